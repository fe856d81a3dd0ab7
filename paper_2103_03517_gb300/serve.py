"""A request loop in front of the library's server (mc_server_*, mc_submit,
mc_poll): jobs arrive as JSON lines, each is submitted as soon as it is read,
and each result is written as a JSON line when its job finishes, with its
latency.  The server admits jobs by device memory, keeps their lattices and
RNG state resident between epochs and batches the resident ones into shared
launches (continuous batching); this module only reads, submits, polls and
writes.

    python -m paper_2103_03517_gb300.serve < jobs.jsonl > results.jsonl

A job is a JSON object.  Lattice keys (defaults as in make_desc): dims
(required), J, K_u, axis, K_c, H, T, seed, precision ("fp32" | "fp64"),
boundary (three of "periodic" | "open" | "pinned" | "antiperiodic"),
lattice ("sc" | "bcc" | "fcc" | "hcp"), J2, theta0_deg, adapt_in_measure,
init ("uniform" | "wall"), init_dir, ring_capacity, sample_torque.  Job keys:
kind ("sweep" for Table A1, "constrained" for Table A2), theta_c_deg,
phi_c_deg (constraint direction), n_equilibrate, n_measure, and an optional
id echoed in the result.  Unknown keys are rejected.
"""
from __future__ import annotations

import json
import sys
import time

from . import _mc as mc

__all__ = ["job_from_dict", "result_to_dict", "serve", "main"]

_PRECISION = {"fp32": mc.MC_FP32, "fp64": mc.MC_FP64}
_BOUNDARY = {"periodic": mc.MC_PERIODIC, "open": mc.MC_OPEN, "pinned": mc.MC_PINNED,
             "antiperiodic": mc.MC_ANTIPERIODIC}
_LATTICE = {"sc": mc.MC_SC, "bcc": mc.MC_BCC, "fcc": mc.MC_FCC, "hcp": mc.MC_HCP}
_INIT = {"uniform": mc.MC_INIT_UNIFORM, "wall": mc.MC_INIT_WALL}
_KIND = {"sweep": mc.MC_JOB_SWEEP, "constrained": mc.MC_JOB_CONSTRAINED}
_LATTICE_KEYS = {"dims", "J", "K_u", "axis", "K_c", "H", "T", "seed", "precision", "boundary", "lattice", "J2",
                 "theta0_deg", "adapt_in_measure", "init", "init_dir", "ring_capacity", "sample_torque"}
_JOB_KEYS = {"kind", "theta_c_deg", "phi_c_deg", "n_equilibrate", "n_measure", "id"}


def _choice(table, value, key):
    if value not in table:
        raise ValueError(f"{key}: {value!r} is not one of {sorted(table)}")
    return table[value]


def _vec3(value, key):
    v = [float(x) for x in value]
    if len(v) != 3:
        raise ValueError(f"{key}: three components expected")
    return tuple(v)


def job_from_dict(d: dict) -> mc.mc_job:
    """mc_job of one JSON job.  Raises ValueError for unknown keys and for
    values outside the lists above; the library checks the physics (even
    periodic sizes, T > 0, ...) when the job is submitted."""
    unknown = set(d) - _LATTICE_KEYS - _JOB_KEYS
    if unknown:
        raise ValueError(f"unknown keys {sorted(unknown)}")
    if "dims" not in d:
        raise ValueError("dims is required")
    dims = [int(x) for x in d["dims"]]
    if len(dims) != 3:
        raise ValueError("dims: three sizes expected")
    kw = {}
    for key in ("J", "K_u", "K_c", "T", "J2"):
        if key in d:
            kw[key] = float(d[key])
    for key in ("axis", "H", "init_dir"):
        if key in d:
            kw[key] = _vec3(d[key], key)
    for key in ("seed", "theta0_deg", "adapt_in_measure", "ring_capacity", "sample_torque"):
        if key in d:
            kw[key] = int(d[key])
    if "precision" in d:
        kw["precision"] = _choice(_PRECISION, d["precision"], "precision")
    if "boundary" in d:
        b = list(d["boundary"])
        if len(b) != 3:
            raise ValueError("boundary: three modes expected")
        kw["boundary"] = tuple(_choice(_BOUNDARY, x, "boundary") for x in b)
    if "lattice" in d:
        kw["lattice"] = _choice(_LATTICE, d["lattice"], "lattice")
    if "init" in d:
        kw["init"] = _choice(_INIT, d["init"], "init")
    kind = _choice(_KIND, d.get("kind", "sweep"), "kind")
    n_eq, n_meas = int(d.get("n_equilibrate", 0)), int(d.get("n_measure", 0))
    if n_eq < 0 or n_meas < 0:
        raise ValueError("sweep counts must be >= 0")
    desc = mc.make_desc(dims, **kw)
    return mc.make_job(desc, kind, theta_c_deg=float(d.get("theta_c_deg", 0.0)),
                       phi_c_deg=float(d.get("phi_c_deg", 0.0)), n_equilibrate=n_eq, n_measure=n_meas)


def result_to_dict(job_id, tag, res) -> dict:
    """JSON-ready result: the job's id (and the caller's tag), status, the
    observables of mc_measure, and submit / admit / finish times with the
    latency (finish - submit), in seconds on the server's clock."""
    out = {"job": int(job_id), "status": int(res.status)}
    if tag is not None:
        out["id"] = tag
    out["obs"] = res.obs.asdict()
    out["t_submit"], out["t_admit"], out["t_finish"] = res.t_submit, res.t_admit, res.t_finish
    out["latency_s"] = res.t_finish - res.t_submit
    return out


def serve(lines, write, submit, poll, poll_interval=0.002, forget=None):
    """The request loop.  lines yields JSON job lines as they arrive (blank
    lines are skipped); each is parsed and submitted at once.  submit(job)
    returns a job id; poll(job_id) returns (status, result) with status
    MC_PENDING or MC_OK.  Finished jobs are written (write(dict)) as they
    complete, between reads and after the input ends.  A line that does not
    parse, or a job the server refuses, is written as an error record with its
    line number and the loop goes on.  forget(job_id), if given, is called
    once a result is written, so that the server drops the finished job's
    record and a long stream keeps only the jobs in flight.  Returns the
    number of results written (errors included)."""
    pending = {}  # job id -> caller's tag
    written = 0

    def drain():
        nonlocal written
        for jid in list(pending):
            rc, res = poll(jid)
            if rc == mc.MC_OK:
                write(result_to_dict(jid, pending.pop(jid), res))
                written += 1
                if forget is not None:
                    forget(jid)

    for n, line in enumerate(lines, 1):
        line = line.strip()
        if not line:
            continue
        try:
            d = json.loads(line)
            if not isinstance(d, dict):
                raise ValueError("a job is a JSON object")
            jid = submit(job_from_dict(d))
        except (ValueError, TypeError, mc.MCError) as e:
            write({"line": n, "error": str(e)})
            written += 1
            continue
        pending[jid] = d.get("id")
        drain()
    while pending:
        drain()
        if pending:
            time.sleep(poll_interval)
    return written


def main(argv=None) -> int:
    import argparse

    ap = argparse.ArgumentParser(description="JSON-lines request loop in front of the libmc server")
    ap.add_argument("--device", type=int, default=0)
    ap.add_argument("--memory-budget", type=int, default=0, help="bytes of device memory for jobs (0: 90%% free)")
    ap.add_argument("--max-resident", type=int, default=256)
    ap.add_argument("--max-epoch-sweeps", type=int, default=50)
    a = ap.parse_args(argv)
    srv = mc.mc_server_create(device=a.device, memory_budget=a.memory_budget, max_resident=a.max_resident,
                              max_epoch_sweeps=a.max_epoch_sweeps)
    try:
        def write(rec):
            sys.stdout.write(json.dumps(rec) + "\n")
            sys.stdout.flush()

        serve(sys.stdin, write, lambda job: mc.mc_submit(srv, job), lambda jid: mc.mc_poll(srv, jid),
              forget=lambda jid: mc.mc_forget(srv, jid))
    finally:
        mc.mc_server_destroy(srv)
    return 0


if __name__ == "__main__":
    sys.exit(main())
