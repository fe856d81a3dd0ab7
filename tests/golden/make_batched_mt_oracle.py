"""Write tests/golden/batched_mt_oracle.json: the serial FP64 oracle's
ensemble averages for the FP32 precision check of the batched m(T) workload.

For every case of workloads.precision_cases() (the 32 lattices of the
batched temperature sweep and two extra 16^3 points near T_C) the oracle runs
K independent chains (seeds workloads.precision_seed(PRECISION_ORACLE_SEED0,
spec, k)), each n_eq unmeasured + n_meas measured sweeps of Table A1 from the
all +z state (workloads.PRECISION_SWEEPS).  Per chain it records the means
over the measured sweeps of |m|, |m|^2, |m_z|, m_z and E/N; the file holds,
per case and observable, the mean over the K chains and their standard
deviation (ddof 1), so the standard error is sd / sqrt(K).

K is chosen per case: a pilot of 8 chains gives the spread of <|m|>, then K
grows until the standard error of <|m|> is at most SIGMA_TARGET (at least 8
chains, at most K_MAX); the spread is re-estimated from all chains after
each round, for up to four rounds.  Only the oracle runs here; nothing comes
from the CUDA library.

    python tests/golden/make_batched_mt_oracle.py [--jobs N] [--scratch PATH]

Runs take about an hour on 8 cores; partial results go to the scratch file
so an interrupted run resumes.
"""
from __future__ import annotations

import argparse
import json
import math
import multiprocessing as mp
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import workloads  # noqa: E402

OUT = os.path.join(HERE, "batched_mt_oracle.json")
SIGMA_TARGET = 4e-4
K_PILOT = 8
K_MAX = 20000
OBS = ("ml", "ml2", "mabs_z", "mz", "e")


def run_chain(task):
    """One oracle chain: (case, k) -> (case, k, {observable: mean})."""
    name, k = task
    import oracle

    spec = workloads.precision_cases()[name]
    n_eq, n_meas = workloads.PRECISION_SWEEPS[spec.dims[0]]
    seed = workloads.precision_seed(workloads.PRECISION_ORACLE_SEED0, spec, k)
    o = oracle.Lattice(spec.dims, J=spec.J, Ku=spec.Ku, axis=spec.axis, T=spec.T, seed=seed,
                       theta0=spec.theta0, adapt_in_measure=1, ring_cap=1)
    o.sweep(n_eq, measure=False)
    o.sweep(n_meas, measure=True)
    s = o.stats()
    n = s["n"]
    return name, k, {"ml": s["ml"] / n, "ml2": s["ml2"] / n, "mabs_z": s["mabsz"] / n, "mz": s["mz"] / n,
                     "e": s["e"] / n}


def summarise(runs: dict) -> dict:
    out = {}
    vals = list(runs.values())
    K = len(vals)
    for key in OBS:
        xs = [v[key] for v in vals]
        mean = math.fsum(xs) / K
        sd = math.sqrt(math.fsum((x - mean) ** 2 for x in xs) / (K - 1)) if K > 1 else float("nan")
        out[key] = {"mean": mean, "sd": sd}
    return out


def main(argv=None) -> int:
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--jobs", type=int, default=os.cpu_count() or 1)
    ap.add_argument("--scratch", default=os.path.join("/tmp", "batched_mt_oracle.partial.json"))
    a = ap.parse_args(argv)

    import oracle
    oracle.build()
    cases = workloads.precision_cases()
    done = {name: {} for name in cases}
    if os.path.exists(a.scratch):
        with open(a.scratch) as f:
            for name, runs in json.load(f).items():
                done[name] = {int(k): v for k, v in runs.items()}

    def save():
        tmp = a.scratch + ".tmp"
        with open(tmp, "w") as f:
            json.dump(done, f)
        os.replace(tmp, a.scratch)

    def cost(name):
        spec = cases[name]
        return spec.N * sum(workloads.PRECISION_SWEEPS[spec.dims[0]])

    ctx = mp.get_context("spawn")
    t0 = time.time()
    with ctx.Pool(a.jobs) as pool:
        for phase in ("pilot", "main", "main", "main", "main"):
            tasks = []
            for name in cases:
                if phase == "pilot":
                    want = K_PILOT
                else:
                    s = summarise(done[name])["ml"]["sd"]
                    want = min(K_MAX, max(K_PILOT, math.ceil((s / SIGMA_TARGET) ** 2)))
                tasks += [(name, k) for k in range(want) if k not in done[name]]
            tasks.sort(key=lambda t: -cost(t[0]))
            print(f"{phase}: {len(tasks)} chains", flush=True)
            if not tasks:
                continue
            last = time.time()
            for i, (name, k, obs) in enumerate(pool.imap_unordered(run_chain, tasks, chunksize=1), 1):
                done[name][k] = obs
                if time.time() - last > 30 or i == len(tasks):
                    save()
                    last = time.time()
                    print(f"  {phase} {i}/{len(tasks)}  {time.time() - t0:.0f} s", flush=True)

    result = {"protocol": {"sweeps": {str(L): list(v) for L, v in workloads.PRECISION_SWEEPS.items()},
                           "oracle_seed0": workloads.PRECISION_ORACLE_SEED0,
                           "sigma_target_ml": SIGMA_TARGET, "k_pilot": K_PILOT, "k_max": K_MAX,
                           "observables": list(OBS),
                           "note": "per chain: means over the measured sweeps; per case: mean over chains "
                                   "and their standard deviation (ddof 1)"},
              "cases": {}}
    for name, spec in cases.items():
        K = len(done[name])
        result["cases"][name] = {"L": spec.dims[0], "T": spec.T, "K_u": spec.Ku, "seed_index": spec.seed,
                                 "sweeps": list(workloads.PRECISION_SWEEPS[spec.dims[0]]), "chains": K,
                                 "obs": summarise(done[name])}
    with open(OUT, "w") as f:
        json.dump(result, f, indent=1)
    print(f"wrote {OUT} in {time.time() - t0:.0f} s", flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
