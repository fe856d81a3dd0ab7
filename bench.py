"""Throughput of the batched parallel Metropolis sweep on GB300.

Workload (one step = one measurement sweep of the whole batch: red pass, black
pass with the fused sample, cone adaptation, for every lattice):
32 independent periodic simple-cubic lattices, L = 16, 32, 64, 128 cycled,
T_i = 0.05 (i + 1), J = 1, K_u = 0.01 along z, FP32 spins with fixed-point
sample sums, 19,169,280 spins in total (230 MB of spins: larger than L2, so
no flush is needed between steps), advanced by one graph-replayed launch per
colour pass.

Usage:  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
                       [--side all|none|fp64|constrained|anisotropy|cubes|general|stiffness|films|precision|
                               serving|torque|wall|wave|slabs|paper]
                       [--no-cpu]
Under torchrun (N > 1) the ranks split the batch: each lattice runs on one
rank, shares balanced by spins (strong scaling, no collective on the data
path); the time is the max over ranks and the value the batch's updates.
`--impl reference` times the serial FP64 CPU oracle on the host cores instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads  # noqa: E402

METRIC = "spin-updates/s & HBM roofline frac (128^3 FP32); served m(T) req/s, p50/p99"
UNIT = "spin-updates/s"
# launch shapes of the FP32 row kernel (mc_group_autotune's row candidates)
ROW_SHAPES = ["3 blocks per SM", "2 blocks per SM"]
RESIDENT_SHAPES = ["blocks of 512 threads", "blocks of 640 threads"]
BYTES_PER_UPDATE = 24          # FP32: read + write 3 x 4 B of every spin once per sweep
FALLBACK_HBM_GBS = 6800.0
LATSTATE_BYTES = 400           # device state block read back by mc_measure
PROFILE_SUMMARY = os.path.join(ROOT, "profiles", "row_pass_f32_batched_mT.txt")
KERNEL_SOURCES = ["paper_2103_03517_gb300/csrc/row_pass.cuh", "paper_2103_03517_gb300/csrc/pair_math.cuh",
                  "paper_2103_03517_gb300/csrc/pass_impl.cuh",
                  "paper_2103_03517_gb300/csrc/device_common.cuh", "paper_2103_03517_gb300/csrc/kernels_f32.cu",
                  "paper_2103_03517_gb300/csrc/launchers_common.cuh", "paper_2103_03517_gb300/csrc/mc_internal.h"]


def workload_config():
    specs = workloads.batched_mt_32()
    n = sum(s.N for s in specs)
    return specs, n, {
        "workload": "batched m(T) sweep: 32 periodic sc lattices 16^3/32^3/64^3/128^3 cycled, "
                    "T = 0.05..1.60, J = 1, K_u = 0.01 z; FP32 spins, fixed-point sample sums; "
                    "one measurement sweep per step (sample: m vector and energy parts of every lattice)",
        "lattices": len(specs),
        "spins": n,
        "l2": "inputs larger than L2 (230 MB of spins), no flush",
    }


def kernel_hash() -> str:
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def read_traffic():
    """Per-launch DRAM bytes of the row colour-pass kernel from the committed ncu
    summary, or None if absent or taken on a different kernel source."""
    try:
        kv = {}
        with open(PROFILE_SUMMARY) as f:
            for ln in f:
                if ":" in ln:
                    k, v = ln.split(":", 1)
                    kv[k.strip()] = v.strip()
        if kv.get("kernel_source_sha256_16") != kernel_hash():
            return None
        return float(kv["dram_bytes_per_launch"])
    except (OSError, KeyError, ValueError):
        return None


def measured_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return FALLBACK_HBM_GBS, "fallback"


# ------------------------------------------------------------ clocks
class Clocks:
    """nvidia-smi samples (every 50 ms) over a loaded window of the GPU that
    contains the timed region: the caller starts it, keeps the GPU busy with
    untimed sweeps for about a second, runs the timed region, and stops it.
    A timed region of a few milliseconds falls between two samples, so the
    window around it is what is sampled."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu):
        self.gpu = gpu
        self.proc = None
        self.lines = []
        self.error = None

    def __enter__(self):
        import threading
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True, bufsize=1)
        except OSError as e:
            self.proc, self.error = None, f"nvidia-smi unavailable: {e}"
            return self

        def reader():
            for ln in self.proc.stdout:
                self.lines.append(ln)
        self.thread = threading.Thread(target=reader, daemon=True)
        self.thread.start()
        return self

    def __exit__(self, *a):
        if self.proc:
            import signal
            self.proc.send_signal(signal.SIGINT)  # nvidia-smi ends a -lms loop on Ctrl-C
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.proc.wait()
            self.thread.join(timeout=5)
            if self.proc.returncode not in (0, -2, 130) and not self.lines:
                self.error = (self.proc.stderr.read() or "").strip()[:200]

    def summary(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0, "error": self.error}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax.append(float(p[2]))
            except ValueError:
                continue
            for n, v in zip(names, p[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        out = {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
               "reasons": sorted(reasons), "samples": len(sm),
               "window": "nvidia-smi every 50 ms over about 1 s of untimed sweeps and the timed region"}
        if not sm:
            out["error"] = self.error or "no clock samples recorded"
            print(f"bench.py: WARNING: {out['error']}", file=sys.stderr, flush=True)
        return out


# ------------------------------------------------------------ ranks
def job_time_and_value(ms_local: float, updates_total: float, world: int, reduce_max=None):
    """Whole-job numbers: the ranks split one batch (each lattice on one
    rank), the job time is the max over ranks (reduce_max, a collective, is
    given for world > 1) and the value is the batch's updates over it."""
    ms = reduce_max(ms_local) if world > 1 else ms_local
    return ms, updates_total / (ms * 1e-3)


def torch_reduce_max(device):
    import torch
    import torch.distributed as dist

    def f(x):
        t = torch.tensor([x], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())
    return f


# ------------------------------------------------------------ oracle legs
def _oracle_worker(args):
    idx, n_warm, n_steps, barrier = args
    import oracle

    specs = workloads.batched_mt_32()
    lats = []
    for i in idx:
        s = specs[i]
        lats.append(oracle.Lattice(s.dims, Ku=s.Ku, T=s.T, seed=s.seed, ring_cap=1))
    for o in lats:
        o.sweep(n_warm, measure=True)
    if barrier is not None:
        barrier.wait()
    t = time.perf_counter()
    for o in lats:
        o.sweep(n_steps, measure=True)
    return time.perf_counter() - t


def oracle_single_thread():
    """Single-thread cost of the serial oracle in ns per spin-update, in this
    process: the 16^3 point (K_u = 0.01, T = 0.5) over 1 + 40 measured sweeps
    and one 128^3 lattice of the batch (T = 0.2) over 1 + 2."""
    import oracle
    oracle.build()
    out = {}
    for name, spec, n in (("16^3", workloads.point_16c(), 40), ("128^3", workloads.batched_mt_32()[3], 2)):
        o = oracle.Lattice(spec.dims, Ku=spec.Ku, T=spec.T, seed=spec.seed, ring_cap=1)
        o.sweep(1, measure=True)
        t = time.perf_counter()
        o.sweep(n, measure=True)
        out[name] = round((time.perf_counter() - t) / (spec.N * n) * 1e9, 2)
    return out


def run_oracle(lattice_ids, n_warm, n_steps):
    """Run the serial oracle on the given batched m(T) lattices, one process per
    core (spawned), every lattice n_warm + n_steps measurement sweeps; return
    (updates per second over the timed sweeps, cores used)."""
    import oracle
    oracle.build()
    specs = workloads.batched_mt_32()
    cores = max(1, min(len(lattice_ids), os.cpu_count() or 1))
    # balance by size: largest first onto the least loaded core
    bins = [[] for _ in range(cores)]
    load = [0] * cores
    for i in sorted(lattice_ids, key=lambda i: -specs[i].N):
        k = load.index(min(load))
        bins[k].append(i)
        load[k] += specs[i].N
    ctx = mp.get_context("spawn")
    with ctx.Manager() as man:
        barrier = man.Barrier(cores + 1)
        with ctx.Pool(cores) as pool:
            res = pool.map_async(_oracle_worker, [(b, n_warm, n_steps, barrier) for b in bins])
            barrier.wait()
            t = time.perf_counter()
            res.get()
            wall = time.perf_counter() - t
    updates = sum(specs[i].N for i in lattice_ids) * n_steps
    return updates / wall, cores


def reference_arm(args, cfg):
    """--impl reference: the serial FP64 oracle on the host cores, on the GPU
    arm's own workload: one step = one measurement sweep of all 32 lattices
    (19,169,280 updates), lattices spread over the cores by size."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    specs = workloads.batched_mt_32()
    # the whole batch per step while the run stays within about two minutes
    # on the host's cores (the oracle does about 5e6 updates/s per core);
    # for longer runs the largest set of the smallest lattices that fits
    budget = 120.0 * 5e6 * (os.cpu_count() or 1) / max(1, args.steps + args.warmup)
    sample = []
    for i in sorted(range(32), key=lambda i: specs[i].N):
        if sum(specs[j].N for j in sample) + specs[i].N <= budget or not sample:
            sample.append(i)
    sample.sort()
    rate, cores = run_oracle(sample, args.warmup, args.steps)
    per_step = sum(specs[i].N for i in sample)
    which = "all 32 lattices of the workload" if len(sample) == 32 else \
        f"{len(sample)} of the workload's 32 lattices (the smallest, to bound the run)"
    sample_desc = f"{which}, {args.warmup} warm-up + {args.steps} measurement sweeps each, one spawned process per core"
    line = {
        "impl": "reference", "metric": METRIC, "value": rate, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": per_step / rate * 1e3,
        "higher_is_better": True, "scaling": "strong", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": cfg,
        "cpu_baseline": {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample_desc},
        "e2e": {"value": rate, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------ GPU arm
def gpu_arm(args, cfg):
    import torch

    import paper_2103_03517_gb300 as mc
    from paper_2103_03517_gb300 import build as libbuild

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    libbuild.build()
    specs_all, n_spins, _ = workload_config()
    # the ranks split the batch: each lattice runs on one rank, shares
    # balanced by spins (every lattice takes the same sweeps)
    from paper_2103_03517_gb300 import shard
    mine = shard.partition_by_cost([sp.N for sp in specs_all], world)[rank]
    specs = [specs_all[i] for i in mine]
    n_local = sum(sp.N for sp in specs)

    # cpu baseline first (spawned pool; rank 0, N = 1 only)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        rate, cores = run_oracle(list(range(32)), 1, 4)
        cpu = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": "all 32 lattices of the workload, 4 measurement sweeps each after 1 warm-up "
                         "(76.7M updates), one spawned process per core",
               "single_thread_ns_per_update": oracle_single_thread()}

    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        hs = [mc.mc_create_ex(mc.make_desc(s.dims, K_u=s.Ku, T=s.T, seed=s.seed, precision=mc.MC_FP32,
                                           ring_capacity=16, sample_torque=0, stream=stream.cuda_stream,
                                           device=local))
              for s in specs]
        g = mc.mc_group_create(hs)
        # launch shapes picked by the autotuner (the chains are left unchanged)
        if not args.no_autotune:
            tuned = mc.mc_group_autotune(g, 4, mc.MC_TUNE_SWEEP)
            cfg["autotuned"] = {"row_shape": ROW_SHAPES[tuned["row"]],
                                "ms_per_sweep": [round(x, 4) for x in tuned["row_ms"][:2]]}
        mc.mc_group_sweep(g, args.warmup, measure=True)
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        try:
            gpu_id = "GPU-" + str(torch.cuda.get_device_properties(local).uuid)
        except Exception:
            gpu_id = str(local)
        with Clocks(gpu_id) as clk:
            # about a second of untimed measured sweeps under the sampler, so
            # that the clocks of a loaded GPU are on record around the timed region
            t_load = time.perf_counter()
            while time.perf_counter() - t_load < 1.0:
                mc.mc_group_sweep(g, 256, measure=True)
                torch.cuda.synchronize()
            start.record(stream)
            mc.mc_group_sweep(g, args.steps, measure=True)
            stop.record(stream)
            torch.cuda.synchronize()
        ms, value = job_time_and_value(start.elapsed_time(stop), n_spins * args.steps, world,
                                       torch_reduce_max("cuda") if world > 1 else None)

        # dominant kernel: the row colour pass (a red and a measured black pass
        # per step, every launch of the timed region; with the wavefront path
        # asked for, the wavefront launch).  Its launch duration: CUDA events
        # around every launch over the same kind of sweeps, right after the
        # timed region (events between launches would change the timed region)
        n_time = max(8, min(args.steps, 200)) // 2 * 2
        kern_ms, kern_n = mc.mc_group_time_kernels(g, n_time, measure=True, constrained=False)
        wave_spins = sum(sp.N for sp in specs if sp.dims[0] == 128)
        if kern_n[0]:
            kernel_name, avg_ms, bytes_per_launch = "wave_sweep_kernel<float>", kern_ms[0], wave_spins * BYTES_PER_UPDATE
        else:
            kernel_name, avg_ms, bytes_per_launch = "row_pass_kernel<float>", kern_ms[1], (n_local // 2) * BYTES_PER_UPDATE
        achieved = bytes_per_launch / (avg_ms * 1e-3) / 1e9
        peak, peak_kind = measured_peak()
        traffic = read_traffic()
        # launches of the timed region: a wavefront pair is 2 x (1 + 2) launches;
        # an odd last sweep runs every lattice on the two row passes
        launches = 3 * (args.steps - args.steps % 2) + 2 * (args.steps % 2) if kern_n[0] else 2 * args.steps

        # end to end through the C ABI with host buffers: per step the whole
        # spin state goes host -> device from pinned memory, one measurement
        # sweep runs, and every lattice's observables come back (one wait).
        # Serial: each step's copy, sweep and read in turn.  Pipelined: a
        # second set of the same lattices on a second stream, the steps
        # alternating between the sets, so that step k + 1's copy runs while
        # step k sweeps; every step still copies all of its state and reads
        # its results.
        sizes = [mc.mc_state_bytes(h) for h in hs]
        host = [torch.empty(b, dtype=torch.uint8, pin_memory=True) for b in sizes]
        for h, buf, b in zip(hs, host, sizes):
            mc.mc_export_state(h, buf.data_ptr(), b)
        e2e_steps = max(4, min(args.steps, 50)) // 2 * 2

        def e2e_issue(lats, grp):
            for h, buf, b in zip(lats, host, sizes):
                mc.mc_import_state(h, buf.data_ptr(), b)
            mc.mc_group_sweep(grp, 1, measure=True)

        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            e2e_issue(hs, g)
            mc.mc_group_measure(g, len(hs))
        torch.cuda.synchronize()
        serial_s = time.perf_counter() - t0
        stream2 = torch.cuda.Stream()
        hs2 = [mc.mc_create_ex(mc.make_desc(s.dims, K_u=s.Ku, T=s.T, seed=s.seed, precision=mc.MC_FP32,
                                            ring_capacity=16, sample_torque=0, stream=stream2.cuda_stream,
                                            device=local))
               for s in specs]
        g2 = mc.mc_group_create(hs2)
        sets = [(hs, g), (hs2, g2)]
        e2e_issue(hs2, g2)  # the second set's first sweep (graph capture) outside the timed region
        mc.mc_group_measure(g2, len(hs2))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e2e_issue(*sets[0])
        for k in range(e2e_steps):
            if k + 1 < e2e_steps:
                e2e_issue(*sets[(k + 1) % 2])
            mc.mc_group_measure(sets[k % 2][1], len(hs))
        torch.cuda.synchronize()
        e2e_s = time.perf_counter() - t0
        mc.mc_group_destroy(g2)
        for h in hs2:
            mc.mc_destroy(h)
        if world > 1:
            e2e_s, serial_s = torch_reduce_max("cuda")(e2e_s), torch_reduce_max("cuda")(serial_s)
        e2e = {"value": n_spins * e2e_steps / e2e_s, "unit": UNIT,
               "h2d_bytes_per_step": int(sum(sizes)), "d2h_bytes_per_step": LATSTATE_BYTES * len(hs),
               "steps": e2e_steps, "serial_value": n_spins * e2e_steps / serial_s,
               "how": "two sets of the lattices on two streams, step k + 1's host-to-device copy during step k's "
                      "sweep; serial_value: one set, copy, sweep and read in turn"}

        extra = {}
        side = "none" if args.quick else args.side
        if rank == 0 and side != "none":
            extra = secondary(mc, torch, stream, local, side, tune=not args.no_autotune)
            if side in ("all", "serving"):
                extra["serving"] = serving(mc)
        mc.mc_group_destroy(g)
        for h in hs:
            mc.mc_destroy(h)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "strong",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": cfg,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic, "peak_kind": peak_kind,
                         "kernel": kernel_name, "launch_avg_ms": avg_ms,
                         "launch_avg_ms_source": f"CUDA events around each of {kern_n[0] or kern_n[1]} launches "
                                                 f"of {n_time} measured sweeps after the timed region",
                         "algorithmic_bytes_per_launch": bytes_per_launch,
                         "other_launches_avg_ms": kern_ms[1] if kern_n[0] else None,
                         "step_frac": n_spins * BYTES_PER_UPDATE / (ms / args.steps * 1e-3) / 1e9 / (peak * world),
                         "step_frac_note": "whole step (all 32 lattices, every launch) against 24 B per update "
                                           "and the peak of every GPU of the job"},
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": launches,
            "clocks": clk.summary(),
        }
        line.update(extra)
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def secondary(mc, torch, stream, dev, side="all", tune=True):
    """Side measurements reported with the headline: the same batch as 32
    sequential one-lattice FP64 runs (per-launch baseline of the batched
    path), and the constrained workload (80 x 64^3 pair sweeps)."""
    out = {}
    if side in ("all", "fp64"):
        out.update(fp64_per_lattice(mc, torch, stream, dev))
    if side in ("all", "constrained"):
        out.update(constrained(mc, torch, stream, dev, tune))
    if side in ("all", "anisotropy"):
        out.update(anisotropy(mc, torch, stream, dev))
    if side in ("all", "cubes"):
        out.update(cubes(mc, torch, stream, dev, tune))
    if side in ("all", "general"):
        out.update(general_geometry(mc, torch, stream, dev))
    if side in ("all", "stiffness"):
        out.update(stiffness(mc, torch, stream, dev))
    if side in ("all", "films"):
        out.update(films(mc, torch, stream, dev))
    if side in ("all", "precision"):
        out.update(precision(mc, torch, stream, dev))
    if side in ("all", "wave"):
        out.update(wavefront(mc, torch, stream, dev))
    if side in ("all", "torque"):
        out.update(torque_study(stream, dev))
    if side in ("all", "wall"):
        out.update(wall_study(stream, dev))
    if side in ("all", "slabs"):
        out.update(slabs_side(mc, torch, stream, dev))
    if side == "paper":  # not in "all": about ten minutes
        out.update(paper_size(mc, torch, stream, dev))
    return out


def wavefront(mc, torch, stream, dev, sweeps=200):
    """The eight 128^3 lattices of the batched workload on the wavefront path
    (kernel_path MC_PATH_WAVE: one launch per sweep, each spin read and
    written once) and on the row passes, measured sweeps: time per sweep
    (CUDA events around the replayed graphs) and the wavefront launch timed
    alone, against 24 B per update and the measured HBM peak."""
    peak, _ = measured_peak()
    specs = [sp for sp in workloads.batched_mt_32() if sp.dims[0] == 128]
    n = sum(sp.N for sp in specs)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    res = {}
    for name, path in (("wavefront", mc.MC_PATH_WAVE), ("row", mc.MC_PATH_ROW)):
        hs = [mc.mc_create_ex(mc.make_desc(sp.dims, K_u=sp.Ku, T=sp.T, seed=sp.seed, kernel_path=path,
                                           ring_capacity=16, sample_torque=0, stream=stream.cuda_stream,
                                           device=dev)) for sp in specs]
        g = mc.mc_group_create(hs)
        mc.mc_group_sweep(g, 10, measure=True)
        torch.cuda.synchronize()
        a.record(stream)
        mc.mc_group_sweep(g, sweeps, measure=True)
        b.record(stream)
        torch.cuda.synchronize()
        ms = a.elapsed_time(b) / sweeps
        kms, kn = mc.mc_group_time_kernels(g, 20, measure=True)
        res[name] = {"us_per_sweep": round(ms * 1e3, 2), "sweep_frac": round(n * 24 / (ms * 1e-3) / 1e9 / peak, 4),
                     "launch_ms": round(kms[0] if kn[0] else kms[1], 5)}
        mc.mc_group_destroy(g)
        for h in hs:
            mc.mc_destroy(h)
    return {"wavefront": {"workload": "the eight 128^3 lattices of the batch (16.8M spins), measured sweeps, FP32",
                          **res}}


def slabs_side(mc, torch, stream, dev, sweeps=40):
    """The Bloch-wall lattice (1024 x 128 x 128, x pinned, z periodic) swept
    whole and split along z into 1, 2 and 4 slabs on this one GPU
    (mc_slab_sweep: the slab passes, the halo-plane copies after each colour
    pass, the count export, sum and close of every sweep), measured sweeps,
    CUDA events: the cost of the multi-device decomposition's protocol
    without the interconnect."""
    spec = workloads.bloch_wall_1024()[3]
    dims = spec.dims
    n = dims[0] * dims[1] * dims[2]
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def desc():
        return mc.make_desc(dims, K_u=spec.Ku, T=spec.T, seed=spec.seed, boundary=spec.bc, init=mc.MC_INIT_WALL,
                            ring_capacity=16, stream=stream.cuda_stream, device=dev)

    def timed(run):
        run(4)
        torch.cuda.synchronize()
        a.record(stream)
        run(sweeps)
        b.record(stream)
        torch.cuda.synchronize()
        return n * sweeps / (a.elapsed_time(b) * 1e-3)

    out = {}
    h = mc.mc_create_ex(desc())
    out["whole"] = timed(lambda k: mc.mc_sweep(h, k, measure=True))
    mc.mc_destroy(h)
    for ns in (1, 2, 4):
        nz = dims[2] // ns
        hs = [mc.mc_slab_create(desc(), i * nz, nz) for i in range(ns)]
        out[f"slabs_{ns}"] = timed(lambda k: mc.mc_slab_sweep(hs, k, measure=True))
        for x in hs:
            mc.mc_destroy(x)
    plane_bytes = dims[0] * dims[1] // 2 * 12
    return {"slabs": {"unit": UNIT, **{k: round(v, 1) for k, v in out.items()},
                      "halo_bytes_per_slab_per_sweep": 4 * plane_bytes,
                      "workload": f"Bloch-wall lattice {dims[0]}x{dims[1]}x{dims[2]}, x pinned, FP32, {sweeps} "
                                  "measured sweeps; slabs of equal planes on one GPU, halo planes copied device "
                                  "to device"}}


def torque_study(stream, dev):
    """Config 3 as stated: 64^3, K_u = 0.05 z, K_c = 0.02, constraint theta
    0..90 by 10 at phi 0 and 45 deg, T in {0.2, 0.6, 1.0, 1.3}, 3000 + 5000
    constrained sweeps (80 runs, FP32), K_u(T) and K_c(T) by least squares of
    the torque against theta (Sec. 3, Fig. 1(a))."""
    from paper_2103_03517_gb300 import studies
    r = studies.anisotropy_torque_study((64, 64, 64), K_u=0.05, K_c=0.02, temps=(0.2, 0.6, 1.0, 1.3),
                                        n_eq=3000, n_meas=5000, stream=stream.cuda_stream, device=dev)
    fits = {str(T): {k: round(v, 6) for k, v in f.items()} for T, f in r["fits"].items()}
    return {"torque_fit": {"workload": "80 x 64^3 constrained runs, 3000 + 5000 sweeps, FP32", "fits": fits,
                           "seconds": round(r["seconds"], 2), "pair_half_updates_per_s": r["updates"] / r["seconds"],
                           "tau_theta_phi0_T0.2": [round(x["tau"], 6) for x in r["runs"]
                                                   if x["T"] == 0.2 and x["phi"] == 0.0]}}


def wall_study(stream, dev):
    """Config 4 as stated: 1024 x 128 x 128, x pinned (+z / -z end planes), y
    and z periodic, K_u = 0.05 z, T = 0.1 .. 1.4 in 8 steps, 2000 + 4000
    sweeps with a profile every 10; K(T) from constrained 64^3 lattices at
    theta = 45 deg; the wall width from the tanh fit of the re-centred
    average profile and A(T) = K(T) (Delta / pi)^2 (Sec. 3, Eq. 5)."""
    from paper_2103_03517_gb300 import studies
    temps = [round(0.1 + i * (1.4 - 0.1) / 7, 4) for i in range(8)]
    r = studies.pinned_wall_study(temps, dims=(1024, 128, 128), K_u=0.05, n_eq=2000, n_meas=4000, every=10,
                                  stream=stream.cuda_stream, device=dev)
    rows = [{k: (round(v, 5) if isinstance(v, float) else v) for k, v in x.items() if k != "profile"}
            for x in r["rows"]]
    mid = [x["profile"][512 - 24:512 + 24:4] for x in r["rows"]]
    return {"wall": {"workload": "8 x 1024x128x128 pinned walls + 8 x 64^3 constrained, FP32, 2000 + 4000 sweeps",
                     "rows": rows, "profile_centre_every_4th_plane": [[round(v, 4) for v in m] for m in mid],
                     "seconds": round(r["seconds"], 2), "updates_per_s": r["updates"] / r["seconds"]}}


def fp64_per_lattice(mc, torch, stream, dev):
    out = {}
    specs = workloads.batched_mt_32()
    n = sum(s.N for s in specs)
    sweeps = 10
    hs = [mc.mc_create_ex(mc.make_desc(s.dims, K_u=s.Ku, T=s.T, seed=s.seed, precision=mc.MC_FP64,
                                       ring_capacity=16, stream=stream.cuda_stream, device=dev)) for s in specs]
    for h in hs:
        mc.mc_sweep(h, 2, measure=True)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for h in hs:
        mc.mc_sweep(h, sweeps, measure=True)
    b.record(stream)
    torch.cuda.synchronize()
    out["fp64_per_lattice"] = {"value": n * sweeps / (a.elapsed_time(b) * 1e-3), "unit": UNIT,
                               "workload": "same 32 lattices, FP64, one lattice per launch sequence"}
    for h in hs:
        mc.mc_destroy(h)
    return out


def constrained(mc, torch, stream, dev, tune=True):
    out = {}
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    sweeps = 10
    runs = workloads.constrained_64c_runs()
    hs = []
    for spec, th, ph in runs:
        t, p = math.radians(th), math.radians(ph)
        e = (math.sin(t) * math.cos(p), math.sin(t) * math.sin(p), math.cos(t))
        hs.append(mc.mc_create_ex(mc.make_desc(spec.dims, K_u=spec.Ku, K_c=spec.Kc, T=spec.T, seed=spec.seed,
                                               init_dir=e, ring_capacity=16, stream=stream.cuda_stream,
                                               device=dev)))
    g = mc.mc_group_create(hs)
    th = [r[1] for r in runs]
    ph = [r[2] for r in runs]
    mc.mc_group_constrained_sweep(g, th, ph, 4, measure=True)
    tuned = mc.mc_group_autotune(g, 2, mc.MC_TUNE_CONSTRAINED) if tune else None
    torch.cuda.synchronize()
    a.record(stream)
    mc.mc_group_constrained_sweep(g, th, ph, sweeps, measure=True)
    b.record(stream)
    torch.cuda.synchronize()
    nc = sum(r[0].N for r in runs)
    # the pair pass against the HBM roofline: 24 B per pair-half update (each
    # spin of the pass's colour read and written once), one launch per colour
    kms, kn = mc.mc_group_time_kernels(g, 8, measure=True, constrained=True)
    peak, _ = measured_peak()
    pair_gbs = (nc // 2) * BYTES_PER_UPDATE / (kms[2] * 1e-3) / 1e9 if kn[2] else None
    out["constrained_roofline"] = {
        "kernel": "pair_pass_kernel<float> (site order)", "launch_avg_ms": kms[2], "launches": kn[2],
        "algorithmic_bytes_per_launch": (nc // 2) * BYTES_PER_UPDATE, "achieved": pair_gbs, "peak": peak,
        "unit": "GB/s", "frac": pair_gbs / peak if pair_gbs else None,
        "sweep_frac": nc * sweeps / (a.elapsed_time(b) * 1e-3) * BYTES_PER_UPDATE / 1e9 / peak}
    out["constrained"] = {"value": nc * sweeps / (a.elapsed_time(b) * 1e-3), "unit": UNIT,
                          "workload": "80 x 64^3 constrained runs (theta_c 0..90, phi_c 0/45, 4 T), FP32, "
                                      "pair halves counted as updates",
                          "autotuned": None if tuned is None else {
                              "field_tiles_per_step": [4, 8, 2][tuned["field"]],
                              "pair_shape": ["4 tiles per step", "8 tiles per step", "2 tiles per step",
                                             "4 tiles per step, more resident warps"][tuned["pair"]],
                              "field_ms": [round(x, 4) for x in tuned["field_ms"][:3]],
                              "pair_ms": [round(x, 4) for x in tuned["pair_ms"][:4]]}}
    mc.mc_group_destroy(g)
    for h in hs:
        mc.mc_destroy(h)
    return out


def anisotropy(mc, torch, stream, dev, n_eq=200, n_meas=500):
    """Anisotropy scaling k_u(T) at 8 temperatures, 64^3 FP32, K_u = 0.05
    along z: by Eq. 4 from standard sweeps, against the constrained torque at
    theta_c = 45 deg (tau_theta / N = -K(T) sin 2 theta); the same sweep
    counts, timed with CUDA events."""
    K, dims = 0.05, (64, 64, 64)
    Ts = [round(0.1 + 0.15 * i, 2) for i in range(8)]
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    res = {}
    for route in ("eq4", "torque"):
        init = (1 / math.sqrt(2), 0.0, 1 / math.sqrt(2)) if route == "torque" else (0.0, 0.0, 1.0)
        hs = [mc.mc_create_ex(mc.make_desc(dims, K_u=K, T=T, seed=i, init_dir=init, ring_capacity=16,
                                           stream=stream.cuda_stream, device=dev)) for i, T in enumerate(Ts)]
        g = mc.mc_group_create(hs)
        torch.cuda.synchronize()
        a.record(stream)
        if route == "eq4":
            mc.mc_group_sweep(g, n_eq)
            mc.mc_group_sweep(g, n_meas, measure=True)
        else:
            th, ph = [45.0] * len(Ts), [0.0] * len(Ts)
            mc.mc_group_constrained_sweep(g, th, ph, n_eq)
            mc.mc_group_constrained_sweep(g, th, ph, n_meas, measure=True)
        b.record(stream)
        torch.cuda.synchronize()
        if route == "eq4":
            k = [mc.mc_anisotropy_scaling(h)[0] for h in hs]
        else:
            k = [-mc.mc_measure(h).torque[1] / K for h in hs]
        res[route] = {"ms": a.elapsed_time(b), "k_u": [round(x, 4) for x in k]}
        mc.mc_group_destroy(g)
        for h in hs:
            mc.mc_destroy(h)
    return {"anisotropy": {
        "workload": f"k_u(T) of 8 x 64^3 FP32 lattices, K_u = 0.05, T = {Ts[0]}..{Ts[-1]}, "
                    f"{n_eq} + {n_meas} sweeps per route",
        "temperatures": Ts, "eq4": res["eq4"], "torque": res["torque"],
        "torque_over_eq4_time": res["torque"]["ms"] / res["eq4"]["ms"],
        "max_abs_diff": max(abs(x - y) for x, y in zip(res["eq4"]["k_u"], res["torque"]["k_u"]))}}


def stiffness(mc, torch, stream, dev):
    """Table I of the paper at reduced size: for K/J = 8.33e-3 .. 4.2e-2 and
    7 temperatures, a 256 x 64 x 64 wall lattice (x anti-periodic, Bloch-wall
    start) and a 64^3 uniform lattice per point, 2000 + 4000 sweeps, one
    profile fit every 20 sweeps; A(T) = K(T) (Delta/pi)^2 with K(T) from
    Eq. 4, and the exponent of A ~ m^k over m > 0.6.  Wall time of the whole
    study (sweeps, profile reads and fits)."""
    from paper_2103_03517_gb300.studies import exchange_stiffness_study
    table1 = [8.33e-3, 1.67e-2, 2.5e-2, 3.33e-2, 4.2e-2]
    temps = [0.2, 0.35, 0.5, 0.65, 0.8, 0.95, 1.1]
    r = exchange_stiffness_study(table1, temps, stream=stream.cuda_stream, device=dev)
    # the free-energy route of Eq. 5 for K/J = 4.2e-2: walls and uniform
    # lattices of the same size, from the paramagnet (T = 20) down to 0.2
    df_temps = [20.0, 10.0, 6.0, 4.0, 3.0, 2.5, 2.0, 1.7, 1.5, 1.35, 1.2, 1.1, 0.95, 0.8, 0.65, 0.5, 0.35, 0.2]
    f = exchange_stiffness_study([4.2e-2], df_temps, wall_dims=(128, 48, 48), uniform_dims=(128, 48, 48),
                                 stream=stream.cuda_stream, device=dev)
    return {"stiffness": {
        "workload": "Table I at reduced size: 5 K/J x 7 T, wall 256x64x64 (x anti-periodic) + uniform 64^3 "
                    "per point, FP32, 2000 + 4000 sweeps, profile fit every 20 sweeps",
        "k": {f"{K:.4g}": [round(v[0], 3), round(v[1], 3)] for K, v in r["exponents"].items()},
        "paper_k": {"0.00833": 1.48, "0.0167": 1.55, "0.025": 1.75, "0.0333": 1.75, "0.042": 1.79},
        "seconds": round(r["seconds"], 2), "updates_per_s": r["updates"] / r["seconds"],
        "points": [{k: (round(v, 5) if isinstance(v, float) else v) for k, v in x.items()} for x in r["rows"]],
        "free_energy_route": {
            "workload": "K/J = 4.2e-2, wall and uniform 128x48x48 per T, T = 20 .. 0.2 (18 points), "
                        "2000 + 4000 sweeps",
            "seconds": round(f["seconds"], 2),
            "points": [{k: round(x[k], 5) for k in ("T", "m", "K_T", "delta", "A", "dF", "A_dF")}
                       for x in f["rows"]]}}}


def films(mc, torch, stream, dev):
    """Sec. 4 at reduced size: granular films 512 x 512 x Lz (Lz = 4, 8; x, y
    periodic, z open), Voronoi grains of mean diameter 32, 64 and 128 sites
    with a random easy axis each (K_u = 0.02), m(T) at T = 0.1 .. 1.7 from
    per-grain samples; the continuous film of each thickness by Eq. 3 (T_C
    and beta), and the average Curie temperature of Eq. 8 (20 terms, every
    term with the continuous film's beta).  1500 + 3000 sweeps per point, a
    grain sample every 20; wall time of each study."""
    from paper_2103_03517_gb300.studies import film_curie_study
    temps = [round(0.1 * i, 2) for i in range(1, 18)]
    kw = dict(n_eq=1500, n_meas=3000, stream=stream.cuda_stream, device=dev)
    out = {}
    for Lz in (4, 8):
        dims = (512, 512, Lz)
        c = film_curie_study(dims, None, None, None, temps, **kw)
        row = {"continuous": {"T_C": round(c["fit"]["T_C"], 4), "beta": round(c["fit"]["beta"], 3),
                              "seconds": round(c["seconds"], 2)}}
        for d in (32, 64, 128):
            gid, mask, axes = workloads.voronoi_film(512, 512, Lz, float(d), seed=d + Lz)
            r = film_curie_study(dims, gid, mask, axes, temps, beta=c["fit"]["beta"], **kw)
            row[f"grains_d{d}"] = {"grains": int(gid.max()) + 1, "T_C_mean": round(r["fit"]["T_C_mean"], 4),
                                   "beta": r["fit"]["beta"], "rms": round(r["fit"]["rms"], 5),
                                   "m": [round(x, 4) for x in r["m"]], "seconds": round(r["seconds"], 2),
                                   "updates_per_s": r["updates"] / r["seconds"]}
        out[f"Lz{Lz}"] = row
    return {"films": {"workload": "Sec. 4 at reduced size: 512x512xLz films, Lz = 4, 8; Voronoi grains d = 32, "
                                  "64, 128; T = 0.1..1.7 (17 points), 1500 + 3000 sweeps, FP32",
                      "temperatures": temps, "results": out}}


def paper_size(mc, torch, stream, dev):
    """The two studies of the paper at its own sizes and run lengths (not part
    of `--side all`: about ten minutes of GPU time).

    * Table I (Sec. 3): 5 K/J x 7 T, a 256 x 128 x 128 wall (x anti-periodic,
      4.2M spins, as many as the paper's 160^3 mesh) and a 128^3 uniform
      lattice per point, 10,000 + 40,000 sweeps (the paper's 50,000 steps),
      a profile fit every 100 sweeps; A(T) and the exponent of A ~ m^k.
    * Granular films (Sec. 4): 768 x 768 x Lz, Lz = 4, 8, 16, 24 (the paper's
      1 - 6 nm), Voronoi grains of mean diameter 20, 40, 80 and 160 sites (its
      5 - 40 nm), K_u = 0.02 random axes, T = 0.1 .. 1.7, 1500 + 3000 sweeps,
      a grain sample every 20; T_C of the continuous film of each thickness
      (Eq. 3) and the average T_C of the granular films (Eq. 8)."""
    from paper_2103_03517_gb300.studies import exchange_stiffness_study, film_curie_study
    table1 = [8.33e-3, 1.67e-2, 2.5e-2, 3.33e-2, 4.2e-2]
    temps = [0.2, 0.35, 0.5, 0.65, 0.8, 0.95, 1.1]
    r = exchange_stiffness_study(table1, temps, wall_dims=(256, 128, 128), uniform_dims=(128, 128, 128),
                                 n_eq=10000, n_meas=40000, every=100, stream=stream.cuda_stream, device=dev)
    t1 = {"workload": "Table I: 5 K/J x 7 T, wall 256x128x128 (x anti-periodic) + uniform 128^3 per point, FP32, "
                      "10000 + 40000 sweeps, profile fit every 100 sweeps",
          "k": {f"{K:.4g}": [round(v[0], 3), round(v[1], 3)] for K, v in r["exponents"].items()},
          "paper_k": {"0.00833": 1.48, "0.0167": 1.55, "0.025": 1.75, "0.0333": 1.75, "0.042": 1.79},
          "seconds": round(r["seconds"], 1), "updates_per_s": r["updates"] / r["seconds"],
          "points": [{k: (round(v, 5) if isinstance(v, float) else v) for k, v in x.items()} for x in r["rows"]]}
    ftemps = [round(0.1 * i, 2) for i in range(1, 18)]
    kw = dict(n_eq=1500, n_meas=3000, stream=stream.cuda_stream, device=dev)
    films_out = {}
    for Lz in (4, 8, 16, 24):
        dims = (768, 768, Lz)
        c = film_curie_study(dims, None, None, None, ftemps, **kw)
        row = {"continuous": {"T_C": round(c["fit"]["T_C"], 4), "beta": round(c["fit"]["beta"], 3),
                              "seconds": round(c["seconds"], 1)}}
        for d in (20, 40, 80, 160):
            gid, mask, axes = workloads.voronoi_film(768, 768, Lz, float(d), seed=d + Lz)
            g = film_curie_study(dims, gid, mask, axes, ftemps, beta=c["fit"]["beta"], **kw)
            row[f"grains_d{d}"] = {"grains": int(gid.max()) + 1, "T_C_mean": round(g["fit"]["T_C_mean"], 4),
                                   "rms": round(g["fit"]["rms"], 5), "m": [round(x, 4) for x in g["m"]],
                                   "seconds": round(g["seconds"], 1)}
            del gid, mask, axes
        films_out[f"Lz{Lz}"] = row
    return {"paper_size": {"table1": t1, "films": {
        "workload": "768x768xLz films, Lz = 4, 8, 16, 24; Voronoi grains d = 20, 40, 80, 160; T = 0.1..1.7 "
                    "(17 points), 1500 + 3000 sweeps, FP32", "temperatures": ftemps, "results": films_out}}}


def precision(mc, torch, stream, dev):
    """FP32 against FP64, so that each FP32 result's error is stated.  The
    16^3 point (K_u = 0.01, T = 0.5, 1000 + 1000 sweeps) over 8 seeds per
    precision (FP64 on the GPU is the oracle's chain bit for bit):
    differences of the seed means of <|m|>, <m_z>, chi_l and <E/N>, with the
    standard error of the difference from the spread between seeds.  The 32
    lattices of the batched m(T) workload against the serial oracle's stored
    ensembles: per lattice the difference of <|m|> and its standard error,
    both sides from many independent chains, and the count within the
    the benchmark spec's |d| <= 2e-3 and 3 sigma."""
    import numpy as np

    from paper_2103_03517_gb300.analysis import blocking_error

    out = {}
    res = {}
    for prec in (mc.MC_FP32, mc.MC_FP64):
        hs = [mc.mc_create_ex(mc.make_desc((16, 16, 16), K_u=0.01, T=0.5, seed=s, precision=prec, ring_capacity=16,
                                           stream=stream.cuda_stream, device=dev)) for s in range(8)]
        g = mc.mc_group_create(hs)
        mc.mc_group_sweep(g, 1000)
        mc.mc_group_sweep(g, 1000, measure=True)
        mc.mc_group_sync(g)
        mc.mc_group_destroy(g)
        obs = [mc.mc_measure(h) for h in hs]
        res[prec] = {k: np.array(v) for k, v in {"ml": [o.ml for o in obs], "mz": [o.m[2] for o in obs],
                                                  "chi_l": [o.chi[0] for o in obs], "e": [o.e for o in obs]}.items()}
        for h in hs:
            mc.mc_destroy(h)
    c1 = {}
    for k in ("ml", "mz", "chi_l", "e"):
        a, b = res[mc.MC_FP32][k], res[mc.MC_FP64][k]
        c1[k] = {"fp32": round(float(a.mean()), 6), "fp64": round(float(b.mean()), 6),
                 "diff": float(a.mean() - b.mean()),
                 "sigma": float(np.hypot(a.std(ddof=1), b.std(ddof=1)) / np.sqrt(len(a)))}
    out["point_16c_T0.5_8_seeds"] = c1
    # the 32 lattices against the oracle's FP64 chains stored in
    # tests/golden/batched_mt_oracle.json (written by an oracle-only script):
    # per lattice many independent chains on each side (same protocol,
    # disjoint seeds), sigma from the spread between chains
    import json

    from paper_2103_03517_gb300 import studies

    golden_path = os.path.join(ROOT, "tests", "golden", "batched_mt_oracle.json")
    if os.path.exists(golden_path):
        with open(golden_path) as f:
            golden = json.load(f)["cases"]
        cases = workloads.precision_cases()
        names = [f"mT_{i}" for i in range(32)]
        chosen = {n: cases[n] for n in names}
        n_chains = {n: min(20000, max(8, math.ceil((golden[n]["obs"]["ml"]["sd"] / 2e-4) ** 2))) for n in names}
        t0 = time.perf_counter()
        res = studies.chain_ensembles(
            chosen, n_chains, lambda n, k: workloads.precision_seed(workloads.PRECISION_GPU_SEED0, cases[n], k),
            lambda n: workloads.PRECISION_SWEEPS[cases[n].dims[0]], stream=stream.cuda_stream, device=dev)
        secs = time.perf_counter() - t0
        rows, ok = [], 0
        for n in names:
            a, o = res[n]["ml"], golden[n]["obs"]["ml"]
            d = float(a.mean()) - o["mean"]
            sg = math.sqrt(a.var(ddof=1) / a.size + o["sd"] ** 2 / golden[n]["chains"])
            within = abs(d) <= 2e-3 and abs(d) <= 3 * sg
            ok += within
            rows.append({"lattice": n, "L": cases[n].dims[0], "T": round(cases[n].T, 2), "fp32_chains": int(a.size),
                         "oracle_chains": golden[n]["chains"], "diff_ml": round(d, 6), "sigma": round(sg, 6),
                         "within": bool(within)})
        out["batched_mT_32_lattices"] = {
            "criterion": "|d<|m|>| <= 2e-3 and <= 3 sigma, sigma from the spread between chains of each side",
            "lattices_within": ok, "max_abs_diff_ml": max(abs(r["diff_ml"]) for r in rows),
            "max_abs_diff_over_sigma": max(abs(r["diff_ml"]) / r["sigma"] for r in rows), "rows": rows,
            "fp32_seconds": round(secs, 2),
            "protocol": "all +z, n_eq + n_meas = 200 + 500 sweeps (100 + 200 for 128^3), cone adapting; "
                        "FP32 chains on the GPU, FP64 chains of the serial oracle from the stored file"}
    else:
        out["batched_mT_32_lattices"] = {"unavailable": "tests/golden/batched_mt_oracle.json missing"}
    return {"precision": out}


def cubes(mc, torch, stream, dev, tune=True, sweeps=400):
    """The standard FP32 sweep on periodic cubes alone: one 128^3 lattice
    (25 MB of spins) held in shared memory (resident sweeps, the automatic
    path) and on row passes, sixteen 128^3 lattices in one group (403 MB;
    the automatic path sweeps them resident one after another, and on
    batched row passes) and one 256^3 lattice (201 MB).  K_u = 0.01 z, T = 0.5 ..
    1.25, all +z.  Per case: spin-updates/s over unmeasured and measured
    sweeps (CUDA events around the calls), and one launch timed alone
    against the HBM roofline (24 B per update): a colour pass, a wavefront
    sweep, or a resident launch of 100 sweeps."""
    peak, _ = measured_peak()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    cases = [("128c_single", [128], mc.MC_PATH_AUTO), ("128c_single_row", [128], mc.MC_PATH_ROW),
             ("128c_x16", [128] * 16, mc.MC_PATH_AUTO), ("128c_x16_row", [128] * 16, mc.MC_PATH_ROW),
             ("256c_single", [256], mc.MC_PATH_AUTO), ("128c_single_wavefront", [128], mc.MC_PATH_WAVE),
             ("128c_x16_wavefront", [128] * 16, mc.MC_PATH_WAVE)]
    out = {}
    for name, sizes, path in cases:
        torch.cuda.nvtx.range_push(f"cubes_{name}")  # lets a profiler select one case
        hs = [mc.mc_create_ex(mc.make_desc((L, L, L), K_u=0.01, T=0.5 + 0.05 * i, seed=100 + i,
                                           ring_capacity=16, sample_torque=0, stream=stream.cuda_stream,
                                           device=dev, kernel_path=path)) for i, L in enumerate(sizes)]
        g = mc.mc_group_create(hs)
        tuned = mc.mc_group_autotune(g, 4, mc.MC_TUNE_SWEEP) if tune else None
        n = sum(L ** 3 for L in sizes)
        mc.mc_group_sweep(g, 20, measure=True)
        torch.cuda.synchronize()
        res = {"spins": n}
        for meas in (False, True):
            a.record(stream)
            mc.mc_group_sweep(g, sweeps, measure=meas)
            b.record(stream)
            torch.cuda.synchronize()
            rate = n * sweeps / (a.elapsed_time(b) * 1e-3)
            res["measured" if meas else "unmeasured"] = rate
            res["sweep_frac_measured" if meas else "sweep_frac"] = round(rate * BYTES_PER_UPDATE / 1e9 / peak, 4)
            # one launch timed alone: a resident launch of 100 sweeps, a
            # wavefront sweep (128-wide lattices) or a colour pass
            kms, kn = mc.mc_group_time_kernels(g, 100, measure=meas)
            wave, resident = kn[0] > 0, kn[3] > 0
            avg_ms = kms[3] if resident else (kms[0] if wave else kms[1])
            # a resident launch runs one lattice's 100 sweeps (the group's
            # lattices one after another)
            per_launch = (n * 100 // kn[3] if resident else (n if wave else n // 2)) * BYTES_PER_UPDATE
            gbs = per_launch / (avg_ms * 1e-3) / 1e9
            res["kernel"] = ("resident_sweep_kernel (100 sweeps of one lattice per launch)" if resident else
                             "wave_sweep_kernel (one sweep per launch)" if wave else
                             "row_pass_kernel (one colour per launch)")
            shapes = RESIDENT_SHAPES if resident else ROW_SHAPES
            res["row_shape"] = shapes[tuned["row"]] if tuned else shapes[0]
            res["launch_ms_measured" if meas else "launch_ms"] = round(avg_ms, 5)
            res["frac_measured" if meas else "frac"] = round(gbs / peak, 4)
        out[name] = res
        mc.mc_group_destroy(g)
        for h in hs:
            mc.mc_destroy(h)
        torch.cuda.nvtx.range_pop()
    return {"cubes": {"unit": UNIT, "peak_gbs": peak, "cases": out,
                      "workload": f"periodic FP32 cubes, {sweeps} sweeps timed per mode; sweep_frac = updates/s x "
                                  "24 B / measured HBM peak over the timed sweeps; frac = one launch timed alone "
                                  "(algorithmic bytes of the launch over its event time)"}}


def general_geometry(mc, torch, stream, dev, sweeps=40):
    """FP32 throughput of the lattices that are not all-periodic simple
    cubes: the Bloch-wall lattice (1024 x 128 x 128, x pinned, T = 0.66), a
    granular film (1024 x 1024 x 15, Voronoi grains of mean diameter 10, bond
    mask and grain axes, z open) and an fcc lattice of 128^3 cells (8,388,608
    spins, T = 2.0), measured sweeps, CUDA events."""
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    spec = workloads.bloch_wall_1024()[3]
    gid, mask, axes = workloads.voronoi_film(1024, 1024, 15, 10.0, seed=1)
    cases = [("wall", spec.dims, mc.make_desc(spec.dims, K_u=spec.Ku, T=spec.T, seed=spec.seed, boundary=spec.bc,
                                              init=mc.MC_INIT_WALL, ring_capacity=16, stream=stream.cuda_stream,
                                              device=dev)),
             ("film", (1024, 1024, 15), mc.make_desc((1024, 1024, 15), K_u=0.02, T=0.6, seed=3, boundary=(0, 0, 1),
                                                     bond_mask=mask, grain_id=gid, grain_axis=axes, ring_capacity=16,
                                                     stream=stream.cuda_stream, device=dev)),
             ("fcc", (128, 128, 128), mc.make_desc((128, 128, 128), K_u=0.02, T=2.0, seed=4, lattice=mc.MC_FCC,
                                                ring_capacity=16, stream=stream.cuda_stream, device=dev))]
    out = {}
    for name, dims, d in cases:
        h = mc.mc_create_ex(d)
        mc.mc_sweep(h, 4, measure=True)
        torch.cuda.synchronize()
        a.record(stream)
        mc.mc_sweep(h, sweeps, measure=True)
        b.record(stream)
        torch.cuda.synchronize()
        n = dims[0] * dims[1] * dims[2] * (4 if name == "fcc" else 1)
        out[name] = n * sweeps / (a.elapsed_time(b) * 1e-3)
        mc.mc_destroy(h)
    peak, _ = measured_peak()
    return {"general_geometry": {"unit": UNIT, "wall_1024x128x128_pinned_x": out["wall"],
                                 "film_1024x1024x15": out["film"], "fcc_128c": out["fcc"],
                                 "wall_sweep_frac": round(out["wall"] * BYTES_PER_UPDATE / 1e9 / peak, 4),
                                 "film_sweep_frac": round(out["film"] * BYTES_PER_UPDATE / 1e9 / peak, 4),
                                 "workload": f"{sweeps} measured sweeps each, FP32; sweep_frac = updates/s x 24 B "
                                             "over the measured HBM peak"}}


def _serve_trace(mc, trace, n_eq, n_meas, film_tables):
    """Submit the trace's jobs at their arrival times to one server, poll
    until all finish (forgetting each finished record), and return the
    latencies and the work done."""
    gid, mask, axes = film_tables
    jobs, work = [], 0
    for r in trace:
        if r["kind"] == "film":
            d = mc.make_desc((1024, 1024, 15), K_u=0.02, T=r["T"], seed=r["seed"], boundary=(0, 0, 1),
                             bond_mask=mask, grain_id=gid, grain_axis=axes, ring_capacity=16, sample_torque=0)
            jobs.append(mc.make_job(d, mc.MC_JOB_SWEEP, n_equilibrate=n_eq, n_measure=n_meas))
            work += 1024 * 1024 * 15 * (n_eq + n_meas)
        elif r["kind"] == "constrained":
            t = math.radians(r["theta_c"])
            d = mc.make_desc((r["L"],) * 3, K_u=0.05, K_c=0.02, T=r["T"], seed=r["seed"], ring_capacity=16,
                             init_dir=(math.sin(t), 0.0, math.cos(t)))
            jobs.append(mc.make_job(d, mc.MC_JOB_CONSTRAINED, theta_c_deg=r["theta_c"], phi_c_deg=0.0,
                                    n_equilibrate=n_eq, n_measure=n_meas))
            work += r["L"] ** 3 * (n_eq + n_meas)
        else:
            d = mc.make_desc((r["L"],) * 3, K_u=0.01, T=r["T"], seed=r["seed"], ring_capacity=16, sample_torque=0)
            jobs.append(mc.make_job(d, mc.MC_JOB_SWEEP, n_equilibrate=n_eq, n_measure=n_meas))
            work += r["L"] ** 3 * (n_eq + n_meas)
    srv = mc.mc_server_create(max_epoch_sweeps=50)
    done = {}
    try:
        ids = []
        t0 = time.perf_counter()
        for r, j in zip(trace, jobs):
            while time.perf_counter() - t0 < r["t"]:
                for i in ids:  # collect finished jobs while waiting for the next arrival
                    if i not in done:
                        rc, res = mc.mc_poll(srv, i)
                        if rc == mc.MC_OK:
                            done[i] = (res.t_submit, res.t_finish, res.status)
                            mc.mc_forget(srv, i)
                time.sleep(0.0005)
            ids.append(mc.mc_submit(srv, j))
        while len(done) < len(ids):
            for i in ids:
                if i not in done:
                    rc, res = mc.mc_poll(srv, i)
                    if rc == mc.MC_OK:
                        done[i] = (res.t_submit, res.t_finish, res.status)
                        mc.mc_forget(srv, i)
            time.sleep(0.002)
    finally:
        mc.mc_server_destroy(srv)
    res = [done[i] for i in ids]
    lat = sorted(f - s for s, f, _ in res)
    span = max(f for _, f, _ in res) - min(s for s, _, _ in res)
    q = lambda f: lat[min(len(lat) - 1, int(round(f * (len(lat) - 1))))]
    return {"requests": len(trace), "req_per_s": len(trace) / span, "p50_s": q(0.5), "p99_s": q(0.99),
            "updates_per_s": work / span, "ok": sum(st == 0 for _, _, st in res), "span_s": span}


def serving(mc, n_requests=400, rate=20.0, load_frac=0.6, n_eq=200, n_meas=500):
    """The serving mix: Poisson arrivals (seed 1) of m(T) points, constrained
    points and granular films (45/45/10%), cubes L in {8, ..., 256}, T uniform
    in (0.05, 1.6), 200 + 500 sweeps per job, submitted at their arrival
    times to one server; latency = finish - arrival on the server's clock.
    First the configured 20 req/s, which offers more work than the GPU does:
    the queue grows, and the completion rate of that run is the capacity for
    the mix.  Then the same trace shape at load_frac of that capacity, the
    steady state, where p50 / p99 describe a server that keeps up."""
    film = workloads.voronoi_film(1024, 1024, 15, 10.0, seed=1)
    desc = ("Poisson trace (seed 1) of m(T) / constrained / film jobs 45/45/10%, cubes 8^3..256^3, films "
            "1024x1024x15 Voronoi (d = 10), 200 + 500 sweeps per job")
    over = _serve_trace(mc, workloads.poisson_trace(rate, n_requests, seed=1), n_eq, n_meas, film)
    capacity = over["req_per_s"]
    over.update(rate_per_s=rate, offered_load_frac=rate / capacity)
    steady_rate = load_frac * capacity
    steady = _serve_trace(mc, workloads.poisson_trace(steady_rate, n_requests, seed=1), n_eq, n_meas, film)
    steady.update(rate_per_s=steady_rate, offered_load_frac=load_frac)
    return {"requests": n_requests, "capacity_req_per_s": capacity,
            "capacity_note": "completion rate of the 20 req/s run, which the GPU cannot keep up with",
            "configured_20_per_s": over, "steady_state": steady, "offered_load_frac": load_frac,
            "workload": desc}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=4000)
    ap.add_argument("--warmup", type=int, default=50)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle CPU baseline")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the default launch shapes (for profiler runs, whose timings would mislead the tuner)")
    ap.add_argument("--quick", action="store_true", help="skip the side measurements (same as --side none)")
    ap.add_argument("--side", default="all",
                    choices=["all", "none", "fp64", "constrained", "anisotropy", "cubes", "general", "stiffness", "films",
                             "precision", "serving", "torque", "wall", "wave", "slabs", "paper"],
                    help="which side measurements to add to the line")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    _, _, cfg = workload_config()
    if args.impl == "reference":
        reference_arm(args, cfg)
    else:
        gpu_arm(args, cfg)


if __name__ == "__main__":
    main()
