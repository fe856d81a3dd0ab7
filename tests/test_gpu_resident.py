"""Resident sweeps (csrc/resident_pass.cuh): a lattice held in the SMs'
shared memory for a whole run of sweeps, one block per brick of rows, the
blocks waiting on their neighbours between the colour passes of Table A1
and on all blocks between sweeps, against the row passes.

The resident kernel keys the same Philox draws to the same sites and moves a
row with the row kernel's operations in the same order, and the cone rule
and the sample take the same integer totals, so the spins, the cone angle,
the per-sweep samples and the ensemble averages must equal the row passes'
bit for bit.  The lattices below split into bricks of every kind the planner
makes: the 128^3 lattice (8 x 19 bricks of up to 16 x 7 rows, ragged in z),
ragged in both y and z (64 x 64 rows in 11 x 13 bricks), bricks of one row,
bricks spanning all of y (the y neighbours wrap inside the brick) or all of
z; blocks of 512 and of 640 threads.  A host-set fault makes the wait for
every block's count of the first sweep wait for an arrival that never
comes: the launch ends with MC_ERR_TIMEOUT instead of hanging.
"""
import os
import subprocess
import sys

import numpy as np
import pytest

import paper_2103_03517_gb300 as mc
import workloads

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2103_03517_gb300 import build as libbuild
    libbuild.build()


def _run(dims, kw, spins, plan, path):
    ring = sum(n for n, meas in plan if meas)
    h = mc.mc_create_ex(mc.make_desc(dims, kernel_path=path, ring_capacity=max(1, ring), **kw))
    try:
        mc.mc_set_spins(h, spins)
        for n, meas in plan:
            mc.mc_sweep(h, n, measure=meas)
        N = dims[0] * dims[1] * dims[2]
        return (mc.mc_get_spins(h, N), mc.mc_get_theta(h), mc.mc_measure(h).asdict(),
                mc.mc_samples(h, max(1, ring)))
    finally:
        mc.mc_destroy(h)


def _assert_same(a, b, what):
    assert np.array_equal(a[0], b[0]), (what, int(np.sum(np.any(a[0] != b[0], axis=1))))
    assert a[1] == b[1], what
    assert a[2] == b[2], what
    assert np.array_equal(a[3], b[3]), what


RES_DIMS = [(128, 128, 128), (128, 64, 64), (128, 16, 16), (128, 4, 300), (128, 300, 4), (128, 2, 4)]


@pytest.mark.parametrize("dims", RES_DIMS)
def test_resident_sweeps_equal_row_passes_bit_for_bit(dims):
    """Unmeasured then measured sweeps (with the torque sums) from random
    spins, with cubic anisotropy and a field."""
    N = dims[0] * dims[1] * dims[2]
    spins = workloads.random_spins(N, 11)
    kw = dict(K_u=0.05, K_c=0.02, H=(0.02, 0.0, 0.05), T=0.9, seed=5)
    plan = [(3, False), (4, True)]
    a = _run(dims, kw, spins, plan, mc.MC_PATH_RESIDENT)
    b = _run(dims, kw, spins, plan, mc.MC_PATH_ROW)
    moved = np.any(a[0] != spins, axis=1).mean()
    assert moved > 0.5, moved
    _assert_same(a, b, dims)


def test_resident_sample_without_torques_and_fixed_cone():
    """Measured sweeps without the torque sums and without cone adaptation
    (adapt_in_measure = 0), near T_C."""
    dims = (128, 32, 8)
    spins = workloads.random_spins(128 * 32 * 8, 3)
    kw = dict(K_u=0.01, T=1.4, seed=2, sample_torque=0, adapt_in_measure=0)
    plan = [(5, False), (6, True), (2, False), (3, True)]
    _assert_same(_run(dims, kw, spins, plan, mc.MC_PATH_RESIDENT), _run(dims, kw, spins, plan, mc.MC_PATH_ROW),
                 "no torques")


def test_resident_run_longer_than_one_launch():
    """2050 sweeps in one call take two launches (2048 + 2): the chain
    continues across them, the cone angle adapting all the way."""
    dims = (128, 2, 4)
    spins = workloads.random_spins(128 * 8, 5)
    kw = dict(K_u=0.02, T=0.3, seed=9, theta0_deg=90)
    plan = [(2050, False), (3, True)]
    _assert_same(_run(dims, kw, spins, plan, mc.MC_PATH_RESIDENT), _run(dims, kw, spins, plan, mc.MC_PATH_ROW),
                 "two launches")


def test_automatic_path_sweeps_a_lone_lattice_resident():
    """On the automatic path a group of the one 128-wide lattice sweeps
    resident (the timed launches are of the resident kind) and equals the
    lattice swept by row passes."""
    dims = (128, 64, 32)
    N = dims[0] * dims[1] * dims[2]
    spins = workloads.random_spins(N, 8)
    kw = dict(K_u=0.01, T=1.1, seed=4, sample_torque=0)
    h = mc.mc_create_ex(mc.make_desc(dims, kernel_path=mc.MC_PATH_AUTO, ring_capacity=8, **kw))
    g = mc.mc_group_create([h])
    try:
        mc.mc_set_spins(h, spins)
        ms, n = mc.mc_group_time_kernels(g, 5, measure=True)
        assert n[3] == 1 and n[0] == n[1] == n[2] == 0, n
        assert ms[3] > 0.0
        mc.mc_group_sweep(g, 3)
        mc.mc_group_sync(g)
        a = (mc.mc_get_spins(h, N), mc.mc_get_theta(h), mc.mc_measure(h).asdict(), mc.mc_samples(h, 5))
    finally:
        mc.mc_group_destroy(g)
        mc.mc_destroy(h)
    _assert_same(a, _run(dims, kw, spins, [(5, True), (3, False)], mc.MC_PATH_ROW), "group")


def test_short_calls_mix_with_resident_launches():
    """Calls of one and two sweeps take the row passes (too short to pay for
    the lattice's load and store), longer ones resident launches; the chain
    is the row passes' chain throughout."""
    dims = (128, 32, 16)
    spins = workloads.random_spins(128 * 32 * 16, 14)
    kw = dict(K_u=0.03, K_c=0.01, T=0.8, seed=13)
    plan = [(1, False), (2, True), (5, False), (1, True), (4, True), (3, False)]
    _assert_same(_run(dims, kw, spins, plan, mc.MC_PATH_AUTO), _run(dims, kw, spins, plan, mc.MC_PATH_ROW),
                 "short calls")


def test_temperature_and_field_changes_between_resident_runs():
    """mc_set_temperature and mc_set_field between calls reach the next
    resident launch (the parameters are read from the lattice, not cached)."""
    dims = (128, 16, 32)
    N = dims[0] * dims[1] * dims[2]
    spins = workloads.random_spins(N, 15)
    out = []
    for path in (mc.MC_PATH_AUTO, mc.MC_PATH_ROW):
        h = mc.mc_create_ex(mc.make_desc(dims, K_u=0.02, T=1.2, seed=17, ring_capacity=8, kernel_path=path))
        try:
            mc.mc_set_spins(h, spins)
            mc.mc_sweep(h, 4)
            mc.mc_set_temperature(h, 0.6)
            mc.mc_set_field(h, (0.0, 0.05, 0.1))
            mc.mc_sweep(h, 5, measure=True)
            out.append((mc.mc_get_spins(h, N), mc.mc_get_theta(h), mc.mc_measure(h).asdict(), mc.mc_samples(h, 5)))
        finally:
            mc.mc_destroy(h)
    _assert_same(out[0], out[1], "T and H changes")


def test_resident_run_resumes_from_a_checkpoint(tmp_path):
    """A lattice saved between resident runs and loaded again continues the
    same chain as the one that kept running."""
    dims = (128, 32, 32)
    N = dims[0] * dims[1] * dims[2]
    spins = workloads.random_spins(N, 16)
    path = str(tmp_path / "res.ckpt")
    h = mc.mc_create_ex(mc.make_desc(dims, K_u=0.01, T=1.0, seed=18, ring_capacity=8))
    try:
        mc.mc_set_spins(h, spins)
        mc.mc_sweep(h, 6)
        mc.mc_save(h, path)
        mc.mc_sweep(h, 5, measure=True)
        a = (mc.mc_get_spins(h, N), mc.mc_get_theta(h), mc.mc_measure(h).asdict(), mc.mc_samples(h, 5))
    finally:
        mc.mc_destroy(h)
    c = mc.mc_load(path)
    try:
        mc.mc_sweep(c, 5, measure=True)
        b = (mc.mc_get_spins(c, N), mc.mc_get_theta(c), mc.mc_measure(c).asdict(), mc.mc_samples(c, 5))
    finally:
        mc.mc_destroy(c)
    _assert_same(a, b, "resume")


def test_two_resident_lattices_on_two_streams():
    """Two resident lattices swept at the same time on two streams: each
    launch wants every SM and neither waits on the other, so the second
    starts as the first drains; both give their row-pass chains."""
    import torch
    dims = [(128, 128, 64), (128, 64, 96)]
    spins = [workloads.random_spins(d[0] * d[1] * d[2], 20 + i) for i, d in enumerate(dims)]
    kws = [dict(K_u=0.02, T=0.7, seed=21), dict(K_u=0.01, K_c=0.01, T=1.1, seed=22)]
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    hs = [mc.mc_create_ex(mc.make_desc(d, ring_capacity=8, stream=int(st.cuda_stream), **kw))
          for d, kw, st in zip(dims, kws, streams)]
    try:
        for h, sp in zip(hs, spins):
            mc.mc_set_spins(h, sp)
        for _ in range(3):
            for h in hs:
                mc.mc_sweep(h, 40)
        for h in hs:
            mc.mc_sweep(h, 6, measure=True)
        got = []
        for h, d in zip(hs, dims):
            N = d[0] * d[1] * d[2]
            got.append((mc.mc_get_spins(h, N), mc.mc_get_theta(h), mc.mc_measure(h).asdict(), mc.mc_samples(h, 6)))
    finally:
        for h in hs:
            mc.mc_destroy(h)
    for d, kw, sp, g in zip(dims, kws, spins, got):
        _assert_same(g, _run(d, kw, sp, [(40, False)] * 3 + [(6, True)], mc.MC_PATH_ROW), d)


def test_group_of_large_resident_lattices_sweeps_them_one_after_another():
    """A group made only of resident lattices of at least 2^21 spins (two
    128^3) sweeps each held in shared memory in turn: one resident launch
    per lattice per call, each lattice on its row-pass chain.  A group with
    a smaller member keeps the batched row passes."""
    dims = (128, 128, 128)
    N = dims[0] * dims[1] * dims[2]
    spins = [workloads.random_spins(N, 30 + i) for i in range(2)]
    kws = [dict(K_u=0.01, T=0.9, seed=31), dict(K_u=0.02, K_c=0.01, T=1.2, seed=32)]
    hs = [mc.mc_create_ex(mc.make_desc(dims, ring_capacity=8, **kw)) for kw in kws]
    g = mc.mc_group_create(hs)
    try:
        for h, sp in zip(hs, spins):
            mc.mc_set_spins(h, sp)
        _, n = mc.mc_group_time_kernels(g, 4)
        assert n[3] == 2 and n[1] == 0, n
        mc.mc_group_sweep(g, 5, measure=True)
        mc.mc_group_sync(g)
        got = [(mc.mc_get_spins(h, N), mc.mc_get_theta(h), mc.mc_measure(h).asdict(), mc.mc_samples(h, 5))
               for h in hs]
    finally:
        mc.mc_group_destroy(g)
        for h in hs:
            mc.mc_destroy(h)
    for kw, sp, gt in zip(kws, spins, got):
        _assert_same(gt, _run(dims, kw, sp, [(4, False), (5, True)], mc.MC_PATH_ROW), "group")
    small = mc.mc_create_ex(mc.make_desc((128, 32, 32), T=1.0, seed=33))
    big = mc.mc_create_ex(mc.make_desc(dims, T=1.0, seed=34))
    g = mc.mc_group_create([small, big])
    try:
        _, n = mc.mc_group_time_kernels(g, 4)
        assert n[3] == 0 and n[1] == 8, n
    finally:
        mc.mc_group_destroy(g)
        mc.mc_destroy(small)
        mc.mc_destroy(big)


def test_both_resident_shapes_give_the_same_chain():
    """Blocks of 512 and of 640 threads (the tuner's two candidates) hand
    the rows out differently and give the same chain."""
    dims = (128, 64, 32)
    N = dims[0] * dims[1] * dims[2]
    spins = workloads.random_spins(N, 12)
    out = []
    for shape in (0, 1):
        h = mc.mc_create_ex(mc.make_desc(dims, K_u=0.02, T=1.0, seed=6, ring_capacity=4,
                                         kernel_path=mc.MC_PATH_RESIDENT))
        g = mc.mc_group_create([h])
        try:
            mc.mc_set_spins(h, spins)
            mc.mc_group_set_shapes(g, shape, 0, 0)
            mc.mc_group_sweep(g, 3)
            mc.mc_group_sweep(g, 4, measure=True)
            mc.mc_group_sync(g)
            out.append((mc.mc_get_spins(h, N), mc.mc_get_theta(h), mc.mc_measure(h).asdict(), mc.mc_samples(h, 4)))
        finally:
            mc.mc_group_destroy(g)
            mc.mc_destroy(h)
    _assert_same(out[0], out[1], "shapes")


def test_lattice_too_large_for_shared_memory_runs_row_passes():
    """128 x 128 x 160 (31 MB of spins) does not fit the blocks' shared
    memory: MC_PATH_RESIDENT then sweeps it by row passes."""
    dims = (128, 128, 160)
    h = mc.mc_create_ex(mc.make_desc(dims, kernel_path=mc.MC_PATH_RESIDENT, T=1.0, ring_capacity=4))
    g = mc.mc_group_create([h])
    try:
        _, n = mc.mc_group_time_kernels(g, 1)
        assert n[3] == 0 and n[1] == 2, n
    finally:
        mc.mc_group_destroy(g)
        mc.mc_destroy(h)


_TIMEOUT_CHILD = r"""
import sys
sys.path.insert(0, {root!r})
import paper_2103_03517_gb300 as mc
h = mc.mc_create_ex(mc.make_desc((128, 16, 16), T=1.0, seed=1, kernel_path=mc.MC_PATH_RESIDENT))
mc.mc_sweep(h, 3)
try:
    mc.mc_sync(h)
    print("NO_ERROR")
except mc.MCError as e:
    print("CODE", e.code)
mc.mc_destroy(h)
h = mc.mc_create_ex(mc.make_desc((128, 16, 16), T=1.0, seed=1, kernel_path=mc.MC_PATH_ROW))
mc.mc_sweep(h, 3)
mc.mc_sync(h)
print("CONTEXT_OK")
mc.mc_destroy(h)
"""


def test_a_missing_arrival_ends_in_a_timeout_error():
    """Fault injection on the host (MC_RESIDENT_INJECT_TIMEOUT=1): the wait
    for every block's count of a sweep expects one arrival more than there
    are blocks.  Every block's bounded wait gives up after about a second (or
    on the abort flag the first one raises), the launch ends, the lattice
    reports MC_ERR_TIMEOUT, and the context still runs other work (row
    passes: every resident lattice of the process has the fault)."""
    env = dict(os.environ, MC_RESIDENT_INJECT_TIMEOUT="1")
    r = subprocess.run([sys.executable, "-c", _TIMEOUT_CHILD.format(root=ROOT)], env=env, capture_output=True,
                       text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    assert f"CODE {mc.MC_ERR_TIMEOUT}" in r.stdout, r.stdout + r.stderr
    assert "CONTEXT_OK" in r.stdout, r.stdout + r.stderr
