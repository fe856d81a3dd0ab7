"""The FP32 wavefront sweep (red and black pass of Table A1 in one launch,
csrc/wave_pass.cuh) against the two row passes it replaces.

Both key the same Philox draws to the same sites and evaluate the trial
point, Eq. 2 and Eq. 1 with the same operations in the same order, so a
wavefront sweep must give the spins, cone angle, accepted count and sample
of a red and a black row pass bit for bit, on any band / slab split of the
lattice (bands of at most 15 rows, slabs down to one plane, halo rows and planes
that wrap onto the band itself).  The per-sweep samples then agree too.  A
host-set fault makes a staged copy's wait run out: the launch ends with
MC_ERR_TIMEOUT instead of hanging.
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


def _run(dims, kw, spins, n_sweeps, path, calls=1):
    h = mc.mc_create_ex(mc.make_desc(dims, kernel_path=path, ring_capacity=max(1, n_sweeps * calls), **kw))
    try:
        mc.mc_set_spins(h, spins)
        for _ in range(calls):
            mc.mc_sweep(h, n_sweeps, measure=True)
        N = dims[0] * dims[1] * dims[2]
        return (mc.mc_get_spins(h, N), mc.mc_get_theta(h), mc.mc_measure(h).asdict(),
                mc.mc_samples(h, n_sweeps * calls))
    finally:
        mc.mc_destroy(h)


WAVE_DIMS = [(128, 16, 16), (128, 32, 8), (128, 48, 6), (128, 16, 2), (128, 64, 10), (128, 18, 4), (128, 30, 6),
             (128, 128, 128)]


@pytest.mark.parametrize("dims", WAVE_DIMS)
def test_wavefront_sweeps_equal_row_passes_bit_for_bit(dims):
    """Two, three (a wavefront pair then two row passes) and sixteen sweeps
    (a captured graph of eight wavefront pairs) from random spins."""
    N = dims[0] * dims[1] * dims[2]
    spins = workloads.random_spins(N, 11)
    kw = dict(K_u=0.05, K_c=0.02, H=(0.02, 0.0, 0.05), T=0.9, seed=5)
    for n in (2, 3, 16):
        w = _run(dims, kw, spins, n, mc.MC_PATH_WAVE)
        r = _run(dims, kw, spins, n, mc.MC_PATH_ROW)
        moved = np.any(w[0] != spins, axis=1).mean()
        assert moved > 0.5, moved
        assert np.array_equal(w[0], r[0]), (dims, n, int(np.sum(np.any(w[0] != r[0], axis=1))))
        assert w[1] == r[1]
        assert w[2] == r[2]
        assert np.array_equal(w[3], r[3])


def test_wavefront_lattice_in_a_group_equals_row_passes():
    """The batched temperature sweep with the wavefront path asked for (32
    lattices; the eight 128^3 ones take the wavefront launch, the others the
    row passes beside it) equals the same group on row passes, lattice by
    lattice."""
    specs = workloads.batched_mt_32()
    res = {}
    for path in (mc.MC_PATH_WAVE, mc.MC_PATH_ROW):
        hs = [mc.mc_create_ex(mc.make_desc(s.dims, K_u=s.Ku, T=s.T, seed=s.seed, kernel_path=path,
                                           ring_capacity=8, sample_torque=0)) for s in specs]
        g = mc.mc_group_create(hs)
        try:
            mc.mc_group_sweep(g, 6)
            mc.mc_group_sweep(g, 4, measure=True)
            mc.mc_group_sync(g)
            res[path] = [(mc.mc_get_spins(h, s.N), mc.mc_get_theta(h), mc.mc_measure(h).asdict())
                         for h, s in zip(hs, specs)]
        finally:
            mc.mc_group_destroy(g)
            for h in hs:
                mc.mc_destroy(h)
    for i, (a, b) in enumerate(zip(res[mc.MC_PATH_WAVE], res[mc.MC_PATH_ROW])):
        assert np.array_equal(a[0], b[0]), i
        assert a[1] == b[1] and a[2] == b[2], i


def test_wavefront_chain_continues_across_calls():
    """Calls of one, two and three sweeps in a row (pairs, odd tails) give
    the chain of one call of the same total length."""
    dims = (128, 32, 12)
    spins = workloads.random_spins(128 * 32 * 12, 4)
    kw = dict(K_u=0.01, T=1.2, seed=8)
    h = mc.mc_create_ex(mc.make_desc(dims, ring_capacity=16, kernel_path=mc.MC_PATH_WAVE, **kw))
    try:
        mc.mc_set_spins(h, spins)
        for n in (1, 2, 3):
            mc.mc_sweep(h, n, measure=True)
        a = mc.mc_get_spins(h, spins.shape[0]), mc.mc_get_theta(h)
    finally:
        mc.mc_destroy(h)
    b = _run(dims, kw, spins, 6, mc.MC_PATH_ROW)
    assert np.array_equal(a[0], b[0]) and a[1] == b[1]


_TIMEOUT_CHILD = r"""
import sys
sys.path.insert(0, {root!r})
import paper_2103_03517_gb300 as mc
h = mc.mc_create_ex(mc.make_desc((128, 16, 4), T=1.0, seed=1, kernel_path=mc.MC_PATH_WAVE))
mc.mc_sweep(h, 2)
try:
    mc.mc_sync(h)
    print("NO_ERROR")
except mc.MCError as e:
    print("CODE", e.code)
mc.mc_destroy(h)
"""


def test_a_staged_copy_that_never_completes_ends_in_a_timeout_error():
    """Fault injection on the host (MC_WAVE_INJECT_TIMEOUT=1): block 0's
    first staged copy expects 16 bytes more than are sent, so its mbarrier
    never completes.  The bounded wait gives up after about a second, the
    block drains its copies and leaves, and the lattice reports
    MC_ERR_TIMEOUT; the process is not hung and exits normally."""
    env = dict(os.environ, MC_WAVE_INJECT_TIMEOUT="1")
    r = subprocess.run([sys.executable, "-c", _TIMEOUT_CHILD.format(root=ROOT)], env=env, capture_output=True,
                       text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    assert f"CODE {mc.MC_ERR_TIMEOUT}" in r.stdout, r.stdout + r.stderr
