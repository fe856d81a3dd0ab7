"""One lattice split into z slabs (the domain decomposition of the paper's
multi-GPU projection, Sec. 2), run on one GPU: each slab holds its planes
plus a halo plane each side, the halos are refreshed after every colour
pass, the accepted counts and sample sums are summed over the slabs before
the sweep closes.  Draws are keyed by global site and colour, so the split
chain must equal the unsplit lattice's bit for bit: the spins of every
plane, the cone angle, the per-sweep samples and the ensemble averages
(samples are exact integer sums of the same per-site-pair parts).  Covered:
one slab wrapping onto itself, two and three slabs, slabs starting on odd
planes (their local colours are the global ones flipped), rows of 64 and of
16 sites per colour, a wall with pinned x planes, the one-device driver
(mc_slab_sweep), the rank driver of shard.py with one rank, and the
step-by-step protocol (planes and count words moved by the caller, as
between devices).
"""
import numpy as np
import pytest
import torch

import paper_2103_03517_gb300 as mc
from paper_2103_03517_gb300 import shard
import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2103_03517_gb300 import build as libbuild
    libbuild.build()


def _slab_spins(spins, dims, z0, nz):
    """The slab's local spins: global planes z0 - 1 .. z0 + nz (mod Lz)."""
    Lx, Ly, Lz = dims
    g = spins.reshape(Lz, Ly, Lx, 3)
    return g[[(z0 - 1 + k) % Lz for k in range(nz + 2)]].reshape(-1, 3)


def _gather(hs, splits, dims):
    Lx, Ly, Lz = dims
    out = np.zeros((Lz, Ly, Lx, 3))
    for h, (z0, nz) in zip(hs, splits):
        loc = mc.mc_get_spins(h, Lx * Ly * (nz + 2)).reshape(nz + 2, Ly, Lx, 3)
        out[z0:z0 + nz] = loc[1:nz + 1]
    return out.reshape(-1, 3)


def _unsplit(dims, kw, spins, plan):
    h = mc.mc_create_ex(mc.make_desc(dims, ring_capacity=64, **kw))
    try:
        mc.mc_set_spins(h, spins)
        for n, meas in plan:
            mc.mc_sweep(h, n, measure=meas)
        N = dims[0] * dims[1] * dims[2]
        return mc.mc_get_spins(h, N), mc.mc_get_theta(h), mc.mc_measure(h).asdict(), mc.mc_samples(h, 64)
    finally:
        mc.mc_destroy(h)


def _make_slabs(dims, kw, spins, splits, stream=None):
    hs = []
    for z0, nz in splits:
        h = mc.mc_slab_create(mc.make_desc(dims, ring_capacity=64, stream=stream, **kw), z0, nz)
        hs.append(h)
        mc.mc_set_spins(h, _slab_spins(spins, dims, z0, nz))
    return hs


def _results(hs, splits, dims):
    res = [(mc.mc_get_theta(h), mc.mc_measure(h).asdict(), mc.mc_samples(h, 64)) for h in hs]
    for r in res[1:]:  # every slab closes the same sweeps with the same totals
        assert r[0] == res[0][0]
        assert r[1] == res[0][1]
        assert np.array_equal(r[2], res[0][2])
    return (_gather(hs, splits, dims),) + res[0]


def _split(dims, kw, spins, splits, plan):
    stream = torch.cuda.Stream()  # mc_slab_sweep runs the slabs on one stream
    hs = _make_slabs(dims, kw, spins, splits, stream=int(stream.cuda_stream))
    try:
        for n, meas in plan:
            mc.mc_slab_sweep(hs, n, measure=meas)
        return _results(hs, splits, dims)
    finally:
        for h in hs:
            mc.mc_destroy(h)


def _assert_same(a, b):
    assert np.array_equal(a[0], b[0]), int(np.sum(np.any(a[0] != b[0], axis=1)))
    assert a[1] == b[1]
    assert a[2] == b[2]
    assert np.array_equal(a[3], b[3])


CASES = [
    ((128, 16, 16), [(0, 16)]),
    ((128, 16, 16), [(0, 8), (8, 8)]),
    ((128, 16, 16), [(0, 5), (5, 11)]),
    ((128, 16, 16), [(0, 6), (6, 3), (9, 7)]),
    ((32, 32, 12), [(0, 7), (7, 5)]),
]


@pytest.mark.parametrize("dims,splits", CASES)
def test_slabs_equal_the_unsplit_lattice_bit_for_bit(dims, splits):
    N = dims[0] * dims[1] * dims[2]
    spins = workloads.random_spins(N, 3)
    kw = dict(K_u=0.05, K_c=0.02, H=(0.02, 0.0, 0.05), T=0.9, seed=5)
    plan = [(3, False), (4, True)]
    a = _unsplit(dims, kw, spins, plan)
    b = _split(dims, kw, spins, splits, plan)
    moved = np.any(a[0] != spins, axis=1).mean()
    assert moved > 0.5, moved
    _assert_same(a, b)


def test_pinned_wall_in_slabs_equals_the_unsplit_wall():
    """The Bloch-wall geometry (x planes pinned at +z and -z, y and z
    periodic): pinned x planes inside every slab, halo planes on top."""
    dims = (128, 16, 16)
    kw = dict(K_u=0.05, T=0.4, seed=9, boundary=(mc.MC_PINNED, mc.MC_PERIODIC, mc.MC_PERIODIC))
    N = dims[0] * dims[1] * dims[2]
    x = np.arange(N) % dims[0]
    spins = np.zeros((N, 3))
    spins[:, 2] = np.where(x < dims[0] // 2, 1.0, -1.0)
    plan = [(5, False), (3, True)]
    _assert_same(_unsplit(dims, kw, spins, plan), _split(dims, kw, spins, [(0, 10), (10, 6)], plan))


def _stream():
    s = torch.cuda.Stream()
    return s, int(s.cuda_stream)


def test_rank_driver_with_one_rank_equals_the_unsplit_lattice():
    """shard.slab_sweep_ranks moves the planes and count words with torch
    on the library's stream; with one rank the slab is its own neighbour."""
    dims = (128, 16, 8)
    N = dims[0] * dims[1] * dims[2]
    spins = workloads.random_spins(N, 7)
    kw = dict(K_u=0.02, T=1.1, seed=2)
    a = _unsplit(dims, kw, spins, [(2, False), (3, True)])
    s, sp = _stream()
    with torch.cuda.stream(s):
        hs = _make_slabs(dims, kw, spins, [(0, 8)], stream=sp)
        try:
            shard.slab_sweep_ranks(hs[0], 2, measure=False)
            shard.slab_sweep_ranks(hs[0], 3, measure=True)
            s.synchronize()
            b = _results(hs, [(0, 8)], dims)
        finally:
            mc.mc_destroy(hs[0])
    _assert_same(a, b)


def test_step_by_step_protocol_equals_the_unsplit_lattice():
    """Two slabs driven call by call, the caller moving each colour's
    boundary planes into the neighbour's halo planes and summing the
    exported count words (what send/recv and an all-reduce do between
    devices)."""
    dims = (128, 16, 12)
    splits = [(0, 7), (7, 5)]
    N = dims[0] * dims[1] * dims[2]
    spins = workloads.random_spins(N, 8)
    kw = dict(K_u=0.03, H=(0.0, 0.01, 0.0), T=0.7, seed=11)
    a = _unsplit(dims, kw, spins, [(4, True)])
    s, sp = _stream()
    with torch.cuda.stream(s):
        hs = _make_slabs(dims, kw, spins, splits, stream=sp)
        try:
            for _ in range(4):
                for colour in (0, 1):
                    for h in hs:
                        mc.mc_slab_pass(h, colour, measure=colour == 1)
                    planes = []
                    for h in hs:
                        per = []
                        for which in range(4):
                            ptrs, n = mc.mc_slab_plane(h, colour, which)
                            per.append([shard.device_array(p, n, torch.float32) for p in ptrs])
                        planes.append(per)
                    for i in range(2):
                        j = 1 - i
                        for c in range(3):
                            planes[i][3][c].copy_(planes[j][0][c])  # upper halo <- neighbour's first plane
                            planes[i][2][c].copy_(planes[j][1][c])  # lower halo <- neighbour's last plane
                words = [shard.device_array(mc.mc_slab_export(h), mc.MC_SLAB_WORDS, torch.int64) for h in hs]
                total = words[0] + words[1]
                for w in words:
                    w.copy_(total)
                for h in hs:
                    mc.mc_slab_close(h, measure=True)
            s.synchronize()
            b = _results(hs, splits, dims)
        finally:
            for h in hs:
                mc.mc_destroy(h)
    _assert_same(a, b)


def test_slab_misuse_is_refused():
    dims = (128, 16, 16)
    h = mc.mc_slab_create(mc.make_desc(dims, T=1.0), 0, 8)
    try:
        assert mc.mc_slab_info(h) == (0, 8, 16)
        with pytest.raises(mc.MCError) as e:
            mc.mc_sweep(h, 1)
        assert e.value.code == mc.MC_ERR_STATE
        with pytest.raises(mc.MCError) as e:
            mc.mc_group_create([h])
        assert e.value.code == mc.MC_ERR_ARG
        with pytest.raises(mc.MCError) as e:
            mc.mc_slab_pass(h, 0, measure=True)  # the sample belongs to the black pass
        assert e.value.code == mc.MC_ERR_ARG
        with pytest.raises(mc.MCError) as e:
            mc.mc_slab_sweep([h], 1)  # one slab of 8 planes does not cover Lz = 16
        assert e.value.code == mc.MC_ERR_ARG
        with pytest.raises(mc.MCError) as e:
            mc.mc_save(h, "/dev/null")
        assert e.value.code == mc.MC_ERR_STATE
        with pytest.raises(mc.MCError):
            mc.mc_profile_sample(h)
    finally:
        mc.mc_destroy(h)
    for bad in (dict(precision=mc.MC_FP64), dict(boundary=(0, 0, mc.MC_PINNED))):
        with pytest.raises(mc.MCError) as e:
            mc.mc_slab_create(mc.make_desc(dims, **bad), 0, 8)
        assert e.value.code == mc.MC_ERR_ARG
    with pytest.raises(mc.MCError):
        mc.mc_slab_create(mc.make_desc(dims), 12, 8)  # planes beyond Lz
    h = mc.mc_create_ex(mc.make_desc(dims))
    try:
        with pytest.raises(mc.MCError):
            mc.mc_slab_pass(h, 0)  # not a slab
    finally:
        mc.mc_destroy(h)
