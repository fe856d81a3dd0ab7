"""The launch-shape autotuner (mc_group_autotune, mc_autotune): it leaves the
chains exactly as they were, every later result is the same whatever shape
it picked, and its report is well formed."""
import numpy as np
import pytest

import paper_2103_03517_gb300 as mc
import workloads

pytestmark = pytest.mark.gpu


def _group(prec):
    """Lattices of every colour-pass kind: row layout (periodic), row layout
    with an open face, and the general kernel (Lh = 10)."""
    descs = [((32, 16, 16), (0, 0, 0)), ((64, 32, 8), (0, 0, 1)), ((20, 12, 8), (0, 0, 0)), ((64, 64, 64), (0, 0, 0))]
    return [mc.mc_create_ex(mc.make_desc(d, K_u=0.05, K_c=0.02, T=0.7, seed=i + 5, precision=prec, boundary=bc,
                                         init_dir=(0.6, 0.0, 0.8), ring_capacity=32)) for i, (d, bc) in enumerate(descs)]


@pytest.mark.parametrize("prec", [mc.MC_FP32, mc.MC_FP64])
def test_group_autotune_leaves_chains_unchanged(prec):
    runs = []
    for tune in (False, True):
        hs = _group(prec)
        g = mc.mc_group_create(hs)
        try:
            mc.mc_group_sweep(g, 5)
            mc.mc_group_constrained_sweep(g, [40.0] * 4, [10.0] * 4, 3)
            if tune:
                rep = mc.mc_group_autotune(g, 2)
                assert 0 <= rep["row"] < 2 and 0 <= rep["field"] < 3 and 0 <= rep["pair"] < 4
                assert all(t > 0 for t in rep["field_ms"][:3]) and all(t > 0 for t in rep["pair_ms"][:4])
                if prec == mc.MC_FP32:
                    assert all(t > 0 for t in rep["row_ms"][:2])
            mc.mc_group_sweep(g, 20, measure=True)
            mc.mc_group_constrained_sweep(g, [40.0] * 4, [10.0] * 4, 18, measure=True)
            mc.mc_group_sync(g)
        finally:
            mc.mc_group_destroy(g)
        dims = [(32, 16, 16), (64, 32, 8), (20, 12, 8), (64, 64, 64)]
        runs.append([(mc.mc_get_spins(h, int(np.prod(d))), mc.mc_measure(h).asdict(), mc.mc_get_theta(h))
                     for h, d in zip(hs, dims)])
        for h in hs:
            mc.mc_destroy(h)
    for a, b in zip(*runs):
        assert np.array_equal(a[0], b[0])
        assert a[1] == b[1] and a[2] == b[2]


def test_lone_lattice_autotune_and_errors():
    dims = (128, 128, 128)
    h = mc.mc_create_ex(mc.make_desc(dims, K_u=0.05, T=0.6, seed=3, init_dir=(0.0, 0.6, 0.8), ring_capacity=8))
    ref = mc.mc_create_ex(mc.make_desc(dims, K_u=0.05, T=0.6, seed=3, init_dir=(0.0, 0.6, 0.8), ring_capacity=8))
    try:
        rep = mc.mc_autotune(h, 2)
        for x in (h, ref):
            mc.mc_constrained_sweep(x, 35.0, 90.0, 17, measure=True)
            mc.mc_sweep(x, 17, measure=True)
        N = dims[0] * dims[1] * dims[2]
        assert np.array_equal(mc.mc_get_spins(h, N), mc.mc_get_spins(ref, N)), rep
        with pytest.raises(Exception):
            mc.mc_autotune(h, 0)
        with pytest.raises(Exception):
            mc.mc_autotune(h, 2, 0)
    finally:
        mc.mc_destroy(h)
        mc.mc_destroy(ref)
    x = mc.mc_create_ex(mc.make_desc((8, 8, 8), lattice=mc.MC_FCC, T=1.0))
    try:
        with pytest.raises(Exception):
            mc.mc_autotune(x, 2)
    finally:
        mc.mc_destroy(x)


def test_every_row_shape_gives_the_same_chain():
    """The row kernel's launch shapes (3 or 2 blocks per SM) change no bit:
    rows of 64, 128, 32 and 8 sites per colour, unmeasured and measured
    sweeps, runs of tiles of every length."""
    dims = [(128, 32, 16), (256, 16, 8), (64, 64, 16), (16, 16, 16), (32, 8, 8)]
    ref = None
    for shape in range(2):
        hs = [mc.mc_create_ex(mc.make_desc(d, K_u=0.05, K_c=0.01, H=(0.0, 0.02, 0.0), T=0.6 + 0.1 * i, seed=i + 3,
                                           init_dir=(0.3, 0.0, 0.95), ring_capacity=16)) for i, d in enumerate(dims)]
        g = mc.mc_group_create(hs)
        try:
            mc.mc_group_set_shapes(g, row=shape)
            mc.mc_group_sweep(g, 5)
            mc.mc_group_sweep(g, 6, measure=True)
            mc.mc_group_sync(g)
            got = [(mc.mc_get_spins(h, int(np.prod(d))), mc.mc_measure(h).asdict(), mc.mc_get_theta(h),
                    mc.mc_samples(h, 16)) for h, d in zip(hs, dims)]
        finally:
            mc.mc_group_destroy(g)
            for h in hs:
                mc.mc_destroy(h)
        if ref is None:
            ref = got
            continue
        for a, b in zip(ref, got):
            assert np.array_equal(a[0], b[0]), shape
            assert a[1] == b[1] and a[2] == b[2], shape
            assert np.array_equal(a[3], b[3]), shape
    with pytest.raises(mc.MCError):
        hs = [mc.mc_create_ex(mc.make_desc((16, 16, 16)))]
        g = mc.mc_group_create(hs)
        try:
            mc.mc_group_set_shapes(g, row=2)
        finally:
            mc.mc_group_destroy(g)
            mc.mc_destroy(hs[0])
