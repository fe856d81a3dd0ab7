"""Parity of the CUDA path (through the C ABI) with the serial FP64 oracle.

FP64 mode: the spin trajectory, the cone angle and the per-sweep accepted
counts are bit-identical to the oracle's, on every geometry (ragged tails,
open, pinned and periodic axes, films, constrained pairs) and at the full
batched workload; observables agree to 1e-9 relative.  FP32 mode: ensemble
averages agree within |delta| <= 2e-3 and 3 sigma of the sampling error.
"""
import math

import numpy as np
import pytest

import oracle
import paper_2103_03517_gb300 as mc
import workloads
from _stats import blocking_error

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2103_03517_gb300 import build as libbuild
    libbuild.build()
    oracle.build()


def make_pair(dims, prec=mc.MC_FP64, J=1.0, Ku=0.0, axis=(0, 0, 1.0), Kc=0.0, H=(0, 0, 0), T=1.0, seed=0,
              bc=(0, 0, 0), theta0=30, adapt=1, ring=4096, spins=None, film=None):
    kw = {}
    if film is not None:
        gid, mask, axes = film
        kw = dict(bond_mask=mask, grain_id=gid, grain_axis=axes)
    d = mc.make_desc(dims, J=J, K_u=Ku, axis=axis, K_c=Kc, H=H, T=T, seed=seed, precision=prec, boundary=bc,
                     theta0_deg=theta0, adapt_in_measure=adapt, ring_capacity=ring, **kw)
    h = mc.mc_create_ex(d)
    o = oracle.Lattice(dims, J=J, Ku=Ku, axis=axis, Kc=Kc, H=H, T=T, seed=seed, bc=bc, theta0=theta0,
                       adapt_in_measure=adapt, ring_cap=ring)
    if film is not None:
        o.set_bonds(film[1])
        o.set_grains(film[0], film[2])
    if spins is not None:
        mc.mc_set_spins(h, spins)
        o.set_spins(spins)
    return h, o


def assert_same_state(h, o, where=""):
    N = o.N
    g = mc.mc_get_spins(h, N)
    r = o.spins()
    diff = np.any(g != r, axis=1)
    assert not diff.any(), f"{where}: {diff.sum()} sites differ, first {int(np.argmax(diff))}: {g[diff][0]} vs {r[diff][0]}"
    theta, sweeps = mc.mc_get_theta(h)
    assert theta == o.theta, f"{where}: theta {theta} vs {o.theta}"
    assert sweeps == o.sweep_count


def assert_same_samples(h, o, n):
    gs = mc.mc_samples(h, n)
    os_ = o.samples(n)
    assert len(gs) == len(os_) == n
    assert np.array_equal(gs["sweep"], os_[:, 0].astype(np.int64))
    assert np.array_equal(gs["theta_deg"], os_[:, 1].astype(np.int32))
    assert np.array_equal(gs["accepted"], os_[:, 2].astype(np.int64))
    np.testing.assert_allclose(gs["m"], os_[:, 3:6], rtol=0, atol=1e-9)
    np.testing.assert_allclose(gs["e_parts"], os_[:, 6:10], rtol=0, atol=1e-9)
    np.testing.assert_allclose(gs["torque"], os_[:, 10:13], rtol=0, atol=1e-9)


def assert_same_stats(h, o):
    ob = mc.mc_measure(h)
    s = o.stats()
    n = s["n"]
    assert ob.n_samples == n
    if n == 0:
        return
    pairs = [(ob.ml, s["ml"]), (ob.ml2, s["ml2"]), (ob.ml4, s["ml4"]), (ob.e, s["e"]), (ob.e2, s["e2"])]
    pairs += [(ob.m[a], s["m" + c]) for a, c in enumerate("xyz")]
    pairs += [(ob.m2[a], s["m2" + c]) for a, c in enumerate("xyz")]
    pairs += [(ob.m_abs[a], s["mabs" + c]) for a, c in enumerate("xyz")]
    pairs += [(ob.torque[a], s["tq" + c]) for a, c in enumerate("xyz")]
    pairs += [(ob.e_parts[k], s[f]) for k, f in enumerate(("e_ex", "e_u", "e_c", "e_z"))]
    for g, r in pairs:
        assert abs(g - r / n) <= 1e-9 * max(1.0, abs(r / n)), (g, r / n)


# ------------------------------------------------------- FP64 bit-exactness
def test_fp64_point_16c_bit_exact():
    """16^3 periodic, K_u = 0.01 z, T = 0.5, seed 0, all +z: 1, 10 and
    1000 + 1000 sweeps."""
    c = workloads.point_16c()
    h, o = make_pair(c.dims, Ku=c.Ku, T=c.T, seed=c.seed, ring=1000)
    try:
        mc.mc_sweep(h, 1)
        o.sweep(1)
        assert_same_state(h, o, "after 1 sweep")
        mc.mc_sweep(h, 9)
        o.sweep(9)
        assert_same_state(h, o, "after 10 sweeps")
        mc.mc_sweep(h, 990)
        o.sweep(990)
        mc.mc_sweep(h, 1000, measure=True)
        o.sweep(1000, measure=True)
        assert_same_state(h, o, "after 2000 sweeps")
        assert_same_samples(h, o, 1000)
        assert_same_stats(h, o)
    finally:
        mc.mc_destroy(h)


GEOMETRIES = [
    ((24, 18, 10), (0, 0, 0)),   # several blocks per colour, ragged tail
    ((6, 3, 1), (1, 1, 1)),      # all open, odd sizes, a single plane
    ((4, 2, 6), (2, 0, 1)),      # pinned x planes, open z
    ((2, 1, 1), (1, 1, 1)),      # two spins
    ((2, 2, 2), (0, 0, 0)),      # every neighbour doubled by the wrap
    ((10, 6, 4), (0, 1, 0)),
    ((34, 1, 1), (0, 1, 1)),     # a periodic chain
    ((64, 6, 4), (0, 0, 0)),     # row fast path: one 32-site segment per row
    ((128, 2, 2), (0, 0, 0)),    # row fast path, y and z neighbours doubled by the wrap
    ((192, 4, 2), (0, 0, 0)),    # row fast path, three segments per row
    ((24, 6, 4), (3, 0, 0)),     # anti-periodic x (the wall setup)
    ((8, 6, 4), (3, 3, 1)),      # anti-periodic x and y, open z
    ((2, 2, 4), (3, 0, 3)),      # anti-periodic with doubled neighbours
    ((64, 4, 2), (3, 0, 0)),     # a row-sized lattice that must leave the row path
]


@pytest.mark.parametrize("dims,bc", GEOMETRIES)
@pytest.mark.parametrize("measure_all", [False, True])
def test_fp64_geometries_bit_exact(dims, bc, measure_all):
    N = dims[0] * dims[1] * dims[2]
    rng = np.random.default_rng(N)
    axis = rng.standard_normal(3)
    spins = workloads.random_spins(N, N + 1)
    h, o = make_pair(dims, J=1.0, Ku=0.3, axis=axis, Kc=0.2, H=(0.1, -0.2, 0.15), T=0.8, seed=N * 7 + 1, bc=bc,
                     spins=spins, ring=64)
    try:
        mc.mc_sweep(h, 7, measure=measure_all)
        o.sweep(7, measure=measure_all)
        assert_same_state(h, o, f"{dims} {bc}")
        mc.mc_sweep(h, 23, measure=True)
        o.sweep(23, measure=True)
        assert_same_state(h, o, f"{dims} {bc}")
        assert_same_samples(h, o, 23)
        assert_same_stats(h, o)
    finally:
        mc.mc_destroy(h)


def test_fp64_film_bit_exact():
    film = workloads.voronoi_film(32, 32, 4, 8.0, seed=3)
    h, o = make_pair((32, 32, 4), J=1.0, Ku=0.02, T=0.6, seed=11, bc=(0, 0, 1), film=film, ring=64)
    try:
        mc.mc_sweep(h, 10)
        o.sweep(10)
        mc.mc_sweep(h, 20, measure=True)
        o.sweep(20, measure=True)
        assert_same_state(h, o, "film")
        assert_same_samples(h, o, 20)
        assert_same_stats(h, o)
    finally:
        mc.mc_destroy(h)


@pytest.mark.parametrize("dims,th,ph,anti", [((16, 16, 16), 30.0, 20.0, False), ((12, 10, 8), 60.0, 45.0, False),
                                             ((6, 3, 1), 90.0, 0.0, False), ((34, 6, 6), 0.0, 0.0, False),
                                             ((12, 6, 4), 45.0, 0.0, True)])
def test_fp64_constrained_bit_exact(dims, th, ph, anti):
    N = dims[0] * dims[1] * dims[2]
    bc = tuple(0 if d % 2 == 0 else 1 for d in dims)
    if anti:
        bc = (3,) + bc[1:]
    R = oracle.constraint_frame(th, ph)
    spins = workloads.uniform_spins(N, R[0])
    h, o = make_pair(dims, J=1.0, Ku=0.05, Kc=0.02, H=(0.0, 0.05, 0.0), T=0.6, seed=5, bc=bc, spins=spins, ring=64)
    try:
        mc.mc_constrained_sweep(h, th, ph, 20)
        o.constrained_sweep(th, ph, 20)
        assert_same_state(h, o, "constrained")
        mc.mc_constrained_sweep(h, th, ph, 30, measure=True)
        o.constrained_sweep(th, ph, 30, measure=True)
        assert_same_state(h, o, "constrained measured")
        assert_same_samples(h, o, 30)
        assert_same_stats(h, o)
    finally:
        mc.mc_destroy(h)


def test_fp64_mixed_constrained_and_free_sweeps():
    dims = (8, 8, 8)
    h, o = make_pair(dims, Ku=0.05, T=0.9, seed=21, ring=64)
    try:
        for k in range(3):
            mc.mc_sweep(h, 5, measure=k == 2)
            o.sweep(5, measure=k == 2)
            mc.mc_constrained_sweep(h, 10.0 * k, 5.0, 5, measure=k == 1)
            o.constrained_sweep(10.0 * k, 5.0, 5, measure=k == 1)
        assert_same_state(h, o, "mixed")
        assert_same_stats(h, o)
    finally:
        mc.mc_destroy(h)


def test_fp64_temperature_and_field_changes():
    dims = (8, 6, 4)
    h, o = make_pair(dims, Ku=0.05, T=0.9, seed=2, ring=64)
    try:
        mc.mc_sweep(h, 5)
        o.sweep(5)
        mc.mc_set_temperature(h, 0.3)
        o.set_temperature(0.3)
        mc.mc_sweep(h, 5)
        o.sweep(5)
        assert_same_state(h, o, "after T change")
    finally:
        mc.mc_destroy(h)


def test_fp64_wall_profile():
    """Slice-averaged profile (Sec. 3 domain-wall profile) of a pinned wall:
    three samples at different times equal the mean of the oracle's slice
    averages of the same (bit-identical) states."""
    dims = (32, 8, 8)
    h, o = make_pair(dims, Ku=0.05, T=0.4, seed=9, bc=(2, 0, 0), spins=workloads.wall_spins(dims))
    try:
        ref = []
        for k in range(3):
            mc.mc_sweep(h, 10)
            o.sweep(10)
            mc.mc_profile_sample(h)
            S = o.spins().reshape(dims[2], dims[1], dims[0], 3)
            ref.append(S.mean(axis=(0, 1)))
        assert_same_state(h, o, "wall")
        ref = np.mean(ref, axis=0)
        for a in range(3):
            np.testing.assert_allclose(mc.mc_profile(h, a, dims[0]), ref[:, a], rtol=0, atol=1e-8)
        prof = mc.mc_profile(h, 2, dims[0])
        assert prof[0] == pytest.approx(1.0) and prof[-1] == pytest.approx(-1.0)
        mc.mc_reset_stats(h)
        assert np.all(mc.mc_profile(h, 2, dims[0]) == 0.0)
    finally:
        mc.mc_destroy(h)


def test_zero_sweeps_is_a_no_op():
    h, o = make_pair((4, 4, 4), T=0.5)
    try:
        mc.mc_sweep(h, 0)
        mc.mc_constrained_sweep(h, 0.0, 0.0, 0)
        assert_same_state(h, o, "no-op")
        assert mc.mc_measure(h).n_samples == 0
    finally:
        mc.mc_destroy(h)


def test_constraint_violation_reported():
    dims = (8, 8, 8)
    h = mc.mc_create_ex(mc.make_desc(dims, precision=mc.MC_FP64, init_dir=(0, 0, -1.0)))
    try:
        mc.mc_constrained_sweep(h, 0.0, 0.0, 2)  # M_L = -N <= 0
        with pytest.raises(mc.MCError) as e:
            mc.mc_sync(h)
        assert e.value.code == mc.MC_ERR_CONSTRAINT
    finally:
        mc.mc_destroy(h)


# ---------------------------------------------------------------- batching
@pytest.mark.parametrize("prec", [mc.MC_FP64, mc.MC_FP32])
def test_group_equals_alone_bitwise(prec):
    specs = [((16, 16, 16), 0.5, 1), ((8, 8, 6), 1.1, 2), ((32, 16, 16), 0.9, 3), ((6, 3, 1), 0.4, 4),
             ((64, 8, 4), 0.7, 5)]
    def make(dims, T, seed):
        bc = tuple(0 if d % 2 == 0 else 1 for d in dims)
        return mc.mc_create_ex(mc.make_desc(dims, K_u=0.05, K_c=0.01, T=T, seed=seed, precision=prec, boundary=bc,
                                            ring_capacity=64))
    grouped = [make(*s) for s in specs]
    alone = [make(*s) for s in specs]
    g = mc.mc_group_create(grouped)
    try:
        mc.mc_group_sweep(g, 37)
        mc.mc_group_sweep(g, 21, measure=True)
        batch = mc.mc_group_measure(g, len(grouped))   # one wait, creation order
        mc.mc_group_sync(g)
        for h in alone:
            mc.mc_sweep(h, 37)
            mc.mc_sweep(h, 21, measure=True)
        for (dims, _, _), a, b, ga in zip(specs, grouped, alone, batch):
            N = dims[0] * dims[1] * dims[2]
            assert np.array_equal(mc.mc_get_spins(a, N), mc.mc_get_spins(b, N))
            oa, ob = mc.mc_measure(a).asdict(), mc.mc_measure(b).asdict()
            assert oa == ob
            assert ga.asdict() == oa
    finally:
        mc.mc_group_destroy(g)
        for h in grouped + alone:
            mc.mc_destroy(h)


def test_group_constrained_equals_alone_bitwise():
    specs = [((16, 16, 16), 0.5, 30.0, 0.0), ((12, 10, 8), 0.8, 60.0, 45.0)]
    hs, al = [], []
    for dims, T, th, ph in specs:
        R = oracle.constraint_frame(th, ph)
        for lst in (hs, al):
            h = mc.mc_create_ex(mc.make_desc(dims, K_u=0.05, K_c=0.02, T=T, seed=4, precision=mc.MC_FP64,
                                             init_dir=tuple(R[0]), ring_capacity=64))
            lst.append(h)
    g = mc.mc_group_create(hs)
    try:
        mc.mc_group_constrained_sweep(g, [s[2] for s in specs], [s[3] for s in specs], 20, measure=True)
        mc.mc_group_sync(g)
        for h, s in zip(al, specs):
            mc.mc_constrained_sweep(h, s[2], s[3], 20, measure=True)
        for (dims, *_), a, b in zip(specs, hs, al):
            N = dims[0] * dims[1] * dims[2]
            assert np.array_equal(mc.mc_get_spins(a, N), mc.mc_get_spins(b, N))
            assert mc.mc_measure(a).asdict() == mc.mc_measure(b).asdict()
    finally:
        mc.mc_group_destroy(g)
        for h in hs + al:
            mc.mc_destroy(h)


def _one_sweep_pair(dims, kw_a, kw_b, spins, n_sweeps=1):
    """Spins and energy of two lattices started from the same spins after
    n_sweeps measured sweeps."""
    out = []
    for kw in (kw_a, kw_b):
        h = mc.mc_create_ex(mc.make_desc(dims, **kw))
        try:
            mc.mc_set_spins(h, spins)
            mc.mc_sweep(h, n_sweeps, measure=True)
            out.append((mc.mc_get_spins(h, len(spins)), mc.mc_measure(h).e))
        finally:
            mc.mc_destroy(h)
    return out


def _assert_same_chain(spins, a, b, label):
    (sa, ea), (sb, eb) = a, b
    moved = np.any(sa != spins, axis=1).mean()
    assert moved > 0.2, (label, moved)
    close = np.all(np.abs(sa - sb) < 1e-5, axis=1)
    assert close.mean() > 0.999, (label, close.mean())
    assert abs(ea - eb) < 1e-5, (label, ea, eb)


@pytest.mark.parametrize("dims", [(16, 16, 16), (8, 8, 8), (4, 4, 8), (64, 32, 8), (128, 8, 4), (256, 4, 4),
                                  (384, 2, 2), (64, 64, 16), (128, 16, 32), (128, 8, 16), (256, 8, 16), (512, 4, 16),
                                  (512, 2, 32)])
def test_fp32_row_kernels_match_general_kernel(dims):
    """FP32, every axis periodic: the row kernel (no film tables), the row
    kernel with boundaries and films (an all-ones bond mask, the same
    physics) and the general kernel (forced) key the same draws to the same
    sites, so one sweep gives the same spins up to FP32 rounding; a wrong
    neighbour would change many sites by O(1)."""
    N = dims[0] * dims[1] * dims[2]
    spins = workloads.random_spins(N, 7)
    kw = dict(K_u=0.05, K_c=0.02, H=(0.02, 0.0, 0.05), T=0.9, seed=12, ring_capacity=8)
    row, gen = _one_sweep_pair(dims, kw, dict(kw, kernel_path=mc.MC_PATH_GENERAL), spins)
    _assert_same_chain(spins, row, gen, f"row {dims}")
    rowx, gen2 = _one_sweep_pair(dims, dict(kw, bond_mask=np.full(N, 0x3F, np.uint8)),
                                 dict(kw, kernel_path=mc.MC_PATH_GENERAL), spins)
    _assert_same_chain(spins, rowx, gen2, f"rowx {dims}")


ROWX_CASES = [
    ((64, 16, 8), (3, 0, 0), False),     # anti-periodic x (the wall setup)
    ((128, 8, 6), (2, 0, 0), False),     # pinned x planes
    ((32, 9, 4), (1, 1, 1), False),      # all open, odd Ly
    ((16, 8, 4), (0, 3, 1), False),      # anti-periodic y, open z
    ((256, 6, 4), (3, 2, 3), False),     # long rows, pinned y, anti-periodic z
    ((64, 64, 4), (0, 0, 1), True),      # film: bond mask and grain axes, open z
    ((128, 32, 3), (3, 0, 1), True),     # film on an anti-periodic x
]


@pytest.mark.parametrize("dims,bc,film", ROWX_CASES)
def test_fp32_row_kernel_with_boundaries_matches_general_kernel(dims, bc, film):
    """FP32 lattices in the row layout with open, pinned and anti-periodic
    faces, bond masks and grain axes: the row kernel and the general kernel
    (forced) run the same chain."""
    Lh = dims[0] // 2
    assert (Lh & (Lh - 1) == 0 and Lh <= 64) or Lh % 64 == 0
    assert (Lh * dims[1] * dims[2]) % 64 == 0  # the row layout, so AUTO takes the row kernel
    N = dims[0] * dims[1] * dims[2]
    spins = workloads.random_spins(N, 3)
    kw = dict(K_u=0.05, K_c=0.02, H=(0.01, 0.02, 0.05), T=0.8, seed=21, ring_capacity=8, boundary=bc)
    if film:
        gid, mask, axes = workloads.voronoi_film(dims[0], dims[1], dims[2], 6.0, seed=2)
        kw.update(bond_mask=mask, grain_id=gid, grain_axis=axes)
    for n in (1, 3):
        a, b = _one_sweep_pair(dims, kw, dict(kw, kernel_path=mc.MC_PATH_GENERAL), spins, n_sweeps=n)
        if n == 1:
            _assert_same_chain(spins, a, b, f"{dims} {bc} film={film}")
        else:  # a few sweeps: still the same chain on nearly every site
            assert np.all(np.abs(a[0] - b[0]) < 1e-4, axis=1).mean() > 0.99


@pytest.mark.parametrize("dims", [(16, 16, 16), (64, 8, 4)])
def test_sampling_without_torque_changes_nothing_else(dims):
    """sample_torque = 0 drops only the torque sums: spins, m and energies
    are bit-identical to full sampling, torques read zero."""
    N = dims[0] * dims[1] * dims[2]
    a = mc.mc_create_ex(mc.make_desc(dims, K_u=0.05, K_c=0.02, H=(0, 0.05, 0), T=0.7, seed=3, ring_capacity=64))
    b = mc.mc_create_ex(mc.make_desc(dims, K_u=0.05, K_c=0.02, H=(0, 0.05, 0), T=0.7, seed=3, ring_capacity=64,
                                     sample_torque=0))
    try:
        for h in (a, b):
            mc.mc_sweep(h, 20)
            mc.mc_sweep(h, 40, measure=True)
        assert np.array_equal(mc.mc_get_spins(a, N), mc.mc_get_spins(b, N))
        oa, ob = mc.mc_measure(a), mc.mc_measure(b)
        for f in ("m", "m2", "ml", "ml2", "ml4", "e", "e2", "e_parts", "chi"):
            assert getattr(oa, f) == getattr(ob, f) if not hasattr(getattr(oa, f), "__len__") else \
                list(getattr(oa, f)) == list(getattr(ob, f)), f
        assert list(ob.torque) == [0.0, 0.0, 0.0] and any(x != 0.0 for x in oa.torque)
    finally:
        mc.mc_destroy(a)
        mc.mc_destroy(b)


@pytest.mark.parametrize("prec", [mc.MC_FP64, mc.MC_FP32])
def test_checkpoint_resume_is_bit_exact(prec, tmp_path):
    dims = (16, 12, 8)
    d = mc.make_desc(dims, K_u=0.05, T=0.7, seed=13, precision=prec, ring_capacity=64)
    a = mc.mc_create_ex(d)
    b = mc.mc_create_ex(d)
    try:
        mc.mc_sweep(a, 60)
        mc.mc_sweep(a, 40, measure=True)
        mc.mc_sweep(b, 60)
        mc.mc_sweep(b, 10, measure=True)
        path = str(tmp_path / "ck.bin")
        mc.mc_save(b, path)
        c = mc.mc_load(path)
        mc.mc_sweep(c, 30, measure=True)
        N = dims[0] * dims[1] * dims[2]
        assert np.array_equal(mc.mc_get_spins(a, N), mc.mc_get_spins(c, N))
        assert mc.mc_measure(a).asdict() == mc.mc_measure(c).asdict()
        mc.mc_destroy(c)
    finally:
        mc.mc_destroy(a)
        mc.mc_destroy(b)


# ------------------------------------------- full size, bench launch config
def test_batched_mt_full_size_fp64_two_sweeps_bit_exact():
    """All 32 lattices of the batched m(T) workload (19,169,280 spins) in one
    group, FP64: two sweeps agree with the oracle bit for bit."""
    specs = workloads.batched_mt_32()
    hs = [mc.mc_create_ex(mc.make_desc(s.dims, K_u=s.Ku, T=s.T, seed=s.seed, precision=mc.MC_FP64,
                                       ring_capacity=4)) for s in specs]
    g = mc.mc_group_create(hs)
    try:
        mc.mc_group_sweep(g, 1)
        mc.mc_group_sweep(g, 1, measure=True)
        mc.mc_group_sync(g)
        for s, h in zip(specs, hs):
            o = oracle.Lattice(s.dims, Ku=s.Ku, T=s.T, seed=s.seed, ring_cap=4)
            o.sweep(1)
            o.sweep(1, measure=True)
            assert_same_state(h, o, f"batched m(T) L={s.dims[0]} T={s.T:.2f}")
            assert_same_stats(h, o)
    finally:
        mc.mc_group_destroy(g)
        for h in hs:
            mc.mc_destroy(h)


def test_batched_mt_full_size_fp32_properties():
    """The bench's FP32 group of 32 lattices: after 400 sweeps every spin is a
    unit vector, cone angles settled with acceptance near one half, and the
    coldest lattice obeys equipartition E/N = -3J - K_u + T (any size)."""
    specs = workloads.batched_mt_32()
    hs = [mc.mc_create_ex(mc.make_desc(s.dims, K_u=s.Ku, T=s.T, seed=s.seed, ring_capacity=256)) for s in specs]
    g = mc.mc_group_create(hs)
    try:
        mc.mc_group_sweep(g, 200)
        mc.mc_group_sweep(g, 200, measure=True)
        mc.mc_group_sync(g)
        for s, h in zip(specs, hs):
            S = mc.mc_get_spins(h, s.N)
            assert np.abs(np.linalg.norm(S, axis=1) - 1.0).max() < 2e-6
            ob = mc.mc_measure(h)
            samp = mc.mc_samples(h, 200)
            acc = samp["accepted"] / s.N
            if ob.theta_deg < 180:  # below the cap the cone angle holds acceptance at one half
                assert 1 < ob.theta_deg and abs(acc.mean() - 0.5) < 0.05, (s.dims, s.T, acc.mean())
            else:
                assert acc.mean() > 0.45
        cold = mc.mc_measure(hs[0])  # T = 0.05, 16^3
        assert abs((cold.e + 3.01) / 0.05 - 1.0) < 0.05
        big = mc.mc_measure(hs[3])   # T = 0.2, 128^3: harmonic spin waves
        L = 128
        k = 2 * np.pi * np.arange(L) / L
        c = np.cos(k)
        eps = (3 - c[:, None, None] - c[None, :, None] - c[None, None, :]).ravel()[1:]
        W = (1 / (eps + 0.01)).sum() / L ** 3  # transverse modes gapped by K_u
        ratio = (1 - big.ml) / (0.2 / 2 * W)
        assert 1.0 < ratio < 1.12, ratio  # anharmonic correction ~ +0.3 T
    finally:
        mc.mc_group_destroy(g)
        for h in hs:
            mc.mc_destroy(h)


# ------------------------------------------------------ FP32 ensembles
def _oracle_series(dims, Ku, T, seed, n_eq, n_meas, constrained=None, Kc=0.0):
    o = oracle.Lattice(dims, Ku=Ku, Kc=Kc, T=T, seed=seed, ring_cap=n_meas)
    if constrained:
        th, ph = constrained
        R = oracle.constraint_frame(th, ph)
        o.set_spins(workloads.uniform_spins(o.N, R[0]))
        o.constrained_sweep(th, ph, n_eq)
        o.constrained_sweep(th, ph, n_meas, measure=True)
    else:
        o.sweep(n_eq)
        o.sweep(n_meas, measure=True)
    return o.samples()


@pytest.mark.parametrize("T", [0.5, 1.2])
def test_fp32_ensemble_matches_oracle(T):
    """16^3, K_u = 0.01: 128 independent FP32 chains against 128 FP64 chains
    (FP64 on the GPU is the oracle's chain bit for bit, as the tests above
    show), 500 + 2000 sweeps each from +z.  The mean over chains of <|m|> and
    <|m|^2> agree within |d| <= 2e-3 and 3 sigma, <E/N> within 3 sigma, sigma
    from the spread between chains; enough chains that 2e-3 is more than 3
    sigma.  The near-T_C lattices are covered against the stored oracle
    ensembles in test_gpu_precision.py."""
    from paper_2103_03517_gb300 import studies
    spec = workloads.LatticeSpec(dims=(16, 16, 16), Ku=0.01, T=T)
    res = {}
    for prec in (mc.MC_FP32, mc.MC_FP64):
        res[prec] = studies.chain_ensembles({"c": spec}, {"c": 128}, lambda n, k: 5000 * prec + k,
                                            lambda n: (500, 2000), precision=prec)["c"]
    for key in ("ml", "ml2", "e"):
        a, b = res[mc.MC_FP32][key], res[mc.MC_FP64][key]
        d = float(a.mean() - b.mean())
        sig = math.sqrt(a.var(ddof=1) / a.size + b.var(ddof=1) / b.size)
        assert abs(d) <= 3 * sig, (T, key, d, sig)
        if key != "e":
            assert abs(d) <= 2e-3 and sig < 6.7e-4, (T, key, d, sig)


@pytest.mark.parametrize("H,T", [((0.0, 0.0, 1.5), 1.0), ((0.3, -0.4, 1.2), 0.7)])
def test_fp32_langevin_law(H, T):
    """J = 0 in FP32 mode: independent moments in a field obey
    <S.h^> = coth(|H|/T) - T/|H| (pins the FP32 cone sampler and the
    acceptance test against a closed form).  Sixteen independent lattices;
    the mean of their means lies within the 3-sigma-equivalent bound (t3)
    of its standard error from the spread between lattices."""
    from _stats import langevin, t3
    hs = [mc.mc_create_ex(mc.make_desc((64, 32, 32), J=0.0, H=H, T=T, seed=4 + k, ring_capacity=16))
          for k in range(16)]
    g = mc.mc_group_create(hs)
    try:
        mc.mc_group_sweep(g, 300)
        mc.mc_group_sweep(g, 2000, measure=True)
        hh = np.asarray(H) / np.linalg.norm(H)
        proj = np.array([np.dot(o.m, hh) for o in mc.mc_group_measure(g, len(hs))])
    finally:
        mc.mc_group_destroy(g)
        for h in hs:
            mc.mc_destroy(h)
    expect = langevin(np.linalg.norm(H) / T)
    se = proj.std(ddof=1) / math.sqrt(proj.size)
    assert abs(proj.mean() - expect) <= t3(proj.size - 1) * se + 1e-6, (proj.mean(), expect, se)


def test_fp32_constrained_torque_matches_oracle():
    """FP32 constrained torque tau_y against the oracle's FP64 chain: six
    independent runs on each side; the difference of the mean run means lies
    within the 3-sigma-equivalent bound (the Student-t quantile with the
    two-sided coverage of 3 sigma, 10 degrees of freedom) of the pooled
    spread between runs.  One run's blocking error understates the
    run-to-run spread of this 3000-sample series about twice, so the spread
    is taken between runs."""
    dims, T, th = (16, 16, 16), 0.5, 45.0
    n_eq, n_meas, runs = 500, 3000, 6
    R = oracle.constraint_frame(th, 0.0)
    gm, rm = [], []
    for k in range(runs):
        h = mc.mc_create_ex(mc.make_desc(dims, K_u=0.05, K_c=0.02, T=T, seed=1 + k, init_dir=tuple(R[0]),
                                         ring_capacity=n_meas))
        try:
            mc.mc_constrained_sweep(h, th, 0.0, n_eq)
            mc.mc_constrained_sweep(h, th, 0.0, n_meas, measure=True)
            gm.append(mc.mc_samples(h, n_meas)["torque"][:, 1].mean())
        finally:
            mc.mc_destroy(h)
        rm.append(_oracle_series(dims, 0.05, T, 101 + k, n_eq, n_meas, constrained=(th, 0.0), Kc=0.02)[:, 11].mean())
    gm, rm = np.array(gm), np.array(rm)
    pooled = math.sqrt((gm.var(ddof=1) + rm.var(ddof=1)) / 2)
    sig = pooled * math.sqrt(2.0 / runs)
    from _stats import t3
    assert abs(gm.mean() - rm.mean()) <= t3(2 * runs - 2) * sig, (gm.mean(), rm.mean(), sig)


@pytest.mark.parametrize("dims", [(160, 160, 160), (32, 32, 32), (40, 36, 30)])
def test_fp32_constrained_site_order_equals_pair_order(dims):
    """An FP32 lattice takes its constrained pairs in site order; forced to
    pair order (MC_PATH_GENERAL) it runs the same pairs with the same draws,
    so the spins are equal bit for bit.  160^3: spins and packed copy far
    above L2; 32^3: N_c a power of two (no cycle-walking); 40x36x30: N_c =
    21600, walks in both directions of the shuffle.  The samples agree to
    1e-9: on a row-layout lattice (32^3) the two paths sample with different
    kernels, whose FP32 lane sums round to fixed point in other groups."""
    th = 40.0
    N = dims[0] * dims[1] * dims[2]
    R = oracle.constraint_frame(th, 0.0)
    out = []
    for path in (mc.MC_PATH_AUTO, mc.MC_PATH_GENERAL):
        h = mc.mc_create_ex(mc.make_desc(dims, K_u=0.05, K_c=0.02, T=0.7, seed=9, init_dir=tuple(R[0]),
                                         ring_capacity=8, kernel_path=path))
        try:
            mc.mc_constrained_sweep(h, th, 0.0, 3, measure=True)
            out.append((mc.mc_get_spins(h, N), mc.mc_measure(h)))
        finally:
            mc.mc_destroy(h)
    assert np.array_equal(out[0][0], out[1][0])
    assert abs(out[0][1].torque[1] - out[1][1].torque[1]) <= 1e-9
    assert abs(out[0][1].e - out[1][1].e) <= 1e-9


# ------------------------- full size: constrained 64^3, Bloch wall, granular film (bench workloads)
def test_constrained_64c_full_size_lattice_fp64_bit_exact():
    """One lattice of the constrained workload at its full size (64^3,
    theta_c = 40, phi_c = 45, T = 0.2), FP64: two constrained sweeps, the
    second measured, equal the oracle's chain bit for bit (spins, theta,
    samples with the torque)."""
    spec, th, ph = workloads.constrained_64c_runs()[14]
    R = oracle.constraint_frame(th, ph)
    spins = workloads.uniform_spins(spec.N, R[0])
    h, o = make_pair(spec.dims, Ku=spec.Ku, Kc=spec.Kc, T=spec.T, seed=spec.seed, ring=4, spins=spins)
    try:
        mc.mc_constrained_sweep(h, th, ph, 1)
        o.constrained_sweep(th, ph, 1)
        mc.mc_constrained_sweep(h, th, ph, 1, measure=True)
        o.constrained_sweep(th, ph, 1, measure=True)
        assert_same_state(h, o, "constrained 64^3")
        assert_same_samples(h, o, 1)
    finally:
        mc.mc_destroy(h)


def test_constrained_64c_full_size_fp32_batch_properties():
    """The bench's FP32 constrained batch (80 x 64^3, site order): after 20
    sweeps every lattice keeps its transverse magnetisation at zero and its
    projection on e_C positive (to FP32 rounding of the compensation), spins
    stay unit vectors (the partner is not renormalised: to FP32 rounding),
    and the acceptance sits at one half or the cone is fully open."""
    runs = workloads.constrained_64c_runs()
    hs = []
    for spec, th, ph in runs:
        R = oracle.constraint_frame(th, ph)
        hs.append(mc.mc_create_ex(mc.make_desc(spec.dims, K_u=spec.Ku, K_c=spec.Kc, T=spec.T, seed=spec.seed,
                                               init_dir=tuple(R[0]), ring_capacity=32)))
    g = mc.mc_group_create(hs)
    try:
        mc.mc_group_constrained_sweep(g, [r[1] for r in runs], [r[2] for r in runs], 20, measure=True)
        mc.mc_group_sync(g)
        for (spec, th, ph), h in zip(runs, hs):
            R = oracle.constraint_frame(th, ph)
            S = mc.mc_get_spins(h, spec.N)
            M = S.sum(axis=0)
            assert abs(M @ R[1]) < 1e-3 * spec.N and abs(M @ R[2]) < 1e-3 * spec.N and M @ R[0] > 0, (th, ph, M)
            assert np.abs(np.linalg.norm(S, axis=1) - 1.0).max() < 1e-4
            ob = mc.mc_measure(h)
            acc = mc.mc_samples(h, 20)["accepted"][-10:] / spec.N
            assert ob.theta_deg == 180 or abs(acc.mean() - 0.5) < 0.1, (spec.T, th, ob.theta_deg, acc.mean())
    finally:
        mc.mc_group_destroy(g)
        for h in hs:
            mc.mc_destroy(h)


def test_wall_1024x128x128_full_size_fp64_bit_exact():
    """The Bloch-wall lattice at its full size (1024 x 128 x 128, x pinned,
    16,777,216 spins, T = 0.66), FP64: one sweep and one measured sweep equal
    the oracle's chain bit for bit; the pinned planes keep +z and -z."""
    spec = workloads.bloch_wall_1024()[3]
    spins = workloads.wall_spins(spec.dims)
    h, o = make_pair(spec.dims, Ku=spec.Ku, T=spec.T, seed=spec.seed, bc=spec.bc, ring=4, spins=spins)
    try:
        mc.mc_sweep(h, 1)
        o.sweep(1)
        mc.mc_sweep(h, 1, measure=True)
        o.sweep(1, measure=True)
        assert_same_state(h, o, "Bloch wall 1024x128x128")
        assert_same_samples(h, o, 1)
        S = mc.mc_get_spins(h, spec.N).reshape(spec.dims[2], spec.dims[1], spec.dims[0], 3)
        assert np.all(S[:, :, 0, 2] == 1.0) and np.all(S[:, :, -1, 2] == -1.0)
    finally:
        mc.mc_destroy(h)


def test_film_1024x1024x15_full_size_fp64_bit_exact():
    """The serving mix's granular film at its full size (1024 x 1024 x 15,
    Voronoi grains of mean diameter 10, 15,728,640 spins), FP64: one sweep and
    one measured sweep equal the oracle's chain bit for bit."""
    dims = (1024, 1024, 15)
    film = workloads.voronoi_film(*dims, 10.0, seed=1)
    h, o = make_pair(dims, Ku=0.02, T=0.8, seed=5, bc=(0, 0, 1), ring=4, film=film)
    try:
        mc.mc_sweep(h, 1)
        o.sweep(1)
        mc.mc_sweep(h, 1, measure=True)
        o.sweep(1, measure=True)
        assert_same_state(h, o, "film 1024x1024x15")
        assert_same_samples(h, o, 1)
    finally:
        mc.mc_destroy(h)


# ---------------------------------------------- degenerate cone angles
@pytest.mark.parametrize("T,theta0,limit", [(60.0, 176, 180), (1e-4, 4, 1)])
def test_fp64_cone_at_its_limits_bit_exact(T, theta0, limit):
    """Table A1's cone rule at its ends: far above T_C nearly every move is
    accepted and theta climbs to 180 degrees (the trial point is uniform on
    the whole sphere) and stays; near T = 0 nearly every move is rejected and
    theta falls to 1 degree.  The GPU follows the oracle bit for bit there."""
    dims = (24, 6, 4)
    h, o = make_pair(dims, Ku=0.05, Kc=0.02, H=(0.0, 0.01, 0.03), T=T, seed=13, theta0=theta0, ring=64)
    try:
        mc.mc_sweep(h, 30)
        o.sweep(30)
        mc.mc_sweep(h, 40, measure=True)
        o.sweep(40, measure=True)
        assert_same_state(h, o, f"T = {T}")
        assert_same_samples(h, o, 40)
        assert_same_stats(h, o)
        assert mc.mc_get_theta(h)[0] == limit
    finally:
        mc.mc_destroy(h)


@pytest.mark.parametrize("prec", [mc.MC_FP64, mc.MC_FP32])
def test_cone_frozen_in_measurement_sweeps(prec):
    """adapt_in_measure = 0: the cone angle adapts in the unmeasured sweeps
    only; FP64 follows the oracle bit for bit, FP32 keeps the angle of the
    last unmeasured sweep through every sample."""
    dims = (64, 6, 4)
    h, o = make_pair(dims, prec=prec, Ku=0.02, T=0.9, seed=4, theta0=60, adapt=0, ring=64)
    try:
        mc.mc_sweep(h, 12)
        theta = mc.mc_get_theta(h)[0]
        mc.mc_sweep(h, 25, measure=True)
        s = mc.mc_samples(h, 25)
        assert np.all(s["theta_deg"] == theta)
        if prec == mc.MC_FP64:
            o.sweep(12)
            o.sweep(25, measure=True)
            assert_same_state(h, o, "frozen cone")
            assert_same_samples(h, o, 25)
    finally:
        mc.mc_destroy(h)


def test_fp32_spins_stay_unit_at_the_cone_limits():
    """FP32 renormalises every trial point: after sweeps with theta at 180
    and at 1 degree every spin has unit length to FP32 accuracy."""
    for T, theta0 in ((60.0, 176), (1e-4, 4)):
        dims = (128, 8, 8)
        h = mc.mc_create_ex(mc.make_desc(dims, K_u=0.05, T=T, seed=2, theta0_deg=theta0, ring_capacity=8))
        try:
            mc.mc_sweep(h, 40, measure=True)
            S = mc.mc_get_spins(h, dims[0] * dims[1] * dims[2])
            n = np.linalg.norm(S, axis=1)
            assert np.all(np.abs(n - 1.0) < 2e-6), float(np.max(np.abs(n - 1.0)))
            assert mc.mc_get_theta(h)[0] == (180 if T > 1 else 1)
        finally:
            mc.mc_destroy(h)
