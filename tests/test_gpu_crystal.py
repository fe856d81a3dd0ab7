"""bcc / fcc / hcp lattices (Sec. 2: 2 / 4 simple cubic or 4 simple
tetragonal sub-lattices, each split red/black, the sub-sets updated in
turn) on the GPU: FP64 bit-exact with the oracle's chain, FP32
statistically equal to FP64, and the calls that stay simple-cubic-only
refuse these lattices."""
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


KIND = {mc.MC_BCC: oracle.BCC, mc.MC_FCC: oracle.FCC, mc.MC_HCP: oracle.HCP}


@pytest.mark.parametrize("lattice,cells,J2", [(mc.MC_BCC, (4, 2, 6), 0.0), (mc.MC_BCC, (6, 4, 2), 0.3),
                                              (mc.MC_FCC, (2, 4, 2), 0.0), (mc.MC_FCC, (4, 4, 6), -0.2),
                                              (mc.MC_FCC, (8, 2, 2), 0.1), (mc.MC_HCP, (4, 2, 6), 0.0),
                                              (mc.MC_HCP, (2, 4, 2), 0.0)])
def test_crystal_fp64_bit_exact(lattice, cells, J2):
    nsub = 2 if lattice == mc.MC_BCC else 4
    N = nsub * cells[0] * cells[1] * cells[2]
    spins = workloads.random_spins(N, N + 3)
    kw = dict(Ku=0.2, Kc=0.1, H=(0.05, -0.1, 0.1), T=1.3, seed=N)
    o = oracle.Crystal(KIND[lattice], cells, J1=1.1, J2=J2, axis=(0.2, 0.1, 1.0), **kw)
    o.set_spins(spins)
    h = mc.mc_create_ex(mc.make_desc(cells, J=1.1, J2=J2, K_u=kw["Ku"], K_c=kw["Kc"], H=kw["H"], T=kw["T"],
                                     seed=kw["seed"], axis=(0.2, 0.1, 1.0), precision=mc.MC_FP64, lattice=lattice,
                                     ring_capacity=32))
    try:
        mc.mc_set_spins(h, spins)
        for n, meas in ((7, False), (13, True)):
            mc.mc_sweep(h, n, measure=meas)
            o.sweep(n, measure=meas)
            got = mc.mc_get_spins(h, N)
            assert np.array_equal(got, o.spins()), (lattice, cells, int((got != o.spins()).any(axis=1).sum()))
            assert mc.mc_get_theta(h)[0] == o.theta()
        ob, st = mc.mc_measure(h), o.stats()
        assert ob.n_samples == st["n"] == 13
        np.testing.assert_allclose(list(ob.m), [st["mx"], st["my"], st["mz"]], rtol=0, atol=1e-9)
        np.testing.assert_allclose([ob.ml, ob.e], [st["ml"], st["e"]], rtol=0, atol=1e-9)
        np.testing.assert_allclose(list(ob.e_parts), [st["e_ex"], st["e_u"], st["e_c"], st["e_z"]], rtol=0, atol=1e-9)
    finally:
        mc.mc_destroy(h)


@pytest.mark.parametrize("lattice", [mc.MC_BCC, mc.MC_FCC, mc.MC_HCP])
def test_crystal_fp32_matches_fp64(lattice):
    """Below T_C (bcc 2.05, fcc and hcp near 3.2 for J = 1): FP32 and FP64
    ensembles, six independent runs each, agree on <|m|> and <E> within the
    3-sigma-equivalent bound (t3) of the spread between runs."""
    from _stats import diff_within_t3
    cells, T, n, runs = (8, 8, 8), (1.4 if lattice == mc.MC_BCC else 2.2), 3000, 6
    means = {}
    for p in (mc.MC_FP32, mc.MC_FP64):
        ml, e = [], []
        for k in range(runs):
            h = mc.mc_create_ex(mc.make_desc(cells, K_u=0.02, T=T, seed=1 + 2 * k + p, precision=p, lattice=lattice,
                                             ring_capacity=16))
            try:
                mc.mc_sweep(h, 500)
                mc.mc_sweep(h, n, measure=True)
                o = mc.mc_measure(h)
                ml.append(o.ml)
                e.append(o.e)
            finally:
                mc.mc_destroy(h)
        means[p] = (np.array(ml), np.array(e))
    for k in range(2):
        d, se, bound = diff_within_t3(means[mc.MC_FP32][k], means[mc.MC_FP64][k])
        assert abs(d) <= max(bound, 1e-5), (lattice, k, d, se)
    assert means[mc.MC_FP32][0].mean() > 0.3  # ordered


def test_crystal_refused_where_simple_cubic_only():
    h = mc.mc_create_ex(mc.make_desc((4, 4, 4), lattice=mc.MC_FCC))
    try:
        with pytest.raises(mc.MCError):
            mc.mc_group_create([h])
        with pytest.raises(mc.MCError):
            mc.mc_profile_sample(h)
    finally:
        mc.mc_destroy(h)
    with pytest.raises(mc.MCError):
        mc.mc_create_ex(mc.make_desc((4, 4, 4), lattice=mc.MC_BCC, boundary=(1, 0, 0)))



# --------------------------------------- constrained sweeps (Table A2, Sec. 2)
@pytest.mark.parametrize("lattice,cells,J2", [(mc.MC_BCC, (4, 2, 6), 0.0), (mc.MC_FCC, (2, 4, 2), 0.15),
                                              (mc.MC_HCP, (4, 2, 2), 0.0), (mc.MC_FCC, (6, 4, 4), 0.0)])
def test_crystal_constrained_fp64_bit_exact(lattice, cells, J2):
    """Constrained sweeps of a crystal, FP64: spins, theta and the samples
    (torque included) equal the oracle's chain; 7 sweeps enqueued directly,
    then 20 (one captured graph of 16 and 4 more) with samples."""
    nsub = 2 if lattice == mc.MC_BCC else 4
    N = nsub * cells[0] * cells[1] * cells[2]
    th, ph = 35.0, 20.0
    R = oracle.constraint_frame(th, ph)
    kw = dict(Ku=0.2, Kc=0.1, H=(0.02, -0.03, 0.05), T=0.9, seed=N + 1)
    o = oracle.Crystal(KIND[lattice], cells, J1=1.1, J2=J2, axis=(0.2, 0.1, 1.0), **kw)
    spins = np.tile(R[0], (N, 1))
    o.set_spins(spins)
    h = mc.mc_create_ex(mc.make_desc(cells, J=1.1, J2=J2, K_u=kw["Ku"], K_c=kw["Kc"], H=kw["H"], T=kw["T"],
                                     seed=kw["seed"], axis=(0.2, 0.1, 1.0), precision=mc.MC_FP64, lattice=lattice,
                                     ring_capacity=32))
    try:
        mc.mc_set_spins(h, spins)
        for n, meas in ((7, False), (20, True)):
            mc.mc_constrained_sweep(h, th, ph, n, measure=meas)
            assert o.constrained_sweep(th, ph, n, measure=meas) == 0
            got = mc.mc_get_spins(h, N)
            assert np.array_equal(got, o.spins()), (lattice, cells, int((got != o.spins()).any(axis=1).sum()))
            assert mc.mc_get_theta(h)[0] == o.theta()
        ob, st = mc.mc_measure(h), o.stats()
        assert ob.n_samples == st["n"] == 20
        np.testing.assert_allclose(list(ob.m), [st["mx"], st["my"], st["mz"]], rtol=0, atol=1e-9)
        np.testing.assert_allclose(list(ob.torque), [st["tqx"], st["tqy"], st["tqz"]], rtol=0, atol=1e-9)
        np.testing.assert_allclose([ob.e], [st["e"]], rtol=0, atol=1e-9)
    finally:
        mc.mc_destroy(h)


def test_crystal_constrained_fp32_torque_matches_fp64():
    """fcc 6^3 cells at T = 0.6, theta_c = 45 deg: the FP32 torque tau_y
    (site order, FP32 moves) agrees with the FP64 chain's within the
    3-sigma-equivalent Student-t bound of the spread between 6 runs per
    precision (10 degrees of freedom, 3.96 standard errors); both near the T -> 0 law
    -(K_u sin 2 theta) softened by temperature."""
    th, Ku = 45.0, 0.05
    R = oracle.constraint_frame(th, 0.0)
    means = {}
    for prec in (mc.MC_FP32, mc.MC_FP64):
        vals = []
        for k in range(6):
            h = mc.mc_create_ex(mc.make_desc((6, 6, 6), K_u=Ku, T=0.6, seed=40 + k, precision=prec,
                                             lattice=mc.MC_FCC, init_dir=tuple(R[0]), ring_capacity=16))
            try:
                mc.mc_constrained_sweep(h, th, 0.0, 300)
                mc.mc_reset_stats(h)
                mc.mc_constrained_sweep(h, th, 0.0, 1500, measure=True)
                vals.append(mc.mc_measure(h).torque[1])
            finally:
                mc.mc_destroy(h)
        means[prec] = np.array(vals)
    from _stats import diff_within_t3
    a, b = means[mc.MC_FP32], means[mc.MC_FP64]
    d, se, bound = diff_within_t3(a, b)
    assert abs(d) <= bound + 1e-6, (a.mean(), b.mean(), se)
    assert -Ku < b.mean() < -0.5 * Ku, b.mean()
