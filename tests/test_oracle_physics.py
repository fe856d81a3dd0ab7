"""Statistical pins of the oracle's Markov chains (Eq. 1, Eq. 2, Tables A1/A2)
against closed forms, quadratures and invariants -- never against itself.

Every expected value here comes from mathematics: the Langevin function, the
two-spin Boltzmann integral, equipartition, harmonic spin waves, the Binder
cumulant crossing at the known Curie point, and the invariants of the
constrained pair move.  A dropped term, a wrong sign or a transposed operand
in the oracle moves one of these by many standard errors.
"""
import math
import os

import numpy as np
import pytest

import oracle
import workloads
from _stats import blocking_error, langevin


def _series(lat, word):
    return lat.samples()[:, word]


# --------------------------------------------------------------- closed forms
@pytest.mark.parametrize("H,T", [((0.0, 0.0, 1.5), 1.0), ((0.3, -0.4, 1.2), 0.7), ((0.0, 0.2, 0.0), 0.5)])
def test_langevin_law_independent_spins(H, T):
    """J = 0: every spin is an independent moment in a field; <S.h^> = L(|h|/T)."""
    lat = workloads.LatticeSpec(dims=(16, 16, 16), J=0.0, H=H, T=T)
    o = oracle.Lattice(lat.dims, J=0.0, H=H, T=T, seed=1, ring_cap=4000)
    o.sweep(300)
    o.sweep(3000, measure=True)
    s = o.samples()
    h = np.asarray(H) / np.linalg.norm(H)
    proj = s[:, 3:6] @ h
    expect = langevin(np.linalg.norm(H) / T)
    err = blocking_error(proj)
    assert abs(proj.mean() - expect) < max(5 * err, 2e-4), (proj.mean(), expect, err)


def test_two_spins_exchange_closed_form():
    """Two spins, one bond (2 x 1 x 1, open): <S1.S2> = coth(J/T) - T/J."""
    for T in (0.25, 1.0, 3.0):
        o = oracle.Lattice((2, 1, 1), J=1.0, T=T, bc=(1, 1, 1), seed=2, ring_cap=200000)
        o.sweep(1000)
        o.sweep(200000, measure=True)
        x = -2.0 * _series(o, 6)  # e_ex per spin = -J S1.S2 / 2
        err = blocking_error(x)
        assert abs(x.mean() - langevin(1.0 / T)) < max(5 * err, 1e-3), (T, x.mean(), langevin(1.0 / T), err)


def _two_spin_quadrature(J, K, H, T, n=96):
    """<S1.S2>, <S1z + S2z>/2 for E = -J S1.S2 - K(S1z^2+S2z^2) - H(S1z+S2z)
    by Gauss-Legendre quadrature over (cos t1, cos t2, dphi)."""
    xg, wg = np.polynomial.legendre.leggauss(n)
    pg = (xg + 1) * math.pi  # dphi in (0, 2 pi)
    wp = wg * math.pi
    c1, c2, ph = np.meshgrid(xg, xg, pg, indexing="ij")
    w = wg[:, None, None] * wg[None, :, None] * wp[None, None, :]
    s1, s2 = np.sqrt(1 - c1 ** 2), np.sqrt(1 - c2 ** 2)
    dot = c1 * c2 + s1 * s2 * np.cos(ph)
    E = -J * dot - K * (c1 ** 2 + c2 ** 2) - H * (c1 + c2)
    b = np.exp(-(E - E.min()) / T) * w
    Z = b.sum()
    return (b * dot).sum() / Z, (b * (c1 + c2) / 2).sum() / Z


def test_two_spins_with_anisotropy_and_field_quadrature():
    J, K, H, T = 1.0, 0.6, 0.3, 0.8
    o = oracle.Lattice((2, 1, 1), J=J, Ku=K, H=(0, 0, H), T=T, bc=(1, 1, 1), seed=5, ring_cap=300000)
    o.sweep(1000)
    o.sweep(300000, measure=True)
    s = o.samples()
    dot = -2.0 * s[:, 6] / J
    mz = s[:, 5]
    e_dot, e_mz = _two_spin_quadrature(J, K, H, T)
    assert abs(dot.mean() - e_dot) < max(5 * blocking_error(dot), 1e-3)
    assert abs(mz.mean() - e_mz) < max(5 * blocking_error(mz), 1e-3)


def test_single_spin_uniaxial_quadrature():
    """One spin, uniaxial only: <Sz^2> = int t^2 e^{Kt^2/T} / int e^{Kt^2/T} over [0,1]."""
    K, T = 1.0, 0.4
    o = oracle.Lattice((1, 1, 1), Ku=K, T=T, bc=(1, 1, 1), seed=9, ring_cap=400000)
    o.sweep(1000)
    o.sweep(400000, measure=True)
    sz2 = -_series(o, 7) / K
    t, w = np.polynomial.legendre.leggauss(200)
    t = 0.5 * (t + 1)
    w = 0.5 * w
    b = np.exp(K * t ** 2 / T) * w
    expect = (b * t ** 2).sum() / b.sum()
    assert abs(sz2.mean() - expect) < max(5 * blocking_error(sz2), 1e-3)


def test_two_spin_distribution_detailed_balance():
    """With the cone angle frozen the chain is a reversible Metropolis chain:
    x = S1.S2 has density beta J e^{beta J x} / (2 sinh beta J) on [-1, 1]."""
    T = 0.5
    o = oracle.Lattice((2, 1, 1), J=1.0, T=T, bc=(1, 1, 1), seed=21, adapt_in_measure=0, ring_cap=400000)
    o.sweep(2000)
    o.sweep(400000, measure=True)
    x = -2.0 * _series(o, 6)[::20]  # thin to reduce correlation
    b = 1.0 / T
    edges = np.linspace(-1, 1, 17)
    cdf = lambda v: (np.exp(b * v) - np.exp(-b)) / (np.exp(b) - np.exp(-b))
    p = np.diff(cdf(edges))
    h, _ = np.histogram(x, bins=edges)
    n = x.size
    sig = np.sqrt(n * p * (1 - p)) * 2.0  # generous factor for residual correlation
    assert np.all(np.abs(h - n * p) < 5 * sig + 5), (h, n * p)


# --------------------------------------------------------------- low T limits
def test_low_temperature_energy_equipartition():
    """T -> 0: E/N = -3J - K_u + T (two quadratic transverse modes per spin)."""
    for T in (0.01, 0.02):
        o = oracle.Lattice((8, 8, 8), J=1.0, Ku=0.01, T=T, seed=4, ring_cap=3000)
        o.sweep(1000)
        o.sweep(3000, measure=True)
        s = o.stats()
        e = s["e"] / s["n"]
        assert abs(e - (-3.0 - 0.01 + T)) < 0.03 * T, (T, e)


def test_spin_wave_magnetization():
    """K = 0, harmonic spin waves on the periodic 16^3 lattice:
    1 - <|m|> = (T / 2J) (1/N) sum_{k != 0} 1 / (3 - cos kx - cos ky - cos kz),
    up to the O(T) anharmonic correction."""
    L = 16
    k = 2 * np.pi * np.arange(L) / L
    kx, ky, kz = np.meshgrid(k, k, k, indexing="ij")
    eps = (3 - np.cos(kx) - np.cos(ky) - np.cos(kz)).ravel()[1:]
    W = (1 / eps).sum() / L ** 3
    for T, tol in ((0.02, 0.015), (0.05, 0.03)):
        o = oracle.Lattice((L, L, L), J=1.0, T=T, seed=3, ring_cap=3000)
        o.sweep(1000)
        o.sweep(3000, measure=True)
        s = o.stats()
        ratio = (1 - s["ml"] / s["n"]) / (T / 2 * W)
        assert abs(ratio - 1) < tol, (T, ratio)


# ---------------------------------------------------------------- critical point
@pytest.mark.slow
def test_binder_cumulant_brackets_curie_point():
    """U_L = 1 - <m^4>/(3<m^2>^2) grows with L below T_C and shrinks above it;
    the classical sc Heisenberg T_C = 1.443 J/k_B (2 theta_C = 1.446, Sec. 3)."""
    def U(L, T, seed):
        o = oracle.Lattice((L, L, L), J=1.0, T=T, seed=seed, ring_cap=1)
        o.set_spins(workloads.random_spins(L ** 3, seed))
        o.sweep(2000)
        o.sweep(16000, measure=True)
        s = o.stats()
        return 1 - (s["ml4"] / s["n"]) / (3 * (s["ml2"] / s["n"]) ** 2)

    below = (U(10, 1.33, 1), U(6, 1.33, 2))
    above = (U(10, 1.56, 3), U(6, 1.56, 4))
    assert below[0] > below[1], below
    assert above[0] < above[1], above


@pytest.mark.slow
def test_binder_cumulant_crossing_locates_the_curie_point():
    """U_L(T) = 1 - <m^4>/(3 <m^2>^2) at T = 1.42, 1.445 and 1.47 for L = 8, 12
    and 16; the crossing of L = 8 and 16, and of L = 12 and 16 (the root of
    a quadratic through the three differences U_16 - U_L) lies within 0.02
    of the classical simple-cubic Heisenberg T_C = 1.443 J/k_B (the paper's
    theta_C = 0.723 gives 2 theta_C = 1.446, Sec. 3).  The moments pool
    independent chains (8 per L and T for L = 12 and 16, 4 for L = 8) run in
    parallel processes.  A straight line through two temperatures would put
    the crossings about 0.01 low: U_L curves over this range."""
    import multiprocessing as mp

    import _binder

    temps = (1.42, 1.445, 1.47)
    jobs = [(L, T, 1000 * L + 10 * k + i, 1000, 16000)
            for L, k_n in ((8, 4), (12, 8), (16, 8)) for i, T in enumerate(temps) for k in range(k_n)]
    jobs.sort(key=lambda j: -j[0])
    with mp.get_context("spawn").Pool(min(len(jobs), os.cpu_count() or 1)) as pool:
        res = pool.map(_binder.binder_sums, jobs, chunksize=1)
    acc = {}
    for L, T, m2, m4, n in res:
        a = acc.setdefault((L, T), [0.0, 0.0, 0.0])
        a[0] += m2
        a[1] += m4
        a[2] += n
    U = {k: 1 - (v[1] / v[2]) / (3 * (v[0] / v[2]) ** 2) for k, v in acc.items()}
    for La in (8, 12):
        d = np.array([U[(16, T)] - U[(La, T)] for T in temps])
        assert d[0] > 0 > d[2], (La, d)  # the larger lattice orders more below T_C, less above
        roots = [r.real for r in np.roots(np.polyfit(temps, d, 2)) if abs(r.imag) < 1e-12 and temps[0] <= r.real <= temps[2]]
        assert len(roots) == 1, (La, d, roots)
        assert abs(roots[0] - 1.443) < 0.02, (La, roots[0], U)


# ------------------------------------------------- parallel vs serial (Sec. 2)
def test_checkerboard_matches_serial_random_order():
    """The paper checks the parallel chain against the serial random-order
    chain (Sec. 2): same ensemble averages within the sampling error."""
    res = []
    for serial in (False, True):
        o = oracle.Lattice((8, 8, 8), J=1.0, Ku=0.01, T=1.0, seed=7, ring_cap=20000)
        run = o.sweep_serial if serial else o.sweep
        run(3000)
        run(20000, measure=True)
        s = o.samples()
        ml = np.linalg.norm(s[:, 3:6], axis=1)
        e = s[:, 6:10].sum(axis=1)
        res.append(((ml.mean(), blocking_error(ml)), (e.mean(), blocking_error(e))))
    for k in range(2):
        (a, ea), (b, eb) = res[0][k], res[1][k]
        assert abs(a - b) < 3 * math.hypot(ea, eb), (k, a, b, ea, eb)


def test_ordered_and_random_starts_agree():
    for T in (1.0, 1.6):
        vals = []
        for start in ("ordered", "random"):
            o = oracle.Lattice((8, 8, 8), J=1.0, T=T, seed=11, ring_cap=10000)
            if start == "random":
                o.set_spins(workloads.random_spins(512, 99))
            o.sweep(3000)
            o.sweep(10000, measure=True)
            ml = np.linalg.norm(o.samples()[:, 3:6], axis=1)
            vals.append((ml.mean(), blocking_error(ml)))
        assert abs(vals[0][0] - vals[1][0]) < 3 * math.hypot(vals[0][1], vals[1][1]), (T, vals)


def test_cone_angle_adaptation_targets_half():
    o = oracle.Lattice((8, 8, 8), J=1.0, Ku=0.01, T=0.8, seed=1, ring_cap=2000)
    o.sweep(500)
    o.sweep(2000, measure=True)
    s = o.samples()
    th = s[:, 1]
    assert np.all(np.abs(np.diff(th)) == 1)  # one degree per iteration
    assert 1 < th.min() and th.max() < 180
    acc = s[:, 2] / o.n_mov
    assert abs(acc.mean() - 0.5) < 0.02


def test_pinned_planes_never_move():
    dims = (12, 4, 4)
    o = oracle.Lattice(dims, J=1.0, Ku=0.05, T=0.8, bc=(2, 0, 0), seed=3)
    S0 = workloads.wall_spins(dims)
    o.set_spins(S0)
    assert o.n_mov == 12 * 16 - 2 * 16
    o.sweep(200)
    S = o.spins().reshape(4, 4, 12, 3)
    S0 = S0.reshape(4, 4, 12, 3)
    assert np.array_equal(S[:, :, 0], S0[:, :, 0]) and np.array_equal(S[:, :, -1], S0[:, :, -1])
    assert not np.array_equal(S[:, :, 1:-1], S0[:, :, 1:-1])


# ------------------------------------------------- constrained MC (Table A2)
def test_constrained_pair_move_conserves_transverse_magnetization():
    th, ph = 30.0, 20.0
    R = oracle.constraint_frame(th, ph)
    N = 8 ** 3
    o = oracle.Lattice((8, 8, 8), J=1.0, Ku=0.05, Kc=0.02, T=0.6, seed=5)
    o.set_spins(workloads.uniform_spins(N, R[0]))
    for _ in range(20):
        o.constrained_sweep(th, ph, 10)
        M = o.spins().sum(axis=0)
        assert abs(M @ R[1]) < 1e-9 * N and abs(M @ R[2]) < 1e-9 * N
        assert M @ R[0] > 0
    assert np.allclose(np.linalg.norm(o.spins(), axis=1), 1.0, atol=1e-10)


def test_constrained_low_temperature_torque():
    """T -> 0 along e_C(theta, phi = 0): tau_theta / N = -(K_u sin 2 theta +
    (K_c / 2) sin 4 theta), from F = -K_u cos^2 theta + K_c sin^2 2theta / 4,
    reduced by O(T) thermal softening."""
    Ku, Kc, T = 0.05, 0.02, 0.01
    for th in (30.0, 60.0):
        R = oracle.constraint_frame(th, 0.0)
        o = oracle.Lattice((8, 8, 8), J=1.0, Ku=Ku, Kc=Kc, T=T, seed=8, ring_cap=3000)
        o.set_spins(workloads.uniform_spins(512, R[0]))
        o.constrained_sweep(th, 0.0, 500)
        o.constrained_sweep(th, 0.0, 2000, measure=True)
        s = o.stats()
        n_hat = np.array([0.0, 1.0, 0.0])
        tau = np.array([s["tqx"], s["tqy"], s["tqz"]]) / s["n"] @ n_hat
        t = math.radians(th)
        expect = -(Ku * math.sin(2 * t) + 0.5 * Kc * math.sin(4 * t))
        assert abs(tau / expect - 1) < 0.03, (th, tau, expect)


def test_constrained_low_temperature_torque_at_45_degrees_azimuth():
    """T -> 0 along e_C(theta, phi = 45): with e_C = (s/sqrt2, s/sqrt2, c),
    s = sin theta, c = cos theta, the cubic energy per spin is
    K_c (s^4/4 + s^2 c^2), so F = -K_u c^2 + K_c (s^4/4 + s^2 c^2) and
    tau_theta / N = -dF/dtheta = -(K_u sin 2 theta + K_c s c (2 c^2 - s^2)),
    tau_theta = n.tau with n = (-sin phi, cos phi, 0).  At theta = 60 this
    differs from the phi = 0 law by 19%, so a frame that ignored phi fails."""
    Ku, Kc, T, ph = 0.05, 0.02, 0.01, 45.0
    for th in (30.0, 60.0):
        R = oracle.constraint_frame(th, ph)
        o = oracle.Lattice((8, 8, 8), J=1.0, Ku=Ku, Kc=Kc, T=T, seed=18, ring_cap=3000)
        o.set_spins(workloads.uniform_spins(512, R[0]))
        o.constrained_sweep(th, ph, 500)
        o.constrained_sweep(th, ph, 2000, measure=True)
        s = o.stats()
        p = math.radians(ph)
        n_hat = np.array([-math.sin(p), math.cos(p), 0.0])
        tau = np.array([s["tqx"], s["tqy"], s["tqz"]]) / s["n"] @ n_hat
        t = math.radians(th)
        st, ct = math.sin(t), math.cos(t)
        expect = -(Ku * math.sin(2 * t) + Kc * st * ct * (2 * ct * ct - st * st))
        assert abs(tau / expect - 1) < 0.03, (th, tau, expect)
        at_phi0 = -(Ku * math.sin(2 * t) + 0.5 * Kc * math.sin(4 * t))
        if th == 60.0:
            assert abs(tau / at_phi0 - 1) > 0.1


def test_constrained_zero_angle_torque_vanishes():
    o = oracle.Lattice((8, 8, 8), J=1.0, Ku=0.05, T=0.6, seed=9, ring_cap=4000)
    o.constrained_sweep(0.0, 0.0, 500)
    o.constrained_sweep(0.0, 0.0, 4000, measure=True)
    s = o.samples()
    for a in (10, 11):
        assert abs(s[:, a].mean()) < 5 * blocking_error(s[:, a]) + 1e-5


def test_parallel_constrained_matches_serial_asselin():
    """Sec. 2: the parallel form (M_L frozen per iteration, same-colour pairs)
    gives the same torque as the serial algorithm of Asselin et al."""
    th, ph, T = 45.0, 0.0, 0.7
    R = oracle.constraint_frame(th, ph)
    res = []
    for serial in (False, True):
        o = oracle.Lattice((8, 8, 8), J=1.0, Ku=0.05, Kc=0.02, T=T, seed=13, ring_cap=12000)
        o.set_spins(workloads.uniform_spins(512, R[0]))
        run = o.constrained_sweep_serial if serial else o.constrained_sweep
        run(th, ph, 2000)
        run(th, ph, 12000, measure=True)
        tau = o.samples()[:, 10:13] @ np.array([0.0, 1.0, 0.0])
        res.append((tau.mean(), blocking_error(tau)))
    (a, ea), (b, eb) = res
    assert abs(a - b) < 3 * math.hypot(ea, eb), res


# ------------------------------------------------------ Eq. 4 anisotropy scaling
def _sphere_average(f, weight, n_t=200, n_phi=400):
    """<f> under the weight over the unit sphere: Gauss-Legendre in cos(theta),
    periodic trapezoid in phi."""
    t, w = np.polynomial.legendre.leggauss(n_t)
    phi = np.linspace(0.0, 2 * np.pi, n_phi, endpoint=False)
    T, P = np.meshgrid(t, phi, indexing="ij")
    r = np.sqrt(1 - T ** 2)
    x, y, z = r * np.cos(P), r * np.sin(P), T
    b = weight(x, y, z) * w[:, None]
    return float((b * f(x, y, z)).sum() / b.sum())


def test_eq4_uniaxial_single_spin_is_p2():
    """One spin, uniaxial only: Eq. 4 with K_easy = <E_u> + K_u and K_0,hard =
    K_u gives k_u = (3 <cos^2> - 1) / 2, the Boltzmann average of P_2 by
    quadrature."""
    K, T = 1.0, 0.4
    o = oracle.Lattice((1, 1, 1), Ku=K, T=T, bc=(1, 1, 1), seed=19, ring_cap=300000)
    o.sweep(1000)
    o.sweep(300000, measure=True)
    k_u, k_c = o.anisotropy_scaling()
    assert math.isnan(k_c)
    per_sweep = 1 - 3 * (_series(o, 7) + K) / (2 * K)
    expect = _sphere_average(lambda x, y, z: 1.5 * z ** 2 - 0.5, lambda x, y, z: np.exp(K * z ** 2 / T))
    assert abs(k_u - expect) < max(5 * blocking_error(per_sweep), 1e-3), (k_u, expect)


def test_eq4_cubic_single_spin_quadrature():
    """One spin, cubic only (K_c > 0, easy <100>): k_c = 1 - 5 <q> with q =
    x^2 y^2 + x^2 z^2 + y^2 z^2 averaged by quadrature over the sphere."""
    K, T = 1.0, 0.15
    o = oracle.Lattice((1, 1, 1), Kc=K, T=T, bc=(1, 1, 1), seed=23, ring_cap=300000)
    o.sweep(1000)
    o.sweep(300000, measure=True)
    k_u, k_c = o.anisotropy_scaling()
    assert math.isnan(k_u)
    q = lambda x, y, z: x * x * y * y + x * x * z * z + y * y * z * z  # noqa: E731
    expect = 1 - 5 * _sphere_average(q, lambda x, y, z: np.exp(-K * q(x, y, z) / T))
    per_sweep = 1 - 5 * _series(o, 8) / K
    assert 0.2 < expect < 0.9
    assert abs(k_c - expect) < max(5 * blocking_error(per_sweep), 1e-3), (k_c, expect)


def test_eq4_limits():
    """Eq. 4 is 1 at T -> 0 (every spin on the easy axis) and 0 in the
    paramagnetic limit (<cos^2> = 1/3, <q> = 1/5 for spins uniform on the
    sphere), for both constants at once."""
    # at T = 1e-4 the thermal softening (k_c ~ 1 - 5 <delta^2>, <delta^2> ~ T)
    # is about 2e-4
    cold = oracle.Lattice((8, 8, 8), J=1.0, Ku=0.05, Kc=0.02, T=1e-4, seed=3, ring_cap=1)
    cold.sweep(50)
    cold.sweep(200, measure=True)
    k_u, k_c = cold.anisotropy_scaling()
    assert abs(k_u - 1) < 1e-3 and abs(k_c - 1) < 1e-3, (k_u, k_c)
    hot = oracle.Lattice((8, 8, 8), J=0.0, Ku=1.0, Kc=1.0, T=1e3, seed=4, ring_cap=4000)
    hot.sweep(200)
    hot.sweep(4000, measure=True)
    k_u, k_c = hot.anisotropy_scaling()
    s = hot.samples()
    err_u = blocking_error(1 - 3 * (s[:, 7] + 1.0) / 2)
    err_c = blocking_error(1 - 5 * s[:, 8])
    assert abs(k_u) < 5 * err_u + 2e-3 and abs(k_c) < 5 * err_c + 2e-3, (k_u, k_c, err_u, err_c)


# ------------------------------------------------ anti-periodic wall (Sec. 3)
def _discrete_wall(Lx, J, K):
    """Minimum of the 1-D chain energy -J sum cos(phi_{x+1} - phi_x) - K sum
    cos^2 phi_x with the anti-periodic closure phi_Lx = phi_0 + pi (one
    Bloch wall), by L-BFGS from a tanh start.  Returns (phi, E_min)."""
    from scipy.optimize import minimize

    def energy(phi):
        nxt = np.append(phi[1:], phi[0] + np.pi)
        d = nxt - phi
        e = -J * np.cos(d).sum() - K * (np.cos(phi) ** 2).sum()
        g = -J * np.sin(d) + J * np.roll(np.sin(d), 1) + K * np.sin(2 * phi)
        return e, g

    x = np.arange(Lx)
    width = np.pi * math.sqrt(J / (2 * K))
    phi0 = 2 * np.arctan(np.exp(np.pi * (x - Lx / 2) / width))  # 0 -> pi across the wall
    r = minimize(energy, phi0, jac=True, method="L-BFGS-B", options={"gtol": 1e-12, "maxiter": 10000})
    return r.x, r.fun


def test_antiperiodic_wall_energy_at_low_temperature():
    """x anti-periodic holds one Bloch wall.  Started on the discrete
    minimum of the wall, the chain at T = 1e-3 keeps the minimum energy plus
    equipartition (two transverse modes per spin: E = E_min + N T); the
    discrete wall energy is the continuum 4 sqrt(A K) = 2 sqrt(2 J K) to
    within the lattice correction."""
    Lx, Ly, Lz, J, K, T = 64, 2, 2, 1.0, 0.05, 1e-3
    phi, e_chain = _discrete_wall(Lx, J, K)
    wall = e_chain + (J + K) * Lx
    assert abs(wall / (2 * math.sqrt(2 * J * K)) - 1) < 0.01
    N = Lx * Ly * Lz
    S = np.zeros((N, 3))
    xs = np.arange(N) % Lx
    S[:, 0], S[:, 2] = np.sin(phi[xs]), np.cos(phi[xs])
    o = oracle.Lattice((Lx, Ly, Lz), J=J, Ku=K, T=T, bc=(3, 0, 0), seed=6, ring_cap=1)
    o.set_spins(S)
    o.sweep(200)
    o.sweep(400, measure=True)
    s = o.stats()
    e_total = s["e"] / s["n"] * N
    ground = Ly * Lz * e_chain - 2 * J * N  # y and z bonds aligned
    assert abs(e_total - (ground + N * T)) < 0.02 * Ly * Lz * wall, (e_total, ground + N * T)
    mz = o.spins()[:, 2].reshape(Lz, Ly, Lx).mean(axis=(0, 1))
    assert mz.max() > 0.9 and mz.min() < -0.9  # the wall is still there
