"""Host analysis of Sec. 3 (paper_2103_03517_gb300.analysis) against closed
forms and the discrete minimum-energy Bloch wall."""
import math

import numpy as np
import pytest

from paper_2103_03517_gb300 import analysis as an
from test_oracle_physics import _discrete_wall


@pytest.mark.parametrize("x0", [64.3, 2.2, 127.6, 0.0])
@pytest.mark.parametrize("m", [0.8, -0.55])
def test_fit_wall_recovers_antiperiodic_tanh(x0, m):
    """An exact anti-periodic tanh profile, the wall anywhere (at the
    boundary too) and either orientation: m, x0 and the width come back."""
    Lx, delta = 128, 15.3
    mz = an.wall_model(np.arange(Lx), m, x0, delta, Lx)
    mf, cf, df, _ = an.fit_wall(mz)
    assert abs(df - delta) < 1e-6
    # x0 comes back in [0, Lx) with the sign of m that goes with it
    assert abs(mf - m) < 1e-6 and abs((cf - x0 + Lx / 2) % Lx - Lx / 2) < 1e-5, (mf, cf, df)


@pytest.mark.parametrize("K", [0.01, 0.04])
def test_zero_temperature_wall_gives_stiffness_half_J(K):
    """The discrete minimum-energy wall of the anti-periodic chain (J = 1):
    its m_z = cos(phi) fitted by the tanh of Sec. 3 gives Delta close to
    pi sqrt(J / 2K), and Eq. 5 then gives A = J/2 (the continuum stiffness
    of the simple cubic lattice, a = 1) to the discreteness error."""
    J, Lx = 1.0, 256
    phi, _ = _discrete_wall(Lx, J, K)
    m, x0, delta, _ = an.fit_wall(np.cos(phi))
    assert abs(delta / (math.pi * math.sqrt(J / (2 * K))) - 1) < 0.02
    assert abs(an.exchange_stiffness(delta, K) / (J / 2) - 1) < 0.04
    assert abs(abs(m) - 1) < 1e-3


def test_free_energy_difference_closed_forms():
    """beta dF = int_0^beta dU with dU(0) = 0: dU = c beta (trapezoid-exact)
    gives dF = c beta / 2, the temperatures in any order; dU = E0 (1 -
    exp(-beta)) gives dF = E0 (1 - (1 - exp(-beta)) / beta) on a fine grid."""
    T = np.array([0.5, 2.0, 1.0, 0.25])
    c = 1.7
    assert np.allclose(an.free_energy_difference(T, c / T), c / (2 * T), rtol=0, atol=1e-12)
    beta = np.linspace(0.0, 5.0, 20001)[1:]
    E0 = 2.3
    dF = an.free_energy_difference(1.0 / beta, E0 * (1 - np.exp(-beta)))
    assert np.allclose(dF, E0 * (1 - (1 - np.exp(-beta)) / beta), rtol=0, atol=1e-7)  # O(h^2) trapezoid


def test_free_energy_route_at_zero_temperature_gives_half_J():
    """At T -> 0 the wall's free energy is its energy; for the discrete wall
    per unit cross-section that is close to 2 sqrt(2 J K), and Eq. 5 turns it
    into A = J/2."""
    J, K, Lx = 1.0, 0.02, 256
    _, e_min = _discrete_wall(Lx, J, K)
    e_wall = e_min + (J + K) * Lx
    beta = np.linspace(0.0, 400.0, 4001)[1:]
    dF = an.free_energy_difference(1.0 / beta, np.full(beta.size, e_wall))
    assert abs(an.stiffness_from_free_energy(dF[-1], 1.0, K) / (J / 2) - 1) < 0.02


def test_power_exponent_and_bloch_law():
    m = np.linspace(0.3, 0.98, 30)
    k, err, c = an.power_exponent(m, 2.5 * m ** 1.48, m_min=0.6)
    assert abs(k - 1.48) < 1e-10 and abs(c - 2.5) < 1e-10 and err < 1e-8
    T = np.linspace(0.05, 1.35, 40)
    Tc, beta, _ = an.bloch_fit(T, (1 - T / 1.443) ** 0.34)
    assert abs(Tc - 1.443) < 1e-6 and abs(beta - 0.34) < 1e-6


def test_transverse_susceptibility_low_temperature_single_spin():
    """Eq. 7 at T -> 0 for one spin with uniaxial K (m = 1, K_u(T) = K): the
    variance of S_x over the Boltzmann weight exp(K cos^2 theta / T), by
    quadrature over the sphere, divided by T equals 1 / (2K) to O(T/K)."""
    K, T = 1.0, 1e-3
    th = np.linspace(0.0, math.pi, 400001)
    w = np.exp(K * (np.cos(th) ** 2 - 1) / T) * np.sin(th)
    sx2 = np.trapezoid(0.5 * np.sin(th) ** 2 * w, th) / np.trapezoid(w, th)  # <cos^2 phi> = 1/2
    assert abs((sx2 / T) / an.chi_perp_uniaxial(1.0, K) - 1) < 5e-3


def test_multi_bloch_fit_recovers_one_and_two_terms():
    """Eq. 8 with the T_C grid holding the true values: one Bloch law comes
    back as one term (T_C, beta exact), two as their weights."""
    T = np.linspace(0.05, 1.25, 40)
    grid = (0.1, 1.6)  # 15 terms: 0.2, 0.3, ..., 1.6
    f = an.multi_bloch_fit(T, (1 - T / 1.3) ** 0.35, 15, tc_range=grid)
    assert abs(f["T_C_mean"] - 1.3) < 1e-6 and abs(f["beta"] - 0.35) < 1e-9 and f["rms"] < 1e-6
    m = 0.6 * np.clip(1 - T / 1.0, 0, None) ** 0.35 + 0.4 * np.clip(1 - T / 1.4, 0, None) ** 0.35
    f = an.multi_bloch_fit(T, m, 15, tc_range=grid)
    assert abs(f["T_C_mean"] - 1.16) < 1e-6 and abs(f["w"].sum() - 1) < 1e-6


def test_multi_bloch_fit_converges_with_terms():
    """T_C spread uniformly over [0.9, 1.3] (m(T) by quadrature over the
    spread): the average of Eq. 8 approaches 1.1 as the number of terms
    grows, and settles (20 vs 40 terms)."""
    T = np.linspace(0.05, 1.35, 60)
    tcs = np.linspace(0.9, 1.3, 4001)
    m = np.mean(np.clip(1 - T[:, None] / tcs[None, :], 0, None) ** 0.35, axis=1)
    f20 = an.multi_bloch_fit(T, m, 20, tc_range=(0.5, 1.5))
    f40 = an.multi_bloch_fit(T, m, 40, tc_range=(0.5, 1.5))
    assert abs(f40["T_C_mean"] - 1.1) < 0.01 and abs(f20["T_C_mean"] - f40["T_C_mean"]) < 0.01


# ------------------------------------------------------- blocking error bars
def _ar1(rho, n, rng):
    """Stationary AR(1) series y_i = rho y_(i-1) + e_i with unit innovations."""
    from scipy.signal import lfilter
    e = rng.standard_normal(n)
    e[0] /= math.sqrt(1.0 - rho * rho)
    return lfilter([1.0], [1.0, -rho], e)


def test_blocking_error_independent_samples():
    """Independent samples: level 0 is std / sqrt(n) and the deeper levels
    scatter about it, so the largest is at least that and, averaged over
    replicas, within about 10% of it."""
    rng = np.random.default_rng(11)
    ratios = []
    for _ in range(32):
        x = rng.standard_normal(2 ** 14)
        exact = x.std(ddof=1) / math.sqrt(x.size)
        r = an.blocking_error(x) / exact
        assert r >= 1.0 - 1e-12
        ratios.append(r)
    assert 1.0 <= np.mean(ratios) < 1.15


def test_blocking_error_ar1_closed_form():
    """AR(1): the standard error of the mean of n samples is
    sqrt(var_y (1 + rho) / ((1 - rho) n)) with var_y = 1 / (1 - rho^2), and
    the naive error is sqrt((1 - rho) / (1 + rho)) times that.  Averaged over
    replicas the blocking estimate matches the closed form; each replica is
    far above the naive error."""
    rng = np.random.default_rng(12)
    for rho, n in ((0.9, 2 ** 15), (0.5, 5000)):
        exact = math.sqrt((1.0 / (1.0 - rho * rho)) * (1.0 + rho) / ((1.0 - rho) * n))
        naive = exact * math.sqrt((1.0 - rho) / (1.0 + rho))
        ratios = []
        for _ in range(32):
            got = an.blocking_error(_ar1(rho, n, rng))
            assert got > 0.5 * (exact + naive)
            ratios.append(got / exact)
        assert 0.9 < np.mean(ratios) < 1.15, (rho, np.mean(ratios))


def test_blocking_error_exact_cases():
    assert an.blocking_error(np.full(1024, 0.7)) == pytest.approx(0.0, abs=1e-15)
    assert an.blocking_error(np.arange(10.0)) == 0.0  # fewer than 32 samples: no level
    # perfectly alternating series: pair averages vanish, so level 0 is the largest
    x = np.tile([1.0, -1.0], 512)
    assert an.blocking_error(x) == pytest.approx(math.sqrt(np.var(x, ddof=1) / x.size), rel=1e-12)


def test_sample_errors_of_a_sample_series():
    n = 4096
    rng = np.random.default_rng(13)
    s = np.zeros(n, dtype=[("m", "f8", 3), ("e_parts", "f8", 4), ("torque", "f8", 3)])
    s["m"] = [0.0, 0.6, -0.8] + 0.01 * rng.standard_normal((n, 3))
    s["e_parts"] = [-2.0, -0.01, 0.0, 0.0]
    s["torque"] = 0.0
    out = an.sample_errors(s)
    assert set(out) == {"ml", "mx", "my", "mz", "mz_abs", "e", "tx", "ty", "tz"}
    assert out["ml"][0] == pytest.approx(1.0, abs=1e-3)
    assert out["mz"][0] == pytest.approx(-0.8, abs=1e-3) and out["mz_abs"][0] == pytest.approx(0.8, abs=1e-3)
    assert out["e"][0] == pytest.approx(-2.01) and out["e"][1] == pytest.approx(0.0, abs=1e-15)
    assert 0.01 / math.sqrt(n) * 0.9 < out["mx"][1] < 0.01 / math.sqrt(n) * 1.3


def test_magnetization_curve_rejects_bad_arguments_on_the_host():
    from paper_2103_03517_gb300 import studies as st
    with pytest.raises(ValueError):
        st.magnetization_curve((16, 16, 16), [])
    with pytest.raises(ValueError):
        st.magnetization_curve([(16, 16, 16), (32, 32, 32)], [0.5])
    with pytest.raises(ValueError):
        st.magnetization_curve((16, 16, 16), [0.5], n_meas=0)


def test_torque_basis_is_the_theta_derivative_of_the_anisotropy_energy():
    """g_u and g_c against a central difference of the energy per spin
    written from the direction cosines themselves: -(e_C . z)^2 and
    a1^2 a2^2 + a1^2 a3^2 + a2^2 a3^2 (Eq. 2's anisotropy terms)."""
    def energies(t, p):
        a = np.array([np.sin(t) * np.cos(p), np.sin(t) * np.sin(p), np.cos(t)])
        return -(a[2] ** 2), a[0] ** 2 * a[1] ** 2 + a[0] ** 2 * a[2] ** 2 + a[1] ** 2 * a[2] ** 2
    h = 1e-6
    for th in (0.0, 7.0, 30.0, 45.0, 61.0, 90.0, 133.0):
        for ph in (0.0, 17.0, 45.0, 90.0):
            t, p = math.radians(th), math.radians(ph)
            up, cp = energies(t + h, p)
            um, cm = energies(t - h, p)
            g_u, g_c = an.torque_basis(th, ph)
            assert abs(g_u - (up - um) / (2 * h)) < 1e-8 and abs(g_c - (cp - cm) / (2 * h)) < 1e-8, (th, ph)


def test_torque_fit_recovers_the_constants_exactly():
    """The closed-form torque of config 3's grid (theta 0..90 by 10, phi 0
    and 45 deg) gives back K_u and K_c; with phi = 0 alone the cubic term
    sin(4 theta)/2 still separates from sin(2 theta)."""
    th = np.array(list(range(0, 91, 10)) * 2, float)
    ph = np.array([0.0] * 10 + [45.0] * 10)
    for Ku, Kc in ((0.05, 0.02), (0.031, -0.007), (0.0, 0.013)):
        g_u, g_c = an.torque_basis(th, ph)
        tau = -(Ku * g_u + Kc * g_c)
        f = an.torque_fit(th, ph, tau)
        assert abs(f["K_u"] - Ku) < 1e-14 and abs(f["K_c"] - Kc) < 1e-14
        f0 = an.torque_fit(th[:10], ph[:10], tau[:10], sigma=np.full(10, 1e-3))
        assert abs(f0["K_u"] - Ku) < 1e-14 and abs(f0["K_c"] - Kc) < 1e-14 and f0["chi2_dof"] < 1e-20
    with pytest.raises(ValueError):  # theta = 0 and 90 only: both factors vanish
        an.torque_fit([0.0, 90.0], [0.0, 0.0], [0.0, 0.0])


def test_torque_theta_projects_on_increasing_theta():
    tq = np.array([[0.3, -0.2, 0.7], [1.0, 2.0, 3.0]])
    np.testing.assert_allclose(an.torque_theta(tq, [0.0, 90.0]), [-0.2, -1.0])


def test_torque_fit_on_the_oracle_chain_at_low_temperature():
    """Table A2 on the serial oracle (8^3, K_u = 0.05, K_c = 0.02, T = 0.02)
    at five constraint directions, fitted by torque_fit: K_u(T) and K_c(T)
    come back just below their T = 0 values: spin waves lower them as
    K_u ~ m^3 and K_c ~ m^10 (Callen-Callen, Sec. 3) with m ~ 1 - 0.25 T,
    about 1.5% and 5% here, and never raise them."""
    import oracle
    import workloads

    Ku, Kc, T = 0.05, 0.02, 0.02
    th = np.array([20.0, 45.0, 70.0, 30.0, 60.0])
    ph = np.array([0.0, 0.0, 0.0, 45.0, 45.0])
    tau = []
    for t, p in zip(th, ph):
        R = oracle.constraint_frame(t, p)
        o = oracle.Lattice((8, 8, 8), J=1.0, Ku=Ku, Kc=Kc, T=T, seed=int(t + p), ring_cap=1)
        o.set_spins(workloads.uniform_spins(512, R[0]))
        o.constrained_sweep(t, p, 200)
        o.constrained_sweep(t, p, 600, measure=True)
        s = o.stats()
        tau.append(float(an.torque_theta(np.array([s["tqx"], s["tqy"], s["tqz"]]) / s["n"], p)))
    f = an.torque_fit(th, ph, tau)
    assert 0.97 < f["K_u"] / Ku < 1.0 and 0.9 < f["K_c"] / Kc < 1.0, f
