"""Host analysis of the library's outputs for Sec. 3 and 4 of arXiv:2103.03517:
the domain-wall width fit and the exchange stiffness of Eq. 5, the free-energy
route dF(T) of Eq. 5, the m^k scaling exponent of Table I, the Bloch law of
Eq. 3, the transverse susceptibility of Eq. 7, the weighted Bloch series of
Eq. 8 for granular films, the anisotropy constants from the constrained
torque (Sec. 3, Fig. 1(a)), and error bars of the per-sweep series by blocking.  Plain numpy / scipy on the host; reduced units
(J = 1, k_B = 1, mu_S = 1, lattice constant 1).
"""
from __future__ import annotations

import math

import numpy as np

__all__ = ["wall_model", "fit_wall", "exchange_stiffness", "free_energy_difference",
           "stiffness_from_free_energy", "power_exponent", "bloch_fit", "chi_perp_uniaxial", "multi_bloch_fit",
           "blocking_error", "sample_errors", "torque_basis", "torque_fit", "torque_theta"]


def wall_model(x, m, x0, delta, Lx=None):
    """Bloch-wall profile of Sec. 3: m_z(x) = m tanh(-pi (x - x0) / delta).
    With Lx given the profile is anti-periodic, m_z(x + Lx) = -m_z(x) (the
    wall setup with x anti-periodic): x - x0 is folded into [-Lx/2, Lx/2) and
    each fold by Lx flips the sign."""
    x = np.asarray(x, np.float64)
    d = x - x0
    sign = np.ones_like(d)
    if Lx is not None:
        k = np.floor((d + 0.5 * Lx) / Lx)
        d = d - k * Lx
        sign = np.where(np.mod(k, 2) == 0, 1.0, -1.0)
    return sign * m * np.tanh(-math.pi * d / delta)


def fit_wall(mz, antiperiodic=True, x=None):
    """Least-squares fit of wall_model to a slice profile m_z(x) (one value
    per x-plane, from mc_profile), returning (m, x0, delta, errors).  The
    start is the profile's own sign change; with antiperiodic the wall may sit
    anywhere, the boundary included."""
    from scipy.optimize import curve_fit

    mz = np.asarray(mz, np.float64)
    Lx = mz.size
    x = np.arange(Lx, dtype=np.float64) if x is None else np.asarray(x, np.float64)
    m0 = max(float(np.abs(mz).max()), 1e-3)
    # start: the + to - crossing of the (anti-periodically extended) profile
    ext = np.concatenate([mz, -mz]) if antiperiodic else mz
    cross = [i for i in range(ext.size - 1) if ext[i] > 0 >= ext[i + 1]]
    x0 = float(cross[0]) + 0.5 if cross else 0.5 * Lx  # in [Lx, 2 Lx): a reversed wall
    width = max(2.0, float(np.sum(np.abs(mz) < 0.76 * m0)) * math.pi / 2.0)  # |tanh| < 0.76 over ~delta/pi*2
    f = (lambda xx, m, c, d: wall_model(xx, m, c, d, Lx)) if antiperiodic else (lambda xx, m, c, d: wall_model(xx, m, c, d))
    import warnings

    with warnings.catch_warnings():  # a flat profile leaves the covariance undefined (inf errors)
        warnings.simplefilter("ignore")
        p, cov = curve_fit(f, x, mz, p0=[m0, x0, width], maxfev=20000)
    m, c, d = p
    if d < 0:  # the model is symmetric under (m, delta) -> (-m, -delta)
        m, d = -m, -d
    if antiperiodic:  # x0 into [0, Lx); each fold by Lx flips the sign of m
        k = math.floor(c / Lx)
        c -= k * Lx
        m = -m if k % 2 else m
    err = np.sqrt(np.maximum(np.diag(cov), 0.0))
    return float(m), float(c), float(d), err


def exchange_stiffness(delta, K):
    """Eq. 5 solved for A: Delta = pi sqrt(A / K), so A = K (Delta / pi)^2."""
    return np.asarray(K, np.float64) * (np.asarray(delta, np.float64) / math.pi) ** 2


def free_energy_difference(T, dU):
    """dF(T) of a wall from internal energies (Eq. 5 and the text after it):
    with beta = 1/T, d(beta F)/d beta = U, and at beta = 0 the two states
    have the same free energy, so beta dF(beta) = int_0^beta dU(b) db.  dU
    is <E>_wall - <E>_uniform at the temperatures T (any order); at beta = 0
    every state has the same weight in both, so dU(0) = 0 and the integral is
    the trapezoid rule over the beta grid from (0, 0)."""
    T = np.asarray(T, np.float64)
    dU = np.asarray(dU, np.float64)
    order = np.argsort(1.0 / T)
    beta = np.concatenate([[0.0], 1.0 / T[order]])
    u = np.concatenate([[0.0], dU[order]])
    integral = np.concatenate([[0.0], np.cumsum(0.5 * (u[1:] + u[:-1]) * np.diff(beta))])
    dF = np.empty_like(T)
    dF[order] = integral[1:] / beta[1:]
    return dF


def stiffness_from_free_energy(dF, C, K):
    """Eq. 5, dF = 4 C sqrt(A K), solved for A = dF^2 / (16 C^2 K); C is the
    wall's cross-section (Ly Lz)."""
    return np.asarray(dF, np.float64) ** 2 / (16.0 * float(C) ** 2 * np.asarray(K, np.float64))


def power_exponent(m, y, m_min=0.0, sigma_y=None):
    """Exponent k of y ~ m^k (Table I: A(T) against m(T), low-temperature
    range m > m_min) by least squares on log y = log c + k log m; returns
    (k, its standard error, c).  sigma_y weights the points (relative error
    sigma_y / y in log space)."""
    m = np.asarray(m, np.float64)
    y = np.asarray(y, np.float64)
    sel = (m > m_min) & (y > 0)
    X = np.stack([np.ones(sel.sum()), np.log(m[sel])], axis=1)
    Y = np.log(y[sel])
    w = np.ones(sel.sum()) if sigma_y is None else (y[sel] / np.asarray(sigma_y, np.float64)[sel])
    Xw, Yw = X * w[:, None], Y * w
    coef, res, *_ = np.linalg.lstsq(Xw, Yw, rcond=None)
    dof = max(1, X.shape[0] - 2)
    s2 = float(np.sum((Yw - Xw @ coef) ** 2)) / dof if sigma_y is None else 1.0
    cov = s2 * np.linalg.inv(Xw.T @ Xw)
    return float(coef[1]), float(math.sqrt(cov[1, 1])), float(math.exp(coef[0]))


def bloch_fit(T, m, T_max=None):
    """Eq. 3, m(T) = (1 - T/T_C)^beta, fitted to (T, m) with T < T_max;
    returns (T_C, beta, errors)."""
    from scipy.optimize import curve_fit

    T = np.asarray(T, np.float64)
    m = np.asarray(m, np.float64)
    sel = T < (T_max if T_max is not None else np.inf)
    f = lambda t, tc, b: np.power(np.clip(1.0 - t / tc, 1e-12, None), b)
    p, cov = curve_fit(f, T[sel], m[sel], p0=[1.05 * T[sel].max(), 0.35], maxfev=20000)
    return float(p[0]), float(p[1]), np.sqrt(np.maximum(np.diag(cov), 0.0))


def chi_perp_uniaxial(m, Ku_T, Ms0=1.0):
    """Eq. 7: transverse susceptibility below T_C, M_S(0) m^2 / (2 K_u(T))."""
    return float(Ms0) * np.asarray(m, np.float64) ** 2 / (2.0 * np.asarray(Ku_T, np.float64))


def multi_bloch_fit(T, m, n_terms, tc_range=None, betas=None):
    """Eq. 8: m(T) = sum_i w_i (1 - T/T_C,i)^beta_i with sum w_i = 1 (a term
    is zero above its T_C,i), and the average Curie temperature T_C =
    sum_i w_i T_C,i.  The paper fixes only the series; this fit places the
    n_terms values T_C,i on an even grid over tc_range (default: from the
    lowest T to 1.25 times the highest), gives every term one exponent beta
    (the best of `betas`, default 0.15 .. 0.80 in steps of 0.01) and finds
    the weights w_i >= 0 by non-negative least squares with the sum held to 1
    by a heavily weighted extra row.  More terms refine the grid; the paper's
    average converges once n_terms exceeds about 10.  Returns a dict: w, T_C,
    beta, T_C_mean, rms (of the fit)."""
    from scipy.optimize import nnls

    T = np.asarray(T, np.float64)
    m = np.asarray(m, np.float64)
    lo, hi = tc_range if tc_range is not None else (float(T.min()), 1.25 * float(T.max()))
    Tc = np.linspace(lo, hi, int(n_terms) + 1)[1:]
    betas = np.round(np.arange(0.15, 0.8001, 0.01), 10) if betas is None else np.asarray(betas, np.float64)
    lam = 1e3 * math.sqrt(T.size)
    best = None
    for b in betas:
        X = np.clip(1.0 - T[:, None] / Tc[None, :], 0.0, None) ** b
        w, _ = nnls(np.vstack([X, lam * np.ones(Tc.size)]), np.concatenate([m, [lam]]))
        rms = float(np.sqrt(np.mean((X @ w - m) ** 2)))
        if best is None or rms < best["rms"]:
            best = {"w": w, "T_C": Tc, "beta": float(b), "T_C_mean": float(w @ Tc), "rms": rms}
    return best


def blocking_error(x, min_blocks: int = 32) -> float:
    """Standard error of the mean of a correlated series, by the blocking
    method of Flyvbjerg and Petersen (J. Chem. Phys. 91, 461 (1989)).

    The series is coarsened by averaging neighbouring pairs (an odd last
    element is dropped) while at least min_blocks blocks remain; level k with
    n_k blocks gives the naive error sqrt(var_k / n_k).  Once the blocks are
    longer than the correlation time these sit on a plateau at the true
    error.  The largest over the levels is returned: a conservative reading of
    the plateau, which on series of a few thousand correlated samples is
    within a few percent of the true error on average, where stopping at the
    first level that agrees with the deeper ones comes out 10-25% low; for
    independent samples it is std / sqrt(n) or a little above (about 8% on
    average with 32 blocks at the deepest level).  0 for a series too short
    for one level."""
    x = np.asarray(x, np.float64).ravel()
    best = 0.0
    while x.size >= max(2, min_blocks):
        n = x.size
        best = max(best, float(np.sqrt(np.var(x, ddof=1) / n)))
        x = 0.5 * (x[: n // 2 * 2: 2] + x[1: n // 2 * 2: 2])
    return best


def sample_errors(samples, min_blocks: int = 32) -> dict:
    """Means and blocking errors of the per-sweep series of one lattice, from
    the structured array mc_samples returns (fields m, e_parts, torque).

    Returns {name: (mean, error)} for |m|, m_x, m_y, m_z, |m_z|, the total
    energy per spin E/N (sum of the four parts of Eq. 2) and the three torque
    components per spin."""
    m = np.asarray(samples["m"], np.float64)
    series = {"ml": np.linalg.norm(m, axis=1), "mx": m[:, 0], "my": m[:, 1], "mz": m[:, 2],
              "mz_abs": np.abs(m[:, 2]), "e": np.asarray(samples["e_parts"], np.float64).sum(axis=1)}
    tq = np.asarray(samples["torque"], np.float64)
    for a, name in enumerate(("tx", "ty", "tz")):
        series[name] = tq[:, a]
    return {k: (float(v.mean()), blocking_error(v, min_blocks)) for k, v in series.items()}


def torque_basis(theta_deg, phi_deg):
    """The angular factors of the anisotropy torque of Sec. 3 (Fig. 1(a)).
    The free energy per spin of a magnetisation held along
    e_C = (sin t cos p, sin t sin p, cos t) is F = K_u(T) sin^2 t + K_c(T) q
    with q = a1^2 a2^2 + a1^2 a3^2 + a2^2 a3^2 = sin^4 t sin^2(2p) / 4 +
    sin^2 t cos^2 t, so dF/dt = K_u g_u + K_c g_c with
    g_u = sin 2t and g_c = sin t cos t (sin^2 t sin^2 2p + 2 cos 2t)
    (g_c = sin(4t) / 2 at p = 0, sin t cos t (2 cos^2 t - sin^2 t) at
    p = 45 deg).  Returns (g_u, g_c) as arrays."""
    t = np.radians(np.asarray(theta_deg, np.float64))
    p = np.radians(np.asarray(phi_deg, np.float64))
    g_u = np.sin(2.0 * t)
    g_c = np.sin(t) * np.cos(t) * (np.sin(t) ** 2 * np.sin(2.0 * p) ** 2 + 2.0 * np.cos(2.0 * t))
    return g_u, g_c


def torque_theta(torque, phi_deg):
    """tau_theta = n . tau of a mean torque vector per spin (mc_measure's
    torque), n = (-sin p, cos p, 0): the component along increasing theta,
    so that dF/dtheta = -<tau_theta>."""
    tq = np.asarray(torque, np.float64)
    p = np.radians(np.asarray(phi_deg, np.float64))
    return -np.sin(p) * tq[..., 0] + np.cos(p) * tq[..., 1]


def torque_fit(theta_deg, phi_deg, tau, sigma=None):
    """K_u(T) and K_c(T) from constrained runs at one temperature (Asselin's
    torque method, Sec. 3): linear least squares of
    tau_theta(theta, phi) = -[K_u g_u(theta, phi) + K_c g_c(theta, phi)]
    over the runs (weighted by 1 / sigma^2 when the errors are given).
    Returns {"K_u", "K_c", "K_u_err", "K_c_err", "chi2_dof"}; the errors are
    the fit's standard errors (from sigma, else from the residual scatter)."""
    g_u, g_c = torque_basis(theta_deg, phi_deg)
    y = -np.asarray(tau, np.float64)
    A = np.stack([g_u, g_c], axis=1)
    w = np.ones_like(y) if sigma is None else 1.0 / np.maximum(np.asarray(sigma, np.float64), 1e-300)
    Aw, yw = A * w[:, None], y * w
    coef, _, rank, _ = np.linalg.lstsq(Aw, yw, rcond=None)
    if rank < 2:
        raise ValueError("torque_fit: the angles do not separate the uniaxial and cubic terms")
    resid = yw - Aw @ coef
    dof = max(1, y.size - 2)
    chi2 = float(resid @ resid) / dof
    cov = np.linalg.inv(Aw.T @ Aw) * (1.0 if sigma is not None else chi2)
    return {"K_u": float(coef[0]), "K_c": float(coef[1]), "K_u_err": float(math.sqrt(max(cov[0, 0], 0.0))),
            "K_c_err": float(math.sqrt(max(cov[1, 1], 0.0))), "chi2_dof": chi2}
