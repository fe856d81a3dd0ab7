"""Studies of arXiv:2103.03517 driven through the library's public API: the
magnetisation curve m(T) with the susceptibilities of Eq. 6 and the Bloch law
of Eq. 3 (Sec. 3, Fig. 1); the exchange stiffness A(T) by the Bloch-wall method (Sec. 3, Eq. 5) with K(T)
from the easy-axis estimator (Eq. 4) and its low-temperature m^k exponent as a
function of K/J (Table I); the anisotropy constants K_u(T), K_c(T) from the
constrained torque against the constraint direction (Sec. 3, Fig. 1(a)); the
pinned Bloch wall's averaged profile, width and A(T) (Sec. 3, Eq. 5, Fig. 2);
the average Curie temperature of granular films from the weighted Bloch
series of Eq. 8 (Sec. 4).  Every sweep and sample runs
in libmc; the fits are host post-processing (``analysis``).
"""
from __future__ import annotations

import math
import time

import numpy as np

from . import _mc as mc
from . import analysis as an

__all__ = ["magnetization_curve", "exchange_stiffness_study", "bloch_wall_spins", "film_curie_study",
           "anisotropy_torque_study", "pinned_wall_study", "chain_ensembles"]


def magnetization_curve(dims, temps, K_u=0.01, K_c=0.0, n_eq=2000, n_meas=5000, seed=0, precision=mc.MC_FP32,
                        m_fit_min=0.2, stream=None, device=0):
    """m(T) of Sec. 3 (Fig. 1): one periodic lattice per temperature, all
    advanced as one group (one launch per colour pass for every
    temperature), easy axis z, all spins starting along +z.  dims is one
    (Lx, Ly, Lz) for every temperature or a list with one per temperature
    (uneven sizes batch like equal ones).  n_eq sweeps of equilibration, then
    n_meas measured sweeps with one sample each; lattice i takes seed + i.

    Per temperature: <|m|> and its blocking error, <m_z>, the susceptibilities
    of Eq. 6 in reduced units (mu_S = 1): chi_par = N (<m_z^2> - <|m_z|>^2) / T
    along the easy axis (the |m_z| form is not spoiled by the sign flips of a
    small lattice near T_C), chi_perp = (chi_x + chi_y) / 2 over the hard
    axes, chi_l from |m|; <E/N> and its error; k(T) of Eq. 4 (k_u if
    K_u != 0, else k_c if K_c != 0); the acceptance of the last sweep.  Eq. 3
    is fitted to the temperatures with <|m|> >= m_fit_min when at least three
    qualify.  Returns a dict of per-temperature lists, the fit (T_C, beta or
    None), spin-updates and wall time."""
    temps = [float(t) for t in temps]
    if not temps:
        raise ValueError("no temperatures")
    if n_eq < 0 or n_meas < 1:
        raise ValueError("need n_eq >= 0 and n_meas >= 1")
    sizes = [tuple(int(v) for v in dims)] * len(temps) if np.ndim(dims[0]) == 0 else [tuple(d) for d in dims]
    if len(sizes) != len(temps):
        raise ValueError("one dims per temperature")
    hs = []
    try:
        for i, (d, T) in enumerate(zip(sizes, temps)):
            hs.append(mc.mc_create_ex(mc.make_desc(d, K_u=K_u, K_c=K_c, T=T, seed=seed + i, precision=precision,
                                                   ring_capacity=n_meas, sample_torque=0, stream=stream,
                                                   device=device)))
        g = mc.mc_group_create(hs)
        t0 = time.perf_counter()
        try:
            mc.mc_group_sweep(g, n_eq)
            for h in hs:
                mc.mc_reset_stats(h)
            mc.mc_group_sweep(g, n_meas, measure=True)
            obs = mc.mc_group_measure(g, len(hs))
        finally:
            mc.mc_group_destroy(g)
        wall = time.perf_counter() - t0
        out = {k: [] for k in ("T", "N", "m", "m_err", "mz", "chi_par", "chi_perp", "chi_l", "e", "e_err", "k",
                               "accept")}
        for h, o, d, T in zip(hs, obs, sizes, temps):
            N = int(np.prod(d))
            err = an.sample_errors(mc.mc_samples(h, n_meas))
            k = mc.mc_anisotropy_scaling(h)
            out["T"].append(T)
            out["N"].append(N)
            out["m"].append(o.ml)
            out["m_err"].append(err["ml"][1])
            out["mz"].append(o.m[2])
            out["chi_par"].append(N * (o.m2[2] - o.m_abs[2] ** 2) / T)
            out["chi_perp"].append(0.5 * (o.chi[1] + o.chi[2]))
            out["chi_l"].append(o.chi[0])
            out["e"].append(o.e)
            out["e_err"].append(err["e"][1])
            out["k"].append(float(k[0] if K_u != 0.0 else k[1]))
            out["accept"].append(o.accept_last)
    finally:
        for h in hs:
            mc.mc_destroy(h)
    Tf = [T for T, m in zip(out["T"], out["m"]) if m >= m_fit_min]
    mf = [m for m in out["m"] if m >= m_fit_min]
    out["T_C"], out["beta"] = None, None
    if len(Tf) >= 3:
        try:
            out["T_C"], out["beta"], _ = an.bloch_fit(Tf, mf)
        except RuntimeError:  # no convergence: leave the fit out
            pass
    out["updates"] = float(sum(out["N"])) * (n_eq + n_meas)
    out["seconds"] = wall
    return out


def bloch_wall_spins(dims, K, J=1.0):
    """Spins (N x 3, site order x + Lx (y + Ly z)) of the continuum Bloch wall
    centred in x: phi(x) = 2 arctan(exp(pi (x - Lx/2) / Delta0)), Delta0 =
    pi sqrt(J / 2K), S = (0, sin phi, cos phi); with x anti-periodic the
    closure S(Lx) = -S(0) matches the wall's far side."""
    Lx, Ly, Lz = dims
    x = np.arange(Lx, dtype=np.float64) + 0.5
    phi = 2.0 * np.arctan(np.exp(math.pi * (x - Lx / 2) / (math.pi * math.sqrt(J / (2.0 * K)))))
    row = np.stack([np.zeros(Lx), np.sin(phi), np.cos(phi)], axis=1)
    return np.tile(row, (Ly * Lz, 1))


def exchange_stiffness_study(K_over_J, temps, wall_dims=(256, 64, 64), uniform_dims=(64, 64, 64), n_eq=2000,
                             n_meas=4000, every=20, m_min=0.6, seed=1, precision=mc.MC_FP32, stream=None,
                             device=0):
    """For every K/J (uniaxial K along z, J = 1) and temperature T:

    * a wall lattice, x anti-periodic and y, z periodic, started on the
      continuum Bloch wall of width pi sqrt(J / 2K) (the wall setup of Sec. 3,
      rotating in the y-z plane); every `every` measured sweeps one
      slice profile m_z(x) is taken and fitted by the tanh of Sec. 3, and the
      width Delta(T) is the mean of the fits that find a wall (amplitude above
      0.05, width below Lx; above T_C none does and Delta is NaN);
    * a uniform periodic lattice, whose samples give m(T) = <|m|> and
      K(T) = K k_u(T) by Eq. 4;
    * A(T) = K(T) (Delta / pi)^2 (Eq. 5), and for each K/J the exponent k of
      A ~ m^k over the points with m > m_min (Table I);
    * when the uniform lattice has the wall lattice's size, the free-energy
      route of Eq. 5 as well: dU = N (e_wall - e_uniform), dF(T) from dU over
      the given temperatures (which should then reach well above T_C, the
      integral starting at beta = 0), and A_dF = dF^2 / (16 C^2 K(T)) with C
      = Ly Lz.

    All lattices advance together as one group.  Returns a dict with the
    per-point table, the exponents, the spin-updates run and the wall time.
    """
    K_over_J = [float(k) for k in K_over_J]
    temps = [float(t) for t in temps]
    points = [(k, t) for k in K_over_J for t in temps]
    walls, unis = [], []
    try:
        for i, (K, T) in enumerate(points):
            walls.append(mc.mc_create_ex(mc.make_desc(
                wall_dims, K_u=K, T=T, seed=seed + 2 * i, precision=precision,
                boundary=(mc.MC_ANTIPERIODIC, mc.MC_PERIODIC, mc.MC_PERIODIC), ring_capacity=16,
                sample_torque=0, stream=stream, device=device)))
            mc.mc_set_spins(walls[-1], bloch_wall_spins(wall_dims, K))
            unis.append(mc.mc_create_ex(mc.make_desc(
                uniform_dims, K_u=K, T=T, seed=seed + 2 * i + 1, precision=precision, ring_capacity=16,
                sample_torque=0, stream=stream, device=device)))
        g = mc.mc_group_create(walls + unis)
        t0 = time.perf_counter()
        try:
            mc.mc_group_sweep(g, n_eq)
            for h in walls + unis:
                mc.mc_reset_stats(h)
            Lx = wall_dims[0]
            prev = [np.zeros(Lx) for _ in walls]
            deltas = [[] for _ in walls]
            blocks = max(1, n_meas // every)
            for b in range(blocks):
                mc.mc_group_sweep(g, every, measure=True)
                for w, h in enumerate(walls):
                    mc.mc_profile_sample(h)
                    avg = mc.mc_profile(h, 2, Lx)  # mean over the b + 1 samples so far
                    one = avg * (b + 1) - prev[w] * b
                    prev[w] = avg
                    try:
                        m_w, _, d_w, _ = an.fit_wall(one)
                    except RuntimeError:  # a profile the fit cannot follow (near T_C)
                        continue
                    if abs(m_w) > 0.05 and 0.0 < d_w < Lx:  # a wall (none above T_C)
                        deltas[w].append(d_w)
            mc.mc_group_sync(g)
        finally:
            mc.mc_group_destroy(g)
        seconds = time.perf_counter() - t0
        rows = []
        for w, (K, T) in enumerate(points):
            ow, ou = mc.mc_measure(walls[w]), mc.mc_measure(unis[w])
            k_u = float(mc.mc_anisotropy_scaling(unis[w])[0])
            d = np.asarray(deltas[w])
            delta = float(d.mean()) if d.size else float("nan")
            d_err = float(d.std(ddof=1) / math.sqrt(d.size)) if d.size > 1 else float("nan")
            K_T = K * k_u
            rows.append({"K": K, "T": T, "m": float(ou.ml), "k_u": k_u, "K_T": K_T, "delta": delta,
                         "delta_err": d_err, "A": float(an.exchange_stiffness(delta, K_T)),
                         "e_wall": float(ow.e), "e_uniform": float(ou.e), "profiles": int(d.size)})
    finally:
        for h in walls + unis:
            mc.mc_destroy(h)
    if tuple(uniform_dims) == tuple(wall_dims):  # the free-energy route
        N, C = int(np.prod(wall_dims)), wall_dims[1] * wall_dims[2]
        for K in K_over_J:
            r = [x for x in rows if x["K"] == K]
            dU = np.array([N * (x["e_wall"] - x["e_uniform"]) for x in r])
            dF = an.free_energy_difference([x["T"] for x in r], dU)
            for x, f in zip(r, dF):
                x["dF"] = float(f)
                x["A_dF"] = float(an.stiffness_from_free_energy(f, C, x["K_T"])) if x["K_T"] > 0 else float("nan")
    exponents = {}
    for K in K_over_J:
        r = [x for x in rows if x["K"] == K and np.isfinite(x["A"]) and x["A"] > 0]
        m = np.array([x["m"] for x in r])
        A = np.array([x["A"] for x in r])
        if int(np.sum(m > m_min)) >= 3:
            k, k_err, _ = an.power_exponent(m, A, m_min=m_min)
            exponents[K] = (k, k_err)
    updates = len(points) * (n_eq + blocks * every) * (int(np.prod(wall_dims)) + int(np.prod(uniform_dims)))
    return {"rows": rows, "exponents": exponents, "updates": updates, "seconds": seconds}


def film_curie_study(dims, grain_id, bond_mask, grain_axis, temps, K_u=0.02, n_eq=1000, n_meas=2000, every=20,
                     n_terms=20, beta=None, seed=1, precision=mc.MC_FP32, stream=None, device=0):
    """m(T) of a granular film and its average Curie temperature (Sec. 4,
    Eq. 8).  The film (x, y periodic, z open; grain tables as for
    mc_create_ex: bonds only inside a grain, one uniaxial easy axis per
    grain) is run independently at every temperature, all runs as one group;
    every `every` measured sweeps each run takes a grain sample.  The film's
    m(T) = sum_g w_g <m_g>(T), w_g = N_g / N (columnar grains: weight by
    area), and the weighted Bloch series of Eq. 8 with n_terms terms gives
    T_C_mean; beta fixes the exponent of every term (the continuous film's
    own, from Eq. 3, is the natural choice: the grains are the same material
    at the same thickness), None searches it.  With grain_id None the film is
    continuous (one grain, no bond mask, easy axis z): m(T) = <|m|> and Eq. 3
    gives its T_C and beta.  Returns a dict: T, m, the fit, spin-updates and
    wall time."""
    temps = [float(t) for t in temps]
    N = int(np.prod(dims))
    grains = grain_id is not None
    if grains:
        grain_id = np.ascontiguousarray(grain_id, np.int32)
        ng = int(grain_id.max()) + 1
        w = np.bincount(grain_id, minlength=ng) / float(N)
    hs = []
    try:
        for i, T in enumerate(temps):
            kw = dict(bond_mask=bond_mask, grain_id=grain_id, grain_axis=grain_axis) if grains else {}
            hs.append(mc.mc_create_ex(mc.make_desc(dims, K_u=K_u, T=T, seed=seed + i, precision=precision,
                                                   boundary=(mc.MC_PERIODIC, mc.MC_PERIODIC, mc.MC_OPEN),
                                                   ring_capacity=16, sample_torque=0, stream=stream,
                                                   device=device, **kw)))
        g = mc.mc_group_create(hs)
        t0 = time.perf_counter()
        try:
            mc.mc_group_sweep(g, n_eq)
            for h in hs:
                mc.mc_reset_stats(h)
            blocks = max(1, n_meas // every)
            for _ in range(blocks):
                mc.mc_group_sweep(g, every, measure=True)
                if grains:
                    for h in hs:
                        mc.mc_grain_sample(h)
            mc.mc_group_sync(g)
        finally:
            mc.mc_group_destroy(g)
        if grains:
            m = np.array([float(w @ mc.mc_grain_magnetization(h, ng)[0]) for h in hs])
        else:
            m = np.array([float(mc.mc_measure(h).ml) for h in hs])
        seconds = time.perf_counter() - t0
    finally:
        for h in hs:
            mc.mc_destroy(h)
    T = np.array(temps)
    if grains:
        fit = an.multi_bloch_fit(T, m, n_terms, betas=None if beta is None else [round(float(beta), 2)])
        fit = {"T_C_mean": fit["T_C_mean"], "beta": fit["beta"], "rms": fit["rms"],
               "w": fit["w"].tolist(), "T_C": fit["T_C"].tolist()}
    else:  # Eq. 3 over the ordered range (m above 0.3, below it the finite film's tail)
        tc, beta, err = an.bloch_fit(T[m > 0.3], m[m > 0.3])
        fit = {"T_C": tc, "beta": beta, "errors": err.tolist()}
    updates = len(temps) * (n_eq + blocks * every) * N
    return {"T": temps, "m": m.tolist(), "fit": fit, "updates": updates, "seconds": seconds}


def _unit(theta_deg, phi_deg):
    t, p = math.radians(theta_deg), math.radians(phi_deg)
    return (math.sin(t) * math.cos(p), math.sin(t) * math.sin(p), math.cos(t))


def anisotropy_torque_study(dims=(64, 64, 64), K_u=0.05, K_c=0.02, temps=(0.2, 0.6, 1.0, 1.3),
                            thetas=tuple(range(0, 91, 10)), phis=(0.0, 45.0), n_eq=3000, n_meas=5000, seed=0,
                            precision=mc.MC_FP32, stream=None, device=0):
    """Asselin's torque method of Sec. 3 (Fig. 1(a)) with the parallel
    constrained algorithm (Table A2): one periodic lattice per (T, phi,
    theta), started along its constraint direction e_C(theta, phi) and
    held there, all advanced as one group; n_eq sweeps, then n_meas measured
    sweeps with the torque sampled every sweep.  Per run: <tau_theta> (per
    spin, along increasing theta) with its blocking error.  Per temperature:
    K_u(T) and K_c(T) from analysis.torque_fit over that temperature's runs,
    weighted by the errors.  Run i takes seed + i.  Returns {"runs": [...],
    "fits": {T: fit}, "updates", "seconds"} (pair halves count as updates)."""
    runs = [(float(T), float(ph), float(th)) for T in temps for ph in phis for th in thetas]
    hs = []
    try:
        for i, (T, ph, th) in enumerate(runs):
            hs.append(mc.mc_create_ex(mc.make_desc(dims, K_u=K_u, K_c=K_c, T=T, seed=seed + i, precision=precision,
                                                   init_dir=_unit(th, ph), ring_capacity=n_meas, stream=stream,
                                                   device=device)))
        g = mc.mc_group_create(hs)
        th_l, ph_l = [r[2] for r in runs], [r[1] for r in runs]
        t0 = time.perf_counter()
        try:
            mc.mc_group_constrained_sweep(g, th_l, ph_l, n_eq)
            for h in hs:
                mc.mc_reset_stats(h)
            mc.mc_group_constrained_sweep(g, th_l, ph_l, n_meas, measure=True)
            obs = mc.mc_group_measure(g, len(hs))
        finally:
            mc.mc_group_destroy(g)
        seconds = time.perf_counter() - t0
        rows = []
        for h, o, (T, ph, th) in zip(hs, obs, runs):
            series = an.torque_theta(mc.mc_samples(h, n_meas)["torque"], ph)
            rows.append({"T": T, "phi": ph, "theta": th, "tau": float(an.torque_theta(np.array(o.torque), ph)),
                         "tau_err": float(an.blocking_error(series)), "m_l": float(o.ml)})
    finally:
        for h in hs:
            mc.mc_destroy(h)
    fits = {}
    for T in sorted({r["T"] for r in rows}):
        r = [x for x in rows if x["T"] == T]
        sig = np.array([max(x["tau_err"], 1e-12) for x in r])
        fits[T] = an.torque_fit([x["theta"] for x in r], [x["phi"] for x in r], [x["tau"] for x in r], sigma=sig)
    updates = float(len(runs)) * float(np.prod(dims)) * (n_eq + n_meas)
    return {"runs": rows, "fits": fits, "updates": updates, "seconds": seconds}


def pinned_wall_study(temps, dims=(1024, 128, 128), K_u=0.05, n_eq=2000, n_meas=4000, every=10,
                      uniform_dims=(64, 64, 64), uniform_sweeps=(1000, 2000), seed=0, precision=mc.MC_FP32,
                      stream=None, device=0):
    """The Bloch-wall method of Sec. 3 (Eq. 5, Fig. 2) on walls held by
    pinned end planes: x = 0 at +z and x = Lx - 1 at -z, y and z periodic,
    started as a step at Lx / 2 (the wall workload of 1024 x 128 x 128 spins).
    Every `every` measured sweeps one slice profile m_z(x) is taken and
    fitted by the tanh of Sec. 3; the wall drifts, so each profile is
    shifted by its fitted centre (rounded) to the middle before it enters the
    average.  Per temperature: the re-centred average profile, its width
    Delta from the tanh fit, the mean width of the single-profile fits, and
    K(T) from a constrained uniform lattice held at theta = 45 deg (tau_theta
    = -K(T) sin 2 theta per spin, Fig. 1(a)), so A(T) = K(T) (Delta / pi)^2.
    Returns {"rows": [...], "updates", "seconds"}."""
    temps = [float(t) for t in temps]
    Lx = int(dims[0])
    walls, unis = [], []
    try:
        for i, T in enumerate(temps):
            walls.append(mc.mc_create_ex(mc.make_desc(
                dims, K_u=K_u, T=T, seed=seed + 2 * i, precision=precision, init=mc.MC_INIT_WALL,
                boundary=(mc.MC_PINNED, mc.MC_PERIODIC, mc.MC_PERIODIC), ring_capacity=16, sample_torque=0,
                stream=stream, device=device)))
            unis.append(mc.mc_create_ex(mc.make_desc(
                uniform_dims, K_u=K_u, T=T, seed=seed + 2 * i + 1, precision=precision, init_dir=_unit(45.0, 0.0),
                ring_capacity=16, stream=stream, device=device)))
        t0 = time.perf_counter()
        gu = mc.mc_group_create(unis)
        try:
            th, ph = [45.0] * len(unis), [0.0] * len(unis)
            mc.mc_group_constrained_sweep(gu, th, ph, uniform_sweeps[0])
            for h in unis:
                mc.mc_reset_stats(h)
            mc.mc_group_constrained_sweep(gu, th, ph, uniform_sweeps[1], measure=True)
            K_T = [-float(an.torque_theta(np.array(o.torque), 0.0)) for o in mc.mc_group_measure(gu, len(unis))]
        finally:
            mc.mc_group_destroy(gu)
        gw = mc.mc_group_create(walls)
        acc = [np.zeros(Lx) for _ in walls]
        cnt = [np.zeros(Lx) for _ in walls]
        widths = [[] for _ in walls]
        try:
            mc.mc_group_sweep(gw, n_eq)
            for h in walls:
                mc.mc_reset_stats(h)
            prev = [np.zeros(Lx) for _ in walls]
            blocks = max(1, n_meas // every)
            x = np.arange(Lx)
            for b in range(blocks):
                mc.mc_group_sweep(gw, every, measure=True)
                for w, h in enumerate(walls):
                    mc.mc_profile_sample(h)
                    avg = mc.mc_profile(h, 2, Lx)  # mean over the b + 1 samples so far
                    one = avg * (b + 1) - prev[w] * b
                    prev[w] = avg
                    try:
                        m_w, x0, d_w, _ = an.fit_wall(one, antiperiodic=False)
                    except RuntimeError:
                        continue
                    if not (abs(m_w) > 0.05 and 0.0 < d_w < Lx and 0.0 <= x0 < Lx):
                        continue  # no wall (near or above T_C)
                    widths[w].append(d_w)
                    s = int(round(x0 - Lx / 2))
                    src = x + s
                    ok = (src >= 0) & (src < Lx)
                    acc[w][ok] += one[src[ok]]
                    cnt[w][ok] += 1.0
            mc.mc_group_sync(gw)
        finally:
            mc.mc_group_destroy(gw)
        seconds = time.perf_counter() - t0
        rows = []
        for w, T in enumerate(temps):
            prof = np.where(cnt[w] > 0, acc[w] / np.maximum(cnt[w], 1.0), np.nan)
            delta = float("nan")
            m_amp = float("nan")
            good = np.isfinite(prof)
            if widths[w] and good.sum() > 16:
                # planes no shifted profile reached (next to the pinned ends)
                # take the nearest averaged value: the profile is flat there
                idx = np.arange(Lx)
                filled = np.interp(idx, idx[good], prof[good])
                try:
                    m_amp, _, delta, _ = an.fit_wall(filled, antiperiodic=False)
                except RuntimeError:
                    pass
            d = np.asarray(widths[w])
            rows.append({"T": T, "K_T": K_T[w], "delta": delta, "m_wall": m_amp,
                         "delta_single_mean": float(d.mean()) if d.size else float("nan"),
                         "delta_single_err": float(d.std(ddof=1) / math.sqrt(d.size)) if d.size > 1 else float("nan"),
                         "profiles": int(d.size), "A": float(an.exchange_stiffness(delta, K_T[w])),
                         "profile": [float(v) for v in prof]})
    finally:
        for h in walls + unis:
            mc.mc_destroy(h)
    updates = float(len(temps)) * (float(np.prod(dims)) * (n_eq + max(1, n_meas // every) * every)
                                   + float(np.prod(uniform_dims)) * sum(uniform_sweeps))
    return {"rows": rows, "updates": updates, "seconds": seconds}


def chain_ensembles(cases, n_chains, seed_of, sweeps_of, precision=mc.MC_FP32, max_group=4096, stream=None,
                    device=0):
    """Independent chains of Table A1 for each case: cases maps a name to a
    lattice description (dims, K_u, T, J, axis attributes, as
    workloads.LatticeSpec), n_chains maps a name to a chain count, seed_of(name,
    k) gives chain k's seed and sweeps_of(name) its (n_eq, n_meas).  Every chain
    starts along +z, runs n_eq sweeps, then n_meas measured sweeps (the cone
    adapting in every sweep).  Chains run as groups of at most max_group
    lattices.  Returns {name: {"ml", "ml2", "mabs_z", "mz", "e": arrays of the
    per-chain means over the measured sweeps}}."""
    jobs = [(name, k) for name in cases for k in range(int(n_chains[name]))]
    out = {name: {key: [] for key in ("ml", "ml2", "mabs_z", "mz", "e")} for name in cases}
    # chains of equal sweep counts share a group
    by_sweeps = {}
    for name, k in jobs:
        by_sweeps.setdefault(tuple(sweeps_of(name)), []).append((name, k))
    for (n_eq, n_meas), js in by_sweeps.items():
        for i in range(0, len(js), max_group):
            chunk = js[i:i + max_group]
            hs = []
            try:
                for name, k in chunk:
                    sp = cases[name]
                    hs.append(mc.mc_create_ex(mc.make_desc(sp.dims, J=sp.J, K_u=sp.Ku, axis=sp.axis, T=sp.T,
                                                           seed=seed_of(name, k), theta0_deg=sp.theta0,
                                                           precision=precision, ring_capacity=1, sample_torque=0,
                                                           stream=stream, device=device)))
                g = mc.mc_group_create(hs)
                try:
                    mc.mc_group_sweep(g, n_eq)
                    for h in hs:
                        mc.mc_reset_stats(h)
                    mc.mc_group_sweep(g, n_meas, measure=True)
                    obs = mc.mc_group_measure(g, len(hs))
                finally:
                    mc.mc_group_destroy(g)
                for (name, _), o in zip(chunk, obs):
                    d = out[name]
                    d["ml"].append(o.ml)
                    d["ml2"].append(o.ml2)
                    d["mabs_z"].append(o.m_abs[2])
                    d["mz"].append(o.m[2])
                    d["e"].append(o.e)
            finally:
                for h in hs:
                    mc.mc_destroy(h)
    return {name: {key: np.asarray(v) for key, v in d.items()} for name, d in out.items()}
