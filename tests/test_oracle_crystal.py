"""Pins of the bcc / fcc / hcp oracle (Sec. 2: bcc as 2, fcc as 4 simple
cubic sub-lattices, hcp as 4 simple tetragonal ones, each split red/black).  Expected values come from the atomic
positions, never from the oracle's neighbour table: a brute-force Eq. 2
energy over all pairs at the nearest and next-nearest distances, the
ground-state energy, and harmonic spin waves from the bond graph."""
import math

import numpy as np
import pytest

import oracle

BASIS = {oracle.BCC: [(0, 0, 0), (0.5, 0.5, 0.5)],
         oracle.FCC: [(0, 0, 0), (0.5, 0.5, 0), (0.5, 0, 0.5), (0, 0.5, 0.5)],
         oracle.HCP: [(0, 0, 0), (0.5, 0.5, 0), (0.5, 1 / 6, 0.5), (0, 2 / 3, 0.5)]}
# cell lengths: cubic cells, and the orthohexagonal cell (a, sqrt 3 a, c) with c/a = sqrt(8/3)
ELL = {oracle.BCC: (1.0, 1.0, 1.0), oracle.FCC: (1.0, 1.0, 1.0),
       oracle.HCP: (1.0, math.sqrt(3.0), math.sqrt(8.0 / 3.0))}
NN2 = {oracle.BCC: 0.75, oracle.FCC: 0.5, oracle.HCP: 1.0}
Z1 = {oracle.BCC: 8, oracle.FCC: 12, oracle.HCP: 12}


def positions(kind, cells):
    b = np.array(BASIS[kind], float)
    Lx, Ly, Lz = cells
    out = []
    for z in range(Lz):
        for y in range(Ly):
            for x in range(Lx):
                for s in range(len(b)):
                    out.append((b[s] + (x, y, z)) * ELL[kind])
    return np.array(out)  # site i = s + nsub (x + Lx (y + Ly z))


def bonds(kind, cells, J1, J2):
    """(i, j, J) for every bond, each image once from each end: pairs at the
    nearest (J1) or next-nearest (distance 1, J2) distance, periodic images
    included, so small cells count a doubled bond twice."""
    pos = positions(kind, cells)
    L = np.array(cells, float) * ELL[kind]
    out = []
    for i in range(len(pos)):
        for j in range(len(pos)):
            for n in np.ndindex(3, 3, 3):
                d = pos[j] + (np.array(n) - 1) * L - pos[i]
                r2 = d @ d
                if abs(r2 - NN2[kind]) < 1e-9:
                    out.append((i, j, J1))
                elif abs(r2 - 1.0) < 1e-9 and J2 != 0.0:
                    out.append((i, j, J2))
    return out


def energy(S, bl, Ku, axis, Kc, H):
    E = -0.5 * sum(J * float(S[i] @ S[j]) for i, j, J in bl)
    E -= Ku * float(((S @ axis) ** 2).sum())
    E += Kc * float((S[:, 0] ** 2 * S[:, 1] ** 2 + S[:, 0] ** 2 * S[:, 2] ** 2 + S[:, 1] ** 2 * S[:, 2] ** 2).sum())
    E -= float((S @ np.asarray(H)).sum())
    return E


@pytest.mark.parametrize("kind,cells,J2", [(oracle.BCC, (2, 2, 2), 0.0), (oracle.BCC, (4, 2, 2), 0.3),
                                           (oracle.FCC, (2, 2, 2), 0.0), (oracle.FCC, (2, 4, 2), -0.2),
                                           (oracle.HCP, (2, 2, 2), 0.0), (oracle.HCP, (4, 2, 2), 0.0)])
def test_crystal_delta_e_equals_total_energy_difference(kind, cells, J2):
    rng = np.random.default_rng(int(kind) * 10 + cells[0])
    J1, Ku, Kc = 1.2, 0.3, -0.4
    axis = rng.standard_normal(3)
    axis /= np.linalg.norm(axis)
    H = rng.standard_normal(3) * 0.3
    X = oracle.Crystal(kind, cells, J1=J1, J2=J2, Ku=Ku, axis=axis, Kc=Kc, H=H, T=0.7, seed=1)
    S = rng.standard_normal((X.N, 3))
    S /= np.linalg.norm(S, axis=1, keepdims=True)
    X.set_spins(S)
    bl = bonds(kind, cells, J1, J2)
    assert len([b for b in bl if b[2] == J1]) == Z1[kind] * X.N  # every site has z nearest neighbours
    E0 = energy(S, bl, Ku, axis, Kc, H)
    for _ in range(20):
        i = int(rng.integers(X.N))
        Sn = rng.standard_normal(3)
        Sn /= np.linalg.norm(Sn)
        S1 = S.copy()
        S1[i] = Sn
        assert abs(X.delta_e(i, Sn) - (energy(S1, bl, Ku, axis, Kc, H) - E0)) < 1e-12 * max(1.0, abs(E0))


@pytest.mark.parametrize("kind", [oracle.BCC, oracle.FCC, oracle.HCP])
def test_crystal_sample_energy_equals_brute_force(kind):
    """The measured energy parts of one sweep sum to the brute-force E/N of
    the final state."""
    cells = (2, 2, 2)
    rng = np.random.default_rng(3)
    J2 = 0.0 if kind == oracle.HCP else 0.25
    X = oracle.Crystal(kind, cells, J1=1.0, J2=J2, Ku=0.2, Kc=0.1, H=(0.1, 0.0, -0.2), T=0.8, seed=5)
    S = rng.standard_normal((X.N, 3))
    X.set_spins(S / np.linalg.norm(S, axis=1, keepdims=True))
    X.sweep(1, measure=True)
    st = X.stats()
    E = energy(X.spins(), bonds(kind, cells, 1.0, J2), 0.2, np.array([0, 0, 1.0]), 0.1, (0.1, 0.0, -0.2))
    assert abs(st["e"] - E / X.N) < 1e-13
    assert abs(st["e_ex"] + st["e_u"] + st["e_c"] + st["e_z"] - st["e"]) < 1e-13


@pytest.mark.parametrize("kind,J2", [(oracle.BCC, 0.0), (oracle.FCC, 0.0), (oracle.BCC, 0.2), (oracle.HCP, 0.0)])
def test_crystal_harmonic_spin_waves(kind, J2):
    """Low T, uniaxial K along z: E = 1/2 u^T A u per transverse component
    with A = the bond-weighted graph Laplacian + 2K, so equipartition gives
    1 - <m_z> = (T / N) tr(A^-1) and E/N = E_0 + T, E_0 = -(z1 J1 + z2 J2)/2
    - K.  A comes from the bond list of the positions."""
    cells, K, T = (4, 4, 4), 0.5, 0.03  # a gap of 2K = 1 keeps the uniform mode quick
    X = oracle.Crystal(kind, cells, J1=1.0, J2=J2, Ku=K, T=T, seed=7)
    N = X.N
    A = 2 * K * np.eye(N)
    for i, j, J in bonds(kind, cells, 1.0, J2):
        A[i, i] += J
        A[i, j] -= J
    one_minus_m = T / N * np.trace(np.linalg.inv(A))
    e0 = -(Z1[kind] * 1.0 + 6 * J2) / 2 - K
    X.sweep(500)
    X.sweep(3000, measure=True)
    st = X.stats()
    assert abs((1 - st["mz"]) / one_minus_m - 1) < 0.04, (1 - st["mz"], one_minus_m)
    assert abs(st["e"] - (e0 + T)) < 0.05 * T, (st["e"], e0 + T)


def test_crystal_cone_adaptation_and_order_free_passes():
    """The cone angle adapts toward 50% acceptance over all N spins, and the
    sweep keeps unit spins."""
    X = oracle.Crystal(oracle.FCC, (4, 4, 4), Ku=0.05, T=1.5, seed=9)
    X.sweep(300)
    acc = X.last_accepted() / X.N
    assert abs(acc - 0.5) < 0.05
    S = X.spins()
    assert np.allclose(np.linalg.norm(S, axis=1), 1.0, atol=1e-12)


# --------------------------------------- constrained sweeps (Table A2, Sec. 2)
def _uniform(n, d):
    return np.tile(np.asarray(d, float), (n, 1))


@pytest.mark.parametrize("kind,cells", [(oracle.BCC, (4, 4, 4)), (oracle.FCC, (4, 2, 4)), (oracle.HCP, (4, 2, 2))])
def test_xtal_constrained_conserves_transverse_magnetization(kind, cells):
    """Every accepted pair compensates the transverse components, so the
    total transverse magnetisation stays zero and M_L stays positive."""
    th, ph = 30.0, 20.0
    R = oracle.constraint_frame(th, ph)
    o = oracle.Crystal(kind, cells, J1=1.0, J2=0.1 if kind != oracle.HCP else 0.0, Ku=0.05, Kc=0.02, T=0.8, seed=5)
    o.set_spins(_uniform(o.N, R[0]))
    for _ in range(10):
        assert o.constrained_sweep(th, ph, 5) == 0
        M = o.spins().sum(axis=0)
        assert abs(M @ R[1]) < 1e-9 * o.N and abs(M @ R[2]) < 1e-9 * o.N and M @ R[0] > 0
    assert o.last_accepted() > 0
    assert np.allclose(np.linalg.norm(o.spins(), axis=1), 1.0, atol=1e-10)


@pytest.mark.parametrize("kind", [oracle.FCC, oracle.HCP])
def test_xtal_constrained_low_temperature_torque(kind):
    """T -> 0 along e_C(theta, phi = 0) on a crystal: the anisotropy is per
    site, so tau_theta / N = -(K_u sin 2 theta + (K_c / 2) sin 4 theta) as on
    the simple cubic lattice, reduced by O(T) thermal softening."""
    Ku, Kc, T = 0.05, 0.02, 0.01
    for th in (30.0, 60.0):
        R = oracle.constraint_frame(th, 0.0)
        o = oracle.Crystal(kind, (4, 2, 4), J1=1.0, Ku=Ku, Kc=Kc, T=T, seed=8)
        o.set_spins(_uniform(o.N, R[0]))
        o.constrained_sweep(th, 0.0, 300)
        o.constrained_sweep(th, 0.0, 1500, measure=True)
        tau = o.stats()["tqy"]
        t = math.radians(th)
        expect = -(Ku * math.sin(2 * t) + 0.5 * Kc * math.sin(4 * t))
        assert abs(tau / expect - 1) < 0.03, (th, tau, expect)


def test_xtal_constrained_refuses_negative_projection():
    o = oracle.Crystal(oracle.BCC, (2, 2, 2), Ku=0.05, T=0.5)
    o.set_spins(_uniform(o.N, (0.0, 0.0, -1.0)))
    assert o.constrained_sweep(0.0, 0.0, 1) == -5
