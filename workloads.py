"""Seeded synthetic inputs shared by the tests, the oracle runs and bench.py.

This module holds only workload definitions and seeded input generators
(initial spin states, Voronoi grain maps, request traces).  It contains none
of the Monte Carlo method's arithmetic, and neither the oracle nor the CUDA
library imports it: callers build inputs here and hand the same arrays to
both sides.

Site order everywhere is x + Lx (y + Ly z); spins are (N, 3) arrays.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

PERIODIC, OPEN, PINNED = 0, 1, 2


@dataclass
class LatticeSpec:
    dims: tuple
    J: float = 1.0
    Ku: float = 0.0
    axis: tuple = (0.0, 0.0, 1.0)
    Kc: float = 0.0
    H: tuple = (0.0, 0.0, 0.0)
    T: float = 1.0
    seed: int = 0
    bc: tuple = (PERIODIC, PERIODIC, PERIODIC)
    theta0: int = 30
    extra: dict = field(default_factory=dict)

    @property
    def N(self) -> int:
        return int(self.dims[0] * self.dims[1] * self.dims[2])


# --------------------------------------------------------------------------
# The five workloads (reduced units J = 1, k_B = 1).
# --------------------------------------------------------------------------

# --------------------------------------------------------------------------
# FP32-against-oracle precision check of the batched m(T) workload: the 32
# lattices of batched_mt_32 plus two extra 16^3 points near T_C, each run from
# the all +z state for n_eq unmeasured and n_meas measured sweeps (cone
# adaptation in every sweep), over many independent seeds per side.  The
# oracle's seeds and the GPU's seeds are disjoint ranges of the 64-bit key.
# --------------------------------------------------------------------------

PRECISION_SWEEPS = {16: (200, 500), 32: (200, 500), 64: (200, 500), 128: (100, 200)}
PRECISION_ORACLE_SEED0 = 10 ** 6
PRECISION_GPU_SEED0 = 1 << 40


def precision_cases() -> dict:
    """name -> LatticeSpec of the precision check: 'mT_i' for lattice i of
    batched_mt_32, and 'extra_16c_T1.40', 'extra_16c_T1.50' (16^3 at the
    temperatures either side of lattice 28's T = 1.45).  spec.seed is the
    case's index in the seed ranges (precision_seed)."""
    out = {f"mT_{i}": s for i, s in enumerate(batched_mt_32())}
    out["extra_16c_T1.40"] = LatticeSpec(dims=(16, 16, 16), Ku=0.01, T=1.40, seed=40)
    out["extra_16c_T1.50"] = LatticeSpec(dims=(16, 16, 16), Ku=0.01, T=1.50, seed=41)
    return out


def precision_seed(side_seed0: int, spec: LatticeSpec, k: int) -> int:
    """Seed of run k of a precision case on one side (k < 10^5)."""
    return side_seed0 + 100000 * int(spec.seed) + int(k)


def point_16c() -> LatticeSpec:
    """16^3 periodic, FP64, K_u = 0.01 along z, T = 0.5, seed 0, all +z;
    1000 equilibration + 1000 measurement sweeps."""
    return LatticeSpec(dims=(16, 16, 16), Ku=0.01, T=0.5, seed=0)


POINT_16C_SWEEPS = (1000, 1000)


def batched_mt_32() -> list:
    """Batched m(T) sweep: 32 periodic lattices, L = 16, 32, 64, 128 cycled,
    T_i = 0.05 (i + 1), K_u = 0.01 along z, seed i; FP32 spins."""
    sizes = (16, 32, 64, 128)
    return [LatticeSpec(dims=(sizes[i % 4],) * 3, Ku=0.01, T=0.05 * (i + 1), seed=i)
            for i in range(32)]


BATCHED_MT_SWEEPS = (2000, 5000)


def constrained_64c_runs() -> list:
    """Constrained anisotropy runs: 64^3 periodic, K_u = 0.05 along z,
    K_c = 0.02; theta_c in 0..90 (10 steps), phi_c in {0, 45},
    T in {0.2, 0.6, 1.0, 1.3}.  Returns (spec, theta_c, phi_c) tuples."""
    runs = []
    idx = 0
    for T in (0.2, 0.6, 1.0, 1.3):
        for phi in (0.0, 45.0):
            for th in range(0, 91, 10):
                runs.append((LatticeSpec(dims=(64, 64, 64), Ku=0.05, Kc=0.02, T=T, seed=idx), float(th), phi))
                idx += 1
    return runs


CONSTRAINED_64C_SWEEPS = (3000, 5000)


def bloch_wall_1024() -> list:
    """Bloch wall: 1024 x 128 x 128, x pinned (x = 0 at +z, x = 1023 at -z),
    y, z periodic, K_u = 0.05 along z, 8 temperatures 0.1..1.4, seed = index."""
    Ts = np.linspace(0.1, 1.4, 8)
    return [LatticeSpec(dims=(1024, 128, 128), Ku=0.05, T=float(T), seed=i,
                        bc=(PINNED, PERIODIC, PERIODIC)) for i, T in enumerate(Ts)]


BLOCH_WALL_SWEEPS = (2000, 4000)


# --------------------------------------------------------------------------
# Initial states.
# --------------------------------------------------------------------------

def uniform_spins(N: int, direction=(0.0, 0.0, 1.0)) -> np.ndarray:
    d = np.asarray(direction, np.float64)
    d = d / np.linalg.norm(d)
    return np.tile(d, (N, 1))


def random_spins(N: int, seed: int) -> np.ndarray:
    """Directions uniform on the sphere (normalised Gaussians), seeded."""
    rng = np.random.default_rng(seed)
    v = rng.standard_normal((N, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def wall_spins(dims) -> np.ndarray:
    """Step profile along x: +z for x < Lx/2, -z otherwise."""
    Lx, Ly, Lz = dims
    x = np.arange(Lx)
    sz = np.where(x < Lx // 2, 1.0, -1.0)
    S = np.zeros((Lz, Ly, Lx, 3))
    S[..., 2] = sz[None, None, :]
    return S.reshape(-1, 3)


def perturbed_spins(N: int, seed: int, amplitude: float) -> np.ndarray:
    """+z with a seeded random tilt of the given amplitude, renormalised."""
    rng = np.random.default_rng(seed)
    v = np.zeros((N, 3))
    v[:, 2] = 1.0
    v += amplitude * rng.standard_normal((N, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


# --------------------------------------------------------------------------
# Granular films: seeded in-plane Voronoi tessellation, columnar grains.
# --------------------------------------------------------------------------

def voronoi_film(Lx: int, Ly: int, Lz: int, mean_diameter: float, seed: int):
    """Grain id per site, a bond mask and per-grain easy axes.

    Seeds: n = round(Lx Ly / (pi (d/2)^2)) points uniform in the periodic
    Lx x Ly plane; every column (x, y) (centre at x + 1/2, y + 1/2) belongs
    to the nearest seed under the minimum-image distance.  A bond exists
    iff both ends are in the same grain (zero exchange across grain
    boundaries); x and y are periodic, z is open.  Easy axes are uniform on
    the sphere.  Returns (grain_id (N,), bond_mask (N,) uint8, axes (n, 3)).
    Bond bits: 0 = -x, 1 = +x, 2 = -y, 3 = +y, 4 = -z, 5 = +z.
    """
    rng = np.random.default_rng(seed)
    n = max(1, int(round(Lx * Ly / (math.pi * (mean_diameter / 2.0) ** 2))))
    seeds = rng.uniform(0.0, 1.0, (n, 2)) * np.array([Lx, Ly], np.float64)
    axes = rng.standard_normal((n, 3))
    axes /= np.linalg.norm(axes, axis=1, keepdims=True)
    # nearest seed per column under the periodic (minimum-image) metric
    from scipy.spatial import cKDTree
    tree = cKDTree(seeds, boxsize=[float(Lx), float(Ly)])
    gx, gy = np.meshgrid(np.arange(Lx) + 0.5, np.arange(Ly) + 0.5)
    _, owner = tree.query(np.stack([gx.ravel(), gy.ravel()], axis=1))
    owner = owner.reshape(Ly, Lx)
    col = owner  # (Ly, Lx)
    gid = np.broadcast_to(col[None, :, :], (Lz, Ly, Lx)).reshape(-1).astype(np.int32)
    g3 = gid.reshape(Lz, Ly, Lx)
    mask = np.zeros((Lz, Ly, Lx), np.uint8)
    # -x / +x (periodic)
    mask |= ((g3 == np.roll(g3, 1, axis=2)).astype(np.uint8) << 0)
    mask |= ((g3 == np.roll(g3, -1, axis=2)).astype(np.uint8) << 1)
    mask |= ((g3 == np.roll(g3, 1, axis=1)).astype(np.uint8) << 2)
    mask |= ((g3 == np.roll(g3, -1, axis=1)).astype(np.uint8) << 3)
    zlo = np.ones((Lz, Ly, Lx), bool); zlo[0] = False
    zhi = np.ones((Lz, Ly, Lx), bool); zhi[-1] = False
    mask |= (zlo.astype(np.uint8) << 4)
    mask |= (zhi.astype(np.uint8) << 5)
    return gid, mask.reshape(-1), axes


# --------------------------------------------------------------------------
# Serving trace.
# --------------------------------------------------------------------------

def poisson_trace(rate: float, n: int, seed: int = 1):
    """n request arrival times (s) of a Poisson stream with the given rate,
    and per request a job kind and parameters (seeded).  Kinds: 45% m(T)
    point, 45% constrained point, 10% film; cube L uniform in
    {8, 16, 32, 64, 128, 256}; T uniform in (0.05, 1.6)."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, n))
    u = rng.uniform(size=n)
    kinds = np.where(u < 0.45, "mT", np.where(u < 0.90, "constrained", "film"))
    L = rng.choice(np.array([8, 16, 32, 64, 128, 256]), size=n)
    T = rng.uniform(0.05, 1.6, size=n)
    theta_c = rng.choice(np.arange(0, 91, 10), size=n).astype(float)
    return [dict(t=float(t[i]), kind=str(kinds[i]), L=int(L[i]), T=float(T[i]),
                 theta_c=float(theta_c[i]), seed=1000 + i) for i in range(n)]
