"""Serial FP64 CPU oracle (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this package.  The
product library never does, and this package imports nothing from it.

The arithmetic lives in ``oracle.c`` (plain C, FP64, compiled without
fused multiply-add); this module compiles it with gcc and marshals
arguments through ctypes.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

# Observable sums returned by or_stats, in order (26 words).
STAT_FIELDS = (["n"] + [f"m{a}" for a in "xyz"] + [f"m2{a}" for a in "xyz"]
               + [f"mabs{a}" for a in "xyz"] + ["ml", "ml2", "ml4", "e", "e2",
               "e_ex", "e_u", "e_c", "e_z"] + [f"tq{a}" for a in "xyz"]
               + [f"tq2{a}" for a in "xyz"])
SAMPLE_WORDS = 14

PERIODIC, OPEN, PINNED, ANTIPERIODIC = 0, 1, 2, 3


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so next to it (gcc, no FMA contraction)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math",
           "-fPIC", "-shared", "-Wall", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib() -> C.CDLL:
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB)
        vp, i32, u32, i64, u64, dbl = C.c_void_p, C.c_int, C.c_uint32, C.c_int64, C.c_uint64, C.c_double
        P = C.POINTER
        L.or_philox.argtypes = [P(u32), P(u32), P(u32)]
        L.or_exp.argtypes = [dbl]; L.or_exp.restype = dbl
        L.or_exp_array.argtypes = [P(dbl), P(dbl), i64]; L.or_exp_array.restype = None
        L.or_cone_trial.argtypes = [P(dbl), i32, u32, u32, u32, P(u32), P(dbl), P(dbl)]
        L.or_cone_trial.restype = i32
        L.or_create.argtypes = [P(i32), P(i32), dbl, dbl, P(dbl), dbl, P(dbl), dbl, u64, i32, i32, i32]
        L.or_create.restype = vp
        L.or_destroy.argtypes = [vp]
        L.or_set_spins.argtypes = [vp, P(dbl)]
        L.or_get_spins.argtypes = [vp, P(dbl)]
        L.or_set_temperature.argtypes = [vp, dbl]
        L.or_theta.argtypes = [vp]; L.or_theta.restype = i32
        L.or_sweep_count.argtypes = [vp]; L.or_sweep_count.restype = u32
        L.or_last_accepted.argtypes = [vp]; L.or_last_accepted.restype = i64
        L.or_n_mov.argtypes = [vp]; L.or_n_mov.restype = i64
        L.or_set_bonds.argtypes = [vp, P(C.c_uint8)]
        L.or_set_grains.argtypes = [vp, P(C.c_int32), P(dbl), i32]
        L.or_delta_e.argtypes = [vp, i64, P(dbl)]; L.or_delta_e.restype = dbl
        L.or_stats.argtypes = [vp, P(dbl)]
        L.or_colour_pass_planes.argtypes = [vp, i32, i32, i32]; L.or_colour_pass_planes.restype = i64
        L.or_end_sweep.argtypes = [vp, i64]; L.or_end_sweep.restype = None
        L.or_samples.argtypes = [vp, P(dbl), i64]; L.or_samples.restype = i64
        L.or_anisotropy_scaling.argtypes = [vp, P(dbl)]
        L.or_xtal_create.argtypes = [i32, P(i32), dbl, dbl, dbl, P(dbl), dbl, P(dbl), dbl, u64, i32, i32]
        L.or_xtal_create.restype = vp
        L.or_xtal_destroy.argtypes = [vp]
        L.or_xtal_set_spins.argtypes = [vp, P(dbl)]
        L.or_xtal_get_spins.argtypes = [vp, P(dbl)]
        L.or_xtal_theta.argtypes = [vp]; L.or_xtal_theta.restype = i32
        L.or_xtal_last_accepted.argtypes = [vp]; L.or_xtal_last_accepted.restype = i64
        L.or_xtal_delta_e.argtypes = [vp, i64, P(dbl)]; L.or_xtal_delta_e.restype = dbl
        L.or_xtal_sweep.argtypes = [vp, i32, i32]
        L.or_xtal_stats.argtypes = [vp, P(dbl)]
        L.or_xtal_constrained_sweep.argtypes = [vp, dbl, dbl, i32, i32]
        L.or_xtal_constrained_sweep.restype = i32
        L.or_profile.argtypes = [vp, P(dbl)]
        L.or_reset_stats.argtypes = [vp]
        L.or_sweep.argtypes = [vp, i32, i32]; L.or_sweep.restype = i32
        L.or_sweep_serial.argtypes = [vp, i32, i32]; L.or_sweep_serial.restype = i32
        L.or_fixed_sum.argtypes = [P(dbl), i64]; L.or_fixed_sum.restype = dbl
        L.or_constraint_frame.argtypes = [dbl, dbl, P(dbl)]
        L.or_m_long.argtypes = [vp, dbl, dbl]; L.or_m_long.restype = dbl
        L.or_permutation.argtypes = [u32, u32, i32, P(u32), P(u32)]
        L.or_constrained_sweep.argtypes = [vp, dbl, dbl, i32, i32]; L.or_constrained_sweep.restype = i32
        L.or_constrained_sweep_serial.argtypes = [vp, dbl, dbl, i32, i32]
        L.or_constrained_sweep_serial.restype = i32
        _lib = L
    return _lib


def _p(a: np.ndarray, ct):
    return a.ctypes.data_as(C.POINTER(ct))


def philox(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, np.uint32)
    lib().or_philox(_p(c, C.c_uint32), _p(k, C.c_uint32), _p(out, C.c_uint32))
    return out


def exp(x: float) -> float:
    return lib().or_exp(float(x))


def exp_array(xs) -> np.ndarray:
    """exp_own elementwise over an array (float64)."""
    x = np.ascontiguousarray(xs, dtype=np.float64)
    y = np.empty_like(x)
    lib().or_exp_array(_p(x, C.c_double), _p(y, C.c_double), x.size)
    return y


def cone_trial(S, theta_deg: int, idx: int, sweep: int, tag: int, key):
    s = np.ascontiguousarray(S, dtype=np.float64)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(3)
    P = C.c_double()
    ok = lib().or_cone_trial(_p(s, C.c_double), int(theta_deg), idx, sweep, tag,
                             _p(k, C.c_uint32), _p(out, C.c_double), C.byref(P))
    return bool(ok), out, P.value


def fixed_sum(t) -> float:
    a = np.ascontiguousarray(t, dtype=np.float64)
    return lib().or_fixed_sum(_p(a, C.c_double), a.size)


def grain_magnetization(spins, grain_id, n_grains: int) -> np.ndarray:
    """Magnetisation length of every grain of a film (Sec. 4: each grain
    contributes its own Bloch term to Eq. 8): m_g = |sum_{i in g} S_i| / N_g,
    from (N, 3) spins and the per-site grain ids (site order)."""
    S = np.asarray(spins, np.float64).reshape(-1, 3)
    g = np.asarray(grain_id).reshape(-1)
    M = np.stack([np.bincount(g, weights=S[:, a], minlength=n_grains) for a in range(3)], axis=1)
    N = np.bincount(g, minlength=n_grains)
    return np.linalg.norm(M, axis=1) / np.maximum(N, 1)


def constraint_frame(theta_deg: float, phi_deg: float) -> np.ndarray:
    R = np.zeros(9)
    lib().or_constraint_frame(float(theta_deg), float(phi_deg), _p(R, C.c_double))
    return R.reshape(3, 3)


def permutation(n: int, sweep: int, colour: int, key) -> np.ndarray:
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(n, np.uint32)
    lib().or_permutation(n, sweep, colour, _p(k, C.c_uint32), _p(out, C.c_uint32))
    return out


class Lattice:
    """One lattice of the serial oracle.  Spins are (N, 3) FP64 in site order
    x + Lx (y + Ly z).  bc per axis: 0 periodic, 1 open, 2 pinned."""

    def __init__(self, dims, J=1.0, Ku=0.0, axis=(0.0, 0.0, 1.0), Kc=0.0, H=(0.0, 0.0, 0.0),
                 T=1.0, seed=0, bc=(0, 0, 0), theta0=30, adapt_in_measure=1, ring_cap=1):
        self.dims = tuple(int(d) for d in dims)
        self.N = self.dims[0] * self.dims[1] * self.dims[2]
        self.ring_cap = max(1, int(ring_cap))
        d = np.array(self.dims, np.int32)
        b = np.array(bc, np.int32)
        ax = np.array(axis, np.float64)
        h = np.array(H, np.float64)
        self._h = lib().or_create(_p(d, C.c_int), _p(b, C.c_int), float(J), float(Ku),
                                  _p(ax, C.c_double), float(Kc), _p(h, C.c_double), float(T),
                                  int(seed) & (2**64 - 1), int(theta0), int(adapt_in_measure),
                                  int(ring_cap))
        if not self._h:
            raise MemoryError("or_create failed")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and _lib is not None:
            _lib.or_destroy(h)
            self._h = None

    # state -------------------------------------------------------------
    def set_spins(self, S: np.ndarray) -> None:
        a = np.ascontiguousarray(S, dtype=np.float64).reshape(self.N, 3)
        lib().or_set_spins(self._h, _p(a, C.c_double))

    def spins(self) -> np.ndarray:
        out = np.zeros((self.N, 3))
        lib().or_get_spins(self._h, _p(out, C.c_double))
        return out

    def set_temperature(self, T: float) -> None:
        lib().or_set_temperature(self._h, float(T))

    def set_bonds(self, mask: np.ndarray) -> None:
        self._bonds = np.ascontiguousarray(mask, dtype=np.uint8).reshape(self.N)
        lib().or_set_bonds(self._h, _p(self._bonds, C.c_uint8))

    def set_grains(self, gid: np.ndarray, axes: np.ndarray) -> None:
        g = np.ascontiguousarray(gid, dtype=np.int32).reshape(self.N)
        a = np.ascontiguousarray(axes, dtype=np.float64).reshape(-1, 3)
        lib().or_set_grains(self._h, _p(g, C.c_int32), _p(a, C.c_double), a.shape[0])

    @property
    def theta(self) -> int:
        return lib().or_theta(self._h)

    @property
    def sweep_count(self) -> int:
        return lib().or_sweep_count(self._h)

    @property
    def last_accepted(self) -> int:
        return lib().or_last_accepted(self._h)

    @property
    def n_mov(self) -> int:
        return lib().or_n_mov(self._h)

    # method ------------------------------------------------------------
    def sweep(self, n: int, measure: bool = False) -> None:
        lib().or_sweep(self._h, int(n), int(bool(measure)))

    def colour_pass_planes(self, colour: int, z0: int, z1: int) -> int:
        """One Table A1 colour pass over the planes z0 <= z < z1 only (a
        slab's share of the pass); returns the accepted moves."""
        n = lib().or_colour_pass_planes(self._h, int(colour), int(z0), int(z1))
        if n < 0:
            raise ValueError("or_colour_pass_planes: bad colour or plane range")
        return int(n)

    def end_sweep(self, accepted: int) -> None:
        """End an unmeasured iteration with the whole lattice's accepted
        moves: cone adaptation and the sweep counter."""
        lib().or_end_sweep(self._h, int(accepted))

    def sweep_serial(self, n: int, measure: bool = False) -> None:
        lib().or_sweep_serial(self._h, int(n), int(bool(measure)))

    def constrained_sweep(self, theta_c: float, phi_c: float, n: int, measure: bool = False) -> None:
        rc = lib().or_constrained_sweep(self._h, float(theta_c), float(phi_c), int(n), int(bool(measure)))
        if rc != 0:
            raise RuntimeError(f"or_constrained_sweep returned {rc}")

    def constrained_sweep_serial(self, theta_c: float, phi_c: float, n: int, measure: bool = False) -> None:
        rc = lib().or_constrained_sweep_serial(self._h, float(theta_c), float(phi_c), int(n), int(bool(measure)))
        if rc != 0:
            raise RuntimeError(f"or_constrained_sweep_serial returned {rc}")

    def delta_e(self, i: int, Sn) -> float:
        s = np.ascontiguousarray(Sn, dtype=np.float64)
        return lib().or_delta_e(self._h, int(i), _p(s, C.c_double))

    def m_long(self, theta_c: float, phi_c: float) -> float:
        return lib().or_m_long(self._h, float(theta_c), float(phi_c))

    # measurements ------------------------------------------------------
    def stats(self) -> dict:
        out = np.zeros(len(STAT_FIELDS))
        lib().or_stats(self._h, _p(out, C.c_double))
        return dict(zip(STAT_FIELDS, out.tolist()))

    def anisotropy_scaling(self) -> np.ndarray:
        """(k_u, k_c) of Eq. 4 from the mean anisotropy energies (NaN where
        the constant is zero or nothing was sampled)."""
        out = np.zeros(2)
        lib().or_anisotropy_scaling(self._h, _p(out, C.c_double))
        return out

    def samples(self, max_n: int | None = None) -> np.ndarray:
        """The most recent min(max_n, kept) per-sweep samples, oldest first."""
        if max_n is None:
            max_n = self.ring_cap
        out = np.zeros((max_n, SAMPLE_WORDS))
        n = lib().or_samples(self._h, _p(out, C.c_double), max_n)
        return out[:n]

    def profile(self) -> np.ndarray:
        out = np.zeros(self.dims[0])
        lib().or_profile(self._h, _p(out, C.c_double))
        return out

    def reset_stats(self) -> None:
        lib().or_reset_stats(self._h)


BCC, FCC, HCP = 1, 2, 3
XTAL_STAT_FIELDS = ("n", "mx", "my", "mz", "ml", "e", "e_ex", "e_u", "e_c", "e_z", "tqx", "tqy", "tqz")


class Crystal:
    """A bcc (kind 1), fcc (kind 2) or hcp (kind 3, orthohexagonal cells)
    lattice of the serial oracle: cells (Lx, Ly, Lz), all periodic; site i =
    s + nsub (x + Lx (y + Ly z)) for sub-lattice s of cell (x, y, z).  J1
    nearest, J2 next-nearest exchange (bcc, fcc)."""

    def __init__(self, kind, cells, J1=1.0, J2=0.0, Ku=0.0, axis=(0.0, 0.0, 1.0), Kc=0.0, H=(0.0, 0.0, 0.0),
                 T=1.0, seed=0, theta0=30, adapt_in_measure=1):
        self.kind = int(kind)
        self.cells = tuple(int(c) for c in cells)
        self.nsub = 2 if self.kind == BCC else 4
        self.N = self.nsub * self.cells[0] * self.cells[1] * self.cells[2]
        d = np.array(self.cells, np.int32)
        ax = np.array(axis, np.float64)
        h = np.array(H, np.float64)
        self._h = lib().or_xtal_create(self.kind, _p(d, C.c_int), float(J1), float(J2), float(Ku),
                                       _p(ax, C.c_double), float(Kc), _p(h, C.c_double), float(T),
                                       int(seed) & (2**64 - 1), int(theta0), int(adapt_in_measure))
        if not self._h:
            raise ValueError("or_xtal_create failed")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and _lib is not None:
            _lib.or_xtal_destroy(h)
            self._h = None

    def set_spins(self, S: np.ndarray) -> None:
        a = np.ascontiguousarray(S, dtype=np.float64).reshape(self.N, 3)
        lib().or_xtal_set_spins(self._h, _p(a, C.c_double))

    def spins(self) -> np.ndarray:
        out = np.zeros((self.N, 3))
        lib().or_xtal_get_spins(self._h, _p(out, C.c_double))
        return out

    def theta(self) -> int:
        return lib().or_xtal_theta(self._h)

    def last_accepted(self) -> int:
        return lib().or_xtal_last_accepted(self._h)

    def delta_e(self, i: int, Sn) -> float:
        s = np.ascontiguousarray(Sn, dtype=np.float64)
        return lib().or_xtal_delta_e(self._h, int(i), _p(s, C.c_double))

    def sweep(self, n: int, measure: bool = False) -> None:
        lib().or_xtal_sweep(self._h, int(n), int(bool(measure)))

    def constrained_sweep(self, theta_deg: float, phi_deg: float, n: int, measure: bool = False) -> int:
        """Table A2 over the sub-sets (or_xtal_constrained_sweep); -5 if M_L <= 0."""
        return lib().or_xtal_constrained_sweep(self._h, float(theta_deg), float(phi_deg), int(n), int(bool(measure)))

    def stats(self) -> dict:
        out = np.zeros(len(XTAL_STAT_FIELDS))
        lib().or_xtal_stats(self._h, _p(out, C.c_double))
        return dict(zip(XTAL_STAT_FIELDS, out.tolist()))
