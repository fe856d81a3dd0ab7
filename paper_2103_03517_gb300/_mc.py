"""ctypes binding of libmc (include/mc.h): the same entry points under the same
names, argument marshalling only.  Every step of the Monte Carlo path runs in
the CUDA library; if libmc.so is missing or cannot be loaded this module
raises instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmc.so")

MC_OK, MC_PENDING = 0, 1
MC_ERR_ARG, MC_ERR_NOMEM, MC_ERR_CUDA, MC_ERR_TIMEOUT, MC_ERR_CONSTRAINT, MC_ERR_STATE, MC_ERR_IO = (
    -1, -2, -3, -4, -5, -6, -7)
MC_ERR_CANCELLED = -8
MC_FP32, MC_FP64 = 0, 1
MC_PERIODIC, MC_OPEN, MC_PINNED, MC_ANTIPERIODIC = 0, 1, 2, 3
MC_PATH_AUTO, MC_PATH_GENERAL, MC_PATH_ROW, MC_PATH_WAVE, MC_PATH_RESIDENT = 0, 1, 2, 3, 4
MC_SC, MC_BCC, MC_FCC, MC_HCP = 0, 1, 2, 3
MC_INIT_UNIFORM, MC_INIT_WALL = 0, 1
MC_TUNE_SWEEP, MC_TUNE_CONSTRAINED = 1, 2
MC_JOB_SWEEP, MC_JOB_CONSTRAINED = 0, 1


class MCError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"libmc error {code}: {msg}")
        self.code = code


class mc_desc(C.Structure):
    _fields_ = [("dims", C.c_int * 3), ("boundary", C.c_int * 3), ("precision", C.c_int),
                ("J", C.c_double), ("K_u", C.c_double), ("axis", C.c_double * 3), ("K_c", C.c_double),
                ("H", C.c_double * 3), ("T", C.c_double), ("seed", C.c_uint64),
                ("theta0_deg", C.c_int), ("adapt_in_measure", C.c_int), ("init", C.c_int),
                ("init_dir", C.c_double * 3), ("ring_capacity", C.c_int), ("sample_torque", C.c_int),
                ("bond_mask", C.POINTER(C.c_uint8)), ("grain_id", C.POINTER(C.c_int32)),
                ("grain_axis", C.POINTER(C.c_double)), ("n_grains", C.c_int),
                ("stream", C.c_void_p), ("device", C.c_int), ("kernel_path", C.c_int), ("lattice", C.c_int),
                ("J2", C.c_double)]


class mc_observables(C.Structure):
    _fields_ = [("n_samples", C.c_int64), ("sweeps_done", C.c_int64), ("theta_deg", C.c_int),
                ("error", C.c_int), ("accept_last", C.c_double), ("m", C.c_double * 3),
                ("m2", C.c_double * 3), ("m_abs", C.c_double * 3), ("ml", C.c_double), ("ml2", C.c_double),
                ("ml4", C.c_double), ("e", C.c_double), ("e2", C.c_double), ("e_parts", C.c_double * 4),
                ("torque", C.c_double * 3), ("torque2", C.c_double * 3), ("chi", C.c_double * 4),
                ("binder", C.c_double)]

    def asdict(self) -> dict:
        out = {}
        for name, _ in self._fields_:
            v = getattr(self, name)
            out[name] = list(v) if hasattr(v, "__len__") else v
        return out


class mc_tune_report(C.Structure):
    _fields_ = [("row", C.c_int), ("field", C.c_int), ("pair", C.c_int), ("pad", C.c_int),
                ("row_ms", C.c_double * 4), ("field_ms", C.c_double * 4), ("pair_ms", C.c_double * 4)]

    def asdict(self):
        return {"row": self.row, "field": self.field, "pair": self.pair, "row_ms": list(self.row_ms),
                "field_ms": list(self.field_ms), "pair_ms": list(self.pair_ms)}


class mc_sample(C.Structure):
    _fields_ = [("sweep", C.c_int64), ("theta_deg", C.c_int32), ("pad", C.c_int32), ("accepted", C.c_int64),
                ("m", C.c_double * 3), ("e_parts", C.c_double * 4), ("torque", C.c_double * 3)]


class mc_server_desc(C.Structure):
    _fields_ = [("device", C.c_int), ("memory_budget", C.c_size_t), ("max_resident", C.c_int),
                ("max_epoch_sweeps", C.c_int)]


class mc_job(C.Structure):
    _fields_ = [("lattice", mc_desc), ("kind", C.c_int), ("theta_c_deg", C.c_double), ("phi_c_deg", C.c_double),
                ("n_equilibrate", C.c_int), ("n_measure", C.c_int)]


class mc_result(C.Structure):
    _fields_ = [("obs", mc_observables), ("t_submit", C.c_double), ("t_admit", C.c_double),
                ("t_finish", C.c_double), ("status", C.c_int)]


# every entry point of include/mc.h: name -> (restype, argtypes)
_P = C.POINTER
_SIGS = {
    "mc_desc_default": (None, [_P(mc_desc)]),
    "mc_create": (C.c_int, [_P(C.c_int), C.c_double, C.c_double, _P(C.c_double), C.c_double, _P(C.c_double),
                            C.c_double, C.c_uint64, _P(C.c_void_p)]),
    "mc_create_ex": (C.c_int, [_P(mc_desc), _P(C.c_void_p)]),
    "mc_destroy": (C.c_int, [C.c_void_p]),
    "mc_set_temperature": (C.c_int, [C.c_void_p, C.c_double]),
    "mc_set_field": (C.c_int, [C.c_void_p, _P(C.c_double)]),
    "mc_sweep": (C.c_int, [C.c_void_p, C.c_int, C.c_int]),
    "mc_constrained_sweep": (C.c_int, [C.c_void_p, C.c_double, C.c_double, C.c_int, C.c_int]),
    "mc_sync": (C.c_int, [C.c_void_p]),
    "mc_measure": (C.c_int, [C.c_void_p, _P(mc_observables)]),
    "mc_anisotropy_scaling": (C.c_int, [C.c_void_p, _P(C.c_double)]),
    "mc_profile": (C.c_int, [C.c_void_p, C.c_int, _P(C.c_double), C.c_int]),
    "mc_profile_sample": (C.c_int, [C.c_void_p]),
    "mc_grain_sample": (C.c_int, [C.c_void_p]),
    "mc_grain_magnetization": (C.c_int, [C.c_void_p, _P(C.c_double), C.c_int, _P(C.c_int64)]),
    "mc_samples": (C.c_int, [C.c_void_p, _P(mc_sample), C.c_int, _P(C.c_int)]),
    "mc_reset_stats": (C.c_int, [C.c_void_p]),
    "mc_get_spins": (C.c_int, [C.c_void_p, _P(C.c_double), C.c_size_t]),
    "mc_set_spins": (C.c_int, [C.c_void_p, _P(C.c_double), C.c_size_t]),
    "mc_state_bytes": (C.c_size_t, [C.c_void_p]),
    "mc_export_state": (C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t]),
    "mc_import_state": (C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t]),
    "mc_get_theta": (C.c_int, [C.c_void_p, _P(C.c_int), _P(C.c_int64)]),
    "mc_save": (C.c_int, [C.c_void_p, C.c_char_p]),
    "mc_load": (C.c_int, [C.c_char_p, _P(C.c_void_p)]),
    "mc_group_create": (C.c_int, [_P(C.c_void_p), C.c_int, _P(C.c_void_p)]),
    "mc_group_destroy": (C.c_int, [C.c_void_p]),
    "mc_group_sweep": (C.c_int, [C.c_void_p, C.c_int, C.c_int]),
    "mc_group_constrained_sweep": (C.c_int, [C.c_void_p, _P(C.c_double), _P(C.c_double), C.c_int, C.c_int]),
    "mc_group_time_passes": (C.c_int, [C.c_void_p, C.c_int, C.c_int, _P(C.c_double), _P(C.c_int)]),
    "mc_group_time_kernels": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_int, _P(C.c_double), _P(C.c_int)]),
    "mc_group_measure": (C.c_int, [C.c_void_p, _P(mc_observables), C.c_int]),
    "mc_group_sync": (C.c_int, [C.c_void_p]),
    "mc_group_autotune": (C.c_int, [C.c_void_p, C.c_int, C.c_int, _P(mc_tune_report)]),
    "mc_autotune": (C.c_int, [C.c_void_p, C.c_int, C.c_int, _P(mc_tune_report)]),
    "mc_group_set_shapes": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_int]),
    "mc_server_create": (C.c_int, [_P(mc_server_desc), _P(C.c_void_p)]),
    "mc_server_destroy": (C.c_int, [C.c_void_p]),
    "mc_submit": (C.c_int, [C.c_void_p, _P(mc_job), _P(C.c_uint64)]),
    "mc_poll": (C.c_int, [C.c_void_p, C.c_uint64, _P(mc_result)]),
    "mc_cancel": (C.c_int, [C.c_void_p, C.c_uint64]),
    "mc_forget": (C.c_int, [C.c_void_p, C.c_uint64]),
    "mc_server_stats": (C.c_int, [C.c_void_p, _P(C.c_double), _P(C.c_int), _P(C.c_int), _P(C.c_size_t)]),
    "mc_slab_create": (C.c_int, [_P(mc_desc), C.c_int, C.c_int, _P(C.c_void_p)]),
    "mc_slab_info": (C.c_int, [C.c_void_p, _P(C.c_int), _P(C.c_int), _P(C.c_int)]),
    "mc_slab_pass": (C.c_int, [C.c_void_p, C.c_int, C.c_int]),
    "mc_slab_plane": (C.c_int, [C.c_void_p, C.c_int, C.c_int, _P(C.c_void_p), _P(C.c_size_t)]),
    "mc_slab_export": (C.c_int, [C.c_void_p, _P(C.c_void_p)]),
    "mc_slab_close": (C.c_int, [C.c_void_p, C.c_int]),
    "mc_slab_sweep": (C.c_int, [_P(C.c_void_p), C.c_int, C.c_int, C.c_int]),
    "mc_sweep_noalloc": (C.c_int, [C.c_void_p, _P(C.c_int), C.c_double, C.c_double, _P(C.c_double), C.c_double,
                                   _P(C.c_double), C.c_double, C.c_uint64, C.c_int64, C.c_int, _P(C.c_int),
                                   C.c_void_p, C.c_void_p]),
    "mc_last_error": (C.c_char_p, []),
    "mc_version": (C.c_char_p, []),
}

_lib = None


def lib() -> C.CDLL:
    """Load libmc.so (built by build.py / __graft_entry__.build()); raise if absent."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libmc.so not found at {LIB_PATH}: build it with "
                              "`python -c 'import __graft_entry__ as g; g.build()'`")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(rc: int) -> int:
    if rc < 0:
        raise MCError(rc, lib().mc_last_error().decode(errors="replace"))
    return rc


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _vec3(v):
    return (C.c_double * 3)(*[float(x) for x in v])


# ------------------------------------------------------------------ lattice
def mc_desc_default() -> mc_desc:
    d = mc_desc()
    lib().mc_desc_default(C.byref(d))
    return d


def make_desc(dims, J=1.0, K_u=0.0, axis=(0.0, 0.0, 1.0), K_c=0.0, H=(0.0, 0.0, 0.0), T=1.0, seed=0,
              precision=MC_FP32, boundary=(0, 0, 0), theta0_deg=30, adapt_in_measure=1, init=MC_INIT_UNIFORM,
              init_dir=(0.0, 0.0, 1.0), ring_capacity=4096, sample_torque=1, bond_mask=None, grain_id=None,
              grain_axis=None,
              stream=None, device=0, kernel_path=0, lattice=0, J2=0.0) -> mc_desc:
    """Fill an mc_desc.  Film tables (numpy arrays) are referenced, not
    copied, until mc_create_ex / mc_submit copies them; keep them alive."""
    d = mc_desc_default()
    for a in range(3):
        d.dims[a] = int(dims[a])
        d.boundary[a] = int(boundary[a])
        d.axis[a] = float(axis[a])
        d.H[a] = float(H[a])
        d.init_dir[a] = float(init_dir[a])
    d.precision = int(precision)
    d.J, d.K_u, d.K_c, d.T = float(J), float(K_u), float(K_c), float(T)
    d.seed = int(seed) & (2 ** 64 - 1)
    d.theta0_deg = int(theta0_deg)
    d.adapt_in_measure = int(adapt_in_measure)
    d.init = int(init)
    d.ring_capacity = int(ring_capacity)
    d.kernel_path = int(kernel_path)
    d.lattice = int(lattice)
    d.J2 = float(J2)
    d.sample_torque = int(bool(sample_torque))
    d._keep = []
    if bond_mask is not None:
        bm = np.ascontiguousarray(bond_mask, dtype=np.uint8)
        d._keep.append(bm)
        d.bond_mask = bm.ctypes.data_as(C.POINTER(C.c_uint8))
    if grain_id is not None:
        gi = np.ascontiguousarray(grain_id, dtype=np.int32)
        ga = np.ascontiguousarray(grain_axis, dtype=np.float64).reshape(-1, 3)
        d._keep += [gi, ga]
        d.grain_id = gi.ctypes.data_as(C.POINTER(C.c_int32))
        d.grain_axis = _dp(ga)
        d.n_grains = ga.shape[0]
    d.stream = stream
    d.device = int(device)
    return d


def mc_create(dims, J, K_u, axis, K_c, H, T, seed) -> int:
    h = C.c_void_p()
    d = (C.c_int * 3)(*[int(x) for x in dims])
    _check(lib().mc_create(d, float(J), float(K_u), _vec3(axis), float(K_c), _vec3(H), float(T),
                           int(seed) & (2 ** 64 - 1), C.byref(h)))
    return h.value


def mc_create_ex(desc: mc_desc) -> int:
    h = C.c_void_p()
    _check(lib().mc_create_ex(C.byref(desc), C.byref(h)))
    return h.value


def mc_destroy(h) -> None:
    _check(lib().mc_destroy(h))


def mc_set_temperature(h, T) -> None:
    _check(lib().mc_set_temperature(h, float(T)))


def mc_set_field(h, H) -> None:
    _check(lib().mc_set_field(h, _vec3(H)))


def mc_sweep(h, n_sweeps: int, measure: bool = False) -> None:
    _check(lib().mc_sweep(h, int(n_sweeps), int(bool(measure))))


def mc_constrained_sweep(h, theta_c_deg, phi_c_deg, n_sweeps: int, measure: bool = False) -> None:
    _check(lib().mc_constrained_sweep(h, float(theta_c_deg), float(phi_c_deg), int(n_sweeps), int(bool(measure))))


def mc_sync(h) -> None:
    _check(lib().mc_sync(h))


def mc_measure(h) -> mc_observables:
    o = mc_observables()
    _check(lib().mc_measure(h, C.byref(o)))
    return o


def mc_anisotropy_scaling(h) -> np.ndarray:
    """(k_u, k_c) of Eq. 4 from the samples since the last reset."""
    out = np.zeros(2)
    _check(lib().mc_anisotropy_scaling(h, _dp(out)))
    return out


def mc_profile_sample(h) -> None:
    _check(lib().mc_profile_sample(h))


def mc_profile(h, component: int, Lx: int) -> np.ndarray:
    out = np.zeros(Lx)
    _check(lib().mc_profile(h, int(component), _dp(out), Lx))
    return out


def mc_grain_sample(h) -> None:
    _check(lib().mc_grain_sample(h))


def mc_grain_magnetization(h, n_grains: int):
    """(<m_g> per grain as a numpy array, number of grain samples)."""
    out = np.zeros(int(n_grains))
    n = C.c_int64()
    _check(lib().mc_grain_magnetization(h, _dp(out), int(n_grains), C.byref(n)))
    return out, n.value


def mc_samples(h, max_n: int) -> np.ndarray:
    """Per-sweep samples as a structured numpy array (fields of mc_sample)."""
    buf = (mc_sample * max_n)()
    n = C.c_int()
    _check(lib().mc_samples(h, buf, int(max_n), C.byref(n)))
    arr = np.ctypeslib.as_array(buf)[: n.value].copy()
    return arr


def mc_reset_stats(h) -> None:
    _check(lib().mc_reset_stats(h))


def mc_get_spins(h, N: int) -> np.ndarray:
    out = np.zeros((N, 3))
    _check(lib().mc_get_spins(h, _dp(out), N))
    return out


def mc_set_spins(h, xyz: np.ndarray) -> None:
    a = np.ascontiguousarray(xyz, dtype=np.float64).reshape(-1, 3)
    _check(lib().mc_set_spins(h, _dp(a), a.shape[0]))


def mc_state_bytes(h) -> int:
    return int(lib().mc_state_bytes(h))


def mc_export_state(h, host_ptr: int, nbytes: int) -> None:
    _check(lib().mc_export_state(h, C.c_void_p(host_ptr), nbytes))


def mc_import_state(h, host_ptr: int, nbytes: int) -> None:
    _check(lib().mc_import_state(h, C.c_void_p(host_ptr), nbytes))


def mc_get_theta(h):
    t = C.c_int()
    s = C.c_int64()
    _check(lib().mc_get_theta(h, C.byref(t), C.byref(s)))
    return t.value, s.value


def mc_save(h, path: str) -> None:
    _check(lib().mc_save(h, path.encode()))


def mc_load(path: str) -> int:
    h = C.c_void_p()
    _check(lib().mc_load(path.encode(), C.byref(h)))
    return h.value


# ---------------------------------------------------------------- batching
def mc_group_create(handles) -> int:
    arr = (C.c_void_p * len(handles))(*handles)
    g = C.c_void_p()
    _check(lib().mc_group_create(arr, len(handles), C.byref(g)))
    return g.value


def mc_group_destroy(g) -> None:
    _check(lib().mc_group_destroy(g))


def mc_group_sweep(g, n_sweeps: int, measure: bool = False) -> None:
    _check(lib().mc_group_sweep(g, int(n_sweeps), int(bool(measure))))


def mc_group_constrained_sweep(g, theta_c_deg, phi_c_deg, n_sweeps: int, measure: bool = False) -> None:
    th = np.ascontiguousarray(theta_c_deg, dtype=np.float64)
    ph = np.ascontiguousarray(phi_c_deg, dtype=np.float64)
    _check(lib().mc_group_constrained_sweep(g, _dp(th), _dp(ph), int(n_sweeps), int(bool(measure))))


def mc_group_set_shapes(g, row: int = 0, field: int = 0, pair: int = 0) -> None:
    """Launch shapes of the group's kernels by candidate index (see mc_group_autotune)."""
    _check(lib().mc_group_set_shapes(g, int(row), int(field), int(pair)))


def mc_group_autotune(g, sweeps: int = 4, what: int = MC_TUNE_SWEEP | MC_TUNE_CONSTRAINED) -> dict:
    """Autotune the group's launch shapes (chains unchanged); returns the report."""
    r = mc_tune_report()
    _check(lib().mc_group_autotune(g, int(sweeps), int(what), C.byref(r)))
    return r.asdict()


def mc_autotune(h, sweeps: int = 4, what: int = MC_TUNE_SWEEP | MC_TUNE_CONSTRAINED) -> dict:
    """Autotune the launch shapes of one lattice swept alone; returns the report."""
    r = mc_tune_report()
    _check(lib().mc_autotune(h, int(sweeps), int(what), C.byref(r)))
    return r.asdict()


def mc_group_time_passes(g, n_sweeps: int, measure: bool = False):
    avg = C.c_double()
    n = C.c_int()
    _check(lib().mc_group_time_passes(g, int(n_sweeps), int(bool(measure)), C.byref(avg), C.byref(n)))
    return avg.value, n.value


def mc_group_time_kernels(g, n_sweeps: int, measure: bool = False, constrained: bool = False):
    """Per launch kind (wavefront sweeps, colour passes, pair passes,
    resident launches of up to 2048 sweeps): the mean launch duration in ms
    and the number of launches timed."""
    ms = (C.c_double * 4)()
    n = (C.c_int * 4)()
    _check(lib().mc_group_time_kernels(g, int(n_sweeps), int(bool(measure)), int(bool(constrained)), ms, n))
    return list(ms), list(n)


def mc_group_measure(g, n: int) -> list:
    """Observables of the group's n lattices (creation order), one wait."""
    arr = (mc_observables * int(n))()
    _check(lib().mc_group_measure(g, arr, int(n)))
    return list(arr)


def mc_group_sync(g) -> None:
    _check(lib().mc_group_sync(g))


# ----------------------------------------------------------------- serving
def mc_server_create(device=0, memory_budget=0, max_resident=256, max_epoch_sweeps=50) -> int:
    d = mc_server_desc(int(device), int(memory_budget), int(max_resident), int(max_epoch_sweeps))
    s = C.c_void_p()
    _check(lib().mc_server_create(C.byref(d), C.byref(s)))
    return s.value


def mc_server_destroy(s) -> None:
    _check(lib().mc_server_destroy(s))


def make_job(desc: mc_desc, kind=MC_JOB_SWEEP, theta_c_deg=0.0, phi_c_deg=0.0, n_equilibrate=0,
             n_measure=0) -> mc_job:
    j = mc_job()
    j.lattice = desc
    j.kind = int(kind)
    j.theta_c_deg = float(theta_c_deg)
    j.phi_c_deg = float(phi_c_deg)
    j.n_equilibrate = int(n_equilibrate)
    j.n_measure = int(n_measure)
    j._keep = getattr(desc, "_keep", [])
    return j


def mc_submit(s, job: mc_job) -> int:
    jid = C.c_uint64()
    _check(lib().mc_submit(s, C.byref(job), C.byref(jid)))
    return jid.value


def mc_poll(s, job_id: int):
    """(status, mc_result or None): status MC_PENDING or MC_OK."""
    r = mc_result()
    rc = _check(lib().mc_poll(s, int(job_id), C.byref(r)))
    return rc, (r if rc == MC_OK else None)


def mc_cancel(s, job_id: int) -> None:
    """Cancel a queued or resident job (its result then reads MC_ERR_CANCELLED)."""
    _check(lib().mc_cancel(s, int(job_id)))


MC_SLAB_WORDS = 16


def mc_slab_create(desc: mc_desc, z0: int, nz: int) -> int:
    """Slab of global planes [z0, z0 + nz) of the lattice desc describes,
    with one halo plane each side (Lx x Ly x (nz + 2) local sites)."""
    h = C.c_void_p()
    _check(lib().mc_slab_create(C.byref(desc), int(z0), int(nz), C.byref(h)))
    return h.value


def mc_slab_info(h):
    z0, nz, Lz = C.c_int(), C.c_int(), C.c_int()
    _check(lib().mc_slab_info(h, C.byref(z0), C.byref(nz), C.byref(Lz)))
    return z0.value, nz.value, Lz.value


def mc_slab_pass(h, colour: int, measure: bool = False) -> None:
    _check(lib().mc_slab_pass(h, int(colour), int(bool(measure))))


def mc_slab_plane(h, colour: int, which: int):
    """((x, y, z) component device addresses, sites) of one plane: which = 0
    first own, 1 last own, 2 lower halo, 3 upper halo."""
    ptrs = (C.c_void_p * 3)()
    n = C.c_size_t()
    _check(lib().mc_slab_plane(h, int(colour), int(which), ptrs, C.byref(n)))
    return tuple(int(p) for p in ptrs), n.value


def mc_slab_export(h) -> int:
    """Queue the export of the sweep's counts; returns the device address of
    the MC_SLAB_WORDS int64 words."""
    p = C.c_void_p()
    _check(lib().mc_slab_export(h, C.byref(p)))
    return int(p.value)


def mc_slab_close(h, measure: bool = False) -> None:
    _check(lib().mc_slab_close(h, int(bool(measure))))


def mc_slab_sweep(slabs, n_sweeps: int, measure: bool = False) -> None:
    """Sweeps of the slabs of one lattice held on one device and stream."""
    arr = (C.c_void_p * len(slabs))(*slabs)
    _check(lib().mc_slab_sweep(arr, len(slabs), int(n_sweeps), int(bool(measure))))


def mc_forget(s, job_id: int) -> None:
    """Drop a finished job's record (poll its result first)."""
    _check(lib().mc_forget(s, int(job_id)))


def mc_server_stats(s):
    now = C.c_double()
    q = C.c_int()
    r = C.c_int()
    b = C.c_size_t()
    _check(lib().mc_server_stats(s, C.byref(now), C.byref(q), C.byref(r), C.byref(b)))
    return now.value, q.value, r.value, b.value


# ------------------------------------------------------------ no allocation
def mc_sweep_noalloc(spins_ptr: int, dims, J, K_u, axis, K_c, H, T, seed, first_sweep: int, n_sweeps: int,
                     theta_deg: int, samples_ptr: int | None = None, stream: int | None = None) -> int:
    """FP32 sweeps on caller-owned device spins (colour-split layout) without
    any device allocation; returns the cone angle after the sweeps."""
    d = (C.c_int * 3)(*[int(x) for x in dims])
    th = C.c_int(int(theta_deg))
    _check(lib().mc_sweep_noalloc(C.c_void_p(spins_ptr), d, float(J), float(K_u), _vec3(axis), float(K_c), _vec3(H),
                                  float(T), int(seed) & (2 ** 64 - 1), int(first_sweep), int(n_sweeps), C.byref(th),
                                  C.c_void_p(samples_ptr) if samples_ptr else None,
                                  C.c_void_p(stream) if stream else None))
    return th.value


def mc_last_error() -> str:
    return lib().mc_last_error().decode(errors="replace")


def mc_version() -> str:
    return lib().mc_version().decode()
