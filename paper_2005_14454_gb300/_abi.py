"""ctypes binding of the engine's C ABI (include/ahs.h), with the same names.

Argument marshalling only: every step of the evolution and of the diagnostics
runs in the CUDA kernels of ``_ahs.so``.  Importing this module loads the shared
library and fails loudly if it has not been built; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_ahs.so")

AHS_OK, AHS_EINVAL, AHS_ENOMEM, AHS_ECUDA, AHS_ESTATE, AHS_ENONFINITE, AHS_ETIMEOUT = 0, -1, -2, -3, -4, -5, -6
AHS_MINKOWSKI, AHS_RADIATION, AHS_MATTER = 0, 1, 2
AHS_FIELD_PHI, AHS_FIELD_PI, AHS_FIELD_THETA, AHS_FIELD_E, AHS_FIELD_ALL, AHS_FIELD_LOW = 0, 1, 2, 3, 4, 5
FIELD_PLANES = {AHS_FIELD_PHI: 2, AHS_FIELD_PI: 2, AHS_FIELD_THETA: 3, AHS_FIELD_E: 3, AHS_FIELD_ALL: 10,
                AHS_FIELD_LOW: 5}
AHS_PREC_FP32, AHS_PREC_FP32_COMPENSATED, AHS_PREC_FP64 = 0, 1, 2
(AHS_OPT_MEASURE_EVERY, AHS_OPT_ALPHA, AHS_OPT_TAU0, AHS_OPT_STEP, AHS_OPT_WRAP_THETA,
 AHS_OPT_PROFILE, AHS_OPT_N, AHS_OPT_TILE_Y, AHS_OPT_ZCHUNK, AHS_OPT_GRAPH, AHS_OPT_PRECISION,
 AHS_OPT_COOLING, AHS_OPT_MOMENTA_IN_PLACE, AHS_OPT_CORE_GROWTH_S, AHS_OPT_CORE_GROWTH_TAU,
 AHS_OPT_STEPS_PER_PASS, AHS_OPT_MEASURE_TILE_Y) = range(17)
AHS_KERNEL_STEP, AHS_KERNEL_STEP_MEASURE, AHS_KERNEL_STEP_PAIR = 0, 1, 2

# every symbol include/ahs.h declares
EXPORTS = (
    "ahs_create", "ahs_init", "ahs_step", "ahs_measure", "ahs_records", "ahs_fields",
    "ahs_set_fields", "ahs_fields_box", "ahs_windings", "ahs_set_option", "ahs_get_option",
    "ahs_set_stream", "ahs_kernel_time", "ahs_device_bytes", "ahs_destroy", "ahs_last_error",
    "ahs_last_error_message", "ahs_strerror", "ahs_sizeof_obs", "ahs_measure_noalloc", "ahs_autotune",
    "ahs_batch_create", "ahs_batch_init", "ahs_batch_run", "ahs_batch_records", "ahs_batch_fields",
    "ahs_batch_set_fields", "ahs_batch_step_info", "ahs_batch_set_option", "ahs_batch_get_option",
    "ahs_batch_member_zchunk", "ahs_batch_autotune", "ahs_batch_kernel_time", "ahs_batch_set_stream",
    "ahs_batch_destroy", "ahs_batch_measure", "ahs_stable_dt", "ahs_bounds_check",
)
_NON_INT = ("ahs_create", "ahs_destroy", "ahs_last_error_message", "ahs_strerror", "ahs_sizeof_obs",
            "ahs_batch_create", "ahs_batch_destroy")


class ahs_obs_t(ctypes.Structure):
    _fields_ = [("step", ctypes.c_int64), ("tau", ctypes.c_double), ("a", ctypes.c_double),
                ("n_wind", ctypes.c_int64), ("string_length", ctypes.c_double),
                ("xi_w", ctypes.c_double), ("xi_l", ctypes.c_double),
                ("lagrangian", ctypes.c_double), ("v2_phi", ctypes.c_double),
                ("v2_omega", ctypes.c_double), ("e_kin", ctypes.c_double),
                ("e_grad", ctypes.c_double), ("e_pot", ctypes.c_double),
                ("e_elec", ctypes.c_double), ("e_mag", ctypes.c_double),
                ("e_total", ctypes.c_double), ("gauss_rms", ctypes.c_double),
                ("gauss_max", ctypes.c_double), ("nonfinite", ctypes.c_int64),
                ("sum_K", ctypes.c_double), ("sum_G", ctypes.c_double),
                ("sum_V", ctypes.c_double), ("sum_El", ctypes.c_double),
                ("sum_B", ctypes.c_double), ("sum_L", ctypes.c_double),
                ("sum_KL", ctypes.c_double), ("sum_GL", ctypes.c_double),
                ("sum_pL", ctypes.c_double), ("sum_rhoL", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class AHSError(RuntimeError):
    def __init__(self, status: int, where: str, message: str):
        super().__init__(f"{where}: {message} (status {status})")
        self.status = status


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load _ahs.so and declare the prototypes.  Raises if the library is missing."""
    if not os.path.exists(path):
        raise ImportError(f"engine library {path} is not built; run "
                          "`python -c 'import __graft_entry__ as g; g.build()'`")
    L = ctypes.CDLL(path)
    H = ctypes.c_void_p
    i, d, sz = ctypes.c_int, ctypes.c_double, ctypes.c_size_t
    vp = ctypes.c_void_p
    L.ahs_create.argtypes = [i, d, d, d, d, d, d, i]
    L.ahs_create.restype = H
    L.ahs_init.argtypes = [H, ctypes.c_uint64]
    L.ahs_step.argtypes = [H, i]
    L.ahs_measure.argtypes = [H, ctypes.POINTER(ahs_obs_t)]
    L.ahs_records.argtypes = [H, ctypes.POINTER(ahs_obs_t), i]
    L.ahs_fields.argtypes = [H, i, vp, sz]
    L.ahs_set_fields.argtypes = [H, i, vp, sz]
    L.ahs_fields_box.argtypes = [H, i, i, i, i, i, i, i, vp, sz]
    L.ahs_windings.argtypes = [H, vp, sz, ctypes.POINTER(ctypes.c_int64)]
    L.ahs_set_option.argtypes = [H, i, d]
    L.ahs_get_option.argtypes = [H, i, ctypes.POINTER(d)]
    L.ahs_set_stream.argtypes = [H, vp]
    L.ahs_kernel_time.argtypes = [H, i, ctypes.POINTER(d), ctypes.POINTER(ctypes.c_int64), i]
    L.ahs_device_bytes.argtypes = [H, ctypes.POINTER(sz)]
    L.ahs_destroy.argtypes = [H]
    L.ahs_destroy.restype = None
    L.ahs_last_error.argtypes = []
    L.ahs_last_error_message.restype = ctypes.c_char_p
    L.ahs_strerror.argtypes = [i]
    L.ahs_strerror.restype = ctypes.c_char_p
    L.ahs_sizeof_obs.restype = sz
    L.ahs_measure_noalloc.argtypes = [i, d, d, d, d, d, d, i, d, d, ctypes.c_int64, vp, vp, vp]
    L.ahs_autotune.argtypes = [H]
    L.ahs_stable_dt.argtypes = [d, d, d, d, d, i, d, d, d, d, d, ctypes.POINTER(d)]
    L.ahs_bounds_check.argtypes = [i, ctypes.POINTER(ctypes.c_int64)]
    i64p = ctypes.POINTER(ctypes.c_int64)
    L.ahs_batch_create.argtypes = [i, ctypes.POINTER(i), ctypes.POINTER(i), ctypes.POINTER(ctypes.c_uint64), i64p,
                                   d, d, d, d, d, d]
    L.ahs_batch_create.restype = H
    L.ahs_batch_init.argtypes = [H]
    L.ahs_batch_run.argtypes = [H, i]
    L.ahs_batch_records.argtypes = [H, i, ctypes.POINTER(ahs_obs_t), i]
    L.ahs_batch_measure.argtypes = [H, i, ctypes.POINTER(ahs_obs_t)]
    L.ahs_batch_fields.argtypes = [H, i, i, vp, sz]
    L.ahs_batch_set_fields.argtypes = [H, i, i, vp, sz]
    L.ahs_batch_step_info.argtypes = [H, i, i64p, i64p]
    L.ahs_batch_set_option.argtypes = [H, i, d]
    L.ahs_batch_get_option.argtypes = [H, i, ctypes.POINTER(d)]
    L.ahs_batch_member_zchunk.argtypes = [H, i, ctypes.POINTER(i)]
    L.ahs_batch_autotune.argtypes = [H]
    L.ahs_batch_kernel_time.argtypes = [H, ctypes.POINTER(d), i64p, i]
    L.ahs_batch_set_stream.argtypes = [H, vp]
    L.ahs_batch_destroy.argtypes = [H]
    L.ahs_batch_destroy.restype = None
    for name in EXPORTS:
        if name not in _NON_INT:
            getattr(L, name).restype = i
    if L.ahs_sizeof_obs() != ctypes.sizeof(ahs_obs_t):
        raise ImportError("ahs_obs_t layout mismatch between include/ahs.h and the binding")
    return L


_lib = None


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        _lib = load()
    return _lib


def check(status: int, where: str) -> int:
    if status < 0:
        msg = lib().ahs_last_error_message().decode(errors="replace")
        raise AHSError(status, where, msg or lib().ahs_strerror(status).decode())
    return status


# ---- thin wrappers with the ABI's names ------------------------------------
def ahs_create(N, dx, dt, lambda0, e0, sigma, s, era):
    h = lib().ahs_create(N, dx, dt, lambda0, e0, sigma, s, era)
    if not h:
        check(lib().ahs_last_error() or AHS_EINVAL, "ahs_create")
    return h


def ahs_init(h, seed):
    return check(lib().ahs_init(h, seed), "ahs_init")


def ahs_step(h, n):
    return check(lib().ahs_step(h, n), "ahs_step")


def ahs_measure(h) -> dict:
    o = ahs_obs_t()
    check(lib().ahs_measure(h, ctypes.byref(o)), "ahs_measure")
    return o.as_dict()


def ahs_records(h, max_records: int = 1 << 20):
    pending = check(lib().ahs_records(h, None, 0), "ahs_records")
    m = min(pending, max_records)
    if m == 0:
        return []
    buf = (ahs_obs_t * m)()
    got = check(lib().ahs_records(h, buf, m), "ahs_records")
    return [buf[i].as_dict() for i in range(got)]


def storage_dtype(h):
    return np.float64 if int(ahs_get_option(h, AHS_OPT_PRECISION)) == AHS_PREC_FP64 else np.float32


def ahs_fields(h, which, out: np.ndarray | None = None) -> np.ndarray:
    N = int(ahs_get_option(h, AHS_OPT_N))
    shape = (FIELD_PLANES[which], N, N, N)
    dt = storage_dtype(h)
    if out is None:
        out = np.empty(shape, dtype=dt)
    assert out.dtype == dt and out.flags.c_contiguous and out.shape == shape
    check(lib().ahs_fields(h, which, out.ctypes.data, out.nbytes), "ahs_fields")
    return out


def ahs_set_fields(h, which, src: np.ndarray):
    src = np.ascontiguousarray(src, dtype=storage_dtype(h))
    return check(lib().ahs_set_fields(h, which, src.ctypes.data, src.nbytes), "ahs_set_fields")


def ahs_fields_box(h, which, x0, y0, z0, nx, ny, nz) -> np.ndarray:
    out = np.empty((FIELD_PLANES[which], nz, ny, nx), dtype=np.float32)
    check(lib().ahs_fields_box(h, which, x0, y0, z0, nx, ny, nz, out.ctypes.data, out.nbytes), "ahs_fields_box")
    return out


def ahs_windings(h):
    N = int(ahs_get_option(h, AHS_OPT_N))
    W = np.empty((3, N, N, N), dtype=np.int8)
    n = ctypes.c_int64()
    check(lib().ahs_windings(h, W.ctypes.data, W.nbytes, ctypes.byref(n)), "ahs_windings")
    return W, n.value


def ahs_set_option(h, key, value):
    return check(lib().ahs_set_option(h, key, float(value)), "ahs_set_option")


def ahs_get_option(h, key) -> float:
    v = ctypes.c_double()
    check(lib().ahs_get_option(h, key, ctypes.byref(v)), "ahs_get_option")
    return v.value


def ahs_set_stream(h, stream_ptr: int):
    return check(lib().ahs_set_stream(h, ctypes.c_void_p(stream_ptr)), "ahs_set_stream")


def ahs_kernel_time(h, kind: int = AHS_KERNEL_STEP, reset: bool = False):
    ms, n = ctypes.c_double(), ctypes.c_int64()
    check(lib().ahs_kernel_time(h, kind, ctypes.byref(ms), ctypes.byref(n), int(reset)), "ahs_kernel_time")
    return ms.value, n.value


def ahs_device_bytes(h) -> int:
    b = ctypes.c_size_t()
    check(lib().ahs_device_bytes(h, ctypes.byref(b)), "ahs_device_bytes")
    return b.value


def ahs_destroy(h):
    if h:
        lib().ahs_destroy(h)


def ahs_stable_dt(dx, lambda0, e0, sigma, s, era, tau0, tau_end, s_cg=0.0, tau_cg=0.0, safety=0.9) -> float:
    v = ctypes.c_double()
    check(lib().ahs_stable_dt(dx, lambda0, e0, sigma, s, era, tau0, tau_end, s_cg, tau_cg, safety,
                              ctypes.byref(v)), "ahs_stable_dt")
    return v.value


def ahs_autotune(h):
    return check(lib().ahs_autotune(h), "ahs_autotune")


# ---- batched ensembles --------------------------------------------------------
def ahs_batch_create(N, era, seed, n_end=None, dx=0.5, dt=0.1, lambda0=2.0, e0=1.0, sigma=1.0, s=0.0):
    count = len(N)
    Na = (ctypes.c_int * count)(*N)
    Ea = (ctypes.c_int * count)(*era)
    Sa = (ctypes.c_uint64 * count)(*seed)
    Ta = (ctypes.c_int64 * count)(*n_end) if n_end is not None else None
    h = lib().ahs_batch_create(count, Na, Ea, Sa, Ta, dx, dt, lambda0, e0, sigma, s)
    if not h:
        check(lib().ahs_last_error() or AHS_EINVAL, "ahs_batch_create")
    return h


def ahs_batch_init(b):
    return check(lib().ahs_batch_init(b), "ahs_batch_init")


def ahs_batch_run(b, max_steps):
    return check(lib().ahs_batch_run(b, max_steps), "ahs_batch_run")


def ahs_batch_measure(b, m) -> dict:
    o = ahs_obs_t()
    check(lib().ahs_batch_measure(b, m, ctypes.byref(o)), "ahs_batch_measure")
    return o.as_dict()


def ahs_batch_records(b, m):
    pending = check(lib().ahs_batch_records(b, m, None, 0), "ahs_batch_records")
    if pending == 0:
        return []
    buf = (ahs_obs_t * pending)()
    got = check(lib().ahs_batch_records(b, m, buf, pending), "ahs_batch_records")
    return [buf[k].as_dict() for k in range(got)]


def ahs_batch_step_info(b, m):
    n, e = ctypes.c_int64(), ctypes.c_int64()
    check(lib().ahs_batch_step_info(b, m, ctypes.byref(n), ctypes.byref(e)), "ahs_batch_step_info")
    return n.value, e.value


def ahs_batch_fields(b, m, which, N) -> np.ndarray:
    out = np.empty((FIELD_PLANES[which], N, N, N), dtype=np.float32)
    check(lib().ahs_batch_fields(b, m, which, out.ctypes.data, out.nbytes), "ahs_batch_fields")
    return out


def ahs_batch_set_fields(b, m, which, src: np.ndarray):
    src = np.ascontiguousarray(src, dtype=np.float32)
    return check(lib().ahs_batch_set_fields(b, m, which, src.ctypes.data, src.nbytes), "ahs_batch_set_fields")


def ahs_batch_set_option(b, key, value):
    return check(lib().ahs_batch_set_option(b, key, float(value)), "ahs_batch_set_option")


def ahs_batch_get_option(b, key) -> float:
    v = ctypes.c_double()
    check(lib().ahs_batch_get_option(b, key, ctypes.byref(v)), "ahs_batch_get_option")
    return v.value


def ahs_batch_member_zchunk(b, m) -> int:
    v = ctypes.c_int()
    check(lib().ahs_batch_member_zchunk(b, m, ctypes.byref(v)), "ahs_batch_member_zchunk")
    return v.value


def ahs_batch_autotune(b):
    return check(lib().ahs_batch_autotune(b), "ahs_batch_autotune")


def ahs_batch_kernel_time(b, reset=False):
    ms, n = ctypes.c_double(), ctypes.c_int64()
    check(lib().ahs_batch_kernel_time(b, ctypes.byref(ms), ctypes.byref(n), int(reset)), "ahs_batch_kernel_time")
    return ms.value, n.value


def ahs_batch_set_stream(b, stream_ptr: int):
    return check(lib().ahs_batch_set_stream(b, ctypes.c_void_p(stream_ptr)), "ahs_batch_set_stream")


def ahs_batch_destroy(b):
    if b:
        lib().ahs_batch_destroy(b)
