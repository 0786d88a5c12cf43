"""ctypes binding of ``libols.so`` (C ABI declared in include/ols.h).

Argument marshalling only: every function here has the name and argument
order of its C counterpart and forwards plain integers and pointers.  The
library must exist: there is no fallback of any kind, a missing or stale
build raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
# OLS_LIBRARY selects another build of the library (e.g. the bounds-checked
# debug build, libols_check.so); default: the in-tree libols.so.
LIB_PATH = os.environ.get("OLS_LIBRARY") or os.path.join(_HERE, "libols.so")

OLS_OK = 0
OLS_ERR_INVALID = 1
OLS_ERR_UNSUPPORTED = 2
OLS_ERR_ALLOC = 3
OLS_ERR_CUDA = 4
OLS_ERR_NOT_READY = 5
OLS_ERR_TIMEOUT = 6
OLS_ERR_WORKSPACE = 7
OLS_ERR_TOO_LARGE = 8
OLS_NOALLOC_SCRATCH_BYTES = 32 << 20

OLS_FLAG_FP32 = 0
OLS_TUNE_MODEL = 1 << 8
OLS_BATCH_PER_N = 1 << 9
OLS_FLAG_TC_FP16SPLIT = 1
OLS_FLAG_TC_BF16SPLIT = 2
OLS_FLAG_R2R = 4

# (name, restype, argtypes) of every exported symbol declared in include/ols.h
i32, i64, u32 = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32
vp, cint = ctypes.c_void_p, ctypes.c_int
P_i64, P_i32 = ctypes.POINTER(i64), ctypes.POINTER(i32)
SIGNATURES = [
    ("ols_status_string", ctypes.c_char_p, [cint]),
    ("ols_version", cint, []),
    ("ols_geometry", cint, [i64, i32, i64, P_i64, P_i64, P_i64]),
    ("ols_spectrum_order", cint, [i64, P_i32]),
    ("ols_plan", cint, [ctypes.POINTER(vp), i64, i32, i32, u32]),
    ("ols_plan_destroy", cint, [vp]),
    ("ols_plan_query", cint, [vp, i64, P_i64, P_i32, P_i32, P_i64, P_i64, P_i64]),
    ("ols_set_filters", cint, [vp, vp, vp]),
    ("ols_get_spectra", cint, [vp, vp, vp]),
    ("ols_convolve", cint, [vp, vp, i64, vp, vp]),
    ("ols_convolve_host", cint, [vp, vp, i64, vp, vp]),
    ("ols_host_timing", cint, [vp, cint]),
    ("ols_host_stage_ms", cint, [vp, ctypes.POINTER(ctypes.c_double)]),
    ("ols_convolve_split", cint, [vp, vp, vp, i64, vp, vp]),
    ("ols_split_signal", cint, [vp, vp, i64, vp, vp, vp]),
    ("ols_convolve_power", cint, [vp, vp, i64, vp, vp]),
    ("ols_convolve_detect", cint, [vp, vp, i64, ctypes.c_float, vp, i64, vp, vp]),
    ("ols_convolve_peaks", cint, [vp, vp, i64, ctypes.c_float, vp, i64, vp, vp]),
    ("ols_convolve_derivative", cint, [vp, vp, i64, vp, vp]),
    ("ols_set_filters_real", cint, [vp, vp, vp]),
    ("ols_convolve_real", cint, [vp, vp, i64, vp, vp]),
    ("ols_backward_workspace", cint, [vp, i64, cint, cint, ctypes.POINTER(ctypes.c_size_t)]),
    ("ols_convolve_backward", cint, [vp, vp, i64, vp, vp, vp, vp, ctypes.c_size_t, vp]),
    ("ols_convolve_backward_noalloc", cint, [vp, vp, i64, vp, vp, vp, vp]),
    ("ols_last_launch_count", cint, [vp]),
    ("ols_plan_status", cint, [vp, P_i32, cint]),
    ("ols_autotune", cint, [i32, i32, u32, P_i64]),
    ("ols_batch_plan", cint, [ctypes.POINTER(vp), i32, P_i64, P_i32, P_i32, P_i64, u32]),
    ("ols_batch_destroy", cint, [vp]),
    ("ols_batch_query", cint, [vp, i32, P_i64, P_i64, P_i32]),
    ("ols_batch_set_filters", cint, [vp, ctypes.POINTER(vp), vp]),
    ("ols_convolve_batched", cint, [vp, vp, vp, vp]),
    ("ols_batch_last_launch_count", cint, [vp]),
    ("ols_batch_plan_tiles", cint, [ctypes.POINTER(vp), i32, P_i64, P_i32, P_i32, P_i64, P_i32, u32]),
    ("ols_autotune_tiles", cint, [i32, i32, i64, i32, u32, P_i32]),
    ("ols_batch_schedule", cint, [vp, i32, P_i32, P_i64]),
    ("ols_batch_status", cint, [vp, P_i32, cint]),
]

_lib = None
_lock = threading.Lock()


class OLSError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        msg = lib().ols_status_string(status).decode() if _lib is not None else str(status)
        super().__init__("%s: %s" % (where, msg))


def lib():
    """The loaded library (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libols.so is not built (run __graft_entry__.build() or "
                               "python -m paper_1910_01972_gb300.build); there is no fallback path")
        L = ctypes.CDLL(LIB_PATH)
        for name, res, args in SIGNATURES:
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
        return L


def check(status: int, where: str) -> None:
    if status != OLS_OK:
        raise OLSError(status, where)


def ols_status_string(status: int) -> str:
    return lib().ols_status_string(status).decode()


def ols_version() -> int:
    return lib().ols_version()


def ols_geometry(N: int, M: int, Ns: int):
    L, nseg, Nout = i64(), i64(), i64()
    rc = lib().ols_geometry(N, M, Ns, ctypes.byref(L), ctypes.byref(nseg), ctypes.byref(Nout))
    return rc, L.value, nseg.value, Nout.value


def ols_spectrum_order(N: int):
    arr = (i32 * N)()
    rc = lib().ols_spectrum_order(N, arr)
    return rc, list(arr)


def ols_plan(N: int, M: int, F: int, flags: int = OLS_FLAG_FP32):
    h = vp()
    rc = lib().ols_plan(ctypes.byref(h), N, M, F, flags)
    return rc, h.value


def ols_plan_destroy(plan) -> int:
    return lib().ols_plan_destroy(plan)


def ols_plan_query(plan, Ns: int = 0):
    N, M, F, L, nseg, Nout = i64(), i32(), i32(), i64(), i64(), i64()
    rc = lib().ols_plan_query(plan, Ns, ctypes.byref(N), ctypes.byref(M), ctypes.byref(F),
                              ctypes.byref(L), ctypes.byref(nseg), ctypes.byref(Nout))
    return rc, dict(N=N.value, M=M.value, F=F.value, L=L.value, nseg=nseg.value, Nout=Nout.value)


def ols_set_filters(plan, h_ptr: int, stream: int) -> int:
    return lib().ols_set_filters(plan, h_ptr, stream)


def ols_get_spectra(plan, H_ptr: int, stream: int) -> int:
    return lib().ols_get_spectra(plan, H_ptr, stream)


def ols_convolve(plan, s_ptr: int, Ns: int, y_ptr: int, stream: int) -> int:
    return lib().ols_convolve(plan, s_ptr, Ns, y_ptr, stream)


def ols_convolve_power(plan, s_ptr: int, Ns: int, p_ptr: int, stream: int) -> int:
    return lib().ols_convolve_power(plan, s_ptr, Ns, p_ptr, stream)


def ols_convolve_detect(plan, s_ptr: int, Ns: int, threshold: float, cand_ptr, capacity: int, count_ptr: int,
                        stream: int) -> int:
    return lib().ols_convolve_detect(plan, s_ptr, Ns, threshold, cand_ptr, capacity, count_ptr, stream)


def ols_convolve_peaks(plan, s_ptr: int, Ns: int, threshold: float, cand_ptr, capacity: int, count_ptr: int,
                        stream: int) -> int:
    return lib().ols_convolve_peaks(plan, s_ptr, Ns, threshold, cand_ptr, capacity, count_ptr, stream)


def ols_convolve_derivative(plan, s_ptr: int, Ns: int, d_ptr: int, stream: int) -> int:
    return lib().ols_convolve_derivative(plan, s_ptr, Ns, d_ptr, stream)


def ols_set_filters_real(plan, h_ptr: int, stream: int) -> int:
    return lib().ols_set_filters_real(plan, h_ptr, stream)


def ols_convolve_real(plan, s_ptr: int, Ns: int, y_ptr: int, stream: int) -> int:
    return lib().ols_convolve_real(plan, s_ptr, Ns, y_ptr, stream)


def ols_convolve_host(plan, s_ptr: int, Ns: int, y_ptr: int, stream: int) -> int:
    return lib().ols_convolve_host(plan, s_ptr, Ns, y_ptr, stream)


def ols_host_timing(plan, on: bool) -> int:
    return lib().ols_host_timing(plan, int(on))


def ols_host_stage_ms(plan):
    ms = (ctypes.c_double * 5)()
    rc = lib().ols_host_stage_ms(plan, ms)
    return rc, list(ms)


def ols_backward_workspace(plan, Ns: int, want_ds: bool, want_dh: bool):
    nb = ctypes.c_size_t()
    rc = lib().ols_backward_workspace(plan, Ns, int(want_ds), int(want_dh), ctypes.byref(nb))
    return rc, nb.value


def ols_convolve_backward(plan, s_ptr, Ns: int, g_ptr: int, ds_ptr, dh_ptr, ws_ptr, ws_bytes: int,
                          stream: int) -> int:
    return lib().ols_convolve_backward(plan, s_ptr, Ns, g_ptr, ds_ptr, dh_ptr, ws_ptr, ws_bytes, stream)


def ols_convolve_split(plan, hi_ptr: int, lo_ptr: int, Ns: int, y_ptr: int, stream: int) -> int:
    return lib().ols_convolve_split(plan, hi_ptr, lo_ptr, Ns, y_ptr, stream)


def ols_split_signal(plan, s_ptr: int, Ns: int, hi_ptr: int, lo_ptr: int, stream: int) -> int:
    return lib().ols_split_signal(plan, s_ptr, Ns, hi_ptr, lo_ptr, stream)


def ols_convolve_backward_noalloc(plan, s_ptr, Ns: int, g_ptr: int, ds_ptr, dh_ptr, stream: int) -> int:
    return lib().ols_convolve_backward_noalloc(plan, s_ptr, Ns, g_ptr, ds_ptr, dh_ptr, stream)


def ols_last_launch_count(plan) -> int:
    return lib().ols_last_launch_count(plan)


def ols_plan_status(plan, reset: bool = True):
    v = i32()
    rc = lib().ols_plan_status(plan, ctypes.byref(v), int(reset))
    return rc, v.value


def ols_autotune(M: int, F: int, flags: int = 0):
    n = i64()
    rc = lib().ols_autotune(M, F, flags, ctypes.byref(n))
    return rc, n.value


def ols_batch_plan(Ns, M, F, N=None, flags: int = 0):
    B = len(Ns)
    a_ns = (i64 * B)(*Ns)
    a_m = (i32 * B)(*M)
    a_f = (i32 * B)(*F)
    a_n = (i64 * B)(*N) if N is not None else None
    h = vp()
    rc = lib().ols_batch_plan(ctypes.byref(h), B, a_ns, a_m, a_f, a_n, flags)
    return rc, h.value


def ols_batch_plan_tiles(Ns, M, F, N=None, tiles=None, flags: int = 0):
    B = len(Ns)
    a_ns = (i64 * B)(*Ns)
    a_m = (i32 * B)(*M)
    a_f = (i32 * B)(*F)
    a_n = (i64 * B)(*N) if N is not None else None
    a_t = (i32 * B)(*tiles) if tiles is not None else None
    h = vp()
    rc = lib().ols_batch_plan_tiles(ctypes.byref(h), B, a_ns, a_m, a_f, a_n, a_t, flags)
    return rc, h.value


def ols_autotune_tiles(M: int, F: int, N: int, block: int, flags: int = 0):
    r = i32()
    rc = lib().ols_autotune_tiles(M, F, N, block, flags, ctypes.byref(r))
    return rc, r.value


def ols_batch_schedule(batch, b: int):
    r, n = i32(), i64()
    rc = lib().ols_batch_schedule(batch, b, ctypes.byref(r), ctypes.byref(n))
    return rc, r.value, n.value


def ols_batch_status(batch, reset: bool = True):
    v = i32()
    rc = lib().ols_batch_status(batch, ctypes.byref(v), int(reset))
    return rc, v.value


def ols_batch_destroy(batch) -> int:
    return lib().ols_batch_destroy(batch)


def ols_batch_query(batch, b: int):
    N, Nout, ng = i64(), i64(), i32()
    rc = lib().ols_batch_query(batch, b, ctypes.byref(N), ctypes.byref(Nout), ctypes.byref(ng))
    return rc, N.value, Nout.value, ng.value


def ols_batch_set_filters(batch, h_ptrs, stream: int) -> int:
    arr = (vp * len(h_ptrs))(*h_ptrs)
    return lib().ols_batch_set_filters(batch, arr, stream)


def ols_convolve_batched(batch, s_ptrs_dev: int, y_ptrs_dev: int, stream: int) -> int:
    return lib().ols_convolve_batched(batch, s_ptrs_dev, y_ptrs_dev, stream)


def ols_batch_last_launch_count(batch) -> int:
    return lib().ols_batch_last_launch_count(batch)
