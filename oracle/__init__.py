"""FP64 CPU oracle for overlap-and-save convolution -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference
legs of ``bench.py`` may import this package.  The product library
(``paper_1910_01972_gb300``) never imports it and never falls back to it.

The arithmetic lives in ``ols_oracle.c`` (plain C, FP64, OpenMP over output
elements): the valid part of Eq. 1 for a bank of filters (Sec. 3.2 states
that OLS returns exactly this, whatever the segment length), the adjoint
of that linear map, the real-to-real form, and the post-processing of the
output (power, and the derivative read as central differences with
one-sided ends, Sec. 4.3), and the peak rule on the power (Sec. 4.4's peak
finding); ``detect`` and ``peaks`` only select from ``power``.  This module
only compiles the C file and marshals numpy arrays through ctypes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ols_oracle.c")
_LIB_PATH = os.path.join(_HERE, "libols_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile ``ols_oracle.c`` into ``libols_oracle.so`` beside it.

    ``-ffp-contract=off`` keeps every multiply and add separately rounded so
    x86 and Arm hosts give identical results; no fast-math.
    """
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + ".tmp.%d" % os.getpid()
    cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
           "-fPIC", "-shared", "-std=c11", "-o", tmp, _SRC]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        i64, i32 = ctypes.c_int64, ctypes.c_int32
        vp = ctypes.c_void_p
        lib.ols_oracle_conv.argtypes = [i64, vp, i32, i32, vp, vp]
        lib.ols_oracle_conv.restype = ctypes.c_int
        lib.ols_oracle_conv_at.argtypes = [i64, vp, i32, i32, vp, i64, vp, vp, vp]
        lib.ols_oracle_conv_at.restype = ctypes.c_int
        lib.ols_oracle_adjoint.argtypes = [i64, vp, i32, i32, vp, vp, vp, vp]
        lib.ols_oracle_adjoint.restype = ctypes.c_int
        lib.ols_oracle_conv_real.argtypes = [i64, vp, i32, i32, vp, vp]
        lib.ols_oracle_conv_real.restype = ctypes.c_int
        lib.ols_oracle_conv_real_at.argtypes = [i64, vp, i32, i32, vp, i64, vp, vp, vp]
        lib.ols_oracle_conv_real_at.restype = ctypes.c_int
        lib.ols_oracle_power.argtypes = [i64, vp, i32, i32, vp, vp]
        lib.ols_oracle_power.restype = ctypes.c_int
        lib.ols_oracle_derivative.argtypes = [i64, vp, i32, i32, vp, vp]
        lib.ols_oracle_derivative.restype = ctypes.c_int
        lib.ols_oracle_derivative_at.argtypes = [i64, vp, i32, i32, vp, i64, vp, vp, vp]
        lib.ols_oracle_derivative_at.restype = ctypes.c_int
        lib.ols_oracle_peak_mask.argtypes = [i32, i64, vp, ctypes.c_double, vp]
        lib.ols_oracle_peak_mask.restype = ctypes.c_int
        lib.ols_oracle_threads.argtypes = []
        lib.ols_oracle_threads.restype = ctypes.c_int
        lib.ols_oracle_set_threads.argtypes = [ctypes.c_int]
        lib.ols_oracle_set_threads.restype = None
        _lib = lib
        return lib


def _c64(a) -> np.ndarray:
    a = np.ascontiguousarray(a)
    if a.dtype != np.complex64:
        raise TypeError("oracle inputs are complex64 (the FP32 values the GPU consumes), got %s" % a.dtype)
    return a


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def threads() -> int:
    """OpenMP threads the oracle uses."""
    return int(_load().ols_oracle_threads())


def set_threads(n: int) -> None:
    _load().ols_oracle_set_threads(int(n))


def conv(s, h) -> np.ndarray:
    """Valid-mode convolution y[F][Ns-M+1] (complex128) of s[Ns] with h[F][M].

    ``h`` may be 1-D (one filter), giving y of shape [Ns-M+1].
    """
    s = _c64(s)
    h = _c64(h)
    squeeze = h.ndim == 1
    if squeeze:
        h = h[None, :]
    F, M = h.shape
    Ns = s.shape[0]
    if M < 1 or F < 1 or Ns < M:
        raise ValueError("need M >= 1, F >= 1, Ns >= M")
    y = np.empty((F, Ns - M + 1), dtype=np.complex128)
    rc = _load().ols_oracle_conv(Ns, _ptr(s), M, F, _ptr(h), _ptr(y))
    if rc != 0:
        raise ValueError("ols_oracle_conv rejected the sizes")
    return y[0] if squeeze else y


def conv_at(s, h, f_idx, j_idx) -> np.ndarray:
    """y_{f_idx[i]}[j_idx[i]] for each i (complex128)."""
    s = _c64(s)
    h = _c64(h)
    if h.ndim == 1:
        h = h[None, :]
    F, M = h.shape
    fi = np.ascontiguousarray(f_idx, dtype=np.int64)
    ji = np.ascontiguousarray(j_idx, dtype=np.int64)
    if fi.shape != ji.shape:
        raise ValueError("index arrays differ in shape")
    out = np.empty(fi.shape, dtype=np.complex128)
    rc = _load().ols_oracle_conv_at(s.shape[0], _ptr(s), M, F, _ptr(h), fi.size,
                                    _ptr(fi), _ptr(ji), _ptr(out))
    if rc != 0:
        raise ValueError("ols_oracle_conv_at rejected the sizes or an index")
    return out


def _f32(a) -> np.ndarray:
    a = np.ascontiguousarray(a)
    if a.dtype != np.float32:
        raise TypeError("real oracle inputs are float32 (the FP32 values the GPU consumes), got %s" % a.dtype)
    return a


def conv_real(s, h) -> np.ndarray:
    """Real valid-mode convolution y[F][Ns-M+1] (float64) of real s[Ns] with
    real h[F][M] (the R2R form); ``h`` may be 1-D."""
    s = _f32(s)
    h = _f32(h)
    squeeze = h.ndim == 1
    if squeeze:
        h = h[None, :]
    F, M = h.shape
    Ns = s.shape[0]
    if M < 1 or F < 1 or Ns < M:
        raise ValueError("need M >= 1, F >= 1, Ns >= M")
    y = np.empty((F, Ns - M + 1), dtype=np.float64)
    rc = _load().ols_oracle_conv_real(Ns, _ptr(s), M, F, _ptr(h), _ptr(y))
    if rc != 0:
        raise ValueError("ols_oracle_conv_real rejected the sizes")
    return y[0] if squeeze else y


def conv_real_at(s, h, f_idx, j_idx) -> np.ndarray:
    """Real y_{f_idx[i]}[j_idx[i]] for each i (float64)."""
    s = _f32(s)
    h = _f32(h)
    if h.ndim == 1:
        h = h[None, :]
    F, M = h.shape
    fi = np.ascontiguousarray(f_idx, dtype=np.int64)
    ji = np.ascontiguousarray(j_idx, dtype=np.int64)
    if fi.shape != ji.shape:
        raise ValueError("index arrays differ in shape")
    out = np.empty(fi.shape, dtype=np.float64)
    rc = _load().ols_oracle_conv_real_at(s.shape[0], _ptr(s), M, F, _ptr(h), fi.size,
                                         _ptr(fi), _ptr(ji), _ptr(out))
    if rc != 0:
        raise ValueError("ols_oracle_conv_real_at rejected the sizes or an index")
    return out


def _bank(s, h):
    s = _c64(s)
    h = _c64(h)
    squeeze = h.ndim == 1
    if squeeze:
        h = h[None, :]
    F, M = h.shape
    if M < 1 or F < 1 or s.shape[0] < M:
        raise ValueError("need M >= 1, F >= 1, Ns >= M")
    return s, h, F, M, squeeze


def power(s, h) -> np.ndarray:
    """Power of the convolved output, p[F][Ns-M+1] = |y|^2 (float64)."""
    s, h, F, M, squeeze = _bank(s, h)
    p = np.empty((F, s.shape[0] - M + 1), dtype=np.float64)
    if _load().ols_oracle_power(s.shape[0], _ptr(s), M, F, _ptr(h), _ptr(p)) != 0:
        raise ValueError("ols_oracle_power rejected the sizes")
    return p[0] if squeeze else p


def power_at(s, h, f_idx, j_idx) -> np.ndarray:
    """|y_{f_idx[i]}[j_idx[i]]|^2 (float64)."""
    y = conv_at(s, h, f_idx, j_idx)
    return y.real * y.real + y.imag * y.imag


def detect(s, h, threshold: float):
    """Candidates of the power detector: the set of (f, j) with
    |y_f[j]|^2 >= threshold, and their powers (float64)."""
    p = power(s, h)
    if p.ndim == 1:
        p = p[None, :]
    f, j = np.nonzero(p >= threshold)
    return f, j, p[f, j]


def peak_mask(p, threshold: float) -> np.ndarray:
    """Peak rule of ``ols_oracle_peak_mask`` on a power array p[F][Nout] (or
    [Nout]): bool mask of the (f, j) whose power reaches the threshold, is
    above its left neighbour and at least its right one."""
    p = np.ascontiguousarray(p, dtype=np.float64)
    squeeze = p.ndim == 1
    if squeeze:
        p = p[None, :]
    F, Nout = p.shape
    m = np.zeros((F, Nout), dtype=np.uint8)
    if _load().ols_oracle_peak_mask(F, Nout, _ptr(p), float(threshold), _ptr(m)) != 0:
        raise ValueError("ols_oracle_peak_mask rejected the sizes")
    m = m.astype(bool)
    return m[0] if squeeze else m


def peaks(s, h, threshold: float):
    """Peaks of the power of the convolved output (``peak_mask`` of
    ``power``): the (f, j) and their powers (float64)."""
    p = power(s, h)
    if p.ndim == 1:
        p = p[None, :]
    f, j = np.nonzero(peak_mask(p, threshold))
    return f, j, p[f, j]


def derivative(s, h) -> np.ndarray:
    """Derivative of the convolved output along j, d[F][Ns-M+1] (complex128):
    central differences inside, one-sided at both ends (Ns - M + 1 >= 2)."""
    s, h, F, M, squeeze = _bank(s, h)
    d = np.empty((F, s.shape[0] - M + 1), dtype=np.complex128)
    if _load().ols_oracle_derivative(s.shape[0], _ptr(s), M, F, _ptr(h), _ptr(d)) != 0:
        raise ValueError("ols_oracle_derivative rejected the sizes (needs Ns - M + 1 >= 2)")
    return d[0] if squeeze else d


def derivative_at(s, h, f_idx, j_idx) -> np.ndarray:
    """d_{f_idx[i]}[j_idx[i]] for each i (complex128)."""
    s, h, F, M, _ = _bank(s, h)
    fi = np.ascontiguousarray(f_idx, dtype=np.int64)
    ji = np.ascontiguousarray(j_idx, dtype=np.int64)
    if fi.shape != ji.shape:
        raise ValueError("index arrays differ in shape")
    out = np.empty(fi.shape, dtype=np.complex128)
    if _load().ols_oracle_derivative_at(s.shape[0], _ptr(s), M, F, _ptr(h), fi.size, _ptr(fi), _ptr(ji),
                                        _ptr(out)) != 0:
        raise ValueError("ols_oracle_derivative_at rejected the sizes or an index")
    return out


def adjoint(s, h, g, want_ds: bool = True, want_dh: bool = True):
    """Adjoint of ``conv``: returns (ds[Ns], dh[F][M]) as complex128.

    ``g`` is dL/dRe y + i dL/dIm y, shape [F][Ns-M+1]; it is widened to
    complex128 (exact for complex64 input).
    """
    s = _c64(s)
    h = _c64(h)
    g = np.ascontiguousarray(g, dtype=np.complex128)
    squeeze = h.ndim == 1
    if squeeze:
        h = h[None, :]
        g = g[None, :]
    F, M = h.shape
    Ns = s.shape[0]
    if g.shape != (F, Ns - M + 1):
        raise ValueError("g must have shape [F][Ns-M+1]")
    ds = np.empty(Ns, dtype=np.complex128) if want_ds else None
    dh = np.empty((F, M), dtype=np.complex128) if want_dh else None
    rc = _load().ols_oracle_adjoint(Ns, _ptr(s), M, F, _ptr(h), _ptr(g),
                                    _ptr(ds) if ds is not None else None,
                                    _ptr(dh) if dh is not None else None)
    if rc != 0:
        raise ValueError("ols_oracle_adjoint rejected the sizes")
    if squeeze and dh is not None:
        dh = dh[0]
    return ds, dh


def rel_l2(y, y_ref) -> float:
    """||y - y_ref||_2 / ||y_ref||_2 (in FP64)."""
    y = np.asarray(y, dtype=np.complex128)
    y_ref = np.asarray(y_ref, dtype=np.complex128)
    den = np.linalg.norm(y_ref.ravel())
    num = np.linalg.norm((y - y_ref).ravel())
    return float(num / den) if den > 0 else float(num)


def max_stream_rel_l2(y, y_ref, floor=None) -> float:
    """Largest per-stream relative L2 error over the leading (filter) axis.
    floor (one value per stream, e.g. ``stream_scale``): the denominator is
    max(||y_ref_f||, floor_f)."""
    y = np.asarray(y)
    y_ref = np.asarray(y_ref)
    if y.ndim == 1:
        y, y_ref = y[None], y_ref[None]
    out = 0.0
    for f in range(y.shape[0]):
        num = np.linalg.norm((y[f].astype(np.complex128) - y_ref[f]).ravel())
        den = np.linalg.norm(np.asarray(y_ref[f], dtype=np.complex128).ravel())
        if floor is not None:
            den = max(den, float(np.ravel(floor)[f]))
        out = max(out, float(num / den) if den > 0 else float(num))
    return out


def stream_scale(s, h, Nout) -> np.ndarray:
    """Expected norm of each output stream for a white signal:
    sqrt(Nout) ||h_f||_2 rms(s), since E|y_f[j]|^2 = ||h_f||^2 E|s|^2 by
    Eq. 1.  A stream of a few outputs can have a norm far below it by chance
    (one output of a random signal can be near zero), while the rounding
    error of an FFT-based convolution scales with the segment's and the
    filter's energy, not with that output; this is the floor of the
    denominator that makes the relative error of such streams meaningful.
    For long streams ||y_f|| is close to it and the floor has no effect."""
    s = np.asarray(s)
    h = np.asarray(h)
    if h.ndim == 1:
        h = h[None]
    rms = np.linalg.norm(s.astype(np.complex128)) / np.sqrt(max(s.size, 1))
    return np.sqrt(Nout) * np.linalg.norm(h.astype(np.complex128), axis=1) * rms
