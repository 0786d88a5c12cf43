"""The FP64 oracle pinned to the paper and to mathematics (CPU only)."""
import ctypes
import importlib.util
import os
import shutil
import subprocess
import tempfile

import numpy as np
import pytest

import oracle
from tests import oracle_pins as P


def _conv(s, h):
    return oracle.conv(s, h)


def _adj(s, h, g):
    return oracle.adjoint(s, h, g)


@pytest.mark.parametrize("pin", [P.pin_golden_conv, P.pin_golden_adjoint, P.pin_bruteforce_dft,
                                 P.pin_fft_fullconv, P.pin_delta_shift, P.pin_linearity,
                                 P.pin_closed_forms, P.pin_adjoint_dot])
def test_oracle_pin(pin):
    pin(_conv, _adj)


@pytest.mark.parametrize("pin", P.REAL_QUICK_PINS)
def test_oracle_real_pin(pin):
    pin(oracle.conv_real)


def test_oracle_real_matches_complex_on_real_data():
    P.pin_real_is_complex_on_real_data(oracle.conv_real, oracle.conv)


def test_oracle_conv_real_at_matches_conv_real():
    g = np.random.Generator(np.random.PCG64(5))
    s = g.uniform(-1, 1, 900).astype(np.float32)
    h = g.normal(size=(3, 20)).astype(np.float32)
    y = oracle.conv_real(s, h)
    fi = g.integers(0, 3, 100)
    ji = g.integers(0, y.shape[1], 100)
    assert np.array_equal(oracle.conv_real_at(s, h, fi, ji), y[fi, ji])
    with pytest.raises(TypeError):
        oracle.conv_real(s.astype(np.float64), h)
    with pytest.raises(ValueError):
        oracle.conv_real(s[:5], h)


def test_oracle_adjoint_finite_difference():
    worst = P.pin_adjoint_finite_difference(_conv, _adj)
    assert worst < 1e-9


def test_oracle_conv_at_matches_conv():
    g = np.random.Generator(np.random.PCG64(3))
    s = (g.uniform(-1, 1, 1000) + 1j * g.uniform(-1, 1, 1000)).astype(np.complex64)
    h = (g.normal(size=(4, 33)) + 1j * g.normal(size=(4, 33))).astype(np.complex64)
    y = oracle.conv(s, h)
    fi = g.integers(0, 4, 200)
    ji = g.integers(0, y.shape[1], 200)
    assert np.array_equal(oracle.conv_at(s, h, fi, ji), y[fi, ji])
    with pytest.raises(ValueError):
        oracle.conv_at(s, h, [4], [0])
    with pytest.raises(ValueError):
        oracle.conv_at(s, h, [0], [y.shape[1]])


def test_oracle_rejects_bad_sizes():
    s = np.zeros(4, np.complex64)
    with pytest.raises(ValueError):
        oracle.conv(s, np.zeros(5, np.complex64))
    with pytest.raises(TypeError):
        oracle.conv(s.astype(np.complex128), np.zeros(2, np.complex64))


def test_oracle_thread_count_invariant():
    """Each output is one sequential sum, so the thread count cannot change it."""
    g = np.random.Generator(np.random.PCG64(4))
    s = (g.uniform(-1, 1, 3000) + 1j * g.uniform(-1, 1, 3000)).astype(np.complex64)
    h = (g.normal(size=(3, 65)) + 1j * g.normal(size=(3, 65))).astype(np.complex64)
    n0 = oracle.threads()
    try:
        oracle.set_threads(1)
        y1 = oracle.conv(s, h)
        oracle.set_threads(max(2, n0))
        y2 = oracle.conv(s, h)
    finally:
        oracle.set_threads(n0)
    assert np.array_equal(y1, y2)


# ------------------------------------------------------------ mutation test
# Plausible mistakes planted in copies of the oracle source (never in the
# oracle itself).  Each must be caught by at least one quick pin.
MUTANTS = {
    "drop_last_tap": ("for (int32_t k = 0; k < M; ++k) {\n        const int64_t n = j",
                      "for (int32_t k = 0; k < M - 1; ++k) {\n        const int64_t n = j"),
    "off_by_one_index": ("const int64_t n = j + (int64_t)M - 1 - k;",
                         "const int64_t n = j + (int64_t)M - 1 - k + (k > 0);"),
    "conjugated_tap": ("acc_im += sr * hi + si * hr;", "acc_im += si * hr - sr * hi;"),
    "wrong_sign_re": ("acc_re += sr * hr - si * hi;", "acc_re += sr * hr + si * hi;"),
    "adjoint_no_conj_h": ("acc_im += gi * hr - gr * hi;", "acc_im += gi * hr + gr * hi;"),
    "adjoint_dh_index": ("const int64_t n = j + M - 1 - k;", "const int64_t n = j + k;"),
    "adjoint_ds_edge": ("if (j < 0 || j >= Nout) continue;", "if (j < 0 || j >= Nout - 1) continue;"),
}


def _bind(path):
    lib = ctypes.CDLL(path)
    vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32
    lib.ols_oracle_conv.argtypes = [i64, vp, i32, i32, vp, vp]
    lib.ols_oracle_adjoint.argtypes = [i64, vp, i32, i32, vp, vp, vp, vp]

    def conv(s, h):
        s = np.ascontiguousarray(s, np.complex64)
        h = np.ascontiguousarray(h, np.complex64)
        sq = h.ndim == 1
        h2 = h[None] if sq else h
        F, M = h2.shape
        y = np.empty((F, len(s) - M + 1), np.complex128)
        lib.ols_oracle_conv(len(s), s.ctypes.data, M, F, h2.ctypes.data, y.ctypes.data)
        return y[0] if sq else y

    def adjoint(s, h, g):
        s = np.ascontiguousarray(s, np.complex64)
        h = np.ascontiguousarray(h, np.complex64)
        sq = h.ndim == 1
        h2 = h[None] if sq else h
        g2 = np.ascontiguousarray(np.atleast_2d(g), np.complex128)
        F, M = h2.shape
        ds = np.empty(len(s), np.complex128)
        dh = np.empty((F, M), np.complex128)
        lib.ols_oracle_adjoint(len(s), s.ctypes.data, M, F, h2.ctypes.data, g2.ctypes.data,
                               ds.ctypes.data, dh.ctypes.data)
        return ds, (dh[0] if sq else dh)

    return conv, adjoint


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")
@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_planted_mistake(name):
    src = open(os.path.join(os.path.dirname(oracle.__file__), "ols_oracle.c")).read()
    old, new = MUTANTS[name]
    assert src.count(old) == 1, "mutation anchor not unique: " + name
    with tempfile.TemporaryDirectory() as d:
        cpath = os.path.join(d, "mut.c")
        with open(cpath, "w") as fh:
            fh.write(src.replace(old, new))
        so = os.path.join(d, "libmut.so")
        subprocess.run(["gcc", "-O1", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
                        "-std=c11", "-o", so, cpath], check=True)
        conv, adjoint = _bind(so)
        caught = []
        for pin in P.QUICK_PINS:
            try:
                pin(conv, adjoint)
            except AssertionError:
                caught.append(pin.__name__)
        assert caught, "no pin caught mutant " + name


REAL_MUTANTS = {
    "real_drop_last_tap": ("for (int32_t k = 0; k < M; ++k)\n        acc += (double)s[j + (int64_t)M - 1 - k]",
                           "for (int32_t k = 0; k < M - 1; ++k)\n        acc += (double)s[j + (int64_t)M - 1 - k]"),
    "real_off_by_one": ("acc += (double)s[j + (int64_t)M - 1 - k] * (double)hf[k];",
                        "acc += (double)s[j + (int64_t)M - 1 - k + (k > 0)] * (double)hf[k];"),
    "real_unflipped": ("acc += (double)s[j + (int64_t)M - 1 - k] * (double)hf[k];",
                       "acc += (double)s[j + k] * (double)hf[k];"),
}


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")
@pytest.mark.parametrize("name", sorted(REAL_MUTANTS))
def test_real_pins_catch_planted_mistake(name):
    src = open(os.path.join(os.path.dirname(oracle.__file__), "ols_oracle.c")).read()
    old, new = REAL_MUTANTS[name]
    assert src.count(old) == 1, "mutation anchor not unique: " + name
    with tempfile.TemporaryDirectory() as d:
        cpath = os.path.join(d, "mut.c")
        with open(cpath, "w") as fh:
            fh.write(src.replace(old, new))
        so = os.path.join(d, "libmut.so")
        subprocess.run(["gcc", "-O1", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
                        "-std=c11", "-o", so, cpath], check=True)
        lib = ctypes.CDLL(so)
        vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32
        lib.ols_oracle_conv_real.argtypes = [i64, vp, i32, i32, vp, vp]

        def conv_real(s, h):
            s = np.ascontiguousarray(s, np.float32)
            h = np.ascontiguousarray(h, np.float32)
            sq = h.ndim == 1
            h2 = h[None] if sq else h
            F, M = h2.shape
            y = np.empty((F, len(s) - M + 1), np.float64)
            lib.ols_oracle_conv_real(len(s), s.ctypes.data, M, F, h2.ctypes.data, y.ctypes.data)
            return y[0] if sq else y

        caught = []
        for pin in P.REAL_QUICK_PINS:
            try:
                pin(conv_real)
            except AssertionError:
                caught.append(pin.__name__)
        assert caught, "planted mistake %s passed every real pin" % name


@pytest.mark.parametrize("pin", P.POST_PINS)
def test_oracle_post_pin(pin):
    pin(oracle.power, oracle.derivative, oracle.conv)


def test_oracle_post_sampled_and_detect():
    g = np.random.Generator(np.random.PCG64(6))
    s = (g.uniform(-1, 1, 800) + 1j * g.uniform(-1, 1, 800)).astype(np.complex64)
    h = (g.normal(size=(3, 30)) + 1j * g.normal(size=(3, 30))).astype(np.complex64)
    d = oracle.derivative(s, h)
    fi = np.concatenate([g.integers(0, 3, 50), [0, 1, 2]])
    ji = np.concatenate([g.integers(0, d.shape[1], 50), [0, d.shape[1] - 1, 1]])
    assert np.array_equal(oracle.derivative_at(s, h, fi, ji), d[fi, ji])
    p = oracle.power(s, h)
    assert np.array_equal(oracle.power_at(s, h, fi, ji), p[fi, ji])
    thr = float(np.quantile(p, 0.99))
    f, j, pw = oracle.detect(s, h, thr)
    assert f.size == int(np.sum(p >= thr)) and np.all(pw >= thr) and np.array_equal(pw, p[f, j])
    with pytest.raises(ValueError):
        oracle.derivative(s[:30], h)          # Nout = 1: no derivative


POST_MUTANTS = {
    "deriv_no_half": ("const double scale = (hi - lo == 2) ? 0.5 : 1.0;", "const double scale = 1.0;"),
    "deriv_ends_halved": ("const double scale = (hi - lo == 2) ? 0.5 : 1.0;", "const double scale = 0.5;"),
    "deriv_sign": ("*out_re = (br - ar) * scale;\n    *out_im = (bi - ai) * scale;",
                   "*out_re = (ar - br) * scale;\n    *out_im = (ai - bi) * scale;"),
    "deriv_backward_only": ("const int64_t hi = (j == Nout - 1) ? j : j + 1;", "const int64_t hi = j;"),
    "power_minus": ("p[idx] = yr * yr + yi * yi;", "p[idx] = yr * yr - yi * yi;"),
}


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")
@pytest.mark.parametrize("name", sorted(POST_MUTANTS))
def test_post_pins_catch_planted_mistake(name):
    src = open(os.path.join(os.path.dirname(oracle.__file__), "ols_oracle.c")).read()
    old, new = POST_MUTANTS[name]
    assert src.count(old) == 1, "mutation anchor not unique: " + name
    with tempfile.TemporaryDirectory() as d:
        cpath = os.path.join(d, "mut.c")
        with open(cpath, "w") as fh:
            fh.write(src.replace(old, new))
        so = os.path.join(d, "libmut.so")
        subprocess.run(["gcc", "-O1", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
                        "-std=c11", "-o", so, cpath], check=True)
        lib = ctypes.CDLL(so)
        vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32
        for fn in ("ols_oracle_power", "ols_oracle_derivative", "ols_oracle_conv"):
            getattr(lib, fn).argtypes = [i64, vp, i32, i32, vp, vp]

        def call(fn, dtype):
            def run(s, h):
                s = np.ascontiguousarray(s, np.complex64)
                h = np.ascontiguousarray(h, np.complex64)
                sq = h.ndim == 1
                h2 = h[None] if sq else h
                F, M = h2.shape
                out = np.empty((F, len(s) - M + 1), dtype)
                assert getattr(lib, fn)(len(s), s.ctypes.data, M, F, h2.ctypes.data, out.ctypes.data) == 0
                return out[0] if sq else out
            return run

        power, deriv, conv = (call("ols_oracle_power", np.float64), call("ols_oracle_derivative", np.complex128),
                              call("ols_oracle_conv", np.complex128))
        caught = []
        for pin in P.POST_PINS:
            try:
                pin(power, deriv, conv)
            except AssertionError:
                caught.append(pin.__name__)
        assert caught, "planted mistake %s passed every post-processing pin" % name


def test_error_metric_floor():
    """The parity metric: without a floor it is the per-stream relative L2
    error; the floor only replaces a denominator below it; stream_scale is
    the expected stream norm of a white signal (within a few percent on
    long streams, so the floor leaves their error unchanged)."""
    g = np.random.Generator(np.random.PCG64(3))
    y_ref = g.normal(size=(3, 50)) + 1j * g.normal(size=(3, 50))
    y = y_ref + 1e-3 * (g.normal(size=(3, 50)) + 0j)
    plain = max(np.linalg.norm(y[f] - y_ref[f]) / np.linalg.norm(y_ref[f]) for f in range(3))
    assert oracle.max_stream_rel_l2(y, y_ref) == pytest.approx(plain, rel=1e-12)
    assert oracle.max_stream_rel_l2(y, y_ref, floor=[0.0, 0.0, 0.0]) == pytest.approx(plain, rel=1e-12)
    big = [1e6] * 3
    assert oracle.max_stream_rel_l2(y, y_ref, floor=big) == pytest.approx(
        max(np.linalg.norm(y[f] - y_ref[f]) for f in range(3)) / 1e6, rel=1e-12)
    Ns, M, F = 200_000, 33, 2
    s = (g.normal(size=Ns) + 1j * g.normal(size=Ns)).astype(np.complex64)
    h = (g.normal(size=(F, M)) + 1j * g.normal(size=(F, M))).astype(np.complex64)
    yr = oracle.conv(s, h)
    sc = oracle.stream_scale(s, h, Ns - M + 1)
    assert sc.shape == (F,)
    for f in range(F):
        assert np.linalg.norm(yr[f]) == pytest.approx(sc[f], rel=0.05)


@pytest.mark.parametrize("pin", P.PEAK_PINS)
def test_oracle_peak_pin(pin):
    if pin is P.pin_peaks_match_scipy:
        pytest.importorskip("scipy.signal")
    pin(oracle.peak_mask, oracle.power)


PEAK_MUTANTS = {
    "peak_left_not_strict": ("if (j > 0 && !(pf[j] > pf[j - 1])) peak = 0;",
                             "if (j > 0 && !(pf[j] >= pf[j - 1])) peak = 0;"),
    "peak_right_strict": ("if (j < Nout - 1 && !(pf[j] >= pf[j + 1])) peak = 0;",
                          "if (j < Nout - 1 && !(pf[j] > pf[j + 1])) peak = 0;"),
    "peak_threshold_strict": ("int peak = pf[j] >= threshold;", "int peak = pf[j] > threshold;"),
    "peak_first_output_never": ("if (j > 0 && !(pf[j] > pf[j - 1])) peak = 0;",
                                "if (j == 0 || !(pf[j] > pf[j - 1])) peak = 0;"),
    "peak_last_output_never": ("if (j < Nout - 1 && !(pf[j] >= pf[j + 1])) peak = 0;",
                               "if (j == Nout - 1 || !(pf[j] >= pf[j + 1])) peak = 0;"),
    "peak_minimum": ("if (j > 0 && !(pf[j] > pf[j - 1])) peak = 0;\n            "
                     "if (j < Nout - 1 && !(pf[j] >= pf[j + 1])) peak = 0;",
                     "if (j > 0 && !(pf[j] < pf[j - 1])) peak = 0;\n            "
                     "if (j < Nout - 1 && !(pf[j] <= pf[j + 1])) peak = 0;"),
}


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")
@pytest.mark.parametrize("name", sorted(PEAK_MUTANTS))
def test_peak_pins_catch_planted_mistake(name):
    src = open(os.path.join(os.path.dirname(oracle.__file__), "ols_oracle.c")).read()
    old, new = PEAK_MUTANTS[name]
    assert src.count(old) == 1, "mutation anchor not unique: " + name
    with tempfile.TemporaryDirectory() as d:
        cpath = os.path.join(d, "mut.c")
        with open(cpath, "w") as fh:
            fh.write(src.replace(old, new))
        so = os.path.join(d, "libmut.so")
        subprocess.run(["gcc", "-O1", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
                        "-std=c11", "-o", so, cpath], check=True)
        lib = ctypes.CDLL(so)
        lib.ols_oracle_peak_mask.argtypes = [ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p, ctypes.c_double,
                                             ctypes.c_void_p]
        lib.ols_oracle_peak_mask.restype = ctypes.c_int

        def mask(p, thr):
            p = np.ascontiguousarray(p, dtype=np.float64)
            sq = p.ndim == 1
            p2 = p[None, :] if sq else p
            m = np.zeros(p2.shape, np.uint8)
            assert lib.ols_oracle_peak_mask(p2.shape[0], p2.shape[1], p2.ctypes.data, float(thr), m.ctypes.data) == 0
            return m.astype(bool)[0] if sq else m.astype(bool)

        caught = []
        for pin in P.PEAK_PINS:
            if pin is P.pin_peaks_match_scipy and importlib.util.find_spec("scipy") is None:
                continue
            try:
                pin(mask, oracle.power)
            except AssertionError:
                caught.append(pin.__name__)
        assert caught, "planted mistake %s passed every peak pin" % name
