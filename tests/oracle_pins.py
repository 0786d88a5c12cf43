"""Checks that pin the FP64 oracle to facts fixed by the paper and by
mathematics, independent of the oracle's own code.

Each ``pin_*`` function takes the two oracle entry points as callables
(``conv(s, h) -> y`` and ``adjoint(s, h, g) -> (ds, dh)``) and raises
AssertionError on a mismatch, so the same checks run against the real oracle
(tests/test_oracle_pins.py) and against deliberately broken copies of it
(the mutation test), proving that each plausible mistake is caught.
"""
from __future__ import annotations

import math
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


# ----------------------------------------------------------------- fixtures
def read_golden(name):
    """Parse a tests/golden/*.txt fixture into a list of dicts of arrays."""
    cases, cur = [], {}
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                if not line and cur:
                    cases.append(cur)
                    cur = {}
                continue
            key, val = (x.strip() for x in line.split("=", 1))
            if key == "case":
                cur["case"] = val
            else:
                cur[key] = np.array([complex(v) for v in val.split()], dtype=np.complex128)
    if cur:
        cases.append(cur)
    return cases


def _c64(x):
    return np.asarray(x, dtype=np.complex64)


def naive_dft_matrix(P):
    """Explicit P x P DFT matrix exp(-2 pi i n k / P), index product reduced mod P."""
    n = np.arange(P)
    e = (np.outer(n, n) % P).astype(np.float64)
    return np.exp(-2j * math.pi * e / P)


def quantized(g, shape, step):
    """Complex values on a grid of ``step`` in [-1, 1] (exact in FP32)."""
    q = np.round(g.uniform(-1, 1, size=shape) / step) * step
    r = np.round(g.uniform(-1, 1, size=shape) / step) * step
    return (q + 1j * r).astype(np.complex64)


# ----------------------------------------------------------------- pins
def pin_golden_conv(conv, adjoint=None):
    """Hand-worked cases of Eq. 1 (tests/golden/hand_conv.txt): exact."""
    for c in read_golden("hand_conv.txt"):
        y = conv(_c64(c["s"]), _c64(c["h"]))
        assert np.array_equal(y, c["y"]), (c["case"], y, c["y"])


def pin_golden_adjoint(conv, adjoint):
    """Hand-worked adjoint cases (tests/golden/hand_adjoint.txt): exact."""
    for c in read_golden("hand_adjoint.txt"):
        ds, dh = adjoint(_c64(c["s"]), _c64(c["h"]), c["g"])
        assert np.array_equal(ds, c["ds"]), (c["case"], ds, c["ds"])
        assert np.array_equal(np.ravel(dh), c["dh"]), (c["case"], dh, c["dh"])


def pin_bruteforce_dft(conv, adjoint=None, seed=11):
    """Linear convolution equals circular convolution once both operands are
    zero-padded to P >= Ns + M - 1 (Sec. 1, Eq. 2 and its padding rule); the
    circular convolution is evaluated with explicit O(P^2) DFT matrices.  The
    valid outputs are entries M-1 .. Ns-1 of the full linear result."""
    g = np.random.Generator(np.random.PCG64(seed))
    for Ns in (1, 2, 3, 5, 8, 17, 31, 64):
        for M in (1, 2, 3, 4, 7, 16):
            if M > Ns:
                continue
            F = 1 + (Ns + M) % 3
            s = _c64(g.normal(size=Ns) + 1j * g.normal(size=Ns))
            h = _c64(g.normal(size=(F, M)) + 1j * g.normal(size=(F, M)))
            P = Ns + M - 1
            W = naive_dft_matrix(P)
            Winv = np.conj(W) / P
            sp = np.zeros(P, np.complex128)
            sp[:Ns] = s
            S = W @ sp
            y = conv(s, h)
            assert y.shape == (F, Ns - M + 1)
            for f in range(F):
                hp = np.zeros(P, np.complex128)
                hp[:M] = h[f]
                full = Winv @ (S * (W @ hp))
                ref = full[M - 1:Ns]
                err = np.max(np.abs(y[f] - ref)) / max(1.0, np.max(np.abs(ref)))
                assert err < 1e-13, (Ns, M, f, err)


def pin_fft_fullconv(conv, adjoint=None, seed=12):
    """Full-length zero-padded FFT convolution (Sec. 1: padding to at least
    Ns + M - 1 makes the circular result linear), via numpy's FFT."""
    g = np.random.Generator(np.random.PCG64(seed))
    for (Ns, M, F) in ((4096, 64, 1), (4096, 129, 3), (4096, 257, 2)):
        s = _c64(g.uniform(-1, 1, Ns) + 1j * g.uniform(-1, 1, Ns))
        h = _c64(g.normal(size=(F, M)) + 1j * g.normal(size=(F, M)))
        P = 1 << int(math.ceil(math.log2(Ns + M - 1)))
        S = np.fft.fft(s.astype(np.complex128), P)
        y = conv(s, h)
        for f in range(F):
            full = np.fft.ifft(S * np.fft.fft(h[f].astype(np.complex128), P))
            ref = full[M - 1:Ns]
            err = np.linalg.norm(y[f] - ref) / np.linalg.norm(ref)
            assert err < 1e-12, (Ns, M, f, err)


def pin_delta_shift(conv, adjoint=None, seed=13):
    """h = e_d (unit tap at d) gives y[j] = s[j + M - 1 - d], exactly."""
    g = np.random.Generator(np.random.PCG64(seed))
    n = np.arange(300)
    s_int = _c64((n % 1024) + 1j * ((7 * n) % 1024))
    s_rand = _c64(g.uniform(-1, 1, 300) + 1j * g.uniform(-1, 1, 300))
    for s in (s_int, s_rand):
        for M in (1, 2, 5, 64):
            for d in sorted({0, M // 2, M - 1}):
                h = np.zeros(M, np.complex64)
                h[d] = 1
                y = conv(s, h)
                ref = s[M - 1 - d: len(s) - d].astype(np.complex128)
                assert np.array_equal(y, ref), (M, d)


def pin_linearity(conv, adjoint=None, seed=14):
    """Convolution is linear in s and in h; a bank of filters is the stack of
    the single-filter results.  Inputs sit on a 2^-8 grid so the scaled sums
    are exact in FP32."""
    g = np.random.Generator(np.random.PCG64(seed))
    Ns, M = 200, 9
    s1, s2 = quantized(g, Ns, 2.0 ** -8), quantized(g, Ns, 2.0 ** -8)
    h1, h2 = quantized(g, M, 2.0 ** -8), quantized(g, M, 2.0 ** -8)
    a, b = 2.0, -0.5
    lhs = conv(_c64(a * s1.astype(np.complex128) + b * s2), h1)
    rhs = a * conv(s1, h1) + b * conv(s2, h1)
    assert np.max(np.abs(lhs - rhs)) <= 1e-13 * np.max(np.abs(rhs))
    lhs = conv(s1, _c64(a * h1.astype(np.complex128) + b * h2))
    rhs = a * conv(s1, h1) + b * conv(s1, h2)
    assert np.max(np.abs(lhs - rhs)) <= 1e-13 * np.max(np.abs(rhs))
    bank = conv(s1, np.stack([h1, h2]))
    assert np.array_equal(bank[0], conv(s1, h1)) and np.array_equal(bank[1], conv(s1, h2))


def pin_closed_forms(conv, adjoint=None, seed=15):
    """Complex exponentials are eigenfunctions: s[n] = z^n with |z| = 1 gives
    y[j] = z^(j+M-1) * sum_k h[k] z^(-k).  z = i and z = -1 are exact in FP32;
    z = 1 (a constant signal) gives sum_k h[k] everywhere."""
    g = np.random.Generator(np.random.PCG64(seed))
    Ns, M = 257, 13
    h = _c64(g.normal(size=M) + 1j * g.normal(size=M))
    hd = h.astype(np.complex128)
    n = np.arange(Ns)
    for z, pw in ((1j, lambda e: 1j ** (e % 4)), (-1.0, lambda e: (-1.0) ** (e % 2)),
                  (1.0, lambda e: np.ones_like(e, dtype=np.float64))):
        s = _c64(pw(n))
        Hz = sum(hd[k] * np.conj(pw(np.array(k))) for k in range(M))
        j = np.arange(Ns - M + 1)
        ref = pw(j + M - 1) * Hz
        y = conv(s, h)
        assert np.max(np.abs(y - ref)) < 1e-12, z


def pin_adjoint_dot(conv, adjoint, seed=16):
    """The adjoint satisfies Re<g, y(s, h)> = Re<ds, s> = Re<dh, h> (a linear
    map and its adjoint); convention grad = dL/dRe + i dL/dIm."""
    g = np.random.Generator(np.random.PCG64(seed))
    for (Ns, M, F) in ((50, 7, 3), (300, 64, 2), (64, 64, 1), (33, 1, 2)):
        s = _c64(g.normal(size=Ns) + 1j * g.normal(size=Ns))
        h = _c64(g.normal(size=(F, M)) + 1j * g.normal(size=(F, M)))
        gr = g.normal(size=(F, Ns - M + 1)) + 1j * g.normal(size=(F, Ns - M + 1))
        y = conv(s, h)
        ds, dh = adjoint(s, h, gr)
        lhs = np.real(np.vdot(gr, y))
        r1 = np.real(np.vdot(ds, s.astype(np.complex128)))
        r2 = np.real(np.vdot(dh, h.astype(np.complex128)))
        scale = np.linalg.norm(gr) * np.linalg.norm(y) + 1.0
        assert abs(lhs - r1) < 1e-12 * scale, (Ns, M, F, lhs, r1)
        assert abs(lhs - r2) < 1e-12 * scale, (Ns, M, F, lhs, r2)


def weighted_power_loss(y, w):
    """L = sum_f sum_j w[j] |y_f[j]|^2 in FP64."""
    y = np.atleast_2d(y)
    return float(np.sum(w[None, :] * (y.real ** 2 + y.imag ** 2)))


def pin_adjoint_finite_difference(conv, adjoint, seed=17, Ns=4096, F=16, M=129,
                                  h_filters=(0, 7, 15), n_s=512):
    """FP64 central differences of L = sum w|y|^2 (quadratic, so the central
    difference is exact up to rounding) against ds, dh with g = 2 w y.
    Inputs lie on a 2^-10 grid and the step is 2^-6, so every perturbed input
    is exact in FP32."""
    g = np.random.Generator(np.random.PCG64(seed))
    s = quantized(g, Ns, 2.0 ** -10)
    h = quantized(g, (F, M), 2.0 ** -10)
    w = g.uniform(0, 1, Ns - M + 1)
    y = conv(s, h)
    grad_y = 2.0 * w[None, :] * y
    ds, dh = adjoint(s, h, grad_y)
    eps = 2.0 ** -6
    worst = 0.0
    # every real coordinate of the chosen filters
    for f in h_filters:
        for k in range(M):
            for unit in (1.0, 1j):
                hp = h[f].astype(np.complex128).copy()
                hm = hp.copy()
                hp[k] += eps * unit
                hm[k] -= eps * unit
                lp = weighted_power_loss(conv(s, _c64(hp)), w)
                lm = weighted_power_loss(conv(s, _c64(hm)), w)
                fd = (lp - lm) / (2 * eps)
                an = dh[f, k].real if unit == 1.0 else dh[f, k].imag
                worst = max(worst, abs(fd - an) / (abs(an) + 1e-3 * np.max(np.abs(dh))))
    # seeded coordinates of s; only outputs j in [m-M+1, m] depend on s[m]
    Nout = Ns - M + 1
    ms = np.concatenate([[0, 1, M - 1, M, Ns // 2, Ns - M, Ns - 2, Ns - 1],
                         g.integers(0, Ns, size=max(0, n_s - 8))])
    sd = s.astype(np.complex128)
    for m in ms:
        j0, j1 = max(0, m - M + 1), min(Nout - 1, m)
        for unit in (1.0, 1j):
            sp = sd[j0:j1 + M].copy()
            sm = sp.copy()
            sp[m - j0] += eps * unit
            sm[m - j0] -= eps * unit
            lp = weighted_power_loss(conv(_c64(sp), h), w[j0:j1 + 1])
            lm = weighted_power_loss(conv(_c64(sm), h), w[j0:j1 + 1])
            fd = (lp - lm) / (2 * eps)
            an = ds[m].real if unit == 1.0 else ds[m].imag
            worst = max(worst, abs(fd - an) / (abs(an) + 1e-3 * np.max(np.abs(ds))))
    assert worst < 1e-9, worst
    return worst


QUICK_PINS = (pin_golden_conv, pin_golden_adjoint, pin_bruteforce_dft, pin_delta_shift,
              pin_linearity, pin_closed_forms, pin_adjoint_dot)


# ------------------------------------------------------ real-to-real (R2R) form
# The paper's second OLS variant (Sec. 3.4) convolves real signals with real
# filters; its exact result is Eq. 1's valid part on real data.  Each pin
# takes conv_real(s, h) -> y (float64) on float32 inputs.

def pin_real_bruteforce(conv_real, seed=21):
    """Against numpy's direct 'valid' convolution in FP64 (np.convolve flips h,
    as Eq. 1 does), over shapes including M = 1 and M = Ns."""
    g = np.random.Generator(np.random.PCG64(seed))
    for (Ns, M, F) in ((1, 1, 1), (40, 1, 2), (64, 7, 3), (37, 37, 2), (300, 33, 2), (129, 64, 1)):
        s = g.uniform(-1, 1, Ns).astype(np.float32)
        h = g.normal(size=(F, M)).astype(np.float32)
        y = conv_real(s, h)
        for f in range(F):
            ref = np.convolve(s.astype(np.float64), h[f].astype(np.float64), mode="valid")
            assert y[f].shape == ref.shape
            assert np.max(np.abs(y[f] - ref)) <= 1e-13 * (np.max(np.abs(ref)) + 1.0), (Ns, M, f)


def pin_real_delta_shift(conv_real, seed=22):
    """h = e_d gives y[j] = s[j + M - 1 - d], exactly."""
    g = np.random.Generator(np.random.PCG64(seed))
    s = g.uniform(-1, 1, 300).astype(np.float32)
    for M in (1, 2, 5, 64):
        for d in sorted({0, M // 2, M - 1}):
            h = np.zeros(M, np.float32)
            h[d] = 1
            assert np.array_equal(conv_real(s, h), s[M - 1 - d: len(s) - d].astype(np.float64)), (M, d)


def pin_real_closed_forms(conv_real, seed=23):
    """A constant signal gives sum_k h[k]; s[n] = (-1)^n gives
    (-1)^(j+M-1) sum_k (-1)^k h[k] (both exact sums of FP32 taps in FP64
    up to rounding of the reference)."""
    g = np.random.Generator(np.random.PCG64(seed))
    Ns, M = 257, 13
    h = g.normal(size=M).astype(np.float32)
    hd = h.astype(np.float64)
    j = np.arange(Ns - M + 1)
    y = conv_real(np.ones(Ns, np.float32), h)
    assert np.max(np.abs(y - hd.sum())) < 1e-12
    alt = ((-1.0) ** np.arange(Ns)).astype(np.float32)
    ref = ((-1.0) ** (j + M - 1)) * np.sum(hd * (-1.0) ** np.arange(M))
    assert np.max(np.abs(conv_real(alt, h) - ref)) < 1e-12


def pin_real_is_complex_on_real_data(conv_real, conv, seed=24):
    """On real data the complex oracle's sums reduce term by term to the real
    ones (every imaginary product is an exact zero), so the real parts agree
    bit for bit and the imaginary parts are zero."""
    g = np.random.Generator(np.random.PCG64(seed))
    s = g.uniform(-1, 1, 500).astype(np.float32)
    h = g.normal(size=(3, 41)).astype(np.float32)
    yc = conv(s.astype(np.complex64), h.astype(np.complex64))
    assert np.array_equal(yc.real, conv_real(s, h)) and not np.any(yc.imag)


REAL_QUICK_PINS = (pin_real_bruteforce, pin_real_delta_shift, pin_real_closed_forms)


# ------------------------------------------------- post-processing of the output
# Sec. 4.3: per-element post-processing (the power spectrum) and non-local
# post-processing (the numerical derivative of the convolved signal; the
# paper gives no formula, the reading is the central difference with
# one-sided ends).  Each pin takes (power, derivative, conv).

def pin_derivative_is_numpy_gradient(power, derivative, conv, seed=31):
    """numpy.gradient with unit spacing is the same difference scheme (central
    inside, first-order one-sided at both ends); it is an independent
    implementation of the reading."""
    g = np.random.Generator(np.random.PCG64(seed))
    for (Ns, M, F) in ((2, 1, 1), (3, 2, 2), (40, 7, 3), (300, 33, 2)):
        s = (g.uniform(-1, 1, Ns) + 1j * g.uniform(-1, 1, Ns)).astype(np.complex64)
        h = (g.normal(size=(F, M)) + 1j * g.normal(size=(F, M))).astype(np.complex64)
        d = derivative(s, h)
        ref = np.gradient(conv(s, h), axis=1)
        assert d.shape == ref.shape
        assert np.max(np.abs(d - ref)) <= 1e-13 * (np.max(np.abs(ref)) + 1.0), (Ns, M, F)


def pin_derivative_ramp(power, derivative, conv):
    """s[n] = n (exact in FP32) with a delta filter gives y[j] = j + M - 1 - d,
    whose derivative is exactly 1 everywhere, ends included."""
    Ns = 500
    s = np.arange(Ns).astype(np.complex64)
    for M in (1, 2, 17):
        for dpos in sorted({0, M - 1}):
            h = np.zeros(M, np.complex64)
            h[dpos] = 1
            assert np.array_equal(derivative(s, h), np.ones(Ns - M + 1, np.complex128)), (M, dpos)


def pin_derivative_closed_form(power, derivative, conv, seed=32):
    """s[n] = exp(i w n) gives y[j] = A exp(i w j), A = exp(i w (M-1)) sum_k h[k]
    exp(-i w k); its derivative is y[j] i sin(w) inside, y[j] (exp(i w) - 1) at
    j = 0 and y[j] (1 - exp(-i w)) at the last output.  The power is |A|^2."""
    g = np.random.Generator(np.random.PCG64(seed))
    Ns, M, w = 400, 9, 0.3
    n = np.arange(Ns)
    s = np.exp(1j * w * n).astype(np.complex64)
    h = (g.normal(size=M) + 1j * g.normal(size=M)).astype(np.complex64)
    # FP32-rounded input: the closed form uses the rounded samples' exact phases only approximately,
    # so compare at the rounding level of complex64 (~1e-7 relative)
    k = np.arange(M)
    A = np.exp(1j * w * (M - 1)) * np.sum(h.astype(np.complex128) * np.exp(-1j * w * k))
    j = np.arange(Ns - M + 1)
    y = A * np.exp(1j * w * j)
    ref = y * 1j * np.sin(w)
    ref[0] = y[0] * (np.exp(1j * w) - 1)
    ref[-1] = y[-1] * (1 - np.exp(-1j * w))
    d = derivative(s, h)
    assert np.max(np.abs(d - ref)) <= 2e-6 * np.abs(A)
    assert np.max(np.abs(power(s, h) - np.abs(A) ** 2)) <= 2e-6 * np.abs(A) ** 2


def pin_power_is_squared_magnitude(power, derivative, conv, seed=33):
    """p = |y|^2 = Re(y)^2 + Im(y)^2 of the same FP64 outputs, element by element."""
    g = np.random.Generator(np.random.PCG64(seed))
    s = (g.uniform(-1, 1, 700) + 1j * g.uniform(-1, 1, 700)).astype(np.complex64)
    h = (g.normal(size=(3, 21)) + 1j * g.normal(size=(3, 21))).astype(np.complex64)
    y = conv(s, h)
    assert np.array_equal(power(s, h), y.real * y.real + y.imag * y.imag)
    # a delta filter returns |s|^2 of the shifted samples
    e = np.zeros(5, np.complex64)
    e[2] = 1
    sd = s.astype(np.complex128)[2: 700 - 2]
    assert np.array_equal(power(s, e), sd.real * sd.real + sd.imag * sd.imag)


POST_PINS = (pin_derivative_is_numpy_gradient, pin_derivative_ramp, pin_derivative_closed_form,
             pin_power_is_squared_magnitude)


# -- peak finding (Sec. 4.4), pinned through ``peak_mask(p, threshold)`` ------

def pin_peaks_match_scipy(peak_mask, power, seed=41):
    """On tie-free powers of random convolutions, the interior peaks are
    exactly scipy.signal.find_peaks with a height bound (a library routine for
    local maxima; it never reports the two ends, so those are left out)."""
    from scipy.signal import find_peaks
    g = np.random.Generator(np.random.PCG64(seed))
    s = (g.uniform(-1, 1, 3000) + 1j * g.uniform(-1, 1, 3000)).astype(np.complex64)
    h = (g.normal(size=(3, 17)) + 1j * g.normal(size=(3, 17))).astype(np.complex64)
    p = power(s, h)
    for f in range(p.shape[0]):
        assert np.unique(p[f]).size == p.shape[1]           # no ties
        thr = float(np.quantile(p[f], 0.6))
        m = peak_mask(p[f], thr)
        ref, _ = find_peaks(p[f], height=thr)
        assert np.array_equal(np.nonzero(m[1:-1])[0] + 1, ref)


def pin_peaks_spike_train(peak_mask, power, M=7):
    """Delta filters on a spike train (closed form: y_f[j] = s[j + M-1 - d_f],
    so the powers are the squared spikes): a spike on the first and on the
    last output of the stream, a spike exactly at the threshold, a pair of
    equal spikes (one peak, at the left one) and a spike below the
    threshold."""
    Nout = 60
    spikes = {0: 9.0, 10: 4.0, 20: 5.0, 21: 5.0, 33: 3.0, 45: 6.0, Nout - 1: 7.0}
    thr = 16.0                                            # = 4^2: the spike at 10 sits on it
    want = {0, 10, 20, 45, Nout - 1}                      # 33 (power 9) is below it
    for d in (0, M // 2, M - 1):
        s = np.full(Nout + M - 1, 0.5, np.complex64)      # a floor of power 0.25
        for j, a in spikes.items():
            s[j + M - 1 - d] = a
        h = np.zeros((1, M), np.complex64)
        h[0, d] = 1
        p = power(s, h)[0]
        assert set(np.nonzero(peak_mask(p, thr))[0].tolist()) == want, d


def pin_peaks_ramps(peak_mask, power):
    """A rising power has its only peak on the last output, a falling one on
    the first; a flat one on the first (the left end of a run of equals)."""
    n = np.arange(1, 41, dtype=np.float64)
    for p, j in ((n, 39), (n[::-1].copy(), 0), (np.full(40, 3.0), 0)):
        assert np.nonzero(peak_mask(p, 0.5))[0].tolist() == [j]
        assert not peak_mask(p, 1e9).any()
    one = np.array([2.0])
    assert peak_mask(one, 2.0).tolist() == [True] and peak_mask(one, 2.5).tolist() == [False]


PEAK_PINS = (pin_peaks_match_scipy, pin_peaks_spike_train, pin_peaks_ramps)
