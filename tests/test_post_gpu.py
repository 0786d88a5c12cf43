"""Parity of the fused post-processing kernels (power, detection, derivative of
the convolved output, Sec. 4.3) through the C ABI with the FP64 oracle.

Tolerances, derived from the FP32 bar of the convolution (relative L2 error
of y <= 2e-6 per stream):
* power p = |y|^2: relative error of p is about twice that of y, so
  max over streams ||p - p_ref|| / ||p_ref|| <= 4e-6;
* derivative: each d[j] is a difference of two outputs, so its error is
  bounded by that of y: max over streams ||d - d_ref|| / ||y_ref|| <= 2e-6
  (relative to the convolved signal, since d can be much smaller than y);
* detection: the same power, so the candidate sets agree except for powers
  within 1e-5 (relative) of the threshold, and each reported power is within
  4e-6 of the oracle's.
Segment bookkeeping of the derivative (segments advance by L-2) is checked
bit-exactly with delta filters on integer-valued signals.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from paper_1910_01972_gb300 import Plan, _native, decode_candidates
from paper_1910_01972_gb300 import build as _build

pytestmark = pytest.mark.gpu
TOL_Y = 2e-6
TOL_P = 4e-6


@pytest.fixture(scope="module", autouse=True)
def built():
    _build.build()
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")


def to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def rand_inputs(seed, Ns, F, M, window=False):
    g = np.random.Generator(np.random.PCG64(seed))
    return synth.signal(g, Ns), synth.filters(g, F, M, window=window)


def make_plan(h, N):
    plan = Plan(h.shape[1], h.shape[0], N)
    plan.set_filters(to_dev(h))
    return plan


CASES = [
    # (N, M, F, Ns)
    (512, 64, 1, 65536),
    (2048, 257, 8, 40_000),
    (256, 33, 3, 10_000),
    (256, 254, 2, 3_000),      # L = 3: the derivative's step is 1
    (512, 1, 2, 5_000),
    (1024, 129, 5, 50_001),
    (4096, 512, 3, 70_000),
    (8192, 1025, 2, 100_000),
    (1024, 100, 3, 1_000),     # Ns < N
    (2048, 257, 2, 258),       # Nout = 2
]


@pytest.mark.parametrize("N,M,F,Ns", CASES)
def test_power_parity(N, M, F, Ns):
    s, h = rand_inputs(N + 3 * M + F, Ns, F, M)
    plan = make_plan(h, N)
    p = plan.convolve_power(to_dev(s)).cpu().numpy()
    plan.close()
    p_ref = oracle.power(s, h)
    assert p.shape == p_ref.shape and p.dtype == np.float32
    assert oracle.max_stream_rel_l2(p, p_ref) <= TOL_P


@pytest.mark.parametrize("N,M,F,Ns", CASES)
def test_derivative_parity(N, M, F, Ns):
    s, h = rand_inputs(N + 5 * M + F, Ns, F, M)
    plan = make_plan(h, N)
    d = plan.convolve_derivative(to_dev(s)).cpu().numpy()
    plan.close()
    d_ref = oracle.derivative(s, h)
    y_ref = oracle.conv(s, h)
    assert d.shape == d_ref.shape
    worst = max(np.linalg.norm(d[f] - d_ref[f]) / np.linalg.norm(y_ref[f]) for f in range(F))
    assert worst <= TOL_Y


@pytest.mark.parametrize("N", [256, 2048, 8192])
@pytest.mark.parametrize("M", [1, 37, 250])
def test_derivative_delta_filters_bit_exact(N, M):
    """Delta filters on an integer-valued signal: every derivative is a
    multiple of 1/2 and must round back exactly, which pins the shifted
    segment starts (step L-2, one output early), both one-sided ends and the
    ragged tail."""
    Ns = 3 * N + 123
    n = np.arange(Ns)
    s = (((n * n) % 1031) + 1j * ((7 * n) % 1024)).astype(np.complex64)
    ds = sorted({0, M // 2, M - 1})
    h = np.zeros((len(ds), M), np.complex64)
    for i, dpos in enumerate(ds):
        h[i, dpos] = 1.0
    plan = make_plan(h, N)
    d = plan.convolve_derivative(to_dev(s)).cpu().numpy()
    plan.close()
    for i, dpos in enumerate(ds):
        y = s[M - 1 - dpos: Ns - dpos].astype(np.complex128)
        ref = np.gradient(y)
        got2 = np.round(2 * d[i].real) + 1j * np.round(2 * d[i].imag)
        assert np.array_equal(got2, 2 * ref), (N, M, dpos)


def test_detection_matches_oracle_candidates():
    M, F, N, Ns = 129, 6, 1024, 60_000
    s, h = rand_inputs(41, Ns, F, M)
    p_ref = oracle.power(s, h)
    thr = float(np.quantile(p_ref, 0.999))
    plan = make_plan(h, N)
    rec, cnt = plan.convolve_detect(to_dev(s), thr, capacity=4096)
    torch.cuda.synchronize()
    count = int(cnt.item())
    f, j, pw = decode_candidates(rec, count)
    plan.close()
    got = set(zip(f.tolist(), j.tolist()))
    assert len(got) == count <= 4096                   # no duplicates, nothing dropped
    band = 1e-5 * thr
    must = {(a, b) for a, b in zip(*np.nonzero(p_ref >= thr + band))}
    may = {(a, b) for a, b in zip(*np.nonzero(p_ref >= thr - band))}
    assert must <= got <= may
    assert np.all(np.abs(pw - p_ref[f, j]) <= TOL_P * p_ref[f, j])


def test_detection_capacity_overflow_reports_total():
    M, F, N, Ns = 65, 3, 512, 20_000
    s, h = rand_inputs(42, Ns, F, M)
    p_ref = oracle.power(s, h)
    thr = float(np.quantile(p_ref, 0.9))
    plan = make_plan(h, N)
    rec, cnt = plan.convolve_detect(to_dev(s), thr, capacity=100)
    torch.cuda.synchronize()
    count = int(cnt.item())
    band = 1e-5 * thr
    assert int(np.sum(p_ref >= thr + band)) <= count <= int(np.sum(p_ref >= thr - band))
    f, j, pw = decode_candidates(rec, count)
    assert f.size == 100
    assert np.all(p_ref[f, j] >= thr - band)
    # a second call on the same counter starts again from zero
    rec2, cnt2 = plan.convolve_detect(to_dev(s), thr, capacity=0)
    torch.cuda.synchronize()
    assert int(cnt2.item()) == count
    plan.close()


def test_full_size_bank_sampled():
    """Power and derivative of the benchmark's filter bank (Ns = 2^23, F = 32,
    M = 257, N = 2048) at sampled outputs, including segment boundaries of
    both segmentations and both ends."""
    cfg = synth.PLAIN_BANK
    s, h = synth.plain_inputs(cfg)
    plan = make_plan(h, cfg.N)
    sd = to_dev(s)
    q = plan.query(cfg.Ns)
    Nout, L = q["Nout"], q["L"]
    g = np.random.Generator(np.random.PCG64(12))
    b = np.concatenate([np.arange(1, 40) * L, np.arange(1, 40) * (L - 2)])
    ej = np.concatenate([[0, 1, Nout - 1, Nout - 2], b - 1, b, b + 1])
    ji = np.concatenate([g.integers(0, Nout, 6000), ej])
    fi = np.concatenate([g.integers(0, cfg.F, 6000), np.arange(ej.size) % cfg.F])
    fit, jit = torch.from_numpy(fi).cuda(), torch.from_numpy(ji).cuda()
    p = plan.convolve_power(sd)
    got_p = p[fit, jit].cpu().numpy().astype(np.float64)
    del p
    ref_p = oracle.power_at(s, h, fi, ji)
    assert np.linalg.norm(got_p - ref_p) / np.linalg.norm(ref_p) <= TOL_P
    d = plan.convolve_derivative(sd)
    got_d = d[fit, jit].cpu().numpy()
    del d
    ref_d = oracle.derivative_at(s, h, fi, ji)
    ref_y = oracle.conv_at(s, h, fi, ji)
    assert np.linalg.norm(got_d - ref_d) / np.linalg.norm(ref_y) <= TOL_Y
    plan.close()


def test_post_entry_points_check_arguments():
    st = torch.cuda.current_stream().cuda_stream
    s = to_dev(np.zeros(300, np.complex64))
    out = torch.empty(600, dtype=torch.float32, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    h = to_dev(np.ones((1, 255), np.complex64))
    p = Plan(255, 1, 256)                        # L = 2: no room for the derivative's step
    p.set_filters(h)
    assert _native.ols_convolve_derivative(p.handle, s.data_ptr(), 300, out.data_ptr(), st) == \
        _native.OLS_ERR_UNSUPPORTED
    assert _native.ols_convolve_derivative(p.handle, s.data_ptr(), 255, out.data_ptr(), st) == \
        _native.OLS_ERR_INVALID                    # Nout = 1
    assert _native.ols_convolve_detect(p.handle, s.data_ptr(), 300, 1.0, out.data_ptr(), -1, cnt.data_ptr(),
                                       st) == _native.OLS_ERR_INVALID
    assert _native.ols_convolve_detect(p.handle, s.data_ptr(), 300, 1.0, None, 0, None, st) == \
        _native.OLS_ERR_INVALID
    assert _native.ols_convolve_power(p.handle, s.data_ptr(), 300, out.data_ptr() + 2, st) == \
        _native.OLS_ERR_INVALID
    p.close()
    r = Plan(33, 2, 256, flags=_native.OLS_FLAG_R2R)
    assert _native.ols_convolve_power(r.handle, s.data_ptr(), 300, out.data_ptr(), st) == \
        _native.OLS_ERR_UNSUPPORTED
    r.close()
    torch.cuda.synchronize()


# -- peak finding (Sec. 4.4) -------------------------------------------------
# The kernel decides in FP32 on its own powers, the oracle in FP64: a
# candidate must be reported when every comparison of the rule holds with a
# relative margin BAND, and may be reported when each holds within it.
BAND = 2e-5


def peak_bands(p, thr):
    """(must, may) bool masks of the peak rule on p [F][Nout] (numpy or torch)
    with every comparison taken with / without a relative margin BAND."""
    mod = torch if isinstance(p, torch.Tensor) else np
    inf = float("inf")
    if mod is torch:
        left = torch.nn.functional.pad(p[:, :-1], (1, 0), value=-inf)
        right = torch.nn.functional.pad(p[:, 1:], (0, 1), value=-inf)
    else:
        left = np.pad(p[:, :-1], ((0, 0), (1, 0)), constant_values=-inf)
        right = np.pad(p[:, 1:], ((0, 0), (0, 1)), constant_values=-inf)
    must = (p >= thr * (1 + BAND)) & (p > left * (1 + BAND)) & (p >= right * (1 + BAND))
    may = (p >= thr * (1 - BAND)) & (p >= left * (1 - BAND)) & (p >= right * (1 - BAND))
    return must, may


PEAK_CASES = [(2048, 257, 8, 40_000), (256, 33, 3, 10_000), (256, 254, 2, 3_000), (512, 1, 2, 5_000),
              (1024, 129, 5, 50_001), (4096, 512, 3, 70_000), (8192, 1025, 2, 100_000),
              (1024, 100, 3, 1_000), (2048, 257, 2, 257)]


@pytest.mark.parametrize("N,M,F,Ns", PEAK_CASES)
def test_peaks_match_oracle(N, M, F, Ns):
    s, h = rand_inputs(N + 9 * M + F, Ns, F, M)
    p_ref = oracle.power(s, h)
    thr = float(np.quantile(p_ref, 0.9)) if p_ref.size > 10 else float(p_ref.min())
    plan = make_plan(h, N)
    rec, cnt = plan.convolve_peaks(to_dev(s), thr, capacity=p_ref.size + 1)
    torch.cuda.synchronize()
    count = int(cnt.item())
    f, j, pw = decode_candidates(rec, count)
    plan.close()
    got = set(zip(f.tolist(), j.tolist()))
    assert len(got) == count                                   # no duplicates, nothing dropped
    must, may = peak_bands(p_ref, thr)
    must = set(zip(*[a.tolist() for a in np.nonzero(must)]))
    may = set(zip(*[a.tolist() for a in np.nonzero(may)]))
    assert must <= got <= may
    assert count >= 1 and np.all(np.abs(pw - p_ref[f, j]) <= TOL_P * p_ref[f, j])
    exact = set(zip(*[a.tolist() for a in np.nonzero(oracle.peak_mask(p_ref, thr))]))
    assert must <= exact <= may                                # the bands bracket the exact rule


@pytest.mark.parametrize("N", [256, 2048, 8192])
@pytest.mark.parametrize("M", [1, 37, 250])
def test_peaks_spike_train_exact(N, M):
    """Delta filters on a tie-free integer spike train: the peaks are known in
    closed form, including spikes on the first and last output and spikes on
    every segment boundary of the L-2 layout."""
    L = N - M + 1
    if L < 3:
        pytest.skip("needs N - M + 1 >= 3")
    Nout = 3 * N + 123
    g = np.random.Generator(np.random.PCG64(N + M))
    pos = np.unique(np.concatenate([[0, Nout - 1], np.arange(1, 8) * (L - 2), np.arange(1, 8) * (L - 2) - 1,
                                    g.integers(0, Nout, 40)]))
    pos = pos[(pos >= 0) & (pos < Nout)]
    pos = pos[np.concatenate([[True], np.diff(pos) > 1])]      # no two adjacent spikes
    for d in sorted({0, M // 2, M - 1}):
        base = (1 + (np.arange(Nout) % 7)) * 0.25                # small, non-increasing runs never tie a spike
        amp = 10.0 + np.arange(pos.size)                          # distinct spikes, powers 100 and up
        y = base.astype(np.complex64)
        y[pos] = amp
        s = np.zeros(Nout + M - 1, np.complex64)
        s[np.arange(Nout) + M - 1 - d] = y
        h = np.zeros((1, M), np.complex64)
        h[0, d] = 1
        plan = make_plan(h, N)
        rec, cnt = plan.convolve_peaks(to_dev(s), 50.0, capacity=4 * pos.size)
        torch.cuda.synchronize()
        f, j, pw = decode_candidates(rec, int(cnt.item()))
        plan.close()
        assert sorted(j.tolist()) == pos.tolist(), (N, M, d)
        assert np.array_equal(np.sort(pw), np.sort((amp * amp).astype(np.float32))) or \
            np.allclose(np.sort(pw), np.sort(amp * amp), rtol=1e-5)


def test_peaks_capacity_and_arguments():
    M, F, N, Ns = 65, 3, 512, 20_000
    s, h = rand_inputs(43, Ns, F, M)
    p_ref = oracle.power(s, h)
    thr = float(np.quantile(p_ref, 0.5))
    plan = make_plan(h, N)
    rec, cnt = plan.convolve_peaks(to_dev(s), thr, capacity=50)
    torch.cuda.synchronize()
    must, may = peak_bands(p_ref, thr)
    count = int(cnt.item())
    assert int(must.sum()) <= count <= int(may.sum()) and count > 50
    f, j, pw = decode_candidates(rec, count)
    assert f.size == 50 and np.all(may[f, j])
    st = torch.cuda.current_stream().cuda_stream
    sd = to_dev(s)
    # count only: capacity 0, no record array
    cnt2 = torch.full((1,), 7, dtype=torch.int64, device="cuda")
    assert _native.ols_convolve_peaks(plan.handle, sd.data_ptr(), Ns, thr, None, 0, cnt2.data_ptr(), st) == 0
    torch.cuda.synchronize()
    assert int(cnt2.item()) == count
    assert _native.ols_convolve_peaks(plan.handle, sd.data_ptr(), Ns, thr, rec.data_ptr(), -1, cnt.data_ptr(),
                                      st) == _native.OLS_ERR_INVALID
    assert _native.ols_convolve_peaks(plan.handle, sd.data_ptr(), M - 1, thr, rec.data_ptr(), 5, cnt.data_ptr(),
                                      st) == _native.OLS_ERR_INVALID
    plan.close()
    p2 = Plan(255, 1, 256)                                        # L = 2: no room for the L-2 layout
    p2.set_filters(to_dev(np.ones((1, 255), np.complex64)))
    assert _native.ols_convolve_peaks(p2.handle, sd.data_ptr(), 300, 1.0, rec.data_ptr(), 5, cnt.data_ptr(),
                                      st) == _native.OLS_ERR_UNSUPPORTED
    p2.close()


def test_peaks_full_size_bank():
    """The benchmark's filter bank (Ns = 2^23, F = 32, M = 257, N = 2048): the
    peaks bracket those of the kernel's own power array (pinned to the oracle
    by the power tests), and each reported power matches the oracle's."""
    cfg = synth.PLAIN_BANK
    s, h = synth.plain_inputs(cfg)
    plan = make_plan(h, cfg.N)
    sd = to_dev(s)
    p = plan.convolve_power(sd)
    thr = float(torch.quantile(p[0, : 1 << 20].float(), 0.999).item())
    must, may = peak_bands(p, thr)
    del p
    n_must, n_may = int(must.sum().item()), int(may.sum().item())
    rec, cnt = plan.convolve_peaks(sd, thr, capacity=n_may + 16)
    torch.cuda.synchronize()
    count = int(cnt.item())
    assert n_must <= count <= n_may
    j = rec[:count, 0].clone()
    w = torch.empty(count, dtype=torch.int64, device=rec.device)
    w.copy_(rec[:count, 1])                                      # a fresh contiguous column
    f = w.view(torch.int32).view(count, 2)[:, 0].long()
    assert bool(may[f, j].all())
    got = torch.zeros_like(must)
    got[f, j] = True
    assert int(got.sum().item()) == count                       # no duplicates
    assert bool((got | ~must).all())                            # every sure peak reported
    del must, may, got
    fi, ji, pw = decode_candidates(rec, min(count, 3000))
    ref = oracle.power_at(s, h, fi, ji)
    assert np.all(np.abs(pw - ref) <= TOL_P * ref)
    plan.close()
