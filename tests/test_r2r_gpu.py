"""Parity of the real-to-real fused OLS kernel (Sec. 3.4's R2R variant, through
the C ABI) with the FP64 real oracle.

Tolerance: max over filters of ||y - y_ref||_2 / ||y_ref||_2 <= 2e-6, the
FP32 bar of the complex path, with the same floor of the denominator
(oracle.stream_scale) for streams of a few outputs.  Index bookkeeping and the filter pairing
(filter 2p in the real part, 2p+1 in the imaginary part of one inverse FFT)
are checked bit-exactly with delta filters on integer-valued signals.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from paper_1910_01972_gb300 import OLSError, Plan, _native
from paper_1910_01972_gb300 import build as _build

pytestmark = pytest.mark.gpu
TOL = 2e-6
R2R = _native.OLS_FLAG_R2R


@pytest.fixture(scope="module", autouse=True)
def built():
    _build.build()
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")


def to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def run(s, h, N):
    plan = Plan(h.shape[1], h.shape[0], N, flags=R2R)
    plan.set_filters_real(to_dev(h))
    y = plan.convolve_real(to_dev(s))
    torch.cuda.synchronize()
    assert plan.last_launch_count() == 1
    plan.close()
    return y.cpu().numpy()


def rand_inputs(seed, Ns, F, M, window=False):
    g = np.random.Generator(np.random.PCG64(seed))
    return synth.real_signal(g, Ns), synth.real_filters(g, F, M, window=window)


CASES = [
    # (N, M, F, Ns, window)
    (512, 64, 1, 65536, False),          # one filter: the pair's imaginary half is unused
    (2048, 257, 32, 40_000, True),       # filter bank, Hann window, ragged tail
    (2048, 257, 5, 40_000, False),       # odd bank
    (256, 33, 3, 10_000, False),
    (256, 256, 2, 2_000, False),         # M = N: one valid sample per segment
    (512, 1, 2, 5_000, False),           # M = 1: nothing discarded
    (1024, 129, 16, 50_001, False),
    (4096, 512, 4, 70_000, False),
    (8192, 1025, 3, 100_000, False),
    (1024, 100, 7, 1_000, False),        # Ns < N: a single partial segment
    (2048, 257, 2, 257, False),          # Ns = M: one output
    (2048, 257, 3, 1792 * 5 + 256, False),  # Ns = nseg L + M - 1 exactly
]


@pytest.mark.parametrize("N,M,F,Ns,window", CASES)
def test_parity_with_real_oracle(N, M, F, Ns, window):
    s, h = rand_inputs(N * 5 + M + F, Ns, F, M, window)
    y = run(s, h, N)
    y_ref = oracle.conv_real(s, h)
    assert y.shape == y_ref.shape and y.dtype == np.float32
    assert oracle.max_stream_rel_l2(y, y_ref, oracle.stream_scale(s, h, y.shape[1])) <= TOL


@pytest.mark.parametrize("N", [256, 2048, 8192])
@pytest.mark.parametrize("M", [1, 37, 256])
def test_delta_filters_bit_exact(N, M):
    """h_f = e_{d_f} gives y_f[j] = s[j+M-1-d_f]; integer-valued s must come back
    exactly after rounding, for filters in both halves of a pair and for the
    unpaired last filter of an odd bank."""
    Ns = 3 * N + 123
    s = (np.arange(Ns) % 1024).astype(np.float32)
    ds = sorted({0, M // 2, M - 1}) + [M - 1, 0]     # an odd bank
    h = np.zeros((len(ds), M), np.float32)
    for i, d in enumerate(ds):
        h[i, d] = 1.0
    y = run(s, h, N)
    for i, d in enumerate(ds):
        ref = s[M - 1 - d: Ns - d]
        assert np.array_equal(np.round(y[i]), ref), (N, M, d)
        assert np.max(np.abs(y[i] - ref)) < 0.05


def test_matches_complex_path_on_real_data():
    """The R2R form and the complex form agree on real inputs (same Eq. 1)."""
    M, F, N, Ns = 129, 6, 1024, 30_000
    s, h = rand_inputs(11, Ns, F, M)
    yr = run(s, h, N)
    plan = Plan(M, F, N)
    plan.set_filters(to_dev(h.astype(np.complex64)))
    yc = plan.convolve(to_dev(s.astype(np.complex64))).cpu().numpy()
    plan.close()
    assert oracle.max_stream_rel_l2(yr, yc.real) <= 2 * TOL
    assert np.max(np.abs(yc.imag)) <= 1e-5


def test_spectra_are_the_paired_filters():
    """ols_get_spectra of an R2R plan returns FFT(h_{2p} + i h_{2p+1}) / N."""
    M, F, N = 65, 5, 512
    _, h = rand_inputs(3, 10, F, M)
    plan = Plan(M, F, N, flags=R2R)
    plan.set_filters_real(to_dev(h))
    H = torch.empty(((F + 1) // 2, N), dtype=torch.complex64, device="cuda")
    _native.check(_native.ols_get_spectra(plan.handle, H.data_ptr(), 0), "ols_get_spectra")
    hp = np.zeros(((F + 1) // 2, M), np.complex128)
    hp[:, :] = h[0::2]
    hp[: F // 2] += 1j * h[1::2]
    ref = np.fft.fft(hp, N, axis=1) / N
    got = H.cpu().numpy()
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-7
    plan.close()


def test_full_size_real_filter_bank_sampled():
    """Real filter bank of the benchmark shape (Ns = 2^23, F = 32, M = 257,
    N = 2048) in the launch configuration it is timed in; sampled outputs
    (random, segment boundaries, first and last) against the oracle."""
    cfg = synth.R2R_BANK
    s, h = synth.real_inputs(cfg)
    plan = Plan(cfg.M, cfg.F, cfg.N, flags=R2R)
    plan.set_filters_real(to_dev(h))
    y = plan.convolve_real(to_dev(s))
    torch.cuda.synchronize()
    q = plan.query(cfg.Ns)
    Nout, L = q["Nout"], q["L"]
    g = np.random.Generator(np.random.PCG64(8))
    fi = g.integers(0, cfg.F, 20_000)
    ji = g.integers(0, Nout, 20_000)
    b = np.arange(1, 64) * L
    ej = np.concatenate([[0, 1, Nout - 1, Nout - 2], b - 1, b])
    fi = np.concatenate([fi, np.arange(ej.size) % cfg.F])
    ji = np.concatenate([ji, ej])
    got = y[torch.from_numpy(fi).cuda(), torch.from_numpy(ji).cuda()].cpu().numpy().astype(np.float64)
    ref = oracle.conv_real_at(s, h, fi, ji)
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= TOL
    assert bool(torch.isfinite(y).all())
    plan.close()


def test_entry_points_check_the_plan_kind():
    M, F, N = 33, 2, 256
    s = to_dev(np.zeros(1000, np.float32))
    sc = to_dev(np.zeros(1000, np.complex64))
    hr = to_dev(np.zeros((F, M), np.float32))
    hc = to_dev(np.zeros((F, M), np.complex64))
    y = torch.empty((F, 1000 - M + 1), dtype=torch.float32, device="cuda")
    yc = torch.empty((F, 1000 - M + 1), dtype=torch.complex64, device="cuda")
    st = torch.cuda.current_stream().cuda_stream
    pr = Plan(M, F, N, flags=R2R)
    assert _native.ols_convolve_real(pr.handle, s.data_ptr(), 1000, y.data_ptr(), st) == _native.OLS_ERR_NOT_READY
    assert _native.ols_set_filters(pr.handle, hc.data_ptr(), st) == _native.OLS_ERR_UNSUPPORTED
    pr.set_filters_real(hr)
    assert _native.ols_convolve(pr.handle, sc.data_ptr(), 1000, yc.data_ptr(), st) == _native.OLS_ERR_UNSUPPORTED
    assert _native.ols_convolve_real(pr.handle, s.data_ptr(), 10, y.data_ptr(), st) == _native.OLS_ERR_INVALID
    assert _native.ols_convolve_real(pr.handle, s.data_ptr() + 2, 999, y.data_ptr(), st) == _native.OLS_ERR_INVALID
    pc = Plan(M, F, N)
    assert _native.ols_set_filters_real(pc.handle, hr.data_ptr(), st) == _native.OLS_ERR_UNSUPPORTED
    assert _native.ols_convolve_real(pc.handle, s.data_ptr(), 1000, y.data_ptr(), st) == _native.OLS_ERR_UNSUPPORTED
    with pytest.raises(OLSError):
        pc.convolve_real(s)
    torch.cuda.synchronize()
    pr.close()
    pc.close()
