"""Parity of the fused FP32 OLS kernel (through the C ABI) with the FP64 oracle.

Tolerance: max over filters of ||y - y_ref||_2 / ||y_ref||_2 <= 2e-6 (FP32
path against the FP64 direct sum of Eq. 1), the denominator floored at the
stream's expected norm sqrt(Nout) ||h_f|| rms(s) (oracle.stream_scale): a
stream of one or two outputs can be near zero by chance, while the FFT's
rounding error follows the segment's energy.  Index bookkeeping (segment
starts, discarded samples, the ragged tail) is checked bit-exactly with
delta filters on integer-valued signals.
"""
import math

import numpy as np
import pytest
import torch

import oracle
import synth
from paper_1910_01972_gb300 import Plan, _native
from paper_1910_01972_gb300 import build as _build

pytestmark = pytest.mark.gpu
TOL = 2e-6


@pytest.fixture(scope="module", autouse=True)
def built():
    _build.build()
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")


def to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def run(s, h, N):
    plan = Plan(h.shape[1], h.shape[0], N)
    plan.set_filters(to_dev(h))
    y = plan.convolve(to_dev(s))
    torch.cuda.synchronize()
    out = y.cpu().numpy()
    assert plan.last_launch_count() == 1
    plan.close()
    return out


def rand_inputs(seed, Ns, F, M, window=False):
    g = np.random.Generator(np.random.PCG64(seed))
    return synth.signal(g, Ns), synth.filters(g, F, M, window=window)


def test_spectra_match_fft_of_padded_filters():
    for N, M, F in ((256, 33, 2), (2048, 257, 4), (8192, 1025, 2), (512, 512, 1)):
        _, h = rand_inputs(N + M, 10, F, M)
        plan = Plan(M, F, N)
        plan.set_filters(to_dev(h))
        H = plan.spectra().cpu().numpy()
        ref = np.fft.fft(h.astype(np.complex128), N, axis=1) / N
        err = np.linalg.norm(H - ref) / np.linalg.norm(ref)
        assert err < 1e-7, (N, M, err)
        plan.close()


CASES = [
    # (N, M, F, Ns, window)
    (512, 64, 1, 65536, False),          # one signal, one filter (full size)
    (2048, 257, 32, 40_000, True),       # filter bank, Hann window, ragged tail
    (2048, 257, 5, 40_000, False),
    (256, 33, 3, 10_000, False),
    (256, 256, 2, 2_000, False),         # M = N: one valid sample per segment
    (512, 1, 2, 5_000, False),           # M = 1: nothing discarded
    (1024, 129, 16, 50_001, False),
    (4096, 512, 4, 70_000, False),
    (8192, 1025, 3, 100_000, False),
    (8192, 3000, 2, 30_000, False),
    (1024, 100, 7, 1_000, False),        # Ns < N: a single partial segment
    (2048, 257, 2, 257, False),          # Ns = M: one output
    (2048, 257, 3, 1792 * 5 + 256, False),  # Ns = nseg L + M - 1 exactly
]


@pytest.mark.parametrize("N,M,F,Ns,window", CASES)
def test_parity_with_oracle(N, M, F, Ns, window):
    s, h = rand_inputs(N * 7 + M + F, Ns, F, M, window)
    y = run(s, h, N)
    y_ref = oracle.conv(s, h)
    assert y.shape == y_ref.shape
    err = oracle.max_stream_rel_l2(y, y_ref, oracle.stream_scale(s, h, y.shape[1]))
    assert err <= TOL, err


@pytest.mark.parametrize("N", [256, 512, 2048, 8192])
@pytest.mark.parametrize("M", [1, 37, 256])
def test_delta_filters_bit_exact(N, M):
    """h = e_d gives y[j] = s[j+M-1-d]; integer-valued s must come back exactly
    after rounding, which pins every segment start, discard and tail clip."""
    Ns = 3 * N + 123
    n = np.arange(Ns)
    s = ((n % 1024) + 1j * ((7 * n) % 1024)).astype(np.complex64)
    ds = sorted({0, M // 2, M - 1})
    h = np.zeros((len(ds), M), np.complex64)
    for i, d in enumerate(ds):
        h[i, d] = 1.0
    y = run(s, h, N)
    for i, d in enumerate(ds):
        ref = s[M - 1 - d: Ns - d]
        got = np.round(y[i].real) + 1j * np.round(y[i].imag)
        assert np.array_equal(got, ref), (N, M, d)
        assert np.max(np.abs(y[i] - ref)) < 0.05


def test_segment_size_invariance():
    """Sec. 3.2: the result does not depend on the segment length."""
    M, F, Ns = 200, 3, 30_000
    s, h = rand_inputs(99, Ns, F, M)
    y_ref = oracle.conv(s, h)
    outs = []
    for N in (256, 512, 1024, 2048, 4096, 8192):
        y = run(s, h, N)
        assert oracle.max_stream_rel_l2(y, y_ref) <= TOL, N
        outs.append(y)
    for y in outs[1:]:
        assert oracle.max_stream_rel_l2(y, outs[0]) <= 2 * TOL


def test_automatic_segment_length():
    s, h = rand_inputs(5, 20_000, 2, 257)
    plan = Plan(257, 2, 0)
    assert plan.N in (256 * 2 ** i for i in range(6)) and plan.N >= 257
    plan.set_filters(to_dev(h))
    y = plan.convolve(to_dev(s)).cpu().numpy()
    assert oracle.max_stream_rel_l2(y, oracle.conv(s, h)) <= TOL


def _sample_indices(g, F, Nout, L, n):
    fi = g.integers(0, F, n)
    ji = g.integers(0, Nout, n)
    # segment boundaries, the first and last outputs of every stream
    b = np.arange(1, min(Nout // L, 64)) * L
    extra_j = np.concatenate([[0, 1, Nout - 1, Nout - 2], b - 1, b])
    extra_f = np.arange(extra_j.size) % F
    return np.concatenate([fi, extra_f]), np.concatenate([ji, extra_j])


def test_full_size_filter_bank_sampled():
    """The benchmark's workload (Ns = 2^23, F = 32, M = 257, N = 2048) in the
    launch configuration it times; sampled outputs against the oracle."""
    cfg = synth.PLAIN_BANK
    s, h = synth.plain_inputs(cfg)
    plan = Plan(cfg.M, cfg.F, cfg.N)
    plan.set_filters(to_dev(h))
    y = plan.convolve(to_dev(s))
    torch.cuda.synchronize()
    q = plan.query(cfg.Ns)
    g = np.random.Generator(np.random.PCG64(7))
    fi, ji = _sample_indices(g, cfg.F, q["Nout"], q["L"], 20_000)
    got = y[torch.from_numpy(fi).cuda(), torch.from_numpy(ji).cuda()].cpu().numpy()
    ref = oracle.conv_at(s, h, fi, ji)
    err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert err <= TOL, err
    assert bool(torch.isfinite(torch.view_as_real(y)).all())
    plan.close()


def test_host_buffer_path_matches_device_path():
    """ols_convolve_host (chunked, pipelined copies) gives the device result
    bit for bit: chunks start on segment boundaries."""
    M, F, N, Ns = 257, 32, 2048, (1 << 21) + 777
    s, h = rand_inputs(21, Ns, F, M)
    plan = Plan(M, F, N)
    plan.set_filters(to_dev(h))
    y_dev = plan.convolve(to_dev(s)).cpu()
    s_pin = torch.from_numpy(s).pin_memory()
    y_host = plan.convolve_host(s_pin)
    assert plan.last_launch_count() > 1       # several chunks
    assert torch.equal(y_host, y_dev)
    y_pageable = plan.convolve_host(torch.from_numpy(s))
    assert torch.equal(y_pageable, y_dev)
    plan.close()


def test_host_stage_timing():
    """Stage timing of the host-buffer path: NOT_READY until a timed call,
    then per-stage device times for every chunk; the results are unchanged
    (bit for bit) by the events, and turning it off clears it."""
    import time
    M, F, N, Ns = 257, 32, 2048, (1 << 21) + 777
    s, h = rand_inputs(22, Ns, F, M)
    plan = Plan(M, F, N)
    plan.set_filters(to_dev(h))
    s_pin = torch.from_numpy(s).pin_memory()
    ref = plan.convolve_host(s_pin)
    assert _native.ols_host_stage_ms(plan.handle)[0] == _native.OLS_ERR_NOT_READY   # timing off
    plan.host_timing(True)
    assert _native.ols_host_stage_ms(plan.handle)[0] == _native.OLS_ERR_NOT_READY   # no timed call yet
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    y = plan.convolve_host(s_pin)
    wall_ms = (time.perf_counter() - t0) * 1e3
    st = plan.host_stage_ms()
    assert torch.equal(y, ref)
    assert st["chunks"] == plan.last_launch_count() > 1
    assert st["h2d_ms"] > 0 and st["kernel_ms"] > 0 and st["d2h_ms"] > 0
    assert 0 < st["span_ms"] <= wall_ms
    # bytes moved out / summed D2H time: a plausible host-link rate (> 1 GB/s)
    assert 8 * F * (Ns - M + 1) / (st["d2h_ms"] * 1e-3) > 1e9
    plan.host_timing(False)
    assert _native.ols_host_stage_ms(plan.handle)[0] == _native.OLS_ERR_NOT_READY
    plan.close()


def test_graph_capture_and_side_stream():
    M, F, N, Ns = 129, 8, 1024, 100_000
    s, h = rand_inputs(3, Ns, F, M)
    plan = Plan(M, F, N)
    plan.set_filters(to_dev(h))
    sd = to_dev(s)
    ref = plan.convolve(sd).clone()
    out = torch.empty_like(ref)
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=side):
            plan.convolve(sd, out=out)
    torch.cuda.current_stream().wait_stream(side)
    out.zero_()
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(out, ref)
    plan.close()


def test_errors_are_reported_not_raised_in_c():
    plan = Plan(64, 2, 512)
    s = torch.zeros(1000, dtype=torch.complex64, device="cuda")
    y = torch.empty((2, 1000 - 63), dtype=torch.complex64, device="cuda")
    st = torch.cuda.current_stream().cuda_stream
    assert _native.ols_convolve(plan.handle, s.data_ptr(), 1000, y.data_ptr(), st) == _native.OLS_ERR_NOT_READY
    plan.set_filters(torch.zeros((2, 64), dtype=torch.complex64, device="cuda"))
    assert _native.ols_convolve(plan.handle, s.data_ptr() + 4, 1000, y.data_ptr(), st) == _native.OLS_ERR_INVALID
    assert _native.ols_convolve(plan.handle, s.data_ptr(), 63, y.data_ptr(), st) == _native.OLS_ERR_INVALID
    assert _native.ols_convolve(plan.handle, s.data_ptr(), 1000, y.data_ptr(), st) == 0
    torch.cuda.synchronize()
    assert float(y.abs().max()) == 0.0
    plan.close()
