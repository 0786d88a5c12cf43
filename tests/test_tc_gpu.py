"""The tensor-core split-precision form against the FP64 oracle.

Stated bounds (max over filters of the relative L2 error):
* FP16 split: 2e-6.  Each operand carries ~22 significant bits
  (x = x_hi + x_lo in FP16, unit roundoff 2^-22 ~ 2.4e-7 per rounding); a
  radix-16 pass adds about three such roundings (operand split, DFT-matrix
  split, the dropped lo*lo term) on top of FP32 accumulation, and a
  convolution runs 3 + 3 passes at N = 4096: ~1e-6 expected (measured
  0.8e-6 .. 1.2e-6).
* BF16 split: 3e-5.  ~16-17 significant bits (2^-17 ~ 7.6e-6 per rounding),
  same pass count: measured 6e-6 .. 8e-6.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from paper_1910_01972_gb300 import OLSError, Plan, _native
from paper_1910_01972_gb300 import build as _build

pytestmark = pytest.mark.gpu
BOUND = {_native.OLS_FLAG_TC_FP16SPLIT: 2e-6, _native.OLS_FLAG_TC_BF16SPLIT: 3e-5}
FLAGS = [_native.OLS_FLAG_TC_FP16SPLIT, _native.OLS_FLAG_TC_BF16SPLIT]


@pytest.fixture(scope="module", autouse=True)
def built():
    _build.build()
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("flag", FLAGS)
@pytest.mark.parametrize("N,M,F,Ns", [(4096, 512, 4, 200_000), (256, 33, 3, 20_001), (2048, 257, 4, 60_000),
                                      (8192, 1025, 2, 90_000), (1024, 129, 5, 30_000), (512, 1, 2, 3_000),
                                      (4096, 4096, 1, 9_000)])
def test_tc_parity(flag, N, M, F, Ns):
    g = np.random.Generator(np.random.PCG64(N + M + flag))
    s, h = synth.signal(g, Ns), synth.filters(g, F, M)
    p = Plan(M, F, N, flags=flag)
    p.set_filters(dev(h))
    y = p.convolve(dev(s)).cpu().numpy()
    assert p.status() == 0
    err = oracle.max_stream_rel_l2(y, oracle.conv(s, h), oracle.stream_scale(s, h, y.shape[1]))
    assert err <= BOUND[flag], err
    p.close()


@pytest.mark.parametrize("flag", FLAGS)
def test_tc_index_bookkeeping_with_delta_filters(flag):
    """Delta filters on a small-integer signal: rounding the output recovers
    the shifted input exactly (segment starts, discards and tail clip)."""
    N, M, Ns = 4096, 300, 3 * 4096 + 77
    n = np.arange(Ns)
    s = (((n % 3) - 1) + 1j * (((7 * n) % 3) - 1)).astype(np.complex64)
    ds = [0, 150, 299]
    h = np.zeros((3, M), np.complex64)
    for i, d in enumerate(ds):
        h[i, d] = 1.0
    p = Plan(M, 3, N, flags=flag)
    p.set_filters(dev(h))
    y = p.convolve(dev(s)).cpu().numpy()
    for i, d in enumerate(ds):
        ref = s[M - 1 - d: Ns - d]
        got = np.round(y[i].real) + 1j * np.round(y[i].imag)
        assert np.array_equal(got, ref)
    p.close()


@pytest.mark.parametrize("flag", FLAGS)
def test_tc_full_size_sampled(flag):
    """Ns = 2^24, F = 64, M = 512, N = 4096: sampled outputs against the
    oracle; the signal stored as split planes gives the same output."""
    cfg = synth.TC_SPLIT
    s, h = synth.plain_inputs(cfg)
    p = Plan(cfg.M, cfg.F, cfg.N, flags=flag)
    p.set_filters(dev(h))
    y = p.convolve(dev(s))
    torch.cuda.synchronize()
    assert p.status() == 0
    g = np.random.Generator(np.random.PCG64(9))
    Nout = cfg.Ns - cfg.M + 1
    fi = g.integers(0, cfg.F, 20_000)
    ji = np.concatenate([g.integers(0, Nout, 19_996), [0, 1, Nout - 2, Nout - 1]])
    got = y[torch.from_numpy(fi).cuda(), torch.from_numpy(ji).cuda()].cpu().numpy()
    ref = oracle.conv_at(s, h, fi, ji)
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= BOUND[flag]
    # the workload's stored form: the same signal as split hi / lo planes
    hi, lo = p.split_signal(dev(s))
    y2 = p.convolve_split(hi, lo)
    torch.cuda.synchronize()
    assert p.status() == 0 and torch.equal(y, y2)
    del y, y2
    p.close()


def test_tc_plans_reject_the_adjoint():
    p = Plan(65, 2, 512, flags=_native.OLS_FLAG_TC_FP16SPLIT)
    p.set_filters(torch.zeros((2, 65), dtype=torch.complex64, device="cuda"))
    s = torch.zeros(2000, dtype=torch.complex64, device="cuda")
    g = torch.zeros((2, 2000 - 64), dtype=torch.complex64, device="cuda")
    with pytest.raises(OLSError):
        p.convolve_backward(s, g)
    p.close()


# ----------------------------------------------------------- split storage
def _round16(x32, bf16):
    """Round FP32 values to FP16 / BF16 (nearest even); returns (bits as
    uint16, value as FP32)."""
    if not bf16:
        h = x32.astype(np.float16)
        return h.view(np.uint16), h.astype(np.float32)
    u = x32.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16).astype(np.uint16)
    return r, (r.astype(np.uint32) << 16).view(np.float32)


def host_split(s, bf16):
    """hi = round16(x), lo = round16(x - hi) per real / imaginary part, as
    int32 words (Re in the low half): the stored split form."""
    words = []
    parts = []
    for part in (s.real.astype(np.float32), s.imag.astype(np.float32)):
        hb, hv = _round16(part, bf16)
        lb, lv = _round16((part - hv).astype(np.float32), bf16)
        parts.append((hb, lb, hv, lv))
    for k in (0, 1):        # hi, lo
        w = parts[0][k].astype(np.uint32) | (parts[1][k].astype(np.uint32) << 16)
        words.append(w.view(np.int32))
    value = (parts[0][2].astype(np.float64) + parts[0][3]) + 1j * (parts[1][2].astype(np.float64) + parts[1][3])
    return words[0], words[1], value


@pytest.mark.parametrize("flag", FLAGS)
def test_split_signal_rounding(flag):
    g = np.random.Generator(np.random.PCG64(31 + flag))
    s = synth.signal(g, 100_003)
    s[:4] = [0, 1 + 1j, -1e-3 + 2.5j, 3e-5 - 7e-6j]
    p = Plan(33, 1, 256, flags=flag)
    hi, lo = p.split_signal(dev(s))
    rh, rl, _ = host_split(s, flag == _native.OLS_FLAG_TC_BF16SPLIT)
    assert np.array_equal(hi.cpu().numpy(), rh)
    assert np.array_equal(lo.cpu().numpy(), rl)
    p.close()


@pytest.mark.parametrize("flag", FLAGS)
@pytest.mark.parametrize("N,M,F,Ns", [(4096, 512, 3, 100_000), (256, 33, 2, 20_001), (2048, 257, 2, 9_001),
                                      (8192, 1025, 1, 40_000), (512, 1, 2, 700),
                                      (1024, 129, 3, 129),          # Ns = M: one output
                                      (1024, 100, 2, 900),          # Ns < N: one segment, zero-filled
                                      (512, 257, 5, 7_000),         # M - 1 = L: overlaps meet exactly
                                      (4096, 4096, 1, 9_000)])      # M = N: one output per segment
def test_convolve_split_equals_convolve(flag, N, M, F, Ns):
    """Planes from split_signal give bit for bit the FP32-input result: the
    first forward stage gets the same operands either way."""
    g = np.random.Generator(np.random.PCG64(N + M + 7 * flag))
    s, h = synth.signal(g, Ns), synth.filters(g, F, M)
    p = Plan(M, F, N, flags=flag)
    p.set_filters(dev(h))
    sd = dev(s)
    y = p.convolve(sd)
    hi, lo = p.split_signal(sd)
    y2 = p.convolve_split(hi, lo)
    torch.cuda.synchronize()
    assert p.status() == 0
    assert torch.equal(y, y2)
    p.close()


@pytest.mark.parametrize("flag", FLAGS)
def test_convolve_split_parity_host_planes(flag):
    """Planes written on the host; the stored value hi + lo (exact in FP32)
    convolved by the oracle is the reference."""
    N, M, F, Ns = 4096, 512, 3, 150_000
    g = np.random.Generator(np.random.PCG64(57 + flag))
    s, h = synth.signal(g, Ns), synth.filters(g, F, M)
    hi, lo, value = host_split(s, flag == _native.OLS_FLAG_TC_BF16SPLIT)
    v32 = value.astype(np.complex64)
    assert np.array_equal(v32.astype(np.complex128), value)
    p = Plan(M, F, N, flags=flag)
    p.set_filters(dev(h))
    y = p.convolve_split(dev(hi), dev(lo)).cpu().numpy()
    err = oracle.max_stream_rel_l2(y, oracle.conv(v32, h))
    assert err <= BOUND[flag], err
    p.close()


def test_convolve_split_errors():
    p = Plan(65, 2, 512)                               # FP32 plan
    w = torch.zeros(2000, dtype=torch.int32, device="cuda")
    with pytest.raises(OLSError) as ei:
        p.convolve_split(w, w)
    assert ei.value.status == _native.OLS_ERR_UNSUPPORTED
    p.close()
    p = Plan(65, 2, 512, flags=_native.OLS_FLAG_TC_FP16SPLIT)
    with pytest.raises(OLSError) as ei:
        p.convolve_split(w, w)                         # filters not set
    assert ei.value.status == _native.OLS_ERR_NOT_READY
    p.set_filters(torch.zeros((2, 65), dtype=torch.complex64, device="cuda"))
    y = torch.empty((2, 2000 - 64), dtype=torch.complex64, device="cuda")
    rc = _native.ols_convolve_split(p.handle, w.data_ptr() + 2, w.data_ptr(), 2000, y.data_ptr(),
                                    torch.cuda.current_stream().cuda_stream)
    assert rc == _native.OLS_ERR_INVALID                # misaligned plane
    p.close()
