"""Parity of the adjoint kernels (through the C ABI) with the FP64 oracle.

Tolerances (relative L2 per gradient): ds <= 2e-6 (same as the forward
output: each ds sample is one windowed FFT convolution in FP32); dh <= 1e-5
(each dh entry sums ~Nout FP32 products over all windows; the windows'
partials are added with compensated summation).
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from paper_1910_01972_gb300 import Plan, _native, ols_conv
from paper_1910_01972_gb300 import build as _build

pytestmark = pytest.mark.gpu
TOL_DS = 2e-6
TOL_DH = 1e-5


@pytest.fixture(scope="module", autouse=True)
def built():
    _build.build()
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def inputs(seed, Ns, F, M):
    g = np.random.Generator(np.random.PCG64(seed))
    s = synth.signal(g, Ns)
    h = synth.filters(g, F, M)
    gy = (g.normal(size=(F, Ns - M + 1)) + 1j * g.normal(size=(F, Ns - M + 1))).astype(np.complex64)
    return s, h, gy


def gpu_backward(s, h, gy, N, want_ds=True, want_dh=True):
    plan = Plan(h.shape[1], h.shape[0], N)
    plan.set_filters(dev(h))
    ds, dh = plan.convolve_backward(dev(s), dev(gy), want_ds, want_dh)
    torch.cuda.synchronize()
    n = plan.last_launch_count()
    plan.close()
    return (ds.cpu().numpy() if ds is not None else None, dh.cpu().numpy() if dh is not None else None, n)


CASES = [
    # (N, M, F, Ns)
    (1024, 129, 16, 30_000),
    (2048, 257, 4, 20_001),
    (256, 33, 3, 5_000),
    (512, 64, 1, 65_536),
    (512, 1, 2, 3_000),           # M = 1: no overlap, dh is a plain correlation
    (4096, 512, 2, 40_000),
    (8192, 1025, 2, 60_000),
    (1024, 100, 5, 900),          # Ns < N: one window
    (1024, 129, 3, 129),          # Ns = M: one output
    (512, 257, 2, 7_000),         # M - 1 = L: overlaps meet exactly
]


@pytest.mark.parametrize("N,M,F,Ns", CASES)
def test_adjoint_parity(N, M, F, Ns):
    s, h, gy = inputs(N + M + F, Ns, F, M)
    ds, dh, n = gpu_backward(s, h, gy, N)
    ds_ref, dh_ref = oracle.adjoint(s, h, gy)
    # main kernel, then the overlap / spectrum-sum kernel, then the dh inverse FFTs
    assert n == 3
    e_ds = oracle.rel_l2(ds, ds_ref)
    e_dh = oracle.max_stream_rel_l2(dh, dh_ref)
    assert e_ds <= TOL_DS, e_ds
    assert e_dh <= TOL_DH, e_dh


def test_ds_only_and_dh_only_agree_with_both():
    s, h, gy = inputs(5, 25_000, 6, 129)
    ds, dh, _ = gpu_backward(s, h, gy, 1024)
    ds1, none1, _ = gpu_backward(s, h, gy, 1024, True, False)
    none2, dh2, _ = gpu_backward(s, h, gy, 1024, False, True)
    assert none1 is None and none2 is None
    assert oracle.rel_l2(ds1, ds) <= 1e-7
    assert oracle.rel_l2(dh2, dh) <= 1e-7


def test_adjoint_is_deterministic():
    s, h, gy = inputs(6, 50_000, 8, 65)
    a = gpu_backward(s, h, gy, 512)
    b = gpu_backward(s, h, gy, 512)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_adjoint_dot_product_identity_on_gpu():
    """Re<g, conv(s, h)> = Re<ds, s> = Re<dh, h>, all sides from the GPU."""
    s, h, gy = inputs(8, 40_000, 4, 200)
    plan = Plan(200, 4, 1024)
    plan.set_filters(dev(h))
    y = plan.convolve(dev(s)).cpu().numpy().astype(np.complex128)
    ds, dh = plan.convolve_backward(dev(s), dev(gy))
    ds, dh = ds.cpu().numpy().astype(np.complex128), dh.cpu().numpy().astype(np.complex128)
    lhs = np.real(np.vdot(gy.astype(np.complex128), y))
    r1 = np.real(np.vdot(ds, s.astype(np.complex128)))
    r2 = np.real(np.vdot(dh, h.astype(np.complex128)))
    scale = np.linalg.norm(gy) * np.linalg.norm(y)
    assert abs(lhs - r1) <= 1e-5 * scale and abs(lhs - r2) <= 1e-5 * scale
    plan.close()


def test_autograd_weighted_power_loss():
    """L = sum_f sum_n w[n] |y_f[n]|^2 through ols_conv; gradients against the
    oracle adjoint applied to the same output gradient 2 w y."""
    s_np, h_np, w_np = synth.diff_inputs(Ns=20_000)
    s = dev(s_np).requires_grad_(True)
    h = dev(h_np).requires_grad_(True)
    w = dev(w_np)
    y = ols_conv(s, h, N=1024)
    loss = (w[None, :] * (y.real ** 2 + y.imag ** 2)).sum()
    loss.backward()
    gy = (2.0 * w[None, :] * y).detach().cpu().numpy()
    ds_ref, dh_ref = oracle.adjoint(s_np, h_np, gy)
    assert oracle.rel_l2(s.grad.cpu().numpy(), ds_ref) <= TOL_DS
    assert oracle.max_stream_rel_l2(h.grad.cpu().numpy(), dh_ref) <= TOL_DH
    # forward value against the oracle as well
    y_ref = oracle.conv(s_np, h_np)
    assert oracle.max_stream_rel_l2(y.detach().cpu().numpy(), y_ref) <= 2e-6


def test_full_size_differentiable_workload():
    """Ns = 2^22, F = 16, M = 129, N = 1024: the whole gradient against the oracle."""
    cfg = synth.DIFF
    s_np, h_np, w_np = synth.diff_inputs(cfg)
    plan = Plan(cfg.M, cfg.F, cfg.N)
    plan.set_filters(dev(h_np))
    s = dev(s_np)
    y = plan.convolve(s)
    gy = (2.0 * dev(w_np)[None, :] * y).contiguous()
    ds, dh = plan.convolve_backward(s, gy)
    torch.cuda.synchronize()
    ds_ref, dh_ref = oracle.adjoint(s_np, h_np, gy.cpu().numpy())
    assert oracle.rel_l2(ds.cpu().numpy(), ds_ref) <= TOL_DS
    assert oracle.max_stream_rel_l2(dh.cpu().numpy(), dh_ref) <= TOL_DH
    plan.close()


def test_backward_errors():
    plan = Plan(129, 2, 1024)
    st = torch.cuda.current_stream().cuda_stream
    Ns = 5000
    s = torch.zeros(Ns, dtype=torch.complex64, device="cuda")
    g = torch.zeros((2, Ns - 128), dtype=torch.complex64, device="cuda")
    ds = torch.empty(Ns, dtype=torch.complex64, device="cuda")
    dh = torch.empty((2, 129), dtype=torch.complex64, device="cuda")
    assert _native.ols_convolve_backward(plan.handle, s.data_ptr(), Ns, g.data_ptr(), ds.data_ptr(),
                                         dh.data_ptr(), None, 0, st) == _native.OLS_ERR_NOT_READY
    plan.set_filters(torch.zeros((2, 129), dtype=torch.complex64, device="cuda"))
    nb = plan.backward_workspace(Ns)
    assert nb > 0
    ws = torch.empty(nb + 256, dtype=torch.uint8, device="cuda")
    wp = (ws.data_ptr() + 255) & ~255
    assert _native.ols_convolve_backward(plan.handle, s.data_ptr(), Ns, g.data_ptr(), ds.data_ptr(),
                                         dh.data_ptr(), wp, nb - 1, st) == _native.OLS_ERR_WORKSPACE
    assert _native.ols_convolve_backward(plan.handle, s.data_ptr(), Ns, g.data_ptr(), ds.data_ptr(),
                                         dh.data_ptr(), wp + 8, nb, st) == _native.OLS_ERR_WORKSPACE
    assert _native.ols_convolve_backward(plan.handle, s.data_ptr(), Ns, g.data_ptr(), None, None, wp, nb,
                                         st) == _native.OLS_ERR_INVALID
    assert _native.ols_convolve_backward(plan.handle, s.data_ptr(), Ns, g.data_ptr(), ds.data_ptr(),
                                         dh.data_ptr(), wp, nb, st) == 0
    torch.cuda.synchronize()
    assert float(ds.abs().max()) == 0.0 and float(dh.abs().max()) == 0.0
    plan.close()
    big = Plan(600, 1, 1024)   # L = 425 < M - 1 = 599: ds unsupported, dh fine
    big.set_filters(torch.zeros((1, 600), dtype=torch.complex64, device="cuda"))
    s2 = torch.zeros(3000, dtype=torch.complex64, device="cuda")
    g2 = torch.zeros((1, 3000 - 599), dtype=torch.complex64, device="cuda")
    with pytest.raises(Exception):
        big.convolve_backward(s2, g2, True, True)
    _, dh2 = big.convolve_backward(s2, g2, False, True)
    assert dh2 is not None
    big.close()


def test_workspace_contents_do_not_matter():
    """Nothing in the caller's workspace needs to start at zero: a NaN-filled
    workspace gives bit for bit the results of a zero-filled one."""
    Ns, F, M = 60_000, 8, 129
    s, h, gy = inputs(9, Ns, F, M)
    plan = Plan(M, F, 1024)
    plan.set_filters(dev(h))
    sd, gd = dev(s), dev(gy)
    nb = plan.backward_workspace(Ns)
    st = torch.cuda.current_stream().cuda_stream
    outs = []
    for fill in (0.0, float("nan")):
        ws = torch.full(((nb + 512) // 4,), fill, dtype=torch.float32, device="cuda")
        wp = (ws.data_ptr() + 255) & ~255
        ds = torch.empty(Ns, dtype=torch.complex64, device="cuda")
        dh = torch.empty((F, M), dtype=torch.complex64, device="cuda")
        rc = _native.ols_convolve_backward(plan.handle, sd.data_ptr(), Ns, gd.data_ptr(), ds.data_ptr(),
                                           dh.data_ptr(), wp, nb, st)
        assert rc == _native.OLS_OK
        torch.cuda.synchronize()
        outs.append((ds, dh))
    assert torch.equal(outs[0][0], outs[1][0]) and torch.equal(outs[0][1], outs[1][1])
    ds_ref, dh_ref = oracle.adjoint(s, h, gy)
    assert oracle.rel_l2(outs[1][0].cpu().numpy(), ds_ref) <= TOL_DS
    plan.close()
