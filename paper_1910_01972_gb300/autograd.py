"""Differentiable OLS convolution: a torch.autograd.Function over the C ABI.

Forward: ``ols_set_filters`` + ``ols_convolve``.  Backward:
``ols_convolve_backward`` (the adjoint kernels), re-setting the filters that
were used in the forward so interleaved calls cannot mix spectra.  Gradients
follow PyTorch's complex convention (dL/dRe + i dL/dIm), which is the one the
library's adjoint uses.  No arithmetic happens in Python.
"""
from __future__ import annotations

import threading

import torch

_plans = {}
_lock = threading.Lock()


def _plan(M: int, F: int, N: int, device: torch.device):
    from . import Plan
    key = (M, F, N, device.index)
    with _lock:
        p = _plans.get(key)
        if p is None:
            with torch.cuda.device(device):
                p = Plan(M, F, N)
            _plans[key] = p
        return p


class OLSConvFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, s: torch.Tensor, h: torch.Tensor, N: int):
        s = s.contiguous()
        h = h.contiguous()
        plan = _plan(h.shape[1], h.shape[0], N, s.device)
        plan.set_filters(h)
        y = plan.convolve(s)
        ctx.save_for_backward(s, h)
        ctx.N = N
        return y

    @staticmethod
    def backward(ctx, gy: torch.Tensor):
        s, h = ctx.saved_tensors
        want_ds, want_dh = ctx.needs_input_grad[0], ctx.needs_input_grad[1]
        if not (want_ds or want_dh):
            return None, None, None
        plan = _plan(h.shape[1], h.shape[0], ctx.N, s.device)
        plan.set_filters(h)
        ds, dh = plan.convolve_backward(s, gy.contiguous(), want_ds=want_ds, want_dh=want_dh)
        return ds, dh, None


def ols_conv(s: torch.Tensor, h: torch.Tensor, N: int = 0) -> torch.Tensor:
    """Valid-mode convolution of s [Ns] with every filter of h [F][M] (complex64,
    CUDA), differentiable in both.  N: segment length (0 = automatic; the
    adjoint of ds needs N >= 2(M-1))."""
    if h.dim() == 1:
        return OLSConvFunction.apply(s, h.unsqueeze(0), N)[0]
    return OLSConvFunction.apply(s, h, N)
