"""Differentiable OLS convolution: a torch.autograd.Function over the C ABI.

Forward: ``ols_set_filters`` + ``ols_convolve``.  Backward:
``ols_convolve_backward`` (the adjoint kernels), re-setting the filters that
were used in the forward.  Gradients follow PyTorch's complex convention
(dL/dRe + i dL/dIm), which is the one the library's adjoint uses.  No
arithmetic happens in Python.

A plan holds one filter bank's spectra, so two calls must never share a plan
while either one's kernels may still read it.  Plans are cached per (M, F, N,
device, stream): calls on one stream run in stream order, and each call holds
its plan's lock from ``set_filters`` until its convolution is enqueued, so no
other thread's filters can be set in between.  Calls on different streams use
different plans.
"""
from __future__ import annotations

import threading

import torch

_plans = {}
_lock = threading.Lock()


def _plan(M: int, F: int, N: int, device: torch.device):
    """(plan, lock) for the current stream of `device`."""
    from . import Plan
    stream = torch.cuda.current_stream(device).cuda_stream
    key = (M, F, N, device.index, stream)
    with _lock:
        entry = _plans.get(key)
        if entry is None:
            with torch.cuda.device(device):
                entry = (Plan(M, F, N), threading.Lock())
            _plans[key] = entry
        return entry


def _values(t: torch.Tensor) -> torch.Tensor:
    # lazy conjugate / negative views carry a flag, not the values, in memory
    return t.resolve_conj().resolve_neg().contiguous()


class OLSConvFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, s: torch.Tensor, h: torch.Tensor, N: int):
        s = _values(s)
        h = _values(h)
        plan, lock = _plan(h.shape[1], h.shape[0], N, s.device)
        with lock:
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
        plan, lock = _plan(h.shape[1], h.shape[0], ctx.N, s.device)
        with lock:
            plan.set_filters(h)
            ds, dh = plan.convolve_backward(s, _values(gy), want_ds=want_ds, want_dh=want_dh)
        return ds, dh, None


def ols_conv(s: torch.Tensor, h: torch.Tensor, N: int = 0) -> torch.Tensor:
    """Valid-mode convolution of s [Ns] with every filter of h [F][M] (complex64,
    CUDA), differentiable in both.  N: segment length (0 = automatic; the
    adjoint of ds needs N >= 2(M-1))."""
    if h.dim() == 1:
        return OLSConvFunction.apply(s, h.unsqueeze(0), N)[0]
    return OLSConvFunction.apply(s, h, N)
