"""GB300-native overlap-and-save (OLS) convolution.

Fused OLS convolution of a long complex signal with a bank of short filters
(arXiv:1910.01972, Algorithm 2), as hand-written CUDA kernels for sm_103a
behind a C ABI (``include/ols.h``).  This package is the thin Python side:
``_native`` binds the C functions under their own names, and ``Plan`` passes
torch tensors' device pointers and the current CUDA stream to them.  PyTorch
supplies device memory and streams only; every step of the convolution runs
in the library's kernels.
"""
from __future__ import annotations

import numpy as np
import torch

from . import _native
from ._native import OLSError, check

__all__ = ["Plan", "BatchPlan", "OLSError", "geometry", "spectrum_order", "convolve", "ols_conv", "autotune",
           "decode_candidates"]


def _stream_ptr(device) -> int:
    return torch.cuda.current_stream(device).cuda_stream


def _check(t: torch.Tensor, name: str, dtype, device):
    if not isinstance(t, torch.Tensor):
        raise TypeError("%s must be a torch.Tensor" % name)
    if t.dtype != dtype:
        raise TypeError("%s must be %s, got %s" % (name, str(dtype).replace("torch.", ""), t.dtype))
    if device is not None and t.device != device:
        raise ValueError("%s is on %s, expected %s" % (name, t.device, device))


def _lazy(t: torch.Tensor) -> bool:
    # A conjugate (t.conj()) or negative (e.g. t.conj().imag) view shares its
    # base's memory and only flags the operation: the bytes at data_ptr() are
    # not the values the tensor stands for.
    return t.is_conj() or t.is_neg()


def _input(t: torch.Tensor, name: str, device=None, dtype=torch.complex64) -> torch.Tensor:
    """The tensor whose memory holds the values `t` stands for.  Lazy
    conjugate / negative views are materialised into a fresh tensor (the
    kernels read raw memory); any other layout must already be contiguous."""
    _check(t, name, dtype, device)
    if _lazy(t):
        t = t.resolve_conj().resolve_neg()
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    return t


def _output(t: torch.Tensor, name: str, device=None, dtype=torch.complex64) -> torch.Tensor:
    """A caller-supplied output: written in place, so it must be a plain
    contiguous tensor (a lazy conjugate or negative view would be read back
    conjugated or negated)."""
    _check(t, name, dtype, device)
    if _lazy(t):
        raise ValueError("%s must not be a conjugate or negative view (resolve it first)" % name)
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    return t


def geometry(N: int, M: int, Ns: int):
    """(L, nseg, Nout) of Sec. 3.2's segmentation; host arithmetic only."""
    rc, L, nseg, Nout = _native.ols_geometry(N, M, Ns)
    check(rc, "ols_geometry")
    return L, nseg, Nout


def spectrum_order(N: int):
    """Frequency index held at each storage position of the internal spectrum."""
    rc, nu = _native.ols_spectrum_order(N)
    check(rc, "ols_spectrum_order")
    return nu


class Plan:
    """A plan for F filters of M taps with segment length N (0 = automatic).

    The plan lives on the CUDA device current at construction.
    """

    def __init__(self, M: int, F: int, N: int = 0, flags: int = _native.OLS_FLAG_FP32):
        rc, handle = _native.ols_plan(int(N), int(M), int(F), int(flags))
        check(rc, "ols_plan")
        self._h = handle
        self.device = torch.device("cuda", torch.cuda.current_device())
        rc, q = _native.ols_plan_query(self._h, 0)
        check(rc, "ols_plan_query")
        self.N, self.M, self.F, self.L = q["N"], q["M"], q["F"], q["L"]
        self._filters = None

    def close(self):
        if getattr(self, "_h", None):
            _native.ols_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self) -> int:
        return self._h

    def query(self, Ns: int):
        rc, q = _native.ols_plan_query(self._h, int(Ns))
        check(rc, "ols_plan_query")
        return q

    def set_filters(self, h: torch.Tensor) -> None:
        """h: [F][M] complex64 on the plan's device."""
        h = _input(h, "h", self.device)
        if tuple(h.shape) != (self.F, self.M):
            raise ValueError("h must have shape [%d][%d]" % (self.F, self.M))
        check(_native.ols_set_filters(self._h, h.data_ptr(), _stream_ptr(self.device)), "ols_set_filters")
        self._filters = h

    def spectra(self) -> torch.Tensor:
        """The plan's filter spectra in natural order, [F][N] complex64 (1/N folded in)."""
        H = torch.empty((self.F, self.N), dtype=torch.complex64, device=self.device)
        check(_native.ols_get_spectra(self._h, H.data_ptr(), _stream_ptr(self.device)), "ols_get_spectra")
        return H

    def convolve(self, s: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
        """Valid-mode convolution: s [Ns] -> y [F][Ns-M+1] (complex64, device)."""
        s = _input(s, "s", self.device)
        if s.dim() != 1:
            raise ValueError("s must be 1-D")
        Ns = s.shape[0]
        if Ns < self.M:
            raise ValueError("signal shorter than the filter (Ns < M)")
        Nout = Ns - self.M + 1
        if out is None:
            out = torch.empty((self.F, Nout), dtype=torch.complex64, device=self.device)
        else:
            _output(out, "out", self.device)
            if tuple(out.shape) != (self.F, Nout):
                raise ValueError("out must have shape [F][Ns-M+1]")
        check(_native.ols_convolve(self._h, s.data_ptr(), Ns, out.data_ptr(), _stream_ptr(self.device)),
              "ols_convolve")
        return out

    def split_signal(self, s: torch.Tensor):
        """Tensor-core plans: the stored split form (hi, lo) of s [Ns]
        complex64, two int32 tensors [Ns] each holding one sample's 16-bit
        (Re, Im) pair (see ols_split_signal)."""
        s = _input(s, "s", self.device)
        hi = torch.empty(s.shape[0], dtype=torch.int32, device=self.device)
        lo = torch.empty_like(hi)
        check(_native.ols_split_signal(self._h, s.data_ptr(), s.shape[0], hi.data_ptr(), lo.data_ptr(),
                                       _stream_ptr(self.device)), "ols_split_signal")
        return hi, lo

    def convolve_split(self, s_hi: torch.Tensor, s_lo: torch.Tensor, out: torch.Tensor | None = None):
        """Tensor-core plans: convolution of a signal stored split (planes as
        returned by split_signal): -> y [F][Ns-M+1] complex64."""
        s_hi = _input(s_hi, "s_hi", self.device, torch.int32)
        s_lo = _input(s_lo, "s_lo", self.device, torch.int32)
        if s_hi.dim() != 1 or s_hi.shape != s_lo.shape:
            raise ValueError("s_hi and s_lo must be 1-D and of one length")
        Ns = s_hi.shape[0]
        if Ns < self.M:
            raise ValueError("signal shorter than the filter (Ns < M)")
        Nout = Ns - self.M + 1
        if out is None:
            out = torch.empty((self.F, Nout), dtype=torch.complex64, device=self.device)
        else:
            _output(out, "out", self.device)
            if tuple(out.shape) != (self.F, Nout):
                raise ValueError("out must have shape [F][Ns-M+1]")
        check(_native.ols_convolve_split(self._h, s_hi.data_ptr(), s_lo.data_ptr(), Ns, out.data_ptr(),
                                         _stream_ptr(self.device)), "ols_convolve_split")
        return out

    def _signal(self, s: torch.Tensor):
        s = _input(s, "s", self.device)
        if s.dim() != 1:
            raise ValueError("s must be 1-D")
        if s.shape[0] < self.M:
            raise ValueError("signal shorter than the filter (Ns < M)")
        return s, s.shape[0] - self.M + 1

    def convolve_power(self, s: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
        """|y|^2 fused into the convolution: s [Ns] -> p [F][Ns-M+1] float32."""
        s, Nout = self._signal(s)
        if out is None:
            out = torch.empty((self.F, Nout), dtype=torch.float32, device=self.device)
        _output(out, "out", self.device, torch.float32)
        if tuple(out.shape) != (self.F, Nout):
            raise ValueError("out must have shape [F][Ns-M+1]")
        check(_native.ols_convolve_power(self._h, s.data_ptr(), s.shape[0], out.data_ptr(),
                                         _stream_ptr(self.device)), "ols_convolve_power")
        return out

    def convolve_detect(self, s: torch.Tensor, threshold: float, capacity: int):
        """Candidates (f, j) with |y_f[j]|^2 >= threshold.  Returns (records,
        count): records is a device int64 tensor [capacity][2] holding the C
        records (j; f and power packed in the second word, see
        ``decode_candidates``), count a device uint64-as-int64 tensor [1]."""
        s, _ = self._signal(s)
        rec = torch.empty((max(int(capacity), 1), 2), dtype=torch.int64, device=self.device)
        cnt = torch.zeros(1, dtype=torch.int64, device=self.device)
        check(_native.ols_convolve_detect(self._h, s.data_ptr(), s.shape[0], float(threshold), rec.data_ptr(),
                                          int(capacity), cnt.data_ptr(), _stream_ptr(self.device)),
              "ols_convolve_detect")
        return rec, cnt

    def convolve_peaks(self, s: torch.Tensor, threshold: float, capacity: int):
        """Peaks of the power |y_f[j]|^2: at least ``threshold``, above the power
        of j-1 and at least that of j+1.  Returns (records, count) as
        ``convolve_detect``."""
        s, _ = self._signal(s)
        rec = torch.empty((max(int(capacity), 1), 2), dtype=torch.int64, device=self.device)
        cnt = torch.zeros(1, dtype=torch.int64, device=self.device)
        check(_native.ols_convolve_peaks(self._h, s.data_ptr(), s.shape[0], float(threshold), rec.data_ptr(),
                                         int(capacity), cnt.data_ptr(), _stream_ptr(self.device)),
              "ols_convolve_peaks")
        return rec, cnt

    def convolve_derivative(self, s: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
        """Derivative of the convolved output along j (central differences,
        one-sided at the ends): s [Ns] -> d [F][Ns-M+1] complex64."""
        s, Nout = self._signal(s)
        if out is None:
            out = torch.empty((self.F, Nout), dtype=torch.complex64, device=self.device)
        _output(out, "out", self.device)
        if tuple(out.shape) != (self.F, Nout):
            raise ValueError("out must have shape [F][Ns-M+1]")
        check(_native.ols_convolve_derivative(self._h, s.data_ptr(), s.shape[0], out.data_ptr(),
                                              _stream_ptr(self.device)), "ols_convolve_derivative")
        return out

    def set_filters_real(self, h: torch.Tensor) -> None:
        """Real-to-real plans (flags=OLS_FLAG_R2R): h [F][M] float32 on the plan's device."""
        h = _input(h, "h", self.device, torch.float32)
        if tuple(h.shape) != (self.F, self.M):
            raise ValueError("h must have shape [%d][%d]" % (self.F, self.M))
        check(_native.ols_set_filters_real(self._h, h.data_ptr(), _stream_ptr(self.device)), "ols_set_filters_real")
        self._filters = h

    def convolve_real(self, s: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
        """Real valid-mode convolution: s [Ns] float32 -> y [F][Ns-M+1] float32 (R2R plans)."""
        s = _input(s, "s", self.device, torch.float32)
        if s.dim() != 1:
            raise ValueError("s must be 1-D")
        Ns = s.shape[0]
        if Ns < self.M:
            raise ValueError("signal shorter than the filter (Ns < M)")
        Nout = Ns - self.M + 1
        if out is None:
            out = torch.empty((self.F, Nout), dtype=torch.float32, device=self.device)
        else:
            _output(out, "out", self.device, torch.float32)
            if tuple(out.shape) != (self.F, Nout):
                raise ValueError("out must have shape [F][Ns-M+1]")
        check(_native.ols_convolve_real(self._h, s.data_ptr(), Ns, out.data_ptr(), _stream_ptr(self.device)),
              "ols_convolve_real")
        return out

    def convolve_host(self, s_host: torch.Tensor, out_host: torch.Tensor | None = None) -> torch.Tensor:
        """Host-buffer convolution (pinned CPU tensors give overlapped copies)."""
        if s_host.device.type != "cpu":
            raise ValueError("s_host must be a CPU tensor")
        s_host = _input(s_host, "s_host")
        Ns = s_host.shape[0]
        if Ns < self.M:
            raise ValueError("signal shorter than the filter (Ns < M)")
        Nout = Ns - self.M + 1
        if out_host is None:
            out_host = torch.empty((self.F, Nout), dtype=torch.complex64, pin_memory=s_host.is_pinned())
        _output(out_host, "out_host")
        if tuple(out_host.shape) != (self.F, Nout) or out_host.device.type != "cpu":
            raise ValueError("out_host must be a CPU tensor of shape [F][Ns-M+1]")
        check(_native.ols_convolve_host(self._h, s_host.data_ptr(), Ns, out_host.data_ptr(),
                                        _stream_ptr(self.device)), "ols_convolve_host")
        return out_host

    def host_timing(self, on: bool = True) -> None:
        """Record per-stage events in later ``convolve_host`` calls (see host_stage_ms)."""
        check(_native.ols_host_timing(self._h, on), "ols_host_timing")

    def host_stage_ms(self) -> dict:
        """Device time of the last timed ``convolve_host`` call: copies in, kernels,
        copies out (each summed over the chunks), the span, and the chunk count."""
        rc, ms = _native.ols_host_stage_ms(self._h)
        check(rc, "ols_host_stage_ms")
        return {"h2d_ms": ms[0], "kernel_ms": ms[1], "d2h_ms": ms[2], "span_ms": ms[3], "chunks": int(ms[4])}

    def backward_workspace(self, Ns: int, want_ds: bool = True, want_dh: bool = True) -> int:
        rc, nb = _native.ols_backward_workspace(self._h, int(Ns), want_ds, want_dh)
        check(rc, "ols_backward_workspace")
        return nb

    def convolve_backward(self, s: torch.Tensor | None, g: torch.Tensor, want_ds: bool = True,
                          want_dh: bool = True, Ns: int | None = None):
        """Adjoint of ``convolve``: returns (ds [Ns] or None, dh [F][M] or None).

        g: [F][Ns-M+1] complex64, the gradient dL/dRe y + i dL/dIm y.
        """
        g = _input(g, "g", self.device)
        if s is not None:
            s = _input(s, "s", self.device)
            Ns = s.shape[0]
        if Ns is None:
            raise ValueError("Ns is needed when s is not given")
        if want_dh and s is None:
            raise ValueError("dh needs the signal s")
        if tuple(g.shape) != (self.F, Ns - self.M + 1):
            raise ValueError("g must have shape [F][Ns-M+1]")
        ds = torch.empty(Ns, dtype=torch.complex64, device=self.device) if want_ds else None
        dh = torch.empty((self.F, self.M), dtype=torch.complex64, device=self.device) if want_dh else None
        nb = self.backward_workspace(Ns, want_ds, want_dh)
        ws = torch.empty(max(nb, 1) + 256, dtype=torch.uint8, device=self.device)
        wp = (ws.data_ptr() + 255) & ~255
        check(_native.ols_convolve_backward(self._h, s.data_ptr() if s is not None else None, Ns, g.data_ptr(),
                                            ds.data_ptr() if ds is not None else None,
                                            dh.data_ptr() if dh is not None else None, wp, nb,
                                            _stream_ptr(self.device)), "ols_convolve_backward")
        return ds, dh

    def last_launch_count(self) -> int:
        return _native.ols_last_launch_count(self._h)

    def status(self, reset: bool = True) -> int:
        """Device status word: bit 1 a bounded tensor-core wait gave up, bit 2
        (OLS_CHECK builds) a global access failed its bounds check."""
        rc, v = _native.ols_plan_status(self._h, reset)
        check(rc, "ols_plan_status")
        return v


def decode_candidates(records: torch.Tensor, count: int):
    """(f, j, power) numpy arrays of the first min(count, capacity) records
    written by ``Plan.convolve_detect`` (record layout of ols_candidate)."""
    n = min(int(count), records.shape[0])
    r = np.ascontiguousarray(records[:n].cpu().numpy())
    j = r[:, 0].copy()
    w = np.ascontiguousarray(r[:, 1])          # a fresh array whatever n (a [1] column keeps stride 2 in torch)
    f = w.view(np.int32).reshape(n, 2)[:, 0].copy()
    p = w.view(np.float32).reshape(n, 2)[:, 1].copy()
    return f, j, p


def autotune(M: int, F: int, model_only: bool = False) -> int:
    """Segment length the library picks for M taps and F filters (timed on the
    current device unless model_only)."""
    rc, n = _native.ols_autotune(int(M), int(F), _native.OLS_TUNE_MODEL if model_only else 0)
    check(rc, "ols_autotune")
    return n


class BatchPlan:
    """B independent problems of uneven size (Ns[b], M[b], F[b], N[b]; N None
    or 0 entries are autotuned), convolved by one persistent launch (or, with
    per_n, one persistent launch per distinct segment length).  tiles[b]:
    segment tiles per work item of problem b (None or 0: autotuned)."""

    def __init__(self, Ns, M, F, N=None, model_only: bool = False, per_n: bool = False, tiles=None):
        flags = (_native.OLS_TUNE_MODEL if model_only else 0) | (_native.OLS_BATCH_PER_N if per_n else 0)
        rc, handle = _native.ols_batch_plan_tiles(list(Ns), list(M), list(F), None if N is None else list(N),
                                                  None if tiles is None else list(tiles), flags)
        check(rc, "ols_batch_plan_tiles")
        self._h = handle
        self.device = torch.device("cuda", torch.cuda.current_device())
        self.B = len(Ns)
        self.Ns, self.M, self.F = list(Ns), list(M), list(F)
        self.N, self.Nout = [], []
        for b in range(self.B):
            rc, n, nout, ng = _native.ols_batch_query(self._h, b)
            check(rc, "ols_batch_query")
            self.N.append(n)
            self.Nout.append(nout)
            self.ngroups = ng
        # single launch: tiles per item and items of every problem
        self.tiles, self.items = [], []
        if not per_n:
            for b in range(self.B):
                rc, r, n = _native.ols_batch_schedule(self._h, b)
                check(rc, "ols_batch_schedule")
                self.tiles.append(r)
                self.items.append(n)
        self._keep = None

    def close(self):
        if getattr(self, "_h", None):
            _native.ols_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self) -> int:
        return self._h

    def set_filters(self, hs) -> None:
        """hs: list of B device tensors [F[b]][M[b]] complex64."""
        hs = [_input(h, "h[%d]" % b, self.device) for b, h in enumerate(hs)]
        for b, h in enumerate(hs):
            if tuple(h.shape) != (self.F[b], self.M[b]):
                raise ValueError("h[%d] must have shape [%d][%d]" % (b, self.F[b], self.M[b]))
        check(_native.ols_batch_set_filters(self._h, [h.data_ptr() for h in hs], _stream_ptr(self.device)),
              "ols_batch_set_filters")
        self._keep = list(hs)

    def outputs(self):
        """Freshly allocated outputs [F[b]][Nout[b]] for every problem."""
        return [torch.empty((f, n), dtype=torch.complex64, device=self.device) for f, n in zip(self.F, self.Nout)]

    def pointer_table(self, tensors) -> torch.Tensor:
        """Device int64 table of the tensors' data pointers (what the kernels read)."""
        return torch.tensor([t.data_ptr() for t in tensors], dtype=torch.int64, device=self.device)

    def launch(self, s_table: torch.Tensor, y_table: torch.Tensor) -> None:
        """Enqueue the batched convolution for pointer tables already on the
        device (graph-capturable: no allocation, no host synchronisation)."""
        check(_native.ols_convolve_batched(self._h, s_table.data_ptr(), y_table.data_ptr(),
                                           _stream_ptr(self.device)), "ols_convolve_batched")

    def convolve(self, ss, ys=None):
        """ss: list of B device tensors [Ns[b]]; returns the list of outputs."""
        ss = [_input(s, "s[%d]" % b, self.device) for b, s in enumerate(ss)]
        for b, s in enumerate(ss):
            if s.shape != (self.Ns[b],):
                raise ValueError("s[%d] must have %d samples" % (b, self.Ns[b]))
        if ys is None:
            ys = self.outputs()
        for b, y in enumerate(ys):
            _output(y, "y[%d]" % b, self.device)
            if tuple(y.shape) != (self.F[b], self.Nout[b]):
                raise ValueError("y[%d] has the wrong shape" % b)
        st, yt = self.pointer_table(ss), self.pointer_table(ys)
        self.launch(st, yt)
        return ys

    def status(self, reset: bool = True) -> int:
        """OR of the status words of every problem's plan (see Plan.status)."""
        rc, v = _native.ols_batch_status(self._h, reset)
        check(rc, "ols_batch_status")
        return v

    def last_launch_count(self) -> int:
        return _native.ols_batch_last_launch_count(self._h)


def convolve(s: torch.Tensor, h: torch.Tensor, N: int = 0) -> torch.Tensor:
    """One-shot convenience: plan, set filters, convolve (s [Ns], h [F][M])."""
    if h.dim() == 1:
        h = h.unsqueeze(0)
    plan = Plan(h.shape[1], h.shape[0], N)
    plan.set_filters(h.contiguous())
    y = plan.convolve(s.contiguous())
    torch.cuda.current_stream(plan.device).synchronize()
    plan.close()
    return y


from .autograd import ols_conv  # noqa: E402  (needs Plan)
