"""Seeded synthetic inputs for overlap-and-save convolution workloads.

This module serves both the GPU path and the CPU oracle.  It holds no step of
the convolution method: it only draws signals, filter taps, loss weights and
batch shapes.  Every value is drawn with numpy's PCG64 from a fixed seed, in
a fixed order (signal, then filters, then weights, then batch shapes), in
FP64 and then rounded to complex64; the rounded values are what both sides
consume.

The paper names no dataset (Sec. 4 uses generic signals of a stated length
and filter banks of stated sizes), so every workload here is synthetic:

* signal: real and imaginary parts i.i.d. uniform[-1, 1];
* filters: real and imaginary parts i.i.d. N(0, 1/2) ("complex Gaussian"),
  optionally times a symmetric Hann window 0.5(1 - cos(2 pi k/(M-1))), then
  scaled to unit L2 norm per filter;
* loss weights: uniform[0, 1], one weight per output index shared by all
  filters;
* real-to-real workloads: signal i.i.d. uniform[-1, 1], filter taps i.i.d.
  N(0, 1) (optionally Hann-windowed), unit L2 per filter.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List

import numpy as np

SEED_BASE = 1910_01972


def rng(config_index: int, salt: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(SEED_BASE + int(config_index) + 1000 * int(salt)))


def signal(g: np.random.Generator, Ns: int) -> np.ndarray:
    """complex64 signal with re, im i.i.d. uniform[-1, 1]."""
    re = g.uniform(-1.0, 1.0, size=Ns)
    im = g.uniform(-1.0, 1.0, size=Ns)
    return (re + 1j * im).astype(np.complex64)


def hann(M: int) -> np.ndarray:
    """Symmetric Hann window of length M (end taps are zero for M > 1)."""
    if M == 1:
        return np.ones(1)
    k = np.arange(M, dtype=np.float64)
    return 0.5 * (1.0 - np.cos(2.0 * math.pi * k / (M - 1)))


def filters(g: np.random.Generator, F: int, M: int, window: bool = False) -> np.ndarray:
    """complex64 filter bank [F][M]: complex Gaussian taps, unit L2 per filter."""
    re = g.normal(0.0, math.sqrt(0.5), size=(F, M))
    im = g.normal(0.0, math.sqrt(0.5), size=(F, M))
    h = re + 1j * im
    if window:
        h = h * hann(M)[None, :]
    nrm = np.linalg.norm(h, axis=1, keepdims=True)
    nrm[nrm == 0] = 1.0
    return (h / nrm).astype(np.complex64)


def real_signal(g: np.random.Generator, Ns: int) -> np.ndarray:
    """float32 real signal, i.i.d. uniform[-1, 1]."""
    return g.uniform(-1.0, 1.0, size=Ns).astype(np.float32)


def real_filters(g: np.random.Generator, F: int, M: int, window: bool = False) -> np.ndarray:
    """float32 real filter bank [F][M]: i.i.d. N(0, 1) taps (optionally times
    the symmetric Hann window), unit L2 per filter."""
    h = g.normal(0.0, 1.0, size=(F, M))
    if window:
        h = h * hann(M)[None, :]
    nrm = np.linalg.norm(h, axis=1, keepdims=True)
    nrm[nrm == 0] = 1.0
    return (h / nrm).astype(np.float32)


def weights(g: np.random.Generator, n: int) -> np.ndarray:
    """Loss weights w[n] ~ uniform[0, 1] (float32)."""
    return g.uniform(0.0, 1.0, size=n).astype(np.float32)


# --------------------------------------------------------------------------
# Named workloads (the shapes of the paper's experiments, Sec. 4, and the
# benchmark configurations built on them).
# --------------------------------------------------------------------------

@dataclasses.dataclass
class Plain:
    name: str
    Ns: int
    F: int
    M: int
    N: int
    window: bool
    index: int


PLAIN_1x1 = Plain("plain_1x1_Ns65536_M64_N512", 65536, 1, 64, 512, False, 0)
PLAIN_BANK = Plain("bank_Ns8388608_F32_M257_N2048", 1 << 23, 32, 257, 2048, True, 1)
DIFF = Plain("diff_Ns4194304_F16_M129_N1024", 1 << 22, 16, 129, 1024, False, 3)
TC_SPLIT = Plain("tc_Ns16777216_F64_M512_N4096", 1 << 24, 64, 512, 4096, False, 4)


# real-to-real form (Sec. 3.4's R2R variant) on the filter-bank shape
R2R_BANK = Plain("r2r_bank_Ns8388608_F32_M257_N2048", 1 << 23, 32, 257, 2048, True, 5)


def real_inputs(cfg: Plain, Ns: int | None = None):
    """(s, h) float32 for a real-to-real workload; ``Ns`` overrides the signal length."""
    g = rng(cfg.index)
    s = real_signal(g, cfg.Ns if Ns is None else Ns)
    h = real_filters(g, cfg.F, cfg.M, window=cfg.window)
    return s, h


def plain_inputs(cfg: Plain, Ns: int | None = None):
    """(s, h) for a plain workload; ``Ns`` overrides the signal length."""
    g = rng(cfg.index)
    s = signal(g, cfg.Ns if Ns is None else Ns)
    h = filters(g, cfg.F, cfg.M, window=cfg.window)
    return s, h


def diff_inputs(cfg: Plain = DIFF, Ns: int | None = None):
    """(s, h, w) for the differentiable workload (loss sum_f sum_n w[n]|y_f[n]|^2)."""
    g = rng(cfg.index)
    Ns = cfg.Ns if Ns is None else Ns
    s = signal(g, Ns)
    h = filters(g, cfg.F, cfg.M, window=cfg.window)
    w = weights(g, Ns - cfg.M + 1)
    return s, h, w


BATCH_M_CHOICES = (33, 65, 129, 257, 513, 1025)


@dataclasses.dataclass
class BatchSpec:
    Ns: List[int]
    F: List[int]
    M: List[int]


def batch_spec(B: int = 64, lo_log2: float = 16.0, hi_log2: float = 22.0,
               F_lo: int = 8, F_hi: int = 128, index: int = 2) -> BatchSpec:
    """Shapes of an uneven batch: lengths log-uniform in [2^lo, 2^hi],
    F uniform in {F_lo..F_hi}, M uniform over BATCH_M_CHOICES."""
    g = rng(index, salt=1)
    Ns = [int(round(2.0 ** g.uniform(lo_log2, hi_log2))) for _ in range(B)]
    F = [int(g.integers(F_lo, F_hi + 1)) for _ in range(B)]
    M = [int(BATCH_M_CHOICES[g.integers(0, len(BATCH_M_CHOICES))]) for _ in range(B)]
    Ns = [max(n, m) for n, m in zip(Ns, M)]
    return BatchSpec(Ns, F, M)


def batch_inputs(spec: BatchSpec, index: int = 2):
    """Per-problem (s_b, h_b) lists for an uneven batch."""
    g = rng(index)
    ss = [signal(g, n) for n in spec.Ns]
    hs = [filters(g, f, m) for f, m in zip(spec.F, spec.M)]
    return ss, hs


def device_signal(Ns: int, seed: int, real: bool = False, device: str = "cuda"):
    """A signal too large to draw on the host: re (and im) i.i.d. uniform[-1, 1]
    drawn on the device by torch's seeded generator (Philox), complex64 (or
    float32 when real).  Both sides read the same device values: tests gather
    the windows they check and pass them to the oracle."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(SEED_BASE + int(seed))
    n = Ns if real else 2 * Ns
    x = torch.rand(n, generator=g, device=device, dtype=torch.float32)
    x.mul_(2.0).sub_(1.0)
    return x if real else x.view(torch.complex64)
