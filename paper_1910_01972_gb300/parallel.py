"""Splitting one long signal's convolution across ranks (host logic).

Overlap-and-save segments are independent (Sec. 3.2), so the Nout = Ns-M+1
outputs of one signal can be cut into contiguous ranges, one per rank; rank r
computes y[:, j0:j1] from the input slice s[j0 : j1+M-1] (its outputs plus an
M-1 sample halo) with no communication.  The adjoint needs two reductions:
dh is a sum over ranks, and the input gradient of rank r's slice overlaps the
next rank's by M-1 samples, which one point-to-point exchange adds.

The second way to split is along the filter bank: rank r convolves the whole
signal with its own contiguous block of filters, so its outputs are whole
rows of y and the forward pass needs no communication at all; in the adjoint
each rank's dh rows are final and the input gradient ds is a sum over ranks
(one all-reduce of Ns samples).

Collectives use torch.distributed (gloo on CPU tensors, NCCL on CUDA tensors);
the convolution itself is the caller's (the library's kernels on a GPU).
"""
from __future__ import annotations

import torch


def output_range(Nout: int, world: int, rank: int):
    """[j0, j1) of the outputs owned by `rank` (contiguous, sizes differ by at most one)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank / world size")
    base, extra = divmod(Nout, world)
    j0 = rank * base + min(rank, extra)
    j1 = j0 + base + (1 if rank < extra else 0)
    return j0, j1


def shard(Ns: int, M: int, world: int, rank: int):
    """(j0, j1, i0, i1): outputs [j0, j1) of `rank` and the input slice [i0, i1)
    that produces them (i0 = j0, i1 = j1 + M - 1)."""
    if M < 1 or Ns < M:
        raise ValueError("need 1 <= M <= Ns")
    j0, j1 = output_range(Ns - M + 1, world, rank)
    return j0, j1, j0, j1 + M - 1


def input_range(Ns: int, M: int, world: int, rank: int):
    """[a, b) of the input indices whose gradient `rank` finally holds: its
    slice minus the M-1 tail handed to the next rank (the last rank keeps it)."""
    j0, j1, i0, i1 = shard(Ns, M, world, rank)
    return (i0, i1) if rank == world - 1 else (i0, j1)


def reduce_input_gradient(ds_slice: torch.Tensor, M: int, world: int, rank: int, group=None) -> torch.Tensor:
    """ds_slice: the gradient w.r.t. this rank's input slice (length i1 - i0).
    Sends its last M-1 entries to rank+1, adds the M-1 received from rank-1 to
    its head, and returns the entries of input_range() (length b - a)."""
    import torch.distributed as dist
    h = M - 1
    ds = ds_slice.clone()
    if h > 0 and world > 1:
        if rank + 1 < world:
            dist.send(ds[-h:].contiguous(), dst=rank + 1, group=group)
        if rank > 0:
            buf = torch.empty(h, dtype=ds.dtype, device=ds.device)
            dist.recv(buf, src=rank - 1, group=group)
            ds[:h] += buf
    if rank + 1 < world and h > 0:
        return ds[:-h]
    return ds


def reduce_filter_gradient(dh: torch.Tensor, group=None) -> torch.Tensor:
    """Sum of the ranks' filter gradients (all ranks receive it)."""
    import torch.distributed as dist
    out = dh.clone()
    dist.all_reduce(out, op=dist.ReduceOp.SUM, group=group)
    return out


def filter_range(F: int, world: int, rank: int):
    """[f0, f1) of the filters (rows of y, dh) owned by `rank` when the bank is
    split across ranks (contiguous, sizes differ by at most one; a rank may
    own none when F < world)."""
    return output_range(F, world, rank)


def reduce_signal_gradient(ds: torch.Tensor, group=None) -> torch.Tensor:
    """Filter-split adjoint: the input gradient is the sum of every rank's
    contribution (all ranks receive it)."""
    import torch.distributed as dist
    out = ds.clone()
    dist.all_reduce(out, op=dist.ReduceOp.SUM, group=group)
    return out
