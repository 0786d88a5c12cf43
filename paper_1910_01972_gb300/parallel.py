"""Splitting one long signal's convolution across ranks (host logic).

Overlap-and-save segments are independent (Sec. 3.2), so the Nout = Ns-M+1
outputs of one signal can be cut into contiguous ranges, one per rank; rank r
computes y[:, j0:j1] from the input slice s[j0 : j1+M-1] (its outputs plus an
M-1 sample halo) with no communication.  The adjoint needs two reductions:
dh is a sum over ranks, and the input gradient of rank r's slice overlaps the
next rank's by M-1 samples, which a chain of point-to-point exchanges adds.

The second way to split is along the filter bank: rank r convolves the whole
signal with its own contiguous block of filters, so its outputs are whole
rows of y and the forward pass needs no communication at all; in the adjoint
each rank's dh rows are final and the input gradient ds is a sum over ranks
(one all-reduce of Ns samples).

``FilterSplit`` is that second split as a product call: each rank plans its
own block of filters on its own device, runs the library's kernels for it,
and the rows are gathered (forward) or ds is all-reduced (adjoint).
``SignalSplit`` is the first: each rank plans the whole bank and runs the
library's kernels on its own input slice; the output columns are gathered,
and in the adjoint the slices' overlapping input gradients are added and dh
is summed over ranks.

Collectives use torch.distributed: NCCL on the ranks' CUDA tensors, any other
backend (gloo) on host copies.
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
    Adds the M-1 entries received from rank-1 to its head, then sends its last
    M-1 entries -- received part included -- to rank+1, and returns the entries
    of input_range() (length b - a).  The ranks form a chain: a range shorter
    than M-1 has a head and a tail that overlap (an empty one, Nout < world,
    is all overlap), and what such a rank received must travel on."""
    import torch.distributed as dist
    h = M - 1
    ds = ds_slice.clone()
    if h > 0 and world > 1:
        def real(t):      # complex values travel as (re, im) pairs
            return torch.view_as_real(t) if t.is_complex() else t
        if rank > 0:
            buf = torch.empty(h, dtype=ds.dtype, device=ds.device)
            dist.recv(real(buf), src=rank - 1, group=group)
            ds[:h] += buf
        if rank + 1 < world:
            dist.send(real(ds[-h:].contiguous()), dst=rank + 1, group=group)
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


# ------------------------------------------------------------ filter-bank split
def _device_collectives(group=None) -> bool:
    import torch.distributed as dist
    return dist.get_backend(group) == "nccl"


def _rows_of(F: int, world: int):
    return [filter_range(F, world, r) for r in range(world)]


def all_gather_rows(local: torch.Tensor, F: int, group=None) -> torch.Tensor:
    """Every rank's block of rows ([f1-f0][...] as given by filter_range) gathered
    into the whole [F][...] on every rank, on `local`'s device.  Blocks are
    padded to the largest block for the collective."""
    import torch.distributed as dist
    world, rank = dist.get_world_size(group), dist.get_rank(group)
    rows = _rows_of(F, world)
    f0, f1 = rows[rank]
    if local.shape[0] != f1 - f0:
        raise ValueError("rank %d holds %d rows, expected %d" % (rank, local.shape[0], f1 - f0))
    fmax = max(b - a for a, b in rows)
    comm = local.device if _device_collectives(group) else torch.device("cpu")
    buf = torch.zeros((fmax,) + tuple(local.shape[1:]), dtype=local.dtype, device=comm)
    buf[: f1 - f0] = local.to(comm)
    parts = [torch.empty_like(buf) for _ in range(world)]
    if buf.is_complex():
        dist.all_gather([torch.view_as_real(t) for t in parts], torch.view_as_real(buf), group=group)
    else:
        dist.all_gather(parts, buf, group=group)
    whole = torch.cat([parts[r][: b - a] for r, (a, b) in enumerate(rows)], dim=0)
    return whole.to(local.device)


def all_reduce_sum(t: torch.Tensor, group=None) -> torch.Tensor:
    """Sum of every rank's `t` (all ranks receive it), on t's device."""
    import torch.distributed as dist
    comm = t.device if _device_collectives(group) else torch.device("cpu")
    out = t.to(comm, copy=True)
    dist.all_reduce(torch.view_as_real(out) if out.is_complex() else out, op=dist.ReduceOp.SUM, group=group)
    return out.to(t.device)


def all_gather_candidates(rec: torch.Tensor, count, f0: int = 0, group=None, j_shift: int = 0):
    """Candidate records (ols_candidate: int64 j; int32 f; float power, as an
    int64 tensor [capacity][2]) of every rank gathered on every rank, in rank
    order, with this rank's filter offset f0 added to f and j_shift to j.
    count: the rank's count (a device tensor or an int; may exceed the
    capacity: only stored records travel).  Returns (records [kept][2] int64
    on rec's device, total count over ranks)."""
    import torch.distributed as dist
    world = dist.get_world_size(group)
    comm = rec.device if _device_collectives(group) else torch.device("cpu")
    cap = rec.shape[0]
    n_all = torch.tensor([int(count.item()) if torch.is_tensor(count) else int(count), 0], dtype=torch.int64,
                         device=comm)
    n_all[1] = min(int(n_all[0].item()), cap)
    sizes = [torch.empty_like(n_all) for _ in range(world)]
    dist.all_gather(sizes, n_all, group=group)
    kept = [int(t[1].item()) for t in sizes]
    total = sum(int(t[0].item()) for t in sizes)
    nmax = max(kept + [1])
    mine = rec[: kept[dist.get_rank(group)]].clone()
    mine[:, 0] += j_shift                                      # the record's j, made global
    words = mine.view(torch.int32).view(-1, 4)
    words[:, 2] += f0                                          # the record's f, made global
    buf = torch.zeros((nmax, 4), dtype=torch.int32, device=comm)
    buf[: words.shape[0]] = words.to(comm)
    parts = [torch.empty_like(buf) for _ in range(world)]
    dist.all_gather(parts, buf, group=group)
    whole = torch.cat([parts[r][: kept[r]] for r in range(world)], dim=0).contiguous()
    return whole.view(torch.int64).view(-1, 2).to(rec.device), total


class FilterSplit:
    """A bank of F filters of M taps split across the ranks of `group`: this
    rank owns filters [f0, f1) (``filter_range``) and convolves the whole
    signal with them on the current CUDA device through the library's
    kernels.  Segments and filters are independent (Sec. 3.2), so the forward
    pass needs no communication; ``convolve`` gathers the rows so every rank
    gets y [F][Nout]; ``detect`` and ``peaks`` gather only the selected
    candidates (Sec. 4.4).  In the adjoint each rank's dh rows are final and ds is
    the sum of every rank's contribution (one all-reduce of Ns samples).
    A rank without filters (F < world size) contributes zeros."""

    def __init__(self, M: int, F: int, N: int = 0, group=None):
        import torch.distributed as dist
        from . import Plan
        self.group = group
        self.world, self.rank = dist.get_world_size(group), dist.get_rank(group)
        self.M, self.F = int(M), int(F)
        self.f0, self.f1 = filter_range(self.F, self.world, self.rank)
        self.device = torch.device("cuda", torch.cuda.current_device())
        self.plan = Plan(self.M, self.f1 - self.f0, N) if self.f1 > self.f0 else None
        self.N = self.plan.N if self.plan is not None else None

    def close(self):
        if self.plan is not None:
            self.plan.close()
            self.plan = None

    def set_filters(self, h: torch.Tensor) -> None:
        """h: the whole bank [F][M] complex64 (same on every rank); this rank
        keeps its own rows."""
        if tuple(h.shape) != (self.F, self.M):
            raise ValueError("h must have shape [%d][%d]" % (self.F, self.M))
        if self.plan is not None:
            self.plan.set_filters(h[self.f0:self.f1].to(self.device).contiguous())

    def convolve_local(self, s: torch.Tensor) -> torch.Tensor:
        """This rank's rows of y: [f1-f0][Ns-M+1] (no communication)."""
        Nout = s.shape[0] - self.M + 1
        if self.plan is None:
            return torch.empty((0, Nout), dtype=torch.complex64, device=self.device)
        return self.plan.convolve(s)

    def convolve(self, s: torch.Tensor) -> torch.Tensor:
        """y [F][Ns-M+1] on every rank: local rows, then one row gather."""
        return all_gather_rows(self.convolve_local(s), self.F, self.group)

    def _select(self, mode: str, s: torch.Tensor, threshold: float, capacity: int):
        if self.plan is None:
            rec = torch.zeros((max(int(capacity), 1), 2), dtype=torch.int64, device=self.device)
            cnt = torch.zeros(1, dtype=torch.int64, device=self.device)
        elif mode == "peaks":
            rec, cnt = self.plan.convolve_peaks(s, threshold, capacity)
        else:
            rec, cnt = self.plan.convolve_detect(s, threshold, capacity)
        return all_gather_candidates(rec, cnt, self.f0, self.group)

    def detect(self, s: torch.Tensor, threshold: float, capacity: int):
        """Candidates |y_f[j]|^2 >= threshold over the whole bank, on every rank:
        each rank selects among its own filters (at most `capacity` records
        each) and only the records travel.  Returns (records [n][2] int64 in
        the ols_candidate layout with global f, see ``decode_candidates``;
        total count over ranks, which exceeds n when a rank overflowed)."""
        return self._select("detect", s, threshold, capacity)

    def peaks(self, s: torch.Tensor, threshold: float, capacity: int):
        """Peaks of the power over the whole bank (``Plan.convolve_peaks`` on
        each rank's filters), gathered like ``detect``."""
        return self._select("peaks", s, threshold, capacity)

    def convolve_backward(self, s: torch.Tensor, g: torch.Tensor, want_ds: bool = True, want_dh: bool = True):
        """g: the whole output gradient [F][Ns-M+1] (same on every rank).
        Returns (ds [Ns] summed over ranks, dh [F][M] gathered), each None if
        not wanted."""
        Ns = s.shape[0]
        if tuple(g.shape) != (self.F, Ns - self.M + 1):
            raise ValueError("g must have shape [F][Ns-M+1]")
        ds_loc = dh_loc = None
        if self.plan is not None:
            ds_loc, dh_loc = self.plan.convolve_backward(s, g[self.f0:self.f1].contiguous(), want_ds, want_dh)
        ds = dh = None
        if want_ds:
            if ds_loc is None:
                ds_loc = torch.zeros(Ns, dtype=torch.complex64, device=self.device)
            ds = all_reduce_sum(ds_loc, self.group)
        if want_dh:
            if dh_loc is None:
                dh_loc = torch.empty((self.f1 - self.f0, self.M), dtype=torch.complex64, device=self.device)
            dh = all_gather_rows(dh_loc, self.F, self.group)
        return ds, dh


# ------------------------------------------------------------ output-range split
def _comm_device(t: torch.Tensor, group=None) -> torch.device:
    return t.device if _device_collectives(group) else torch.device("cpu")


def all_gather_pieces(local: torch.Tensor, sizes, dim: int, group=None) -> torch.Tensor:
    """Every rank's piece of `local` along `dim` (rank r's is sizes[r] long)
    concatenated in rank order on every rank, on `local`'s device.  Pieces are
    padded to the largest for the collective."""
    import torch.distributed as dist
    world, rank = dist.get_world_size(group), dist.get_rank(group)
    if local.shape[dim] != sizes[rank]:
        raise ValueError("rank %d holds %d entries, expected %d" % (rank, local.shape[dim], sizes[rank]))
    comm = _comm_device(local, group)
    shape = list(local.shape)
    shape[dim] = max(list(sizes) + [1])
    buf = torch.zeros(shape, dtype=local.dtype, device=comm)
    buf.narrow(dim, 0, sizes[rank]).copy_(local.to(comm))
    parts = [torch.empty_like(buf) for _ in range(world)]
    if buf.is_complex():
        dist.all_gather([torch.view_as_real(t) for t in parts], torch.view_as_real(buf), group=group)
    else:
        dist.all_gather(parts, buf, group=group)
    whole = torch.cat([parts[r].narrow(dim, 0, sizes[r]) for r in range(world)], dim=dim)
    return whole.to(local.device)


class SignalSplit:
    """One long signal split across the ranks of `group` by output range
    (``shard``): rank r computes y[:, j0:j1] for the whole bank of F filters
    from the input slice s[j0 : j1+M-1] with the library's kernels on the
    current CUDA device -- no communication on the forward pass, since
    segments are independent (Sec. 3.2).  ``convolve`` gathers the columns so
    every rank gets y [F][Nout].  In the adjoint the gradients of two
    neighbouring slices overlap by M-1 inputs (one send / receive adds them,
    ``reduce_input_gradient``) and dh is summed over ranks.  A rank whose
    output range is empty (Nout < world size) contributes nothing."""

    def __init__(self, M: int, F: int, N: int = 0, group=None):
        import torch.distributed as dist
        from . import Plan
        self.group = group
        self.world, self.rank = dist.get_world_size(group), dist.get_rank(group)
        self.M, self.F = int(M), int(F)
        self.device = torch.device("cuda", torch.cuda.current_device())
        self.plan = Plan(self.M, self.F, N)
        self.N = self.plan.N

    def close(self):
        if self.plan is not None:
            self.plan.close()
            self.plan = None

    def set_filters(self, h: torch.Tensor) -> None:
        """h: the whole bank [F][M] complex64 (same on every rank)."""
        self.plan.set_filters(h.to(self.device).contiguous())

    def shard(self, Ns: int):
        """(j0, j1, i0, i1) of this rank for a signal of Ns samples."""
        return shard(Ns, self.M, self.world, self.rank)

    def convolve_local(self, s: torch.Tensor) -> torch.Tensor:
        """This rank's columns of y, [F][j1-j0], from the whole signal s (only
        its slice is read)."""
        j0, j1, i0, i1 = self.shard(s.shape[0])
        if j1 == j0:
            return torch.empty((self.F, 0), dtype=torch.complex64, device=self.device)
        return self.plan.convolve(s[i0:i1])

    def convolve(self, s: torch.Tensor) -> torch.Tensor:
        """y [F][Ns-M+1] on every rank: local columns, then one column gather."""
        Nout = s.shape[0] - self.M + 1
        sizes = [b - a for a, b in (output_range(Nout, self.world, r) for r in range(self.world))]
        return all_gather_pieces(self.convolve_local(s), sizes, 1, self.group)

    def _select(self, mode: str, s: torch.Tensor, threshold: float, capacity: int):
        Ns = s.shape[0]
        Nout = Ns - self.M + 1
        j0, j1, _, _ = self.shard(Ns)
        if j1 == j0:
            return all_gather_candidates(torch.zeros((0, 2), dtype=torch.int64, device=self.device), 0, 0,
                                         self.group)
        # peaks look at j - 1 and j + 1: the slice is widened by one output on each side
        # that has a neighbouring range, and only this rank's outputs are kept
        a = j0 - 1 if (mode == "peaks" and j0 > 0) else j0
        b = j1 + 1 if (mode == "peaks" and j1 < Nout) else j1
        fn = self.plan.convolve_peaks if mode == "peaks" else self.plan.convolve_detect
        rec, cnt = fn(s[a:b + self.M - 1], threshold, capacity)
        count = int(cnt.item())
        stored = rec[: min(count, rec.shape[0])]
        keep = stored[(stored[:, 0] >= j0 - a) & (stored[:, 0] < j1 - a)]
        # past the capacity the total is what the kernel found (the one-output widening included)
        total = keep.shape[0] if count <= rec.shape[0] else count
        return all_gather_candidates(keep, total, 0, self.group, a)

    def detect(self, s: torch.Tensor, threshold: float, capacity: int):
        """Candidates |y_f[j]|^2 >= threshold over the whole signal, on every
        rank: each rank selects in its own output range, only the records
        travel (j made global).  Returns (records, total) like
        ``FilterSplit.detect``; a rank past its capacity counts what its
        kernel found."""
        return self._select("detect", s, threshold, capacity)

    def peaks(self, s: torch.Tensor, threshold: float, capacity: int):
        """Peaks of the power over the whole signal: each rank's slice is
        widened by one output towards each neighbouring range so that the
        outputs at its range's ends see both neighbours; the two ends of the
        whole stream keep their one-sided rule.  Gathered like ``detect``."""
        return self._select("peaks", s, threshold, capacity)

    def convolve_backward(self, s: torch.Tensor, g: torch.Tensor, want_ds: bool = True, want_dh: bool = True):
        """g: the whole output gradient [F][Ns-M+1] (same on every rank; only
        this rank's columns are read).  Returns (ds [Ns], dh [F][M]) on every
        rank, each None if not wanted."""
        Ns = s.shape[0]
        if tuple(g.shape) != (self.F, Ns - self.M + 1):
            raise ValueError("g must have shape [F][Ns-M+1]")
        j0, j1, i0, i1 = self.shard(Ns)
        ds_loc = torch.zeros(i1 - i0, dtype=torch.complex64, device=self.device)
        dh_loc = torch.zeros((self.F, self.M), dtype=torch.complex64, device=self.device)
        if j1 > j0:
            a, b = self.plan.convolve_backward(s[i0:i1], g[:, j0:j1].contiguous(), want_ds, want_dh)
            ds_loc = a if a is not None else ds_loc
            dh_loc = b if b is not None else dh_loc
        ds = dh = None
        if want_ds:
            comm = _comm_device(ds_loc, self.group)
            mine = reduce_input_gradient(ds_loc.to(comm), self.M, self.world, self.rank, self.group)
            sizes = [b - a for a, b in (input_range(Ns, self.M, self.world, r) for r in range(self.world))]
            ds = all_gather_pieces(mine.to(self.device), sizes, 0, self.group)
        if want_dh:
            dh = all_reduce_sum(dh_loc, self.group)
        return ds, dh
