"""Multi-rank splitting of one signal (paper_1910_01972_gb300.parallel) on CPU:
world size 2 over gloo, each rank's shard computed by the FP64 oracle, the
shards combined by the module's own collectives (row gather, sum).  The same
split with the library's kernels on each rank is tests/test_parallel_gpu.py."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

from paper_1910_01972_gb300 import parallel


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("Ns,M,world", [(1000, 33, 2), (1000, 33, 3), (70, 70, 2), (9, 1, 4), (100, 40, 7)])
def test_shards_tile_the_outputs_and_inputs(Ns, M, world):
    Nout = Ns - M + 1
    seen_out = np.zeros(Nout, int)
    seen_in = np.zeros(Ns, int)
    for r in range(world):
        j0, j1, i0, i1 = parallel.shard(Ns, M, world, r)
        assert i0 == j0 and i1 == j1 + M - 1 and 0 <= i0 <= i1 <= Ns
        seen_out[j0:j1] += 1
        a, b = parallel.input_range(Ns, M, world, r)
        seen_in[a:b] += 1
    assert np.all(seen_out == 1) and np.all(seen_in == 1)


def _worker(rank, world, port, Ns, M, F, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch.distributed as dist
    import oracle
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        g = np.random.Generator(np.random.PCG64(42))
        s = (g.uniform(-1, 1, Ns) + 1j * g.uniform(-1, 1, Ns)).astype(np.complex64)
        h = (g.normal(size=(F, M)) + 1j * g.normal(size=(F, M))).astype(np.complex64)
        gy = g.normal(size=(F, Ns - M + 1)) + 1j * g.normal(size=(F, Ns - M + 1))
        j0, j1, i0, i1 = parallel.shard(Ns, M, world, rank)
        # forward: each rank convolves its slice, no communication
        empty = j1 == j0                      # Nout < world: a rank without outputs
        y_loc = torch.from_numpy(np.zeros((F, 0), np.complex128) if empty else oracle.conv(s[i0:i1], h))
        parts = [None] * world
        dist.all_gather_object(parts, (j0, y_loc.numpy()))
        # adjoint on the slice, then the two reductions
        if empty:
            ds_loc, dh_loc = np.zeros(i1 - i0, np.complex128), np.zeros((F, M), np.complex128)
        else:
            ds_loc, dh_loc = oracle.adjoint(s[i0:i1], h, gy[:, j0:j1])
        ds_mine = parallel.reduce_input_gradient(torch.from_numpy(ds_loc), M, world, rank)
        dh_all = parallel.reduce_filter_gradient(torch.from_numpy(dh_loc))
        ds_parts = [None] * world
        dist.all_gather_object(ds_parts, (parallel.input_range(Ns, M, world, rank), ds_mine.numpy()))
        if rank == 0:
            y = np.concatenate([p[1] for p in sorted(parts, key=lambda p: p[0])], axis=1)
            y_ref = oracle.conv(s, h)
            ds = np.zeros(Ns, np.complex128)
            for (a, b), v in ds_parts:
                ds[a:b] = v
            ds_ref, dh_ref = oracle.adjoint(s, h, gy)
            q.put((bool(np.array_equal(y, y_ref)),
                   float(np.max(np.abs(ds - ds_ref)) / np.max(np.abs(ds_ref))),
                   float(np.max(np.abs(dh_all.numpy() - dh_ref)) / np.max(np.abs(dh_ref)))))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("Ns,M,world", [(3000, 65, 2), (100, 40, 7), (41, 40, 3), (500, 1, 3)])
def test_two_rank_split_equals_whole_signal(Ns, M, world):
    """Output-range split: outputs concatenated, input gradients of neighbouring
    slices added, dh summed.  Ranges shorter than M-1 (a slice's head and tail
    overlap, so a rank must pass on what it received) and an empty range
    (Nout < world) included."""
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    F = 3
    procs = [ctx.Process(target=_worker, args=(r, world, port, Ns, M, F, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    for p in procs:
        assert p.exitcode == 0, "rank failed"
    same_y, e_ds, e_dh = q.get(timeout=5)
    assert same_y                      # each output is the same sequential sum: identical
    assert e_ds < 1e-12 and e_dh < 1e-12


def _filter_worker(rank, world, port, Ns, M, F, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch.distributed as dist
    import oracle
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        g = np.random.Generator(np.random.PCG64(43))
        s = (g.uniform(-1, 1, Ns) + 1j * g.uniform(-1, 1, Ns)).astype(np.complex64)
        h = (g.normal(size=(F, M)) + 1j * g.normal(size=(F, M))).astype(np.complex64)
        gy = g.normal(size=(F, Ns - M + 1)) + 1j * g.normal(size=(F, Ns - M + 1))
        f0, f1 = parallel.filter_range(F, world, rank)
        # forward: whole signal, own filters, no communication; then the
        # library's row gather (gloo: through host tensors)
        y_loc = oracle.conv(s, h[f0:f1]) if f1 > f0 else np.zeros((0, Ns - M + 1), np.complex128)
        y = parallel.all_gather_rows(torch.from_numpy(y_loc), F).numpy()
        # adjoint: own dh rows are final, ds is summed over ranks
        if f1 > f0:
            ds_loc, dh_loc = oracle.adjoint(s, h[f0:f1], gy[f0:f1])
        else:
            ds_loc, dh_loc = np.zeros(Ns, np.complex128), np.zeros((0, M), np.complex128)
        ds_all = parallel.all_reduce_sum(torch.from_numpy(ds_loc)).numpy()
        assert np.array_equal(ds_all, parallel.reduce_signal_gradient(torch.from_numpy(ds_loc)).numpy())
        dh = parallel.all_gather_rows(torch.from_numpy(dh_loc), F).numpy()
        if rank == 0:
            ds_ref, dh_ref = oracle.adjoint(s, h, gy)
            q.put((bool(np.array_equal(y, oracle.conv(s, h))), bool(np.array_equal(dh, dh_ref)),
                   float(np.max(np.abs(ds_all - ds_ref)) / np.max(np.abs(ds_ref)))))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("F", [5, 1, 2])
def test_two_rank_filter_split_equals_whole_bank(F):
    """The filter-bank split (no forward communication; ds summed over ranks)
    reproduces the unsplit result; F = 1 leaves one rank without filters."""
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    Ns, M = 1500, 33
    procs = [ctx.Process(target=_filter_worker, args=(r, world, port, Ns, M, F, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    for p in procs:
        assert p.exitcode == 0, "rank failed"
    same_y, same_dh, e_ds = q.get(timeout=5)
    assert same_y and same_dh
    assert e_ds < 1e-12


@pytest.mark.parametrize("F,world", [(32, 4), (5, 2), (1, 2), (7, 7), (3, 8)])
def test_filter_ranges_tile_the_bank(F, world):
    seen = np.zeros(F, int)
    for r in range(world):
        f0, f1 = parallel.filter_range(F, world, r)
        assert 0 <= f0 <= f1 <= F
        seen[f0:f1] += 1
    assert np.all(seen == 1)


def _records(j, f, p, cap):
    rec = np.zeros(cap, dtype=[("j", "<i8"), ("f", "<i4"), ("power", "<f4")])
    n = min(len(j), cap)
    rec["j"][:n], rec["f"][:n], rec["power"][:n] = j[:n], f[:n], p[:n]
    return torch.from_numpy(rec.view(np.int64).reshape(cap, 2).copy())


def _cand_worker(rank, world, port, F, counts, cap, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch.distributed as dist
    from paper_1910_01972_gb300 import decode_candidates
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        def local(r):
            # rank r's candidates: local filter indices, found count counts[r] (may exceed cap)
            f0, f1 = parallel.filter_range(F, world, r)
            n = counts[r]
            nf = max(f1 - f0, 1)
            j = 1000 * r + np.arange(n, dtype=np.int64) * 7
            fl = (np.arange(n) % nf).astype(np.int32)
            p = (0.5 + r + np.arange(n) / 8).astype(np.float32)
            return f0, j, fl, p
        f0, j, fl, p = local(rank)
        rec, total = parallel.all_gather_candidates(_records(j, fl, p, cap), torch.tensor([counts[rank]]), f0,
                                                    j_shift=100_000 * rank)
        if rank == 0:
            got = decode_candidates(rec, rec.shape[0])
            want = [np.concatenate(a) for a in zip(*[
                (fl_[:cap] + f0_, j_[:cap] + 100_000 * r, p_[:cap])
                for r, (f0_, j_, fl_, p_) in enumerate(local(r) for r in range(world))])]
            q.put((total, [a.tolist() for a in got], [a.tolist() for a in want]))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("F,world,counts", [(5, 2, (3, 4)), (7, 3, (0, 9, 2)), (2, 3, (5, 6, 0)), (4, 2, (0, 0))])
def test_candidates_gathered_with_global_filter_index(F, world, counts):
    """Candidate records of each rank (its own filters, at most `cap` stored,
    any count found) gathered in rank order on every rank, f made global, the
    total count summed; a rank without filters or candidates contributes none."""
    cap = 5
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_cand_worker, args=(r, world, port, F, counts, cap, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    for p in procs:
        assert p.exitcode == 0, "rank failed"
    total, got, want = q.get(timeout=5)
    assert total == sum(counts)
    assert got == want
