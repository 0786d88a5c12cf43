"""The filter-bank split across ranks (parallel.FilterSplit) with the
library's kernels on every rank.

World size 2 and 3 over gloo (host collectives), every rank on cuda:0: the
ranks' kernels are independent launches that never wait on one another, and
the only exchanges (row gather, ds sum) go through host memory.  Blocks of
uneven size and idle ranks (F < world size) included.  Rank 0 checks
y, ds and dh against the FP64 oracle at the parity tolerances, and y and dh
bit for bit against one unsplit plan (each filter's rows come from the same
kernel arithmetic whichever plan holds the filter); threshold and peak
candidates gathered from the ranks equal the unsplit plan's exactly."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

from paper_1910_01972_gb300 import build as _build

pytestmark = pytest.mark.gpu
TOL, TOL_DS, TOL_DH = 2e-6, 2e-6, 1e-5


@pytest.fixture(scope="module", autouse=True)
def built():
    _build.build()
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, Ns, M, F, N, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch.distributed as dist
    import oracle
    import synth
    from paper_1910_01972_gb300 import Plan, parallel
    torch.cuda.set_device(0)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        g = np.random.Generator(np.random.PCG64(700 + F))
        s_np, h_np = synth.signal(g, Ns), synth.filters(g, F, M)
        gy_np = (g.normal(size=(F, Ns - M + 1)) + 1j * g.normal(size=(F, Ns - M + 1))).astype(np.complex64)
        s, h, gy = (torch.from_numpy(a).cuda() for a in (s_np, h_np, gy_np))
        fs = parallel.FilterSplit(M, F, N)
        fs.set_filters(h)
        y = fs.convolve(s)
        ds, dh = fs.convolve_backward(s, gy)
        torch.cuda.synchronize()
        launched = fs.plan.last_launch_count() if fs.plan is not None else 0
        # candidate selection on each rank's filters, only the records gathered
        p_all = (y.real ** 2 + y.imag ** 2)
        thr = float(torch.quantile(p_all.flatten()[: 1 << 16], 0.99).item())
        cand = {m: getattr(fs, m)(s, thr, 1 << 14) for m in ("detect", "peaks")}
        torch.cuda.synchronize()
        fs.close()
        if rank == 0:
            whole = Plan(M, F, N)
            whole.set_filters(h)
            y1 = whole.convolve(s)
            ds1, dh1 = whole.convolve_backward(s, gy)
            same_cand = True
            from paper_1910_01972_gb300 import decode_candidates
            for m, fn in (("detect", whole.convolve_detect), ("peaks", whole.convolve_peaks)):
                rec1, cnt1 = fn(s, thr, 1 << 14)
                torch.cuda.synchronize()
                rec, total = cand[m]
                a1 = set(zip(*[x.tolist() for x in decode_candidates(rec1, int(cnt1.item()))]))
                a2 = set(zip(*[x.tolist() for x in decode_candidates(rec, rec.shape[0])]))
                same_cand = same_cand and total == int(cnt1.item()) and a1 == a2 and len(a1) > 0
            torch.cuda.synchronize()
            whole.close()
            y_ref = oracle.conv(s_np, h_np)
            ds_ref, dh_ref = oracle.adjoint(s_np, h_np, gy_np)
            q.put({"y_err": oracle.max_stream_rel_l2(y.cpu().numpy(), y_ref),
                   "ds_err": oracle.rel_l2(ds.cpu().numpy(), ds_ref),
                   "dh_err": oracle.max_stream_rel_l2(dh.cpu().numpy(), dh_ref),
                   "y_bitwise": bool(torch.equal(y, y1)), "dh_bitwise": bool(torch.equal(dh, dh1)),
                   "ds_vs_whole": oracle.rel_l2(ds.cpu().numpy(), ds1.cpu().numpy().astype(np.complex128)),
                   "launched": launched, "same_candidates": same_cand})
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("F,world", [(5, 2), (1, 2), (7, 3), (2, 3)])
def test_filter_split_ranks_run_the_kernels(F, world):
    Ns, M, N = 50_000, 129, 1024
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, Ns, M, F, N, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
    for p in procs:
        assert p.exitcode == 0, "rank failed"
    r = q.get(timeout=5)
    assert r["y_err"] <= TOL and r["ds_err"] <= TOL_DS and r["dh_err"] <= TOL_DH, r
    assert r["y_bitwise"] and r["dh_bitwise"], r
    # ds: a sum over ranks in another order than the unsplit plan's; within rounding
    assert r["ds_vs_whole"] <= 1e-6, r
    assert r["launched"] == 3                # rank 0's adjoint call: its three kernels
    assert r["same_candidates"], r           # detect and peaks over the split bank = the unsplit plan's


def _signal_worker(rank, world, port, Ns, M, F, N, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch.distributed as dist
    import oracle
    import synth
    from paper_1910_01972_gb300 import parallel
    torch.cuda.set_device(0)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        g = np.random.Generator(np.random.PCG64(800 + Ns + world))
        s_np, h_np = synth.signal(g, Ns), synth.filters(g, F, M)
        gy_np = (g.normal(size=(F, Ns - M + 1)) + 1j * g.normal(size=(F, Ns - M + 1))).astype(np.complex64)
        s, h, gy = (torch.from_numpy(a).cuda() for a in (s_np, h_np, gy_np))
        sp = parallel.SignalSplit(M, F, N)
        sp.set_filters(h)
        y = sp.convolve(s)
        ds, dh = sp.convolve_backward(s, gy)
        pw = (y.real ** 2 + y.imag ** 2).double().cpu().numpy()
        thr = float(np.quantile(pw, 0.95))
        cand = {m: getattr(sp, m)(s, thr, 1 << 14) for m in ("detect", "peaks")}
        torch.cuda.synchronize()
        sp.close()
        if rank == 0:
            import oracle as orc
            from paper_1910_01972_gb300 import decode_candidates
            p_ref = orc.power(s_np, h_np)
            band = 2e-5
            inf = float("inf")
            left = np.pad(p_ref[:, :-1], ((0, 0), (1, 0)), constant_values=-inf)
            right = np.pad(p_ref[:, 1:], ((0, 0), (0, 1)), constant_values=-inf)
            sets_ok = True
            for m, (must, may) in {
                    "detect": (p_ref >= thr * (1 + band), p_ref >= thr * (1 - band)),
                    "peaks": ((p_ref >= thr * (1 + band)) & (p_ref > left * (1 + band)) & (p_ref >= right * (1 + band)),
                              (p_ref >= thr * (1 - band)) & (p_ref >= left * (1 - band)) & (p_ref >= right * (1 - band)))
            }.items():
                rec, total = cand[m]
                f_, j_, _ = decode_candidates(rec, rec.shape[0])
                got = set(zip(f_.tolist(), j_.tolist()))
                must_s = set(zip(*[x.tolist() for x in np.nonzero(must)]))
                may_s = set(zip(*[x.tolist() for x in np.nonzero(may)]))
                sets_ok = sets_ok and total == len(got) == rec.shape[0] and must_s <= got <= may_s
        if rank == 0:
            y_ref = oracle.conv(s_np, h_np)
            ds_ref, dh_ref = oracle.adjoint(s_np, h_np, gy_np)
            q.put({"y_err": oracle.max_stream_rel_l2(y.cpu().numpy(), y_ref,
                                                     oracle.stream_scale(s_np, h_np, y_ref.shape[1])),
                   "ds_err": oracle.rel_l2(ds.cpu().numpy(), ds_ref),
                   "dh_err": oracle.max_stream_rel_l2(dh.cpu().numpy(), dh_ref),
                   "shapes": (tuple(y.shape), tuple(ds.shape), tuple(dh.shape)), "candidates": sets_ok})
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("Ns,M,F,N,world", [(50_000, 129, 5, 1024, 2), (50_000, 129, 3, 1024, 3),
                                            (300, 129, 2, 512, 3), (130, 129, 2, 256, 3)])
def test_signal_split_ranks_run_the_kernels(Ns, M, F, N, world):
    """The output-range split (parallel.SignalSplit): each rank convolves its
    input slice with the whole bank through the library's kernels; columns
    gathered, neighbouring slices' input gradients added, dh summed; threshold
    and peak candidates selected per range (peaks on a slice widened by one
    output each side) and gathered.  Ranges shorter than M-1 and an empty
    range (Nout = 2 over 3 ranks) included."""
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_signal_worker, args=(r, world, port, Ns, M, F, N, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
    for p in procs:
        assert p.exitcode == 0, "rank failed"
    r = q.get(timeout=5)
    assert r["shapes"] == ((F, Ns - M + 1), (Ns,), (F, M)), r
    assert r["y_err"] <= TOL and r["ds_err"] <= TOL_DS and r["dh_err"] <= TOL_DH, r
    assert r["candidates"], r            # threshold and peak candidates over the split = the oracle's rule
