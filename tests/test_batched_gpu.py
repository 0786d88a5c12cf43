"""The batched uneven form (one persistent launch for the whole batch, or one
per segment length; work tickets, autotuned segment lengths, CUDA-graph
capture) against the FP64 oracle and against per-problem plain calls."""
import numpy as np
import pytest
import torch

import oracle
import synth
from paper_1910_01972_gb300 import BatchPlan, Plan, autotune
from paper_1910_01972_gb300 import build as _build

pytestmark = pytest.mark.gpu
TOL = 2e-6


@pytest.fixture(scope="module", autouse=True)
def built():
    _build.build()
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


SMALL = dict(Ns=[1_000, 70_001, 300_000, 257, 45_000, 120_000, 9_999],
             M=[33, 129, 257, 257, 1025, 65, 513],
             F=[3, 8, 2, 1, 5, 11, 4],
             N=[256, 1024, 2048, 512, 4096, 256, 8192])


def small_inputs(seed=3):
    g = np.random.Generator(np.random.PCG64(seed))
    ss = [synth.signal(g, n) for n in SMALL["Ns"]]
    hs = [synth.filters(g, f, m) for f, m in zip(SMALL["F"], SMALL["M"])]
    return ss, hs


@pytest.mark.parametrize("per_n", [False, True])
def test_batched_matches_oracle_and_plain_calls(per_n):
    ss, hs = small_inputs()
    bp = BatchPlan(SMALL["Ns"], SMALL["M"], SMALL["F"], SMALL["N"], per_n=per_n)
    assert bp.N == SMALL["N"]
    bp.set_filters([dev(h) for h in hs])
    sd = [dev(s) for s in ss]
    ys = bp.convolve(sd)
    torch.cuda.synchronize()
    assert bp.last_launch_count() == (len(set(SMALL["N"])) if per_n else 1)
    assert bp.status() == 0                      # every problem's status word, read and reset
    for b in range(bp.B):
        y = ys[b].cpu().numpy()
        assert oracle.max_stream_rel_l2(y, oracle.conv(ss[b], hs[b])) <= TOL, b
        p = Plan(SMALL["M"][b], SMALL["F"][b], SMALL["N"][b])
        p.set_filters(dev(hs[b]))
        yp = p.convolve(sd[b]).cpu().numpy()
        # same segments, same arithmetic: identical (at N = 512, 1024 and 4096 the
        # plain kernel's last FFT exchange goes through TMEM, the batch's through
        # shared memory, so this also checks that exchange moves data exactly)
        assert np.array_equal(y, yp), b
        p.close()
    bp.close()


def test_autotuned_batch():
    ss, hs = small_inputs(4)
    bp = BatchPlan(SMALL["Ns"], SMALL["M"], SMALL["F"])
    for n, m in zip(bp.N, SMALL["M"]):
        assert n >= m and n & (n - 1) == 0 and 256 <= n <= 8192
    bp.set_filters([dev(h) for h in hs])
    ys = bp.convolve([dev(s) for s in ss])
    for b in range(bp.B):
        assert oracle.max_stream_rel_l2(ys[b].cpu().numpy(), oracle.conv(ss[b], hs[b])) <= TOL
    bp.close()


def test_autotune_is_cached_and_model_is_consistent():
    n1 = autotune(257, 32)
    n2 = autotune(257, 32)
    assert n1 == n2 and n1 >= 257
    nm = autotune(257, 32, model_only=True)
    assert nm >= 257 and nm & (nm - 1) == 0


@pytest.mark.parametrize("per_n", [False, True])
def test_graph_capture_and_replay_with_new_data(per_n):
    ss, hs = small_inputs(5)
    bp = BatchPlan(SMALL["Ns"], SMALL["M"], SMALL["F"], SMALL["N"], per_n=per_n)
    bp.set_filters([dev(h) for h in hs])
    sd = [dev(s) for s in ss]
    ys = bp.outputs()
    st, yt = bp.pointer_table(sd), bp.pointer_table(ys)
    torch.cuda.synchronize()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        bp.launch(st, yt)                        # warm-up outside the capture
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=side):
            bp.launch(st, yt)
    torch.cuda.current_stream().wait_stream(side)
    g = np.random.Generator(np.random.PCG64(77))
    new = [synth.signal(g, n) for n in SMALL["Ns"]]
    for s_dev, s_new in zip(sd, new):
        s_dev.copy_(dev(s_new))
    for y in ys:
        y.zero_()
    graph.replay()
    torch.cuda.synchronize()
    for b in range(bp.B):
        assert oracle.max_stream_rel_l2(ys[b].cpu().numpy(), oracle.conv(new[b], hs[b])) <= TOL
    bp.close()


@pytest.mark.parametrize("per_n", [False, True])
def test_full_size_uneven_batch_sampled(per_n):
    """64 signals, lengths log-uniform in [2^16, 2^22], F in {8..128},
    M in {33, ..., 1025}, autotuned N: sampled outputs of every problem
    against the oracle, and three problems against plain calls."""
    spec = synth.batch_spec()
    ss, hs = synth.batch_inputs(spec)
    bp = BatchPlan(spec.Ns, spec.M, spec.F, per_n=per_n)
    bp.set_filters([dev(h) for h in hs])
    sd = [dev(s) for s in ss]
    ys = bp.convolve(sd)
    torch.cuda.synchronize()
    g = np.random.Generator(np.random.PCG64(11))
    for b in range(bp.B):
        nout = bp.Nout[b]
        fi = g.integers(0, spec.F[b], 64)
        ji = np.concatenate([g.integers(0, nout, 60), [0, 1, nout - 2, nout - 1]])
        got = ys[b][torch.from_numpy(fi).cuda(), torch.from_numpy(ji).cuda()].cpu().numpy()
        ref = oracle.conv_at(ss[b], hs[b], fi, ji)
        assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= TOL, b
    for b in (0, 31, 63):
        p = Plan(spec.M[b], spec.F[b], bp.N[b])
        p.set_filters(dev(hs[b]))
        assert torch.equal(p.convolve(sd[b]), ys[b])
        p.close()
    bp.close()


def test_single_launch_block_sizes_cover_every_segment_length():
    """The single launch picks its block from the longest segment (N/16
    threads, at least 128): a batch with N <= 2048 runs 128-thread blocks, one
    with N = 4096 256-thread blocks, one with N = 8192 512-thread blocks (the
    test above).  Each is bitwise equal to per-problem calls."""
    g = np.random.Generator(np.random.PCG64(21))
    for Ns_, M_, F_, N_ in (([5_000, 40_000, 300, 77_777], [33, 200, 65, 129], [3, 2, 4, 5], [256, 512, 1024, 2048]),
                            ([50_000, 9_000, 60_001], [1000, 17, 300], [2, 6, 3], [4096, 256, 2048])):
        ss = [synth.signal(g, n) for n in Ns_]
        hs = [synth.filters(g, f, m) for f, m in zip(F_, M_)]
        bp = BatchPlan(Ns_, M_, F_, N_)
        bp.set_filters([dev(h) for h in hs])
        sd = [dev(s) for s in ss]
        ys = bp.convolve(sd)
        torch.cuda.synchronize()
        assert bp.last_launch_count() == 1
        for b in range(bp.B):
            p = Plan(M_[b], F_[b], N_[b])
            p.set_filters(dev(hs[b]))
            assert torch.equal(p.convolve(sd[b]), ys[b]), (N_, b)
            p.close()
            assert oracle.max_stream_rel_l2(ys[b].cpu().numpy(), oracle.conv(ss[b], hs[b])) <= TOL
        bp.close()


@pytest.mark.parametrize("tiles", [[1] * 7, [3, 1, 2, 8, 5, 4, 7], [8] * 7])
def test_tile_schedules_give_identical_results(tiles):
    """The single launch's items as runs of 1 to 8 tiles (every run length,
    ragged last runs): outputs bit for bit those of per-problem calls."""
    ss, hs = small_inputs(5)
    sd = [dev(s) for s in ss]
    bp = BatchPlan(SMALL["Ns"], SMALL["M"], SMALL["F"], SMALL["N"], tiles=tiles)
    assert bp.tiles == tiles
    bp.set_filters([dev(h) for h in hs])
    ys = bp.convolve(sd)
    torch.cuda.synchronize()
    block = max(128, max(SMALL["N"]) // 16)
    for b in range(bp.B):
        seg_per_tile = block * 16 // SMALL["N"][b]
        nseg = -(-(SMALL["Ns"][b] - SMALL["M"][b] + 1) // (SMALL["N"][b] - SMALL["M"][b] + 1))
        ntiles = -(-nseg // seg_per_tile)
        assert bp.items[b] == -(-ntiles // tiles[b])
        p = Plan(SMALL["M"][b], SMALL["F"][b], SMALL["N"][b])
        p.set_filters(dev(hs[b]))
        assert torch.equal(ys[b], p.convolve(sd[b])), b
        p.close()
    bp.close()


def test_tile_schedule_autotuned():
    """Tuned runs are powers of two up to 8, cached, and the tuned batch
    matches the oracle; the model choice follows its stated rule."""
    from paper_1910_01972_gb300 import _native
    for F in (1, 8, 40):
        rc, r = _native.ols_autotune_tiles(129, F, 1024, 256, 0)
        assert rc == _native.OLS_OK and r in (1, 2, 4, 8)
        rc2, r2 = _native.ols_autotune_tiles(129, F, 1024, 256, 0)
        assert rc2 == _native.OLS_OK and r2 == r
        rc, rm = _native.ols_autotune_tiles(129, F, 1024, 256, _native.OLS_TUNE_MODEL)
        want = max(1, -(-32 // (F + 1)))
        expect = 1
        while expect < want and expect < 8:
            expect *= 2
        assert rm == expect
    assert _native.ols_autotune_tiles(129, 4, 8192, 256, 0)[0] == _native.OLS_ERR_UNSUPPORTED   # block < N/16
    ss, hs = small_inputs(6)
    bp = BatchPlan(SMALL["Ns"], SMALL["M"], SMALL["F"], SMALL["N"])
    assert all(r in (1, 2, 4, 8) for r in bp.tiles)
    bp.set_filters([dev(h) for h in hs])
    ys = bp.convolve([dev(s) for s in ss])
    for b in range(bp.B):
        assert oracle.max_stream_rel_l2(ys[b].cpu().numpy(), oracle.conv(ss[b], hs[b])) <= TOL
    bp.close()
