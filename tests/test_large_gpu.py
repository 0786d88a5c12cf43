"""Maximum sizes: a signal of more than 2^31 samples (outputs past the 32-bit
index range) through the fused complex kernel, the real-to-real kernel, the
post-processing kernels (power, derivative, threshold and peak candidates), the tensor-core kernel (FP32 and split-plane input)
and the adjoint, checked at sampled outputs against the FP64 oracle
(tolerance 2e-6 relative L2, the FP32 bar; the tensor-core form's FP16 bound
is the same).  The signal is drawn on the device (17 GB complex, 8.6 GB
real); each sampled output's M-sample input window is gathered and given to
the oracle."""
import numpy as np
import pytest
import torch

import oracle
import synth
from paper_1910_01972_gb300 import Plan, _native
from paper_1910_01972_gb300 import build as _build

pytestmark = pytest.mark.gpu
TOL = 2e-6
NS = (1 << 31) + 12345


@pytest.fixture(scope="module", autouse=True)
def built():
    _build.build()
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")


def _sample_outputs(Nout, L, seed):
    g = np.random.Generator(np.random.PCG64(seed))
    b31 = 1 << 31
    seg31 = (b31 // L) * L           # segment boundaries around 2^31
    j = np.concatenate([g.integers(0, Nout, 400),
                        [0, 1, Nout - 1, Nout - 2, b31 - 1, b31, b31 + 1, b31 - 64, seg31 - 1, seg31, seg31 + L - 1,
                         seg31 + L, (1 << 30) - 1, 1 << 30]])
    return np.unique(np.clip(j, 0, Nout - 1))


def _windows(s, j, M):
    idx = torch.from_numpy(j[:, None] + np.arange(M)[None, :]).cuda()
    return s[idx].cpu().numpy()                    # [len(j)][M] input windows


def test_complex_signal_beyond_2_to_31():
    M, F, N = 64, 1, 512
    g = np.random.Generator(np.random.PCG64(77))
    h = synth.filters(g, F, M)
    s = synth.device_signal(NS, seed=501)
    plan = Plan(M, F, N)
    plan.set_filters(torch.from_numpy(h).cuda())
    y = plan.convolve(s)
    torch.cuda.synchronize()
    q = plan.query(NS)
    Nout, L = q["Nout"], q["L"]
    assert Nout > (1 << 31)
    j = _sample_outputs(Nout, L, 5)
    got = y[0, torch.from_numpy(j).cuda()].cpu().numpy()
    win = _windows(s, j, M)
    ref = np.array([oracle.conv_at(win[i], h, [0], [0])[0] for i in range(len(j))])
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= TOL
    # nothing left unwritten at the very end of the output
    tail = y[0, Nout - 5000:]
    assert bool(torch.isfinite(torch.view_as_real(tail)).all())
    plan.close()
    del y, s
    torch.cuda.empty_cache()


def test_real_signal_beyond_2_to_31():
    M, F, N = 129, 2, 1024
    g = np.random.Generator(np.random.PCG64(78))
    h = synth.real_filters(g, F, M)
    s = synth.device_signal(NS, seed=502, real=True)
    plan = Plan(M, F, N, flags=_native.OLS_FLAG_R2R)
    plan.set_filters_real(torch.from_numpy(h).cuda())
    y = plan.convolve_real(s)
    torch.cuda.synchronize()
    q = plan.query(NS)
    Nout, L = q["Nout"], q["L"]
    j = _sample_outputs(Nout, L, 6)
    win = _windows(s, j, M)
    for f in range(F):
        got = y[f, torch.from_numpy(j).cuda()].cpu().numpy().astype(np.float64)
        ref = np.array([oracle.conv_real_at(win[i], h[f], [0], [0])[0] for i in range(len(j))])
        assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= TOL, f
    plan.close()
    del y, s
    torch.cuda.empty_cache()


def test_power_and_derivative_beyond_2_to_31():
    """The post-processing kernels at the same size: |y|^2 and the derivative
    (segments advancing by L-2 from an input offset of -1) past index 2^31."""
    M, F, N = 64, 1, 512
    g = np.random.Generator(np.random.PCG64(79))
    h = synth.filters(g, F, M)
    s = synth.device_signal(NS, seed=503)
    plan = Plan(M, F, N)
    plan.set_filters(torch.from_numpy(h).cuda())
    q = plan.query(NS)
    Nout, L = q["Nout"], q["L"]
    j = _sample_outputs(Nout, L, 7)
    jd = np.unique(np.clip(np.concatenate([j, _sample_outputs(Nout, L - 2, 8)]), 0, Nout - 1))
    jt = torch.from_numpy(j).cuda()
    p = plan.convolve_power(s)
    got_p = p[0, jt].cpu().numpy().astype(np.float64)
    del p
    win = _windows(s, j, M)
    ref_p = np.array([oracle.power_at(win[i], h, [0], [0])[0] for i in range(len(j))])
    assert np.linalg.norm(got_p - ref_p) / np.linalg.norm(ref_p) <= 4e-6
    d = plan.convolve_derivative(s)
    got_d = d[0, torch.from_numpy(jd).cuda()].cpu().numpy()
    del d
    # the oracle's derivative on each output's local window: inputs for outputs
    # j-1 .. j+1 (3 outputs, the middle one interior), or for the two outputs at
    # an end of the stream (where the one-sided rule applies)
    ref_d, ref_y = [], []
    for jj in jd:
        if jj == 0:
            w0, k = 0, 0
        elif jj == Nout - 1:
            w0, k = jj - 1, 1
        else:
            w0, k = jj - 1, 1
        n_loc = 2 if jj in (0, Nout - 1) else 3
        w = _windows(s, np.array([w0]), M - 1 + n_loc)[0]
        ref_d.append(oracle.derivative_at(w, h, [0], [k])[0])
        ref_y.append(oracle.conv_at(w, h, [0], [k])[0])
    ref_d, ref_y = np.array(ref_d), np.array(ref_y)
    assert np.linalg.norm(got_d - ref_d) / np.linalg.norm(ref_y) <= TOL
    plan.close()
    del s
    torch.cuda.empty_cache()


def test_tensor_core_split_beyond_2_to_31():
    """The FP16 split tensor-core kernel at the same size, from the FP32
    signal and from its split planes (equal bit for bit)."""
    M, F, N = 64, 1, 512
    g = np.random.Generator(np.random.PCG64(80))
    h = synth.filters(g, F, M)
    s = synth.device_signal(NS, seed=504)
    plan = Plan(M, F, N, flags=_native.OLS_FLAG_TC_FP16SPLIT)
    plan.set_filters(torch.from_numpy(h).cuda())
    y = plan.convolve(s)
    torch.cuda.synchronize()
    assert plan.status() == 0
    q = plan.query(NS)
    Nout, L = q["Nout"], q["L"]
    j = _sample_outputs(Nout, L, 9)
    got = y[0, torch.from_numpy(j).cuda()].cpu().numpy()
    win = _windows(s, j, M)
    ref = np.array([oracle.conv_at(win[i], h, [0], [0])[0] for i in range(len(j))])
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= TOL
    hi, lo = plan.split_signal(s)
    del s
    y2 = plan.convolve_split(hi, lo)
    torch.cuda.synchronize()
    assert plan.status() == 0
    assert torch.equal(y, y2)
    plan.close()
    del y, y2, hi, lo
    torch.cuda.empty_cache()


def test_adjoint_beyond_2_to_31():
    """The adjoint with an output gradient that is zero except at a few
    outputs, some past 2^31 and at segment boundaries there: ds near each
    nonzero gradient entry and dh (a sum over all 2^31 outputs) against the
    oracle's adjoint of local windows, one per cluster of entries (clusters
    are > 2M apart, so each local window sees all the entries that reach
    it)."""
    M, F, N = 64, 2, 512
    rng = np.random.Generator(np.random.PCG64(81))
    h = synth.filters(rng, F, M)
    s = synth.device_signal(NS, seed=505)
    plan = Plan(M, F, N)
    plan.set_filters(torch.from_numpy(h).cuda())
    q = plan.query(NS)
    Nout, L = q["Nout"], q["L"]
    b31 = 1 << 31
    seg31 = (b31 // L) * L
    support = [(0, 3), (1, 5000), (0, seg31 - 1), (1, seg31), (0, b31 - 1), (1, b31 + 700), (0, Nout - 1)]
    vals = (rng.normal(size=len(support)) + 1j * rng.normal(size=len(support))).astype(np.complex64)
    gy = torch.zeros((F, Nout), dtype=torch.complex64, device="cuda")
    for (f, j0), v in zip(support, vals):
        gy[f, j0] = complex(v)
    ds, dh = plan.convolve_backward(s, gy)
    torch.cuda.synchronize()
    del gy
    dh_ref = np.zeros((F, M), np.complex128)
    got, want = [], []
    # entries closer than 2M (the segment boundary pair) share one local window
    order = sorted(range(len(support)), key=lambda i: support[i][1])
    clusters = []
    for i in order:
        if clusters and support[i][1] - support[clusters[-1][-1]][1] <= 2 * M:
            clusters[-1].append(i)
        else:
            clusters.append([i])
    for cl in clusters:
        jmin, jmax = support[cl[0]][1], support[cl[-1]][1]
        a = max(0, jmin - (M - 1))
        nl = min(Nout, jmax + M) - a                   # local outputs [a, a + nl)
        s_loc = _windows(s, np.array([a]), nl + M - 1)[0]
        g_loc = np.zeros((F, nl), np.complex64)
        for i in cl:
            f, j0 = support[i]
            g_loc[f, j0 - a] = vals[i]
        ds_loc, dh_loc = oracle.adjoint(s_loc, h, g_loc)
        dh_ref += dh_loc
        # ds[m] for m in [jmin, jmax + M - 1] sees only this cluster's entries
        m = np.arange(jmin, min(jmax + M, NS))
        assert m.max() < NS and a + nl + M - 1 <= NS
        got.append(ds[torch.from_numpy(m).cuda()].cpu().numpy())
        want.append(ds_loc[m - a])
    got, want = np.concatenate(got), np.concatenate(want)
    assert np.linalg.norm(got - want) / np.linalg.norm(want) <= 2e-6
    far = np.array([1 << 30, (1 << 31) - (1 << 20), 70_000])  # no gradient within 2M of these
    assert far.max() < NS and all(abs(int(x) - j0) > 2 * M for x in far for _, j0 in support)
    assert np.all(ds[torch.from_numpy(far).cuda()].cpu().numpy() == 0)
    assert oracle.max_stream_rel_l2(dh.cpu().numpy(), dh_ref) <= 1e-5
    plan.close()
    del ds, s
    torch.cuda.empty_cache()


def test_detect_and_peaks_beyond_2_to_31():
    """Threshold and peak candidates past index 2^31.  Detection runs the power
    kernel's segments, so its candidates are exactly the (0, j) with p[j] >=
    threshold in the power kernel's output (same FP32 values); peaks run the
    derivative's L-2 segments and are bracketed by the peak rule on that
    power with a relative margin of 2e-5 on every comparison."""
    M, F, N = 64, 1, 512
    g = np.random.Generator(np.random.PCG64(80))
    h = synth.filters(g, F, M)
    s = synth.device_signal(NS, seed=504)
    plan = Plan(M, F, N)
    plan.set_filters(torch.from_numpy(h).cuda())
    p = plan.convolve_power(s)[0]
    thr = float(torch.quantile(p[:: 1 << 10].float(), 0.9999).item())
    above = p >= thr
    n_above = int(above.sum().item())
    cap = n_above + 1024
    rec, cnt = plan.convolve_detect(s, thr, cap)
    torch.cuda.synchronize()
    assert int(cnt.item()) == n_above
    j = rec[:n_above, 0]
    seen = torch.zeros_like(above)
    seen[j] = True
    assert int(seen.sum().item()) == n_above and torch.equal(seen, above)   # masks: no index list of 2^31+
    assert int(j.max().item()) > (1 << 31)
    del above, seen
    band = 2e-5
    left = torch.cat([torch.full((1,), -float("inf"), device=p.device), p[:-1]])
    must = (p >= thr * (1 + band)) & (p > left * (1 + band))
    may = (p >= thr * (1 - band)) & (p >= left * (1 - band))
    del left
    right = torch.cat([p[1:], torch.full((1,), -float("inf"), device=p.device)])
    must &= p >= right * (1 + band)
    may &= p >= right * (1 - band)
    del right
    rec, cnt = plan.convolve_peaks(s, thr, cap)
    torch.cuda.synchronize()
    n = int(cnt.item())
    jp = rec[:n, 0]
    assert int(must.sum().item()) <= n <= int(may.sum().item())
    assert bool(may[jp].all())
    got = torch.zeros_like(must)
    got[jp] = True
    assert bool((got | ~must).all()) and int(got.sum().item()) == n
    assert int(jp.max().item()) > (1 << 31)
    plan.close()
    del s, p, must, may, got
    torch.cuda.empty_cache()
