"""Maximum sizes: a signal of more than 2^31 samples (outputs past the 32-bit
index range) through the fused complex kernel and the real-to-real kernel,
checked at sampled outputs against the FP64 oracle (tolerance 2e-6 relative
L2, the FP32 bar).  The signal is drawn on the device (17 GB complex, 8.6 GB
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
