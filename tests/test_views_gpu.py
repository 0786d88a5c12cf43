"""The binding hands the kernels the values a tensor stands for.

A lazy conjugate view (``t.conj()``) or negative view (``t.conj().imag``)
shares its base's memory and only carries a flag, so passing its data
pointer would convolve the base.  Inputs given as such views must give the
oracle's result on the conjugated / negated values; caller-supplied outputs
must not be such views.  Also: autograd calls in flight on two streams (or
two threads) with different filter banks must not share filter state.
"""
import threading

import numpy as np
import pytest
import torch

import oracle
import synth
from paper_1910_01972_gb300 import Plan, _native, ols_conv
from paper_1910_01972_gb300 import build as _build

pytestmark = pytest.mark.gpu
TOL = 2e-6
TOL_DS = 2e-6
TOL_DH = 1e-5


@pytest.fixture(scope="module", autouse=True)
def built():
    _build.build()
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def draw(seed, Ns, F, M):
    g = np.random.Generator(np.random.PCG64(seed))
    return synth.signal(g, Ns), synth.filters(g, F, M)


def test_conjugate_signal_and_filters():
    s, h = draw(11, 30_000, 4, 65)
    plan = Plan(65, 4, 512)
    plan.set_filters(dev(h).conj())
    sv = dev(s).conj()
    assert sv.is_conj()
    y = plan.convolve(sv).cpu().numpy()
    ref = oracle.conv(np.conj(s), np.conj(h))
    assert oracle.max_stream_rel_l2(y, ref) <= TOL
    # the view itself is left as it was
    assert sv.is_conj()
    plan.close()


def test_negative_view_signal_real():
    g = np.random.Generator(np.random.PCG64(12))
    z = (g.uniform(-1, 1, 20_000) + 1j * g.uniform(-1, 1, 20_000)).astype(np.complex64)
    h = g.normal(size=(3, 33)).astype(np.float32)
    plan = Plan(33, 3, 256, flags=_native.OLS_FLAG_R2R)
    plan.set_filters_real(dev(h))
    x = dev(z).conj().imag          # -Im z, held as a negative view
    assert x.is_neg()
    y = plan.convolve_real(x).cpu().numpy()
    ref = oracle.conv_real(-z.imag.astype(np.float32), h)
    assert oracle.max_stream_rel_l2(y, ref) <= TOL
    plan.close()


def test_conjugate_output_view_is_rejected():
    s, h = draw(13, 5_000, 2, 17)
    plan = Plan(17, 2, 256)
    plan.set_filters(dev(h))
    out = torch.empty((2, 5_000 - 16), dtype=torch.complex64, device="cuda").conj()
    with pytest.raises(ValueError):
        plan.convolve(dev(s), out=out)
    plan.close()


def test_autograd_through_conjugate_views():
    """L = Re sum conj(y) c: the gradient reaching y is c, delivered by
    autograd as a conjugate view; s and h enter as conjugate views too."""
    s_np, h_np = draw(14, 25_000, 3, 129)
    g = np.random.Generator(np.random.PCG64(15))
    Nout = 25_000 - 128
    c_np = (g.normal(size=(3, Nout)) + 1j * g.normal(size=(3, Nout))).astype(np.complex64)
    sb = dev(s_np).requires_grad_(True)
    hb = dev(h_np).requires_grad_(True)
    y = ols_conv(sb.conj(), hb.conj(), N=1024)
    loss = (y.conj() * dev(c_np)).real.sum()
    loss.backward()
    # y = conv(conj s, conj h); d loss / d conj(s) = adjoint at g = c
    ds_ref, dh_ref = oracle.adjoint(np.conj(s_np), np.conj(h_np), c_np)
    y_ref = oracle.conv(np.conj(s_np), np.conj(h_np))
    assert oracle.max_stream_rel_l2(y.detach().cpu().numpy(), y_ref) <= TOL
    # the leaves are s and h: their gradients are the conjugates
    assert oracle.rel_l2(sb.grad.cpu().numpy(), np.conj(ds_ref)) <= TOL_DS
    assert oracle.max_stream_rel_l2(hb.grad.cpu().numpy(), np.conj(dh_ref)) <= TOL_DH


def _bank(seed, F, M):
    g = np.random.Generator(np.random.PCG64(seed))
    return synth.filters(g, F, M)


def test_two_streams_two_banks_in_flight():
    """Alternating calls with two different banks on two streams, no
    synchronisation until the end: each result matches its own bank."""
    s, _ = draw(16, 200_000, 1, 2)
    banks = [_bank(17, 8, 129), _bank(18, 8, 129)]
    sd = dev(s)
    hd = [dev(b) for b in banks]
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    torch.cuda.synchronize()
    outs = []
    for it in range(6):
        k = it % 2
        with torch.cuda.stream(streams[k]):
            outs.append((k, ols_conv(sd, hd[k], N=1024)))
    torch.cuda.synchronize()
    refs = [oracle.conv(s, b) for b in banks]
    for k, y in outs:
        assert oracle.max_stream_rel_l2(y.cpu().numpy(), refs[k]) <= TOL


def test_two_threads_two_banks():
    s, _ = draw(19, 100_000, 1, 2)
    banks = [_bank(20, 4, 65), _bank(21, 4, 65)]
    sd = dev(s)
    hd = [dev(b) for b in banks]
    torch.cuda.synchronize()
    results = {0: [], 1: []}
    errors = []

    def run(k):
        try:
            st = torch.cuda.Stream()
            with torch.cuda.stream(st):
                for _ in range(5):
                    results[k].append(ols_conv(sd, hd[k], N=512))
            st.synchronize()
        except Exception as e:  # reported below
            errors.append(e)

    th = [threading.Thread(target=run, args=(k,)) for k in (0, 1)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    assert not errors, errors
    torch.cuda.synchronize()
    for k in (0, 1):
        ref = oracle.conv(s, banks[k])
        for y in results[k]:
            assert oracle.max_stream_rel_l2(y.cpu().numpy(), ref) <= TOL
