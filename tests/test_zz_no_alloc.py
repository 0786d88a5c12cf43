"""The allocation-free adjoint entry point (ols_convolve_backward_noalloc).

Callers such as real-time pipelines that forbid device allocation once they
run, or hosts that own every device allocation, cannot hand the adjoint a
workspace; this entry point uses scratch built into the library instead.
It must give the results of the workspace entry point, call after call: the
shared scratch keeps the previous call's contents, which must not leak into
the next result.  The adjoint is deterministic, so the two entry points must
agree bit for bit; before the compared calls the scratch is filled with NaN
by a call whose output gradient is all NaN.  Collected last on purpose, and
self-contained so it also passes alone in a fresh process.
"""
import numpy as np
import pytest
import torch

import synth
from paper_1910_01972_gb300 import Plan, _native
from paper_1910_01972_gb300 import build as _build

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    _build.build()
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")


def _noalloc(plan, s, Ns, gy, ds, dh):
    st = torch.cuda.current_stream().cuda_stream
    return _native.ols_convolve_backward_noalloc(plan.handle, s.data_ptr() if s is not None else None, Ns,
                                                 gy.data_ptr(), ds.data_ptr() if ds is not None else None,
                                                 dh.data_ptr() if dh is not None else None, st)


def test_noalloc_adjoint_matches_workspace_adjoint_twice():
    M, F, N, Ns = 129, 16, 1024, 300_000
    g = np.random.Generator(np.random.PCG64(2024))
    plan = Plan(M, F, N)
    assert plan.backward_workspace(Ns) <= _native.OLS_NOALLOC_SCRATCH_BYTES
    s = torch.from_numpy(synth.signal(g, Ns)).cuda()
    plan.set_filters(torch.from_numpy(synth.filters(g, F, M)).cuda())
    # fill the scratch with NaN: every edge and per-CTA spectrum of this size
    junk = torch.full((F, Ns - M + 1), float("nan"), dtype=torch.complex64, device="cuda")
    ds0 = torch.empty(Ns, dtype=torch.complex64, device="cuda")
    dh0 = torch.empty((F, M), dtype=torch.complex64, device="cuda")
    assert _noalloc(plan, s, Ns, junk, ds0, dh0) == _native.OLS_OK
    torch.cuda.synchronize()
    assert torch.isnan(torch.view_as_real(dh0)).all()
    for call in range(2):
        s = torch.from_numpy(synth.signal(g, Ns)).cuda()
        h = torch.from_numpy(synth.filters(g, F, M)).cuda()
        gy = torch.from_numpy((g.normal(size=(F, Ns - M + 1)) + 1j * g.normal(size=(F, Ns - M + 1)))
                              .astype(np.complex64)).cuda()
        plan.set_filters(h)
        ds_ref, dh_ref = plan.convolve_backward(s, gy)
        ds = torch.full((Ns,), float("nan"), dtype=torch.complex64, device="cuda")
        dh = torch.full((F, M), float("nan"), dtype=torch.complex64, device="cuda")
        rc = _noalloc(plan, s, Ns, gy, ds, dh)
        assert rc == _native.OLS_OK, _native.ols_status_string(rc)
        torch.cuda.synchronize()
        assert torch.equal(ds, ds_ref), call
        assert torch.equal(dh, dh_ref), call
        # ds only, then dh only, through the same shared scratch
        ds2 = torch.empty_like(ds)
        assert _noalloc(plan, s, Ns, gy, ds2, None) == _native.OLS_OK
        dh2 = torch.empty_like(dh)
        assert _noalloc(plan, s, Ns, gy, None, dh2) == _native.OLS_OK
        torch.cuda.synchronize()
        assert torch.equal(ds2, ds_ref) and torch.equal(dh2, dh_ref), call
    plan.close()


def test_noalloc_rejects_problems_beyond_the_scratch():
    M, F, N = 257, 8, 512
    plan = Plan(M, F, N)
    plan.set_filters(torch.zeros((F, M), dtype=torch.complex64, device="cuda"))
    Ns = 1 << 26                         # edges alone: ~2 * (Ns / 256) * 256 * 8 B > 32 MiB
    assert plan.backward_workspace(Ns) > _native.OLS_NOALLOC_SCRATCH_BYTES
    dummy = torch.zeros(16, dtype=torch.complex64, device="cuda")
    rc = _noalloc(plan, dummy, Ns, dummy, dummy, dummy)
    assert rc == _native.OLS_ERR_TOO_LARGE
    assert "scratch" in _native.ols_status_string(rc)
    plan.close()


def test_noalloc_reports_the_workspace_entry_points_errors_first():
    """The argument checks of ols_convolve_backward come before the size
    limit: a plan without filters, or a tensor-core plan, gets the same error
    from both entry points even for a problem beyond the scratch."""
    M, F, N, Ns = 257, 8, 512, 1 << 26
    dummy = torch.zeros(16, dtype=torch.complex64, device="cuda")
    plan = Plan(M, F, N)                 # filters never set
    assert _noalloc(plan, dummy, Ns, dummy, dummy, dummy) == _native.OLS_ERR_NOT_READY
    plan.close()
    plan = Plan(M, F, N, flags=_native.OLS_FLAG_TC_FP16SPLIT)
    plan.set_filters(torch.zeros((F, M), dtype=torch.complex64, device="cuda"))
    assert _noalloc(plan, dummy, Ns, dummy, dummy, dummy) == _native.OLS_ERR_UNSUPPORTED
    plan.close()
    plan = Plan(M, F, N)
    plan.set_filters(torch.zeros((F, M), dtype=torch.complex64, device="cuda"))
    raw = torch.zeros(64, dtype=torch.uint8, device="cuda")
    st = torch.cuda.current_stream().cuda_stream
    rc = _native.ols_convolve_backward_noalloc(plan.handle, dummy.data_ptr(), Ns, raw.data_ptr() + 4,
                                               dummy.data_ptr(), None, st)
    assert rc == _native.OLS_ERR_INVALID   # misaligned gradient pointer
    plan.close()
