"""The allocation-free adjoint entry point (ols_convolve_backward_noalloc).

Callers such as real-time pipelines that forbid device allocation once they
run, or hosts that own every device allocation, cannot hand the adjoint a
workspace; this entry point uses scratch built into the library instead.
It must give the results of the workspace entry point, call after call (the
shared scratch keeps the previous call's contents, which must not leak into
the next result).  Collected last on purpose, and self-contained so it also
passes alone in a fresh process.
"""
import numpy as np
import pytest
import torch

import synth
from paper_1910_01972_gb300 import Plan, _native
from paper_1910_01972_gb300 import build as _build

pytestmark = pytest.mark.gpu
TOL_DS = 2e-6   # the adjoint tolerances of tests/test_backward_gpu.py
TOL_DH = 1e-5


def _rel(a, b):
    return float(torch.linalg.vector_norm((a - b).flatten()) / torch.linalg.vector_norm(b.flatten()))


@pytest.fixture(scope="module", autouse=True)
def built():
    _build.build()
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")


def test_noalloc_adjoint_matches_workspace_adjoint_twice():
    M, F, N, Ns = 129, 16, 1024, 300_000
    g = np.random.Generator(np.random.PCG64(2024))
    plan = Plan(M, F, N)
    assert plan.backward_workspace(Ns) <= _native.OLS_NOALLOC_SCRATCH_BYTES
    st = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        s = torch.from_numpy(synth.signal(g, Ns)).cuda()
        h = torch.from_numpy(synth.filters(g, F, M)).cuda()
        gy = torch.from_numpy((g.normal(size=(F, Ns - M + 1)) + 1j * g.normal(size=(F, Ns - M + 1)))
                              .astype(np.complex64)).cuda()
        plan.set_filters(h)
        ds_ref, dh_ref = plan.convolve_backward(s, gy)
        ds = torch.full((Ns,), float("nan"), dtype=torch.complex64, device="cuda")
        dh = torch.full((F, M), float("nan"), dtype=torch.complex64, device="cuda")
        rc = _native.ols_convolve_backward_noalloc(plan.handle, s.data_ptr(), Ns, gy.data_ptr(),
                                                   ds.data_ptr(), dh.data_ptr(), st)
        assert rc == _native.OLS_OK, _native.ols_status_string(rc)
        torch.cuda.synchronize()
        assert _rel(ds, ds_ref) <= TOL_DS, (call, _rel(ds, ds_ref))
        assert _rel(dh, dh_ref) <= TOL_DH, (call, _rel(dh, dh_ref))
        # ds only, then dh only, through the same shared scratch
        ds2 = torch.empty_like(ds)
        assert _native.ols_convolve_backward_noalloc(plan.handle, s.data_ptr(), Ns, gy.data_ptr(),
                                                     ds2.data_ptr(), None, st) == _native.OLS_OK
        dh2 = torch.empty_like(dh)
        assert _native.ols_convolve_backward_noalloc(plan.handle, s.data_ptr(), Ns, gy.data_ptr(),
                                                     None, dh2.data_ptr(), st) == _native.OLS_OK
        torch.cuda.synchronize()
        assert _rel(ds2, ds_ref) <= TOL_DS and _rel(dh2, dh_ref) <= TOL_DH
    plan.close()


def test_noalloc_rejects_problems_beyond_the_scratch():
    M, F, N = 257, 8, 512
    plan = Plan(M, F, N)
    plan.set_filters(torch.zeros((F, M), dtype=torch.complex64, device="cuda"))
    Ns = 1 << 26                         # edges alone: ~2 * (Ns / 256) * 256 * 8 B > 32 MiB
    assert plan.backward_workspace(Ns) > _native.OLS_NOALLOC_SCRATCH_BYTES
    dummy = torch.zeros(16, dtype=torch.complex64, device="cuda")
    rc = _native.ols_convolve_backward_noalloc(plan.handle, dummy.data_ptr(), Ns, dummy.data_ptr(),
                                               dummy.data_ptr(), dummy.data_ptr(),
                                               torch.cuda.current_stream().cuda_stream)
    assert rc == _native.OLS_ERR_TOO_LARGE
    assert "scratch" in _native.ols_status_string(rc)
    plan.close()
