"""Failure detection without a GPU fault.

* Host-side fault injection: OLS_FAIL_ALLOC=k makes the k-th device
  allocation of one ols_plan / ols_batch_plan / ols_convolve_host call fail;
  the call must return OLS_ERR_ALLOC, keep nothing allocated, and the
  library must work normally once the variable is cleared.
* A bounded device wait that runs out: OLS_TC_WAIT_NEVER=1 points the
  tensor-core kernel's in-loop mbarrier waits at a barrier nothing arrives on
  (a flag nothing sets) and OLS_TC_WAIT_LIMIT=4 keeps them short.  The kernel
  must record the failure in the plan's status word, drain the MMA it gave up
  on, release its tensor memory and return; the context stays usable and the
  next plan's results are correct.
"""
import ctypes
import os

import numpy as np
import pytest
import torch

import oracle
import synth
from paper_1910_01972_gb300 import Plan, _native
from paper_1910_01972_gb300 import build as _build

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    _build.build()
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")


@pytest.fixture
def env():
    saved = {k: os.environ.get(k) for k in ("OLS_FAIL_ALLOC", "OLS_TC_WAIT_LIMIT", "OLS_TC_WAIT_NEVER")}
    yield os.environ
    for k, v in saved.items():
        if v is None:
            os.environ.pop(k, None)
        else:
            os.environ[k] = v


def _free_bytes():
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


def test_plan_allocation_failure_at_every_step(env):
    torch.cuda.init()
    lib = _native.lib()
    base = _free_bytes()
    failed = 0
    for k in range(1, 12):
        env["OLS_FAIL_ALLOC"] = str(k)
        h = ctypes.c_void_p()
        rc = lib.ols_plan(ctypes.byref(h), 1024, 129, 8, _native.OLS_FLAG_FP32)
        if rc == _native.OLS_OK:        # k past the plan's allocations: nothing injected
            lib.ols_plan_destroy(h)
            break
        assert rc == _native.OLS_ERR_ALLOC, (k, _native.ols_status_string(rc))
        assert not h.value
        failed += 1
    assert failed >= 5                 # spectra, adjoint spectra, twiddles, FP64 table, order, status
    env.pop("OLS_FAIL_ALLOC")
    # nothing of the failed plans stays allocated (device pages are 2 MB granular)
    assert abs(_free_bytes() - base) < (8 << 20)
    s, h = synth.signal(np.random.Generator(np.random.PCG64(1)), 5000), \
        synth.filters(np.random.Generator(np.random.PCG64(2)), 8, 129)
    plan = Plan(129, 8, 1024)
    plan.set_filters(torch.from_numpy(h).cuda())
    y = plan.convolve(torch.from_numpy(s).cuda()).cpu().numpy()
    assert oracle.max_stream_rel_l2(y, oracle.conv(s, h)) <= 2e-6
    plan.close()


def _batch_until_success(env, make, limit=400):
    """Fail allocation k = 1, 2, ... of one batch-plan call until it succeeds;
    every failed call must report OLS_ERR_ALLOC.  Returns the failures seen."""
    lib = _native.lib()
    for k in range(1, limit):
        env["OLS_FAIL_ALLOC"] = str(k)
        b = ctypes.c_void_p()
        rc = make(lib, b)
        if rc == _native.OLS_OK:
            env.pop("OLS_FAIL_ALLOC")
            assert lib.ols_batch_destroy(b) == _native.OLS_OK
            return k - 1
        assert rc == _native.OLS_ERR_ALLOC, (k, _native.ols_status_string(rc))
        assert not b.value
    raise AssertionError("no success within %d allocations" % limit)


def test_batch_plan_allocation_failure(env):
    """Every allocation of a batch plan, including those of the autotuners'
    timing runs (segment length, tile schedule), fails cleanly."""
    Ns = (ctypes.c_int64 * 3)(20_000, 30_000, 9_000)
    M = (ctypes.c_int32 * 3)(33, 65, 129)
    F = (ctypes.c_int32 * 3)(4, 2, 3)
    N = (ctypes.c_int64 * 3)(512, 1024, 1024)
    one = (ctypes.c_int32 * 3)(1, 1, 1)
    base = _free_bytes()
    # given N and tiles: 6 allocations per FP32 plan, then 3 batch tables
    n = _batch_until_success(env, lambda lib, b: lib.ols_batch_plan_tiles(ctypes.byref(b), 3, Ns, M, F, N, one, 0))
    assert n == 3 * 6 + 3
    # tuned tile schedule (shapes no other test tunes): the tuner's timing runs allocate too
    Mt = (ctypes.c_int32 * 3)(35, 67, 131)
    Ft = (ctypes.c_int32 * 3)(5, 3, 7)
    n = _batch_until_success(env, lambda lib, b: lib.ols_batch_plan(ctypes.byref(b), 3, Ns, Mt, Ft, N, 0))
    assert n > 3 * 6 + 3
    # tuned segment length (an (M, F) no other test tunes): its timing runs too
    Ns1 = (ctypes.c_int64 * 1)(40_000)
    M1 = (ctypes.c_int32 * 1)(77)
    F1 = (ctypes.c_int32 * 1)(3)
    n = _batch_until_success(env, lambda lib, b: lib.ols_batch_plan(ctypes.byref(b), 1, Ns1, M1, F1, None, 0))
    assert n > 6 + 3
    assert abs(_free_bytes() - base) < (8 << 20)


def test_host_pipeline_allocation_failure(env):
    g = np.random.Generator(np.random.PCG64(3))
    s, h = synth.signal(g, 40_000), synth.filters(g, 4, 65)
    plan = Plan(65, 4, 512)
    plan.set_filters(torch.from_numpy(h).cuda())
    sh = torch.from_numpy(s).pin_memory()
    plan.host_timing(True)
    env["OLS_FAIL_ALLOC"] = "2"          # the first chunk's output staging buffer
    with pytest.raises(_native.OLSError) as ei:
        plan.convolve_host(sh)
    assert ei.value.status == _native.OLS_ERR_ALLOC
    # a failed call leaves no stage times behind
    assert _native.ols_host_stage_ms(plan.handle)[0] == _native.OLS_ERR_NOT_READY
    env.pop("OLS_FAIL_ALLOC")
    y = plan.convolve_host(sh).numpy()
    assert oracle.max_stream_rel_l2(y, oracle.conv(s, h)) <= 2e-6
    assert plan.host_stage_ms()["chunks"] == plan.last_launch_count() >= 1
    plan.close()


@pytest.mark.parametrize("flag", [_native.OLS_FLAG_TC_FP16SPLIT, _native.OLS_FLAG_TC_BF16SPLIT])
def test_tensor_core_wait_runs_out(env, flag):
    g = np.random.Generator(np.random.PCG64(4))
    s, h = synth.signal(g, 60_000), synth.filters(g, 4, 200)
    sd, hd = torch.from_numpy(s).cuda(), torch.from_numpy(h).cuda()
    env["OLS_TC_WAIT_LIMIT"] = "4"
    env["OLS_TC_WAIT_NEVER"] = "1"
    plan = Plan(200, 4, 4096, flags=flag)
    env.pop("OLS_TC_WAIT_LIMIT")
    env.pop("OLS_TC_WAIT_NEVER")
    plan.set_filters(hd)
    plan.convolve(sd)
    torch.cuda.synchronize()             # the kernel returned: no hang, no fault
    assert plan.status() != 0
    assert plan.status() == 0            # read-and-reset
    plan.close()
    # the context is intact: a plan with the default limit gives correct results
    plan = Plan(200, 4, 4096, flags=flag)
    plan.set_filters(hd)
    y = plan.convolve(sd).cpu().numpy()
    assert plan.status() == 0
    tol = 2e-6 if flag == _native.OLS_FLAG_TC_FP16SPLIT else 3e-5
    assert oracle.max_stream_rel_l2(y, oracle.conv(s, h)) <= tol
    plan.close()
