"""The bounds-checked debug build (OLS_CHECK=1): the parity edge cases of the
forward, real-to-real, post-processing, tensor-core, adjoint and batched
kernels run in a child process on that build, every global access checked against its buffer; no check may fail
(the plan status words stay 0) and the results keep the parity bounds."""
import json
import os
import subprocess
import sys

import pytest
import torch

from paper_1910_01972_gb300 import build as _build

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    _build.build()
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")


def test_no_access_fails_its_bounds_check():
    lib = _build.build(extra=["-DOLS_CHECK=1"], out=os.path.join(_build.PKG, "libols_check.so"))
    env = dict(os.environ, OLS_LIBRARY=lib)
    r = subprocess.run([sys.executable, "-m", "tests.checked_cases"], cwd=ROOT, env=env, capture_output=True,
                       text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    res = json.loads(r.stdout.strip().splitlines()[-1])
    assert res["library"] == "libols_check.so"
    assert res["cases"] == 32
    assert res["status"] == 0, res                 # no failed bounds check, no expired wait
    w = res["worst"]
    print(json.dumps(res))
    assert w["fwd"] <= 2e-6 and w["tc"] <= 2e-6 and w["ds"] <= 2e-6 and w["dh"] <= 1e-5, w
    assert w["r2r"] <= 2e-6 and w["power"] <= 4e-6 and w["deriv"] <= 2e-6 and w["batch"] <= 2e-6, json.dumps(res)
    assert w["detect"] == 0.0 and w["peaks"] == 0.0, w
    assert res["tc_split_equal"]
