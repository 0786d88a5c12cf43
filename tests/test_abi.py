"""C ABI checks that need no GPU: the library loads, exports every symbol
include/*.h declares, and its host-side bookkeeping is exact."""
import ctypes
import glob
import os
import re

import numpy as np
import pytest

from paper_1910_01972_gb300 import _native
from paper_1910_01972_gb300 import build as _build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    _build.build()


def declared_functions():
    names = []
    for hdr in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(hdr).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"\b(ols_[a-z0-9_]+)\s*\(", text)
    return sorted(set(names))


def test_every_declared_symbol_is_exported_and_bound():
    names = declared_functions()
    assert "ols_convolve" in names and "ols_plan" in names
    lib = ctypes.CDLL(_native.LIB_PATH)
    for n in names:
        assert hasattr(lib, n), n
    bound = {s[0] for s in _native.SIGNATURES}
    assert set(names) == bound, set(names) ^ bound


def test_status_strings():
    for st in range(0, 9):
        assert _native.ols_status_string(st).startswith("OLS_")
    assert _native.ols_version() == 101


@pytest.mark.parametrize("N,M,Ns", [(512, 64, 65536), (2048, 257, 1 << 23), (1024, 129, 1 << 22),
                                    (4096, 512, 1 << 24), (256, 1, 1), (256, 256, 300), (8192, 1025, 9000)])
def test_geometry_is_exact(N, M, Ns):
    rc, L, nseg, Nout = _native.ols_geometry(N, M, Ns)
    assert rc == 0
    assert L == N - M + 1 and Nout == Ns - M + 1
    assert nseg == -(-Nout // L)
    # segments tile the outputs exactly once, each reading inside [0, Ns + N)
    covered = np.zeros(Nout, np.int32) if Nout < 10 ** 7 else None
    if covered is not None:
        for i in range(nseg):
            covered[i * L: min(i * L + L, Nout)] += 1
        assert np.all(covered == 1)
    assert (nseg - 1) * L < Nout <= nseg * L


def test_geometry_of_the_paper_configs():
    assert _native.ols_geometry(512, 64, 65536)[1:] == (449, 146, 65473)
    assert _native.ols_geometry(2048, 257, 1 << 23)[1:] == (1792, 4681, 8388352)
    assert _native.ols_geometry(1024, 129, 1 << 22)[1:] == (896, 4681, 4194176)
    assert _native.ols_geometry(4096, 512, 1 << 24)[1:] == (3585, 4680, 16776705)


@pytest.mark.parametrize("N,M,Ns,rc", [(512, 0, 100, 1), (512, 64, 63, 1), (500, 64, 1000, 2),
                                       (128, 64, 1000, 2), (16384, 64, 100000, 2), (512, 513, 1000, 2)])
def test_geometry_errors(N, M, Ns, rc):
    assert _native.ols_geometry(N, M, Ns)[0] == rc


@pytest.mark.parametrize("N", [256, 512, 1024, 2048, 4096, 8192])
def test_spectrum_order_is_a_permutation(N):
    rc, nu = _native.ols_spectrum_order(N)
    assert rc == 0
    assert sorted(nu) == list(range(N))
    assert nu[0] == 0


def test_spectrum_order_known_values():
    # N = 256 = 16 x 16: two radix-16 passes, position q = 16 a + b holds frequency a + 16 b.
    rc, nu = _native.ols_spectrum_order(256)
    assert all(nu[16 * a + b] == a + 16 * b for a in range(16) for b in range(16))
    # N = 512 = 16 x 16 x 2: q = 32 a + 2 b + c holds a + 16 b + 256 c.
    rc, nu = _native.ols_spectrum_order(512)
    assert all(nu[32 * a + 2 * b + c] == a + 16 * b + 256 * c
               for a in range(16) for b in range(16) for c in range(2))


def test_plan_rejects_bad_arguments_before_touching_cuda():
    assert _native.ols_plan(512, 0, 1)[0] == _native.OLS_ERR_INVALID
    assert _native.ols_plan(512, 4, 0)[0] == _native.OLS_ERR_INVALID
    assert _native.ols_plan(500, 4, 1)[0] == _native.OLS_ERR_UNSUPPORTED
    assert _native.ols_plan(512, 513, 1)[0] == _native.OLS_ERR_UNSUPPORTED
    assert _native.ols_plan(512, 4, 1, flags=99)[0] == _native.OLS_ERR_UNSUPPORTED
    rc, h = _native.ols_plan(512, 4, 1)
    if rc == 0:          # a GPU is present
        _native.ols_plan_destroy(h)
    else:
        assert rc == _native.OLS_ERR_CUDA


def test_null_handles_are_rejected():
    L = _native.lib()
    assert L.ols_convolve(None, None, 10, None, None) == _native.OLS_ERR_INVALID
    assert L.ols_set_filters(None, None, None) == _native.OLS_ERR_INVALID
    assert L.ols_plan_destroy(None) == 0
    assert L.ols_last_launch_count(None) == -1
    assert L.ols_host_timing(None, 1) == _native.OLS_ERR_INVALID
    assert _native.ols_host_stage_ms(None)[0] == _native.OLS_ERR_INVALID
    assert _native.ols_batch_status(None)[0] == _native.OLS_ERR_INVALID


def test_tile_schedule_model_rule_and_argument_checks():
    """ols_autotune_tiles with OLS_TUNE_MODEL is host arithmetic: the shortest
    power of two giving an item ~32 transforms per slot (F + 1 per segment),
    at most 8; invalid sizes are refused before any device call."""
    for F in (1, 2, 3, 7, 8, 15, 16, 31, 32, 128):
        rc, r = _native.ols_autotune_tiles(129, F, 1024, 256, _native.OLS_TUNE_MODEL)
        assert rc == _native.OLS_OK
        want = -(-32 // (F + 1))
        assert r in (1, 2, 4, 8) and (r >= want or r == 8) and (r == 1 or r // 2 < want), (F, r)
    U, I = _native.OLS_ERR_UNSUPPORTED, _native.OLS_ERR_INVALID
    assert _native.ols_autotune_tiles(129, 4, 1000, 256, _native.OLS_TUNE_MODEL)[0] == U    # N not a power of two
    assert _native.ols_autotune_tiles(2000, 4, 1024, 256, _native.OLS_TUNE_MODEL)[0] == U   # M > N
    assert _native.ols_autotune_tiles(129, 4, 8192, 256, _native.OLS_TUNE_MODEL)[0] == U    # block < N / 16
    assert _native.ols_autotune_tiles(129, 4, 1024, 384, _native.OLS_TUNE_MODEL)[0] == U    # block size
    assert _native.ols_autotune_tiles(0, 4, 1024, 256, _native.OLS_TUNE_MODEL)[0] == I
    assert _native.ols_autotune_tiles(129, 0, 1024, 256, _native.OLS_TUNE_MODEL)[0] == I
