"""Host-side marshalling rules of the Python binding (no GPU): lazy
conjugate / negative views are materialised for inputs and refused for
outputs."""
import pytest
import torch

import paper_1910_01972_gb300 as ols
from paper_1910_01972_gb300 import autograd


def test_conjugate_input_is_materialised():
    z = torch.tensor([1 + 2j, -3 + 0.5j, 4 - 1j], dtype=torch.complex64)
    v = z.conj()
    assert v.is_conj() and v.data_ptr() == z.data_ptr()
    m = ols._input(v, "s")
    assert not m.is_conj() and not m.is_neg()
    assert m.data_ptr() != z.data_ptr()
    assert torch.equal(m.view(torch.float32), torch.tensor([1, -2, -3, -0.5, 4, 1], dtype=torch.float32))


def test_negative_input_is_materialised():
    z = torch.tensor([1 + 2j, -3 + 0.5j], dtype=torch.complex64)
    v = z.conj().imag
    assert v.is_neg()
    m = ols._input(v, "s", dtype=torch.float32)
    assert not m.is_neg()
    assert torch.equal(m, torch.tensor([-2.0, -0.5]))


def test_plain_input_is_passed_through():
    z = torch.zeros(8, dtype=torch.complex64)
    assert ols._input(z, "s") is z


def test_outputs_reject_lazy_views():
    z = torch.zeros(4, dtype=torch.complex64)
    with pytest.raises(ValueError):
        ols._output(z.conj(), "out")
    with pytest.raises(ValueError):
        ols._output(z.conj().imag, "out", dtype=torch.float32)
    assert ols._output(z, "out") is z


def test_non_contiguous_and_wrong_dtype_are_refused():
    z = torch.zeros(8, dtype=torch.complex64)
    with pytest.raises(ValueError):
        ols._input(z[::2], "s")
    with pytest.raises(TypeError):
        ols._input(z.real, "s")
    with pytest.raises(TypeError):
        ols._input([1, 2], "s")


def test_autograd_values_resolves_views():
    z = torch.tensor([1 + 2j], dtype=torch.complex64)
    r = autograd._values(z.conj())
    assert not r.is_conj() and r.item() == 1 - 2j


@pytest.mark.parametrize("n", [0, 1, 3])
def test_decode_candidates_any_count(n):
    """Records laid out as ols_candidate (int64 j; int32 f; float power),
    decoded for every count, including one record (a [1] column whose torch
    stride stays 2) and counts above the capacity."""
    import numpy as np
    rec = np.zeros(4, dtype=[("j", "<i8"), ("f", "<i4"), ("power", "<f4")])
    rec["j"] = [10, 2**40, 7, 5]
    rec["f"] = [3, 0, 31, 2]
    rec["power"] = [1.5, 2.25, 1e30, 0.0]
    t = torch.from_numpy(rec.view(np.int64).reshape(4, 2).copy())
    f, j, p = ols.decode_candidates(t[:3], n)
    assert list(j) == list(rec["j"][:n]) and list(f) == list(rec["f"][:n]) and list(p) == list(rec["power"][:n])
    f, j, p = ols.decode_candidates(t[:2], 9)       # count above capacity: the stored records only
    assert list(j) == [10, 2**40] and list(f) == [3, 0]
