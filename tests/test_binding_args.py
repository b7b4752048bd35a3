"""Argument marshalling of the Python binding, without a GPU: field
buffers must be float64 (3, nz, ny, nx); inputs of another dtype or layout
are converted to a fresh contiguous copy, outputs are refused."""
import numpy as np
import pytest

from paper_1405_0942_gb300 import glemur as gl

SHAPE = (3, 4, 5, 6)


def test_contiguous_float64_array_is_passed_in_place():
    a = np.zeros(SHAPE)
    p, mem, keep = gl._field_ptr(a, SHAPE)
    assert mem == gl.MEM_HOST and p == a.ctypes.data and keep is a


def test_other_inputs_are_copied_to_contiguous_float64():
    a = np.arange(np.prod(SHAPE), dtype=np.float32).reshape(SHAPE)
    p, mem, keep = gl._field_ptr(a, SHAPE)
    assert keep.dtype == np.float64 and keep.flags.c_contiguous and keep.shape == SHAPE
    assert p == keep.ctypes.data and np.array_equal(keep, a.astype(np.float64))
    f = np.asfortranarray(np.random.default_rng(0).standard_normal(SHAPE))
    p, _, keep = gl._field_ptr(f, SHAPE)
    assert keep.flags.c_contiguous and np.array_equal(keep, f)


def test_outputs_must_already_fit():
    with pytest.raises(ValueError):
        gl._field_ptr(np.zeros(SHAPE, dtype=np.float32), SHAPE, writable=True)
    with pytest.raises(ValueError):
        gl._field_ptr(np.asfortranarray(np.zeros(SHAPE)), SHAPE, writable=True)


def test_torch_tensors_are_checked_not_copied():
    torch = pytest.importorskip("torch")
    t = torch.zeros(SHAPE, dtype=torch.float64)
    p, mem, keep = gl._field_ptr(t, SHAPE)
    assert mem == gl.MEM_HOST and p == t.data_ptr() and keep is t
    with pytest.raises(ValueError):
        gl._field_ptr(torch.zeros(SHAPE, dtype=torch.float32), SHAPE)
    with pytest.raises(ValueError):
        gl._field_ptr(torch.zeros((3, 4, 6, 5), dtype=torch.float64).transpose(2, 3), SHAPE)
