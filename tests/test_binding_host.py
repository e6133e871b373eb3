"""Argument marshalling of the Python binding (no GPU): every array handed to
the library is contiguous float32 with the element count the call reads or
writes, and host and device arrays are not mixed in one call; anything else
raises before the library sees a pointer."""
import numpy as np
import pytest

from paper_0712_2247_gb300 import lbif


class _FakeCudaTensor:
    is_cuda = True
    dtype = "torch.float32"

    def is_contiguous(self):
        return True

    def numel(self):
        return 4

    def data_ptr(self):
        return 0x1000


def test_pointer_checks_dtype_layout_and_size():
    with pytest.raises(TypeError):
        lbif._ptr(np.zeros(6, np.float64))
    with pytest.raises(TypeError):
        lbif._ptr(np.zeros((3, 4), np.float32).T)
    with pytest.raises(ValueError):
        lbif._ptr(np.zeros(5, np.float32), 6)
    a = np.zeros((2, 3), np.float32)
    assert lbif._ptr(a, 6) == a.ctypes.data
    assert lbif._ptr(None, 6) is None
    assert lbif._ptr(_FakeCudaTensor(), 4) == 0x1000
    with pytest.raises(ValueError):
        lbif._ptr(_FakeCudaTensor(), 5)


def test_torch_host_tensors():
    torch = pytest.importorskip("torch")
    t = torch.zeros(8)
    assert lbif._ptr(t, 8) == t.data_ptr()
    with pytest.raises(TypeError):
        lbif._ptr(torch.zeros(8, dtype=torch.float64))
    with pytest.raises(TypeError):
        lbif._ptr(torch.zeros(4, 4)[:, 1])


def test_host_and_device_not_mixed():
    host = np.zeros(4, np.float32)
    assert lbif._on_device(None, host) == 0
    assert lbif._on_device(_FakeCudaTensor(), None) == 1
    assert lbif._on_device() == 0
    with pytest.raises(ValueError):
        lbif._on_device(host, _FakeCudaTensor())
