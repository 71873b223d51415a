"""The binding's buffer checks (paper_2607_16946_b300/_buffers.py), on the CPU:
a buffer the library would read or write past its end, or in the wrong
memory space, is refused before any call."""
import numpy as np
import pytest
import torch

from paper_2607_16946_b300 import _buffers as B


def test_host_output_checks():
    ok = np.empty(12, np.float32)
    assert B.host_f32(ok, 12, "out", writable=True) is ok
    with pytest.raises(ValueError, match="dtype"):
        B.host_f32(np.empty(12, np.float64), 12, "out")
    with pytest.raises(ValueError, match="12 floats"):
        B.host_f32(np.empty(11, np.float32), 12, "out")
    with pytest.raises(ValueError, match="contiguous"):
        B.host_f32(np.empty(24, np.float32)[::2], 12, "out")
    ro = np.empty(12, np.float32)
    ro.flags.writeable = False
    B.host_f32(ro, 12, "x")
    with pytest.raises(ValueError, match="writable"):
        B.host_f32(ro, 12, "out", writable=True)
    with pytest.raises(ValueError, match="numpy"):
        B.host_f32([0.0] * 12, 12, "out")


def test_device_output_refuses_host_and_wrong_types():
    with pytest.raises(ValueError, match="CUDA device"):
        B.device_f32(torch.empty(5), 5, "out")
    with pytest.raises(ValueError, match="CUDA float32 tensor"):
        B.device_f32(np.empty(5, np.float32), 5, "out")


def test_request_buffers():
    a = np.zeros((7, 3), np.float32)
    assert B.request_buffer(a, 21, "x") == (a.ctypes.data, True)
    t = torch.zeros(7, dtype=torch.float32)
    assert B.request_buffer(t, 7, "out", writable=True) == (t.data_ptr(), True)
    with pytest.raises(ValueError, match="dtype"):
        B.request_buffer(torch.zeros(7, dtype=torch.int32), 7, "out")      # same item size, not float32
    with pytest.raises(ValueError, match="dtype"):
        B.request_buffer(torch.zeros(7, dtype=torch.float64), 7, "out")
    with pytest.raises(ValueError, match="28 floats"):
        B.request_buffer(torch.zeros(7, dtype=torch.float32), 28, "out")   # a GRAD request needs 4q
    with pytest.raises(ValueError, match="contiguous"):
        B.request_buffer(torch.zeros((3, 7), dtype=torch.float32).t(), 21, "x")
    with pytest.raises(ValueError, match="tensor"):
        B.request_buffer(None, 7, "t")
