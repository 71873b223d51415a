"""Checks on the buffers the Python binding hands to the C ABI.

The library reads and writes exactly the number of floats each declaration in
ptsdf.h states, at the address it is given.  A buffer of the wrong dtype, size,
layout or memory space would be read or overwritten past its end, so it is
refused here, before the call, with a ValueError naming the argument.
"""
from __future__ import annotations

import numpy as np


def _is_tensor(a) -> bool:
    return type(a).__module__.startswith("torch") and hasattr(a, "data_ptr")


def device_f32(t, n_floats: int, name: str, device=None):
    """t must be a contiguous CUDA float32 tensor of n_floats elements (on
    `device` when given).  Returns t."""
    import torch
    if not _is_tensor(t):
        raise ValueError(f"{name}: expected a CUDA float32 tensor, got {type(t).__name__}")
    if t.device.type != "cuda":
        raise ValueError(f"{name}: must be on a CUDA device, not {t.device}")
    if device is not None and t.device != device:
        raise ValueError(f"{name}: on {t.device}, the other buffers on {device}")
    if t.dtype != torch.float32:
        raise ValueError(f"{name}: dtype must be float32, not {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name}: must be contiguous")
    if t.numel() != n_floats:
        raise ValueError(f"{name}: must hold {n_floats} floats, holds {t.numel()}")
    return t


def host_f32(a, n_floats: int, name: str, writable: bool = False):
    """a must be a C-contiguous float32 numpy array of n_floats elements
    (writable for an output).  Returns a."""
    if not isinstance(a, np.ndarray):
        raise ValueError(f"{name}: expected a float32 numpy array, got {type(a).__name__}")
    if a.dtype != np.float32:
        raise ValueError(f"{name}: dtype must be float32, not {a.dtype}")
    if not a.flags.c_contiguous:
        raise ValueError(f"{name}: must be C-contiguous")
    if writable and not a.flags.writeable:
        raise ValueError(f"{name}: must be writable")
    if a.size != n_floats:
        raise ValueError(f"{name}: must hold {n_floats} floats, holds {a.size}")
    return a


def request_buffer(a, n_floats: int, name: str, writable: bool = False):
    """A serving request's buffer: a float32 numpy array or CPU tensor (host)
    or a CUDA float32 tensor (device), contiguous, of n_floats elements.
    Returns (address, is_host)."""
    if isinstance(a, np.ndarray):
        host_f32(a, n_floats, name, writable)
        return a.ctypes.data, True
    if not _is_tensor(a):
        raise ValueError(f"{name}: expected a numpy array or a tensor, got {type(a).__name__}")
    import torch
    if a.dtype != torch.float32:
        raise ValueError(f"{name}: dtype must be float32, not {a.dtype}")
    if not a.is_contiguous():
        raise ValueError(f"{name}: must be contiguous")
    if a.numel() != n_floats:
        raise ValueError(f"{name}: must hold {n_floats} floats, holds {a.numel()}")
    return a.data_ptr(), a.device.type != "cuda"
