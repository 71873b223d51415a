"""ptsdf: pointwise signed distance to oriented point clouds ("points as tori")
on one NVIDIA B300.

The computation lives in libptsdf.so (CUDA, sm_103a) behind the C ABI of
include/ptsdf.h; this package marshals torch/numpy arrays into it.  PyTorch
supplies device memory and the current CUDA stream.

    cloud = Cloud(points, normals, params)        # N x 3, N x 3, N x 6
    phi = cloud.query(x)                           # x: Q x 3 (CUDA tensor) -> Q
    phi = cloud.query_host(x_numpy)                # host arrays in and out
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _abi
from ._abi import (SDF_LAMBDA_FIXED, SDF_LAMBDA_GLOBAL, SdfError, check, lib, make_opts)

__all__ = ["Cloud", "SdfError", "SDF_LAMBDA_GLOBAL", "SDF_LAMBDA_FIXED", "make_opts", "lib"]


def _torch():
    import torch
    return torch


def _stream_ptr(stream=None) -> ctypes.c_void_p:
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _dev_f32(a, cols=None):
    torch = _torch()
    t = torch.as_tensor(a)
    if t.device.type != "cuda":
        t = t.to(device="cuda")
    t = t.to(torch.float32).contiguous()
    if cols is not None:
        t = t.reshape(-1, cols)
    return t


class Cloud:
    """A point cloud with one fitted torus per point, resident on the GPU."""

    def __init__(self, points, normals, params, stream=None):
        lib()
        p, n, a = _dev_f32(points, 3), _dev_f32(normals, 3), _dev_f32(params, 6)
        if not (p.shape[0] == n.shape[0] == a.shape[0]):
            raise ValueError("points, normals and params must have the same length")
        h = ctypes.c_void_p()
        check(lib().sdf_build(ctypes.c_void_p(p.data_ptr()), ctypes.c_void_p(n.data_ptr()),
                              ctypes.c_void_p(a.data_ptr()), p.shape[0], _stream_ptr(stream), ctypes.byref(h)),
              "sdf_build")
        self._h = h
        self.n = int(p.shape[0])

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().sdf_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self) -> ctypes.c_void_p:
        return self._h

    def info(self) -> dict:
        n, nd, nk = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        diag = ctypes.c_float()
        check(lib().sdf_cloud_info(self._h, ctypes.byref(n), ctypes.byref(diag), ctypes.byref(nd), ctypes.byref(nk)))
        return {"n": n.value, "aabb_diag": diag.value, "n_direct": nd.value, "n_kappa": nk.value}

    def query(self, x, out=None, stream=None, **opts):
        """phi at the rows of x (Q x 3, CUDA float32) -> Q float32 CUDA tensor."""
        torch = _torch()
        x = _dev_f32(x, 3)
        q = x.shape[0]
        if out is None:
            out = torch.empty(q, device=x.device, dtype=torch.float32)
        o = make_opts(**opts)
        check(lib().sdf_query(self._h, ctypes.c_void_p(x.data_ptr()), q, ctypes.c_void_p(out.data_ptr()),
                              ctypes.byref(o), _stream_ptr(stream)), "sdf_query")
        return out

    def query_host(self, x, out=None, stream=None, **opts):
        """phi with host (numpy) buffers; copies happen inside the library."""
        x = np.ascontiguousarray(x, dtype=np.float32).reshape(-1, 3)
        q = x.shape[0]
        if out is None:
            out = np.empty(q, dtype=np.float32)
        o = make_opts(**opts)
        check(lib().sdf_query_host(self._h, x.ctypes.data_as(ctypes.c_void_p), q,
                                   out.ctypes.data_as(ctypes.c_void_p), ctypes.byref(o), _stream_ptr(stream)),
              "sdf_query_host")
        return out

    def device_status(self, stream=None) -> int:
        code = ctypes.c_int32()
        st = lib().sdf_device_status(self._h, _stream_ptr(stream), ctypes.byref(code))
        if st not in (_abi.SDF_OK, _abi.SDF_EDEVICE):
            check(st, "sdf_device_status")
        return code.value
