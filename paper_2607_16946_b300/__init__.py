"""ptsdf: pointwise signed distance to oriented point clouds ("points as tori")
on one NVIDIA B300.

The computation lives in libptsdf.so (CUDA, sm_103a) behind the C ABI of
include/ptsdf.h; this package marshals torch/numpy arrays into it.  PyTorch
supplies device memory and the current CUDA stream.

    cloud = Cloud(points, normals, params)        # N x 3, N x 3, N x 6
    phi = cloud.query(x)                           # x: Q x 3 (CUDA tensor) -> Q
    phi = cloud.query_host(x_numpy)                # host arrays in and out
    phi = sdf(x, cloud, params)                    # differentiable in x and params

Also on Cloud: query_grad, query_laplacian, backward_params, trace, export /
from_export (checkpoint),
project_level_set, knn_mean_distance / paper_lambda, info, device_status;
module functions combine, mesh_level_set and orient; serving in
paper_2607_16946_b300.serve.  Options (lambda mode, formula, precision,
engine, offset, ...) are keyword arguments mapped onto sdf_query_opts.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _abi, _buffers
from ._abi import (SDF_DIFFERENCE, SDF_ENGINE_ALU, SDF_ENGINE_AUTO, SDF_ENGINE_TENSOR, SDF_FORMULA_BLEND,
                   SDF_FORMULA_LSE, SDF_FORMULA_SHC, SDF_FORMULA_SSPD, SDF_INTERSECT, SDF_LAMBDA_FIXED,
                   SDF_LAMBDA_GLOBAL, SDF_LAMBDA_RADIUS, SDF_UNION, SdfError, check, lib, make_opts)

__all__ = ["Cloud", "SdfError", "SDF_LAMBDA_GLOBAL", "SDF_LAMBDA_FIXED", "SDF_LAMBDA_RADIUS", "SDF_UNION",
           "SDF_INTERSECT", "SDF_DIFFERENCE", "SDF_ENGINE_AUTO", "SDF_ENGINE_ALU", "SDF_ENGINE_TENSOR",
           "SDF_FORMULA_BLEND", "SDF_FORMULA_LSE", "SDF_FORMULA_SSPD", "SDF_FORMULA_SHC", "mesh_level_set",
           "orient", "make_opts", "lib", "sdf", "combine"]


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

    def __init__(self, points, normals, params, weights=None, stream=None):
        """weights: optional per-point weights A_i (N values in [2^-64, 2^64]),
        the area weights of the discretised surface integral; None = all 1."""
        lib()
        p, n, a = _dev_f32(points, 3), _dev_f32(normals, 3), _dev_f32(params, 6)
        if not (p.shape[0] == n.shape[0] == a.shape[0]):
            raise ValueError("points, normals and params must have the same length")
        w = None
        if weights is not None:
            w = _dev_f32(weights, 1).reshape(-1)
            if w.shape[0] != p.shape[0]:
                raise ValueError("weights must have one value per point")
        h = ctypes.c_void_p()
        check(lib().sdf_build_weighted(ctypes.c_void_p(p.data_ptr()), ctypes.c_void_p(n.data_ptr()),
                                       ctypes.c_void_p(a.data_ptr()),
                                       ctypes.c_void_p(w.data_ptr()) if w is not None else None, p.shape[0],
                                       _stream_ptr(stream), ctypes.byref(h)),
              "sdf_build")
        self._h = h
        self.n = int(p.shape[0])
        self.weighted = w is not None

    def export(self) -> bytes:
        """The cloud as a checkpoint (sdf_export): inputs and fitted records."""
        size = ctypes.c_int64()
        check(lib().sdf_export(self._h, None, 0, ctypes.byref(size)), "sdf_export")
        buf = ctypes.create_string_buffer(size.value)
        check(lib().sdf_export(self._h, buf, size.value, ctypes.byref(size)), "sdf_export")
        return buf.raw[: size.value]

    @classmethod
    def from_export(cls, data: bytes, stream=None) -> "Cloud":
        """A cloud rebuilt from Cloud.export() / sdf_export without fitting
        (sdf_import); its queries equal the exported cloud's bit for bit."""
        h = ctypes.c_void_p()
        buf = ctypes.create_string_buffer(bytes(data), len(data))
        check(lib().sdf_import(buf, len(data), _stream_ptr(stream), ctypes.byref(h)), "sdf_import")
        self = cls.__new__(cls)
        self._h = h
        n = ctypes.c_int64()
        check(lib().sdf_cloud_info(h, ctypes.byref(n), None, None, None))
        self.n = int(n.value)
        self.weighted = bool(int.from_bytes(bytes(data[12:16]), "little"))
        return self

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
        nf, ne = ctypes.c_int64(), ctypes.c_int64()
        check(lib().sdf_cloud_forms(self._h, ctypes.byref(nf), ctypes.byref(ne)))
        return {"n": n.value, "aabb_diag": diag.value, "n_direct": nd.value, "n_kappa": nk.value,
                "n_kappa_flat": nf.value, "exact_tiles": ne.value}

    def query(self, x, out=None, stream=None, **opts):
        """phi at the rows of x (Q x 3, CUDA float32) -> Q float32 CUDA tensor."""
        torch = _torch()
        x = _dev_f32(x, 3)
        q = x.shape[0]
        if out is None:
            out = torch.empty(q, device=x.device, dtype=torch.float32)
        else:
            _buffers.device_f32(out, q, "out", x.device)
        o = make_opts(**opts)
        check(lib().sdf_query(self._h, ctypes.c_void_p(x.data_ptr()), q, ctypes.c_void_p(out.data_ptr()),
                              ctypes.byref(o), _stream_ptr(stream)), "sdf_query")
        return out

    def query_laplacian(self, x, stream=None, **opts):
        """(phi, grad phi, lap phi) at the rows of x (sdf_query_laplacian, App. D)."""
        torch = _torch()
        x = _dev_f32(x, 3)
        q = x.shape[0]
        phi = torch.empty(q, device=x.device, dtype=torch.float32)
        grad = torch.empty((q, 3), device=x.device, dtype=torch.float32)
        lap = torch.empty(q, device=x.device, dtype=torch.float32)
        o = make_opts(**opts)
        check(lib().sdf_query_laplacian(self._h, ctypes.c_void_p(x.data_ptr()), q, ctypes.c_void_p(phi.data_ptr()),
                                        ctypes.c_void_p(grad.data_ptr()), ctypes.c_void_p(lap.data_ptr()),
                                        ctypes.byref(o), _stream_ptr(stream)), "sdf_query_laplacian")
        return phi, grad, lap

    def knn_mean_distance(self, k: int = 64, stream=None) -> float:
        """D of Sec. 4.2's lambda heuristic: the mean distance between a point and
        its k nearest other points, averaged over the cloud (sdf_knn_mean_distance)."""
        D = ctypes.c_double()
        check(lib().sdf_knn_mean_distance(self._h, int(k), ctypes.byref(D), _stream_ptr(stream)),
              "sdf_knn_mean_distance")
        return D.value

    def paper_lambda(self, stream=None) -> float:
        """The paper's constant lambda for the radius-limited evaluation, 10^3 / D
        with D = knn_mean_distance(64) (sdf_paper_lambda)."""
        lam = ctypes.c_double()
        check(lib().sdf_paper_lambda(self._h, ctypes.byref(lam), None, _stream_ptr(stream)), "sdf_paper_lambda")
        return lam.value

    def query_grad(self, x, stream=None, saved=True, **opts):
        """(phi, d phi / d x, saved statistics or None) at the rows of x.  With
        formula=SDF_FORMULA_LSE: (d~, grad d~, None)."""
        torch = _torch()
        saved = saved and opts.get("formula", SDF_FORMULA_BLEND) == SDF_FORMULA_BLEND
        x = _dev_f32(x, 3)
        q = x.shape[0]
        phi = torch.empty(q, device=x.device, dtype=torch.float32)
        grad = torch.empty((q, 3), device=x.device, dtype=torch.float32)
        sv = torch.empty((q, 8), device=x.device, dtype=torch.float32) if saved else None
        o = make_opts(**opts)
        check(lib().sdf_query_grad(self._h, ctypes.c_void_p(x.data_ptr()), q, ctypes.c_void_p(phi.data_ptr()),
                                   ctypes.c_void_p(grad.data_ptr()),
                                   ctypes.c_void_p(sv.data_ptr()) if saved else None,
                                   ctypes.byref(o), _stream_ptr(stream)), "sdf_query_grad")
        return phi, grad, sv

    def project_level_set(self, x0, level: float, max_iter: int = 10, tol: float = 0.0, stream=None, **opts):
        """Samples of the `level` set with normals (Sec. 6, morphological
        operations): each seed moved by Newton steps along grad phi
        (sdf_project_level_set).  Returns (x, normals, phi - level)."""
        torch = _torch()
        x0 = _dev_f32(x0, 3)
        q = x0.shape[0]
        x = torch.empty_like(x0)
        nrm = torch.empty_like(x0)
        res = torch.empty(q, device=x0.device, dtype=torch.float32)
        o = make_opts(**opts)
        check(lib().sdf_project_level_set(self._h, ctypes.c_void_p(x0.data_ptr()), q, float(level), int(max_iter),
                                          float(tol), ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(nrm.data_ptr()),
                                          ctypes.c_void_p(res.data_ptr()), ctypes.byref(o), _stream_ptr(stream)),
              "sdf_project_level_set")
        return x, nrm, res

    def backward_params(self, x, saved, grad_phi, stream=None, **opts):
        """d(sum_q grad_phi[q] phi(x_q)) / d params, N x 6 in the input point order."""
        torch = _torch()
        x = _dev_f32(x, 3)
        q = x.shape[0]
        _buffers.device_f32(saved, 8 * q, "saved", x.device)      # from query_grad at the same x
        gphi = _dev_f32(grad_phi).reshape(-1)
        if gphi.numel() != q:
            raise ValueError(f"grad_phi: must hold {q} floats, holds {gphi.numel()}")
        out = torch.empty((self.n, 6), device=x.device, dtype=torch.float32)
        o = make_opts(**opts)
        check(lib().sdf_backward_params(self._h, ctypes.c_void_p(x.data_ptr()), x.shape[0],
                                        ctypes.c_void_p(saved.data_ptr()), ctypes.c_void_p(gphi.data_ptr()),
                                        ctypes.c_void_p(out.data_ptr()), ctypes.byref(o), _stream_ptr(stream)),
              "sdf_backward_params")
        return out

    def trace(self, origins, dirs, max_steps: int = 48, eps: float = 1e-4, t_max: float = 6.0,
              normals: bool = True, stream=None, **opts):
        """Sphere tracing of phi = offset: (t_hit, steps, normals or None); t_hit = -1 for misses."""
        torch = _torch()
        org, d = _dev_f32(origins, 3), _dev_f32(dirs, 3)
        r = org.shape[0]
        t_hit = torch.empty(r, device=org.device, dtype=torch.float32)
        steps = torch.empty(r, device=org.device, dtype=torch.int32)
        nrm = torch.empty((r, 3), device=org.device, dtype=torch.float32) if normals else None
        o = make_opts(**opts)
        check(lib().sdf_trace(self._h, ctypes.c_void_p(org.data_ptr()), ctypes.c_void_p(d.data_ptr()), r,
                              int(max_steps), float(eps), float(t_max), ctypes.c_void_p(t_hit.data_ptr()),
                              ctypes.c_void_p(steps.data_ptr()),
                              ctypes.c_void_p(nrm.data_ptr()) if normals else None,
                              ctypes.byref(o), _stream_ptr(stream)), "sdf_trace")
        return t_hit, steps, nrm

    def query_host(self, x, out=None, stream=None, **opts):
        """phi with host (numpy) buffers; copies happen inside the library."""
        x = np.ascontiguousarray(x, dtype=np.float32).reshape(-1, 3)
        q = x.shape[0]
        if out is None:
            out = np.empty(q, dtype=np.float32)
        else:
            _buffers.host_f32(out, q, "out", writable=True)
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


def _autograd_function():
    torch = _torch()

    class SDFQuery(torch.autograd.Function):
        """phi(x) with hand-written backward kernels: d phi / d x from
        sdf_query_grad (computed in the forward, recomputing no pair terms
        later) and d phi / d params from sdf_backward_params."""

        @staticmethod
        def forward(ctx, x, params, cloud, opts):
            phi, grad, saved = cloud.query_grad(x.detach(), **opts)
            ctx.cloud, ctx.opts = cloud, opts
            ctx.save_for_backward(x.detach(), grad, saved)
            return phi

        @staticmethod
        def backward(ctx, gphi):
            x, grad, saved = ctx.saved_tensors
            gphi = gphi.contiguous().to(torch.float32)
            gx = gparams = None
            if ctx.needs_input_grad[0]:
                gx = (gphi[:, None] * grad).to(x.dtype)
            if ctx.needs_input_grad[1]:
                gparams = ctx.cloud.backward_params(x, saved, gphi, **ctx.opts)
            return gx, gparams, None, None

    return SDFQuery


_SDFQuery = None


def combine(op: int, a, b, out=None, stream=None):
    """Booleans of two phi arrays (CUDA tensors): SDF_UNION, SDF_INTERSECT, SDF_DIFFERENCE."""
    torch = _torch()
    a, b = _dev_f32(a).reshape(-1), _dev_f32(b).reshape(-1)
    if a.numel() != b.numel():
        raise ValueError(f"a and b must have the same length ({a.numel()} and {b.numel()})")
    if out is None:
        out = torch.empty_like(a)
    else:
        _buffers.device_f32(out, a.numel(), "out", a.device)
    check(lib().sdf_combine(int(op), ctypes.c_void_p(a.data_ptr()), ctypes.c_void_p(b.data_ptr()), a.shape[0],
                            ctypes.c_void_p(out.data_ptr()), _stream_ptr(stream)), "sdf_combine")
    return out


def sdf(x, cloud: Cloud, params=None, **opts):
    """Differentiable phi(x).  `params` is the N x 6 coefficient tensor the
    cloud was built from (pass it to receive d phi / d params)."""
    global _SDFQuery
    torch = _torch()
    if _SDFQuery is None:
        _SDFQuery = _autograd_function()
    if params is None:
        params = torch.zeros(0, device=x.device)
    return _SDFQuery.apply(x, params, cloud, opts)


def mesh_level_set(phi, origin, spacing, level: float = 0.0, stream=None):
    """The level-`level` surface of a phi grid (sdf_mesh_level_set): phi is a
    CUDA float32 tensor of shape (nz, ny, nx) (x fastest), node (i, j, k) at
    origin + (i, j, k) * spacing.  Returns (vertices V x 3 float32, triangles
    T x 3 int32) as CUDA tensors; normals point towards phi >= level."""
    torch = _torch()
    if phi.dim() != 3 or phi.dtype != torch.float32 or not phi.is_cuda:
        raise ValueError("phi must be a (nz, ny, nx) CUDA float32 tensor")
    phi = phi.contiguous()
    nz, ny, nx = phi.shape
    o = (ctypes.c_float * 3)(*[float(v) for v in origin])
    h = (ctypes.c_float * 3)(*[float(v) for v in spacing])
    nv, nt = ctypes.c_int64(), ctypes.c_int64()
    sp = _stream_ptr(stream)
    check(lib().sdf_mesh_level_set(ctypes.c_void_p(phi.data_ptr()), nx, ny, nz, o, h, float(level), None, 0, None, 0,
                                   ctypes.byref(nv), ctypes.byref(nt), sp), "sdf_mesh_level_set")
    verts = torch.empty((nv.value, 3), device=phi.device, dtype=torch.float32)
    tris = torch.empty((nt.value, 3), device=phi.device, dtype=torch.int32)
    if nt.value:
        check(lib().sdf_mesh_level_set(ctypes.c_void_p(phi.data_ptr()), nx, ny, nz, o, h, float(level),
                                       ctypes.c_void_p(verts.data_ptr()), nv.value, ctypes.c_void_p(tris.data_ptr()),
                                       nt.value, ctypes.byref(nv), ctypes.byref(nt), sp), "sdf_mesh_level_set")
    return verts, tris


def orient(points, normals, params, k: int = 16, max_iter: int = 10, stream=None, **opts):
    """Orientation repair (sdf_orient, Sec. 6) on copies of the inputs: returns
    (normals, params, flips per iteration) as CUDA tensors and a list."""
    torch = _torch()
    p = _dev_f32(points, 3)
    nrm = _dev_f32(normals, 3).clone()
    prm = torch.as_tensor(params, dtype=torch.float32, device=p.device).reshape(-1, 6).contiguous().clone()
    if nrm.shape[0] != p.shape[0] or prm.shape[0] != p.shape[0]:
        raise ValueError("points, normals and params must have the same length")
    flips = (ctypes.c_int32 * max_iter)()
    iters = ctypes.c_int32()
    o = make_opts(**opts)
    check(lib().sdf_orient(ctypes.c_void_p(p.data_ptr()), ctypes.c_void_p(nrm.data_ptr()),
                           ctypes.c_void_p(prm.data_ptr()), p.shape[0], int(k), int(max_iter), ctypes.byref(o), flips,
                           ctypes.byref(iters), _stream_ptr(stream)), "sdf_orient")
    return nrm, prm, [flips[i] for i in range(iters.value)]
