"""sdf_query_noalloc: the query entry point for callers that may not allocate
device memory while they run (per-frame or per-cycle loops where the CUDA
allocator can block or synchronise, and services that reserve all their
device memory up front).  Its scratch is a fixed array inside the library.

Checked through the C ABI against sdf_query on the same inputs, for two calls
in a row (the second call reuses the array the first one left behind), and
its size limit must be refused with a clear error.  This file is collected
last so that a failure here does not hide the results of the other tests.
"""
import ctypes

import numpy as np
import pytest

import synth
from workloads import TOL_REL, aabb_diag, f32, mixed_cloud

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2607_16946_b300 import build
    build.build()
    import paper_2607_16946_b300 as m
    from paper_2607_16946_b300 import _abi
    return m, _abi, torch


def _call(L, fn, cloud, x, out, opts, stream):
    return fn(cloud.handle, ctypes.c_void_p(x.data_ptr()), x.shape[0], ctypes.c_void_p(out.data_ptr()),
              ctypes.byref(opts), stream)


@pytest.mark.parametrize("q", [2000, 70_000])
def test_noalloc_matches_query_twice(env, q):
    m, abi, torch = env
    L = abi.lib()
    p, n, a = mixed_cloud(31)
    cloud = m.Cloud(p, n, a)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    opts = abi.make_opts()
    tol = TOL_REL * aabb_diag(p)
    for call in range(2):
        x = torch.as_tensor(f32(synth.uniform_queries(q, 900 + 10 * q + call, -1.5, 1.5)),
                            dtype=torch.float32, device="cuda")
        ref = torch.empty(q, device="cuda")
        got = torch.full((q,), float("nan"), device="cuda")
        abi.check(_call(L, L.sdf_query, cloud, x, ref, opts, stream), "sdf_query")
        abi.check(_call(L, L.sdf_query_noalloc, cloud, x, got, opts, stream), "sdf_query_noalloc")
        torch.cuda.synchronize()
        assert cloud.device_status() == 0
        diff = (got - ref).abs().max().item()
        assert diff <= tol, (call, diff, tol)


@pytest.mark.parametrize("q,split,kw", [
    (70_000, 16, {}),          # 16 chunks do not fit: the split drops to 7
    (1_048_000, 4, {}),        # near the limit: the split drops to 1 (no partials)
    (3000, 0, {"formula": 1}),                                   # the log-sum-exp distance
    (3000, 3, {"formula": 1, "lambda_mode": 1, "fixed_lambda": 40.0}),
    (3000, 3, {"lambda_mode": 1, "fixed_lambda": 40.0, "offset": 0.05}),
])
def test_noalloc_split_reduction_and_formulas(env, q, split, kw):
    """The chunk-count reduction that keeps the partials inside the fixed
    array, and the other formulas and lambda modes, against sdf_query on the
    same inputs, twice in a row."""
    m, abi, torch = env
    L = abi.lib()
    p, n, a = mixed_cloud(33)
    cloud = m.Cloud(p, n, a)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    opts = abi.make_opts(split_n=split, **kw)
    tol = TOL_REL * aabb_diag(p)
    for call in range(2):
        x = torch.as_tensor(f32(synth.uniform_queries(q, 950 + call, -1.5, 1.5)), dtype=torch.float32,
                            device="cuda")
        ref = torch.empty(q, device="cuda")
        got = torch.full((q,), float("nan"), device="cuda")
        abi.check(_call(L, L.sdf_query, cloud, x, ref, opts, stream), "sdf_query")
        abi.check(_call(L, L.sdf_query_noalloc, cloud, x, got, opts, stream), "sdf_query_noalloc")
        torch.cuda.synchronize()
        assert cloud.device_status() == 0
        assert bool(torch.isfinite(got).all())
        diff = (got - ref).abs().max().item()
        assert diff <= tol, (q, split, kw, call, diff, tol)


def test_noalloc_rejects_oversized_batch(env):
    m, abi, torch = env
    L = abi.lib()
    p, n, a = mixed_cloud(32)
    cloud = m.Cloud(p, n, a)
    q = (8 << 20) // 8 + 1
    x = torch.zeros((q, 3), device="cuda")
    out = torch.empty(q, device="cuda")
    st = _call(L, L.sdf_query_noalloc, cloud, x, out, abi.make_opts(),
               ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == abi.SDF_EINVAL
    assert b"exceeds the maximum" in L.sdf_last_error()
