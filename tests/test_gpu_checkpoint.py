"""Checkpoint of a built cloud (sdf_export / sdf_import): the imported cloud
answers every query bit for bit like the exported one (both engines, the
gradient, a weighted cloud, the log-sum-exp distance), the reported size
matches the layout, and short buffers are refused."""
import ctypes

import numpy as np
import pytest

import synth
from workloads import f32, mixed_cloud

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ptsdf():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2607_16946_b300 import build
    build.build()
    import paper_2607_16946_b300 as m
    return m


def answers(m, cl, x):
    import torch
    out = [cl.query(x, engine=m.SDF_ENGINE_TENSOR), cl.query(x, engine=m.SDF_ENGINE_ALU),
           cl.query(x, formula=m.SDF_FORMULA_LSE)]
    phi, g, _ = cl.query_grad(x)
    out += [phi, g.reshape(-1)]
    torch.cuda.synchronize()
    return [o.cpu().numpy() for o in out]


@pytest.mark.parametrize("weighted", [False, True])
def test_round_trip_is_bit_exact(ptsdf, weighted):
    import torch
    p, n, a = f32(*mixed_cloud(1500, 81))
    w = f32(np.exp(np.random.Generator(np.random.PCG64(82)).uniform(-1, 1, len(p)))) if weighted else None
    cl = ptsdf.Cloud(p, n, a, weights=w)
    data = cl.export()
    assert len(data) == 24 + len(p) * (12 + (1 if weighted else 0) + 16) * 4 + len(p)
    x = torch.as_tensor(f32(synth.uniform_queries(3000, 83, -1.3, 1.3)), dtype=torch.float32, device="cuda")
    ref = answers(ptsdf, cl, x)
    cl.close()
    back = ptsdf.Cloud.from_export(data)
    assert back.n == len(p) and back.weighted == weighted
    for got, want in zip(answers(ptsdf, back, x), ref):
        np.testing.assert_array_equal(got, want)
    assert back.export() == data                      # the records are fitted again identically


def test_short_buffers_refused(ptsdf):
    from paper_2607_16946_b300 import _abi
    p, n, a = f32(*synth.sphere_fibonacci(500, 84))
    cl = ptsdf.Cloud(p, n, a)
    L = _abi.lib()
    size = ctypes.c_int64()
    assert L.sdf_export(cl.handle, None, 0, ctypes.byref(size)) == _abi.SDF_OK
    buf = ctypes.create_string_buffer(size.value)
    assert L.sdf_export(cl.handle, buf, size.value - 1, ctypes.byref(size)) == _abi.SDF_EINVAL
    data = cl.export()
    h = ctypes.c_void_p()
    assert L.sdf_import(data[:-1], len(data) - 1, None, ctypes.byref(h)) == _abi.SDF_EINVAL
