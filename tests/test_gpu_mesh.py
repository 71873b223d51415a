"""GPU parity of sdf_mesh_level_set (marching tetrahedra, offset surfaces of
Sec. 6) against the oracle's marching tetrahedra on the same phi grids:
identical vertex numbering and the same set of oriented triangles (exact),
vertex positions within FP32 interpolation error; and on the benchmark's
256^3 dense-grid phi, a closed, consistently oriented surface."""
import math

import numpy as np
import pytest

from oracle import mesh as omesh

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


def fields(nx, ny, nz, lo=(-1.5, -1.4, -1.3), hi=(1.5, 1.6, 1.2)):
    xs = [np.linspace(lo[a], hi[a], n) for a, n in enumerate((nx, ny, nz))]
    z, y, x = np.meshgrid(xs[2], xs[1], xs[0], indexing="ij")
    h = tuple((hi[a] - lo[a]) / (n - 1) for a, n in enumerate((nx, ny, nz)))
    sphere = np.sqrt(x * x + y * y + z * z) - 1.0
    torus = np.sqrt((np.sqrt(x * x + y * y) - 0.9) ** 2 + z * z) - 0.35
    two = np.minimum(np.sqrt((x - 0.7) ** 2 + y * y + z * z), np.sqrt((x + 0.7) ** 2 + y * y + z * z)) - 0.5
    rng = np.random.Generator(np.random.PCG64(5))
    bumpy = sphere + 0.05 * np.sin(7 * x) * np.cos(5 * y) + 0.002 * rng.standard_normal(x.shape)
    return {"sphere": sphere, "torus": torus, "two": two, "bumpy": bumpy}, lo, h


def gpu_mesh(ptsdf, phi32, lo, h, level):
    import torch
    v, t = ptsdf.mesh_level_set(torch.as_tensor(phi32, device="cuda"), lo, h, level)
    torch.cuda.synchronize()
    return v.cpu().numpy().astype(np.float64), t.cpu().numpy().astype(np.int64)


@pytest.mark.parametrize("name,level", [("sphere", 0.0), ("sphere", 0.3), ("torus", 0.0), ("two", -0.1),
                                        ("bumpy", 0.0)])
def test_matches_oracle(ptsdf, name, level):
    f, lo, h = fields(29, 23, 31)
    phi32 = f[name].astype(np.float32)
    ov, ot = omesh.marching_tetrahedra(phi32.astype(np.float64), lo, h, np.float32(level))
    gv, gt = gpu_mesh(ptsdf, phi32, lo, h, level)
    assert len(gv) == len(ov) and len(gt) == len(ot)
    np.testing.assert_array_equal(omesh.canonical_triangles(gt), omesh.canonical_triangles(ot))
    assert np.abs(gv - ov).max() <= 1e-5 * max(h)


def test_counts_and_buffers(ptsdf):
    import ctypes
    import torch
    from paper_2607_16946_b300 import _abi
    f, lo, h = fields(17, 17, 17)
    phi = torch.as_tensor(f["sphere"].astype(np.float32), device="cuda")
    L = ptsdf.lib()
    o = (ctypes.c_float * 3)(*lo)
    hh = (ctypes.c_float * 3)(*h)
    nv, nt = ctypes.c_int64(), ctypes.c_int64()
    assert L.sdf_mesh_level_set(ctypes.c_void_p(phi.data_ptr()), 17, 17, 17, o, hh, 0.0, None, 0, None, 0,
                                ctypes.byref(nv), ctypes.byref(nt), None) == 0
    assert nv.value > 0 and nt.value > 0
    v = torch.empty((nv.value, 3), device="cuda")
    t = torch.empty((nt.value - 1, 3), device="cuda", dtype=torch.int32)
    assert L.sdf_mesh_level_set(ctypes.c_void_p(phi.data_ptr()), 17, 17, 17, o, hh, 0.0,
                                ctypes.c_void_p(v.data_ptr()), nv.value, ctypes.c_void_p(t.data_ptr()),
                                nt.value - 1, ctypes.byref(nv), ctypes.byref(nt), None) == _abi.SDF_EINVAL
    assert L.sdf_mesh_level_set(ctypes.c_void_p(phi.data_ptr()), 1, 17, 17, o, hh, 0.0, None, 0, None, 0,
                                ctypes.byref(nv), ctypes.byref(nt), None) == _abi.SDF_EINVAL


def test_dense_grid_surface_closed(ptsdf):
    """The dense-grid workload's phi (N = 100,000 noisy ring torus, 256^3
    grid over [-1.6, 1.6]^3): its zero level is closed and consistently
    oriented, and encloses a volume near the ring torus's 2 pi^2 R r^2."""
    import torch
    import synth
    p, n, a = synth.ring_torus(100_000, 1002, R=1.0, r=0.35, noise=0.005, jitter_deg=2.0)
    cl = ptsdf.Cloud(p, n, a)
    g = torch.linspace(-1.6, 1.6, 256, device="cuda", dtype=torch.float64)
    zz, yy, xx = torch.meshgrid(g, g, g, indexing="ij")
    x = torch.stack([xx.reshape(-1), yy.reshape(-1), zz.reshape(-1)], 1).to(torch.float32).contiguous()
    phi = cl.query(x).reshape(256, 256, 256)
    h = 3.2 / 255
    v, t = ptsdf.mesh_level_set(phi, (-1.6, -1.6, -1.6), (h, h, h))
    torch.cuda.synchronize()
    v = v.cpu().numpy().astype(np.float64)
    t = t.cpu().numpy().astype(np.int64)
    _, counts, has_rev = omesh.directed_edge_counts(t)
    assert (counts == 1).all() and has_rev.all()
    vol = omesh.enclosed_volume(v, t)
    ref = 2 * math.pi ** 2 * 1.0 * 0.35 ** 2
    assert abs(vol - ref) < 0.02 * ref, (vol, ref)
