"""GPU parity of sdf_query against the FP64 oracle, element by element.

Tolerance (FP32 path): |phi_gpu - phi_oracle| <= 1e-4 x AABB diagonal of the
cloud.  Cases span several tiles and query blocks with ragged tails, both
torus record forms, the split-N merge, FIXED lambda, offsets, host buffers,
degenerate inputs, and the full-size 256^3 grid workload on sampled outputs.
"""
import numpy as np
import pytest

import synth
from workloads import TOL_REL, aabb_diag, config1, config2_cloud, f32, mixed_cloud, GRID_RES

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


@pytest.fixture(scope="module")
def torch_mod():
    import torch
    return torch


def run(cloud, x, torch, **kw):
    xt = torch.as_tensor(np.asarray(x, np.float32), device="cuda")
    phi = cloud.query(xt, **kw)
    torch.cuda.synchronize()
    assert cloud.device_status() == 0
    return phi.cpu().numpy().astype(np.float64)


def test_config1_sphere_full(ptsdf, torch_mod, oracle_mod):
    """Plain method, small: N = 4,096 Fibonacci sphere, Q = 32,768 queries;
    against the oracle and the exact sphere SDF |x| - 1."""
    p, n, a, x = config1()
    cl = ptsdf.Cloud(p, n, a)
    info = cl.info()
    assert info["n"] == 4096 and info["n_kappa"] == 0
    got = run(cl, x, torch_mod)
    ref = oracle_mod.Cloud(p, n, a).phi(x)
    tol = TOL_REL * aabb_diag(p)
    err = np.abs(got - ref)
    assert err.max() <= tol, err.max()
    assert np.abs(got - (np.linalg.norm(x, axis=1) - 1)).max() <= tol


@pytest.mark.parametrize("q", [1, 511, 513, 1537])
@pytest.mark.parametrize("split", [0, 1, 3, 7])
def test_mixed_cloud_ragged(ptsdf, torch_mod, oracle_mod, q, split):
    """N = 1,000 mixed cloud (direct and kappa records, every sign case),
    ragged query counts around the 512-query block, explicit split factors."""
    p, n, a = mixed_cloud()
    cl = ptsdf.Cloud(p, n, a)
    info = cl.info()
    assert info["n_direct"] > 0 and info["n_kappa"] > 0
    x = f32(synth.uniform_queries(q, 500 + q, -1.5, 1.5))
    got = run(cl, x, torch_mod, split_n=split)
    ref = oracle_mod.Cloud(p, n, a).phi(x)
    assert np.abs(got - ref).max() <= TOL_REL * aabb_diag(p)


@pytest.mark.parametrize("split", [0, 1, 5])
def test_flat_kappa_tiles(ptsdf, torch_mod, oracle_mod, split):
    """Noisy superquadric, N = 2,000: most kappa-form records have
    kappa_min = 0 (whole tiles of them take the shorter formula), the rest
    are curved, and the tile at the boundary mixes the two."""
    p, n, a = f32(*synth.superquadric(2000, 5))
    cl = ptsdf.Cloud(p, n, a)
    info = cl.info()
    flat = info["n_kappa_flat"]
    assert 64 < flat < info["n_kappa"] and flat % 32 != 0
    x = f32(synth.uniform_queries(1537, 905, -1.3, 1.3))
    got = run(cl, x, torch_mod, split_n=split)
    ref = oracle_mod.Cloud(p, n, a).phi(x)
    assert np.abs(got - ref).max() <= TOL_REL * aabb_diag(p)


def test_split_factors_agree(ptsdf, torch_mod):
    """The merge of split chunks reproduces the unsplit sums (same shift)."""
    p, n, a = mixed_cloud(5)
    cl = ptsdf.Cloud(p, n, a)
    x = f32(synth.uniform_queries(3000, 6))
    base = run(cl, x, torch_mod, split_n=1)
    for s in (2, 5, 31):
        np.testing.assert_allclose(run(cl, x, torch_mod, split_n=s), base, atol=2e-6, rtol=0)


@pytest.mark.parametrize("C", [4.0, 64.0, 87.0])
def test_screening_constant(ptsdf, torch_mod, oracle_mod, C):
    p, n, a = f32(*synth.ring_torus(5000, 9, noise=0.005, jitter_deg=2.0))
    cl = ptsdf.Cloud(p, n, a)
    x = f32(synth.uniform_queries(2000, 10, -1.6, 1.6))
    got = run(cl, x, torch_mod, C=C)
    ref = oracle_mod.Cloud(p, n, a).phi(x, C=C)
    assert np.abs(got - ref).max() <= TOL_REL * aabb_diag(p)


def test_fixed_lambda_and_offset(ptsdf, torch_mod, oracle_mod):
    p, n, a = f32(*synth.ring_torus(3000, 11, noise=0.005, jitter_deg=2.0))
    cl = ptsdf.Cloud(p, n, a)
    x = f32(synth.uniform_queries(1500, 12, -1.6, 1.6))
    lam = 200.0
    got = run(cl, x, torch_mod, lambda_mode=ptsdf.SDF_LAMBDA_FIXED, fixed_lambda=lam, offset=0.1)
    ref = oracle_mod.Cloud(p, n, a).phi(x, mode=oracle_mod.FIXED, lam=lam) - 0.1
    assert np.abs(got - ref).max() <= TOL_REL * aabb_diag(p)


def test_degenerate_inputs(ptsdf, torch_mod, oracle_mod):
    """N = 1 (phi = g_1), a query exactly at the point (d_max = 0), Q = 0."""
    p, n, a = mixed_cloud(3)
    cl = ptsdf.Cloud(p[:1], n[:1], a[:1])
    x = f32(np.concatenate([synth.uniform_queries(40, 13), p[:1]]))
    got = run(cl, x, torch_mod)
    ref = oracle_mod.Cloud(p[:1], n[:1], a[:1]).phi(x)
    assert np.abs(got - ref).max() <= 1e-5
    import torch
    out = cl.query(torch.empty((0, 3), device="cuda"))
    assert out.shape == (0,)


def test_bad_build_input_rejected(ptsdf):
    p, n, a = mixed_cloud(4)
    n = n.copy()
    n[17] = 0.0
    with pytest.raises(ptsdf.SdfError) as ei:
        ptsdf.Cloud(p, n, a)
    assert ei.value.status == 1


def test_host_buffers_match_device(ptsdf, torch_mod):
    p, n, a = mixed_cloud(8)
    cl = ptsdf.Cloud(p, n, a)
    x = synth.uniform_queries(2500, 14).astype(np.float32)
    dev = run(cl, x, torch_mod)
    host = cl.query_host(x)
    np.testing.assert_array_equal(host.astype(np.float64), dev)


def test_config2_subset(ptsdf, torch_mod, oracle_mod):
    """Dense grid cloud (N = 100,000 noisy ring torus) on 65,536 seeded grid
    nodes, element by element."""
    p, n, a = config2_cloud()
    cl = ptsdf.Cloud(p, n, a)
    rng = np.random.Generator(np.random.PCG64(2))
    idx = rng.integers(0, GRID_RES ** 3, size=65_536)
    x = f32(synth.grid_query_index(idx, GRID_RES))
    got = run(cl, x, torch_mod)
    ref = oracle_mod.Cloud(p, n, a).phi(x)
    tol = TOL_REL * aabb_diag(p)
    err = np.abs(got - ref)
    assert err.max() <= tol, (err.max(), tol)


def test_config2_full_grid_sampled(ptsdf, torch_mod, oracle_mod):
    """Full size, in the benchmark's launch configuration: all 256^3 grid
    queries in one call; 512 sampled outputs checked against the oracle and
    every output finite."""
    import torch
    p, n, a = config2_cloud()
    cl = ptsdf.Cloud(p, n, a)
    g = torch.linspace(-1.6, 1.6, GRID_RES, device="cuda", dtype=torch.float64)
    zz, yy, xx = torch.meshgrid(g, g, g, indexing="ij")
    x = torch.stack([xx.reshape(-1), yy.reshape(-1), zz.reshape(-1)], 1).to(torch.float32).contiguous()
    phi = cl.query(x)
    torch.cuda.synchronize()
    assert cl.device_status() == 0
    phi = phi.cpu().numpy().astype(np.float64)
    assert np.isfinite(phi).all()
    rng = np.random.Generator(np.random.PCG64(3))
    idx = rng.integers(0, GRID_RES ** 3, size=512)
    ref = oracle_mod.Cloud(p, n, a).phi(f32(synth.grid_query_index(idx, GRID_RES)))
    assert np.abs(phi[idx] - ref).max() <= TOL_REL * aabb_diag(p)
