"""GPU parity of the two convolutional baselines (Sec. 5, "Signed distance
accuracy"; opts.formula = SDF_FORMULA_SSPD / SDF_FORMULA_SHC) against the
FP64 oracle, element by element, at the FP32 bar 1e-4 x AABB diagonal.

- phi_SSPD (Eq. SmoothedSignedPlanarDistance): mixed cloud with and without
  weights, ragged Q, explicit point splits, GLOBAL and FIXED lambda, offset;
  the dense-grid cloud on 16,384 seeded grid nodes; the full 256^3 grid in
  one call (the benchmark's launch configuration) sampled at 512 nodes.
- phi_SHC (Eq. ScreenedWindingNumber): the same cases on the queries whose
  double-layer sum is not a cancellation (the oracle's condition number
  sum |terms| / |w| <= 1e3: near w = 0 the sign flips and |phi_SHC| diverges,
  so FP32 and FP64 need not agree there; at most 5% of the queries are left
  out); the planar grid whose exact answer is the signed height; the sign on
  a closed sphere cloud.
- Degenerate cases and the options they refuse.
"""
import numpy as np
import pytest

import synth
from workloads import GRID_RES, TOL_REL, aabb_diag, config2_cloud, f32, mixed_cloud

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


def run(cloud, x, **kw):
    import torch
    out = cloud.query(torch.as_tensor(np.asarray(x, np.float32), device="cuda"), **kw)
    torch.cuda.synchronize()
    assert cloud.device_status() == 0
    return out.cpu().numpy().astype(np.float64)


def weights_for(n, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    return f32(np.exp(rng.uniform(np.log(0.1), np.log(10.0), size=n)))


def check_shc(got, ref, cond, tol, max_left_out=0.05):
    ok = cond <= 1e3
    assert ok.mean() >= 1 - max_left_out, ok.mean()
    err = np.abs(got - ref)[ok]
    assert np.isfinite(got[ok]).all()
    assert err.max() <= tol, (err.max(), tol)


@pytest.mark.parametrize("weighted", [False, True])
@pytest.mark.parametrize("split", [0, 3])
@pytest.mark.parametrize("q", [1, 511, 1537])
def test_mixed_cloud(ptsdf, oracle_mod, weighted, split, q):
    p, n, a = mixed_cloud(91)
    w = weights_for(len(p), 92) if weighted else None
    cl = ptsdf.Cloud(p, n, a, weights=w)
    orc = oracle_mod.Cloud(p, n, a, weights=w)
    x = f32(synth.uniform_queries(q, 93 + q, -1.5, 1.5))
    tol = TOL_REL * aabb_diag(p)
    for kw, okw in (({}, {}), ({"lambda_mode": ptsdf.SDF_LAMBDA_FIXED, "fixed_lambda": 40.0},
                                {"mode": oracle_mod.FIXED, "lam": 40.0})):
        got = run(cl, x, formula=ptsdf.SDF_FORMULA_SSPD, split_n=split, offset=0.03, **kw)
        assert np.abs(got - (orc.sspd(x, **okw) - 0.03)).max() <= tol
        got = run(cl, x, formula=ptsdf.SDF_FORMULA_SHC, split_n=split, **kw)
        ref, cond = orc.shc(x, cond=True, **okw)
        check_shc(got, ref, cond, tol, max_left_out=0.05 if q > 100 else 1.0)


def test_dense_grid_cloud(ptsdf, oracle_mod):
    """The dense-grid cloud (N = 100,000 noisy ring torus) on 16,384 seeded
    nodes of its 256^3 grid."""
    p, n, a = config2_cloud()
    cl = ptsdf.Cloud(p, n, a)
    idx = np.random.Generator(np.random.PCG64(94)).integers(0, GRID_RES ** 3, size=16_384)
    x = f32(synth.grid_query_index(idx, GRID_RES))
    orc = oracle_mod.Cloud(p, n, a)
    tol = TOL_REL * aabb_diag(p)
    assert np.abs(run(cl, x, formula=ptsdf.SDF_FORMULA_SSPD) - orc.sspd(x)).max() <= tol
    ref, cond = orc.shc(x, cond=True)
    check_shc(run(cl, x, formula=ptsdf.SDF_FORMULA_SHC), ref, cond, tol)


def test_dense_grid_full_size_sampled(ptsdf, oracle_mod):
    """All 256^3 grid queries in one call each (the benchmark's launch
    configuration); 512 sampled outputs against the oracle, every output of
    SSPD finite."""
    import torch
    p, n, a = config2_cloud()
    cl = ptsdf.Cloud(p, n, a)
    g = torch.linspace(-1.6, 1.6, GRID_RES, device="cuda", dtype=torch.float64)
    zz, yy, xx = torch.meshgrid(g, g, g, indexing="ij")
    x = torch.stack([xx.reshape(-1), yy.reshape(-1), zz.reshape(-1)], 1).to(torch.float32).contiguous()
    idx = np.random.Generator(np.random.PCG64(95)).integers(0, GRID_RES ** 3, size=512)
    xs = f32(synth.grid_query_index(idx, GRID_RES))
    orc = oracle_mod.Cloud(p, n, a)
    tol = TOL_REL * aabb_diag(p)
    out = cl.query(x, formula=ptsdf.SDF_FORMULA_SSPD)
    torch.cuda.synchronize()
    assert cl.device_status() == 0 and bool(torch.isfinite(out).all())
    assert np.abs(out.cpu().numpy()[idx].astype(np.float64) - orc.sspd(xs)).max() <= tol
    out = cl.query(x, formula=ptsdf.SDF_FORMULA_SHC)
    torch.cuda.synchronize()
    ref, cond = orc.shc(xs, cond=True)
    check_shc(out.cpu().numpy()[idx].astype(np.float64), ref, cond, tol)


def test_shc_plane_grid_is_signed_height(ptsdf, oracle_mod):
    """A planar grid with area weights s^2 (the double-layer integral over a
    plane is sign(h) exp(-lambda |h|)): phi_SHC is the signed height h, on the
    GPU as in the oracle."""
    s = 0.01
    g = np.arange(-1 + s / 2, 1, s)
    X, Y = np.meshgrid(g, g)
    P = np.stack([X.ravel(), Y.ravel(), np.zeros(X.size)], 1)
    N = np.tile([0.0, 0.0, 1.0], (P.shape[0], 1))
    cl = ptsdf.Cloud(P, N, np.zeros((P.shape[0], 6)), weights=np.full(P.shape[0], s * s))
    rng = np.random.Generator(np.random.PCG64(96))
    h = rng.uniform(0.02, 0.3, size=200) * rng.choice([-1.0, 1.0], size=200)
    x = f32(np.stack([rng.uniform(-0.3, 0.3, 200), rng.uniform(-0.3, 0.3, 200), h], 1))
    got = run(cl, x, formula=ptsdf.SDF_FORMULA_SHC)
    assert np.abs(got - x[:, 2]).max() <= TOL_REL * aabb_diag(P)
    sspd = run(cl, x, formula=ptsdf.SDF_FORMULA_SSPD)
    assert np.abs(sspd - x[:, 2]).max() <= 1e-6


def test_shc_sign_on_sphere_cloud(ptsdf):
    p, n, a = f32(*synth.sphere_fibonacci(4096, 97))
    cl = ptsdf.Cloud(p, n, a, weights=np.full(4096, 4 * np.pi / 4096))
    x = f32(synth.uniform_queries(5000, 98, -1.5, 1.5))
    r = np.linalg.norm(x, axis=1)
    x, r = x[np.abs(r - 1) > 0.05], r[np.abs(r - 1) > 0.05]
    got = run(cl, x, formula=ptsdf.SDF_FORMULA_SHC)
    assert np.all(np.sign(got) == np.sign(r - 1))
    sspd = run(cl, x, formula=ptsdf.SDF_FORMULA_SSPD)
    assert np.all(np.sign(sspd) == np.sign(r - 1))


def test_degenerate_cases(ptsdf, oracle_mod):
    p, n, a = mixed_cloud(99)
    one = ptsdf.Cloud(p[:1], n[:1], a[:1])
    # a one-point cloud at its point: lambda = 0, phi_SHC = 0; phi_SSPD = 0
    assert run(one, p[:1], formula=ptsdf.SDF_FORMULA_SHC)[0] == 0.0
    assert run(one, p[:1], formula=ptsdf.SDF_FORMULA_SSPD)[0] == 0.0
    # queries exactly at points of a larger cloud: those points add nothing to w
    cl = ptsdf.Cloud(p, n, a)
    orc = oracle_mod.Cloud(p, n, a)
    xs = p[::37]
    ref, cond = orc.shc(xs, cond=True)
    check_shc(run(cl, xs, formula=ptsdf.SDF_FORMULA_SHC), ref, cond, TOL_REL * aabb_diag(p), max_left_out=0.2)
    assert np.abs(run(cl, xs, formula=ptsdf.SDF_FORMULA_SSPD) - orc.sspd(xs)).max() <= TOL_REL * aabb_diag(p)
    import torch
    assert cl.query(torch.empty((0, 3), device="cuda"), formula=ptsdf.SDF_FORMULA_SHC).shape == (0,)


def test_refused_options(ptsdf):
    import torch
    p, n, a = mixed_cloud(100)
    cl = ptsdf.Cloud(p, n, a)
    x = torch.zeros((8, 3), device="cuda")
    for f in (ptsdf.SDF_FORMULA_SSPD, ptsdf.SDF_FORMULA_SHC):
        for kw in ({"engine": ptsdf.SDF_ENGINE_TENSOR}, {"precision": 1},
                   {"lambda_mode": ptsdf.SDF_LAMBDA_RADIUS, "fixed_lambda": 10.0}):
            with pytest.raises(ptsdf.SdfError):
                cl.query(x, formula=f, **kw)
        with pytest.raises(ptsdf.SdfError):
            cl.query_grad(x, formula=f)
    with pytest.raises(ptsdf.SdfError):
        cl.query(x, formula=ptsdf.SDF_FORMULA_SHC, lambda_mode=ptsdf.SDF_LAMBDA_FIXED, fixed_lambda=0.0)
