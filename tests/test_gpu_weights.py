"""GPU parity of per-point weights (sdf_build_weighted) and of the
log-sum-exp distance (opts.formula = SDF_FORMULA_LSE) against the FP64
oracle, element by element.

Weights A_i are the area weights of the discretised surface integral of Eq.
SelfNormalizedConvolutionalDistanceFormula; the log-sum-exp distance is Eq.
ConvolutionalDistanceFormula with h = 1.  Tolerances are the FP32 bars of
the unweighted tests: 1e-4 x AABB diagonal for phi and d~ (the packed-half
precisions: their own bounds), the gradient, Laplacian and parameter-gradient
bars of their own tests.

Cases: weights log-uniform in [0.1, 10] on the mixed cloud (both record
forms, ragged tiles) for the blend (FP32 and the packed-half weights), its
gradient, Laplacian, parameter gradient and the radius-limited sum; integer
weights against the unweighted cloud with repeated points (GPU against
GPU); d~ on the tensor engine, the FP32-unit engine, split point chunks,
FIXED and RADIUS lambda, weighted and not; option errors.
"""
import numpy as np
import pytest

import synth
from test_gpu_grad import check_close, kink_free
from test_gpu_precision import BOUNDS
from test_gpu_radius import check_against_oracle
from workloads import TOL_REL, aabb_diag, config2_cloud, f32, mixed_cloud

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


def weights_for(n, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    return f32(np.exp(rng.uniform(np.log(0.1), np.log(10.0), size=n)))


def run(cloud, x, **kw):
    import torch
    xt = torch.as_tensor(np.asarray(x, np.float32), device="cuda")
    out = cloud.query(xt, **kw)
    torch.cuda.synchronize()
    assert cloud.device_status() == 0
    return out.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("split", [0, 3])
def test_weighted_blend(ptsdf, oracle_mod, split):
    p, n, a = mixed_cloud(31)
    w = weights_for(len(p), 32)
    cl = ptsdf.Cloud(p, n, a, weights=w)
    assert cl.weighted and cl.info()["n_kappa"] > 0
    x = f32(synth.uniform_queries(1537, 33, -1.5, 1.5))
    got = run(cl, x, split_n=split)
    orc = oracle_mod.Cloud(p, n, a, weights=w)
    tol = TOL_REL * aabb_diag(p)
    assert np.abs(got - orc.phi(x)).max() <= tol
    # the weights matter: the unweighted blend differs by far more than the tolerance
    assert np.abs(got - oracle_mod.Cloud(p, n, a).phi(x)).max() > 10 * tol
    # both engines: the tensor cores take the direct tiles (weights in their B
    # tiles' constants), the FP32 units the curvature-form ones
    for engine in (1, 2):
        assert np.abs(run(cl, x, split_n=split, engine=engine) - orc.phi(x)).max() <= tol, engine
    fixed = run(cl, x, lambda_mode=ptsdf.SDF_LAMBDA_FIXED, fixed_lambda=40.0)
    assert np.abs(fixed - orc.phi(x, mode=oracle_mod.FIXED, lam=40.0)).max() <= tol
    # packed-half weights of the FP32-unit loop, within their own stated bounds
    for prec, name in ((1, "f16x2"), (2, "bf16x2")):
        half = run(cl, x, precision=prec)
        err = np.abs(half - orc.phi(x)).max() / aabb_diag(p)
        print("weighted mixed", name, err)
        assert err <= BOUNDS[(name, "mixed_weighted")], (name, err)


def test_weighted_direct_tiles_on_tensor_cores(ptsdf, oracle_mod):
    """A direct-form cloud (ring torus) with weights: all of it on the tensor
    cores, including weights up to 2^40 whose scaled B-tile constants leave
    the f16 split's range (those tiles are flagged and take the record
    formula); log-sum-exp as well."""
    import ctypes
    p, n, a = f32(*synth.ring_torus(3000, 55, noise=0.005, jitter_deg=2.0))
    w = weights_for(len(p), 56)
    w[::97] = 2.0 ** 40
    cl = ptsdf.Cloud(p, n, a, weights=w)
    info = cl.info()
    assert info["exact_tiles"] > 0 and info["n_direct"] > 0.9 * len(p)
    x = f32(synth.uniform_queries(1200, 57, -1.6, 1.6))
    orc = oracle_mod.Cloud(p, n, a, weights=w)
    tol = TOL_REL * aabb_diag(p)
    tc, alu = run(cl, x, engine=2), run(cl, x, engine=1)
    assert np.abs(tc - orc.phi(x)).max() <= tol
    assert np.abs(alu - orc.phi(x)).max() <= tol
    lse = run(cl, x, engine=2, formula=ptsdf.SDF_FORMULA_LSE)
    assert np.abs(lse - orc.lse(x)).max() <= tol
    # the tensor-core loop did run
    from paper_2607_16946_b300 import _abi
    L = ptsdf.lib()
    _abi.check(L.sdf_profile_enable(1))
    run(cl, x, engine=2)
    cnt, ms = ctypes.c_int64(0), ctypes.c_double(0)
    _abi.check(L.sdf_profile_read(_abi.SDF_K_FWD_TC, ctypes.byref(cnt), ctypes.byref(ms)))
    L.sdf_profile_enable(0)
    assert cnt.value >= 1


def test_integer_weights_equal_repeated_points(ptsdf):
    """GPU against GPU: weights k_i against the unweighted cloud with point i
    repeated k_i times (the engines differ: the repeated cloud takes the
    tensor cores)."""
    p, n, a = mixed_cloud(34)
    k = np.random.Generator(np.random.PCG64(35)).integers(1, 4, size=len(p))
    rep = np.repeat(np.arange(len(p)), k)
    cw = ptsdf.Cloud(p, n, a, weights=k.astype(np.float32))
    cd = ptsdf.Cloud(p[rep], n[rep], a[rep])
    x = f32(synth.uniform_queries(900, 36, -1.5, 1.5))
    tol = TOL_REL * aabb_diag(p)
    assert np.abs(run(cw, x) - run(cd, x)).max() <= tol
    lse = {"formula": ptsdf.SDF_FORMULA_LSE}
    assert np.abs(run(cw, x, **lse) - run(cd, x, **lse)).max() <= tol


def test_weighted_gradient_and_laplacian(ptsdf, oracle_mod):
    import torch
    p, n, a = mixed_cloud(37)
    w = weights_for(len(p), 38)
    cl = ptsdf.Cloud(p, n, a, weights=w)
    orc = oracle_mod.Cloud(p, n, a, weights=w)
    x = f32(synth.uniform_queries(2000, 39, -1.5, 1.5))
    x = x[kink_free(p, x, 1e-5)][:500]
    phi, g, _ = cl.query_grad(torch.as_tensor(x, device="cuda"))
    torch.cuda.synchronize()
    ophi, og = orc.grad_x(x)
    assert np.abs(phi.cpu().numpy() - ophi).max() <= TOL_REL * aabb_diag(p)
    check_close(g.cpu().numpy().astype(np.float64), og)
    xl = x[kink_free(p, x, 0.02, 0.3)][:200]
    assert len(xl) >= 50
    _, gl, lap = cl.query_laplacian(torch.as_tensor(xl, device="cuda"))
    _, rg, rlap = orc.laplacian(xl)
    err = np.abs(lap.cpu().numpy() - rlap) / (1.0 + np.abs(rlap))
    assert err.max() <= 1e-2, err.max()
    assert np.abs(gl.cpu().numpy() - rg).max() <= 1e-3 * (1 + np.abs(rg).max())


def test_weighted_backward_params(ptsdf, oracle_mod):
    import torch
    p, n, a = f32(*synth.ellipsoid(1500, 40, perturb=0.05))
    w = weights_for(len(p), 41)
    x = f32(synth.uniform_queries(400, 42, -1.5, 1.5))
    x = x[kink_free(p, x, 1e-5)][:300]
    G = f32(np.random.Generator(np.random.PCG64(43)).normal(size=x.shape[0]))
    cl = ptsdf.Cloud(p, n, a, weights=w)
    xt = torch.as_tensor(x, device="cuda")
    _, _, saved = cl.query_grad(xt)
    gp = cl.backward_params(xt, saved, torch.as_tensor(G, device="cuda"))
    torch.cuda.synchronize()
    assert cl.device_status() == 0
    ref = oracle_mod.Cloud(p, n, a, weights=w).grad_params(x, G)
    scale = np.abs(ref).max()
    assert np.abs(gp.cpu().numpy() - ref).max() <= 2e-3 * scale


@pytest.mark.parametrize("lse", [False, True])
def test_weighted_radius(ptsdf, oracle_mod, lse):
    """Radius-limited sums (both branches: points inside R_eval and the
    32-nearest fallback) with weights, blend and log-sum-exp."""
    p, n, a = mixed_cloud(44)
    w = weights_for(len(p), 45)
    cl = ptsdf.Cloud(p, n, a, weights=w)
    orc = oracle_mod.Cloud(p, n, a, weights=w)
    x = f32(synth.uniform_queries(1500, 46, -1.5, 1.5))
    lam = 300.0
    kw = {"formula": ptsdf.SDF_FORMULA_LSE} if lse else {}
    got = run(cl, x, lambda_mode=ptsdf.SDF_LAMBDA_RADIUS, fixed_lambda=lam, **kw)
    _, used = orc.phi_radius(x, lam, used=True)
    assert (used > 0).sum() > 50 and (used < 0).sum() > 50
    check_against_oracle(orc, p, x, got, lam, lse=lse)


@pytest.mark.parametrize("engine", [0, 1, 2])
@pytest.mark.parametrize("split", [0, 1, 5])
def test_lse_engines(ptsdf, oracle_mod, engine, split):
    """d~ with lambda_x on the tensor engine (engine 2; 0 chooses it) and the
    FP32-unit engine (1), direct output and merged point chunks."""
    p, n, a = mixed_cloud(47)
    cl = ptsdf.Cloud(p, n, a)
    x = f32(synth.uniform_queries(1537, 48, -1.5, 1.5))
    got = run(cl, x, formula=ptsdf.SDF_FORMULA_LSE, engine=engine, split_n=split)
    ref = oracle_mod.Cloud(p, n, a).lse(x)
    assert np.abs(got - ref).max() <= TOL_REL * aabb_diag(p)


def test_lse_fixed_offset_weighted_and_grid(ptsdf, oracle_mod):
    p, n, a = mixed_cloud(49)
    w = weights_for(len(p), 50)
    x = f32(synth.uniform_queries(1000, 51, -1.5, 1.5))
    tol = TOL_REL * aabb_diag(p)
    cl = ptsdf.Cloud(p, n, a)
    got = run(cl, x, formula=ptsdf.SDF_FORMULA_LSE, lambda_mode=ptsdf.SDF_LAMBDA_FIXED, fixed_lambda=70.0,
              offset=0.05)
    ref = oracle_mod.Cloud(p, n, a).lse(x, mode=oracle_mod.FIXED, lam=70.0) - 0.05
    assert np.abs(got - ref).max() <= tol
    cw = ptsdf.Cloud(p, n, a, weights=w)
    got = run(cw, x, formula=ptsdf.SDF_FORMULA_LSE)
    assert np.abs(got - oracle_mod.Cloud(p, n, a, weights=w).lse(x)).max() <= tol
    # the dense-grid cloud on grid nodes, tensor engine
    p2, n2, a2 = config2_cloud()
    idx = np.random.Generator(np.random.PCG64(52)).choice(256 ** 3, size=1024, replace=False)
    xg = f32(synth.grid_query_index(idx, 256))
    got = run(ptsdf.Cloud(p2, n2, a2), xg, formula=ptsdf.SDF_FORMULA_LSE)
    ref = oracle_mod.Cloud(p2, n2, a2).lse(xg)
    assert np.abs(got - ref).max() <= TOL_REL * aabb_diag(p2)


def test_option_errors(ptsdf):
    import torch
    p, n, a = mixed_cloud(53)
    x = torch.as_tensor(f32(synth.uniform_queries(64, 54)), device="cuda")
    cl = ptsdf.Cloud(p, n, a)
    with pytest.raises(ptsdf.SdfError):
        cl.query(x, formula=7)
    with pytest.raises(ptsdf.SdfError):   # FIXED lambda 0 has no log-sum-exp distance
        cl.query(x, formula=ptsdf.SDF_FORMULA_LSE, lambda_mode=ptsdf.SDF_LAMBDA_FIXED, fixed_lambda=0.0)
    for call in (lambda: cl.query_laplacian(x, formula=ptsdf.SDF_FORMULA_LSE),
                 lambda: cl.project_level_set(x, 0.0, formula=ptsdf.SDF_FORMULA_LSE)):
        with pytest.raises(ptsdf.SdfError):
            call()
    for bad in (0.0, -1.0, float("nan"), 1e30):
        w = np.ones(len(p), np.float32)
        w[5] = bad
        with pytest.raises(ptsdf.SdfError):
            ptsdf.Cloud(p, n, a, weights=w)
    torch.cuda.synchronize()


@pytest.mark.parametrize("weighted", [False, True])
@pytest.mark.parametrize("mode", ["global", "fixed"])
def test_lse_gradient(ptsdf, oracle_mod, mode, weighted):
    """sdf_query_grad with the log-sum-exp formula: d~ and grad d~ against the
    oracle's duals (lambda_x(x) included for GLOBAL), away from ties of the
    farthest point; the C ABI refuses a saved-statistics buffer for it."""
    import ctypes
    import torch
    from paper_2607_16946_b300 import _abi
    p, n, a = mixed_cloud(58)
    w = weights_for(len(p), 59) if weighted else None
    cl = ptsdf.Cloud(p, n, a, weights=w)
    orc = oracle_mod.Cloud(p, n, a, weights=w)
    x = f32(synth.uniform_queries(1500, 60, -1.5, 1.5))
    x = x[kink_free(p, x, 1e-5)][:500]
    kw, okw = ({}, {}) if mode == "global" else (
        {"lambda_mode": ptsdf.SDF_LAMBDA_FIXED, "fixed_lambda": 40.0}, {"mode": oracle_mod.FIXED, "lam": 40.0})
    xt = torch.as_tensor(x, dtype=torch.float32, device="cuda")
    d, g, sv = cl.query_grad(xt, formula=ptsdf.SDF_FORMULA_LSE, **kw)
    torch.cuda.synchronize()
    assert sv is None and cl.device_status() == 0
    od, og = orc.lse_grad(x, **okw)
    assert np.abs(d.cpu().numpy() - od).max() <= TOL_REL * aabb_diag(p)
    check_close(g.cpu().numpy().astype(np.float64), og)
    saved = torch.empty((len(x), 8), device="cuda")
    o = _abi.make_opts(formula=ptsdf.SDF_FORMULA_LSE, **kw)
    assert ptsdf.lib().sdf_query_grad(cl.handle, ctypes.c_void_p(xt.data_ptr()), len(x), ctypes.c_void_p(d.data_ptr()),
                                      ctypes.c_void_p(g.data_ptr()), ctypes.c_void_p(saved.data_ptr()),
                                      ctypes.byref(o), None) != 0
