"""GPU parity of the tensor-core pair loop (engine SDF_ENGINE_TENSOR) against
the FP64 oracle, element by element, and against the FP32-unit loop.

Tolerance: |phi_gpu - phi_oracle| <= 1e-4 x AABB diagonal (the FP32 bar).
Cases: direct-only clouds over several 32-point tiles and 128-query blocks
with ragged tails; mixed clouds (direct, flat and curved kappa-form tiles,
each segment ending in a partial tile); explicit split factors; queries on
and next to the torus axis; queries far outside the cloud (the exact-only
lanes) for both forms; tiles flagged exact because a curvature leaves the
f16 split's range; FIXED lambda and offsets; the dense-grid cloud on
sampled nodes.
"""
import numpy as np
import pytest

import synth
from workloads import GRID_RES, TOL_REL, aabb_diag, config1, config2_cloud, f32, mixed_cloud

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


def run(cloud, x, engine, **kw):
    import torch
    xt = torch.as_tensor(np.asarray(x, np.float32), device="cuda")
    phi = cloud.query(xt, engine=engine, **kw)
    torch.cuda.synchronize()
    assert cloud.device_status() == 0
    return phi.cpu().numpy().astype(np.float64)


def tc_launches(ptsdf, fn):
    """Runs fn with kernel profiling on; returns the number of k_fwd_tc launches."""
    import ctypes
    from paper_2607_16946_b300 import _abi
    L = ptsdf.lib()
    _abi.check(L.sdf_profile_enable(1))
    try:
        fn()
        cnt, ms = ctypes.c_int64(0), ctypes.c_double(0)
        _abi.check(L.sdf_profile_read(_abi.SDF_K_FWD_TC, ctypes.byref(cnt), ctypes.byref(ms)))
        return cnt.value
    finally:
        L.sdf_profile_enable(0)


def test_sphere_direct_only(ptsdf, oracle_mod):
    """N = 4,096 sphere (direct records only), Q = 32,768: the tensor-core
    loop runs, and matches the oracle and the exact SDF |x| - 1."""
    p, n, a, x = config1()
    cl = ptsdf.Cloud(p, n, a)
    got = {}
    launches = tc_launches(ptsdf, lambda: got.setdefault("tc", run(cl, x, ptsdf.SDF_ENGINE_TENSOR)))
    assert launches >= 1
    ref = oracle_mod.Cloud(p, n, a).phi(x)
    tol = TOL_REL * aabb_diag(p)
    assert np.abs(got["tc"] - ref).max() <= tol
    assert np.abs(got["tc"] - (np.linalg.norm(x, axis=1) - 1)).max() <= tol
    alu = run(cl, x, ptsdf.SDF_ENGINE_ALU)
    assert np.abs(got["tc"] - alu).max() <= tol


@pytest.mark.parametrize("n_pts,q", [(33, 1), (95, 127), (1000, 129), (2017, 1000)])
def test_ragged_direct(ptsdf, oracle_mod, n_pts, q):
    """Point counts that leave partial 32-point tiles and query counts around
    the 128-query block."""
    p, n, a = f32(*synth.ring_torus(n_pts, 40 + n_pts, noise=0.005, jitter_deg=2.0))
    cl = ptsdf.Cloud(p, n, a)
    assert cl.info()["n_direct"] > 0
    x = f32(synth.uniform_queries(q, 41 + q, -1.6, 1.6))
    got = run(cl, x, ptsdf.SDF_ENGINE_TENSOR)
    ref = oracle_mod.Cloud(p, n, a).phi(x)
    assert np.abs(got - ref).max() <= TOL_REL * aabb_diag(p)


@pytest.mark.parametrize("q", [1, 127, 129, 1537])
@pytest.mark.parametrize("split", [0, 1, 3, 7])
def test_mixed_cloud(ptsdf, oracle_mod, q, split):
    """Direct and kappa-form tiles (flat and curved) on the tensor cores,
    point chunks merged from partials."""
    p, n, a = mixed_cloud()
    cl = ptsdf.Cloud(p, n, a)
    info = cl.info()
    assert info["n_direct"] > 0 and info["n_kappa"] > 0
    x = f32(synth.uniform_queries(q, 600 + q, -1.5, 1.5))
    got = run(cl, x, ptsdf.SDF_ENGINE_TENSOR, split_n=split)
    ref = oracle_mod.Cloud(p, n, a).phi(x)
    assert np.abs(got - ref).max() <= TOL_REL * aabb_diag(p)


@pytest.mark.parametrize("split", [0, 1, 4])
def test_kappa_form_clouds(ptsdf, oracle_mod, split):
    """Noisy superquadric, N = 2,000: curvature-form records only, most of
    them with kappa_min = 0 (the flat formula), the rest curved; queries
    inside, around and far outside the cloud."""
    p, n, a = f32(*synth.superquadric(2000, 5))
    cl = ptsdf.Cloud(p, n, a)
    info = cl.info()
    assert info["n_direct"] == 0 and info["n_kappa"] == 2000 and info["exact_tiles"] == 0
    flat = sum(oracle_mod.fit_record(p[i], n[i], a[i])["flat"] == 1.0 for i in range(len(p)))
    assert 64 < info["n_kappa_flat"] < 2000 and abs(info["n_kappa_flat"] - flat) <= 20
    rng = np.random.Generator(np.random.PCG64(91))
    dirs = rng.normal(size=(300, 3))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    x = f32(np.concatenate([synth.uniform_queries(1100, 92, -1.3, 1.3), dirs[:150] * 40.0, dirs[150:] * 900.0]))
    got = {}
    launches = tc_launches(ptsdf, lambda: got.setdefault("tc", run(cl, x, ptsdf.SDF_ENGINE_TENSOR, split_n=split)))
    assert launches >= 1
    ref = oracle_mod.Cloud(p, n, a).phi(x)
    tol = TOL_REL * aabb_diag(p)
    assert (np.abs(got["tc"] - ref) <= tol + 2e-6 * np.abs(ref)).all(), np.abs(got["tc"] - ref).max()


def test_out_of_range_curvature_tiles(ptsdf, oracle_mod):
    """Points whose kappa_max s exceeds the f16 split's range (tube radii of
    1e-5): their tiles are flagged and take the record formula, flat and
    curved kappa forms both, next to ordinary tiles."""
    p1, n1, a1 = synth.plane_patch(300, 93)
    a1[:40, 5] = 4e4                       # kappa_max ~ 8e4, kappa_min = 0
    a1[40:70, 5] = 4e4
    a1[40:70, 4] = 1e-3                    # kappa_min ~ 2e-3: curved kappa form
    p2, n2, a2 = synth.superquadric(500, 94)
    p, n, a = f32(np.concatenate([p1 * 0.9, p2]), np.concatenate([n1, n2]), np.concatenate([a1, a2]))
    cl = ptsdf.Cloud(p, n, a)
    info = cl.info()
    assert 2 <= info["exact_tiles"] < (info["n_kappa"] + 31) // 32
    x = f32(synth.uniform_queries(700, 95, -1.3, 1.3))
    got = run(cl, x, ptsdf.SDF_ENGINE_TENSOR)
    ref = oracle_mod.Cloud(p, n, a).phi(x)
    assert np.abs(got - ref).max() <= TOL_REL * aabb_diag(p)
    alu = run(cl, x, ptsdf.SDF_ENGINE_ALU)
    assert np.abs(got - alu).max() <= TOL_REL * aabb_diag(p)


def test_split_factors_agree(ptsdf):
    p, n, a = f32(*synth.ring_torus(6000, 50, noise=0.005, jitter_deg=2.0))
    cl = ptsdf.Cloud(p, n, a)
    x = f32(synth.uniform_queries(3000, 51))
    base = run(cl, x, ptsdf.SDF_ENGINE_TENSOR, split_n=1)
    for s in (2, 5, 31):
        np.testing.assert_allclose(run(cl, x, ptsdf.SDF_ENGINE_TENSOR, split_n=s), base, atol=2e-6, rtol=0)


def test_axis_and_centre(ptsdf, oracle_mod):
    """Ring torus (every fitted torus shares the z axis and the centre):
    queries on the axis, next to it and at the centre, where vv - h^2 cancels."""
    p, n, a = f32(*synth.ring_torus(4000, 60, noise=0.0, jitter_deg=0.0))
    cl = ptsdf.Cloud(p, n, a)
    z = np.linspace(-1.5, 1.5, 301)
    rng = np.random.Generator(np.random.PCG64(61))
    rows = [np.stack([np.zeros_like(z), np.zeros_like(z), z], 1)]
    for r in (1e-6, 1e-4, 1e-3, 1e-2, 3e-2, 0.1):
        ang = rng.uniform(0, 2 * np.pi, z.size)
        rows.append(np.stack([r * np.cos(ang), r * np.sin(ang), z], 1))
    rows.append(np.zeros((1, 3)))
    x = f32(np.concatenate(rows))
    got = run(cl, x, ptsdf.SDF_ENGINE_TENSOR)
    ref = oracle_mod.Cloud(p, n, a).phi(x)
    assert np.abs(got - ref).max() <= TOL_REL * aabb_diag(p)


def test_far_queries(ptsdf, oracle_mod):
    """Queries from just inside to 1e4 diagonals outside the cloud (beyond
    32 s every pair takes the exact formula)."""
    p, n, a = f32(*synth.ring_torus(3000, 70, noise=0.005, jitter_deg=2.0))
    cl = ptsdf.Cloud(p, n, a)
    rng = np.random.Generator(np.random.PCG64(71))
    dirs = rng.normal(size=(640, 3))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    radii = np.repeat([0.5, 2.0, 10.0, 60.0, 130.0, 1000.0, 3e4], 1)
    x = f32(np.concatenate([dirs[i::7] * r for i, r in enumerate(radii)]))
    got = run(cl, x, ptsdf.SDF_ENGINE_TENSOR)
    ref = oracle_mod.Cloud(p, n, a).phi(x)
    tol = TOL_REL * aabb_diag(p)
    # far away phi grows with the distance; FP32 keeps ~1e-7 of it
    assert (np.abs(got - ref) <= tol + 2e-6 * np.abs(ref)).all(), np.abs(got - ref).max()


def test_fixed_lambda_offset(ptsdf, oracle_mod):
    p, n, a = f32(*synth.ring_torus(3000, 11, noise=0.005, jitter_deg=2.0))
    cl = ptsdf.Cloud(p, n, a)
    x = f32(synth.uniform_queries(1500, 12, -1.6, 1.6))
    got = run(cl, x, ptsdf.SDF_ENGINE_TENSOR, lambda_mode=ptsdf.SDF_LAMBDA_FIXED, fixed_lambda=200.0, offset=0.1)
    ref = oracle_mod.Cloud(p, n, a).phi(x, mode=oracle_mod.FIXED, lam=200.0) - 0.1
    assert np.abs(got - ref).max() <= TOL_REL * aabb_diag(p)


@pytest.mark.parametrize("C", [4.0, 64.0, 87.0])
def test_screening_constant(ptsdf, oracle_mod, C):
    p, n, a = f32(*synth.ring_torus(5000, 9, noise=0.005, jitter_deg=2.0))
    cl = ptsdf.Cloud(p, n, a)
    x = f32(synth.uniform_queries(2000, 10, -1.6, 1.6))
    got = run(cl, x, ptsdf.SDF_ENGINE_TENSOR, C=C)
    ref = oracle_mod.Cloud(p, n, a).phi(x, C=C)
    assert np.abs(got - ref).max() <= TOL_REL * aabb_diag(p)


def test_shapes_offset_from_origin(ptsdf, oracle_mod):
    """An ellipsoid cloud translated far from the origin (the centring of the
    features) and a superquadric cloud (curvatures up to the cap)."""
    pe, ne, ae = synth.ellipsoid(3000, 80, (1.0, 0.6, 0.4))
    ps, ns, as_ = synth.superquadric(3000, 81)
    for k, (pts, nrm, prm) in enumerate([(pe + np.array([500.0, -200.0, 80.0]), ne, ae), (ps, ns, as_)]):
        p, n, a = f32(pts, nrm, prm)
        cl = ptsdf.Cloud(p, n, a)
        lo, hi = p.min(0).astype(np.float64), p.max(0).astype(np.float64)
        x = f32(lo - 0.2 * (hi - lo) + synth.uniform_queries(1500, 82 + k, 0.0, 1.0) * (hi - lo) * 1.4)
        got = run(cl, x, ptsdf.SDF_ENGINE_TENSOR)
        ref = oracle_mod.Cloud(p, n, a).phi(x)
        assert np.abs(got - ref).max() <= TOL_REL * aabb_diag(p)


def test_dense_grid_subset(ptsdf, oracle_mod):
    """Dense-grid cloud (N = 100,000 noisy ring torus) on 8,192 sampled grid
    nodes."""
    p, n, a = config2_cloud()
    cl = ptsdf.Cloud(p, n, a)
    rng = np.random.Generator(np.random.PCG64(2))
    idx = rng.integers(0, GRID_RES ** 3, size=8192)
    x = f32(synth.grid_query_index(idx, GRID_RES))
    got = run(cl, x, ptsdf.SDF_ENGINE_TENSOR)
    ref = oracle_mod.Cloud(p, n, a).phi(x)
    assert np.abs(got - ref).max() <= TOL_REL * aabb_diag(p)


def test_engine_option_checks(ptsdf):
    p, n, a = mixed_cloud(4)
    cl = ptsdf.Cloud(p, n, a)
    import torch
    x = torch.zeros((4, 3), device="cuda")
    with pytest.raises(ptsdf.SdfError):
        cl.query(x, engine=ptsdf.SDF_ENGINE_TENSOR, precision=1)
    with pytest.raises(ptsdf.SdfError):
        cl.query(x, engine=7)
    with pytest.raises(ptsdf.SdfError):
        cl.query_grad(x, engine=ptsdf.SDF_ENGINE_TENSOR)


def test_probe_rates(ptsdf):
    """sdf_probe_rates returns plausible per-SM, per-clock unit rates: the
    special-function unit slower than FMA, exp2 at least as fast as sqrt."""
    import ctypes
    buf = (ctypes.c_double * 8)()
    assert ptsdf.lib().sdf_probe_rates(buf) == 0
    sqrt_r, rsqrt_r, ex2_r, fma_r, rcp_r, direct, flat, curved = list(buf)
    for r in (sqrt_r, rsqrt_r, ex2_r, rcp_r):
        assert 2.0 <= r <= 64.0, list(buf)
    assert 32.0 <= fma_r <= 260.0, list(buf)
    assert ex2_r >= 0.9 * sqrt_r and fma_r > ex2_r
    # a whole pair's mix is slower than any of its operations alone, and the
    # curved curvature form (six operations) the slowest
    assert 0.5 <= curved < flat <= 1.1 * direct < sqrt_r, list(buf)


def test_wait_timeout_reports_and_recovers(ptsdf):
    """Failure detection without a fault: a bounded wait on an mbarrier phase
    that nothing completes gives up after its limit, the kernel records
    SDF_DEV_WAIT_TIMEOUT and returns, and the context keeps working."""
    import ctypes
    import torch
    from paper_2607_16946_b300 import _abi
    bits, ms = ctypes.c_int32(), ctypes.c_double()
    assert ptsdf.lib().sdf_selftest_wait_timeout(2000, ctypes.byref(bits), ctypes.byref(ms)) == 0
    assert bits.value == _abi.SDF_DEV_WAIT_TIMEOUT
    assert 2.0 <= ms.value < 1000.0
    p, n, a, x = config1()
    cl = ptsdf.Cloud(p, n, a)
    phi = run(cl, x[:1000], ptsdf.SDF_ENGINE_TENSOR)
    assert np.isfinite(phi).all()


def test_fma_pipe_square_root_matches_sqrtf(ptsdf):
    """The tensor-core epilogue takes the weight's distance d = sqrt(d^2) on
    the FMA pipe (Lomont's bit-level estimate of 1/sqrt and two Newton steps,
    within 4.8e-6 by the CPU emulation): against CUDA's correctly rounded
    sqrtf over 2^25 normal floats it stays within 5e-6."""
    import ctypes
    err = ctypes.c_double()
    assert ptsdf.lib().sdf_selftest_soft_sqrt(ctypes.byref(err)) == 0
    print("soft sqrt max relative error", err.value)
    assert 0.0 <= err.value <= 5e-6
