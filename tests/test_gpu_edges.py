"""GPU edge cases of the query path against the FP64 oracle.

- Clouds translated far from the origin and rescaled by 1e-3 and 1e3: the
  tensor-core loop centres its coordinates on the bounding box and divides
  by a power of two at least the diagonal, so both engines must keep the
  relative FP32 bar (1e-4 x AABB diagonal) at every scale.
- A cloud of coincident points: queries away from it (every pair the same)
  and on it (d_max = 0, lambda_x = 0).
- Non-finite queries share query blocks with ordinary ones: their own
  results are not finite, and every other query of the block is unaffected.
"""
import numpy as np
import pytest

import synth
from workloads import TOL_REL, aabb_diag, f32, mixed_cloud

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
    xt = torch.as_tensor(np.asarray(x, np.float32), device="cuda")
    out = cloud.query(xt, **kw)
    torch.cuda.synchronize()
    assert cloud.device_status() == 0
    return out.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("scale,shift", [(1.0, (100.0, -50.0, 30.0)), (1e-3, (0.0, 0.0, 0.0)),
                                         (1e3, (2e3, 0.0, -1e3))])
def test_translated_and_rescaled_clouds(ptsdf, oracle_mod, scale, shift):
    p0, n, a = mixed_cloud(61)
    shift = np.asarray(shift)
    p = f32(p0 * scale + shift)
    # the same surfaces at the new scale: curvature coefficients scale by 1 / scale
    a = f32(a.astype(np.float64) * np.array([scale, 1, 1, 1 / scale, 1 / scale, 1 / scale]))
    x = f32(synth.uniform_queries(1200, 62, -1.5, 1.5) * scale + shift)
    cl = ptsdf.Cloud(p, n, a)
    orc = oracle_mod.Cloud(p, n, a)
    tol = TOL_REL * aabb_diag(p)
    ref = orc.phi(x)
    for engine in (1, 2):
        assert np.abs(run(cl, x, engine=engine) - ref).max() <= tol, engine
    assert np.abs(run(cl, x, formula=ptsdf.SDF_FORMULA_LSE) - orc.lse(x)).max() <= tol


def test_coincident_points(ptsdf, oracle_mod):
    p = f32(np.tile([[0.2, -0.1, 0.3]], (70, 1)))
    n = f32(np.tile([[0.0, 0.6, 0.8]], (70, 1)))
    a = f32(np.tile([[0.0, 0.0, 0.0, 0.0, -0.5, -0.5]], (70, 1)))   # unit sphere through the point
    cl = ptsdf.Cloud(p, n, a)
    x = f32(np.concatenate([synth.uniform_queries(300, 63, -1.5, 1.5), p[:2]]))
    got = run(cl, x)
    ref = oracle_mod.Cloud(p, n, a).phi(x)
    assert np.isfinite(got).all()
    assert np.abs(got - ref).max() <= 1e-5


@pytest.mark.parametrize("engine", [1, 2])
def test_non_finite_queries_stay_local(ptsdf, oracle_mod, engine):
    p, n, a = mixed_cloud(64)
    x = f32(synth.uniform_queries(700, 65, -1.5, 1.5))
    bad = [3, 130, 131, 520]
    x[bad[0]] = np.nan
    x[bad[1], 1] = np.inf
    x[bad[2], 0] = -np.inf
    x[bad[3], 2] = np.nan
    cl = ptsdf.Cloud(p, n, a)
    got = run(cl, x, engine=engine)
    good = np.setdiff1d(np.arange(len(x)), bad)
    assert not np.isfinite(got[bad]).any()
    ref = oracle_mod.Cloud(p, n, a).phi(x[good])
    assert np.abs(got[good] - ref).max() <= TOL_REL * aabb_diag(p)
