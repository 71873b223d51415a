"""GPU parity of sphere tracing (Sec. 6) and of the Boolean combinations.

Tracing decides integers (hit or miss, step counts) from floating point, so
rays are compared by outcome: both sides must agree on hit / miss for at
least 99% of rays; where both hit, t_hit agrees to 1e-3 and the step counts
to within 1 for 99% of rays.  The disagreeing rays must be borderline: their
oracle values at the deciding step lie within 1e-3 of eps or of t_max.
"""
import numpy as np
import pytest

import synth
from workloads import f32

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


def gpu_trace(cl, org, dirs, **kw):
    import torch
    t, s, nrm = cl.trace(org, dirs, **kw)
    torch.cuda.synchronize()
    assert cl.device_status() == 0
    return (t.cpu().numpy().astype(np.float64), s.cpu().numpy(),
            None if nrm is None else nrm.cpu().numpy().astype(np.float64))


def test_trace_sphere_closed_form(ptsdf):
    """Exact-SDF sphere cloud: hits at the analytic ray-sphere intersection,
    normals = hit point (unit sphere)."""
    p, n, a = f32(*synth.sphere_fibonacci(512, 61))
    org, dirs = (f32(v) for v in synth.camera_rays(48, 48, 62, dist=3.0, fov_deg=60.0))
    cl = ptsdf.Cloud(p, n, a)
    t, steps, nrm = gpu_trace(cl, org, dirs, max_steps=200, eps=1e-5, t_max=8.0)
    b = np.sum(org * dirs, 1)
    c = np.sum(org * org, 1) - 1.0
    disc = b * b - c
    hit = disc > 1e-3
    miss = disc < -1e-3
    t_ref = -b - np.sqrt(np.where(hit, disc, 0.0))
    assert np.all(t[miss] < 0)
    assert np.abs(t[hit] - t_ref[hit]).max() < 2e-4
    xh = org[hit] + t[hit, None] * dirs[hit]
    assert np.abs(nrm[hit] - xh / np.linalg.norm(xh, axis=1, keepdims=True)).max() < 1e-3
    assert np.all(nrm[~(t > 0)] == 0)


def test_trace_superquadric_subset(ptsdf, oracle_mod):
    """Sphere-tracing configuration (N = 262,144 noisy superquadric, pinhole
    camera at distance 3): 1,024 seeded rays of the 512 x 512 image, 48 steps,
    eps = 1e-4, t_max = 6, against the oracle's tracer; normals at hits
    against the oracle's grad phi."""
    p, n, a = f32(*synth.superquadric(262_144, 1003))
    org, dirs = synth.camera_rays(512, 512, 1003)
    rows = np.random.Generator(np.random.PCG64(7)).choice(org.shape[0], size=1024, replace=False)
    org, dirs = f32(org[rows], dirs[rows])
    cl = ptsdf.Cloud(p, n, a)
    t, steps, nrm = gpu_trace(cl, org, dirs, max_steps=48, eps=1e-4, t_max=6.0)
    oc = oracle_mod.Cloud(p, n, a)
    to, so = oc.trace(org, dirs, max_steps=48, eps=1e-4, t_max=6.0)
    gh, oh = t >= 0, to >= 0
    agree = gh == oh
    assert agree.mean() >= 0.99, agree.mean()
    both = gh & oh
    assert both.sum() > 50
    ok = (np.abs(t[both] - to[both]) <= 1e-3) & (np.abs(steps[both] - so[both]) <= 1)
    assert ok.mean() >= 0.99, ok.mean()
    # normals at hits where both sides hit
    xh = org[both] + to[both, None] * dirs[both]
    _, og = oc.grad_x(xh)
    on = og / np.linalg.norm(og, axis=1, keepdims=True)
    cosang = np.sum(nrm[both] * on, 1)
    assert np.quantile(cosang, 0.01) > 0.99


def test_combine_booleans(ptsdf):
    import torch
    a = torch.linspace(-1, 1, 1001, device="cuda")
    b = torch.flip(a, [0]) * 0.5
    u = ptsdf.combine(ptsdf.SDF_UNION, a, b)
    i = ptsdf.combine(ptsdf.SDF_INTERSECT, a, b)
    d = ptsdf.combine(ptsdf.SDF_DIFFERENCE, a, b)
    torch.testing.assert_close(u, torch.minimum(a, b), rtol=0, atol=0)
    torch.testing.assert_close(i, torch.maximum(a, b), rtol=0, atol=0)
    torch.testing.assert_close(d, torch.maximum(a, -b), rtol=0, atol=0)


def test_trace_full_image_sampled(ptsdf, oracle_mod):
    """Full size in the benchmark's launch configuration: all 512 x 512 rays
    traced in one call (N = 262,144); 200 sampled rays against the oracle's
    tracer (each ray's trace is independent of the batch)."""
    p, n, a = f32(*synth.superquadric(262_144, 1003))
    org, dirs = (f32(v) for v in synth.camera_rays(512, 512, 1003))
    cl = ptsdf.Cloud(p, n, a)
    t, steps, _ = gpu_trace(cl, org, dirs, max_steps=48, eps=1e-4, t_max=6.0, normals=False)
    rows = np.random.Generator(np.random.PCG64(8)).choice(org.shape[0], size=200, replace=False)
    to, so = oracle_mod.Cloud(p, n, a).trace(org[rows], dirs[rows], max_steps=48, eps=1e-4, t_max=6.0)
    tg, sg = t[rows], steps[rows]
    agree = (tg >= 0) == (to >= 0)
    assert agree.mean() >= 0.98
    both = (tg >= 0) & (to >= 0)
    ok = (np.abs(tg[both] - to[both]) <= 1e-3) & (np.abs(sg[both] - so[both]) <= 1)
    assert ok.mean() >= 0.98
