"""GPU parity of the gradient paths against the FP64 oracle.

  sdf_query_grad       d phi / d x (App. D plus the lambda_x(x) term) vs the
                       oracle's forward-mode duals, and vs central finite
                       differences of the oracle (h = 1e-3, Richardson).
  sdf_backward_params  d(sum G phi) / d a vs the oracle's duals through the fit,
                       and vs central differences of the oracle's phi in the
                       coefficients (N = 65,536).
  autograd             the torch.autograd.Function routes both.
Tolerance: 1e-3 relative to max(1, |reference|) per entry (FP32 path).
Queries where a distant point ties for the farthest (within 1e-5 of d_max,
or within the finite-difference stencil) are left out: lambda_x has a kink
there and the two sides may pick different points.
"""
import numpy as np
import pytest

import synth
from workloads import f32, mixed_cloud

pytestmark = pytest.mark.gpu
GTOL = 1e-3


@pytest.fixture(scope="module")
def ptsdf():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2607_16946_b300 import build
    build.build()
    import paper_2607_16946_b300 as m
    return m


def kink_free(p, x, tau, sep=0.05):
    """True for queries whose farthest point is unambiguous: no point lying
    more than `sep` away from the farthest one is within `tau` of d_max.  (At a
    tie between distant far points lambda_x has a kink; ties between close
    neighbours change grad lambda_x by a negligible amount.)  Squared
    distances from |x|^2 + |p|^2 - 2 <x, p> in float32 on the host cores
    (torch), with the band widened by 1e-5 to cover their rounding; the
    spread is computed for the points in the band only."""
    import torch
    P = torch.as_tensor(np.asarray(p, np.float32))
    X = torch.as_tensor(np.asarray(x, np.float32))
    pp = (P * P).sum(1)
    keep = torch.empty(X.shape[0], dtype=torch.bool)
    for i0 in range(0, X.shape[0], 1024):
        xs = X[i0:i0 + 1024]
        d2 = torch.addmm(pp[None] + (xs * xs).sum(1, keepdim=True), xs, P.T, alpha=-2.0)
        dmax2, j = d2.max(1)
        lo = (dmax2.clamp_min(0).sqrt() - tau - 1e-5).clamp_min(0)
        rows, cols = torch.nonzero(d2 >= (lo * lo)[:, None], as_tuple=True)
        far = ((P[cols] - P[j[rows]]) ** 2).sum(1) > sep * sep
        bad = torch.zeros(xs.shape[0], dtype=torch.bool)
        bad[rows[far]] = True
        keep[i0:i0 + 1024] = ~bad
    return keep.numpy()


def config4(n=65536, q=1_000_000):
    p, nn, a = synth.ellipsoid(n, 1004, axes=(1.0, 0.6, 0.4), perturb=0.05)
    x = synth.uniform_queries(q, 1004, -1.5, 1.5)
    return f32(p, nn, a, x)


def gpu_grad(cl, x, **kw):
    import torch
    phi, g, saved = cl.query_grad(torch.as_tensor(x, dtype=torch.float32, device="cuda"), **kw)
    torch.cuda.synchronize()
    assert cl.device_status() == 0
    return phi.cpu().numpy().astype(np.float64), g.cpu().numpy().astype(np.float64), saved


def check_close(got, ref, tol=GTOL):
    err = np.abs(got - ref) / np.maximum(1.0, np.abs(ref))
    assert err.max() <= tol, (err.max(), np.unravel_index(err.argmax(), err.shape))


def test_grad_config4_subset(ptsdf, oracle_mod):
    """Differentiation config (N = 65,536 perturbed ellipsoid), 65,536 seeded
    queries of the 1e6 in one call: phi against the oracle on all of them,
    d phi / d x against the oracle's duals on 2,048 of them and against
    Richardson-extrapolated central differences of the oracle's phi (h = 1e-4,
    h / 2; a wider stencil would straddle the kink of lambda_x for a third of
    the queries of this dense cloud) in one seeded component of each of the
    65,536 queries away from such a kink."""
    p, n, a, x = config4(q=65_536)
    cl = ptsdf.Cloud(p, n, a)
    phi, g, _ = gpu_grad(cl, x)
    oc = oracle_mod.Cloud(p, n, a)
    assert np.abs(phi - oc.phi(x)).max() <= 1e-4 * np.linalg.norm(p.max(0) - p.min(0))
    sub = np.flatnonzero(kink_free(p, x[:2600], 1e-5))[:2048]
    assert sub.size == 2048
    _, og = oc.grad_x(x[sub])
    check_close(g[sub], og)
    keep = np.flatnonzero(kink_free(p, x, 2e-4))     # the stencil moves x by at most 1e-4
    assert keep.size > 0.95 * x.shape[0], keep.size
    comp = np.random.Generator(np.random.PCG64(6)).integers(0, 3, size=keep.size)
    e = np.zeros((keep.size, 3))
    e[np.arange(keep.size), comp] = 1.0
    xs = x[keep]
    fd = [(oc.phi(xs + h * e) - oc.phi(xs - h * e)) / (2 * h) for h in (1e-4, 5e-5)]
    check_close(g[keep, comp], (4 * fd[1] - fd[0]) / 3, tol=2e-3)


def test_backward_params_config4_finite_differences(ptsdf, oracle_mod):
    """d(sum_q G_q phi_q) / d a on the differentiation cloud (N = 65,536):
    512 entries against central differences of the oracle's phi in that
    coefficient (the point's torus refitted at a +- h, h = 1e-3 and h / 2,
    Richardson), 64 seeded queries and upstream gradients.  The entries are
    drawn from the 2,000 largest of the oracle's dual-number gradient, so each
    one is carried by queries near its point."""
    import torch
    p, n, a, x = config4(q=400)
    x = x[kink_free(p, x, 1e-5)][:64]
    G = f32(np.random.Generator(np.random.PCG64(44)).normal(size=x.shape[0]))
    cl = ptsdf.Cloud(p, n, a)
    xt = torch.as_tensor(x, dtype=torch.float32, device="cuda")
    _, _, saved = cl.query_grad(xt)
    gp = cl.backward_params(xt, saved, torch.as_tensor(G, dtype=torch.float32, device="cuda"))
    torch.cuda.synchronize()
    assert cl.device_status() == 0
    gp = gp.cpu().numpy().astype(np.float64)
    oc = oracle_mod.Cloud(p, n, a)
    dual = oc.grad_params(x, G)
    top = np.argsort(-np.abs(dual).ravel())[:2000]
    # away from near-umbilic points, where a step of h can swap which principal
    # curvature is kappa_min (the fit is not differentiable across that swap)
    gap = {}
    for i in set(int(f) // 6 for f in top):
        fr = oracle_mod.fit_record(p[i], n[i], a[i])
        gap[i] = abs(abs(fr["kplus"]) - abs(fr["kminus"])) / max(abs(fr["kplus"]), abs(fr["kminus"]))
    top = np.array([f for f in top if gap[int(f) // 6] > 0.05])
    pick = np.random.Generator(np.random.PCG64(45)).choice(top, size=512, replace=False)
    rich = np.empty(512)
    for m, flat in enumerate(pick):
        i, k = divmod(int(flat), 6)
        fd = []
        for h in (1e-3, 5e-4):
            L = []
            for sgn in (1.0, -1.0):
                ai = a[i].copy()
                ai[k] += sgn * h
                oc.set_params(i, ai)
                L.append(float(np.dot(G, oc.phi(x))))
            fd.append((L[0] - L[1]) / (2 * h))
        oc.set_params(i, a[i])
        rich[m] = (4 * fd[1] - fd[0]) / 3
    got = gp.ravel()[pick]
    scale = np.abs(rich).max()
    assert np.abs(got - rich).max() <= 2e-3 * scale, (np.abs(got - rich).max(), scale)


@pytest.mark.parametrize("split", [0, 1, 4])
@pytest.mark.parametrize("q", [1, 255, 257, 700])
def test_grad_mixed_ragged(ptsdf, oracle_mod, q, split):
    """Both torus record forms, ragged query counts around the 256-query
    block, explicit splits (the 13-sum merge)."""
    p, n, a = mixed_cloud(21)
    x = f32(synth.uniform_queries(3 * q + 10, 600 + q, -1.5, 1.5))
    x = x[kink_free(p, x, 1e-5)][:q]
    cl = ptsdf.Cloud(p, n, a)
    phi, g, _ = gpu_grad(cl, x, split_n=split)
    ophi, og = oracle_mod.Cloud(p, n, a).grad_x(x)
    assert np.abs(phi - ophi).max() <= 1e-4 * np.linalg.norm(p.max(0) - p.min(0))
    check_close(g, og)


def test_grad_fixed_lambda(ptsdf, oracle_mod):
    p, n, a = f32(*synth.ring_torus(3000, 31, noise=0.005, jitter_deg=2.0))
    x = f32(synth.uniform_queries(500, 32, -1.6, 1.6))
    cl = ptsdf.Cloud(p, n, a)
    _, g, _ = gpu_grad(cl, x, lambda_mode=ptsdf.SDF_LAMBDA_FIXED, fixed_lambda=150.0)
    _, og = oracle_mod.Cloud(p, n, a).grad_x(x, mode=oracle_mod.FIXED, lam=150.0)
    check_close(g, og)


def test_backward_params(ptsdf, oracle_mod):
    """d(sum_q G_q phi_q)/d a: ellipsoid (direct records) and the mixed
    cloud without zero curvatures (kappa records), against the oracle."""
    import torch
    for p, n, a in (f32(*synth.ellipsoid(1500, 41, perturb=0.05)),
                    mixed_cloud(22)):
        keep = np.ones(p.shape[0], bool)
        if p.shape[0] == 1000:      # mixed cloud: drop plane / cylinder points (zero curvature)
            fit = [oracle_mod.fit_record(p[i], n[i], a[i]) for i in range(p.shape[0])]
            keep = np.array([abs(f["kmin"]) > 1e-6 for f in fit])
            p, n, a = p[keep], n[keep], a[keep]
        x = f32(synth.uniform_queries(400, 42, -1.5, 1.5))
        x = x[kink_free(p, x, 1e-5)][:300]
        G = f32(np.random.Generator(np.random.PCG64(43)).normal(size=x.shape[0]))
        cl = ptsdf.Cloud(p, n, a)
        info = cl.info()
        xt = torch.as_tensor(x, dtype=torch.float32, device="cuda")
        _, _, saved = cl.query_grad(xt)
        gp = cl.backward_params(xt, saved, torch.as_tensor(G, dtype=torch.float32, device="cuda"))
        torch.cuda.synchronize()
        assert cl.device_status() == 0
        gp = gp.cpu().numpy().astype(np.float64)
        ref = oracle_mod.Cloud(p, n, a).grad_params(x, G)
        scale = np.abs(ref).max()
        assert np.abs(gp - ref).max() <= 2e-3 * scale, (info, np.abs(gp - ref).max(), scale)


def test_autograd_function(ptsdf):
    import torch
    p, n, a = f32(*synth.ellipsoid(2000, 51, perturb=0.05))
    params = torch.as_tensor(a, dtype=torch.float32, device="cuda").requires_grad_(True)
    cl = ptsdf.Cloud(p, n, a)
    x = torch.as_tensor(f32(synth.uniform_queries(300, 52)), dtype=torch.float32, device="cuda")
    x.requires_grad_(True)
    phi = ptsdf.sdf(x, cl, params)
    w = torch.linspace(-1, 1, 300, device="cuda")
    (phi * w).sum().backward()
    _, g, saved = cl.query_grad(x.detach())
    torch.testing.assert_close(x.grad, w[:, None] * g)
    gp = cl.backward_params(x.detach(), saved, w)
    torch.testing.assert_close(params.grad, gp)


def test_grad_config4_full_size_sampled(ptsdf, oracle_mod):
    """Full size in the benchmark's launch configuration: all 1e6 queries in
    one sdf_query_grad call (N = 65,536); 200 sampled outputs against the
    oracle's duals.  The parameter backward over all 1e6 queries with a
    one-hot upstream gradient equals the oracle's d phi_j / d a for that query."""
    import torch
    p, n, a, x = config4()
    cl = ptsdf.Cloud(p, n, a)
    xt = torch.as_tensor(x, dtype=torch.float32, device="cuda")
    phi, g, saved = cl.query_grad(xt)
    torch.cuda.synchronize()
    assert cl.device_status() == 0
    rng = np.random.Generator(np.random.PCG64(9))
    idx = rng.choice(x.shape[0], size=400, replace=False)
    idx = idx[kink_free(p, x[idx], 1e-5)][:200]
    ophi, og = oracle_mod.Cloud(p, n, a).grad_x(x[idx])
    assert np.abs(phi.cpu().numpy()[idx] - ophi).max() <= 1e-4 * np.linalg.norm(p.max(0) - p.min(0))
    check_close(g.cpu().numpy()[idx].astype(np.float64), og)
    for j in idx[:2]:
        G = torch.zeros(x.shape[0], device="cuda")
        G[int(j)] = 1.0
        gp = cl.backward_params(xt, saved, G).cpu().numpy().astype(np.float64)
        ref = oracle_mod.Cloud(p, n, a).grad_params(x[j:j + 1], np.ones(1))
        assert np.abs(gp - ref).max() <= 2e-3 * np.abs(ref).max()
