"""Pins of the oracle's two convolutional baselines (Sec. 5, "Signed distance
accuracy"), CPU only:

  phi_SSPD  Eq. SmoothedSignedPlanarDistance: the self-normalised blend of the
            signed distances <x - p_i, n_i> to the points' tangent planes;
  phi_SHC   Eq. ScreenedWindingNumber: sign(w) (-(1/lambda) log|w| + sigma_x)
            of the screened double-layer sum w.

What fixes them, independently of the oracle's own formulas:
  - a plane cloud: phi_SSPD is the exact signed plane distance (every term is
    the same); for phi_SHC a dense grid on a plane with area weights s^2
    approximates the double-layer integral over the plane, which is exactly
    sign(h) exp(-lambda |h|) (the kernel is a derivative in d), so phi_SHC
    converges to the signed height h as the spacing s shrinks;
  - phi_SSPD equals the oracle's torus blend on patches with all six
    coefficients zero (each torus degenerates to the tangent plane), and
    reduces to the weighted mean (lambda -> 0) and the nearest point's
    planar distance (lambda -> infinity);
  - phi_SHC -> sign(<x - p_nn, n_nn>) d_min as lambda -> infinity, its sign
    on a closed convex cloud (inside: every term is negative), and its
    degenerate cases (X26);
  - invariances of both: rigid motions, uniform scale (with the area weights
    scaled by s^2 for phi_SHC), every normal flipped (both negate), point
    order, integer weights equal to repeated points.
"""
import numpy as np
import pytest

import synth
from workloads import f32, mixed_cloud


@pytest.fixture(scope="module")
def orc(oracle_mod):
    return oracle_mod


def plane_grid(s, half=1.0):
    g = np.arange(-half + s / 2, half, s)
    X, Y = np.meshgrid(g, g)
    P = np.stack([X.ravel(), Y.ravel(), np.zeros(X.size)], 1)
    N = np.tile([0.0, 0.0, 1.0], (P.shape[0], 1))
    return P, N, np.zeros((P.shape[0], 6))


def unit(v):
    return v / np.linalg.norm(v)


def random_rotation(seed):
    q, r = np.linalg.qr(np.random.Generator(np.random.PCG64(seed)).normal(size=(3, 3)))
    return q * np.sign(np.diag(r))


def mixed(seed=5):
    p, n, a = mixed_cloud(seed, rounded=False)
    return p, n, a


# --------------------------------------------------------------------------
# phi_SSPD
# --------------------------------------------------------------------------
def test_sspd_plane_is_exact(orc):
    rng = np.random.Generator(np.random.PCG64(1))
    n0 = unit(rng.normal(size=3))
    u = unit(np.cross(n0, [0.3, 0.5, 0.7]))
    v = np.cross(n0, u)
    c = rng.uniform(size=(400, 2)) * 2 - 1
    p0 = np.array([0.1, -0.2, 0.3])
    P = p0 + c[:, :1] * u + c[:, 1:] * v
    N = np.tile(n0, (400, 1))
    w = np.exp(rng.uniform(-1, 1, size=400))
    x = rng.uniform(-1.5, 1.5, size=(300, 3))
    cl = orc.Cloud(P, N, np.zeros((400, 6)), weights=w)
    exact = (x - p0) @ n0
    assert np.abs(cl.sspd(x) - exact).max() < 1e-12
    assert np.abs(cl.sspd(x, mode=orc.FIXED, lam=30.0) - exact).max() < 1e-12


@pytest.mark.parametrize("weighted", [False, True])
def test_sspd_equals_blend_of_flat_patches(orc, weighted):
    """With all six coefficients zero every torus is the point's tangent plane
    (the blend's own plane pin), so the blend is phi_SSPD."""
    p, n, _ = mixed()
    w = np.exp(np.random.Generator(np.random.PCG64(2)).uniform(-1, 1, size=len(p))) if weighted else None
    x = synth.uniform_queries(400, 3, -1.5, 1.5)
    cl = orc.Cloud(p, n, np.zeros((len(p), 6)), weights=w)
    for kw in ({}, {"mode": orc.FIXED, "lam": 25.0}):
        ref = cl.phi(x, **kw)
        assert np.abs(cl.sspd(x, **kw) - ref).max() < 1e-11 * max(1.0, np.abs(ref).max())


def test_sspd_lambda_limits(orc):
    p, n, a = mixed()
    w = np.exp(np.random.Generator(np.random.PCG64(4)).uniform(-1, 1, size=len(p)))
    cl = orc.Cloud(p, n, a, weights=w)
    x = synth.uniform_queries(200, 5, -1.5, 1.5)
    plane = np.einsum("qik,ik->qi", x[:, None, :] - p[None], n)       # <x - p_i, n_i>
    mean = np.average(plane, axis=1, weights=w)
    assert np.abs(cl.sspd(x, mode=orc.FIXED, lam=1e-9) - mean).max() < 1e-7
    d = np.linalg.norm(x[:, None, :] - p[None], axis=2)
    order = np.argsort(d, axis=1)
    gap = np.take_along_axis(d, order[:, 1:2], 1)[:, 0] - np.take_along_axis(d, order[:, :1], 1)[:, 0]
    keep = gap > 2e-3                                  # runner-up weight below e^-200 at lambda = 1e5
    near = plane[np.arange(len(x)), order[:, 0]]
    got = cl.sspd(x[keep], mode=orc.FIXED, lam=1e5)
    assert keep.sum() > 150
    assert np.abs(got - near[keep]).max() < 1e-12


def test_sspd_invariances(orc):
    p, n, a = mixed()
    x = synth.uniform_queries(300, 6, -1.5, 1.5)
    base = orc.Cloud(p, n, a).sspd(x)
    Rm, t = random_rotation(7), np.array([0.3, -1.1, 0.4])
    moved = orc.Cloud(p @ Rm.T + t, n @ Rm.T, a).sspd(x @ Rm.T + t)
    assert np.abs(moved - base).max() < 1e-11
    assert np.abs(orc.Cloud(2.5 * p, n, a).sspd(2.5 * x) - 2.5 * base).max() < 1e-11
    assert np.abs(orc.Cloud(p, -n, a).sspd(x) + base).max() < 1e-12
    perm = np.random.Generator(np.random.PCG64(8)).permutation(len(p))
    assert np.abs(orc.Cloud(p[perm], n[perm], a[perm]).sspd(x) - base).max() < 1e-12
    k = np.random.Generator(np.random.PCG64(9)).integers(1, 4, size=len(p))
    rep = np.repeat(np.arange(len(p)), k)
    wc = orc.Cloud(p, n, a, weights=k.astype(float)).sspd(x)
    assert np.abs(wc - orc.Cloud(p[rep], n[rep], a[rep]).sspd(x)).max() < 1e-12


# --------------------------------------------------------------------------
# phi_SHC
# --------------------------------------------------------------------------
def test_shc_plane_grid_converges_to_signed_height(orc):
    heights = np.array([-0.1, -0.05, -0.02, 0.02, 0.05, 0.1])
    q = np.stack([np.full(6, 0.013), np.full(6, -0.021), heights], 1)
    err = {}
    for s in (0.02, 0.01):
        P, N, A = plane_grid(s)
        cl = orc.Cloud(P, N, A, weights=np.full(len(P), s * s))
        phi, cond = cl.shc(q, cond=True)
        assert np.all(np.abs(cond - 1.0) < 1e-12)       # every term has the sign of h
        err[s] = np.abs(phi - heights)
        fixed = cl.shc(q, mode=orc.FIXED, lam=60.0)
        assert np.abs(fixed - heights).max() < (1e-4 if s == 0.02 else 2e-6)
    assert err[0.01].max() < 2e-6
    near = np.abs(heights) == 0.02
    assert np.all(err[0.01][near] < err[0.02][near] / 10)


def test_shc_large_lambda_limit(orc):
    """-(1/lambda) log|w| -> d_min and sign(w) -> the nearest point's planar
    sign as lambda grows (the correction is O(log(lambda) / lambda))."""
    p, n, a = mixed()
    cl = orc.Cloud(p, n, a)
    x = synth.uniform_queries(300, 10, -1.5, 1.5)
    d = np.linalg.norm(x[:, None, :] - p[None], axis=2)
    order = np.argsort(d, axis=1)
    i0 = order[:, 0]
    dmin = d[np.arange(len(x)), i0]
    gap = d[np.arange(len(x)), order[:, 1]] - dmin
    plane = np.einsum("qk,qk->q", x - p[i0], n[i0])
    keep = (gap > 0.02) & (np.abs(plane) > 0.05 * dmin)
    assert keep.sum() > 100
    dev = []
    for lam in (1e3, 1e4, 1e5):
        phi = cl.shc(x[keep], mode=orc.FIXED, lam=lam)
        assert np.all(np.sign(phi) == np.sign(plane[keep]))
        dev.append(np.abs(np.abs(phi) - dmin[keep]))
    assert np.all(dev[1] < dev[0] / 5) and np.all(dev[2] < dev[1] / 5)
    assert dev[2].max() < 2e-4


def test_shc_sign_on_closed_convex_cloud(orc):
    """Clean unit-sphere cloud, area weights 4 pi / N: inside every term is
    negative (w < 0 exactly, condition number 1); outside the screened near
    side dominates.  So sign(phi_SHC) = sign(|x| - 1) away from the surface."""
    p, n, a = synth.sphere_fibonacci(2048, 11)
    cl = orc.Cloud(p, n, a, weights=np.full(2048, 4 * np.pi / 2048))
    x = synth.uniform_queries(3000, 12, -1.5, 1.5)
    r = np.linalg.norm(x, axis=1)
    x = x[np.abs(r - 1) > 0.05]
    phi, cond = cl.shc(x, cond=True)
    inside = np.linalg.norm(x, axis=1) < 1
    assert np.all(np.sign(phi) == np.where(inside, -1.0, 1.0))
    assert np.all(np.abs(cond[inside] - 1.0) < 1e-12)


def test_shc_invariances(orc):
    p, n, a = mixed()
    A = np.exp(np.random.Generator(np.random.PCG64(13)).uniform(-1, 1, size=len(p)))
    x = synth.uniform_queries(300, 14, -1.5, 1.5)
    base, cond = orc.Cloud(p, n, a, weights=A).shc(x, cond=True)
    ok = cond < 1e6            # well away from w = 0, where the sign flips and |phi| -> infinity
    Rm, t = random_rotation(15), np.array([-0.4, 0.9, 0.2])
    moved = orc.Cloud(p @ Rm.T + t, n @ Rm.T, a, weights=A).shc(x @ Rm.T + t)
    assert np.abs(moved - base)[ok].max() < 1e-9
    s = 1.7
    scaled = orc.Cloud(s * p, n, a, weights=s * s * A).shc(s * x)
    assert np.abs(scaled - s * base)[ok].max() < 1e-9
    assert np.abs(orc.Cloud(p, -n, a, weights=A).shc(x) + base)[ok].max() < 1e-12
    perm = np.random.Generator(np.random.PCG64(16)).permutation(len(p))
    assert np.abs(orc.Cloud(p[perm], n[perm], a[perm], weights=A[perm]).shc(x) - base)[ok].max() < 1e-10
    k = np.random.Generator(np.random.PCG64(17)).integers(1, 4, size=len(p))
    rep = np.repeat(np.arange(len(p)), k)
    wc = orc.Cloud(p, n, a, weights=k.astype(float)).shc(x)
    assert np.abs(wc - orc.Cloud(p[rep], n[rep], a[rep]).shc(x)).max() < 1e-10
    # halving every weight moves -(1/lambda) log|w| by ln 2 / lambda_x, so phi
    # by that much in the direction sign(w)
    half = orc.Cloud(p, n, a, weights=A / 2).shc(x)
    _, st = orc.Cloud(p, n, a, weights=A).phi(x, stats=True)
    assert np.abs(np.abs(half - base) - np.log(2.0) / st[:, 0])[ok].max() < 1e-10


def test_shc_degenerate_cases(orc):
    p, n, a = mixed()
    one = orc.Cloud(p[:1], n[:1], a[:1])
    # a one-point cloud queried at its point: lambda_x = 0 (X9), phi_SHC = 0 (X26)
    assert one.shc(p[:1])[0] == 0.0
    # a query in the point's tangent plane: w = 0, phi_SHC = +inf (X26)
    flat = orc.Cloud(np.zeros((1, 3)), np.array([[0.0, 0.0, 1.0]]), np.zeros((1, 6)))
    assert flat.shc(np.array([[0.5, -0.25, 0.0]]))[0] == np.inf
    t = unit(np.cross(n[0], [0.2, 0.3, 0.9]))
    # a query exactly at one point of a cloud: that point adds nothing to w
    # (lambda_x, set by the farthest point, does not change without it)
    j = 17
    rest = np.delete(np.arange(len(p)), j)
    at = orc.Cloud(p, n, a).shc(p[j:j + 1])
    assert np.abs(at - orc.Cloud(p[rest], n[rest], a[rest]).shc(p[j:j + 1])).max() < 1e-12
    # one point elsewhere: the sign is the planar sign
    y = p[:1] + 0.3 * n[:1] + 0.1 * t
    assert one.shc(y)[0] > 0 and one.shc(p[:1] - 0.3 * n[:1])[0] < 0
