"""Invariances of the blend on noisy clouds with per-query lambda: properties
of the method (Sec. 4.1 fit, Eq. SingleTorusSDF, Eqs. BasicFormulaShifted and
RelationshipBetweenLambdaAndRadius, Eq. ConvolutionalDistanceFormula) that
hold for any cloud, with no closed form of the blend needed.

- Isometries.  Move points, normals and queries by x -> M x + t with M
  orthogonal (rotations and reflections).  The coefficients are expressed in
  the frame (s, t) of each normal (Eq. BivariatePolynomial), and the frame of
  M n is not M applied to the frame of n.  So the same patch gets new
  coefficients: in-plane coordinates w' = B w with
  B = [[<M s, s'>, <M t, s'>], [<M s, t'>, <M t, t'>]], the linear part maps
  to B l and the quadratic form to B Q B^T, and the height is unchanged.
  Every torus is built from distances, curvatures and the normal, so phi,
  the log-sum-exp distance and the Laplacian are unchanged, and grad phi
  turns by M.  A rotation mixes a10 with a01 and a20, a11, a02 with each
  other, so a swapped or mis-signed coefficient anywhere in the fit fails it.
- Scale.  x -> c x with a00 -> c a00, linear terms unchanged and quadratic
  terms divided by c: every length scales by c, lambda_x = C / sigma_x by 1/c,
  so phi and the log-sum-exp distance scale by c, grad phi is unchanged and
  the Laplacian scales by 1/c.  With a fixed lambda, lambda / c.
- Every point twice: W and S double, d_max is unchanged, so phi is unchanged
  and the log-sum-exp distance drops by ln 2 / lambda_x = ln 2 d_max / (2 C).
- Point order: no effect beyond rounding.
- Every normal flipped (the same patches written over the frames of -n_i,
  heights negated): kappa_min and kappa_max are chosen by magnitude, so each
  torus keeps its shape and changes its sign (Eq. TorusSigns).  phi, grad phi
  and the Laplacian negate; the log-sum-exp distance, which has no sign,
  does not change.
- The radius-limited sums (Sec. 4.2) under isometries, scale (lambda / c,
  R_eval c) and the flip, and D, the mean k-nearest distance of the lambda
  heuristic, under isometries (unchanged) and scale (times c).

The cloud is the mixed test cloud in float64: its cylinder patches keep a
curvature of exactly zero up to rounding at every scale.  (Rounded to FP32
they carry kappa_min ~ 5e-8, just above the fit's absolute flatness threshold
of 1e-8, and a scale by 1/250 moves them across it.)
"""
import numpy as np
import pytest

import synth
from workloads import mixed_cloud


def rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def orthogonal(seed, proper=True):
    q, r = np.linalg.qr(rng(seed).normal(size=(3, 3)))
    q = q * np.sign(np.diag(r))
    if (np.linalg.det(q) > 0) != proper:
        q[:, 2] = -q[:, 2]
    return q


def moved_coefficients(n, a, M, flip=False):
    """Coefficients a = (a00, a01, a10, a11, a02, a20) of the same patches
    after the normals are moved to M n (frames recomputed from M n); with
    flip, to -M n, the height then measured along the flipped normal."""
    s, t = synth.frame(n)
    n2 = -(n @ M.T) if flip else n @ M.T
    s2, t2 = synth.frame(n2)
    Ms, Mt = s @ M.T, t @ M.T
    B = np.empty((len(n), 2, 2))
    B[:, 0, 0] = (Ms * s2).sum(1)
    B[:, 0, 1] = (Mt * s2).sum(1)
    B[:, 1, 0] = (Ms * t2).sum(1)
    B[:, 1, 1] = (Mt * t2).sum(1)
    lin = np.stack([a[:, 2], a[:, 1]], 1)                              # (a10, a01)
    Q = np.empty((len(n), 2, 2))
    Q[:, 0, 0], Q[:, 1, 1] = a[:, 5], a[:, 4]                          # a20, a02
    Q[:, 0, 1] = Q[:, 1, 0] = 0.5 * a[:, 3]                            # a11 / 2
    lin2 = np.einsum("mij,mj->mi", B, lin)
    Q2 = B @ Q @ np.transpose(B, (0, 2, 1))
    out = np.empty_like(a)
    out[:, 0] = a[:, 0]
    out[:, 1], out[:, 2] = lin2[:, 1], lin2[:, 0]
    out[:, 3] = 2.0 * Q2[:, 0, 1]
    out[:, 4], out[:, 5] = Q2[:, 1, 1], Q2[:, 0, 0]
    return n2, -out if flip else out


@pytest.fixture(scope="module")
def cloud():
    p, n, a = mixed_cloud(91, rounded=False)
    x = synth.uniform_queries(160, 92, -1.5, 1.5)
    w = np.exp(rng(93).uniform(np.log(0.5), np.log(2.0), size=len(p)))
    return p, n, a, x, w


@pytest.mark.parametrize("flip", [False, True])
def test_moved_coefficients_describe_the_same_surface(cloud, flip):
    """The coefficient map itself: surface points of Eq. BivariatePolynomial
    before and after the move coincide (checked on the patches, not through
    the oracle)."""
    p, n, a, _, _ = cloud
    M = orthogonal(94)
    n2, a2 = moved_coefficients(n, a, M, flip)
    s, t = synth.frame(n)
    s2, t2 = synth.frame(n2)
    g = rng(95)
    for _ in range(5):
        u, v = g.uniform(-0.3, 0.3, size=(2, len(p)))
        h = a[:, 0] + a[:, 2] * u + a[:, 1] * v + a[:, 3] * u * v + a[:, 5] * u * u + a[:, 4] * v * v
        y = (p + u[:, None] * s + v[:, None] * t + h[:, None] * n) @ M.T
        rel = y - p @ M.T
        u2, v2 = (rel * s2).sum(1), (rel * t2).sum(1)
        h2 = a2[:, 0] + a2[:, 2] * u2 + a2[:, 1] * v2 + a2[:, 3] * u2 * v2 + a2[:, 5] * u2 * u2 + a2[:, 4] * v2 * v2
        np.testing.assert_allclose((rel * n2).sum(1), h2, atol=1e-13)


@pytest.mark.parametrize("proper", [True, False])
@pytest.mark.parametrize("weighted", [False, True])
def test_isometry(oracle_mod, cloud, proper, weighted):
    p, n, a, x, w = cloud
    wt = w if weighted else None
    M = orthogonal(96 + proper, proper)
    tr = np.array([0.7, -1.9, 0.4])
    n2, a2 = moved_coefficients(n, a, M)
    c1 = oracle_mod.Cloud(p, n, a, weights=wt)
    c2 = oracle_mod.Cloud(p @ M.T + tr, n2, a2, weights=wt)
    x2 = x @ M.T + tr
    for C in (8.0, 64.0):
        np.testing.assert_allclose(c2.phi(x2, C=C), c1.phi(x, C=C), atol=1e-9)
        np.testing.assert_allclose(c2.lse(x2, C=C), c1.lse(x, C=C), atol=1e-9)
    np.testing.assert_allclose(c2.phi(x2, mode=oracle_mod.FIXED, lam=40.0),
                               c1.phi(x, mode=oracle_mod.FIXED, lam=40.0), atol=1e-9)
    f1, g1 = c1.grad_x(x)
    f2, g2 = c2.grad_x(x2)
    np.testing.assert_allclose(f2, f1, atol=1e-9)
    np.testing.assert_allclose(g2, g1 @ M.T, atol=1e-8)
    np.testing.assert_allclose(c2.laplacian(x2[:40])[2], c1.laplacian(x[:40])[2], atol=1e-6)


@pytest.mark.parametrize("c", [0.01, 3.0, 250.0])
def test_uniform_scale(oracle_mod, cloud, c):
    p, n, a, x, w = cloud
    a2 = a * np.array([c, 1.0, 1.0, 1.0 / c, 1.0 / c, 1.0 / c])
    c1 = oracle_mod.Cloud(p, n, a, weights=w)
    c2 = oracle_mod.Cloud(c * p, n, a2, weights=w)
    np.testing.assert_allclose(c2.phi(c * x), c * c1.phi(x), rtol=1e-10, atol=1e-12 * c)
    np.testing.assert_allclose(c2.lse(c * x), c * c1.lse(x), rtol=1e-10, atol=1e-12 * c)
    np.testing.assert_allclose(c2.phi(c * x, mode=oracle_mod.FIXED, lam=40.0 / c),
                               c * c1.phi(x, mode=oracle_mod.FIXED, lam=40.0), rtol=1e-10, atol=1e-12 * c)
    _, g1 = c1.grad_x(x)
    _, g2 = c2.grad_x(c * x)
    np.testing.assert_allclose(g2, g1, atol=1e-8)
    np.testing.assert_allclose(c2.laplacian(c * x[:40])[2], c1.laplacian(x[:40])[2] / c, rtol=1e-6, atol=1e-9 / c)


def test_every_point_twice(oracle_mod, cloud):
    p, n, a, x, _ = cloud
    C = 16.0
    c1 = oracle_mod.Cloud(p, n, a)
    c2 = oracle_mod.Cloud(np.concatenate([p, p]), np.concatenate([n, n]), np.concatenate([a, a]))
    np.testing.assert_allclose(c2.phi(x, C=C), c1.phi(x, C=C), atol=1e-12)
    dmax = np.linalg.norm(x[:, None, :] - p[None], axis=2).max(1)
    np.testing.assert_allclose(c2.lse(x, C=C), c1.lse(x, C=C) - np.log(2.0) * dmax / (2.0 * C), atol=1e-12)
    np.testing.assert_allclose(c2.grad_x(x, C=C)[1], c1.grad_x(x, C=C)[1], atol=1e-10)


def test_point_order(oracle_mod, cloud):
    p, n, a, x, w = cloud
    perm = rng(97).permutation(len(p))
    c1 = oracle_mod.Cloud(p, n, a, weights=w)
    c2 = oracle_mod.Cloud(p[perm], n[perm], a[perm], weights=w[perm])
    np.testing.assert_allclose(c2.phi(x), c1.phi(x), atol=1e-12)
    np.testing.assert_allclose(c2.lse(x), c1.lse(x), atol=1e-12)


def test_every_normal_flipped(oracle_mod, cloud):
    p, n, a, x, w = cloud
    n2, a2 = moved_coefficients(n, a, np.eye(3), flip=True)
    c1 = oracle_mod.Cloud(p, n, a, weights=w)
    c2 = oracle_mod.Cloud(p, n2, a2, weights=w)
    np.testing.assert_allclose(c2.phi(x), -c1.phi(x), atol=1e-9)
    np.testing.assert_allclose(c2.lse(x), c1.lse(x), atol=1e-12)
    _, g1 = c1.grad_x(x)
    _, g2 = c2.grad_x(x)
    np.testing.assert_allclose(g2, -g1, atol=1e-8)
    np.testing.assert_allclose(c2.laplacian(x[:40])[2], -c1.laplacian(x[:40])[2], atol=1e-6)
    lam = 12.0
    np.testing.assert_allclose(c2.phi_radius(x, lam), -c1.phi_radius(x, lam), atol=1e-9)


@pytest.mark.parametrize("proper", [True, False])
def test_radius_limited_isometry(oracle_mod, cloud, proper):
    p, n, a, x, w = cloud
    M = orthogonal(98 + proper, proper)
    tr = np.array([-3.0, 0.25, 1.5])
    n2, a2 = moved_coefficients(n, a, M)
    c1 = oracle_mod.Cloud(p, n, a, weights=w)
    c2 = oracle_mod.Cloud(p @ M.T + tr, n2, a2, weights=w)
    x2 = x @ M.T + tr
    for lam, reval in ((12.0, None), (300.0, 0.05)):       # sums within R_eval, and the 32-nearest fallback
        r1, u1 = c1.phi_radius(x, lam, reval, used=True)
        r2, u2 = c2.phi_radius(x2, lam, reval, used=True)
        np.testing.assert_array_equal(u2, u1)
        np.testing.assert_allclose(r2, r1, atol=1e-9)
        np.testing.assert_allclose(c2.phi_radius(x2, lam, reval, lse=True), c1.phi_radius(x, lam, reval, lse=True),
                                   atol=1e-9)
    assert (u1 < 0).any() and (u1 > 0).any()
    np.testing.assert_allclose(oracle_mod.knn_mean_distance(p @ M.T + tr, 16), oracle_mod.knn_mean_distance(p, 16),
                               rtol=1e-12)


@pytest.mark.parametrize("c", [0.05, 40.0])
def test_radius_limited_scale(oracle_mod, cloud, c):
    p, n, a, x, w = cloud
    a2 = a * np.array([c, 1.0, 1.0, 1.0 / c, 1.0 / c, 1.0 / c])
    c1 = oracle_mod.Cloud(p, n, a, weights=w)
    c2 = oracle_mod.Cloud(c * p, n, a2, weights=w)
    for lam, reval in ((12.0, None), (300.0, 0.05)):
        r1, u1 = c1.phi_radius(x, lam, reval, used=True)
        r2, u2 = c2.phi_radius(c * x, lam / c, None if reval is None else reval * c, used=True)
        np.testing.assert_array_equal(u2, u1)
        np.testing.assert_allclose(r2, c * r1, rtol=1e-9, atol=1e-12 * c)
    np.testing.assert_allclose(oracle_mod.knn_mean_distance(c * p, 16), c * oracle_mod.knn_mean_distance(p, 16),
                               rtol=1e-12)
