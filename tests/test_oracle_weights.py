"""Pins of the oracle's per-point weights and its log-sum-exp distance.

Weights A_i discretise the surface integral of Eq.
SelfNormalizedConvolutionalDistanceFormula (Eq. BasicFormulaShifted leaves
them out: all A_i = 1).  The log-sum-exp distance is Eq.
ConvolutionalDistanceFormula with h = 1:
d~(x) = -(1/lambda) log sum_i A_i exp(-lambda |x - p_i|).

Pinned against facts outside the oracle's own code:
- integer weights are the same as repeating each point that many times
  (brute force, for phi, grad_x, the Laplacian, the parameter gradient,
  the radius-limited sum and the log-sum-exp distance);
- equal weights c leave every blend unchanged and shift d~ by -ln(c)/lambda;
- d~ of one point is |x - p| - ln(A)/lambda (closed form);
- d~ equals scipy.special.logsumexp with b = A (library routine);
- Laplace's method: d_min - ln(sum A)/lambda <= d~ <= d_min - ln(A_nearest)/lambda,
  and d~ -> d_min as lambda grows.
"""
import numpy as np
import pytest
from scipy.special import logsumexp

import oracle
import synth
from workloads import mixed_cloud


def small_cloud(n=60, seed=5):
    p, nrm, a = mixed_cloud(seed)
    rng = np.random.Generator(np.random.PCG64(seed))
    idx = rng.choice(len(p), size=n, replace=False)
    return p[idx], nrm[idx], a[idx]


def queries(m=40, seed=6, lo=-1.2, hi=1.2):
    return synth.uniform_queries(m, seed, lo, hi)


def test_integer_weights_equal_repeated_points():
    p, n, a = small_cloud()
    rng = np.random.Generator(np.random.PCG64(7))
    k = rng.integers(1, 4, size=len(p))
    rep = np.repeat(np.arange(len(p)), k)
    cw = oracle.Cloud(p, n, a, weights=k.astype(float))
    cd = oracle.Cloud(p[rep], n[rep], a[rep])
    x = queries()
    np.testing.assert_allclose(cw.phi(x), cd.phi(x), rtol=1e-11, atol=1e-12)
    np.testing.assert_allclose(cw.lse(x), cd.lse(x), rtol=1e-11, atol=1e-12)
    for mode, lam in ((oracle.GLOBAL, 0.0), (oracle.FIXED, 9.0)):
        pw, gw = cw.grad_x(x, mode=mode, lam=lam)
        pd, gd = cd.grad_x(x, mode=mode, lam=lam)
        np.testing.assert_allclose(pw, pd, rtol=1e-11, atol=1e-12)
        np.testing.assert_allclose(gw, gd, rtol=1e-9, atol=1e-10)
    _, gl, ll = cw.laplacian(x[:12])
    _, gdl, ldl = cd.laplacian(x[:12])
    np.testing.assert_allclose(gl, gdl, rtol=1e-9, atol=1e-10)
    np.testing.assert_allclose(ll, ldl, rtol=1e-8, atol=1e-9)
    # d (sum_q G_q phi_q) / d a_i: the weighted point carries the sum over its copies
    G = rng.normal(size=len(x))
    gpw = cw.grad_params(x, G)
    gpd = cd.grad_params(x, G)
    summed = np.zeros_like(gpw)
    np.add.at(summed, rep, gpd)
    np.testing.assert_allclose(gpw, summed, rtol=1e-9, atol=1e-11)
    # radius-limited: queries near the cloud, every one with points inside R_eval
    lam = 40.0
    xs = p[:20] + 0.02
    fw, uw = cw.phi_radius(xs, lam, used=True)
    fd, ud = cd.phi_radius(xs, lam, used=True)
    assert (uw > 0).all()
    np.testing.assert_allclose(fw, fd, rtol=1e-11, atol=1e-12)
    np.testing.assert_allclose(cw.phi_radius(xs, lam, lse=True), cd.phi_radius(xs, lam, lse=True),
                               rtol=1e-11, atol=1e-12)


@pytest.mark.parametrize("c", [1e-3, 0.37, 250.0])
def test_equal_weights(c):
    p, n, a = small_cloud(seed=8)
    x = queries(seed=9)
    c0 = oracle.Cloud(p, n, a)
    cw = oracle.Cloud(p, n, a, weights=np.full(len(p), c))
    np.testing.assert_allclose(cw.phi(x), c0.phi(x), rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose(cw.grad_x(x)[1], c0.grad_x(x)[1], rtol=1e-10, atol=1e-11)
    lam_x = c0.phi(x, stats=True)[1][:, 0]
    np.testing.assert_allclose(cw.lse(x), c0.lse(x) - np.log(c) / lam_x, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("A", [1.0, 0.2, 7.5])
def test_lse_single_point(A):
    p = np.array([[0.3, -0.2, 0.1]])
    n = np.array([[0.0, 0.0, 1.0]])
    a = np.array([[0.0, 0.0, 0.0, 0.0, -0.5, -0.5]])
    cl = oracle.Cloud(p, n, a, weights=[A])
    x = queries(25, 10)
    d = np.linalg.norm(x - p, axis=1)
    lam = 13.0
    np.testing.assert_allclose(cl.lse(x, mode=oracle.FIXED, lam=lam), d - np.log(A) / lam, rtol=1e-13, atol=1e-14)
    # GLOBAL: d_max = d, lambda_x = C / (d / 2)
    np.testing.assert_allclose(cl.lse(x), d - np.log(A) * d / (2 * 64.0), rtol=1e-13, atol=1e-14)


def test_lse_equals_logsumexp():
    p, n, a = small_cloud(seed=11)
    rng = np.random.Generator(np.random.PCG64(12))
    A = np.exp(rng.uniform(np.log(0.1), np.log(10.0), size=len(p)))
    cl = oracle.Cloud(p, n, a, weights=A)
    x = queries(seed=13)
    d = np.linalg.norm(x[:, None, :] - p[None], axis=2)
    for lam in (3.0, 40.0, 900.0):
        ref = -logsumexp(-lam * d, b=A[None, :], axis=1) / lam
        np.testing.assert_allclose(cl.lse(x, mode=oracle.FIXED, lam=lam), ref, rtol=1e-12, atol=1e-13)
    lam_x = oracle.Cloud(p, n, a).phi(x, stats=True)[1][:, 0]
    ref = -logsumexp(-lam_x[:, None] * d, b=A[None, :], axis=1) / lam_x
    np.testing.assert_allclose(cl.lse(x), ref, rtol=1e-12, atol=1e-13)


def test_lse_laplace_bounds_and_limit():
    p, n, a = small_cloud(seed=14)
    rng = np.random.Generator(np.random.PCG64(15))
    A = rng.uniform(0.5, 2.0, size=len(p))
    cl = oracle.Cloud(p, n, a, weights=A)
    x = queries(seed=16)
    d = np.linalg.norm(x[:, None, :] - p[None], axis=2)
    dmin = d.min(1)
    Anear = A[d.argmin(1)]
    prev = None
    for lam in (10.0, 100.0, 1e3, 1e4):
        v = cl.lse(x, mode=oracle.FIXED, lam=lam)
        assert (v >= dmin - np.log(A.sum()) / lam - 1e-12).all()
        assert (v <= dmin - np.log(Anear) / lam + 1e-12).all()
        gap = np.abs(v - dmin).max()
        if prev is not None:
            assert gap < prev
        prev = gap
    assert prev < 1e-3


def test_radius_lse_brute_force():
    p, n, a = small_cloud(seed=17)
    rng = np.random.Generator(np.random.PCG64(18))
    A = rng.uniform(0.5, 2.0, size=len(p))
    cl = oracle.Cloud(p, n, a, weights=A)
    lam = 30.0
    reval = 2 * 64.0 / lam
    x = np.concatenate([p[:10] + 0.01, np.array([[30.0, 0.0, 0.0]])])   # the last one has no point inside R_eval
    got, used = cl.phi_radius(x, lam, lse=True, used=True)
    d = np.linalg.norm(x[:, None, :] - p[None], axis=2)
    for j in range(len(x)):
        inside = d[j] <= reval
        sel = inside if inside.any() else np.argsort(d[j], kind="stable")[:32]
        ref = -logsumexp(-lam * d[j][sel], b=A[sel]) / lam
        assert got[j] == pytest.approx(ref, rel=1e-12, abs=1e-12)
    assert used[-1] == -32 and (used[:-1] > 0).all()


@pytest.mark.parametrize("bad", [0.0, -1.0, np.nan, np.inf])
def test_invalid_weights_rejected(bad):
    p, n, a = small_cloud(10, seed=19)
    w = np.ones(len(p))
    w[3] = bad
    with pytest.raises(ValueError):
        oracle.Cloud(p, n, a, weights=w)


@pytest.mark.parametrize("A", [1.0, 0.2, 7.5])
def test_lse_gradient_single_point(A):
    """One point: grad d~ = (x - p)/|x - p| for a fixed lambda, and
    (1 - ln(A) / (2C)) (x - p)/|x - p| for lambda_x = 2C/|x - p|."""
    p = np.array([[0.3, -0.2, 0.1]])
    n = np.array([[0.0, 0.0, 1.0]])
    a = np.array([[0.0, 0.0, 0.0, 0.0, -0.5, -0.5]])
    cl = oracle.Cloud(p, n, a, weights=[A])
    x = queries(25, 20)
    u = (x - p) / np.linalg.norm(x - p, axis=1, keepdims=True)
    _, g = cl.lse_grad(x, mode=oracle.FIXED, lam=13.0)
    np.testing.assert_allclose(g, u, atol=1e-12)
    _, g = cl.lse_grad(x)
    np.testing.assert_allclose(g, (1 - np.log(A) / (2 * 64.0)) * u, atol=1e-12)


@pytest.mark.parametrize("mode,lam", [(oracle.GLOBAL, 0.0), (oracle.FIXED, 25.0)])
def test_lse_gradient_finite_differences(mode, lam):
    """Central differences of d~ (h = 1e-4 and h / 2, Richardson) on a
    weighted mixed cloud, lambda_x(x) included for GLOBAL."""
    p, n, a = small_cloud(seed=21)
    rng = np.random.Generator(np.random.PCG64(22))
    A = rng.uniform(0.5, 2.0, size=len(p))
    cl = oracle.Cloud(p, n, a, weights=A)
    x = queries(30, 23)
    v, g = cl.lse_grad(x, mode=mode, lam=lam)
    np.testing.assert_allclose(v, cl.lse(x, mode=mode, lam=lam), rtol=1e-14, atol=1e-14)
    fd = np.empty_like(g)
    for k in range(3):
        e = np.zeros(3)
        e[k] = 1.0
        est = []
        for h in (1e-4, 5e-5):
            est.append((cl.lse(x + h * e, mode=mode, lam=lam) - cl.lse(x - h * e, mode=mode, lam=lam)) / (2 * h))
        fd[:, k] = (4 * est[1] - est[0]) / 3
    np.testing.assert_allclose(g, fd, rtol=1e-6, atol=1e-7)
