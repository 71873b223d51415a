"""Pins of the FP64 oracle to facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: closed forms,
brute-force geometry, limits of the blend, finite differences, or the textbook
definition of normal curvature.  A dropped term, a wrong sign, a swapped index
or a transposed operand anywhere in the fit, the torus SDF or the blend fails
at least one of them (the comment on each test names what it guards).
"""
import math
import os

import numpy as np
import pytest

import synth

HERE = os.path.dirname(os.path.abspath(__file__))


def rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


# --------------------------------------------------------------------------
# Frame convention (Duff et al. 2017): orthonormal, right-handed, fixed values
# --------------------------------------------------------------------------
def test_frame_convention(oracle_mod):
    """Guards the (s, t) convention the coefficients are expressed in."""
    for n in [np.array([0.0, 0.0, 1.0]), np.array([0.0, 0.0, -1.0]),
              *list(synth._unit(rng(1).normal(size=(20, 3))))]:
        s, t = oracle_mod.frame(n)
        M = np.stack([s, t, n])
        np.testing.assert_allclose(M @ M.T, np.eye(3), atol=1e-14)
        np.testing.assert_allclose(np.cross(s, t), n, atol=1e-14)
        s2, t2 = synth.frame(n[None])
        np.testing.assert_allclose(s, s2[0], atol=1e-15)
        np.testing.assert_allclose(t, t2[0], atol=1e-15)
    s, t = oracle_mod.frame([0.0, 0.0, 1.0])
    np.testing.assert_array_equal(s, [1.0, 0.0, 0.0])
    np.testing.assert_array_equal(t, [0.0, 1.0, 0.0])
    s, t = oracle_mod.frame([0.0, 0.0, -1.0])
    np.testing.assert_array_equal(s, [1.0, 0.0, 0.0])
    np.testing.assert_array_equal(t, [0.0, -1.0, 0.0])


# --------------------------------------------------------------------------
# Eq. SingleTorusSDF: hand-worked closed forms and brute force
# --------------------------------------------------------------------------
def test_torus_sdf_golden(oracle_mod):
    """Hand-derived values (axis, centre, equatorial plane, centre circle)."""
    rows = np.loadtxt(os.path.join(HERE, "golden", "torus_closed_forms.txt"))
    for r in rows:
        got = oracle_mod.torus_sdf(r[0:3], r[3:6], r[6], r[7], r[8:11][None])[0]
        assert abs(got - r[11]) < 1e-13, (r, got)


def _brute_torus(c, u, R, r, x):
    """Signed distance to a ring torus by brute force: distance to the centre
    circle from 20000 samples refined by golden-section search, minus r."""
    b1, b2 = synth.frame(u[None])
    b1, b2 = b1[0], b2[0]
    ang = np.linspace(0.0, 2 * math.pi, 20000, endpoint=False)
    circ = c + R * (np.cos(ang)[:, None] * b1 + np.sin(ang)[:, None] * b2)
    out = []
    for xi in x:
        d = np.linalg.norm(circ - xi, axis=1)
        k = int(np.argmin(d))
        lo, hi = ang[k] - 2e-3, ang[k] + 2e-3
        f = lambda a: np.linalg.norm(c + R * (math.cos(a) * b1 + math.sin(a) * b2) - xi)
        g = (math.sqrt(5) - 1) / 2
        for _ in range(80):
            m1, m2 = hi - g * (hi - lo), lo + g * (hi - lo)
            if f(m1) < f(m2):
                hi = m2
            else:
                lo = m1
        out.append(f(0.5 * (lo + hi)) - r)
    return np.array(out)


def test_torus_sdf_bruteforce(oracle_mod):
    """Eq. SingleTorusSDF against brute-force distance to the torus's centre
    circle (ring tori with random pose)."""
    g = rng(7)
    for trial in range(4):
        c = g.normal(size=3)
        u = synth._unit(g.normal(size=(1, 3)))[0]
        R = 0.5 + g.random()
        r = 0.1 + 0.3 * g.random()
        x = c + g.normal(size=(40, 3)) * 1.5
        got = oracle_mod.torus_sdf(c, u, R, r, x)
        ref = _brute_torus(c, u, R, r, x)
        np.testing.assert_allclose(got, ref, atol=1e-9)


# --------------------------------------------------------------------------
# Fit (Sec. 4.1, App. C): normal curvatures by the textbook definition
# --------------------------------------------------------------------------
def _random_coeffs(g, m, tilt=0.4, curv=2.0):
    a = np.zeros((m, 6))
    a[:, 0] = g.normal(size=m) * 0.05
    a[:, 1:3] = g.normal(size=(m, 2)) * tilt
    a[:, 3:6] = g.normal(size=(m, 3)) * curv
    return a


def _poly_surface(p, n, a, s, t):
    """Q*(s, t) = p + s s_i + t t_i + Q(s, t) n_i  (Eq. BivariatePolynomial)."""
    fs, ft = synth.frame(n[None])
    fs, ft = fs[0], ft[0]
    Q = a[0] + a[2] * s + a[1] * t + a[3] * s * t + a[5] * s * s + a[4] * t * t
    return p + np.outer(s, fs) + np.outer(t, ft) + np.outer(Q, n)


def test_curvatures_are_extremal_normal_curvatures(oracle_mod):
    """kappa_+- and v_min against the extremal normal curvatures of Q*,
    measured by finite differences of surface curves through Q*(0,0)
    (Meusnier: kappa_n = <c''(0), n*> / |c'(0)|^2).  Guards A, H, K, the
    kappa_min/kappa_max selection, w_+-, and the tilt terms of n*."""
    g = rng(11)
    for a in _random_coeffs(g, 12):
        p = g.normal(size=3)
        n = synth._unit(g.normal(size=(1, 3)))[0]
        fit = oracle_mod.fit_record(p, n, a)
        th = np.linspace(0.0, math.pi, 3601)
        h = 1e-4
        c0 = _poly_surface(p, n, a, np.zeros(1), np.zeros(1))[0]
        kn, tang = [], []
        for ang in th:
            al, be = math.cos(ang), math.sin(ang)
            cp = _poly_surface(p, n, a, np.array([h * al]), np.array([h * be]))[0]
            cm = _poly_surface(p, n, a, np.array([-h * al]), np.array([-h * be]))[0]
            d1 = (cp - cm) / (2 * h)
            d2 = (cp - 2 * c0 + cm) / (h * h)
            nstar = np.cross(*[(_poly_surface(p, n, a, np.array([e[0]]), np.array([e[1]]))[0]
                                - _poly_surface(p, n, a, np.array([-e[0]]), np.array([-e[1]]))[0]) / (2 * h)
                               for e in ([h, 0.0], [0.0, h])])
            nstar /= np.linalg.norm(nstar)
            kn.append(np.dot(d2, nstar) / np.dot(d1, d1))
            tang.append(d1 / np.linalg.norm(d1))
        kn = np.array(kn)
        kmin_num, kmax_num = kn.min(), kn.max()
        assert abs(fit["kplus"] - kmax_num) < 1e-5 * (1 + abs(kmax_num))
        assert abs(fit["kminus"] - kmin_num) < 1e-5 * (1 + abs(kmin_num))
        np.testing.assert_allclose(fit["nstar"], nstar, atol=1e-7)
        # v_min is the tangent direction whose normal curvature is kappa_min
        j = int(np.argmin(np.abs(kn - fit["kmin"])))
        if abs(fit["kplus"] - fit["kminus"]) > 1e-2:
            assert abs(abs(np.dot(tang[j], fit["vmin"])) - 1.0) < 1e-4
        assert abs(fit["kmin"]) <= abs(fit["kmax"])


def test_untilted_principal_directions_degenerate_row(oracle_mod):
    """With a11 = a10 = a01 = 0 the printed w_+- vanishes for kappa = 2 a20;
    the principal directions must still be the frame axes (reading X4)."""
    n = np.array([0.0, 0.0, 1.0])
    for a20, a02 in [(-0.2, -1.5), (-1.5, -0.2), (0.3, -2.0), (-0.3, 2.0)]:
        fit = oracle_mod.fit_record(np.zeros(3), n, [0, 0, 0, 0, a02, a20])
        vmin_expected = np.array([1.0, 0.0, 0.0]) if abs(a20) < abs(a02) else np.array([0.0, 1.0, 0.0])
        assert abs(abs(np.dot(fit["vmin"], vmin_expected)) - 1.0) < 1e-14
        assert abs(fit["kmin"] - 2 * (a20 if abs(a20) < abs(a02) else a02)) < 1e-14


def test_osculation_order(oracle_mod):
    """The fitted torus touches Q* to second order (Sec. 4.1): on a circle of
    radius eps around Q*(0,0), max |g_i| shrinks about 8x when eps halves.
    Guards every fit quantity at once, including tilt and the saddle centre."""
    g = rng(13)
    coeffs = _random_coeffs(g, 16)
    coeffs[:4, 1:3] = 0.0                     # untilted cases as well
    coeffs[4:8, 3] = 0.0
    for a in coeffs:
        p = g.normal(size=3)
        n = synth._unit(g.normal(size=(1, 3)))[0]
        cl = oracle_mod.Cloud(p[None], n[None], a[None])
        ang = np.linspace(0, 2 * math.pi, 64, endpoint=False)
        m = []
        for eps in (4e-3, 2e-3):
            pts = _poly_surface(p, n, a, eps * np.cos(ang), eps * np.sin(ang))
            m.append(np.abs(cl.g(0, pts)).max())
        assert m[0] / m[1] > 7.0, (a, m)
        assert m[0] < 50 * 4e-3 ** 3 * (1 + np.abs(a).max()) ** 4


# --------------------------------------------------------------------------
# Exact reproduction (sphere / plane / cylinder / ring-torus equators)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("C", [1.0, 8.0, 64.0, 87.0, 400.0])
def test_sphere_exact(oracle_mod, C):
    """a20 = a02 = -1/2 makes every torus the unit sphere (R = 0, r = 1, c = 0):
    phi(x) = |x| - 1 for every x and every lambda (pins the sign convention
    with the paper's sphere initialisation)."""
    p, n, a = synth.sphere_fibonacci(256, 3)
    x = synth.uniform_queries(300, 5)
    ref = np.linalg.norm(x, axis=1) - 1.0
    cl = oracle_mod.Cloud(p, n, a)
    np.testing.assert_allclose(cl.phi(x, C=C), ref, atol=1e-12)
    np.testing.assert_allclose(cl.phi(x, mode=oracle_mod.FIXED, lam=C), ref, atol=1e-12)
    # concave reading: inward normals, a20 = a02 = +1/2 -> phi = 1 - |x|
    cl2 = oracle_mod.Cloud(p, -n, -a)
    np.testing.assert_allclose(cl2.phi(x, C=C), -ref, atol=1e-12)


def test_plane_exact(oracle_mod):
    """kappa_min = kappa_max = 0 (reading X5): phi(x) = z for a z = 0 patch."""
    p, n, a = synth.plane_patch(200, 9)
    x = synth.uniform_queries(200, 10)
    cl = oracle_mod.Cloud(p, n, a)
    np.testing.assert_allclose(cl.phi(x), x[:, 2], atol=1e-13)
    cl2 = oracle_mod.Cloud(p, -n, a)
    np.testing.assert_allclose(cl2.phi(x), -x[:, 2], atol=1e-13)


@pytest.mark.parametrize("inward", [False, True])
def test_cylinder_exact(oracle_mod, inward):
    """kappa_min = 0, kappa_max = -+1/r (reading X5): phi = +-(rho - r)."""
    p, n, a = synth.cylinder_cloud(300, 12, radius=0.5, inward=inward)
    x = synth.uniform_queries(200, 13)
    rho = np.linalg.norm(x[:, :2], axis=1)
    ref = (rho - 0.5) * (-1.0 if inward else 1.0)
    cl = oracle_mod.Cloud(p, n, a)
    np.testing.assert_allclose(cl.phi(x), ref, atol=1e-12)


@pytest.mark.parametrize("flip", [False, True])
def test_ring_torus_equators_exact(oracle_mod, flip):
    """Points on the outer (convex) and inner (saddle) equators of a ring torus
    with analytic curvatures: every fitted torus IS the ring torus, so phi is
    its exact SDF.  The inner equator pins the saddle centre (reading X1) and
    the sign table; flipped normals pin the other saddle branch."""
    R, r = 1.0, 0.35
    psi = np.linspace(0, 2 * math.pi, 24, endpoint=False)
    theta = np.concatenate([np.zeros(24), np.full(24, math.pi)])
    p, n, a = synth.ring_torus(48, 0, R=R, r=r, noise=0.0, jitter_deg=0.0,
                               theta=theta, psi=np.concatenate([psi, psi + 0.1]), inward=flip)
    x = synth.uniform_queries(300, 14, -1.6, 1.6)
    ref = np.sqrt((np.linalg.norm(x[:, :2], axis=1) - R) ** 2 + x[:, 2] ** 2) - r
    cl = oracle_mod.Cloud(p, n, a)
    np.testing.assert_allclose(cl.phi(x), -ref if flip else ref, atol=1e-12)
    for i in (0, 30):
        fit = oracle_mod.fit_record(p[i], n[i], a[i])
        np.testing.assert_allclose(fit["c"], 0.0, atol=1e-14)
        assert abs(fit["R"] - R) < 1e-14 and abs(fit["r"] - r) < 1e-14
        assert abs(abs(fit["u"][2]) - 1.0) < 1e-14


# --------------------------------------------------------------------------
# The blend (Eqs. BasicFormulaShifted, RelationshipBetweenLambdaAndRadius)
# --------------------------------------------------------------------------
def _torus_cloud(m, seed, noise=0.01, jitter=5.0):
    return synth.ring_torus(m, seed, noise=noise, jitter_deg=jitter)


def test_single_point_is_its_torus(oracle_mod):
    """N = 1: phi = g_1 for every lambda (including d_max = 0, reading X9)."""
    p, n, a = _torus_cloud(5, 21)
    cl = oracle_mod.Cloud(p[:1], n[:1], a[:1])
    x = np.concatenate([synth.uniform_queries(50, 22), p[:1]])
    np.testing.assert_allclose(cl.phi(x), cl.g(0, x), atol=1e-14)


def test_lambda_zero_is_mean(oracle_mod):
    """lambda -> 0: phi = mean_i g_i(x)."""
    p, n, a = _torus_cloud(40, 23)
    cl = oracle_mod.Cloud(p, n, a)
    x = synth.uniform_queries(30, 24)
    ref = np.mean([cl.g(i, x) for i in range(40)], axis=0)
    np.testing.assert_allclose(cl.phi(x, mode=oracle_mod.FIXED, lam=0.0), ref, atol=1e-13)
    np.testing.assert_allclose(cl.phi(x, C=1e-9), ref, atol=1e-9)


def test_lambda_infinity_is_nearest_torus(oracle_mod):
    """lambda -> infinity: phi = g of the nearest point (brute-force NN), on
    queries whose nearest / runner-up gap makes the runner-up weight < 1e-30."""
    p, n, a = _torus_cloud(60, 25)
    cl = oracle_mod.Cloud(p, n, a)
    x = synth.uniform_queries(400, 26)
    d = np.linalg.norm(x[:, None, :] - p[None], axis=2)
    srt = np.sort(d, axis=1)
    lam = 2e4
    keep = (srt[:, 1] - srt[:, 0]) * lam > 70.0
    assert keep.sum() > 200
    x, near = x[keep], np.argmin(d[keep], axis=1)
    ref = np.array([cl.g(int(i), xi[None])[0] for i, xi in zip(near, x)])
    np.testing.assert_allclose(cl.phi(x, mode=oracle_mod.FIXED, lam=lam), ref, atol=1e-12)


def test_shift_invariance(oracle_mod):
    """The exponent shift (sigma_x in the paper, d_min alternatively) cancels."""
    p, n, a = _torus_cloud(300, 27)
    cl = oracle_mod.Cloud(p, n, a)
    x = synth.uniform_queries(100, 28)
    a1 = cl.phi(x, shift=oracle_mod.SHIFT_SIGMA)
    a2 = cl.phi(x, shift=oracle_mod.SHIFT_DMIN)
    np.testing.assert_allclose(a1, a2, atol=1e-12)


def test_lambda_rule_two_points(oracle_mod):
    """lambda_x = C / sigma_x with sigma_x = d_max / 2: with two points the
    blend is g_1 + (g_2 - g_1) w_2 / (w_1 + w_2), so the weight ratio recovered
    from phi must be exp(-(2C / d_max)(d_2 - d_1)); and the farthest point's
    shifted exponent equals -C exactly."""
    p, n, a = _torus_cloud(2, 29)
    cl = oracle_mod.Cloud(p, n, a)
    x = synth.uniform_queries(50, 30)
    C = 3.0
    phi, st = cl.phi(x, C=C, stats=True)
    g1, g2 = cl.g(0, x), cl.g(1, x)
    d = np.linalg.norm(x[:, None, :] - p[None], axis=2)
    ratio = (phi - g1) / (g2 - phi)                      # = w_2 / w_1
    dmax = d.max(1)
    np.testing.assert_allclose(np.log(ratio), -(2 * C / dmax) * (d[:, 1] - d[:, 0]), atol=1e-8)
    np.testing.assert_allclose(st[:, 0] * (dmax - dmax / 2), C, rtol=1e-14)
    np.testing.assert_allclose(st[:, 1], dmax, rtol=1e-15)


def test_sign_on_clean_clouds(oracle_mod):
    """Method property on clean clouds: sgn phi = sgn(F(x) - 1) where the query
    is farther than 5 sample spacings from the surface."""
    pts, nrm, a = synth.ring_torus(3000, 31, noise=0.0, jitter_deg=0.0)
    cl = oracle_mod.Cloud(pts, nrm, a)
    x = synth.uniform_queries(600, 32, -1.6, 1.6)
    sd = np.sqrt((np.linalg.norm(x[:, :2], axis=1) - 1.0) ** 2 + x[:, 2] ** 2) - 0.35
    spacing = math.sqrt(4 * math.pi ** 2 * 0.35 / 3000)
    far = np.abs(sd) > 5 * spacing
    phi = cl.phi(x[far])
    assert np.all(np.sign(phi) == np.sign(sd[far]))
    pts, nrm, a = synth.ellipsoid(3000, 33, perturb=0.0)
    cl = oracle_mod.Cloud(pts, nrm, a)
    F = np.sum((x / np.array([1.0, 0.6, 0.4])) ** 2, axis=1) - 1.0
    far = np.abs(F) > 0.15
    assert np.all(np.sign(cl.phi(x[far])) == np.sign(F[far]))


# --------------------------------------------------------------------------
# Gradients: central finite differences with Richardson behaviour
# --------------------------------------------------------------------------
def _mixed_cloud(m, seed):
    """Torus-sampled points with random coefficients (both curvature signs,
    saddles, tilt, shift) so that every sign(T) branch carries weight."""
    p, n, _ = _torus_cloud(m, seed)
    a = _random_coeffs(rng(seed + 1), m, tilt=0.3, curv=1.5)
    signs = {oracle_fit_sign(p[i], n[i], a[i]) for i in range(m)}
    assert signs == {-1.0, 1.0}
    return p, n, a


def oracle_fit_sign(p, n, a):
    import oracle
    return oracle.fit_record(p, n, a)["sign"]


def test_grad_x_matches_finite_differences(oracle_mod):
    """d phi / d x including the x-dependence of lambda_x (App. D plus the
    lambda term): central differences at h and h/2 shrink ~4x and the
    Richardson extrapolation matches to 1e-8."""
    p, n, a = _mixed_cloud(200, 35)
    cl = oracle_mod.Cloud(p, n, a)
    x = synth.uniform_queries(60, 36)
    # lambda_x has a kink where the farthest point changes: keep queries whose
    # two farthest points are separated by more than the stencil
    dd = np.sort(np.linalg.norm(x[:, None, :] - p[None], axis=2), axis=1)
    x = x[(dd[:, -1] - dd[:, -2]) > 4e-3][:40]
    phi, g = cl.grad_x(x)
    np.testing.assert_allclose(phi, cl.phi(x), atol=1e-13)
    for h in (1e-3,):
        fd = np.zeros_like(g)
        fd2 = np.zeros_like(g)
        for k in range(3):
            e = np.zeros(3)
            e[k] = 1.0
            fd[:, k] = (cl.phi(x + h * e) - cl.phi(x - h * e)) / (2 * h)
            fd2[:, k] = (cl.phi(x + h / 2 * e) - cl.phi(x - h / 2 * e)) / h
        rich = (4 * fd2 - fd) / 3
        err1, err2 = np.abs(fd - g), np.abs(fd2 - g)
        big = err1 > 1e-9
        assert np.median(err1[big] / np.maximum(err2[big], 1e-300)) > 3.0
        np.testing.assert_allclose(rich, g, atol=1e-7)
    # the lambda term matters: the frozen-lambda gradient differs
    assert np.abs(g).max() > 0.1


def test_grad_params_matches_finite_differences(oracle_mod):
    """d(sum_q G_q phi_q)/d a_i through the fit: central differences on
    rebuilt clouds, Richardson-extrapolated, for 24 sampled entries."""
    p, n, a = _mixed_cloud(60, 37)
    x = synth.uniform_queries(30, 38)
    G = rng(39).normal(size=30)
    cl = oracle_mod.Cloud(p, n, a)
    ga = cl.grad_params(x, G)
    pick = rng(40).integers(0, 60, size=24)
    comp = rng(41).integers(0, 6, size=24)

    def loss(aa):
        return float(np.dot(G, oracle_mod.Cloud(p, n, aa).phi(x)))

    for i, k in zip(pick, comp):
        vals = []
        for h in (1e-4, 5e-5):
            ap, am = a.copy(), a.copy()
            ap[i, k] += h
            am[i, k] -= h
            vals.append((loss(ap) - loss(am)) / (2 * h))
        rich = (4 * vals[1] - vals[0]) / 3
        assert abs(rich - ga[i, k]) < 1e-7 * (1 + abs(ga[i, k])), (i, k, rich, ga[i, k])


# --------------------------------------------------------------------------
# Sphere tracing on an exact-SDF cloud
# --------------------------------------------------------------------------
def test_trace_sphere_closed_form(oracle_mod):
    """On the sphere cloud phi is exact, so tracing converges to the analytic
    ray-sphere intersection (to within eps); missing rays miss."""
    p, n, a = synth.sphere_fibonacci(128, 2)
    cl = oracle_mod.Cloud(p, n, a)
    org, dirs = synth.camera_rays(24, 24, 3, dist=3.0, fov_deg=60.0)
    t, steps = cl.trace(org, dirs, max_steps=200, eps=1e-9, t_max=8.0)
    b = np.sum(org * dirs, 1)
    c = np.sum(org * org, 1) - 1.0
    disc = b * b - c
    hit = disc > 1e-6
    t_ref = -b - np.sqrt(np.where(hit, disc, 0.0))
    assert np.all(t[~hit] < 0)
    np.testing.assert_allclose(t[hit], t_ref[hit], atol=2e-9)
    assert steps.max() <= 200


def test_trace_offset_steps_and_limits(oracle_mod):
    """Sphere tracing of phi = c on the exact sphere cloud (Sec. 6): rays hit
    the sphere of radius 1 + c; a ray aimed at the centre reaches it in one
    step, so it stops at the second evaluation; a ray leaving the cloud stops
    once t passes t_max; with too few steps a ray reports a miss after
    exactly max_steps evaluations."""
    p, n, a = synth.sphere_fibonacci(128, 2)
    cl = oracle_mod.Cloud(p, n, a)
    org, dirs = synth.camera_rays(16, 16, 4, dist=3.0, fov_deg=60.0)
    for c in (-0.3, 0.2):
        t, _ = cl.trace(org, dirs, max_steps=300, eps=1e-9, t_max=8.0, offset=c)
        b = np.sum(org * dirs, 1)
        disc = b * b - (np.sum(org * org, 1) - (1.0 + c) ** 2)
        hit, miss = disc > 1e-2, disc < -1e-2      # near-tangent rays converge too slowly to compare
        assert hit.sum() > 20 and miss.sum() > 20
        # tracing stops once phi - c < eps; the ray then still has eps / cos(incidence) to go,
        # cos(incidence) = sqrt(disc) / (1 + c)
        tol = 2e-9 * (1.0 + c) / np.sqrt(np.where(hit, disc, 1.0))
        t_ref = -b - np.sqrt(np.where(hit, disc, 0.0))
        assert np.all(np.abs(t[hit] - t_ref[hit]) <= tol[hit])
        assert np.all(t[hit] <= t_ref[hit] + 1e-12)  # from outside, never past the surface
        assert np.all(t[miss] < 0)
    o = np.array([[0.0, 0.0, 3.0], [0.0, 0.0, 3.0], [0.0, 0.0, 3.0]])
    d = np.array([[0.0, 0.0, -1.0], [0.0, 0.0, 1.0], [0.0, 0.0, -1.0]])
    t, steps = cl.trace(o[:1], d[:1], max_steps=10, eps=1e-9, t_max=8.0, offset=0.25)
    np.testing.assert_allclose(t, [3.0 - 1.25], atol=1e-12)
    assert steps[0] == 2
    t, steps = cl.trace(o[1:2], d[1:2], max_steps=100, eps=1e-9, t_max=8.0)
    assert t[0] < 0 and steps[0] == 3          # phi = 2 + t: t = 0 -> 2 -> 6 -> 14 > t_max after 3 evaluations
    # a ray passing 0.95 from the centre hits, but slowly near the tangent
    sa = 0.95 / 3.0
    g = np.array([[sa, 0.0, -np.sqrt(1.0 - sa * sa)]])
    t, steps = cl.trace(o[2:], g, max_steps=3, eps=1e-9, t_max=8.0)
    assert t[0] < 0 and steps[0] == 3
    t, steps = cl.trace(o[2:], g, max_steps=300, eps=1e-9, t_max=8.0)
    assert t[0] > 0 and 3 < steps[0] < 300
