"""The seeded input generators (synth/) against the analytic surfaces they
sample, on the CPU and without the oracle: points on the surface, normals
along the implicit gradient, and coefficients whose fundamental forms give
the surface's own principal curvatures (negative for convex with outward
normals: the unit sphere has a20 = a02 = -1/2, kappa = -1), in the paper's
coefficient order (a00, a01, a10, a11, a02, a20) over the frame of each
normal.  Also the sampling densities the workloads state, and determinism."""
import math

import numpy as np
import pytest

import synth


def curvatures(a):
    """Principal curvatures (ascending) and their eigenvectors in the (s, t)
    frame of patches with a10 = a01 = 0: II = [[2 a20, a11], [a11, 2 a02]]
    against I = identity."""
    II = np.stack([np.stack([2 * a[:, 5], a[:, 3]], -1), np.stack([a[:, 3], 2 * a[:, 4]], -1)], -2)
    return np.linalg.eigh(II)


def test_sphere_fibonacci():
    p, n, a = synth.sphere_fibonacci(4096, 1001)
    np.testing.assert_allclose(np.linalg.norm(p, axis=1), 1.0, atol=1e-14)
    np.testing.assert_allclose(n, p, atol=1e-14)
    np.testing.assert_array_equal(a, np.tile([0.0, 0.0, 0.0, 0.0, -0.5, -0.5], (4096, 1)))
    # the lattice's heights are the midpoints of N equal bands: area-uniform
    np.testing.assert_allclose(np.sort(p[:, 2]), np.sort(1.0 - (2 * np.arange(4096) + 1) / 4096), atol=1e-14)


def test_ring_torus_clean_geometry_and_curvatures():
    R, r = 1.0, 0.35
    p, n, a = synth.ring_torus(5000, 7, R=R, r=r, noise=0.0, jitter_deg=0.0)
    rho = np.hypot(p[:, 0], p[:, 1])
    np.testing.assert_allclose((rho - R) ** 2 + p[:, 2] ** 2, r * r, atol=1e-13)
    centre = np.stack([R * p[:, 0] / rho, R * p[:, 1] / rho, np.zeros(len(p))], 1)
    np.testing.assert_allclose(n, (p - centre) / r, atol=1e-12)
    assert np.all(a[:, :3] == 0.0)
    k, V = curvatures(a)
    cos_t = (rho - R) / r
    k_par = -cos_t / (R + r * cos_t)                 # along the parallel
    k_mer = np.full(len(p), -1.0 / r)                # around the tube
    np.testing.assert_allclose(k, np.sort(np.stack([k_mer, k_par], 1), axis=1), atol=1e-12)
    # the -1/r direction is the meridian: orthogonal to the parallel (-sin psi, cos psi, 0)
    s, t = synth.frame(n)
    v = V[:, 0, 0][:, None] * s + V[:, 1, 0][:, None] * t
    e_par = np.stack([-p[:, 1] / rho, p[:, 0] / rho, np.zeros(len(p))], 1)
    np.testing.assert_allclose(np.abs((v * e_par).sum(1)), 0.0, atol=1e-9)


def test_ring_torus_area_uniform():
    """Area element (R + r cos theta) dtheta dpsi: E[cos theta] = r / (2 R),
    psi uniform."""
    R, r = 1.0, 0.35
    p, _, _ = synth.ring_torus(200_000, 8, R=R, r=r, noise=0.0, jitter_deg=0.0)
    rho = np.hypot(p[:, 0], p[:, 1])
    assert abs(np.mean((rho - R) / r) - r / (2 * R)) < 0.01
    psi = np.arctan2(p[:, 1], p[:, 0])
    assert abs(np.mean(np.cos(psi))) < 0.01 and abs(np.mean(np.sin(psi))) < 0.01


def test_normal_jitter_and_noise():
    """von Mises-Fisher jitter of concentration kappa = 1 / (2 deg)^2:
    E[1 - cos angle] = 1 / kappa (for large kappa); position noise sigma
    0.005 off the clean surface."""
    R, r = 1.0, 0.35
    p0, n0, _ = synth.ring_torus(50_000, 9, R=R, r=r, noise=0.0, jitter_deg=0.0)
    p, n, _ = synth.ring_torus(50_000, 9, R=R, r=r, noise=0.005, jitter_deg=2.0)
    np.testing.assert_allclose(np.linalg.norm(n, axis=1), 1.0, atol=1e-12)
    kappa = 1.0 / math.radians(2.0) ** 2
    assert np.mean(1.0 - (n * n0).sum(1)) == pytest.approx(1.0 / kappa, rel=0.05)
    assert np.std(p - p0) == pytest.approx(0.005, rel=0.02)


def test_ellipsoid_curvatures_closed_form():
    """Unperturbed: K = 1 / (a b c)^2 / |D|^4 and H = (|x|^2 - a^2 - b^2 - c^2)
    / (2 (a b c)^2 |D|^3) with D = (x / a^2, y / b^2, z / c^2) (negative for
    the convex surface with outward normals)."""
    ax = np.array([1.0, 0.6, 0.4])
    p, n, a = synth.ellipsoid(4000, 10, axes=tuple(ax), perturb=0.0)
    np.testing.assert_allclose(((p / ax) ** 2).sum(1), 1.0, atol=1e-12)
    D = p / ax ** 2
    Dn = np.linalg.norm(D, axis=1)
    np.testing.assert_allclose(n, D / Dn[:, None], atol=1e-12)
    k, _ = curvatures(a)
    abc2 = np.prod(ax) ** 2
    np.testing.assert_allclose(k[:, 0] * k[:, 1], 1.0 / (abc2 * Dn ** 4), rtol=1e-9)
    H = ((p ** 2).sum(1) - (ax ** 2).sum()) / (2.0 * abc2 * Dn ** 3)
    np.testing.assert_allclose(0.5 * (k[:, 0] + k[:, 1]), H, rtol=1e-9)
    # perturbed: the same directions, each curvature scaled by 1 + 0.05 N(0, 1)
    _, _, ap = synth.ellipsoid(4000, 10, axes=tuple(ax), perturb=0.05)
    kp, _ = curvatures(ap)
    ratio = np.concatenate([kp[:, 0] / k[:, 0], kp[:, 1] / k[:, 1]])
    assert np.std(ratio) == pytest.approx(0.05, rel=0.1)


def test_superquadric_on_its_level_set():
    axes, e1, e2 = (1.0, 0.7, 0.5), 0.5, 2.0
    p, n, a = synth.superquadric(3000, 11, axes=axes, e1=e1, e2=e2, noise=0.0, grid=192)
    X = np.abs(p) / np.array(axes)
    F = (X[:, 0] ** (2 / e2) + X[:, 1] ** (2 / e2)) ** (e2 / e1) + X[:, 2] ** (2 / e1)
    np.testing.assert_allclose(F, 1.0, atol=1e-9)
    np.testing.assert_allclose(np.linalg.norm(n, axis=1), 1.0, atol=1e-12)
    assert np.all((n * p).sum(1) > 0.0)                    # outward on a star-shaped surface
    k, _ = curvatures(a)
    assert np.all(np.abs(k) <= 1e3 + 1e-9)                 # capped at the edges
    # flat directions set to 0 (read back through the coefficients: rounding only)
    assert np.all((np.abs(k) < 1e-9) | (np.abs(k) >= 1e-6 - 1e-9))
    assert (np.abs(k) < 1e-9).any()
    assert np.all(k <= 1e-9)                               # convex (e1, e2 <= 2)


@pytest.mark.parametrize("inward", [False, True])
def test_plane_and_cylinder(inward):
    p, n, a = synth.plane_patch(300, 12, extent=2.0)
    assert np.all(p[:, 2] == 0.0) and np.all(np.abs(p[:, :2]) <= 2.0)
    np.testing.assert_array_equal(n, np.tile([0.0, 0.0, 1.0], (300, 1)))
    assert not a.any()
    rad = 0.4
    p, n, a = synth.cylinder_cloud(500, 13, radius=rad, half_len=0.8, inward=inward)
    np.testing.assert_allclose(np.hypot(p[:, 0], p[:, 1]), rad, atol=1e-14)
    assert np.all(np.abs(p[:, 2]) <= 0.8)
    out = np.stack([p[:, 0], p[:, 1], np.zeros(500)], 1) / rad
    np.testing.assert_allclose(n, -out if inward else out, atol=1e-14)
    k, _ = curvatures(a)
    sgn = 1.0 if inward else -1.0
    np.testing.assert_allclose(k, np.sort(np.stack([np.zeros(500), np.full(500, sgn / rad)], 1), axis=1),
                               atol=1e-12)


def test_queries_and_cameras():
    x = synth.uniform_queries(10_000, 14, -1.5, 1.5)
    assert x.shape == (10_000, 3) and x.min() >= -1.5 and x.max() < 1.5
    g = synth.grid_queries(5)
    assert g.shape == (125, 3)
    np.testing.assert_array_equal(synth.grid_query_index(np.arange(125), 5), g)
    np.testing.assert_array_equal(g[:5, 0], np.linspace(-1.6, 1.6, 5))    # x fastest
    assert np.all(g[:5, 1:] == -1.6)
    org, d = synth.camera_rays(32, 24, 15, dist=3.0)
    assert org.shape == d.shape == (32 * 24, 3)
    np.testing.assert_allclose(np.linalg.norm(d, axis=1), 1.0, atol=1e-14)
    np.testing.assert_allclose(np.linalg.norm(org, axis=1), 3.0, atol=1e-14)
    centre = d[12 * 32 + 16] + d[11 * 32 + 15]                           # the four rays around the centre
    centre += d[12 * 32 + 15] + d[11 * 32 + 16]
    np.testing.assert_allclose(centre / np.linalg.norm(centre), -org[0] / 3.0, atol=1e-12)


def test_seeded_and_deterministic():
    for gen in (lambda s: synth.ring_torus(500, s), lambda s: synth.ellipsoid(500, s),
                lambda s: synth.superquadric(500, s, grid=64)):
        a1, a2, b = gen(21), gen(21), gen(22)
        for u, v in zip(a1, a2):
            np.testing.assert_array_equal(u, v)
        assert not np.array_equal(a1[0], b[0])
