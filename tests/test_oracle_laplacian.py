"""Pins of the oracle's Laplacian (App. D, "Laplacian"), computed by
second-order jets: closed forms where every torus equals the shape (sphere,
plane, cylinder, ring-torus equators), central second differences of the
oracle's phi elsewhere (GLOBAL lambda, so the lambda_x(x) terms are pinned
too), and its first derivatives against the dual-number gradient."""
import math

import numpy as np
import pytest

import synth


@pytest.mark.parametrize("mode", ["global", "fixed"])
def test_sphere(oracle_mod, mode):
    p, n, a = synth.sphere_fibonacci(256, 3)
    cl = oracle_mod.Cloud(p, n, a)
    x = synth.uniform_queries(200, 5)
    kw = {} if mode == "global" else {"mode": oracle_mod.FIXED, "lam": 40.0}
    phi, g, lap = cl.laplacian(x, **kw)
    r = np.linalg.norm(x, axis=1)
    np.testing.assert_allclose(lap, 2.0 / r, rtol=1e-10)
    np.testing.assert_allclose(g, x / r[:, None], atol=1e-12)


def test_plane_and_cylinder(oracle_mod):
    p, n, a = synth.plane_patch(200, 9)
    x = synth.uniform_queries(100, 10)
    _, g, lap = oracle_mod.Cloud(p, n, a).laplacian(x)
    assert np.abs(lap).max() < 1e-10
    np.testing.assert_allclose(g, np.tile([0.0, 0.0, 1.0], (len(x), 1)), atol=1e-12)
    for inward in (False, True):
        p, n, a = synth.cylinder_cloud(300, 12, radius=0.5, inward=inward)
        x = synth.uniform_queries(100, 13)
        rho = np.linalg.norm(x[:, :2], axis=1)
        _, _, lap = oracle_mod.Cloud(p, n, a).laplacian(x)
        np.testing.assert_allclose(lap, (-1.0 if inward else 1.0) / rho, rtol=1e-9)


def test_ring_torus_equators(oracle_mod):
    """Every torus is the ring torus: lap phi = lap D = 1/D + (rho - R)/(rho D)
    with D the distance to the centre circle."""
    R, r = 1.0, 0.35
    psi = np.linspace(0, 2 * math.pi, 24, endpoint=False)
    theta = np.concatenate([np.zeros(24), np.full(24, math.pi)])
    p, n, a = synth.ring_torus(48, 0, R=R, r=r, noise=0.0, jitter_deg=0.0, theta=theta,
                               psi=np.concatenate([psi, psi + 0.1]))
    x = synth.uniform_queries(200, 14, -1.6, 1.6)
    rho = np.linalg.norm(x[:, :2], axis=1)
    D = np.sqrt((rho - R) ** 2 + x[:, 2] ** 2)
    _, _, lap = oracle_mod.Cloud(p, n, a).laplacian(x)
    np.testing.assert_allclose(lap, 1.0 / D + (rho - R) / (rho * D), rtol=1e-9)


def test_finite_differences(oracle_mod):
    """Generic clouds, GLOBAL lambda: lap phi against the 7-point stencil of the
    oracle's own phi, which converges at O(h^2) to it (h = 5e-4 and 2.5e-4),
    away from farthest-point ties; and grad phi against the dual numbers.
    (Clouds with near-flat points are left to the closed-form pins: there the
    literal radius form carries rounding noise of ~1e-9 that the stencil
    divides by h^2.)"""
    from test_gpu_grad import kink_free
    clouds = (synth.ellipsoid(300, 80), synth.ring_torus(300, 21, noise=0.01, jitter_deg=5.0),
              synth.superquadric(300, 81, kappa_cap=20.0))
    for p, n, a in clouds:
        cl = oracle_mod.Cloud(p, n, a)
        x = synth.uniform_queries(600, 22, -1.4, 1.4)
        x = x[kink_free(p, x, 0.02, 0.3)][:120]
        assert len(x) >= 60
        phi, g, lap = cl.laplacian(x)
        errs = []
        for h in (5e-4, 2.5e-4):
            fd = -6.0 * cl.phi(x)
            for ax in range(3):
                e = np.zeros(3)
                e[ax] = h
                fd = fd + cl.phi(x + e) + cl.phi(x - e)
            fd /= h * h
            errs.append((np.abs(fd - lap) / (1.0 + np.abs(lap))).max())
        assert errs[1] <= 1e-3 and errs[1] < errs[0] / 3.0, errs
        _, g2 = cl.grad_x(x)
        np.testing.assert_allclose(g, g2, atol=1e-10)
