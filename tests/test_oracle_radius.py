"""Pins of the oracle's radius-limited evaluation and of the mean k-nearest
distance D of the lambda heuristic (Sec. 4.2, "Acceleration and adaptive
lambda"), each against a value fixed by construction or by an already
pinned function:

- R_eval beyond every distance: the all-pairs blend with the same constant
  lambda (FIXED mode, itself pinned in test_oracle_pins.py);
- a line of plane points with lambda = 0: the in-radius set and the
  32-nearest fallback set are known from the geometry, and phi is the plain
  mean of g_k = z - z_k over them;
- the sphere cloud: every torus is the unit sphere, so phi = |x| - 1 whatever
  the set and the weights;
- D on a regular polygon (closed form) and with fewer than k other points.
"""
import math

import numpy as np
import pytest

import synth
from workloads import f32, mixed_cloud


def line_cloud(h=0.1, kmax=40):
    k = np.arange(-kmax, kmax + 1)
    z = 0.001 * ((7 * k) % 5)
    p = np.stack([k * h, np.zeros_like(z), z], 1)
    n = np.tile([0.0, 0.0, 1.0], (k.size, 1))
    a = np.zeros((k.size, 6))
    return k, z, p, n, a


def test_radius_beyond_all_points_is_all_pairs(oracle_mod):
    p, n, a = mixed_cloud(2)
    cl = oracle_mod.Cloud(p, n, a)
    x = synth.uniform_queries(200, 3)
    for lam in (0.0, 5.0, 40.0):
        got = cl.phi_radius(x, lam=lam, reval=1e6)
        ref = cl.phi(x, mode=oracle_mod.FIXED, lam=lam, shift=oracle_mod.SHIFT_DMIN)
        np.testing.assert_allclose(got, ref, atol=1e-12, rtol=0)


def test_line_in_radius_set(oracle_mod):
    h = 0.1
    k, z, p, n, a = line_cloud(h)
    cl = oracle_mod.Cloud(p, n, a)
    z0 = 0.01
    x = np.array([[0.0, 0.0, z0]])
    for R, half in ((2.5 * h, 2), (3.5 * h, 3), (0.5 * h, 0)):
        got, used = cl.phi_radius(x, lam=0.0, reval=R, used=True)
        sel = np.abs(k) <= half
        assert used[0] == sel.sum()
        assert abs(got[0] - (z0 - z[sel].mean())) < 1e-14


def test_line_fallback_set(oracle_mod):
    """No point within R_eval: the 32 nearest are k = -15..16 for a query
    above x = 0.25 h (the 33rd, k = -16, is 0.5 h farther)."""
    h = 0.1
    k, z, p, n, a = line_cloud(h)
    cl = oracle_mod.Cloud(p, n, a)
    H = 1.0
    x = np.array([[0.25 * h, 0.0, H]])
    got, used = cl.phi_radius(x, lam=0.0, reval=0.5 * H, used=True)
    sel = (k >= -15) & (k <= 16)
    assert used[0] == -32
    assert abs(got[0] - (H - z[sel].mean())) < 1e-14
    # the fallback size is an argument: 8 nearest are k = -3..4
    got8 = cl.phi_radius(x, lam=0.0, reval=0.5 * H, kfb=8)
    sel8 = (k >= -3) & (k <= 4)
    assert abs(got8[0] - (H - z[sel8].mean())) < 1e-14


@pytest.mark.parametrize("lam,R", [(50.0, 0.3), (1e3, 0.05), (10.0, 2.0)])
def test_sphere_exact_any_set(oracle_mod, lam, R):
    p, n, a = synth.sphere_fibonacci(512, 4)
    cl = oracle_mod.Cloud(p, n, a)
    x = synth.uniform_queries(300, 5)
    got, used = cl.phi_radius(x, lam=lam, reval=R, used=True)
    np.testing.assert_allclose(got, np.linalg.norm(x, axis=1) - 1.0, atol=1e-12)
    assert (used > 0).any() or R < 0.1          # both branches are exercised across the cases
    assert (used < 0).any() or R > 1.0


def test_knn_mean_distance_polygon(oracle_mod):
    """A regular N-gon of radius rho: every vertex's 64 nearest are the 32
    neighbours on each side, at chords 2 rho sin(pi m / N)."""
    N, rho = 200, 1.3
    t = 2 * np.pi * np.arange(N) / N
    pts = np.stack([rho * np.cos(t), rho * np.sin(t), np.zeros(N)], 1)
    ref = sum(2 * 2 * rho * math.sin(math.pi * m / N) for m in range(1, 33)) / 64
    assert abs(oracle_mod.knn_mean_distance(pts, 64) - ref) < 1e-12
    # k = 2: the two adjacent vertices
    assert abs(oracle_mod.knn_mean_distance(pts, 2) - 2 * rho * math.sin(math.pi / N)) < 1e-12


def test_knn_mean_distance_few_points(oracle_mod):
    """Fewer than k other points: all of them (an equilateral triangle of side
    a gives D = a); one point gives 0."""
    a = 0.7
    pts = np.array([[0, 0, 0], [a, 0, 0], [a / 2, a * math.sqrt(3) / 2, 0]])
    assert abs(oracle_mod.knn_mean_distance(pts, 64) - a) < 1e-14
    assert oracle_mod.knn_mean_distance(pts[:1], 64) == 0.0
