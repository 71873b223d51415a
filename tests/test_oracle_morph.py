"""Pins of the oracle's level-set sampling (Sec. 6, "Morphological
operations"): Newton steps along grad phi onto the c level set, normals from
grad phi.

- A unit-sphere cloud has phi(x) = |x| - 1 exactly (pinned in
  test_oracle_pins.py), so every seed lands on the sphere of radius 1 + c,
  x0 (1 + c) / |x0|, in one step, with normal x0 / |x0| (closed form); with
  no step the residual is the signed |x0| - 1 - c.
- A plane cloud on z = 0 has phi = z: seeds land on z = c with normal +z.
- On a noisy mixed cloud the residual |phi - c| falls quadratically (Newton)
  to rounding within a few steps, the normals are unit vectors, and seeds
  already on the level set do not move.
"""
import numpy as np

import oracle
import synth
from oracle.morph import project_level_set
from workloads import mixed_cloud


def test_sphere_closed_form():
    p, n, a = synth.sphere_fibonacci(400, 3)
    cl = oracle.Cloud(p, n, a)
    x0 = synth.uniform_queries(60, 4, -1.5, 1.5)
    x0 = x0[np.linalg.norm(x0, axis=1) > 0.2]
    for c in (-0.1, 0.0, 0.25):
        x, nrm, res = project_level_set(cl, x0, c, max_iter=3)
        r0 = np.linalg.norm(x0, axis=1, keepdims=True)
        np.testing.assert_allclose(x, x0 * (1 + c) / r0, atol=1e-12)
        np.testing.assert_allclose(nrm, x0 / r0, atol=1e-12)
        assert np.abs(res).max() < 1e-12
        # no step: the seeds themselves, and the signed residual phi - c = |x0| - 1 - c
        x, nrm, res = project_level_set(cl, x0, c, max_iter=0)
        np.testing.assert_array_equal(x, x0)
        np.testing.assert_allclose(res, r0[:, 0] - 1.0 - c, atol=1e-12)
        np.testing.assert_allclose(nrm, x0 / r0, atol=1e-12)


def test_plane_closed_form():
    p, n, a = synth.plane_patch(200, 5, extent=2.0)
    cl = oracle.Cloud(p, n, a)
    x0 = synth.uniform_queries(40, 6, -0.8, 0.8)
    x, nrm, res = project_level_set(cl, x0, 0.07, max_iter=2)
    np.testing.assert_allclose(x[:, :2], x0[:, :2], atol=1e-12)
    np.testing.assert_allclose(x[:, 2], 0.07, atol=1e-12)
    np.testing.assert_allclose(nrm, np.tile([0.0, 0.0, 1.0], (len(x0), 1)), atol=1e-12)


def test_newton_convergence_on_noisy_cloud():
    p, n, a = mixed_cloud(7)
    rng = np.random.Generator(np.random.PCG64(8))
    cl = oracle.Cloud(p, n, a)
    seeds = p[rng.choice(len(p), size=40, replace=False)]
    res = []
    for k in (1, 2, 3, 6):
        _, nrm, r = project_level_set(cl, seeds, -0.05, max_iter=k)
        res.append(np.abs(r))
    np.testing.assert_allclose(np.linalg.norm(nrm, axis=1), 1.0, atol=1e-12)
    assert np.median(res[3]) < 1e-9
    # quadratic convergence where the first step left a residual above rounding
    big = res[0] > 1e-6
    assert big.any() and (res[2][big] < 10 * res[0][big] ** 2 + 1e-12).mean() > 0.9
    # seeds already on the level set (to the tolerance) do not move
    x6, _, r6 = project_level_set(cl, seeds, -0.05, max_iter=6)
    on = np.abs(r6) <= 1e-8
    assert on.sum() >= 30
    x7, _, _ = project_level_set(cl, x6[on], -0.05, max_iter=3, tol=1e-8)
    assert np.abs(x7 - x6[on]).max() == 0.0
