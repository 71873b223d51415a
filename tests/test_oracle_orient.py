"""Pins of the oracle's orientation repair (Sec. 6): the coefficient flip
keeps the torus and negates its SDF (checked through the independently
pinned fit and torus SDF), flipping twice is the identity, and clouds with
30% of their normals reversed come back to the known outward orientation."""
import numpy as np
import pytest

import synth
from oracle import orient


def _random_coeffs(rng, m):
    a = np.zeros((m, 6))
    a[:, 0] = rng.uniform(-0.05, 0.05, m)              # a00
    a[:, 1:3] = rng.uniform(-0.4, 0.4, (m, 2))         # a01, a10 (tilt)
    a[:, 3] = rng.uniform(-1.0, 1.0, m)                # a11
    a[:, 4:6] = rng.uniform(-2.0, 2.0, (m, 2))         # a02, a20
    return a


def test_flip_keeps_the_torus(oracle_mod):
    rng = np.random.Generator(np.random.PCG64(90))
    n = rng.normal(size=(40, 3))
    n /= np.linalg.norm(n, axis=1, keepdims=True)
    n[0] = [0.0, 0.0, 1.0]
    n[1] = [0.0, 0.0, -1.0]                            # both branches of the frame
    p = rng.uniform(-1, 1, (40, 3))
    a = _random_coeffs(rng, 40)
    x = rng.uniform(-2, 2, (50, 3))
    for i in range(40):
        a2 = orient.flip_coefficients(n[i], a[i])
        g1 = oracle_mod.Cloud(p[i:i + 1], n[i:i + 1], a[i:i + 1]).g(0, x)
        g2 = oracle_mod.Cloud(p[i:i + 1], -n[i:i + 1], a2[None]).g(0, x)
        np.testing.assert_allclose(g2, -g1, atol=1e-9)
        f1 = oracle_mod.fit_record(p[i], n[i], a[i])
        f2 = oracle_mod.fit_record(p[i], -n[i], a2)
        np.testing.assert_allclose(f2["q"], f1["q"], atol=1e-12)
        np.testing.assert_allclose(f2["nstar"], -f1["nstar"], atol=1e-12)
        np.testing.assert_allclose(np.abs(f2["kmin"]), np.abs(f1["kmin"]), rtol=1e-9, atol=1e-12)
        np.testing.assert_allclose(orient.flip_coefficients(-n[i], a2), a[i], atol=1e-12)


def _scramble(p, n, a, frac, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    idx = rng.choice(len(p), int(frac * len(p)), replace=False)
    n2, a2 = n.copy(), a.copy()
    for i in idx:
        a2[i] = orient.flip_coefficients(n[i], a[i])
        n2[i] = -n[i]
    return n2, a2, idx


@pytest.mark.parametrize("shape", ["sphere", "ellipsoid"])
def test_recovers_orientation(shape):
    if shape == "sphere":
        p, n, a = synth.sphere_fibonacci(600, 91)
    else:
        p, n, a = synth.ellipsoid(600, 92, (1.0, 0.6, 0.4), perturb=0.0)
    n2, a2, idx = _scramble(p, n, a, 0.3, 93)
    nf, af, flips = orient.orient(p, n2, a2, k=16, max_iter=10)
    assert flips[0] > 0 and flips[-1] == 0
    np.testing.assert_allclose(nf, n / np.linalg.norm(n, axis=1, keepdims=True), atol=1e-12)
    np.testing.assert_allclose(af, a, atol=1e-9)
