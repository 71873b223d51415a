"""Pins of the oracle's orientation repair (Sec. 6): the coefficient flip
keeps the torus and negates its SDF (checked through the independently
pinned fit and torus SDF), flipping twice is the identity, one step's
scores equal the neighbour sums with the Mahalanobis length built from
principal curvatures and directions computed here, and clouds with 30% of
their normals reversed come back to the known outward orientation."""
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


def _principal(n, a):
    """|kappa_min|, |kappa_max| and unit 3-D principal directions (v_min,
    v_max) of the patch Q*(s, t) = p + s s_i + t t_i + f(s, t) n_i at (0, 0):
    the generalised eigenproblem II w = kappa I w of the second and first
    fundamental forms (I = [[1 + a10^2, a10 a01], [a10 a01, 1 + a01^2]],
    II = [[2 a20, a11], [a11, 2 a02]] / sqrt(1 + a10^2 + a01^2)), with each
    w mapped to w_s (s + a10 n) + w_t (t + a01 n)."""
    import scipy.linalg
    a00, a01, a10, a11, a02, a20 = a
    I = np.array([[1 + a10 ** 2, a10 * a01], [a10 * a01, 1 + a01 ** 2]])
    II = np.array([[2 * a20, a11], [a11, 2 * a02]]) / np.sqrt(1 + a10 ** 2 + a01 ** 2)
    kap, W = scipy.linalg.eigh(II, I)
    s, t = synth.frame(n[None])
    Qs, Qt = s[0] + a10 * n, t[0] + a01 * n
    V = [w[0] * Qs + w[1] * Qt for w in W.T]
    V = [v / np.linalg.norm(v) for v in V]
    lo = int(np.argmin(np.abs(kap)))
    return abs(kap[lo]), abs(kap[1 - lo]), V[lo], V[1 - lo]


def test_step_scores_use_the_principal_mahalanobis_length(oracle_mod):
    """score_i = sum_j exp(-M_i(p_i - p_j)) <n_i, grad phi(p_j)> with
    M_i(r)^2 = kmin^2 <r, v_min>^2 + kmax^2 <r, v_max>^2 + eps^2 <r, n_i>^2:
    curvatures and directions from _principal, grad phi from the oracle's
    pinned gradient, neighbours and eps given."""
    rng = np.random.Generator(np.random.PCG64(95))
    m = 60
    p = rng.uniform(-0.5, 0.5, (m, 3))
    n = rng.normal(size=(m, 3))
    n /= np.linalg.norm(n, axis=1, keepdims=True)
    a = _random_coeffs(rng, m)
    nbr = orient.knn_indices(p, 6)
    eps = 3.0
    _, score = orient.orientation_step(p, n, a, nbr, eps)
    _, g = oracle_mod.Cloud(p, n, a).grad_x(p)
    for i in range(m):
        kmin, kmax, vmin, vmax = _principal(n[i], a[i])
        r = p[i] - p[nbr[i]]
        M = np.sqrt((kmin * (r @ vmin)) ** 2 + (kmax * (r @ vmax)) ** 2 + (eps * (r @ n[i])) ** 2)
        np.testing.assert_allclose(score[i], np.exp(-M) @ (g[nbr[i]] @ n[i]), rtol=1e-9, atol=1e-12)


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
