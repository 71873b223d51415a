"""The general curvature-form pair of the tensor-core epilogue
(tile_pairs_kappa2 in csrc/query_tc.cu), on the CPU: its two half-angle
steps (Sec. 4.1, the form without 1/kappa) put over one denominator,

    D1 = 1 + sqrt(1 + k m),   Nn = kM (m^2 + h^2 D1^2) + 2 zeta m D1,
    g  = Nn / (D1 (D1 + sqrt(D1^2 + kM Nn))),

against the two-reciprocal form a' = m / D1, N' = kM (a'^2 + h^2) + 2 zeta a',
g = N' / (1 + sqrt(1 + kM N')) that it replaces (kM is the record's
-kappa_max, in units of the tile scale).  In FP64 the two agree to rounding;
emulated in FP32 (each operation rounded, fused multiply-adds rounded once)
they carry the same error against an FP64 evaluation, over inputs that span
the clouds' curvatures and query distances.  The GPU parity tests check the
kernel itself against the oracle."""
import numpy as np
import pytest

F = np.float32


def inputs(n=200_000, seed=7):
    """Random pair quantities in units of the tile scale: h, |y|^2 >= h^2, m0,
    |kappa_min| s, -kappa_max s, 2 zeta."""
    rng = np.random.Generator(np.random.PCG64(seed))
    scale = lambda *v: rng.choice(v, n)  # noqa: E731
    h = rng.normal(size=n) * scale(1e-3, 0.1, 1.0)
    yy = h * h + np.abs(rng.normal(size=n)) * scale(1e-4, 0.1, 1.0)
    m0 = rng.normal(size=n) * scale(1e-3, 0.1, 1.0)
    k = np.abs(rng.normal(size=n)) * scale(1e-3, 1.0, 100.0, 4000.0)
    kM = rng.normal(size=n) * scale(1e-3, 1.0, 100.0, 4000.0)
    z2 = rng.choice([-2.0, 2.0], n)
    return h, yy, m0, k, kM, z2


def fma32(a, b, c):
    """a * b + c with one rounding to FP32 (the product of two FP32 values is
    exact in FP64)."""
    return (a.astype(np.float64) * b.astype(np.float64) + c.astype(np.float64)).astype(F)


def two_rcp(h, yy, m0, k, kM, z2, fp32):
    if not fp32:
        hh = h * h
        m = k * (yy - hh) + m0
        d1 = 1.0 + np.sqrt(np.maximum(k * m + 1.0, 0.0))
        ap = m / d1
        npr = kM * (ap * ap + hh) + z2 * ap
        return npr / (1.0 + np.sqrt(np.maximum(kM * npr + 1.0, 0.0)))
    one = np.ones_like(h)
    hh = (h * h).astype(F)
    m = fma32(k, (yy - hh).astype(F), m0)
    d1 = (one + np.sqrt(np.maximum(fma32(k, m, one), F(0)))).astype(F)
    ap = (m * (one / d1).astype(F)).astype(F)
    npr = fma32(kM, fma32(ap, ap, hh), (z2 * ap).astype(F))
    d2 = (one + np.sqrt(np.maximum(fma32(kM, npr, one), F(0)))).astype(F)
    return (npr * (one / d2).astype(F)).astype(F)


def one_rcp(h, yy, m0, k, kM, z2, fp32):
    if not fp32:
        hh = h * h
        m = k * (yy - hh) + m0
        d1 = 1.0 + np.sqrt(np.maximum(k * m + 1.0, 0.0))
        nn = kM * (m * m + hh * d1 * d1) + z2 * (m * d1)
        return nn / (d1 * (d1 + np.sqrt(np.maximum(kM * nn + d1 * d1, 0.0))))
    one = np.ones_like(h)
    hh = (h * h).astype(F)
    m = fma32(k, (yy - hh).astype(F), m0)
    d1 = (one + np.sqrt(np.maximum(fma32(k, m, one), F(0)))).astype(F)
    d1sq = (d1 * d1).astype(F)
    nn = fma32(kM, fma32(m, m, (hh * d1sq).astype(F)), (z2 * (m * d1).astype(F)).astype(F))
    u = fma32(kM, nn, d1sq)
    den = (d1 * (d1 + np.sqrt(np.maximum(u, F(0)))).astype(F)).astype(F)
    return (nn * (one / den).astype(F)).astype(F)


def test_one_denominator_is_the_same_function():
    q = inputs()
    a, b = two_rcp(*q, fp32=False), one_rcp(*q, fp32=False)
    assert np.isfinite(a).all() and np.isfinite(b).all()
    err = np.abs(a - b) / np.maximum(np.abs(a), 1.0)
    assert err.max() < 1e-12


def test_second_root_argument_is_a_sum_of_squares():
    """With zeta = +-1, 1 + kM N' = (1 + zeta kM a')^2 + (kM h)^2, so the
    second root's argument D1^2 + kM Nn = D1^2 (1 + kM N') is never negative
    but by rounding: the kernel's clamp at zero only guards that."""
    h, yy, m0, k, kM, z2 = inputs()
    m = k * (yy - h * h) + m0
    d1 = 1.0 + np.sqrt(np.maximum(k * m + 1.0, 0.0))
    ap = m / d1
    nn = kM * (m * m + h * h * d1 * d1) + z2 * (m * d1)
    u = kM * nn + d1 * d1
    squares = d1 * d1 * ((1.0 + 0.5 * z2 * kM * ap) ** 2 + (kM * h) ** 2)
    assert np.allclose(u, squares, rtol=1e-9, atol=1e-9)
    assert (u >= -1e-9 * np.abs(squares).max()).all()


def test_denominator_at_least_one():
    """D1 >= 1, so the one reciprocal never sees a denominator below 1."""
    q = [v.astype(F) for v in inputs()]
    h, yy, m0, k, kM, z2 = q
    one = np.ones_like(h)
    m = fma32(k, (yy - (h * h).astype(F)).astype(F), m0)
    d1 = (one + np.sqrt(np.maximum(fma32(k, m, one), F(0)))).astype(F)
    assert (d1 >= 1).all()


@pytest.mark.parametrize("seed", [7, 8])
def test_fp32_error_not_larger(seed):
    q32 = [v.astype(F) for v in inputs(seed=seed)]
    ref = two_rcp(*[v.astype(np.float64) for v in q32], fp32=False)
    sc = np.maximum(np.abs(ref), 1.0)
    e_two = np.abs(two_rcp(*q32, fp32=True).astype(np.float64) - ref) / sc
    e_one = np.abs(one_rcp(*q32, fp32=True).astype(np.float64) - ref) / sc
    assert np.isfinite(e_one).all()
    # the same error profile: the largest errors come from the shared first
    # step (m = k (|y|^2 - h^2) + m0), not from the denominators
    assert e_one.max() <= 1.01 * e_two.max()
    assert np.quantile(e_one, 0.999) <= 1.5 * np.quantile(e_two, 0.999) + 1e-7
    assert np.median(e_one) <= 2.0 * np.median(e_two) + 1e-8
