"""Seeded synthetic inputs for the points-as-tori SDF workloads.

This module only *makes inputs*: oriented point clouds, their six per-point
coefficients (a00, a01, a10, a11, a02, a20) and query positions / rays.  It
holds none of the method's arithmetic (no torus fit, no torus SDF, no blend)
and imports neither the CUDA library nor the oracle; both sides consume what
it returns.

Coefficient convention (the input format of the method, Sec. 4.1, Eq.
BivariatePolynomial): the surface near p_i is
    Q*(s, t) = p_i + s s_i + t t_i + Q(s, t) n_i,
    Q(s, t) = a00 + a10 s + a01 t + a11 s t + a20 s^2 + a02 t^2,
with (s_i, t_i, n_i) the right-handed orthonormal frame of Duff et al. 2017
("Building an Orthonormal Basis, Revisited").  With a10 = a01 = 0 the second
fundamental form in that frame is [[2 a20, a11], [a11, 2 a02]], so an analytic
shape operator projected into the frame gives the coefficients directly.
Curvature sign: negative where the surface bends away from the outward
normal (a unit sphere with outward normals has kappa = -1, a20 = a02 = -0.5).

Every generator takes an explicit seed and uses numpy's PCG64.
"""
from __future__ import annotations

import math

import numpy as np

__all__ = [
    "frame", "coeffs_from_shape_operator", "sphere_fibonacci", "ring_torus",
    "ellipsoid", "superquadric", "uniform_queries", "grid_queries",
    "camera_rays", "vmf_jitter", "plane_patch", "cylinder_cloud",
]


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def frame(n: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """Duff et al. 2017 orthonormal basis (s, t) of unit normals n (M x 3)."""
    n = np.asarray(n, dtype=np.float64)
    sg = np.where(n[:, 2] >= 0.0, 1.0, -1.0)
    a = -1.0 / (sg + n[:, 2])
    b = n[:, 0] * n[:, 1] * a
    s = np.stack([1.0 + sg * n[:, 0] ** 2 * a, sg * b, -sg * n[:, 0]], axis=1)
    t = np.stack([b, sg + n[:, 1] ** 2 * a, -n[:, 1]], axis=1)
    return s, t


def coeffs_from_shape_operator(n: np.ndarray, k1: np.ndarray, e1: np.ndarray,
                               k2: np.ndarray, e2: np.ndarray) -> np.ndarray:
    """Coefficients (a00=a01=a10=0) whose second fundamental form in the frame
    of ``n`` equals k1 e1 e1^T + k2 e2 e2^T restricted to that frame's plane."""
    s, t = frame(n)
    es1, et1 = np.sum(e1 * s, 1), np.sum(e1 * t, 1)
    es2, et2 = np.sum(e2 * s, 1), np.sum(e2 * t, 1)
    ii_ss = k1 * es1 * es1 + k2 * es2 * es2
    ii_st = k1 * es1 * et1 + k2 * es2 * et2
    ii_tt = k1 * et1 * et1 + k2 * et2 * et2
    a = np.zeros((n.shape[0], 6))
    a[:, 3] = ii_st
    a[:, 4] = 0.5 * ii_tt
    a[:, 5] = 0.5 * ii_ss
    return a


def _unit(v: np.ndarray) -> np.ndarray:
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def vmf_jitter(n: np.ndarray, kappa: float, rng: np.random.Generator) -> np.ndarray:
    """Rotate unit vectors n by von Mises-Fisher noise of concentration kappa
    (Wood 1994; the 3-D inverse-CDF form of the cosine)."""
    m = n.shape[0]
    u = rng.random(m)
    w = 1.0 + np.log(u + (1.0 - u) * np.exp(-2.0 * kappa)) / kappa
    ang = rng.random(m) * 2.0 * math.pi
    b1, b2 = frame(n)
    sw = np.sqrt(np.clip(1.0 - w * w, 0.0, None))
    out = w[:, None] * n + sw[:, None] * (np.cos(ang)[:, None] * b1 + np.sin(ang)[:, None] * b2)
    return _unit(out)


def sphere_fibonacci(n: int, seed: int, radius: float = 1.0):
    """Golden-angle Fibonacci lattice on a sphere, exact outward normals and the
    sphere's coefficients a20 = a02 = -1/(2 radius)."""
    rng = _rng(seed)
    theta0 = rng.random() * 2.0 * math.pi
    i = np.arange(n, dtype=np.float64)
    z = 1.0 - (2.0 * i + 1.0) / n
    rxy = np.sqrt(np.clip(1.0 - z * z, 0.0, None))
    th = i * math.pi * (3.0 - math.sqrt(5.0)) + theta0
    nrm = np.stack([rxy * np.cos(th), rxy * np.sin(th), z], axis=1)
    pts = radius * nrm
    a = np.zeros((n, 6))
    a[:, 4] = a[:, 5] = -0.5 / radius
    return pts, nrm, a


def ring_torus(n: int, seed: int, R: float = 1.0, r: float = 0.35, noise: float = 0.005,
               jitter_deg: float = 2.0, theta: np.ndarray | None = None,
               psi: np.ndarray | None = None, inward: bool = False):
    """Area-uniform samples of a ring torus about the z axis (psi uniform, theta
    by rejection with density proportional to R + r cos theta), Gaussian
    position noise, von Mises-Fisher normal jitter (kappa = 1/jitter^2), and
    coefficients from the analytic principal curvatures and directions at the
    noise-free sample projected into the jittered normal's frame.

    Explicit ``theta``/``psi`` arrays bypass the sampling (used for equator
    clouds); ``noise=0`` and ``jitter_deg=0`` give a clean cloud; ``inward``
    flips the normals (and with them the curvature signs)."""
    rng = _rng(seed)
    if theta is None:
        th = np.empty(0)
        while th.size < n:
            cand = rng.random(2 * n + 16) * 2.0 * math.pi
            acc = rng.random(cand.size) * (R + r) < (R + r * np.cos(cand))
            th = np.concatenate([th, cand[acc]])
        th = th[:n]
        ps = rng.random(n) * 2.0 * math.pi
    else:
        th = np.asarray(theta, dtype=np.float64)
        ps = np.asarray(psi, dtype=np.float64)
        n = th.size
    ct, st, cp, sp = np.cos(th), np.sin(th), np.cos(ps), np.sin(ps)
    rad = R + r * ct
    pts = np.stack([rad * cp, rad * sp, r * st], axis=1)
    nrm = np.stack([ct * cp, ct * sp, st], axis=1)
    e_mer = np.stack([-st * cp, -st * sp, ct], axis=1)       # meridian direction
    e_par = np.stack([-sp, cp, np.zeros_like(sp)], axis=1)   # parallel direction
    k_mer = np.full(n, -1.0 / r)
    k_par = -ct / rad
    if noise > 0.0:
        pts = pts + rng.normal(0.0, noise, size=pts.shape)
    nj = vmf_jitter(nrm, 1.0 / math.radians(jitter_deg) ** 2, rng) if jitter_deg > 0.0 else nrm
    if inward:
        nj, k_mer, k_par = -nj, -k_mer, -k_par
    a = coeffs_from_shape_operator(nj, k_mer, e_mer, k_par, e_par)
    return pts, nj, a


def _shape_operator_from_implicit(grad: np.ndarray, hess: np.ndarray):
    """Principal curvatures / directions of the level set F = 0 with outward
    normal grad F / |grad F|: eigenpairs of -P Hess P / |grad F| on the
    tangent plane (Goldman 2005).  Returns (nrm, k1, e1, k2, e2)."""
    g = np.linalg.norm(grad, axis=1)
    nrm = grad / g[:, None]
    b1, b2 = frame(nrm)
    basis = np.stack([b1, b2], axis=2)                        # M x 3 x 2
    m2 = -np.einsum("mia,mij,mjb->mab", basis, hess, basis) / g[:, None, None]
    m2 = 0.5 * (m2 + np.transpose(m2, (0, 2, 1)))
    w, v = np.linalg.eigh(m2)
    e1 = np.einsum("mia,ma->mi", basis, v[:, :, 0])
    e2 = np.einsum("mia,ma->mi", basis, v[:, :, 1])
    return nrm, w[:, 0], _unit(e1), w[:, 1], _unit(e2)


def ellipsoid(n: int, seed: int, axes=(1.0, 0.6, 0.4), perturb: float = 0.05):
    """Area-uniform samples of an axis-aligned ellipsoid (uniform sphere
    directions mapped by the axes, accepted with probability proportional to
    the area stretch), exact normals, and analytic principal curvatures each
    scaled by (1 + perturb N(0,1)), directions analytic."""
    rng = _rng(seed)
    a, b, c = axes
    out = np.empty((0, 3))
    gmax = max(b * c, a * c, a * b)
    while out.shape[0] < n:
        u = _unit(rng.normal(size=(2 * n + 16, 3)))
        stretch = np.sqrt((b * c * u[:, 0]) ** 2 + (a * c * u[:, 1]) ** 2 + (a * b * u[:, 2]) ** 2)
        acc = rng.random(u.shape[0]) * gmax < stretch
        out = np.concatenate([out, u[acc] * np.array([a, b, c])])
    pts = out[:n]
    inv2 = np.array([1.0 / a ** 2, 1.0 / b ** 2, 1.0 / c ** 2])
    grad = 2.0 * pts * inv2
    hess = np.broadcast_to(np.diag(2.0 * inv2), (n, 3, 3)).copy()
    nrm, k1, e1, k2, e2 = _shape_operator_from_implicit(grad, hess)
    if perturb > 0.0:
        k1 = k1 * (1.0 + perturb * rng.normal(size=n))
        k2 = k2 * (1.0 + perturb * rng.normal(size=n))
    return pts, nrm, coeffs_from_shape_operator(nrm, k1, e1, k2, e2)


def _sq_implicit(x: np.ndarray, axes, e1: float, e2: float):
    """Barr superellipsoid F = ((|x/a|^(2/e2) + |y/b|^(2/e2))^(e2/e1) + |z/c|^(2/e1)),
    its gradient and Hessian (analytic, away from the coordinate planes)."""
    a, b, c = axes
    p, qexp = 2.0 / e2, e2 / e1
    rz = 2.0 / e1
    X, Y, Z = np.abs(x[:, 0]) / a, np.abs(x[:, 1]) / b, np.abs(x[:, 2]) / c
    sx, sy, sz = np.sign(x[:, 0]), np.sign(x[:, 1]), np.sign(x[:, 2])
    X = np.maximum(X, 1e-12); Y = np.maximum(Y, 1e-12); Z = np.maximum(Z, 1e-12)
    u = X ** p + Y ** p
    F = u ** qexp + Z ** rz
    du_dx = p * X ** (p - 1) * sx / a
    du_dy = p * Y ** (p - 1) * sy / b
    d2u_dx2 = p * (p - 1) * X ** (p - 2) / a ** 2
    d2u_dy2 = p * (p - 1) * Y ** (p - 2) / b ** 2
    f1 = qexp * u ** (qexp - 1)
    f2 = qexp * (qexp - 1) * u ** (qexp - 2)
    grad = np.stack([f1 * du_dx, f1 * du_dy, rz * Z ** (rz - 1) * sz / c], axis=1)
    hess = np.zeros((x.shape[0], 3, 3))
    hess[:, 0, 0] = f2 * du_dx ** 2 + f1 * d2u_dx2
    hess[:, 1, 1] = f2 * du_dy ** 2 + f1 * d2u_dy2
    hess[:, 0, 1] = hess[:, 1, 0] = f2 * du_dx * du_dy
    hess[:, 2, 2] = rz * (rz - 1) * Z ** (rz - 2) / c ** 2
    return F, grad, hess


def superquadric(n: int, seed: int, axes=(1.0, 0.7, 0.5), e1: float = 0.5, e2: float = 2.0,
                 noise: float = 0.003, kappa_cap: float = 1e3, grid: int = 768):
    """Area-uniform samples of a Barr superellipsoid: a fine (eta, omega)
    triangle mesh of the surface, triangles drawn by area, uniform barycentric
    points projected back to F = 1 by Newton steps along grad F.  Normals and
    principal curvatures come from the implicit function (Goldman 2005);
    |kappa| is capped at ``kappa_cap`` (edges) and values below 1e-6 (flat
    directions) are set to exactly 0.  Gaussian position noise ``noise``."""
    rng = _rng(seed)
    a, b, c = axes

    def spow(v, e):
        return np.sign(v) * np.abs(v) ** e

    eta = np.linspace(-math.pi / 2, math.pi / 2, grid + 1)
    om = np.linspace(-math.pi, math.pi, 2 * grid + 1)
    E, O = np.meshgrid(eta, om, indexing="ij")
    V = np.stack([a * spow(np.cos(E), e1) * spow(np.cos(O), e2),
                  b * spow(np.cos(E), e1) * spow(np.sin(O), e2),
                  c * spow(np.sin(E), e1)], axis=-1)
    v00, v01, v10, v11 = V[:-1, :-1], V[:-1, 1:], V[1:, :-1], V[1:, 1:]
    tris = np.concatenate([np.stack([v00, v01, v11], -2).reshape(-1, 3, 3),
                           np.stack([v00, v11, v10], -2).reshape(-1, 3, 3)])
    area = 0.5 * np.linalg.norm(np.cross(tris[:, 1] - tris[:, 0], tris[:, 2] - tris[:, 0]), axis=1)
    prob = area / area.sum()
    idx = rng.choice(tris.shape[0], size=n, p=prob)
    r1, r2 = rng.random(n), rng.random(n)
    s1 = np.sqrt(r1)
    bary = np.stack([1 - s1, s1 * (1 - r2), s1 * r2], axis=1)
    x = np.einsum("mk,mki->mi", bary, tris[idx])
    for _ in range(30):
        F, g, _ = _sq_implicit(x, axes, e1, e2)
        x = x - ((F - 1.0) / np.sum(g * g, 1))[:, None] * g
    _, g, h = _sq_implicit(x, axes, e1, e2)
    nrm, k1, v1, k2, v2 = _shape_operator_from_implicit(g, h)
    k1 = np.clip(k1, -kappa_cap, kappa_cap)
    k2 = np.clip(k2, -kappa_cap, kappa_cap)
    k1 = np.where(np.abs(k1) < 1e-6, 0.0, k1)
    k2 = np.where(np.abs(k2) < 1e-6, 0.0, k2)
    pts = x + rng.normal(0.0, noise, size=x.shape) if noise > 0.0 else x
    return pts, nrm, coeffs_from_shape_operator(nrm, k1, v1, k2, v2)


def plane_patch(n: int, seed: int, extent: float = 1.0):
    """Points on z = 0 with normals +z and zero coefficients."""
    rng = _rng(seed)
    xy = (rng.random((n, 2)) * 2.0 - 1.0) * extent
    pts = np.concatenate([xy, np.zeros((n, 1))], axis=1)
    nrm = np.tile([0.0, 0.0, 1.0], (n, 1))
    return pts, nrm, np.zeros((n, 6))


def cylinder_cloud(n: int, seed: int, radius: float = 0.5, half_len: float = 1.0, inward: bool = False):
    """Points on a cylinder about the z axis with exact normals (outward, or
    inward for ``inward=True``) and the cylinder's curvatures (-1/radius around,
    0 along; signs flip with the normal)."""
    rng = _rng(seed)
    ang = rng.random(n) * 2.0 * math.pi
    z = (rng.random(n) * 2.0 - 1.0) * half_len
    nrm = np.stack([np.cos(ang), np.sin(ang), np.zeros(n)], axis=1)
    pts = radius * nrm + np.stack([np.zeros(n), np.zeros(n), z], axis=1)
    e_around = np.stack([-np.sin(ang), np.cos(ang), np.zeros(n)], axis=1)
    e_along = np.tile([0.0, 0.0, 1.0], (n, 1))
    k_around = np.full(n, -1.0 / radius)
    if inward:
        nrm = -nrm
        k_around = -k_around
    return pts, nrm, coeffs_from_shape_operator(nrm, k_around, e_around, np.zeros(n), e_along)


def uniform_queries(q: int, seed: int, lo: float = -1.5, hi: float = 1.5) -> np.ndarray:
    return lo + (hi - lo) * _rng(seed).random((q, 3))


def grid_queries(res: int, lo: float = -1.6, hi: float = 1.6) -> np.ndarray:
    """res^3 nodes of linspace(lo, hi, res)^3, x fastest (row-major z, y, x)."""
    g = np.linspace(lo, hi, res)
    zz, yy, xx = np.meshgrid(g, g, g, indexing="ij")
    return np.stack([xx.ravel(), yy.ravel(), zz.ravel()], axis=1)


def grid_query_index(idx: np.ndarray, res: int, lo: float = -1.6, hi: float = 1.6) -> np.ndarray:
    """Positions of grid nodes by flat index (same ordering as grid_queries)."""
    g = np.linspace(lo, hi, res)
    idx = np.asarray(idx, dtype=np.int64)
    return np.stack([g[idx % res], g[(idx // res) % res], g[idx // (res * res)]], axis=1)


def camera_rays(width: int, height: int, seed: int, dist: float = 3.0, fov_deg: float = 45.0):
    """Pinhole camera on a seeded direction at distance ``dist`` looking at the
    origin, up = +z, vertical field of view ``fov_deg``; one ray per pixel
    centre.  Returns (origins, unit directions), row-major pixels."""
    rng = _rng(seed)
    d = rng.normal(size=3)
    d[2] = abs(d[2]) * 0.5
    d /= np.linalg.norm(d)
    eye = dist * d
    fwd = -d
    right = np.cross(fwd, [0.0, 0.0, 1.0])
    right /= np.linalg.norm(right)
    up = np.cross(right, fwd)
    th = math.tan(math.radians(fov_deg) / 2.0)
    aspect = width / height
    px = ((np.arange(width) + 0.5) / width * 2.0 - 1.0) * th * aspect
    py = (1.0 - (np.arange(height) + 0.5) / height * 2.0) * th
    PY, PX = np.meshgrid(py, px, indexing="ij")
    dirs = fwd + PX[..., None] * right + PY[..., None] * up
    dirs = (dirs / np.linalg.norm(dirs, axis=-1, keepdims=True)).reshape(-1, 3)
    org = np.broadcast_to(eye, dirs.shape).copy()
    return org, dirs
