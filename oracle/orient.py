"""Orientation repair of inconsistently oriented clouds (Sec. 6, "Orienting
inconsistently oriented point clouds"): the oracle.

TEST INFRASTRUCTURE ONLY (as the rest of `oracle/`): numpy plus the FP64
oracle's fit and gradient; shares nothing with the CUDA library.

One iteration, every point deciding from the same cloud:
  1. fit the tori of the current (points, normals, coefficients) and take
     grad phi at every point of the cloud (GLOBAL lambda);
  2. for each point i, n~_i = sum over its k nearest other points j of
     exp(-M_i(p_i - p_j)) grad phi(p_j), with the Mahalanobis length
     M_i(r) = sqrt(kmin^2 <r, v_min>^2 + kmax^2 <r, v_max>^2 + eps^2 <r, n_i>^2)
     from point i's principal curvatures and directions (v_max is the torus
     axis u, v_min = u x n*);
  3. flip n_i when <n_i, n~_i> < 0.  Without the paper's network the
     coefficients of a flipped point are those of the same quadratic patch
     written in the frame of -n_i (see flip_coefficients), so the flipped
     point's torus is the same torus with the opposite sign.
Repeat until no point flips or max_iter iterations.  Readings (the paper
leaves them open): k = 16 neighbours, ties to the lower index; eps = 1/D_k,
D_k the mean distance to the k nearest; FP64 throughout.
"""
from __future__ import annotations

import numpy as np

from . import Cloud, fit_record, frame, knn_mean_distance


def flip_coefficients(n, a):
    """Coefficients (a00, a01, a10, a11, a02, a20) of the patch
    f(s, t) = a00 + a10 s + a01 t + a11 s t + a20 s^2 + a02 t^2 over the frame
    (s, t) of n, re-expressed over the frame (s', t') of -n with height along
    -n: (s, t) = M (s', t'), f' = -f o M."""
    n = np.asarray(n, dtype=np.float64)
    s, t = frame(n)
    s2, t2 = frame(-n)
    M = np.array([[s2 @ s, t2 @ s], [s2 @ t, t2 @ t]])
    a00, a01, a10, a11, a02, a20 = [float(v) for v in a]
    lin = np.array([a10, a01]) @ M                 # coefficients of s', t'
    H = np.array([[a20, 0.5 * a11], [0.5 * a11, a02]])
    H2 = M.T @ H @ M
    return np.array([-a00, -lin[1], -lin[0], -2.0 * H2[0, 1], -H2[1, 1], -H2[0, 0]])


def knn_indices(points, k):
    """The k nearest other points of every point (ascending distance, ties to
    the lower index)."""
    p = np.asarray(points, dtype=np.float64)
    out = np.empty((len(p), k), dtype=np.int64)
    for i0 in range(0, len(p), 256):
        d = np.linalg.norm(p[i0:i0 + 256, None, :] - p[None], axis=2)
        d[np.arange(d.shape[0]), np.arange(i0, i0 + d.shape[0])] = np.inf
        order = np.lexsort((np.broadcast_to(np.arange(len(p)), d.shape), d), axis=1)
        out[i0:i0 + 256] = order[:, :k]
    return out


def orientation_step(points, normals, params, nbr, eps, C=64.0):
    """One iteration: returns (flip mask, <n_i, n~_i>)."""
    p = np.asarray(points, dtype=np.float64)
    cl = Cloud(p, normals, params)
    _, g = cl.grad_x(p, C=C)
    score = np.empty(len(p))
    for i in range(len(p)):
        f = fit_record(p[i], normals[i], params[i])
        u, ns = f["u"], f["nstar"]
        vmin = np.cross(u, ns)
        r = p[i] - p[nbr[i]]
        m = np.sqrt((f["kmin"] * (r @ vmin)) ** 2 + (f["kmax"] * (r @ u)) ** 2 + (eps * (r @ normals[i])) ** 2)
        nt = (np.exp(-m)[:, None] * g[nbr[i]]).sum(0)
        score[i] = normals[i] @ nt
    return score < 0.0, score


def orient(points, normals, params, k=16, max_iter=10, C=64.0):
    """Iterates orientation_step; returns (normals, params, flips per iteration)."""
    p = np.asarray(points, dtype=np.float64)
    nrm = np.asarray(normals, dtype=np.float64).copy()
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    prm = np.asarray(params, dtype=np.float64).copy()
    nbr = knn_indices(p, k)
    eps = 1.0 / knn_mean_distance(p, k)
    flips = []
    for _ in range(max_iter):
        flip, _ = orientation_step(p, nrm, prm, nbr, eps, C)
        flips.append(int(flip.sum()))
        if not flip.any():
            break
        for i in np.nonzero(flip)[0]:
            prm[i] = flip_coefficients(nrm[i], prm[i])
            nrm[i] = -nrm[i]
    return nrm, prm, flips
