"""Sampling a level set of phi with normals (Sec. 6, "Morphological
operations"): the oracle.

TEST INFRASTRUCTURE ONLY (as the rest of `oracle/`): numpy plus the FP64
oracle's phi and gradient; shares nothing with the CUDA library.

The paper erodes a point cloud by sampling the -c level set of phi, taking
the normals at the moved points from grad phi, re-fitting tori (its network)
and sampling the +c level set of the new SDF.  Without the network the
re-fit is out of reach; the sampling is not.  Readings (the paper does not
say how it samples): each seed x_0 (for erosion, the cloud's points) moves by
Newton steps along the gradient,

    x_{k+1} = x_k - (phi(x_k) - c) grad phi(x_k) / |grad phi(x_k)|^2,

a seed stops moving once |phi - c| <= tol (or its gradient vanishes), for at
most max_iter steps; the returned normal is grad phi / |grad phi| at the final
point and the residual phi - c there.  Lambda as in the blend (GLOBAL).
"""
from __future__ import annotations

import numpy as np


def project_level_set(cloud, x0, level: float, max_iter: int = 10, tol: float = 0.0, C: float = 64.0,
                      path: bool = False):
    """(x, normals, residual) after at most max_iter Newton steps onto the
    `level` set of the oracle cloud's phi.  path=True also returns, per
    iterate k = 0..max_iter, the points x_k (max_iter + 1, Q, 3), their
    residuals phi - level and gradient norms |grad phi| (max_iter + 1, Q)."""
    x = np.array(x0, dtype=np.float64).reshape(-1, 3)
    xs, rs, gs = [], [], []
    for _ in range(max_iter):
        phi, g = cloud.grad_x(x, C=C)
        r = phi - level
        g2 = (g * g).sum(1)
        xs.append(x.copy())
        rs.append(r)
        gs.append(np.sqrt(g2))
        move = (np.abs(r) > tol) & (g2 > 1e-30)
        x[move] -= (r[move] / g2[move])[:, None] * g[move]
    phi, g = cloud.grad_x(x, C=C)
    gn = np.linalg.norm(g, axis=1, keepdims=True)
    out = (x, g / np.maximum(gn, 1e-30), phi - level)
    if path:
        xs.append(x.copy())
        rs.append(phi - level)
        gs.append(gn[:, 0])
        out = out + (np.stack(xs), np.stack(rs), np.stack(gs))
    return out
