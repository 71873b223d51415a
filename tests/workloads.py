"""Seeded workloads used by the GPU parity tests (same recipes as bench.py).

Config k uses seed 1000 + k.  Shapes, sizes and distributions follow the
benchmark configurations: a Fibonacci sphere (N = 4,096, Q = 32,768 uniform
in [-1.5, 1.5]^3), a noisy ring torus (N = 100,000, R = 1, r = 0.35,
sigma = 0.005, 2-degree vMF normal jitter) queried on the 256^3 grid over
[-1.6, 1.6]^3, and a mixed cloud that exercises both record forms.
"""
import numpy as np

import synth

TOL_REL = 1e-4     # FP32 tolerance: |phi_gpu - phi_oracle| <= 1e-4 * AABB diagonal


def f32(*arrays):
    """Round to float32 values (kept as float64) so that the GPU and the
    oracle evaluate exactly the same inputs."""
    out = tuple(np.asarray(a, np.float32).astype(np.float64) for a in arrays)
    return out if len(out) > 1 else out[0]


def aabb_diag(p):
    return float(np.linalg.norm(p.max(0) - p.min(0)))


def config1():
    p, n, a = synth.sphere_fibonacci(4096, 1001)
    x = synth.uniform_queries(32768, 1001, -1.5, 1.5)
    return f32(p, n, a, x)


def config2_cloud():
    return f32(*synth.ring_torus(100_000, 1002, R=1.0, r=0.35, noise=0.005, jitter_deg=2.0))


GRID_RES = 256


def mixed_cloud(seed=77, rounded=True):
    """Plane, cylinder, large-radius sphere cap and random-coefficient points
    (both torus record forms, all sign cases, tilt and shift), N = 1,000 (not
    a multiple of the 32-record tile).  rounded=False keeps the float64 values
    (exactly rank-one cylinder forms, unit normals)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    p1, n1, a1 = synth.plane_patch(150, seed + 1)
    p1 = p1 * 0.8 + np.array([0.0, 0.0, -1.0])
    p2, n2, a2 = synth.cylinder_cloud(250, seed + 2, radius=0.4, half_len=0.8)
    # cap of a radius-60 sphere (r = 60 exceeds 8 AABB diagonals: kappa form)
    uv = rng.uniform(-0.8, 0.8, size=(200, 2))
    zc = np.sqrt(60.0 ** 2 - np.sum(uv ** 2, 1))
    n3 = np.concatenate([uv, zc[:, None]], 1) / 60.0
    p3 = np.concatenate([uv, (zc - 60.0 + 0.5)[:, None]], 1)
    a3 = np.zeros((200, 6))
    a3[:, 4] = a3[:, 5] = -0.5 / 60.0
    m = 1000 - p1.shape[0] - p2.shape[0] - p3.shape[0]
    p4 = rng.uniform(-1.0, 1.0, size=(m, 3))
    n4 = synth._unit(rng.normal(size=(m, 3)))
    a4 = np.zeros((m, 6))
    a4[:, 0] = rng.normal(size=m) * 0.02
    a4[:, 1:3] = rng.normal(size=(m, 2)) * 0.2
    a4[:, 3:6] = rng.normal(size=(m, 3)) * 1.5
    a4[: m // 5, 3:6] *= 1e-3          # nearly flat: huge radii
    P = np.concatenate([p1, p2, p3, p4])
    N = np.concatenate([n1, n2, n3, n4])
    A = np.concatenate([a1, a2, a3, a4])
    perm = rng.permutation(P.shape[0])
    out = (P[perm], N[perm], A[perm])
    return f32(*out) if rounded else out
