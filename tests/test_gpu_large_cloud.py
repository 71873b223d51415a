"""Accuracy of the FP32 sums on a cloud of 2^21 = 2,097,152 points.

Every query's W and S are sums over two million weights, all in FP32:
accumulated per epilogue lane in two running halves (tensor-core engine) or
per 32-point tile (FP32 units), per point chunk, and in the fixed-order merge
of the chunks' partials.  Against the FP64 oracle on 512 queries (half of them
near the surface), on both engines and with explicit point chunks (the merge
of 64 partials): the FP32 bar (1e-4 x AABB diagonal) holds, so the merge needs
no FP64.  The measured errors are printed (pytest -s).
"""
import numpy as np
import pytest

import synth
from workloads import TOL_REL, aabb_diag, f32

pytestmark = pytest.mark.gpu

N_LARGE = 1 << 21


@pytest.fixture(scope="module")
def ptsdf():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2607_16946_b300 import build
    build.build()
    import paper_2607_16946_b300 as m
    return m


@pytest.fixture(scope="module")
def large(ptsdf, oracle_mod):
    p, n, a = f32(*synth.ring_torus(N_LARGE, 71, R=1.0, r=0.35, noise=0.005, jitter_deg=2.0))
    rng = np.random.Generator(np.random.PCG64(72))
    near = p[rng.choice(len(p), size=256, replace=False)] + rng.normal(0.0, 0.02, size=(256, 3))
    x = f32(np.concatenate([synth.uniform_queries(256, 73, -1.6, 1.6), near]))
    ref = oracle_mod.Cloud(p, n, a).phi(x)
    return p, n, a, x, ref


@pytest.mark.parametrize("engine,split", [(2, 0), (1, 0), (2, 64), (1, 64)])
def test_two_million_points(ptsdf, large, engine, split):
    import torch
    p, n, a, x, ref = large
    cl = ptsdf.Cloud(p, n, a)
    got = cl.query(torch.as_tensor(x, device="cuda"), engine=engine, split_n=split)
    torch.cuda.synchronize()
    assert cl.device_status() == 0
    err = np.abs(got.cpu().numpy().astype(np.float64) - ref) / aabb_diag(p)
    print(f"N={N_LARGE} engine={engine} split={split}: max |err| / diag = {err.max():.2e}, "
          f"p99 {np.quantile(err, 0.99):.2e}")
    assert err.max() <= TOL_REL
