"""The pruned prepasses (bounding spheres of 64-point Morton tiles) must
return exactly the d_max, d_min and farthest point of the full scan.

Large batches (at least two waves of query blocks) take the pruned prepass
with a thread per query, smaller ones the pruned prepass with a warp per
query, and an explicit split_n the point-split full scan.  The same queries
evaluated these ways must give bit-identical per-query statistics (lambda_x
log2 e and the shift term, saved by sdf_query_grad) and phi within rounding
of the pair-loop split; against the oracle on a sample as well.
"""
import numpy as np
import pytest

import synth
from workloads import TOL_REL, aabb_diag, config2_cloud, f32

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ptsdf():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2607_16946_b300 import build
    build.build()
    import paper_2607_16946_b300 as m
    return m


@pytest.mark.parametrize("which", ["torus", "superquadric"])
def test_pruned_prepass_exact(ptsdf, oracle_mod, which):
    import torch
    if which == "torus":
        p, n, a = config2_cloud()
        lo, hi = -1.6, 1.6
    else:
        p, n, a = f32(*synth.superquadric(60_000, 77, grid=384))
        lo, hi = -1.5, 1.5
    cl = ptsdf.Cloud(p, n, a)
    q = 320_000                        # 625 blocks of 512 queries: the pruned path
    x = torch.as_tensor(f32(synth.uniform_queries(q, 88, lo, hi)), dtype=torch.float32, device="cuda")
    phi_big, g_big, s_big = cl.query_grad(x)
    phi_q = cl.query(x)
    torch.cuda.synchronize()
    for start in (0, 150_000, q - 3000):
        xs = x[start:start + 3000].contiguous()      # 6 blocks: the warp-per-query prepass
        for kw in ({}, {"split_n": 4}):              # and the point-split full scan
            phi_s, g_s, s_s = cl.query_grad(xs, **kw)
            torch.cuda.synchronize()
            assert torch.equal(s_big[start:start + 3000, 3:5], s_s[:, 3:5])   # L and L d_min bit for bit
            # the pair loop splits the points differently for the batch sizes:
            # same terms, different FP32 summation order
            assert (phi_big[start:start + 3000] - phi_s).abs().max().item() <= 2e-5
            assert (g_big[start:start + 3000] - g_s).abs().max().item() <= 1e-3   # the gradient tolerance
            phi_b = cl.query(xs, **kw)                # the query's prepass (no farthest index)
            torch.cuda.synchronize()
            assert (phi_q[start:start + 3000] - phi_b).abs().max().item() <= 2e-5
    assert cl.device_status() == 0
    xs = x[::1000].cpu().numpy().astype(np.float64)
    ref = oracle_mod.Cloud(p, n, a).phi(xs)
    assert np.abs(phi_q[::1000].cpu().numpy() - ref).max() <= TOL_REL * aabb_diag(p)
