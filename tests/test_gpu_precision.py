"""Packed-half weights (SDF_F16X2, SDF_BF16X2): the exponentials of a lane's
two queries evaluated by one packed exp2, everything else FP32.  Their error
against the FP64 oracle is measured and bounded here (it is stated per
configuration by the benchmark); gradients refuse them."""
import numpy as np
import pytest

import synth
from workloads import aabb_diag, config2_cloud, f32, mixed_cloud

pytestmark = pytest.mark.gpu

# max |phi - phi_oracle| / AABB diagonal allowed for each variant and cloud,
# about 3x the error measured on a B300 (max over the 3,000 queries of the
# test; dense-grid torus: F16X2 4.4e-7, BF16X2 7.1e-6; mixed cloud: F16X2
# 1.4e-4, BF16X2 6.9e-4; mixed cloud with weights log-uniform in [0.1, 10]:
# F16X2 5.1e-5, BF16X2 8.4e-4).  On the mixed cloud both exceed the FP32
# bar (1e-4): rounding the exponent A0 - L d to 11 (8) bits costs up to
# 2^-11 (2^-8) of |A0 - L d| in it, and the cloud's points spread their g_i
# widely within the screening length.
BOUNDS = {("f16x2", "torus"): 1.5e-6, ("bf16x2", "torus"): 2.5e-5,
          ("f16x2", "mixed"): 4.5e-4, ("bf16x2", "mixed"): 2.2e-3,
          ("f16x2", "mixed_weighted"): 1.6e-4, ("bf16x2", "mixed_weighted"): 2.6e-3}


@pytest.fixture(scope="module")
def ptsdf():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2607_16946_b300 import build
    build.build()
    import paper_2607_16946_b300 as m
    return m


@pytest.mark.parametrize("prec", ["f16x2", "bf16x2"])
@pytest.mark.parametrize("cloud", ["mixed", "torus"])
def test_packed_weights_error(ptsdf, oracle_mod, prec, cloud):
    import torch
    from paper_2607_16946_b300 import _abi
    p, n, a = mixed_cloud(41) if cloud == "mixed" else config2_cloud()
    x = f32(synth.uniform_queries(3000, 42, -1.6, 1.6))
    cl = ptsdf.Cloud(p, n, a)
    code = _abi.SDF_F16X2 if prec == "f16x2" else _abi.SDF_BF16X2
    got = cl.query(torch.as_tensor(x, dtype=torch.float32, device="cuda"), precision=code)
    f32r = cl.query(torch.as_tensor(x, dtype=torch.float32, device="cuda"))
    torch.cuda.synchronize()
    assert cl.device_status() == 0
    ref = oracle_mod.Cloud(p, n, a).phi(x)
    err = np.abs(got.cpu().numpy() - ref) / aabb_diag(p)
    err32 = np.abs(f32r.cpu().numpy() - ref) / aabb_diag(p)
    print(prec, cloud, "max", err.max(), "p99", np.quantile(err, 0.99), "fp32 max", err32.max())
    assert np.isfinite(err).all()
    assert err.max() <= BOUNDS[(prec, cloud)]
    assert err32.max() <= 1e-4


def test_gradients_refuse_packed_weights(ptsdf):
    import torch
    from paper_2607_16946_b300 import _abi
    p, n, a = mixed_cloud(43)
    cl = ptsdf.Cloud(p, n, a)
    with pytest.raises(ptsdf.SdfError):
        cl.query_grad(torch.zeros((10, 3), device="cuda"), precision=_abi.SDF_F16X2)
