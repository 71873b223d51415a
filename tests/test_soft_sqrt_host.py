"""The FMA-pipe square root of the tensor-core epilogue (sqrt2_newton in
csrc/device_common.cuh), on the CPU: Lomont's bit-level estimate of 1/sqrt
and two Newton steps (the integer and the steps' constants read from the
source; the centred constants of the build option too) emulated in FP32,
against the exact square root over one full period of the estimate (every
seventh float in [1, 4)) and a sweep of 40 decades.  The GPU self-test
(tests/test_gpu_tensor.py) checks the device code against CUDA's sqrtf."""
import os
import re

import numpy as np

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2607_16946_b300", "csrc",
                   "device_common.cuh")


def constants():
    """The magic integer and the two steps' constants, read from the source."""
    body = open(SRC).read().split("f32x2 sqrt2_newton(", 1)[1].split("\n}\n", 1)[0]
    magic = int(re.search(r"0x([0-9a-f]+) - \(__float_as_int", body).group(1), 16)
    src = open(SRC).read()
    steps = [float(re.search(r"#define PTSDF_SQRT_%s ([0-9.]+)f" % c, src).group(1)) for c in ("C1", "C2")]
    assert "PTSDF_SQRT_C1, PTSDF_SQRT_C1" in body and "PTSDF_SQRT_C2, PTSDF_SQRT_C2" in body
    return magic, steps


def emulate(x, steps=None):
    """The device's operations in FP32: y*y, fma(-x/2, y*y, c) (one rounding),
    y * that, and x * y."""
    f = np.float32
    magic, cs = constants()
    cs = cs if steps is None else steps
    x = np.maximum(x.astype(f), f(1e-30))
    y = (np.int32(magic) - (x.view(np.int32) >> 1)).view(f)
    nh = (x * f(-0.5)).astype(f)
    for c in cs:
        yy = (y * y).astype(f)
        t = (nh.astype(np.float64) * yy.astype(np.float64) + np.float64(f(c))).astype(f)
        y = (y * t).astype(f)
    return (x * y).astype(f)


def rel_err(x, **kw):
    return emulate(x, **kw).astype(np.float64) / np.sqrt(np.maximum(x, np.float32(1e-30)).astype(np.float64)) - 1.0


def test_two_newton_steps_stay_within_5e_6():
    magic, cs = constants()
    assert magic == 0x5f375a86 and cs == [1.5, 1.5]
    period = np.arange(0x3f800000, 0x40800000, 7, dtype=np.uint32).view(np.float32)   # [1, 4)
    sweep = np.float32(10.0) ** np.linspace(-20, 20, 200001).astype(np.float32)
    for x in (period, sweep):
        # one-sided (each step approaches 1/sqrt(x) from below), up to 1.5 (1.75e-3)^2
        rel = rel_err(x)
        assert rel.max() < 5e-7 and 4e-6 < -rel.min() <= 5e-6, (rel.min(), rel.max())
        assert np.abs(rel_err(x, steps=[1.5])).max() > 1e-3
        # the centred constants of the build option: both signs, within 8e-7
        cen = rel_err(x, steps=[1.5009, 1.5000006])
        assert 5e-7 < np.abs(cen).max() <= 8e-7 and cen.min() < -5e-7 and cen.max() > 5e-7


def test_zero_is_clamped_not_nan():
    out = emulate(np.array([0.0, 1e-38], np.float32))
    assert np.all(np.isfinite(out)) and np.all(out <= 1.1e-15)
