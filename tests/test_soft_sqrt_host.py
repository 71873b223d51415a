"""The FMA-pipe square root of the tensor-core epilogue (sqrt2_newton<2> in
csrc/device_common.cuh), on the CPU: Lomont's bit-level estimate of 1/sqrt
(the magic integer read from the source) and two Newton steps emulated in
FP32, against the exact square root over one full period of the estimate
(every seventh float in [1, 4)) and a sweep of 40 decades.  The GPU self-test
(tests/test_gpu_tensor.py) checks the device code against CUDA's sqrtf."""
import os
import re

import numpy as np

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2607_16946_b300", "csrc",
                   "device_common.cuh")


def magic():
    body = open(SRC).read().split("f32x2 sqrt2_newton(", 1)[1].split("\n}\n", 1)[0]
    return int(re.search(r"0x([0-9a-f]+) - \(__float_as_int", body).group(1), 16)


def emulate(x, steps=2):
    f = np.float32
    x = np.maximum(x.astype(f), f(1e-30))
    y = (np.int32(magic()) - (x.view(np.int32) >> 1)).view(f)
    nh = (x * f(-0.5)).astype(f)
    for _ in range(steps):
        y = (y * (f(1.5) + nh * (y * y))).astype(f)
    return (x * y).astype(f)


def test_two_newton_steps_stay_within_5e_6():
    period = np.arange(0x3f800000, 0x40800000, 7, dtype=np.uint32).view(np.float32)   # [1, 4)
    sweep = np.float32(10.0) ** np.linspace(-20, 20, 200001).astype(np.float32)
    for x in (period, sweep):
        rel = np.abs(emulate(x).astype(np.float64) / np.sqrt(x.astype(np.float64)) - 1.0)
        assert 4e-6 < rel.max() <= 5e-6, rel.max()      # the quadratic convergence bound, 1.5 (1.75e-3)^2
        assert np.abs(emulate(x, 1).astype(np.float64) / np.sqrt(x.astype(np.float64)) - 1.0).max() > 1e-3


def test_zero_is_clamped_not_nan():
    out = emulate(np.array([0.0, 1e-38], np.float32))
    assert np.all(np.isfinite(out)) and np.all(out <= 1.1e-15)
