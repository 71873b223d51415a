"""A reduced case of the dense-grid workload for profiler captures
(measurement tooling beside bench.py, not part of the library).

    python profile_case.py [--queries Q] [--launches K] [--warmup W]
    python profile_case.py --mode probe      # the unit-rate probe's readings

Builds the dense-grid cloud (ring torus, N = 100,000; or, with --cloud
superquadric, the sphere-tracing cloud of N = 262,144 curvature-form points)
and evaluates an evenly strided subset of Q nodes of the 256^3 grid over
[-1.6, 1.6]^3 (--grid-res, --extent) with sdf_query (or the gradient,
Laplacian and backward calls), W times
untimed and then K times, printing the device time of each call.  Used to give ncu a short, self-terminating run of the
same kernels the benchmark times.  --mode probe prints, for each of the
eight probes of sdf_probe_rates, the four readings of sdf_probe_timing (one
JSON line) and builds no cloud.
"""
from __future__ import annotations

import argparse
import os
import sys

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--queries", type=int, default=1 << 20)
    ap.add_argument("--launches", type=int, default=1)
    ap.add_argument("--warmup", type=int, default=1)
    ap.add_argument("--points", type=int, default=None, help="default 100,000 (torus) / 262,144 (superquadric)")
    ap.add_argument("--cloud", choices=["torus", "superquadric"], default="torus")
    ap.add_argument("--seed", type=int, default=None, help="cloud seed (default 1002 torus, 1003 superquadric)")
    ap.add_argument("--grid-res", type=int, default=256, help="query grid nodes per axis")
    ap.add_argument("--extent", type=float, default=1.6, help="query grid over [-extent, extent]^3")
    ap.add_argument("--mode", choices=["query", "grad", "backward", "laplacian", "radius", "probe", "sspd", "shc"],
                    default="query",
                    help="query: sdf_query; grad: sdf_query_grad; backward: sdf_query_grad then "
                         "sdf_backward_params (each call); laplacian: sdf_query_laplacian; radius: sdf_query "
                         "with SDF_LAMBDA_RADIUS and lambda = 10^3 / D; sspd / shc: sdf_query with the SSPD / "
                         "SHC baseline")
    ap.add_argument("--precision", type=int, default=0, help="sdf_precision of the query")
    ap.add_argument("--engine", type=int, default=0, help="sdf_engine of the query (0 auto, 1 ALU, 2 tensor)")
    args = ap.parse_args()

    import torch

    import paper_2607_16946_b300 as ptsdf
    import synth

    if args.mode == "probe":
        import ctypes
        import json
        from paper_2607_16946_b300 import _abi
        L = _abi.lib()
        names = ["sqrt", "rsqrt", "ex2", "fma", "rcp", "pair_direct", "pair_flat", "pair_curved"]
        out = {}
        for op, nm in enumerate(names):
            buf = (ctypes.c_double * 4)()
            _abi.check(L.sdf_probe_timing(op, buf))
            out[nm] = {"clock64_longest_cta_per_clk": buf[0], "globaltimer_union_per_clk": buf[1],
                       "event_per_sm_per_ns": buf[2], "event_per_clk": buf[2] / buf[3] if buf[3] else None,
                       "sm_ghz_measured": buf[3]}
        print(json.dumps(out), flush=True)
        return

    if args.cloud == "torus":
        args.points = args.points or 100_000
        p, n, a = synth.ring_torus(args.points, args.seed or 1002, R=1.0, r=0.35, noise=0.005, jitter_deg=2.0)
    else:
        args.points = args.points or 262_144
        p, n, a = synth.superquadric(args.points, args.seed or 1003)
    cloud = ptsdf.Cloud(p, n, a)
    res = args.grid_res
    g = torch.linspace(-args.extent, args.extent, res, device="cuda", dtype=torch.float64)
    zz, yy, xx = torch.meshgrid(g, g, g, indexing="ij")
    x = torch.stack([xx.reshape(-1), yy.reshape(-1), zz.reshape(-1)], 1).to(torch.float32)
    stride = max(1, x.shape[0] // args.queries)
    x = x[::stride][: args.queries].contiguous()
    phi = torch.empty(x.shape[0], device="cuda")
    G = torch.ones(x.shape[0], device="cuda")
    lam = cloud.paper_lambda() if args.mode == "radius" else 0.0

    def call():
        nonlocal phi
        if args.mode == "query":
            cloud.query(x, out=phi, precision=args.precision, engine=args.engine)
        elif args.mode == "radius":
            cloud.query(x, out=phi, lambda_mode=ptsdf.SDF_LAMBDA_RADIUS, fixed_lambda=lam)
        elif args.mode in ("sspd", "shc"):
            cloud.query(x, out=phi, formula=ptsdf.SDF_FORMULA_SSPD if args.mode == "sspd" else ptsdf.SDF_FORMULA_SHC)
        elif args.mode == "laplacian":
            phi, _, _ = cloud.query_laplacian(x)
        else:
            phi, _, saved = cloud.query_grad(x)
            if args.mode == "backward":
                cloud.backward_params(x, saved, G)

    for _ in range(args.warmup):
        call()
    torch.cuda.synchronize()
    for i in range(args.launches):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        call()
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        print(f"call {i}: Q={x.shape[0]} N={args.points} {ms:.3f} ms "
              f"{x.shape[0] * args.points / ms / 1e6:.1f} Gpairs/s", flush=True)
    assert cloud.device_status() == 0
    assert bool(torch.isfinite(phi).all())


if __name__ == "__main__":
    main()
