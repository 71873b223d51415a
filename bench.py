#!/usr/bin/env python
"""Benchmark of the points-as-tori SDF query path on B300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Workload (the dense-grid configuration): a ring torus cloud, N = 100,000
area-uniform samples (R = 1, r = 0.35, Gaussian noise sigma = 0.005, normals
jittered by 2-degree von Mises-Fisher noise, coefficients from the analytic
principal curvatures), queried at every node of the 256^3 grid over
[-1.6, 1.6]^3 (Q = 16,777,216 queries, 1.678e12 (query, point) pairs per step).
A step is one sdf_query over the whole grid: prepass (d_max per query) and
the pair loop.  FP32, lambda_x = C / sigma_x with C = 64.

One JSON line on stdout (rank 0):
  value   whole-job Gpairs/s (device-timed, inputs resident in HBM)
  e2e     the same metric through sdf_query_host with pinned host buffers,
          host<->device copies inside the timed region
  roofline  the pair-loop kernel's pairs/s from CUDA events on its stream
          against the instruction-issue ceiling of the SM array
  cpu_baseline  the FP64 CPU oracle on a bounded sample of the same workload
Under torchrun every rank evaluates its own full grid (weak scaling); the
timed region is bracketed by barriers and the slowest rank's time is used.
"""
from __future__ import annotations

import argparse
import ctypes
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "SDF Gpairs/s and queries/s at N=100k (FP32 vs mixed vs served); p50/p99 latency"
UNIT = "Gpairs/s"
N_POINTS = 100_000
GRID_RES = 256
SEED = 1002
WORKLOAD = ("dense_grid: ring torus N=100000 (R=1, r=0.35, noise 0.005, 2deg vMF normals, analytic "
            "curvature coefficients), Q=256^3 grid over [-1.6,1.6]^3")
# Issue-slot ceiling of the pair loop.  Algorithmic work per pair (direct torus
# form): 25 FP32 instructions (two 3-vector differences, two dots, the
# perpendicular component and its norm, the tube distance, the blend and two
# accumulations) + 4 MUFU (three square roots and exp2) = 29 issue slots; an SM
# issues 4 warp-instructions (128 thread-instructions) per clock.  The MUFU pipe
# sustains about 32 results/clk/SM on this part (ncu: 4 MUFU/pair keep it at 40%
# while issue is at 82%), so issue, not MUFU, binds.
INSTR_PER_PAIR = 29
THREAD_INSTR_PER_SM_CLK = 128
FALLBACK_MAX_SM_MHZ = 2032.0


def make_cloud():
    import synth
    return synth.ring_torus(N_POINTS, SEED, R=1.0, r=0.35, noise=0.005, jitter_deg=2.0)


def grid_device(torch, device):
    g = torch.linspace(-1.6, 1.6, GRID_RES, device=device, dtype=torch.float64)
    zz, yy, xx = torch.meshgrid(g, g, g, indexing="ij")
    return torch.stack([xx.reshape(-1), yy.reshape(-1), zz.reshape(-1)], 1).to(torch.float32).contiguous()


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.thread.join(timeout=5)

    def summary(self):
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [s.strip() for s in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def kernel_source_sha() -> str:
    h = hashlib.sha256()
    for f in ("query.cu", "device_common.cuh", "internal.h"):
        with open(os.path.join(ROOT, "paper_2607_16946_b300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def committed_traffic():
    """dram bytes per pair-loop launch from the committed ncu summary, if it was
    taken on the current kernel source; else None."""
    path = os.path.join(ROOT, "profiles", "fwd_dense_grid_traffic.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
    except (OSError, ValueError):
        return None
    if d.get("kernel_sha") != kernel_source_sha():
        return None
    return d.get("dram_bytes_per_launch")


def _timed_oracle_sample(cl, rng, threads, target_s: float, chunk: int = 2048, max_chunks: int = 64):
    """Runs seeded chunks of grid queries through the oracle until about
    target_s seconds have passed; returns (queries, seconds)."""
    import synth
    done, t_total = 0, 0.0
    for _ in range(max_chunks):
        xs = synth.grid_query_index(rng.integers(0, GRID_RES ** 3, size=chunk), GRID_RES)
        t0 = time.perf_counter()
        cl.phi(xs, threads=threads)
        t_total += time.perf_counter() - t0
        done += chunk
        if t_total >= target_s:
            break
    return done, t_total


def cpu_baseline(points, normals, params, target_s: float = 12.0):
    """FP64 CPU oracle on a bounded, seeded sample of grid queries."""
    import oracle
    threads = oracle.default_threads()
    cl = oracle.Cloud(points, normals, params)
    rng = np.random.Generator(np.random.PCG64(SEED))
    m, dt = _timed_oracle_sample(cl, rng, threads, target_s)
    return {"value": m * N_POINTS / dt / 1e9, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"{m} seeded grid nodes of the 256^3 grid x all {N_POINTS} points, FP64, "
                      f"{threads} threads, {dt:.1f} s"}


def run_reference(args, rank, world):
    """The oracle as it stands on the host cores, same workload and metric."""
    if rank != 0:
        return
    import oracle
    import synth
    p, n, a = make_cloud()
    cl = oracle.Cloud(p, n, a)
    threads = oracle.default_threads()
    rng = np.random.Generator(np.random.PCG64(SEED + 7))
    for _ in range(args.warmup):
        _timed_oracle_sample(cl, rng, threads, 1.0, max_chunks=1)
    m, dt = 0, 0.0
    for _ in range(args.steps):           # each step: about 6 s of seeded grid queries
        mi, ti = _timed_oracle_sample(cl, rng, threads, 6.0)
        m += mi
        dt += ti
    m_step = m // args.steps
    value = m * N_POINTS / dt / 1e9
    sample_desc = f"each step about {m_step} seeded grid nodes x all {N_POINTS} points, FP64, {threads} threads"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "N": N_POINTS, "Q": GRID_RES ** 3, "C": 64, "lambda": "global"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": sample_desc},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args, rank, world, local):
    import torch

    import paper_2607_16946_b300 as ptsdf
    from paper_2607_16946_b300 import _abi, dist

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    L = _abi.lib()
    p, n, a = make_cloud()
    cloud = ptsdf.Cloud(p, n, a)
    x = grid_device(torch, dev)
    q = x.shape[0]
    phi = torch.empty(q, device=dev, dtype=torch.float32)
    stream = torch.cuda.current_stream(dev)
    pairs_per_step = q * N_POINTS

    for _ in range(args.warmup):
        cloud.query(x, out=phi)
    torch.cuda.synchronize(dev)
    assert cloud.device_status() == 0, "kernel reported a fault during warm-up"

    # ---- device-timed region ------------------------------------------------
    L.sdf_profile_enable(1)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        dist.barrier()
        torch.cuda.synchronize(dev)
        ev0.record(stream)
        for _ in range(args.steps):
            cloud.query(x, out=phi)
        ev1.record(stream)
        torch.cuda.synchronize(dev)
        dist.barrier()
    L.sdf_profile_enable(0)
    elapsed_s = dist.max_over_ranks(ev0.elapsed_time(ev1) / 1e3, device=dev if world > 1 else None)
    prof = {}
    launches_total = 0
    for name, kid in _abi.KERNEL_IDS.items():
        cnt, ms = ctypes.c_int64(), ctypes.c_double()
        _abi.check(L.sdf_profile_read(kid, ctypes.byref(cnt), ctypes.byref(ms)))
        if cnt.value:
            prof[name] = {"launches": cnt.value, "ms": ms.value}
            launches_total += cnt.value
    assert cloud.device_status() == 0, "kernel reported a fault in the timed region"

    # ---- end to end through the host-buffer call ----------------------------
    hx = torch.empty((q, 3), dtype=torch.float32, pin_memory=True)
    hx.copy_(x.cpu())
    hphi = torch.empty(q, dtype=torch.float32, pin_memory=True)
    hxp = ctypes.c_void_p(hx.data_ptr())
    hpp = ctypes.c_void_p(hphi.data_ptr())
    opts = _abi.make_opts()
    sptr = ctypes.c_void_p(stream.cuda_stream)
    _abi.check(L.sdf_query_host(cloud.handle, hxp, q, hpp, ctypes.byref(opts), sptr))
    dist.barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        _abi.check(L.sdf_query_host(cloud.handle, hxp, q, hpp, ctypes.byref(opts), sptr))
    e2e_s = dist.max_over_ranks(time.perf_counter() - t0, device=dev if world > 1 else None)
    dist.barrier()
    finite = bool(torch.isfinite(hphi).all())

    if rank != 0:
        return
    value = world * pairs_per_step * args.steps / elapsed_s / 1e9
    cs = clk.summary()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    fmax = cs["sm_max_mhz"] or FALLBACK_MAX_SM_MHZ
    peak = sms * fmax * 1e6 * THREAD_INSTR_PER_SM_CLK / INSTR_PER_PAIR / 1e9
    fwd = prof.get("fwd", {"launches": 0, "ms": float("nan")})
    per_launch_s = fwd["ms"] / max(fwd["launches"], 1) / 1e3
    achieved = pairs_per_step / per_launch_s / 1e9
    traffic = committed_traffic()
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": elapsed_s / args.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "N": N_POINTS, "Q": q, "C": 64, "lambda": "global",
                   "precision": "fp32", "parallelism": f"replicas{world}" if world > 1 else "single",
                   "l2": "inputs larger than L2 (queries 201 MB, phi 67 MB); not flushed"},
        "queries_per_s": world * q * args.steps / elapsed_s,
        "e2e": {"value": world * pairs_per_step * args.steps / e2e_s / 1e9, "unit": UNIT,
                "h2d_bytes_per_step": q * 12, "d2h_bytes_per_step": q * 4},
        "gpu_launches": launches_total,
        "kernels": prof,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": UNIT, "frac": achieved / peak,
                     "traffic": traffic,
                     "peak_basis": f"issue ceiling: {sms} SMs x {fmax:.0f} MHz x {THREAD_INSTR_PER_SM_CLK} "
                                   f"thread-instr/clk / {INSTR_PER_PAIR} instr per pair (derived from unit "
                                   f"counts and the max SM clock, not measured)"},
        "clocks": cs,
        "outputs_finite": finite,
    }
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(p, n, a)
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true", help="omit the CPU oracle leg")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    from paper_2607_16946_b300 import dist
    rank, world, local = dist.init()
    if world != args.gpus:
        print(f"warning: --gpus {args.gpus} but WORLD_SIZE={world}", file=sys.stderr)
    try:
        if args.impl == "reference":
            run_reference(args, rank, world)
        else:
            run_ours(args, rank, world, local)
    finally:
        dist.finalize()


if __name__ == "__main__":
    main()
