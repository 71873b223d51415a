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
          against the ceiling of the SM array's MUFU (XU) pipe, which
          binds: three square roots and one exp2 per pair
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
# Ceilings of the pair loop, per SM and clock.
#  FP32-unit loop, direct torus form: 25 FP32 operations (two 3-vector
#    differences, two dots, the perpendicular component and its norm, the tube
#    distance, the blend and two accumulations), issued as .f32x2 for two
#    points at a time, + 4 MUFU.
#  MUFU (XU pipe): sdf_probe_rates measures, on the box, the single
#    operations (on B300 sqrt / rsqrt / rcp.approx 16.0 results per SM per
#    clock, ex2.approx 32.0, timed over the union of each SM's CTA windows and
#    confirmed by CUDA events and by ncu's XU instruction counts) and the
#    per-pair mixes as dependent chains.  The FP32-unit loop's direct pair
#    needs three square roots (|x - p|, the axis distance, the tube distance)
#    and one exp2: 3 x 8 + 4 = 28 XU cycles per 32 pairs per SM sub-partition,
#    4.571 pairs per SM per clock, which the measured mix matches, below that
#    loop's FMA-pipe ceiling (124 / 25 = 4.96).
#  FMA pipe: 128 FP32 lanes per SM (sdf_probe_rates: 124.1 results per clock);
#    an .f32x2 instruction occupies it for two operations.
FP32_PER_PAIR = 25
NOMINAL_RATES = {"sqrt": 16.0, "rsqrt": 16.0, "ex2": 32.0, "fma": 128.0, "rcp": 16.0}
# probe mixes timed whole (the FP32-unit loop's three-root direct pair and
# the scalar curvature-form pairs); the single-operation sums equal them
PAIR_MIX_KEYS = {"direct": "pair_direct", "flat": "pair_flat", "curved": "pair_curved"}


def probe_rates(L):
    """Unit rates (results per SM per clock) measured by sdf_probe_rates, or
    the nominal ones if the probe fails."""
    buf = (ctypes.c_double * 8)()
    if L.sdf_probe_rates(buf) != 0:
        return dict(NOMINAL_RATES, source="nominal (probe failed)")
    return {"sqrt": buf[0], "rsqrt": buf[1], "ex2": buf[2], "fma": buf[3], "rcp": buf[4],
            "pair_direct": buf[5], "pair_flat": buf[6], "pair_curved": buf[7],
            "source": "measured (sdf_probe_rates)"}


def single_op_cost(rates, mix):
    """SM-clocks of special-function work of one pair with `mix` = (sqrt, rcp,
    exp2) operations: the sum of the single-operation costs."""
    return mix[0] / rates["sqrt"] + mix[1] / rates.get("rcp", rates["sqrt"]) + mix[2] / rates["ex2"]


def pair_ceiling(rates, fp32_per_pair):
    """FP32-unit loop, pairs per SM clock: the lower of the MUFU ceiling (its
    3 sqrt + 1 exp2 mix, measured whole, else the single-operation sum) and
    the FMA-pipe ceiling."""
    mufu = rates.get("pair_direct") or 1.0 / single_op_cost(rates, (3, 0, 1))
    issue = rates["fma"] / fp32_per_pair
    return min(mufu, issue), mufu, issue


# Tensor-core loop, per pair by record form: special-function operations
# (sqrt, rcp, ex2) and FP32 operations on the FMA pipe (the products come from
# the tensor cores).  Every form takes d = sqrt(d^2) on the FMA pipe by two
# Newton steps (8 of its FP32 operations, as .f32x2 pairs) and the rest of
# its arithmetic as .f32x2.  Direct: a, b -> rho (MUFU sqrt), the tube
# distance (MUFU sqrt), the weight's exp2; flat curvature form: one half-angle
# step (sqrt + rcp); curved: two square roots and, with the two steps over a
# common denominator, one reciprocal (26 FP32 operations).  The probe does
# not time these mixes whole, so their cost is the sum of the single-operation
# costs (the mixes it does time equal those sums).
TC_FORM_COST = {"direct": ((2, 0, 1), 17), "flat": ((1, 1, 1), 19), "curved": ((2, 1, 1), 26)}


def mix_cost(rates, form):
    """SM-clocks of special-function work per tensor-core pair of a record
    form: the sum of its single-operation costs."""
    return single_op_cost(rates, TC_FORM_COST[form][0])


def tc_pair_ceiling(rates, counts):
    """pairs per SM clock of the tensor-core loop over a cloud with `counts`
    points of each record form (pairs weighted by form): the lower of the
    MUFU and the FMA-pipe ceilings."""
    total = sum(counts.values())
    mufu_clk = sum(c * mix_cost(rates, f) for f, c in counts.items())
    fma_clk = sum(c * TC_FORM_COST[f][1] / rates["fma"] for f, c in counts.items())
    mufu, fma = total / mufu_clk, total / fma_clk
    return min(mufu, fma), mufu, fma
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


TC_SOURCES = ("query_tc.cu", "tc_common.cuh", "query_common.cuh", "device_common.cuh", "internal.h")
RADIUS_SOURCES = ("radius.cu", "sphere_index.h", "query_common.cuh", "device_common.cuh", "internal.h")


def kernel_source_sha(files=TC_SOURCES) -> str:
    """Hash of a kernel's sources with comments and blank space removed, so
    that a comment-only edit keeps a committed capture valid."""
    import re
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, "paper_2607_16946_b300", "csrc", f), encoding="utf-8") as fh:
            src = fh.read()
        src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
        src = re.sub(r"//[^\n]*", " ", src)
        h.update(" ".join(src.split()).encode())
    return h.hexdigest()[:16]


def _committed_capture(name, files):
    """A committed ncu summary (profiles/<name>) if it was taken on the
    current source of the kernel it describes; else None."""
    try:
        with open(os.path.join(ROOT, "profiles", name)) as fh:
            d = json.load(fh)
    except (OSError, ValueError):
        return None
    return d if isinstance(d, dict) and d.get("kernel_sha") == kernel_source_sha(files) else None


def committed_traffic():
    """dram bytes per step of the tensor-core pair loop (its launches of one
    query call) from the committed ncu summary, if it was taken on the
    current kernel source; else None."""
    d = _committed_capture("fwd_tc_dense_grid_traffic.json", TC_SOURCES)
    return d.get("dram_bytes_per_step") if d else None


def radius_issue_roofline(step_s, sms, fmax_mhz):
    """Issue-slot roofline of the radius-limited query on the 2^21-point
    workload: the warp-instructions ncu counted for one query call (both
    kernels), over the measured time of a call, against 4 warp-instructions
    per SM per clock.  None without a capture of the current source."""
    d = _committed_capture("radius_large_cloud_counts.json", RADIUS_SOURCES)
    if not d or not step_s:
        return None
    achieved = d["warp_instructions_per_call"] / step_s / 1e9
    peak = 4 * sms * fmax_mhz * 1e6 / 1e9
    return {"bound": "issue", "kernel": "k_radius_query + k_radius_fallback", "achieved": achieved,
            "peak": peak, "unit": "G warp-instructions/s", "frac": achieved / peak,
            "traffic": d.get("dram_bytes_per_call"),
            "peak_basis": f"{sms} SMs x {fmax_mhz:.0f} MHz x 4 warp-instructions per clock; "
                          f"{d['warp_instructions_per_call']:.4g} warp-instructions per call counted by ncu "
                          f"on this workload"}


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


SERVE_SEED = 1005
SERVE_SPLIT_GPAIRS = 100        # requests above 1e11 (query, point) pairs run as interleaved query chunks
SERVE_EXPRESS_GPAIRS = 10.0     # requests of at most 1e10 pairs (about three in four) on high-priority streams
SERVE_STREAMS = 8               # four express and four bulk streams for the eight slots


def make_serving_clouds(n_clouds: int, seed: int):
    """Serving configuration: clouds with N log-uniform in [2,048, 500,000] drawn
    from the sphere / ring torus / superquadric / ellipsoid generators."""
    import synth
    rng = np.random.Generator(np.random.PCG64(seed))
    gens = [lambda n, s: synth.sphere_fibonacci(n, s),
            lambda n, s: synth.ring_torus(n, s),
            lambda n, s: synth.superquadric(n, s, grid=256),
            lambda n, s: synth.ellipsoid(n, s)]
    out = []
    for i in range(n_clouds):
        n = int(np.exp(rng.uniform(np.log(2048), np.log(500_000))))
        out.append(gens[int(rng.integers(0, 4))](n, seed + 1 + i))
    return out


def run_served(args, dev, pair_rate_gps: float, policy: int = 0, clouds_np=None, precision: int = 0,
               load: float | None = None):
    """Continuous-batching run: Poisson arrivals at `load` (default
    --serve-load) x the measured pair
    rate, requests of Q log-uniform in [1,024, 4,194,304] against random
    resident clouds; kinds QUERY 70%, OFFSET 10%, UNION / DIFFERENCE 10%,
    TRACE_STEP 10%; every request at `precision` (0 FP32 with the tensor
    engine, 1 F16X2 packed-half weights).  Returns the latency / throughput
    summary."""
    import torch

    import paper_2607_16946_b300 as ptsdf
    from paper_2607_16946_b300 import serve as S

    if clouds_np is None:
        clouds_np = make_serving_clouds(args.serve_clouds, SERVE_SEED)
    clouds = [ptsdf.Cloud(*c) for c in clouds_np]
    ns = [c.n for c in clouds]
    rng = np.random.Generator(np.random.PCG64(SERVE_SEED))
    qmax = 4_194_304
    pool = torch.rand((qmax, 3), device=dev, generator=torch.Generator(device=dev).manual_seed(SERVE_SEED)) * 3.0 - 1.5
    dpool = torch.nn.functional.normalize(torch.randn((qmax, 3), device=dev), dim=1).contiguous()
    tpool = (torch.rand(qmax, device=dev) * 0.5).contiguous()
    reqs = []
    for _ in range(args.serve_requests):
        u = rng.random()
        kind = (S.SDF_REQ_QUERY if u < 0.8 else
                (S.SDF_REQ_UNION if u < 0.85 else S.SDF_REQ_DIFFERENCE) if u < 0.9 else S.SDF_REQ_TRACE_STEP)
        q = int(np.exp(rng.uniform(np.log(1024), np.log(qmax))))
        ca, cb = int(rng.integers(0, len(clouds))), int(rng.integers(0, len(clouds)))
        off = int(rng.integers(0, qmax - q + 1))
        pairs = q * ns[ca] + (q * ns[cb] if kind in (S.SDF_REQ_UNION, S.SDF_REQ_DIFFERENCE) else 0)
        reqs.append(dict(kind=kind, q=q, ca=ca, cb=cb, off=off, pairs=pairs, offset=0.05 if 0.7 <= u < 0.8 else 0.0))
    mean_pairs = float(np.mean([r["pairs"] for r in reqs]))
    load = args.serve_load if load is None else load
    rate = load * pair_rate_gps * 1e9 / mean_pairs          # requests per second
    arrivals = np.cumsum(rng.exponential(1.0 / rate, size=len(reqs)))
    srv = S.Server(mem_budget_bytes=16 << 30, max_inflight=8, n_streams=args.serve_streams, policy=policy,
                   starve_ms=2000, split_gpairs=SERVE_SPLIT_GPAIRS, express_gpairs=args.serve_express)
    ids = [srv.register(c) for c in clouds]
    outs = [torch.empty(r["q"], device=dev) for r in reqs]
    torch.cuda.synchronize(dev)
    tickets = [None] * len(reqs)
    t0 = time.perf_counter()

    def submitter():
        for i, r in enumerate(reqs):
            dt = arrivals[i] - (time.perf_counter() - t0)
            if dt > 0:
                time.sleep(dt)
            x = pool[r["off"]:r["off"] + r["q"]]
            kw = {}
            if r["kind"] == S.SDF_REQ_TRACE_STEP:
                kw = dict(dirs=dpool[r["off"]:r["off"] + r["q"]], t=tpool[r["off"]:r["off"] + r["q"]])
            tickets[i] = srv.submit(r["kind"], ids[r["ca"]], x, outs[i], cloud_id_b=ids[r["cb"]],
                                    offset=r["offset"], precision=precision, **kw)

    th = threading.Thread(target=submitter)
    th.start()
    stats = []
    for i in range(len(reqs)):
        while tickets[i] is None:
            time.sleep(0.0005)
        stats.append(srv.poll(tickets[i]))
    th.join()
    srv.shutdown()
    lat = np.array([(s["done_ns"] - s["arrive_ns"]) / 1e6 for s in stats])
    queue = np.array([(s["admit_ns"] - s["arrive_ns"]) / 1e6 for s in stats])
    service = np.array([(s["done_ns"] - s["admit_ns"]) / 1e6 for s in stats])
    span_s = (max(s["done_ns"] for s in stats) - min(s["arrive_ns"] for s in stats)) / 1e9
    total_pairs = float(sum(r["pairs"] for r in reqs))
    finite = all(bool(torch.isfinite(o).all()) for o in outs)
    # each request's time alone at the measured pair rate (at least 1 ms): the
    # slowdown says how much sharing the device delayed a request for its size,
    # and the largest request's time alone is a floor under the latency tail
    alone = np.array([max(r["pairs"] / (pair_rate_gps * 1e9) * 1e3, 1.0) for r in reqs])
    slow = lat / alone
    return {"value": total_pairs / span_s / 1e9, "unit": UNIT, "requests": len(reqs),
            "queries_per_s": float(sum(r["q"] for r in reqs)) / span_s,
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "queue_p50_ms": float(np.percentile(queue, 50)), "queue_p99_ms": float(np.percentile(queue, 99)),
            "service_p50_ms": float(np.percentile(service, 50)), "service_p99_ms": float(np.percentile(service, 99)),
            "slowdown_p50": float(np.percentile(slow, 50)), "slowdown_p99": float(np.percentile(slow, 99)),
            "largest_request_alone_ms": float(alone.max()),
            # the three requests of largest slowdown: pairs, latency, queueing, service (ms), chunks
            "worst_slowdown": [{"pairs": float(reqs[i]["pairs"]), "latency_ms": float(lat[i]),
                                "queue_ms": float(queue[i]), "service_ms": float(service[i]),
                                "chunks": int(stats[i]["chunks"])} for i in np.argsort(-slow)[:3]],
            "offered_load": load, "arrival_rate_per_s": rate, "mean_pairs_per_request": mean_pairs,
            "clouds": len(clouds), "points_total": int(sum(ns)), "outputs_finite": finite,
            "server": {"max_inflight": 8, "n_streams": args.serve_streams, "mem_budget_bytes": 16 << 30,
                       "express_pairs": args.serve_express * 1e9,
                       "policy": "smallest_first (starve 2 s)" if policy else "fifo",
                       "split_pairs": SERVE_SPLIT_GPAIRS * 1e9,
                       "requests_split": sum(1 for st in stats if st["chunks"] > 1)},
            "workload": f"{len(clouds)} resident clouds N~logU[2048,500000] (sphere/torus/superquadric/ellipsoid), "
                        f"{len(reqs)} requests Q~logU[1024,4194304], Poisson arrivals at "
                        f"{load} x measured capacity; "
                        f"{'FP32 (tensor engine)' if precision == 0 else 'F16X2 packed-half weights, FP32 sums'}"}


# Algorithmic FP32 work per pair of the other pair loops (direct torus form,
# counted from their arithmetic), against the FMA pipe's measured rate (the
# .f32x2 instructions issue half as often but occupy the pipe for both
# operations, and the pipe is what binds them): the gradient term is 54 FP32
# operations (distance, torus, grad g, weight, 13 accumulations) + 4 MUFU; the
# parameter-backward term is 47 FP32 (distance, weight, torus, 8 record
# derivatives) + 4 MUFU.  The a-priori per-pair counts of the hot-path plan
# are reported beside them: the gradient is the forward's 23 FP32 plus about
# 20 (43), the backward about twice the forward's 23 (46).
GRAD_FP32_PER_PAIR = 54
BWD_FP32_PER_PAIR = 47
GRAD_PLAN_FP32 = 43
BWD_PLAN_FP32 = 46


def _profile_window(L, abi):
    out = {}
    for name, kid in abi.KERNEL_IDS.items():
        cnt, ms = ctypes.c_int64(), ctypes.c_double()
        abi.check(L.sdf_profile_read(kid, ctypes.byref(cnt), ctypes.byref(ms)))
        if cnt.value:
            out[name] = {"launches": cnt.value, "ms": ms.value}
    return out


# FP32 operations per pair of the baselines' loop: x - p (3), d^2 (3), <x - p, n> (3), then SSPD
# the exponent, W and S (3); SHC d = d^2 / sqrt(d^2), the exponent, lambda d + 1, 1 / d^3 (2)
# and the dipole term into S (3)
PLANE_FP32_PER_PAIR = {"sspd": 12, "shc": 17}


def run_grad_leg(dev, peak_instr_rate, steps: int = 3):
    """Differentiation configuration: N = 65,536 perturbed ellipsoid, Q = 1e6
    uniform queries; forward + d phi / dx (sdf_query_grad) and the parameter
    backward (sdf_backward_params), each timed on the device."""
    import torch

    import paper_2607_16946_b300 as ptsdf
    from paper_2607_16946_b300 import _abi
    import synth
    L = _abi.lib()
    p, n, a = synth.ellipsoid(65536, 1004, axes=(1.0, 0.6, 0.4), perturb=0.05)
    cl = ptsdf.Cloud(p, n, a)
    x = torch.as_tensor(synth.uniform_queries(1_000_000, 1004, -1.5, 1.5), dtype=torch.float32, device=dev)
    G = torch.ones(x.shape[0], device=dev)
    for _ in range(2):
        _, _, saved = cl.query_grad(x)
        cl.backward_params(x, saved, G)
    torch.cuda.synchronize(dev)
    L.sdf_profile_enable(1)
    for _ in range(steps):
        _, _, saved = cl.query_grad(x)
        cl.backward_params(x, saved, G)
    torch.cuda.synchronize(dev)
    L.sdf_profile_enable(0)
    prof = _profile_window(L, _abi)
    pairs = x.shape[0] * 65536
    fg = prof["fwd_grad"]["ms"] / prof["fwd_grad"]["launches"] / 1e3
    bw = prof["bwd_params"]["ms"] / prof["bwd_params"]["launches"] / 1e3
    pre = prof.get("prepass", {"ms": 0.0, "launches": 1})
    # diagnostics (App. D): lap phi and the eikonal residual |grad phi| - 1
    phi, g, lap = cl.query_laplacian(x)
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    phi, g, lap = cl.query_laplacian(x)
    e1.record()
    torch.cuda.synchronize(dev)
    lap_s = e0.elapsed_time(e1) / 1e3
    eik = (g.norm(dim=1) - 1.0).abs()
    near = phi.abs() < 0.05
    diag = {"laplacian_gpairs_s": pairs / lap_s / 1e9, "laplacian_ms": lap_s * 1e3,
            "eikonal_residual_median": float(eik.median()), "eikonal_residual_p99": float(eik.quantile(0.99)),
            "eikonal_residual_median_near_surface": float(eik[near].median()) if bool(near.any()) else None,
            "laplacian_median_near_surface": float(lap[near].median()) if bool(near.any()) else None,
            "note": "|grad phi| - 1 over the 1e6 queries and within |phi| < 0.05; lap phi near the surface is "
                    "about twice the mean curvature"}
    return {"workload": "differentiation: ellipsoid N=65536 (axes 1/0.6/0.4, curvatures x(1+0.05N(0,1))), "
                        "Q=1e6 uniform in [-1.5,1.5]^3; FP32",
            "diagnostics": diag,
            "fwd_grad_gpairs_s": pairs / fg / 1e9, "bwd_params_gpairs_s": pairs / bw / 1e9,
            "step_ms": (fg + bw) * 1e3 + pre["ms"] / pre["launches"],
            "kernels": prof,
            "roofline_fwd_grad": grad_roofline(pairs / fg / 1e9, peak_instr_rate, GRAD_FP32_PER_PAIR,
                                               GRAD_PLAN_FP32),
            "roofline_bwd_params": grad_roofline(pairs / bw / 1e9, peak_instr_rate, BWD_FP32_PER_PAIR,
                                                 BWD_PLAN_FP32)}


def grad_roofline(achieved, fma_rate, counted, plan):
    """Roofline of a gradient pair loop against the FMA pipe (G FP32
    operations/s): over the operations counted from its arithmetic, and over
    the plan's a-priori per-pair count."""
    peak = fma_rate / counted
    return {"bound": "alu", "unit_bound": "FMA pipe", "achieved": achieved, "peak": peak, "unit": UNIT,
            "frac": achieved / peak,
            "peak_basis": f"FMA pipe {fma_rate:.0f} G FP32 operations/s / {counted} per pair (counted)",
            "frac_plan_count": achieved / (fma_rate / plan),
            "plan_count_basis": f"/ {plan} FP32 operations per pair (the plan's "
                                + ("forward 23 + about 20 for the gradient)" if plan == GRAD_PLAN_FP32
                                   else "twice the forward's 23)")}


def run_trace_leg(dev, steps: int = 2):
    """Sphere-tracing configuration: N = 262,144 noisy superquadric, 512 x 512
    pinhole rays from distance 3, <= 48 steps, eps = 1e-4, t_max = 6, normals
    at hits; pairs = sum over steps of live rays x N."""
    import torch

    import paper_2607_16946_b300 as ptsdf
    from paper_2607_16946_b300 import _abi
    import synth
    L = _abi.lib()
    p, n, a = synth.superquadric(262_144, 1003)
    cl = ptsdf.Cloud(p, n, a)
    org, dirs = synth.camera_rays(512, 512, 1003)
    org = torch.as_tensor(org, dtype=torch.float32, device=dev)
    dirs = torch.as_tensor(dirs, dtype=torch.float32, device=dev)
    t, s, nrm = cl.trace(org, dirs)
    torch.cuda.synchronize(dev)
    L.sdf_profile_enable(1)
    t0 = time.perf_counter()
    for _ in range(steps):
        t, s, nrm = cl.trace(org, dirs)
    torch.cuda.synchronize(dev)
    wall = (time.perf_counter() - t0) / steps
    L.sdf_profile_enable(0)
    prof = _profile_window(L, _abi)
    evals = int(s.sum().item())                  # query evaluations = sum over steps of live rays
    pairs = evals * 262_144
    dev_ms = sum(v["ms"] for v in prof.values()) / steps
    roof = None
    if "fwd_tc" in prof:
        # the pair loop over every evaluation (all records are curvature form)
        info = cl.info()
        counts = {"direct": info["n_direct"], "flat": info["n_kappa_flat"],
                  "curved": info["n_kappa"] - info["n_kappa_flat"]}
        rates = probe_rates(L)
        per_sm_clk, mufu_c, fma_c = tc_pair_ceiling(rates, counts)
        sms = torch.cuda.get_device_properties(dev).multi_processor_count
        peak = sms * FALLBACK_MAX_SM_MHZ * 1e6 * per_sm_clk / 1e9
        achieved = pairs / (prof["fwd_tc"]["ms"] / steps / 1e3) / 1e9
        roof = {"bound": "alu", "kernel": "k_fwd_tc", "achieved": achieved, "peak": peak, "unit": UNIT,
                "frac": achieved / peak,
                "peak_basis": f"{'MUFU' if mufu_c <= fma_c else 'FMA-pipe'} ceiling at {FALLBACK_MAX_SM_MHZ:.0f} MHz "
                              f"over the points by form {counts}"}
    return {"workload": "sphere tracing: superquadric N=262144 (e1=0.5, e2=2, axes 1/0.7/0.5, noise 0.003), "
                        "512x512 rays, 48 steps, eps 1e-4, t_max 6, normals at hits; FP32",
            "gpairs_s": pairs / wall / 1e9, "device_gpairs_s": pairs / (dev_ms / 1e3) / 1e9,
            "ms_per_image": wall * 1e3, "rays": int(s.numel()), "hits": int((t >= 0).sum().item()),
            "evaluations": evals, "kernels": prof, "roofline": roof}


def run_radius_leg(dev, cloud, x, phi, steps: int = 3):
    """Sec. 4.2's accelerated evaluation (SDF_LAMBDA_RADIUS) with the paper's
    lambda = 10^3 / D (D from sdf_knn_mean_distance, k = 64), R_eval = 2C/lambda,
    32-nearest fallback: the dense grid, and the sphere-tracing configuration
    traced with it.  Queries/s (pairs/s does not apply: each query sums over
    its own small set)."""
    import torch

    import paper_2607_16946_b300 as ptsdf
    from paper_2607_16946_b300 import _abi
    import synth
    L = _abi.lib()
    out = {}
    t0 = time.perf_counter()
    lam = cloud.paper_lambda()            # sdf_paper_lambda: 10^3 / D, D = sdf_knn_mean_distance(64)
    t_knn = time.perf_counter() - t0
    D = 1e3 / lam
    kw = dict(lambda_mode=ptsdf.SDF_LAMBDA_RADIUS, fixed_lambda=lam)
    cloud.query(x, out=phi, **kw)
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        cloud.query(x, out=phi, **kw)
    e1.record()
    torch.cuda.synchronize(dev)
    s = e0.elapsed_time(e1) / 1e3 / steps
    out["dense_grid"] = {"queries_per_s": x.shape[0] / s, "ms_per_step": s * 1e3, "D": D, "lambda": lam,
                         "R_eval": 128.0 / lam, "knn_ms": t_knn * 1e3,
                         "outputs_finite": bool(torch.isfinite(phi).all())}
    p, n, a = synth.superquadric(262_144, 1003)
    cl = ptsdf.Cloud(p, n, a)
    lam_t = cl.paper_lambda()
    org, dirs = synth.camera_rays(512, 512, 1003)
    org = torch.as_tensor(org, dtype=torch.float32, device=dev)
    dirs = torch.as_tensor(dirs, dtype=torch.float32, device=dev)
    tk = dict(lambda_mode=ptsdf.SDF_LAMBDA_RADIUS, fixed_lambda=lam_t)
    t, st_, nrm = cl.trace(org, dirs, **tk)
    torch.cuda.synchronize(dev)
    L.sdf_profile_enable(1)
    t0 = time.perf_counter()
    for _ in range(2):
        t, st_, nrm = cl.trace(org, dirs, **tk)
    torch.cuda.synchronize(dev)
    wall = (time.perf_counter() - t0) / 2
    L.sdf_profile_enable(0)
    out["trace"] = {"ms_per_image": wall * 1e3, "lambda": lam_t, "hits": int((t >= 0).sum().item()),
                    "evaluations": int(st_.sum().item()),
                    "queries_per_s": int(st_.sum().item()) / wall, "kernels": _profile_window(L, _abi)}
    # the paper's scale for this path: a cloud of 2^21 points (the tracing
    # surface, sampled 8x denser), queried on a 128^3 grid and traced
    pL, nL, aL = synth.superquadric(1 << 21, 2021)
    cL = ptsdf.Cloud(pL, nL, aL)
    del pL, nL, aL
    t0 = time.perf_counter()
    lam_L = cL.paper_lambda()
    t_knn_L = time.perf_counter() - t0
    kL = dict(lambda_mode=ptsdf.SDF_LAMBDA_RADIUS, fixed_lambda=lam_L)
    g = torch.linspace(-1.2, 1.2, 128, device=dev, dtype=torch.float64)
    zz, yy, xx = torch.meshgrid(g, g, g, indexing="ij")
    xg = torch.stack([xx.reshape(-1), yy.reshape(-1), zz.reshape(-1)], 1).to(torch.float32).contiguous()
    phiL = torch.empty(xg.shape[0], device=dev)
    cL.query(xg, out=phiL, **kL)
    torch.cuda.synchronize(dev)
    L.sdf_profile_enable(1)
    e0.record()
    for _ in range(steps):
        cL.query(xg, out=phiL, **kL)
    e1.record()
    torch.cuda.synchronize(dev)
    L.sdf_profile_enable(0)
    sL = e0.elapsed_time(e1) / 1e3 / steps
    out["large_cloud"] = {"points": 1 << 21, "queries_per_s": xg.shape[0] / sL, "ms_per_step": sL * 1e3,
                          "queries": xg.shape[0], "lambda": lam_L, "R_eval": 128.0 / lam_L,
                          "paper_lambda_ms": t_knn_L * 1e3, "kernels": _profile_window(L, _abi),
                          "outputs_finite": bool(torch.isfinite(phiL).all())}
    kr = out["large_cloud"]["kernels"].get("radius")
    out["large_cloud"]["roofline"] = radius_issue_roofline(
        kr["ms"] / kr["launches"] / 1e3 if kr else None, torch.cuda.get_device_properties(dev).multi_processor_count,
        FALLBACK_MAX_SM_MHZ)
    t, st_, nrm = cL.trace(org, dirs, **kL)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    t, st_, nrm = cL.trace(org, dirs, **kL)
    torch.cuda.synchronize(dev)
    out["large_cloud"]["trace_ms_per_image"] = (time.perf_counter() - t0) * 1e3
    out["large_cloud"]["trace_hits"] = int((t >= 0).sum().item())
    out["large_cloud"]["workload"] = ("superquadric N=2^21 (e1=0.5, e2=2, axes 1/0.7/0.5, noise 0.003), "
                                      "lambda = 10^3/D; 128^3 grid over [-1.2,1.2]^3, and the 512x512 "
                                      "tracing camera (normals from the all-pairs gradient)")
    cL.close()
    out["note"] = ("lambda = 10^3/D, R_eval = 2C/lambda, C = 64, 32-nearest fallback; normals at hits from "
                   "the all-pairs gradient with the same lambda")
    return out


def run_mesh_leg(dev, cloud, x, phi, steps: int = 3):
    """Offset surfaces (Sec. 6) of the dense-grid phi: the 0- and 0.05-level
    surfaces of the 256^3 grid by marching tetrahedra (sdf_mesh_level_set)."""
    import torch

    import paper_2607_16946_b300 as ptsdf
    cloud.query(x, out=phi)
    grid = phi.reshape(GRID_RES, GRID_RES, GRID_RES)
    h = 3.2 / (GRID_RES - 1)
    out = {}
    for level in (0.0, 0.05):
        v, t = ptsdf.mesh_level_set(grid, (-1.6, -1.6, -1.6), (h, h, h), level)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for _ in range(steps):
            v, t = ptsdf.mesh_level_set(grid, (-1.6, -1.6, -1.6), (h, h, h), level)
        torch.cuda.synchronize(dev)
        s = (time.perf_counter() - t0) / steps
        out[f"level_{level:g}"] = {"ms": s * 1e3, "vertices": int(v.shape[0]), "triangles": int(t.shape[0]),
                                   "grid_nodes_per_s": GRID_RES ** 3 / s}
    out["note"] = "host-timed, including the count pass and the output allocation"
    return out


def run_morph_leg(dev, cloud, points, steps: int = 3, iters: int = 6, level: float = -0.05):
    """Level-set sampling with normals (Sec. 6, morphological operations,
    erosion's first half): the dense-grid cloud's own points moved onto the
    -0.05 level set by 6 Newton steps along grad phi (sdf_project_level_set,
    7 gradient evaluations of N queries against N points each)."""
    import torch
    seeds = torch.as_tensor(np.asarray(points, np.float32), device=dev)
    x, nrm, res = cloud.project_level_set(seeds, level, max_iter=iters)
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        x, nrm, res = cloud.project_level_set(seeds, level, max_iter=iters)
    e1.record()
    torch.cuda.synchronize(dev)
    s = e0.elapsed_time(e1) / 1e3 / steps
    n = len(points)
    r = res.abs().float()
    return {"ms": s * 1e3, "points": n, "newton_steps": iters, "level": level,
            "gpairs_s": (iters + 1) * n * n / s / 1e9,
            "residual_median": float(r.median()), "residual_p99": float(torch.quantile(r, 0.99)),
            "note": "device-timed; pairs = (steps + 1) gradient evaluations x N^2"}


def run_mixed_leg(dev, cloud, x, phi, points, normals, params, steps: int = 2):
    """The dense-grid step on each engine and precision: FP32 on the tensor
    cores (the default), FP32 on the FP32 units, and packed-half weights
    (SDF_F16X2, SDF_BF16X2, FP32 units); and the two other forms of the sum:
    the log-sum-exp distance on the tensor cores, and the blend with seeded
    per-point weights (default engine).  Device Gpairs/s, and the error against
    the FP64 oracle on 4,096 seeded grid nodes, relative to the AABB diagonal."""
    import torch

    import oracle
    import paper_2607_16946_b300 as ptsdf
    import synth
    from paper_2607_16946_b300 import _abi
    rng = np.random.Generator(np.random.PCG64(SEED + 11))
    idx = rng.integers(0, GRID_RES ** 3, size=4096)
    xs = synth.grid_query_index(idx, GRID_RES)
    orc = oracle.Cloud(points, normals, params)
    ref = orc.phi(xs)
    weights = np.exp(np.random.Generator(np.random.PCG64(SEED + 12)).uniform(np.log(0.5), np.log(2.0),
                                                                             size=len(points))).astype(np.float32)
    wcloud = ptsdf.Cloud(points, normals, params, weights=weights)
    shc_ref, shc_cond = orc.shc(xs, cond=True)
    well = shc_cond <= 1e3         # phi_SHC is compared where its double-layer sum is not a cancellation
    cases = (("fp32_tensor", cloud, dict(precision=_abi.SDF_F32, engine=_abi.SDF_ENGINE_TENSOR), ref, None),
             ("fp32_alu", cloud, dict(precision=_abi.SDF_F32, engine=_abi.SDF_ENGINE_ALU), ref, None),
             ("f16x2", cloud, dict(precision=_abi.SDF_F16X2, engine=_abi.SDF_ENGINE_ALU), ref, None),
             ("bf16x2", cloud, dict(precision=_abi.SDF_BF16X2, engine=_abi.SDF_ENGINE_ALU), ref, None),
             ("lse_tensor", cloud, dict(formula=_abi.SDF_FORMULA_LSE, engine=_abi.SDF_ENGINE_TENSOR), orc.lse(xs),
              None),
             ("weighted_fp32", wcloud, dict(), oracle.Cloud(points, normals, params, weights=weights).phi(xs), None),
             ("sspd", cloud, dict(formula=_abi.SDF_FORMULA_SSPD), orc.sspd(xs), None),
             ("shc", cloud, dict(formula=_abi.SDF_FORMULA_SHC), shc_ref, well))
    diag = float(np.linalg.norm(points.max(0) - points.min(0)))
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    rates = probe_rates(_abi.lib())
    L = _abi.lib()
    out = {}
    for name, cl, kw, r, mask in cases:
        cl.query(x, out=phi, **kw)
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        L.sdf_profile_enable(1)
        e0.record()
        for _ in range(steps):
            cl.query(x, out=phi, **kw)
        e1.record()
        torch.cuda.synchronize(dev)
        L.sdf_profile_enable(0)
        prof = _profile_window(L, _abi)
        s = e0.elapsed_time(e1) / 1e3 / steps
        err = np.abs(phi[torch.as_tensor(idx, device=dev)].double().cpu().numpy() - r) / diag
        if mask is not None:
            err = err[mask]
        out[name] = {"value": x.shape[0] * N_POINTS / s / 1e9, "unit": UNIT, "ms_per_step": s * 1e3,
                     "err_max_rel_diag": float(err.max()), "err_p99_rel_diag": float(np.quantile(err, 0.99))}
        if mask is not None:
            out[name]["compared"] = f"{int(mask.sum())} of {mask.size} nodes (oracle condition number <= 1e3)"
        if "plane" in prof:
            # the baselines' pair loop: 1 sqrt (SSPD) or rsqrt (SHC) + 1 exp2 per pair
            # on the XU pipe, and PLANE_FP32_PER_PAIR operations on the FMA pipe
            mufu = 1.0 / (1.0 / rates["sqrt"] + 1.0 / rates["ex2"])
            fma = rates["fma"] / PLANE_FP32_PER_PAIR[name]
            per_clk = min(mufu, fma)
            peak = sms * FALLBACK_MAX_SM_MHZ * 1e6 * per_clk / 1e9
            ach = x.shape[0] * N_POINTS / (prof["plane"]["ms"] / steps / 1e3) / 1e9
            out[name]["roofline"] = {"bound": "alu", "kernel": "k_fwd_plane", "achieved": ach, "peak": peak,
                                     "unit": UNIT, "frac": ach / peak,
                                     "peak_basis": f"{'XU' if mufu <= fma else 'FMA pipe'}: XU 1 sqrt/rsqrt + 1 ex2 "
                                                   f"per pair at the measured rates = {mufu:.2f} pairs/clk/SM, FMA "
                                                   f"pipe {rates['fma']:.1f} / {PLANE_FP32_PER_PAIR[name]} FP32 "
                                                   f"operations = {fma:.2f}; x {sms} SMs x "
                                                   f"{FALLBACK_MAX_SM_MHZ:.0f} MHz"}
    wcloud.close()
    out["note"] = ("fp32_tensor: products on the tensor cores (split f16, FP32 accumulate), pairs finished in "
                   "FP32; fp32_alu: FP32 units only; f16x2/bf16x2: packed-half exp2 of a lane's two weights on "
                   "the FP32-unit loop; lse_tensor: the log-sum-exp distance (Eq. ConvolutionalDistanceFormula, "
                   "h = 1) from the same sums; weighted_fp32: per-point weights log-uniform in [0.5, 2] "
                   "(direct tiles on the tensor cores, curvature-form tiles on the FP32 units); "
                   "sspd / shc: the paper's baselines phi_SSPD (Eq. SmoothedSignedPlanarDistance) and phi_SHC "
                   "(Eq. ScreenedWindingNumber) on the FP32 units with packed .f32x2 arithmetic; "
                   "error = |out - oracle| / AABB diagonal on 4096 seeded grid nodes")
    return out


def compact_summary(line: dict) -> dict:
    """The other legs in a few numbers each (value, roofline fraction,
    error against the oracle), rounded."""
    def r(v, d=4):
        return None if v is None else float(f"{v:.{d}g}")
    out = {"dense_grid": {"gpairs_s": r(line["value"]), "frac": r(line["roofline"]["frac"], 3),
                          "e2e_gpairs_s": r(line["e2e"]["value"])}}
    for k, v in line.get("mixed", {}).items():
        if isinstance(v, dict):
            out[k] = {"gpairs_s": r(v["value"]), "err_max": r(v["err_max_rel_diag"], 2)}
            if "roofline" in v:
                out[k]["frac"] = r(v["roofline"]["frac"], 3)
    g = line.get("grad")
    if g:
        out["grad"] = {"fwd_grad_gpairs_s": r(g["fwd_grad_gpairs_s"]), "bwd_gpairs_s": r(g["bwd_params_gpairs_s"]),
                       "fwd_grad_frac": r(g["roofline_fwd_grad"]["frac"], 3),
                       "bwd_frac": r(g["roofline_bwd_params"]["frac"], 3),
                       "laplacian_gpairs_s": r(g["diagnostics"]["laplacian_gpairs_s"])}
    t = line.get("trace")
    if t:
        out["trace"] = {"gpairs_s": r(t["gpairs_s"]), "ms_per_image": r(t["ms_per_image"]),
                        "frac": r((t.get("roofline") or {}).get("frac"), 3)}
    rd = line.get("radius")
    if rd:
        out["radius"] = {"grid_queries_s": r(rd["dense_grid"]["queries_per_s"]),
                         "trace_ms_per_image": r(rd["trace"]["ms_per_image"])}
        if "large_cloud" in rd:
            out["radius"]["large_cloud_queries_s"] = r(rd["large_cloud"]["queries_per_s"])
            if rd["large_cloud"].get("roofline"):
                out["radius"]["large_cloud_issue_frac"] = r(rd["large_cloud"]["roofline"]["frac"], 3)
    for k in ("served", "served_high", "served_fifo", "served_f16x2"):
        if k in line:
            out[k] = {"gpairs_s": r(line[k]["value"]), "p50_ms": r(line[k]["p50_ms"]), "p99_ms": r(line[k]["p99_ms"]),
                      "slowdown_p99": r(line[k].get("slowdown_p99"), 3)}
    if "cpu_baseline" in line:
        out["cpu_oracle_gpairs_s"] = r(line["cpu_baseline"]["value"])
    return out


def workload_config(q: int, world: int) -> dict:
    """The workload both arms run, the same dict in both lines (how the main
    arm runs it goes under its own "run" key)."""
    return {"workload": WORKLOAD, "N": N_POINTS, "Q": q, "C": 64, "lambda": "global",
            "parallelism": f"replicas{world}" if world > 1 else "single",
            "l2": "inputs larger than L2 (queries 201 MB, phi 67 MB); not flushed"}


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
            "config": workload_config(GRID_RES ** 3, world),
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
    # the dominant kernel: the tensor-core pair loop, over every tile (direct,
    # flat and curved curvature-form records; the curved ones, 2.6% of the
    # points here, cost two reciprocals more per pair), unless the library
    # routes the curved tiles to the FP32-unit loop (k_fwd then also runs)
    info = cloud.info()
    rates = probe_rates(L)
    if "fwd_tc" in prof:
        flat_tc = info["n_kappa_flat"]
        curved = info["n_kappa"] - flat_tc
        if prof.get("fwd", {}).get("launches", 0) > 0:
            flat_tc, curved = 32 * (flat_tc // 32), 0
        counts = {"direct": info["n_direct"], "flat": flat_tc, "curved": curved}
        kname, kpairs = "k_fwd_tc", q * sum(counts.values())
        per_sm_clk, mufu_c, fma_c = tc_pair_ceiling(rates, counts)
        kp = prof["fwd_tc"]
        traffic = committed_traffic()
        nominal = sum(counts.values()) / sum(c * single_op_cost(NOMINAL_RATES, TC_FORM_COST[f][0])
                                             for f, c in counts.items())
        basis = (f"{'MUFU' if mufu_c <= fma_c else 'FMA-pipe'} ceiling: {sms} SMs x {fmax:.0f} MHz x "
                 f"{per_sm_clk:.3f} pairs/clk/SM over the points by form {counts}; MUFU per pair "
                 f"(sqrt, rcp, ex2) = {dict((f, c[0]) for f, c in TC_FORM_COST.items())} at the measured "
                 f"single-operation rates -> {mufu_c:.3f} (nominal 16/16/32 per SM per clock: {nominal:.3f}); FMA pipe "
                 f"{rates['fma']:.1f}/{dict((f, c[1]) for f, c in TC_FORM_COST.items())} FP32 operations "
                 f"-> {fma_c:.3f} (unit rates {rates['source']})")
    else:
        kname, kpairs = "k_fwd", pairs_per_step
        per_sm_clk, mufu_c, issue_c = pair_ceiling(rates, FP32_PER_PAIR)
        kp = prof.get("fwd", {"launches": 0, "ms": float("nan")})
        traffic = None
        basis = (f"{'MUFU' if mufu_c <= issue_c else 'FMA-pipe'} ceiling: {sms} SMs x {fmax:.0f} MHz x "
                 f"{per_sm_clk:.3f} pairs/clk/SM; MUFU: the direct mix (3 sqrt + 1 ex2) measured whole = "
                 f"{mufu_c:.3f}, FMA pipe {rates['fma']:.1f}/"
                 f"{FP32_PER_PAIR} = {issue_c:.3f} (unit rates {rates['source']})")
    peak = sms * fmax * 1e6 * per_sm_clk / 1e9
    # per step: the pair loop runs as one launch per record segment present
    per_step_s = kp["ms"] / args.steps / 1e3
    achieved = kpairs / per_step_s / 1e9
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": elapsed_s / args.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": workload_config(q, world),
        "run": {"precision": "fp32", "engine": "auto (tensor cores for every tile)"},
        "queries_per_s": world * q * args.steps / elapsed_s,
        "e2e": {"value": world * pairs_per_step * args.steps / e2e_s / 1e9, "unit": UNIT,
                "h2d_bytes_per_step": q * 12, "d2h_bytes_per_step": q * 4},
        "gpu_launches": launches_total,
        "kernels": prof,
        "roofline": {"bound": "alu", "kernel": kname, "launches_per_step": kp["launches"] / args.steps,
                     "achieved": achieved, "peak": peak, "unit": UNIT,
                     "frac": achieved / peak, "traffic": traffic, "peak_basis": basis,
                     "unit_rates_per_sm_clk": {k: v for k, v in rates.items()}},
        "clocks": cs,
        "outputs_finite": finite,
    }
    if world == 1 and not args.no_extra_legs:
        line["mixed"] = run_mixed_leg(dev, cloud, x, phi, p, n, a)
        line["grad"] = run_grad_leg(dev, sms * fmax * 1e6 * rates["fma"] / 1e9)
        line["trace"] = run_trace_leg(dev)
        line["radius"] = run_radius_leg(dev, cloud, x, phi)
        line["mesh"] = run_mesh_leg(dev, cloud, x, phi)
        line["morph"] = run_morph_leg(dev, cloud, p)
    if world == 1 and args.serve_requests > 0:
        del hx, hphi
        clouds_np = make_serving_clouds(args.serve_clouds, SERVE_SEED)
        variants = set(args.serve_variants.split(","))
        if "fp32" in variants:
            line["served"] = run_served(args, dev, value, policy=1, clouds_np=clouds_np)
        if "high" in variants:
            # the same requests and arrivals, offered at the higher load
            line["served_high"] = run_served(args, dev, value, policy=1, clouds_np=clouds_np,
                                             load=args.serve_load_high)
        if "fifo" in variants:
            line["served_fifo"] = run_served(args, dev, value, policy=0, clouds_np=clouds_np)
        if "f16x2" in variants:
            # the serving configuration's packed-half form, offered at 0.7 of its own measured rate
            f16_rate = line.get("mixed", {}).get("f16x2", {}).get("value") or value
            line["served_f16x2"] = run_served(args, dev, f16_rate, policy=1, clouds_np=clouds_np, precision=1)
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(p, n, a)
    line["summary"] = compact_summary(line)     # last, so that a truncated record still shows it
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true", help="omit the CPU oracle leg")
    ap.add_argument("--serve-requests", type=int, default=300, help="requests of the served leg (0: skip)")
    ap.add_argument("--serve-streams", type=int, default=SERVE_STREAMS, help="CUDA streams of the served leg")
    ap.add_argument("--serve-express", type=float, default=SERVE_EXPRESS_GPAIRS,
                    help="requests of at most this many Gpairs run on high-priority streams (0: one priority)")
    ap.add_argument("--no-extra-legs", action="store_true", help="omit the gradient and tracing legs")
    ap.add_argument("--serve-clouds", type=int, default=32)
    ap.add_argument("--serve-variants", default="fp32,high,fifo,f16x2",
                    help="served runs: fp32 (smallest-first), high (the same at --serve-load-high), fifo, "
                         "f16x2 (comma-separated)")
    ap.add_argument("--serve-load", type=float, default=0.7, help="offered load as a fraction of capacity")
    ap.add_argument("--serve-load-high", type=float, default=0.9, help="offered load of the 'high' served run")
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
