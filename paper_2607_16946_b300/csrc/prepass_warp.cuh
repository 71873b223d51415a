// The exact prepass (d_max and d_min of each query over the cloud's points,
// for lambda_x = 2 C / d_max of Eq. RelationshipBetweenLambdaAndRadius and the
// exponent shift) with the bounding-sphere pruning of k_prepass_pruned, run a
// warp per query: for GLOBAL-lambda batches too small to fill the GPU with a
// thread per query (sphere-tracing steps, served requests).  The lanes share
// the query: they take the bounding spheres 32 at a time for the bounds
// LB = max_t (|x - c_t| - r_t) <= d_max and UB = min_t (|x - c_t| + r_t) >= d_min,
// scan the two tiles that gave them exactly (two points per lane), tighten
// the bounds with those exact distances less the same rounding margin as
// k_prepass_pruned, and then scan every tile with |x - c_t| + r_t >= LB or
// |x - c_t| - r_t <= UB.  Each point is evaluated with k_prepass's
// arithmetic, so the maxima, minima and the lowest farthest index equal the
// full scan's.
#pragma once

#include <cuda_runtime.h>

#include "query_common.cuh"

#ifndef PTSDF_WARP_PREPASS
#define PTSDF_WARP_PREPASS 1   // 0: such batches take the point-split full scan
#endif
#ifndef PTSDF_WARP_PREPASS_ALL
#define PTSDF_WARP_PREPASS_ALL 0   // 1: large batches too (instead of a thread per query)
#endif

namespace ptsdf {
namespace qk {
namespace {

constexpr int kWarpPreThreads = 256;

struct Extremes {
    float hi, lo;    // max and min of v = |x' - p'|^2 - |x'|^2 (so d^2 = v + |x'|^2)
    int32_t far;     // lowest prepass index of the maximum
};

template <bool ARGMAX>
__device__ __forceinline__ void scan_point(float4 r, int64_t j, float xs0, float xs1, float xs2, Extremes& e) {
    const float v = fmaf(xs0, r.x, fmaf(xs1, r.y, fmaf(xs2, r.z, r.w)));
    if (ARGMAX) {
        if (v > e.hi || (v == e.hi && (int32_t)j < e.far)) {
            e.hi = v;
            e.far = (int32_t)j;
        }
    } else {
        e.hi = fmaxf(e.hi, v);
    }
    e.lo = fminf(e.lo, v);
}

template <bool ARGMAX>
__device__ __forceinline__ void scan_tile(const float4* __restrict__ pre, int64_t n, int64_t t, int lane, float xs0,
                                          float xs1, float xs2, Extremes& e) {
    const int64_t first = t * kSphereTile;
    if (PTSDF_PRE_UNROLL && first + kSphereTile <= n) {   // a full tile: both loads before the arithmetic
        const float4 r0 = __ldg(pre + first + lane), r1 = __ldg(pre + first + 32 + lane);
        scan_point<ARGMAX>(r0, first + lane, xs0, xs1, xs2, e);
        scan_point<ARGMAX>(r1, first + 32 + lane, xs0, xs1, xs2, e);
        return;
    }
#pragma unroll
    for (int h = 0; h < kSphereTile; h += 32) {
        const int64_t j = first + h + lane;
        if (j >= n) break;
        scan_point<ARGMAX>(__ldg(pre + j), j, xs0, xs1, xs2, e);
    }
}

// Two tiles, all four loads issued before the arithmetic (the extremes and
// the lowest farthest index do not depend on the order of the points).
template <bool ARGMAX>
__device__ __forceinline__ void scan_tile_pair(const float4* __restrict__ pre, int64_t n, int64_t t, int64_t u,
                                               int lane, float xs0, float xs1, float xs2, Extremes& e) {
    const int64_t ft = t * kSphereTile, fu = u * kSphereTile;
    if (ft + kSphereTile <= n && fu + kSphereTile <= n) {
        const float4 r0 = __ldg(pre + ft + lane), r1 = __ldg(pre + ft + 32 + lane);
        const float4 r2 = __ldg(pre + fu + lane), r3 = __ldg(pre + fu + 32 + lane);
        scan_point<ARGMAX>(r0, ft + lane, xs0, xs1, xs2, e);
        scan_point<ARGMAX>(r1, ft + 32 + lane, xs0, xs1, xs2, e);
        scan_point<ARGMAX>(r2, fu + lane, xs0, xs1, xs2, e);
        scan_point<ARGMAX>(r3, fu + 32 + lane, xs0, xs1, xs2, e);
    } else {
        scan_tile<ARGMAX>(pre, n, t, lane, xs0, xs1, xs2, e);
        scan_tile<ARGMAX>(pre, n, u, lane, xs0, xs1, xs2, e);
    }
}

template <bool ARGMAX>
__device__ __forceinline__ void warp_reduce(Extremes& e) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float ohi = __shfl_xor_sync(0xffffffffu, e.hi, o), olo = __shfl_xor_sync(0xffffffffu, e.lo, o);
        const int32_t ofar = __shfl_xor_sync(0xffffffffu, e.far, o);
        if (ARGMAX) {
            if (ohi > e.hi || (ohi == e.hi && ofar < e.far)) {
                e.hi = ohi;
                e.far = ofar;
            }
        } else {
            e.hi = fmaxf(e.hi, ohi);
        }
        e.lo = fminf(e.lo, olo);
    }
}

template <bool ARGMAX>
__global__ void __launch_bounds__(kWarpPreThreads) k_prepass_warp(const float4* __restrict__ pre,
                                                                  const float4* __restrict__ spheres, int64_t n,
                                                                  int64_t nsph, QueryArgs a) {
    const int lane = (int)(threadIdx.x & 31);
    const int64_t warps = (int64_t)gridDim.x * (kWarpPreThreads / 32);
    for (int64_t qi = (int64_t)blockIdx.x * (kWarpPreThreads / 32) + threadIdx.x / 32; qi < a.q; qi += warps) {
        const float xs0 = a.x[3 * qi] - a.cx, xs1 = a.x[3 * qi + 1] - a.cy, xs2 = a.x[3 * qi + 2] - a.cz;
        const float xx = xs0 * xs0 + xs1 * xs1 + xs2 * xs2;
        // 1. bounds from the spheres, with the spheres that gave them
        float lb = -INFINITY, ub = INFINITY;
        int64_t tf = 0, tn = 0;
#pragma unroll 4
        for (int64_t t = lane; t < nsph; t += 32) {
            const float4 s = __ldg(spheres + t);
            const float dx = xs0 - s.x, dy = xs1 - s.y, dz = xs2 - s.z;
            const float dc = sqrt_mufu(fmaf(dx, dx, fmaf(dy, dy, dz * dz)));
            if (dc - s.w > lb) {
                lb = dc - s.w;
                tf = t;
            }
            if (dc + s.w < ub) {
                ub = dc + s.w;
                tn = t;
            }
        }
        // the warp's best, and one seed sphere each on which every lane agrees
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float olb = __shfl_xor_sync(0xffffffffu, lb, o), oub = __shfl_xor_sync(0xffffffffu, ub, o);
            const int64_t otf = __shfl_xor_sync(0xffffffffu, tf, o), otn = __shfl_xor_sync(0xffffffffu, tn, o);
            if (olb > lb || (olb == lb && otf < tf)) {
                lb = olb;
                tf = otf;
            }
            if (oub < ub || (oub == ub && otn < tn)) {
                ub = oub;
                tn = otn;
            }
        }
        // 2. the seed tiles exactly; their extremes tighten the bounds
        Extremes e{-INFINITY, INFINITY, 0x7fffffff};
        scan_tile<ARGMAX>(pre, n, tf, lane, xs0, xs1, xs2, e);
        if (tn != tf) scan_tile<ARGMAX>(pre, n, tn, lane, xs0, xs1, xs2, e);
        warp_reduce<ARGMAX>(e);
        // a computed |x' - p'|^2 = xx + v is within 4 eps (|x'| + |p'|)^2 of the
        // exact one, so its distance is within 2^-11 (|x'| + |p'|)
        const float margin = 4.8828125e-4f * (sqrtf(xx) + a.cloud_radius);
        const float lbmax = fmaxf(lb, sqrtf(fmaxf(e.hi + xx, 0.f)) - margin);
        const float ubmin = fminf(ub, sqrtf(fmaxf(e.lo + xx, 0.f)) + margin);
        // 3. every other tile that may hold an extreme
        for (int64_t t0 = 0; t0 < nsph; t0 += 32) {
            const int64_t t = t0 + lane;
            bool need = false;
            if (t < nsph && t != tf && t != tn) {
                const float4 s = __ldg(spheres + t);
                const float dx = xs0 - s.x, dy = xs1 - s.y, dz = xs2 - s.z;
                const float dc = sqrt_mufu(fmaf(dx, dx, fmaf(dy, dy, dz * dz)));
                need = (dc + s.w >= lbmax) || (dc - s.w <= ubmin);
            }
            unsigned m = __ballot_sync(0xffffffffu, need);
            while (m) {
                const int b = __ffs(m) - 1;
                m &= m - 1;
                if (PTSDF_PRE_UNROLL && m) {
                    const int b2 = __ffs(m) - 1;
                    m &= m - 1;
                    scan_tile_pair<ARGMAX>(pre, n, t0 + b, t0 + b2, lane, xs0, xs1, xs2, e);
                } else {
                    scan_tile<ARGMAX>(pre, n, t0 + b, lane, xs0, xs1, xs2, e);
                }
            }
        }
        warp_reduce<ARGMAX>(e);
        if (lane == 0) {
            a.d2[qi] = make_float2(e.hi + xx, e.lo + xx);
            if (ARGMAX) a.far[qi] = e.far;
        }
    }
}

// True when a query batch of plan p should take the warp-per-query prepass:
// GLOBAL lambda, a batch below the thread-per-query pruned prepass, and the
// automatic split (an explicit split_n keeps the point-split full scan, with
// the same results: the tests compare the two that way).
__host__ inline bool use_warp_prepass(const Cloud& c, const Plan& p, const sdf_query_opts& o) {
    return PTSDF_WARP_PREPASS && o.lambda_mode == SDF_LAMBDA_GLOBAL && o.split_n == 0 && c.spheres != nullptr &&
           (PTSDF_WARP_PREPASS_ALL || !use_pruned_prepass(c, p, o));
}

// Writes a.d2[qi] = (d_max^2, d_min^2) for every query (pre_split = 1) and,
// with argmax, a.far[qi] = the lowest prepass index of a farthest point: the
// values of the full scan, bit for bit.  Launch errors are left for the
// caller's cudaGetLastError.
__host__ inline void launch_prepass_warp(const Cloud& c, const QueryArgs& a, bool argmax, cudaStream_t st) {
    if (a.q <= 0) return;
    const int64_t per_block = kWarpPreThreads / 32;
    const int64_t need = (a.q + per_block - 1) / per_block, cap = 16LL * c.num_sms;
    const unsigned blocks = (unsigned)(need < cap ? need : cap);
    if (argmax)
        k_prepass_warp<true><<<blocks, kWarpPreThreads, 0, st>>>(c.pre, c.spheres, c.n, c.n_spheres, a);
    else
        k_prepass_warp<false><<<blocks, kWarpPreThreads, 0, st>>>(c.pre, c.spheres, c.n, c.n_spheres, a);
}


}  // namespace
}  // namespace qk
}  // namespace ptsdf
