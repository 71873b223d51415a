// Shared by the query kernels (query.cu, grad.cu): launch constants, the
// argument block, the d_max / d_min prepass and the two forms of the torus
// SDF pair term.
#pragma once

#include <cuda_runtime.h>

#include <cmath>

#include "device_common.cuh"
#include "internal.h"

namespace ptsdf {
namespace qk {
namespace {

constexpr int kThreads = (kConsumerWarps + 1) * 32;   // + producer warp
constexpr float kLog2e = 1.4426950408889634f;
constexpr uint32_t kTileBytes = kTileRecs * kRecFloats * sizeof(float);
constexpr uint32_t kPreBytes = kPreTile * sizeof(float4);

struct QueryArgs {
    const float* x;          // Q x 3
    int64_t q;
    float* phi;              // Q (split == 1)
    float2* part;            // split x Q (W, S) partials (split > 1)
    float2* d2;              // split x Q prepass partials (max, min of |x - p|^2)
    int32_t* far;            // split x Q index of the farthest point (prepass order), or null
    float cx, cy, cz;        // cloud bounding-box centre (prepass coordinates)
    int split;               // point chunks of the main kernel
    int pre_split;           // prepass partials per query (1 for the pruned prepass)
    int mode;                // sdf_lambda_mode
    float C;
    float lam;               // fixed lambda
    float offset;
    float cloud_radius = 0.f;  // max |p'| (half the AABB diagonal): scale of the prepass's rounding
    int64_t tile_base = 0;   // first tile of chunk 0 (k_fwd)
    int part_base = 0;       // partial row of chunk 0 when several kernels share the partials
    int formula = SDF_FORMULA_BLEND;   // what the sums finish into (finish_sums)
};

// A query's screening from its prepass partials d2p[c * q + qq] (max, min of
// |x - p|^2): L = lambda log2(e) and A0 = L d_min, so that a point's weight is
// exp2(A0 - L d) = exp(-lambda (d - d_min)).  GLOBAL: lambda_x = C / sigma_x =
// 2 C / d_max (Eq. RelationshipBetweenLambdaAndRadius; d_max = 0, every point
// at the query, takes lambda = 0); FIXED: the given lambda.
__device__ __forceinline__ void query_screening(const float2* __restrict__ d2p, int pre_split, int64_t q, int64_t qq,
                                                int mode, float C, float lam_fixed, float& L, float& A0) {
    float2 d2 = d2p[qq];
    for (int c = 1; c < pre_split; ++c) {
        const float2 v = d2p[(size_t)c * q + qq];
        d2.x = fmaxf(d2.x, v.x);
        d2.y = fminf(d2.y, v.y);
    }
    const float dmin = sqrtf(fmaxf(d2.y, 0.f));
    float lam = lam_fixed;
    if (mode == SDF_LAMBDA_GLOBAL) {
        const float dmax = sqrtf(fmaxf(d2.x, 0.f));
        lam = dmax > 0.f ? 2.f * C / dmax : 0.f;
    }
    L = lam * kLog2e;
    A0 = L * dmin;
}

constexpr float kLog2TwoPi = 2.6514961294723187f;   // log2(2 pi)

// What a query's sums W = sum A_i w_i, S = sum A_i w_i g_i finish into, less
// the offset: the blend S / W (Eq. BasicFormulaShifted; with g_i = <x - p_i,
// n_i> it is phi_SSPD, Eq. SmoothedSignedPlanarDistance), or the log-sum-exp
// distance -(1/lambda) log sum_i A_i exp(-lambda d_i) (Eq.
// ConvolutionalDistanceFormula, h = 1) = d_min - ln(W) / lambda =
// (A0 - log2 W) / L; where L = 0 (GLOBAL with every point at the query) it
// is d_min = 0.  SDF_FORMULA_SHC: S = 2 pi w e^(-lambda d_min) for the
// screened double-layer sum w of Eq. ScreenedWindingNumber, and
// phi_SHC = sign(w) (-(1/lambda) ln|w|) = sign(S) (A0 - log2|S| + log2 2pi) / L
// (the paper's + sigma_x cancels its shift inside w); L = 0 gives 0 and S = 0
// gives +inf (the limit as |w| -> 0).
__device__ __forceinline__ float finish_sums(float W, float S, int formula, float L, float A0, float offset) {
    if (formula == SDF_FORMULA_LSE) return (L > 0.f ? (A0 - log2f(W)) / L : 0.f) - offset;
    if (formula == SDF_FORMULA_SHC) {
        if (!(L > 0.f)) return -offset;
        // sign(w) times the distance term, which is negative where |w| > e^(lambda d_min)
        const float v = (A0 - log2f(fabsf(S)) + kLog2TwoPi) / L;
        return (S < 0.f ? -v : v) - offset;
    }
    return __fdiv_rn(S, W) - offset;
}

// Sums the (W, S) partials of every chunk in chunk order and finishes them.
__global__ void k_merge(QueryArgs a) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.q) return;
    float W = 0.f, S = 0.f;
    for (int c = 0; c < a.split; ++c) {
        const float2 v = a.part[(size_t)c * a.q + i];
        W += v.x;
        S += v.y;
    }
    float L = 0.f, A0 = 0.f;
    if (a.formula == SDF_FORMULA_LSE || a.formula == SDF_FORMULA_SHC)
        query_screening(a.d2, a.pre_split, a.q, i, a.mode, a.C, a.lam, L, A0);
    a.phi[i] = finish_sums(W, S, a.formula, L, A0, a.offset);
}

// --------------------------------------------------------------------------
// Prepass
// --------------------------------------------------------------------------
template <int MODE, bool ARGMAX = false>
__global__ void __launch_bounds__(kThreads) k_prepass(const float4* __restrict__ pre, int64_t n, int64_t pre_tiles,
                                                      int64_t tiles_per_chunk, QueryArgs a, int32_t* status) {
    extern __shared__ __align__(128) char smem[];
    __shared__ TileRing<kStages> ring;
    char* buf = smem;
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int chunk = blockIdx.y;
    const int64_t t0 = (int64_t)chunk * tiles_per_chunk;
    const int64_t t1 = t0 + tiles_per_chunk < pre_tiles ? t0 + tiles_per_chunk : pre_tiles;
    const int64_t nt = t1 > t0 ? t1 - t0 : 0;
    if (threadIdx.x == 0) ring.init(kConsumerWarps);
    __syncthreads();
    if (warp == kConsumerWarps) {
        if (lane == 0) ring.produce(buf, reinterpret_cast<const char*>(pre + t0 * kPreTile), nt, kPreBytes, status);
        return;
    }
    float xs[kQueriesPerThread][3], hi[kQueriesPerThread], lo[kQueriesPerThread], xx[kQueriesPerThread];
    int64_t qi[kQueriesPerThread];
    int32_t far[kQueriesPerThread];
#pragma unroll
    for (int k = 0; k < kQueriesPerThread; ++k) {
        qi[k] = (int64_t)blockIdx.x * kQueriesPerCta + k * (kConsumerWarps * 32) + threadIdx.x;
        const int64_t qq = qi[k] < a.q ? qi[k] : a.q - 1;
        xs[k][0] = a.x[3 * qq] - a.cx;
        xs[k][1] = a.x[3 * qq + 1] - a.cy;
        xs[k][2] = a.x[3 * qq + 2] - a.cz;
        xx[k] = xs[k][0] * xs[k][0] + xs[k][1] * xs[k][1] + xs[k][2] * xs[k][2];
        hi[k] = -INFINITY;
        lo[k] = INFINITY;
        far[k] = 0;
    }
    for (int64_t t = 0; t < nt; ++t) {
        if (!ring.wait_full(t, status)) return;
        const float4* tile = reinterpret_cast<const float4*>(buf + (size_t)(t % kStages) * kPreBytes);
        const int64_t first = (t0 + t) * kPreTile;
        const int cnt = (int)(n - first < kPreTile ? n - first : kPreTile);
        if (MODE == SDF_LAMBDA_GLOBAL) {
            // |x'-p'|^2 - |x'|^2 = |p'|^2 - 2 <x', p'>: three FMAs per pair.  Its
            // cancellation near d = 0 only perturbs the shift d_min (harmless
            // for lambda_x = 2 C / d_max); d_max keeps full relative accuracy.
#pragma unroll 4
            for (int j = 0; j < cnt; ++j) {
                const float4 r = tile[j];
#pragma unroll
                for (int k = 0; k < kQueriesPerThread; ++k) {
                    const float v = fmaf(xs[k][0], r.x, fmaf(xs[k][1], r.y, fmaf(xs[k][2], r.z, r.w)));
                    if (ARGMAX) {
                        // first (lowest prepass index) of equal maxima
                        if (v > hi[k]) {
                            hi[k] = v;
                            far[k] = (int32_t)(first + j);
                        }
                    } else {
                        hi[k] = fmaxf(hi[k], v);
                    }
                    lo[k] = fminf(lo[k], v);
                }
            }
        } else {
            // FIXED lambda may be large, so the shift d_min is computed from
            // the difference vector (no cancellation)
#pragma unroll 4
            for (int j = 0; j < cnt; ++j) {
                const float4 r = tile[j];
#pragma unroll
                for (int k = 0; k < kQueriesPerThread; ++k) {
                    const float dx = fmaf(0.5f, r.x, xs[k][0]), dy = fmaf(0.5f, r.y, xs[k][1]),
                                dz = fmaf(0.5f, r.z, xs[k][2]);
                    lo[k] = fminf(lo[k], fmaf(dx, dx, fmaf(dy, dy, dz * dz)));
                }
            }
        }
        ring.release(t, lane);
    }
#pragma unroll
    for (int k = 0; k < kQueriesPerThread; ++k) {
        if (qi[k] < a.q) {
            const float2 v = MODE == SDF_LAMBDA_GLOBAL ? make_float2(hi[k] + xx[k], lo[k] + xx[k])
                                                       : make_float2(-INFINITY, lo[k]);
            a.d2[(size_t)chunk * a.q + qi[k]] = v;
            if (ARGMAX) a.far[(size_t)chunk * a.q + qi[k]] = far[k];
        }
    }
}

// --------------------------------------------------------------------------
// Pruned prepass (GLOBAL lambda): the same d_max / d_min as k_prepass, with
// tiles that cannot hold either extreme skipped.  For every 64-point tile t
// with bounding sphere (c_t, r_t) and a query x, all its points lie between
// |x - c_t| - r_t and |x - c_t| + r_t.  Hence
//   LB = max_t (|x - c_t| - r_t) <= d_max   and   UB = min_t (|x - c_t| + r_t) >= d_min,
// and only tiles with |x - c_t| + r_t >= LB (may hold the farthest point) or
// |x - c_t| - r_t <= UB (may hold the nearest) are scanned, point by point,
// with exactly the arithmetic of k_prepass, so the results are identical.
// A warp scans a tile when any of its lanes needs it.  Plain cached loads: the
// tiles a warp visits differ from warp to warp.
// --------------------------------------------------------------------------
constexpr int kPrunedThreads = kConsumerWarps * 32;
#ifndef PTSDF_PRE_UNROLL
#define PTSDF_PRE_UNROLL 1   // 0: spheres tested one at a time, tiles scanned at a variable trip count
#endif

// One sphere's tile of the prepass array (points first .. first + cnt - 1),
// for the lane's queries, with k_prepass's arithmetic.  A full tile's loop
// has a fixed trip count, so its loads can be issued ahead of the arithmetic.
template <bool ARGMAX>
__device__ __forceinline__ void pruned_scan_tile(const float4* __restrict__ pre, int64_t first, int cnt,
                                                 const float (&xs)[kQueriesPerThread][3],
                                                 float (&hi)[kQueriesPerThread], float (&lo)[kQueriesPerThread],
                                                 int32_t (&far)[kQueriesPerThread]) {
    auto point = [&](int j) {
        const float4 r = __ldg(pre + first + j);
#pragma unroll
        for (int k = 0; k < kQueriesPerThread; ++k) {
            const float v = fmaf(xs[k][0], r.x, fmaf(xs[k][1], r.y, fmaf(xs[k][2], r.z, r.w)));
            if (ARGMAX) {
                if (v > hi[k] || (v == hi[k] && (int32_t)(first + j) < far[k])) {
                    hi[k] = v;
                    far[k] = (int32_t)(first + j);
                }
            } else {
                hi[k] = fmaxf(hi[k], v);
            }
            lo[k] = fminf(lo[k], v);
        }
    };
    if (PTSDF_PRE_UNROLL && cnt == kSphereTile) {
#pragma unroll 8
        for (int j = 0; j < kSphereTile; ++j) point(j);
    } else {
#pragma unroll 1
        for (int j = 0; j < cnt; ++j) point(j);
    }
}

template <bool ARGMAX>
__global__ void __launch_bounds__(kPrunedThreads) k_prepass_pruned(const float4* __restrict__ pre,
                                                                   const float4* __restrict__ spheres, int64_t n,
                                                                   int64_t nsph, QueryArgs a) {
    float xs[kQueriesPerThread][3], hi[kQueriesPerThread], lo[kQueriesPerThread], xx[kQueriesPerThread];
    float lbmax[kQueriesPerThread], ubmin[kQueriesPerThread];
    int64_t qi[kQueriesPerThread];
    int32_t far[kQueriesPerThread];
#pragma unroll
    for (int k = 0; k < kQueriesPerThread; ++k) {
        qi[k] = (int64_t)blockIdx.x * kQueriesPerCta + k * (kConsumerWarps * 32) + threadIdx.x;
        const int64_t qq = qi[k] < a.q ? qi[k] : a.q - 1;
        xs[k][0] = a.x[3 * qq] - a.cx;
        xs[k][1] = a.x[3 * qq + 1] - a.cy;
        xs[k][2] = a.x[3 * qq + 2] - a.cz;
        xx[k] = xs[k][0] * xs[k][0] + xs[k][1] * xs[k][1] + xs[k][2] * xs[k][2];
        hi[k] = -INFINITY;
        lo[k] = INFINITY;
        lbmax[k] = -INFINITY;
        ubmin[k] = INFINITY;
        far[k] = 0;
    }
    // bounds from the spheres; every lane also notes the spheres that gave its
    // first query's bounds
    int32_t t_far = 0, t_near = 0;
    const int32_t ns = (int32_t)nsph;
#pragma unroll 4
    for (int32_t t = 0; t < ns; ++t) {
        const float4 s = __ldg(spheres + t);
#pragma unroll
        for (int k = 0; k < kQueriesPerThread; ++k) {
            const float dx = xs[k][0] - s.x, dy = xs[k][1] - s.y, dz = xs[k][2] - s.z;
            const float dc = sqrt_mufu(fmaf(dx, dx, fmaf(dy, dy, dz * dz)));
            if (k == 0) {
                if (dc - s.w > lbmax[0]) t_far = t;
                if (dc + s.w < ubmin[0]) t_near = t;
            }
            lbmax[k] = fmaxf(lbmax[k], dc - s.w);
            ubmin[k] = fminf(ubmin[k], dc + s.w);
        }
    }
    // Tighten the bounds with exact distances: scan (for every lane) the
    // spheres lanes 0 and 31 found, which are near-best for the whole warp
    // (its queries are neighbours), and take the farthest and nearest of their
    // points (less a rounding margin) as the bounds.  Only the thresholds of the scan below change; every
    // extreme still comes from the same arithmetic.
    const int32_t seeds[4] = {__shfl_sync(0xffffffffu, t_far, 0), __shfl_sync(0xffffffffu, t_near, 0),
                              __shfl_sync(0xffffffffu, t_far, 31), __shfl_sync(0xffffffffu, t_near, 31)};
    for (int seed = 0; seed < 4; ++seed) {
        const int64_t t = seeds[seed];
        bool dup = false;
        for (int o = 0; o < seed; ++o) dup = dup || seeds[o] == t;
        if (dup) continue;
        const int64_t first = t * kSphereTile;
        pruned_scan_tile<ARGMAX>(pre, first, (int)(n - first < kSphereTile ? n - first : kSphereTile), xs, hi, lo,
                                 far);
    }
#pragma unroll
    for (int k = 0; k < kQueriesPerThread; ++k) {
        // a computed |x' - p'|^2 = xx + v is within 4 eps (|x'| + |p'|)^2 of the
        // exact one, so its distance is within 2^-11 (|x'| + |p'|)
        const float margin = 4.8828125e-4f * (sqrtf(xx[k]) + a.cloud_radius);
        lbmax[k] = fmaxf(lbmax[k], sqrtf(fmaxf(hi[k] + xx[k], 0.f)) - margin);
        ubmin[k] = fminf(ubmin[k], sqrtf(fmaxf(lo[k] + xx[k], 0.f)) + margin);
    }
    // exact scan of the tiles that may hold an extreme: the spheres are
    // tested four at a time (their loads and roots issued together), then
    // the tiles any lane needs are scanned in order
    constexpr int kTest = PTSDF_PRE_UNROLL ? 4 : 1;
    for (int32_t t0 = 0; t0 < ns; t0 += kTest) {
        bool need[kTest];
#pragma unroll
        for (int u = 0; u < kTest; ++u) {
            const int32_t t = t0 + u < ns ? t0 + u : ns - 1;
            const float4 s = __ldg(spheres + t);
            need[u] = false;
#pragma unroll
            for (int k = 0; k < kQueriesPerThread; ++k) {
                const float dx = xs[k][0] - s.x, dy = xs[k][1] - s.y, dz = xs[k][2] - s.z;
                const float dc = sqrt_mufu(fmaf(dx, dx, fmaf(dy, dy, dz * dz)));
                need[u] = need[u] || (dc + s.w >= lbmax[k]) || (dc - s.w <= ubmin[k]);
            }
        }
#pragma unroll
        for (int u = 0; u < kTest; ++u) {
            if (t0 + u >= ns || !__any_sync(0xffffffffu, need[u])) continue;
            const int64_t first = (int64_t)(t0 + u) * kSphereTile;
            pruned_scan_tile<ARGMAX>(pre, first, (int)(n - first < kSphereTile ? n - first : kSphereTile), xs,
                                     hi, lo, far);
        }
    }
#pragma unroll
    for (int k = 0; k < kQueriesPerThread; ++k) {
        if (qi[k] < a.q) {
            a.d2[qi[k]] = make_float2(hi[k] + xx[k], lo[k] + xx[k]);
            if (ARGMAX) a.far[qi[k]] = far[k];
        }
    }
}

// Pruned prepass for GLOBAL lambda once the query blocks fill the GPU (one
// wave of 2 CTAs per SM); smaller batches keep the point-split prepass.
__host__ inline bool use_pruned_prepass(const Cloud& c, const Plan& p, const sdf_query_opts& o) {
    return o.lambda_mode == SDF_LAMBDA_GLOBAL && c.spheres != nullptr && p.pre_qblocks >= 2LL * c.num_sms;
}

// --------------------------------------------------------------------------
// Pair terms
// --------------------------------------------------------------------------
// Direct form: v = x - c, h = <v, u>, rho = |v - h u| (the distance to the
// axis, computed from the perpendicular component so it stays accurate near
// the axis), g = sT (||(rho - R, h)|| - r).
__device__ __forceinline__ float g_direct(float x, float y, float z, const float4& r1, const float4& r2, float sT) {
    const float vx = x - r1.x, vy = y - r1.y, vz = z - r1.z;
    const float h = fmaf(vx, r2.x, fmaf(vy, r2.y, vz * r2.z));
    const float wx = fmaf(-h, r2.x, vx), wy = fmaf(-h, r2.y, vy), wz = fmaf(-h, r2.z, vz);
    const float rho = sqrt_mufu(fmaf(wx, wx, fmaf(wy, wy, wz * wz)));
    const float e = rho - r1.w;
    const float D = sqrt_mufu(fmaf(e, e, h * h));
    return fmaf(sT, D, r2.w);
}

// Curvature form around q = Q*(0,0), exact rewrite of the same torus SDF:
// with y = x - q, h = <y, u>, t^2 = |y|^2 - h^2, k = |kappa_min|,
//   m  = k t^2 + 2 zeta <y, n*>,    a' = m / (1 + sqrt(1 + k m))   (= rho - 1/k)
//   N' = -kappa_max (a'^2 + h^2) + 2 zeta a'
//   g  = N' / (1 + sqrt(1 + (-kappa_max) N'))
// which has no 1/k or 1/|kappa_max| and so no cancellation of large radii.
// g_kappa for a record with kappa_min = 0 (k = r1.w = 0): m = <y, 2 zeta n*>,
// s1 = 1 and a' = m / 2, which saves a square root and a reciprocal.
__device__ __forceinline__ float g_kappa_flat(float x, float y, float z, const float4& r0, const float4& r1,
                                              const float4& r2, const float4& r3) {
    const float yx = x - r1.x, yy = y - r1.y, yz = z - r1.z;
    const float h = fmaf(yx, r2.x, fmaf(yy, r2.y, yz * r2.z));
    const float ap = 0.5f * fmaf(yx, r3.x, fmaf(yy, r3.y, yz * r3.z));
    const float Np = fmaf(r2.w, fmaf(ap, ap, h * h), r0.w * ap);
    const float s2 = sqrt_mufu(fmaxf(fmaf(r2.w, Np, 1.f), 0.f));
    return Np * rcp_mufu(1.f + s2);
}

__device__ __forceinline__ float g_kappa(float x, float y, float z, const float4& r0, const float4& r1,
                                         const float4& r2, const float4& r3) {
    const float yx = x - r1.x, yy = y - r1.y, yz = z - r1.z;
    const float h = fmaf(yx, r2.x, fmaf(yy, r2.y, yz * r2.z));
    const float hh = h * h;
    const float t2 = fmaf(yx, yx, fmaf(yy, yy, yz * yz)) - hh;
    const float m = fmaf(r1.w, t2, fmaf(yx, r3.x, fmaf(yy, r3.y, yz * r3.z)));
    const float s1 = sqrt_mufu(fmaxf(fmaf(r1.w, m, 1.f), 0.f));
    const float ap = m * rcp_mufu(1.f + s1);
    const float Np = fmaf(r2.w, fmaf(ap, ap, hh), r0.w * ap);
    const float s2 = sqrt_mufu(fmaxf(fmaf(r2.w, Np, 1.f), 0.f));
    return Np * rcp_mufu(1.f + s2);
}

}  // namespace
}  // namespace qk
}  // namespace ptsdf
