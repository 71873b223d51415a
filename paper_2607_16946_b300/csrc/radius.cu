// Radius-limited evaluation (Sec. 4.2, "Acceleration and adaptive lambda")
// and the mean k-nearest-neighbour distance D of its lambda heuristic.
//
// lambda is one constant for the cloud; a query sums Eq. BasicFormulaShifted
// over the points within R_eval = 2 C / lambda only, and over its 32 nearest
// points when none lies within R_eval.  The paper finds both sets with a
// kd-tree on the CPU.  Here the spatial index is the one the pruned prepass
// already keeps: the points in Morton order, one bounding sphere per 64
// consecutive points (radius inflated against FP32 rounding), and a copy of
// the torus records in the same order.  A query
//   1. bounds every sphere: points of sphere t lie in [|x - c_t| - r_t,
//      |x - c_t| + r_t]; the spheres that can reach within R_eval are
//      scanned point by point and their points inside R_eval summed, with
//      the exponent shift following the smallest distance seen (the sums
//      are rescaled when it drops);
//   2. if no point was inside, seeds a sorted list of the k nearest
//      (distance, then scan order) with the points of the sphere of smallest
//      |x - c_t| + r_t, then scans every other sphere whose lower bound
//      reaches below the current k-th distance, and sums over the k.
// The k-nearest search of D is the same second step with the point itself
// excluded, seeded with its own sphere and the next one in Morton order.
// Both steps walk the spheres group by group (kGroupSpheres per group sphere)
// and pass over a group whose sphere shows that none of its members would be
// scanned, nor become the seed: every per-point decision, the summation order
// and so the results are those of the walk over every sphere.
// Distances come from the 16-byte prepass entries; records are read only for
// the points that enter a sum.  One thread per query (or point); warps scan a
// sphere when any of their lanes needs it.
#include <cuda_runtime.h>

#include <cmath>
#include <vector>

#include "query_common.cuh"
#include "sphere_index.h"

namespace ptsdf {

using namespace qk;

namespace {

constexpr int kRadiusThreads = 128;
constexpr int kKnnMax = 64;

struct RadiusArgs {
    const float* x;
    int64_t q;
    float* phi;
    const float4* spheres;
    int64_t nsph;
    const float4* groups;  // group spheres (after the spheres in the same array)
    int64_t ngroups;
    const float4* mrec;    // n x 4 float4 records in Morton order (r3.w: the point's weight)
    const float4* pre;     // n float4(-2 p', |p'|^2) in the same order (p' = p - AABB centre)
    int64_t n;
    float cx, cy, cz;
    float L;               // lambda log2(e)
    float reval;
    float offset;
    int kfb;
    int lse;               // 1: the log-sum-exp distance of the set instead of the blend
};

// The torus SDF of one record (the form read from r0.w: sT = +-1 direct,
// 2 zeta = +-2 kappa; 0 when only the weights are wanted) and the point's
// weight A_i.
__device__ __forceinline__ float g_record(float x, float y, float z, const float4* __restrict__ r, bool want_g,
                                          float& wa) {
    const float4 r0 = __ldg(r), r3 = __ldg(r + 3);
    wa = r3.w;
    if (!want_g) return 0.f;
    const float4 r1 = __ldg(r + 1), r2 = __ldg(r + 2);
    return fabsf(r0.w) > 1.5f ? g_kappa(x, y, z, r0, r1, r2, r3) : g_direct(x, y, z, r1, r2, r0.w);
}

__device__ __forceinline__ int sphere_count(int64_t t, int64_t n) {
    const int64_t left = n - t * kSphereTile;
    return (int)(left < kSphereTile ? left : kSphereTile);
}

// Squared distance from x' (coordinates centred on the AABB) to point j of
// the Morton-ordered prepass array float4(-2 p', |p'|^2).
__device__ __forceinline__ float dist2_pre(float xs, float ys, float zs, const float4* __restrict__ pre, int64_t j) {
    const float4 e = __ldg(pre + j);
    const float dx = fmaf(0.5f, e.x, xs), dy = fmaf(0.5f, e.y, ys), dz = fmaf(0.5f, e.z, zs);
    return fmaf(dx, dx, fmaf(dy, dy, dz * dz));
}

// Distance from x' to the centre of sphere s (the bounds add or subtract its
// inflated radius; sqrt.approx's relative error is covered by the 1e-6 pad
// the callers apply).
__device__ __forceinline__ float centre_dist(float xs, float ys, float zs, const float4& s) {
    const float dx = xs - s.x, dy = ys - s.y, dz = zs - s.z;
    return sqrt_mufu(fmaf(dx, dx, fmaf(dy, dy, dz * dz)));
}

// Lower bound on |x' - c_t| - r_t and |x' - c_t| + r_t, as centre_dist gives
// them, for every member t of group sphere gs: the relative pad covers the
// rounding of both centre distances (each well inside 1e-6 relative).
__device__ __forceinline__ float group_lower(float xs, float ys, float zs, const float4& gs) {
    return centre_dist(xs, ys, zs, gs) * (1.f - 1e-5f) - gs.w;
}

__device__ __forceinline__ int64_t group_end(int64_t g, int64_t nsph) {
    const int64_t e = (g + 1) * kGroupSpheres;
    return e < nsph ? e : nsph;
}

// Inserts (d2, j) into the ascending top-k list (bd, bi) of cnt entries.
__device__ __forceinline__ void topk_insert(float* bd, int* bi, int& cnt, int k, float d2, int j) {
    if (cnt == k && !(d2 < bd[k - 1])) return;
    int pos = cnt < k ? cnt++ : k - 1;
    while (pos > 0 && d2 < bd[pos - 1]) {
        bd[pos] = bd[pos - 1];
        bi[pos] = bi[pos - 1];
        --pos;
    }
    bd[pos] = d2;
    bi[pos] = j;
}

// Offers the points of sphere t to the top-k list.  The current k-th squared
// distance is kept in a register (the list lives in local memory), so a
// rejected point costs no local load; the acceptance test is topk_insert's.
__device__ __forceinline__ void scan_sphere(const RadiusArgs& a, float xs, float ys, float zs, int64_t t, int64_t self,
                                            int k, float* bd, int* bi, int& cnt) {
    const int64_t j0 = t * kSphereTile;
    const int c = sphere_count(t, a.n);
    float kth = cnt == k ? bd[k - 1] : INFINITY;
    for (int jj = 0; jj < c; ++jj) {
        const int64_t j = j0 + jj;
        if (j == self) continue;
        const float d2 = dist2_pre(xs, ys, zs, a.pre, j);
        if (cnt == k && !(d2 < kth)) continue;
        topk_insert(bd, bi, cnt, k, d2, (int)j);
        if (cnt == k) kth = bd[k - 1];
    }
}

// The k nearest points of x' (Morton positions in bi, squared distances
// ascending in bd), skipping Morton position `self` (or -1).  The list is
// seeded from `seed` (and, for a point of the cloud, its Morton neighbour
// sphere), then every other sphere whose lower bound reaches below the
// current k-th distance is scanned.  (Sweeping outward from the seed in
// Morton order tightens the bound sooner but gives every lane of a warp a
// different sphere at each step; the shared order keeps the sphere loads
// broadcast and measured 25% faster.)  Returns min(k, points available).
__device__ int knn_scan(const RadiusArgs& a, float xs, float ys, float zs, int k, int64_t self, int64_t seed,
                        float* bd, int* bi) {
    int cnt = 0;
    scan_sphere(a, xs, ys, zs, seed, self, k, bd, bi, cnt);
    int64_t seed2 = -1;
    if (self >= 0 && a.nsph > 1) {
        seed2 = seed + 1 < a.nsph ? seed + 1 : seed - 1;
        scan_sphere(a, xs, ys, zs, seed2, self, k, bd, bi, cnt);
    }
    for (int64_t g = 0; g < a.ngroups; ++g) {
        // the bound only tightens as the list fills, so a group beyond it now
        // has no member within it later
        const float glim = cnt < k ? INFINITY : sqrtf(bd[k - 1]) * (1.f + 1e-6f);
        if (group_lower(xs, ys, zs, __ldg(a.groups + g)) > glim) continue;
        for (int64_t t = g * kGroupSpheres, te = group_end(g, a.nsph); t < te; ++t) {
            if (t == seed || t == seed2) continue;
            const float4 s = __ldg(a.spheres + t);
            const float lb = centre_dist(xs, ys, zs, s) - s.w;
            const float lim = cnt < k ? INFINITY : sqrtf(bd[k - 1]) * (1.f + 1e-6f);
            if (!(lb <= lim)) continue;
            scan_sphere(a, xs, ys, zs, t, self, k, bd, bi, cnt);
        }
    }
    return cnt;
}

// Phase 1, one thread per query: the points within R_eval.  A query with
// none of them is appended, with the seed sphere its pass found, to a list
// that phase 2 (k_radius_fallback) works through a warp per query.
// 12 resident blocks per SM: the kernel waits on dependent loads, so
// residency matters more than a few spilled registers.
__global__ void __launch_bounds__(kRadiusThreads, 12) k_radius_query(RadiusArgs a, int* __restrict__ fb_count,
                                                                     int2* __restrict__ fb_list) {
    const int64_t qi = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (qi >= a.q) return;
    const float x = a.x[3 * qi], y = a.x[3 * qi + 1], z = a.x[3 * qi + 2];
    const float xs = x - a.cx, ys = y - a.cy, zs = z - a.cz;
    const float R2 = a.reval * a.reval;
    const float lim = a.reval * (1.f + 1e-6f);
    // 1. the points inside R_eval, online shift by the smallest distance; the
    //    same pass finds the sphere of smallest upper bound holding kfb points
    float W = 0.f, S = 0.f, m = INFINITY;
    int inside = 0;
    float best_ub = INFINITY;
    int64_t best = 0;
    for (int64_t gi = 0; gi < a.ngroups; ++gi) {
        // a group none of whose spheres reaches R_eval or improves on the
        // seed so far is passed over (a NaN bound passes neither test)
        const float lo = group_lower(xs, ys, zs, __ldg(a.groups + gi));
        if (lo > lim && !(lo < best_ub)) continue;
        for (int64_t t = gi * kGroupSpheres, te = group_end(gi, a.nsph); t < te; ++t) {
            const float4 s = __ldg(a.spheres + t);
            const float dc = centre_dist(xs, ys, zs, s);
            if (dc + s.w < best_ub && sphere_count(t, a.n) >= a.kfb) {
                best_ub = dc + s.w;
                best = t;
            }
            if (!(dc - s.w <= lim)) continue;
            const int64_t j0 = t * kSphereTile;
            const int c = sphere_count(t, a.n);
            for (int jj = 0; jj < c; ++jj) {
                const float d2 = dist2_pre(xs, ys, zs, a.pre, j0 + jj);
                if (!(d2 <= R2)) continue;
                const float d = sqrtf(d2);
                float wa;
                const float g = g_record(x, y, z, a.mrec + 4 * (j0 + jj), !a.lse, wa);
                if (d < m) {
                    // a new nearest point: the sums so far are rescaled to its distance
                    const float f = inside ? exp2f(-a.L * (m - d)) : 0.f;
                    W = fmaf(W, f, wa);
                    S = fmaf(S, f, wa * g);
                    m = d;
                } else {
                    const float w = wa * exp2f(-a.L * (d - m));
                    W += w;
                    S = fmaf(w, g, S);
                }
                ++inside;
            }
        }
    }
    if (inside == 0) {
        // 2. the kfb nearest points: deferred to phase 2 (one list slot per
        //    query, claimed by one atomic per warp)
        const unsigned mask = __activemask();
        const int lane = (int)(threadIdx.x & 31);
        const int leader = __ffs(mask) - 1;
        int base = 0;
        if (lane == leader) base = atomicAdd(fb_count, __popc(mask));
        base = __shfl_sync(mask, base, leader);
        fb_list[base + __popc(mask & ((1u << lane) - 1u))] = make_int2((int)qi, (int)best);
        return;
    }
    // the blend, or the log-sum-exp distance m - ln(W) / lambda = m - log2(W) / L
    a.phi[qi] = (a.lse ? m - log2f(W) / a.L : __fdiv_rn(S, W)) - a.offset;
}

// ---------------------------------------------------------------------------
// Phase 2: the k = 32 nearest points of each listed query, a warp per query.
// The list is held one entry per lane, sorted ascending across the lanes by
// (squared distance, Morton position).  Candidates come 32 at a time (half a
// sphere); when any of them beats the 32nd entry they are sorted by a bitonic
// network of shuffles and merged: the elementwise minimum of the ascending
// list and the descending candidates holds the 32 smallest of both as a
// bitonic sequence, which five more shuffle steps sort.  Spheres are visited
// as in knn_scan: the seed first, then every sphere of a group within reach
// whose lower bound reaches below the current 32nd distance, so the list is
// the exact 32 nearest (ties by Morton position).
// ---------------------------------------------------------------------------
constexpr int kFallbackThreads = 256;
constexpr unsigned kFull = 0xffffffffu;
static_assert(kRadiusFallbackK == 32, "the fallback list is one entry per lane");

__device__ __forceinline__ bool lex_less(float da, int ia, float db, int ib) {
    return da < db || (da == db && ia < ib);
}

// Ascending bitonic sort of the 32 (d, i) pairs held by the lanes.
__device__ __forceinline__ void warp_bitonic_sort(float& d, int& i, int lane) {
#pragma unroll
    for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            const float od = __shfl_xor_sync(kFull, d, j);
            const int oi = __shfl_xor_sync(kFull, i, j);
            const bool take_min = ((lane & j) == 0) == ((lane & k) == 0 || k == 32);
            const bool other_less = lex_less(od, oi, d, i);
            if (take_min == other_less) {
                d = od;
                i = oi;
            }
        }
    }
}

// Merges the lanes' candidates (cd, ci) into the sorted list (ld, li).
__device__ __forceinline__ void warp_merge(float cd, int ci, float& ld, int& li, int lane) {
    warp_bitonic_sort(cd, ci, lane);
    const float rd = __shfl_sync(kFull, cd, 31 - lane);
    const int ri = __shfl_sync(kFull, ci, 31 - lane);
    if (lex_less(rd, ri, ld, li)) {
        ld = rd;
        li = ri;
    }
#pragma unroll
    for (int j = 16; j > 0; j >>= 1) {
        const float od = __shfl_xor_sync(kFull, ld, j);
        const int oi = __shfl_xor_sync(kFull, li, j);
        const bool other_less = lex_less(od, oi, ld, li);
        if (((lane & j) == 0) == other_less) {
            ld = od;
            li = oi;
        }
    }
}

// Offers the points of sphere t (two halves of 32) to the list; kd, ki: the
// current 32nd entry (every lane holds it).
__device__ __forceinline__ void warp_scan_sphere(const RadiusArgs& a, float xs, float ys, float zs, int64_t t,
                                                 int lane, float& ld, int& li, float& kd, int& ki) {
    const int64_t j0 = t * kSphereTile;
    const int c = sphere_count(t, a.n);
#pragma unroll
    for (int h = 0; h < kSphereTile; h += 32) {
        float d2 = INFINITY;
        int idx = 0x7fffffff;
        if (h + lane < c) {
            d2 = dist2_pre(xs, ys, zs, a.pre, j0 + h + lane);
            idx = (int)(j0 + h + lane);
        }
        if (!__any_sync(kFull, lex_less(d2, idx, kd, ki))) continue;
        warp_merge(d2, idx, ld, li, lane);
        kd = __shfl_sync(kFull, ld, 31);
        ki = __shfl_sync(kFull, li, 31);
    }
}

__global__ void __launch_bounds__(kFallbackThreads) k_radius_fallback(RadiusArgs a, const int* __restrict__ fb_count,
                                                                      const int2* __restrict__ fb_list) {
    const int lane = (int)(threadIdx.x & 31);
    const int64_t warps = (int64_t)gridDim.x * (kFallbackThreads / 32);
    const int count = *fb_count;
    for (int64_t e = (int64_t)blockIdx.x * (kFallbackThreads / 32) + threadIdx.x / 32; e < count; e += warps) {
        const int2 job = fb_list[e];
        const int64_t qi = job.x, seed = job.y;
        const float x = a.x[3 * qi], y = a.x[3 * qi + 1], z = a.x[3 * qi + 2];
        const float xs = x - a.cx, ys = y - a.cy, zs = z - a.cz;
        float ld = INFINITY, kd = INFINITY;
        int li = 0x7fffffff, ki = 0x7fffffff;
        warp_scan_sphere(a, xs, ys, zs, seed, lane, ld, li, kd, ki);
        for (int64_t g0 = 0; g0 < a.ngroups; g0 += 32) {
            // the bound only tightens as the list fills, so a group beyond it now
            // has no member within it later
            const float glim = kd < INFINITY ? sqrtf(kd) * (1.f + 1e-6f) : INFINITY;
            const int64_t g = g0 + lane;
            const bool reach = g < a.ngroups && group_lower(xs, ys, zs, __ldg(a.groups + g)) <= glim;
            unsigned gm = __ballot_sync(kFull, reach);
            while (gm) {
                const int64_t gg = g0 + __ffs(gm) - 1;
                gm &= gm - 1;
                const int64_t te = group_end(gg, a.nsph);
                for (int64_t t0 = gg * kGroupSpheres; t0 < te; t0 += 32) {
                    // lanes past the group's last sphere, and the seed, take no part
                    const int64_t t = t0 + lane;
                    const bool real = t < te && t != seed;
                    float lb = INFINITY;
                    if (real) {
                        const float4 sp = __ldg(a.spheres + t);
                        lb = centre_dist(xs, ys, zs, sp) - sp.w;
                    }
                    const float slim = kd < INFINITY ? sqrtf(kd) * (1.f + 1e-6f) : INFINITY;
                    unsigned sm = __ballot_sync(kFull, real && lb <= slim);
                    while (sm) {
                        const int b = __ffs(sm) - 1;
                        sm &= sm - 1;
                        // re-checked against the bound as it stands now
                        const float lbb = __shfl_sync(kFull, lb, b);
                        if (!(lbb <= (kd < INFINITY ? sqrtf(kd) * (1.f + 1e-6f) : INFINITY))) continue;
                        warp_scan_sphere(a, xs, ys, zs, t0 + b, lane, ld, li, kd, ki);
                    }
                }
            }
        }
        // the blend (or log-sum-exp distance) over the list, shifted by its
        // nearest.  Far from the surface lambda d is large (lambda = 10^3 / D
        // gives 10^4 - 10^5 there), so the weights would amplify the FP32
        // rounding of d by that much: the 32 distances are taken again in
        // FP64 from the input coordinates (the records' p), and only their
        // differences to the nearest enter the exponent.
        double dd = 0.0;
        if (li != 0x7fffffff) {
            const float4 r0 = __ldg(a.mrec + 4 * (int64_t)li);
            const double ex = (double)x - r0.x, ey = (double)y - r0.y, ez = (double)z - r0.z;
            dd = sqrt(ex * ex + ey * ey + ez * ez);
        }
        const double m0 = __shfl_sync(kFull, dd, 0);
        const float m = (float)m0;
        float W = 0.f, S = 0.f;
        if (li != 0x7fffffff) {
            float wa;
            const float g = g_record(x, y, z, a.mrec + 4 * (int64_t)li, !a.lse, wa);
            W = wa * exp2f(-a.L * (float)(dd - m0));
            S = W * g;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            W += __shfl_xor_sync(kFull, W, o);
            S += __shfl_xor_sync(kFull, S, o);
        }
        if (lane == 0) a.phi[qi] = (a.lse ? m - log2f(W) / a.L : __fdiv_rn(S, W)) - a.offset;
    }
}

// Per point: mean of the distances to its k nearest other points; one
// partial sum (double) per block.
__global__ void __launch_bounds__(kRadiusThreads) k_knn_mean(RadiusArgs a, int k, double* __restrict__ partial) {
    __shared__ double red[kRadiusThreads];
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double v = 0.0;
    if (i < a.n) {
        const float4 e = __ldg(a.pre + i);
        float bd[kKnnMax];
        int bi[kKnnMax];
        const int cnt = knn_scan(a, -0.5f * e.x, -0.5f * e.y, -0.5f * e.z, k, i, i / kSphereTile, bd, bi);
        double s = 0.0;
        for (int j = 0; j < cnt; ++j) s += sqrt((double)bd[j]);
        v = cnt > 0 ? s / cnt : 0.0;
    }
    red[threadIdx.x] = v;
    __syncthreads();
    for (int w = kRadiusThreads / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

// The k nearest of the point at Morton position i, written as input indices
// at its input row; one partial sum of the mean distances per block.
__global__ void __launch_bounds__(kRadiusThreads) k_knn_index(RadiusArgs a, int k, const int32_t* __restrict__ mperm,
                                                              int32_t* __restrict__ idx, double* __restrict__ partial) {
    __shared__ double red[kRadiusThreads];
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double v = 0.0;
    if (i < a.n) {
        const float4 e = __ldg(a.pre + i);
        float bd[kKnnMax];
        int bi[kKnnMax];
        const int cnt = knn_scan(a, -0.5f * e.x, -0.5f * e.y, -0.5f * e.z, k, i, i / kSphereTile, bd, bi);
        const int64_t row = mperm[i];
        double s = 0.0;
        for (int j = 0; j < k; ++j) {
            idx[row * k + j] = j < cnt ? mperm[bi[j]] : -1;
            if (j < cnt) s += sqrt((double)bd[j]);
        }
        v = cnt > 0 ? s / cnt : 0.0;
    }
    red[threadIdx.x] = v;
    __syncthreads();
    for (int w = kRadiusThreads / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

RadiusArgs radius_args(const Cloud& c) {
    RadiusArgs a;
    a.x = nullptr;
    a.q = 0;
    a.phi = nullptr;
    a.spheres = c.spheres;
    a.nsph = c.n_spheres;
    a.groups = c.spheres ? c.spheres + c.n_spheres : nullptr;
    a.ngroups = c.spheres ? group_count(c.n_spheres) : 0;
    a.mrec = c.mrec;
    a.pre = c.pre;
    a.n = c.n;
    a.cx = 0.5f * (c.aabb[0] + c.aabb[3]);
    a.cy = 0.5f * (c.aabb[1] + c.aabb[4]);
    a.cz = 0.5f * (c.aabb[2] + c.aabb[5]);
    a.L = 0.f;
    a.reval = 0.f;
    a.offset = 0.f;
    a.kfb = kRadiusFallbackK;
    a.lse = 0;
    return a;
}

}  // namespace

sdf_status launch_radius_query(const Cloud& c, const float* d_x, int64_t q, float* d_phi, const sdf_query_opts& o,
                               cudaStream_t st) {
    if (q > 0x7fffffffLL) return set_error(SDF_EINVAL, "sdf_query: SDF_LAMBDA_RADIUS takes at most 2^31 - 1 queries");
    RadiusArgs a = radius_args(c);
    a.x = d_x;
    a.q = q;
    a.phi = d_phi;
    a.L = o.fixed_lambda * 1.4426950408889634f;
    a.reval = 2.f * o.C / o.fixed_lambda;
    a.offset = o.offset;
    a.lse = o.formula == SDF_FORMULA_LSE ? 1 : 0;
    // scratch: the fallback count (16 B) and list (one int2 per query)
    char* scratch = nullptr;
    cudaError_t e = cudaMallocAsync(&scratch, 16 + (size_t)q * sizeof(int2), st);
    if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? set_error(SDF_ENOMEM, "sdf_query: radius scratch")
                                                                : cuda_error(e, "sdf_query: radius scratch");
    int* fb_count = reinterpret_cast<int*>(scratch);
    int2* fb_list = reinterpret_cast<int2*>(scratch + 16);
    e = cudaMemsetAsync(fb_count, 0, sizeof(int), st);
    {
        ProfRange pr(SDF_K_RADIUS, st);
        if (e == cudaSuccess) {
            k_radius_query<<<(unsigned)((q + kRadiusThreads - 1) / kRadiusThreads), kRadiusThreads, 0, st>>>(
                a, fb_count, fb_list);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) {
            // enough warps to cover the list when every query falls back, at
            // most 8 blocks per SM; each warp loops over its share
            const int64_t need = (q + kFallbackThreads / 32 - 1) / (kFallbackThreads / 32);
            const int64_t cap = 8LL * c.num_sms;
            k_radius_fallback<<<(unsigned)(need < cap ? need : cap), kFallbackThreads, 0, st>>>(a, fb_count, fb_list);
            e = cudaGetLastError();
        }
    }
    cudaFreeAsync(scratch, st);
    return e == cudaSuccess ? SDF_OK : cuda_error(e, "sdf_query: radius-limited launch");
}

sdf_status launch_knn_indices(const Cloud& c, int k, int32_t* d_idx, double* mean_dist, cudaStream_t st) {
    if (k < 1 || k > kKnnMax) return set_error(SDF_EINVAL, "k-nearest search: k must be in [1, 64]");
    RadiusArgs a = radius_args(c);
    const int64_t blocks = (c.n + kRadiusThreads - 1) / kRadiusThreads;
    double* part = nullptr;
    cudaError_t e = cudaMallocAsync(&part, (size_t)blocks * sizeof(double), st);
    if (e != cudaSuccess) return cuda_error(e, "k-nearest search: scratch");
    {
        ProfRange pr(SDF_K_KNN, st);
        k_knn_index<<<(unsigned)blocks, kRadiusThreads, 0, st>>>(a, k, c.mperm, d_idx, part);
        e = cudaGetLastError();
    }
    std::vector<double> h((size_t)blocks);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h.data(), part, (size_t)blocks * sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFreeAsync(part, st);
    if (e != cudaSuccess) return cuda_error(e, "k-nearest search");
    double s = 0.0;
    for (double v : h) s += v;
    if (mean_dist) *mean_dist = c.n > 0 ? s / (double)c.n : 0.0;
    return SDF_OK;
}

}  // namespace ptsdf

using namespace ptsdf;

extern "C" sdf_status sdf_knn_mean_distance(sdf_cloud cloud, int32_t k, double* D, void* stream) {
    if (!cloud || !D) return set_error(SDF_EINVAL, "sdf_knn_mean_distance: NULL argument");
    if (k < 1 || k > kKnnMax) return set_error(SDF_EINVAL, "sdf_knn_mean_distance: k must be in [1, 64]");
    const Cloud& c = *reinterpret_cast<const Cloud*>(cloud);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (c.n < 2) {
        *D = 0.0;
        return SDF_OK;
    }
    RadiusArgs a = radius_args(c);
    const int64_t blocks = (c.n + kRadiusThreads - 1) / kRadiusThreads;
    double* part = nullptr;
    cudaError_t e = cudaMallocAsync(&part, (size_t)blocks * sizeof(double), st);
    if (e != cudaSuccess) return cuda_error(e, "sdf_knn_mean_distance: scratch");
    {
        ProfRange pr(SDF_K_KNN, st);
        k_knn_mean<<<(unsigned)blocks, kRadiusThreads, 0, st>>>(a, k, part);
        e = cudaGetLastError();
    }
    std::vector<double> h((size_t)blocks);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h.data(), part, (size_t)blocks * sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFreeAsync(part, st);
    if (e != cudaSuccess) return cuda_error(e, "sdf_knn_mean_distance");
    double s = 0.0;
    for (double v : h) s += v;   // fixed order: the result does not depend on scheduling
    *D = s / (double)c.n;
    return SDF_OK;
}

// Sec. 4.2, "Acceleration and adaptive lambda": the paper's constant lambda =
// 10^3 / D with D the mean distance between a point and its 64 nearest
// neighbours, averaged over the cloud.
extern "C" sdf_status sdf_paper_lambda(sdf_cloud cloud, double* lambda, double* D, void* stream) {
    if (!cloud || !lambda) return set_error(SDF_EINVAL, "sdf_paper_lambda: NULL argument");
    double d = 0.0;
    const sdf_status s = sdf_knn_mean_distance(cloud, 64, &d, stream);
    if (s != SDF_OK) return s;
    if (D) *D = d;
    if (!(d > 0.0)) return set_error(SDF_EINVAL, "sdf_paper_lambda: D = 0 (a single point, or coincident points)");
    *lambda = 1e3 / d;
    return SDF_OK;
}
