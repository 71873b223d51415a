// sdf_query_grad: phi and its gradient in x (App. D, "Gradient expressions"),
// including the dependence of lambda_x = 2 C / d_max(x) on x; and
// sdf_query_laplacian: the same plus lap phi (App. D, "Laplacian"), with 15
// more sums per query (see finalize).
//
// With w_i = exp(-lambda (d_i - d_min)), n_i = (x - p_i) / d_i and phi = S / W:
//
//   grad phi = [ sum w_i grad g_i
//                - lambda ( sum w_i g_i n_i - phi sum w_i n_i )
//                - grad lambda ( sum w_i g_i d_i - phi sum w_i d_i ) ] / W,
//   grad lambda = -(lambda / d_max^2) (x - p_far)       (GLOBAL lambda; 0 if FIXED)
//
// (the first two terms are App. D's A + phi B for a constant lambda; the last
// is the derivative of lambda_x through the farthest point p_far).  The pair
// loop accumulates the 13 sums W, S, sum w grad g (3), sum w n (3),
// sum w g n (3), sum w d, sum w g d per query; nothing per pair is stored.
#include <cuda_runtime.h>

#include <cmath>

#include "query_common.cuh"
#include "f32x2_ops.cuh"
#include "prepass_warp.cuh"

namespace ptsdf {

using namespace qk;

namespace {

constexpr int kGradQPerCta = kConsumerWarps * 32;   // one query per consumer thread
// The Laplacian's 28 sums take 112 registers, so one CTA fills an SM's
// registers; it runs more consumer warps than the gradient (whose two CTAs of
// eight fit at 96): at most four warps of 3,584 registers per 16K sub-partition.
#ifndef PTSDF_LAP_WARPS
#define PTSDF_LAP_WARPS 12
#endif
constexpr int kLapWarps = PTSDF_LAP_WARPS;
static_assert(kLapWarps + 1 <= 16, "four warps per sub-partition at 112 registers");
template <bool LAP>
struct GradGeom {
    static constexpr int warps = LAP ? kLapWarps : kConsumerWarps;   // consumer warps
    static constexpr int threads = (warps + 1) * 32;                 // + producer warp
};
constexpr float kTiny = 1e-30f;                      // zero-length vectors get a zero unit vector

// accumulators: the 13 of the gradient, then the 15 more of the Laplacian
enum {
    A_W, A_S, A_GX, A_GY, A_GZ, A_NX, A_NY, A_NZ, A_HX, A_HY, A_HZ, A_D, A_GD,
    A_LG,                  // sum w lap g
    A_UG,                  // sum w <u, grad g>
    A_GR, A_R,             // sum w g / d, sum w / d
    A_DD, A_DDG,           // sum w d^2, sum w d^2 g
    A_DUX, A_DUY, A_DUZ,   // sum w d u = sum w (x - p)
    A_DHX, A_DHY, A_DHZ,   // sum w d g u
    A_DGX, A_DGY, A_DGZ,   // sum w d grad g
    A_COUNT_
};
template <bool LAP>
struct NAcc {
    static constexpr int value = LAP ? (int)A_COUNT_ : (int)A_LG;
};

struct GradArgs {
    QueryArgs a;
    const float4* pre;       // prepass array (farthest point position)
    float* grad;             // Q x 3 or null
    float* saved;            // Q x 8 or null
    float* lap;              // Q (Laplacian variant)
    float* part;             // split x Q x accumulator partials (split > 1)
};

// Accumulates one tile of pairs for one query into acc[].  WEIGHTED: each
// weight is multiplied by the point's weight A_i (record r3.w); A_i does not
// depend on x, so every sum below is weighted the same way.
template <bool KAPPA, bool LAP, bool WEIGHTED>
__device__ __forceinline__ void grad_tile(const float4* __restrict__ tile, int cnt, float x, float y, float z,
                                          float L, float A0, float (&acc)[NAcc<LAP>::value]) {
#pragma unroll 1
    for (int j = 0; j < cnt; ++j) {
        const float4 r0 = tile[4 * j], r1 = tile[4 * j + 1], r2 = tile[4 * j + 2];
        const float dx = x - r0.x, dy = y - r0.y, dz = z - r0.z;
        const float d2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
        const float rd = rsqrt_mufu(fmaxf(d2, kTiny));
        const float d = d2 * rd;
        float g, gx, gy, gz, lapg = 0.f;
        if (!KAPPA) {
            // direct form: g = sT (||(rho - R, h)|| - r), grad g = alpha v_perp + beta u
            const float vx = x - r1.x, vy = y - r1.y, vz = z - r1.z;
            const float h = fmaf(vx, r2.x, fmaf(vy, r2.y, vz * r2.z));
            const float px = fmaf(-h, r2.x, vx), py = fmaf(-h, r2.y, vy), pz = fmaf(-h, r2.z, vz);
            const float rho2 = fmaf(px, px, fmaf(py, py, pz * pz));
            const float rr = rsqrt_mufu(fmaxf(rho2, kTiny));
            const float e = fmaf(rho2, rr, -r1.w);
            const float Dt2 = fmaf(e, e, h * h);
            const float rD = rsqrt_mufu(fmaxf(Dt2, kTiny));
            g = fmaf(r0.w, Dt2 * rD, r2.w);
            const float sr = r0.w * rD;
            const float alpha = e * rr * sr, beta = h * sr;
            gx = fmaf(alpha, px, beta * r2.x);
            gy = fmaf(alpha, py, beta * r2.y);
            gz = fmaf(alpha, pz, beta * r2.z);
            // lap D = 1/D + (rho - R)/(rho D) for D the distance to the tube's centre circle
            if (LAP) lapg = r0.w * rD * fmaf(e, rr, 1.f);
        } else {
            // kappa form (see g_kappa): with s1 = sqrt(1 + k m), s2 = sqrt(1 + K N'),
            // K = -kappa_max, grad m = 2 k y_perp + m*, d a'/dm = 1/(2 s1),
            // dg/dN' = 1/(2 s2), dN'/da' = 2 K a' + 2 zeta, dN'/dh = 2 K h:
            //   grad g = c1 (2 k y_perp + m*) + (K h / s2) u,
            //   c1 = (2 K a' + 2 zeta) / (4 s1 s2)
            const float4 r3 = tile[4 * j + 3];
            const float yx = x - r1.x, yy = y - r1.y, yz = z - r1.z;
            const float h = fmaf(yx, r2.x, fmaf(yy, r2.y, yz * r2.z));
            const float hh = h * h;
            const float t2 = fmaf(yx, yx, fmaf(yy, yy, yz * yz)) - hh;
            const float m = fmaf(r1.w, t2, fmaf(yx, r3.x, fmaf(yy, r3.y, yz * r3.z)));
            const float z1 = fmaxf(fmaf(r1.w, m, 1.f), 0.f);
            const float rs1 = rsqrt_mufu(fmaxf(z1, kTiny));
            const float ap = m * rcp_mufu(1.f + z1 * rs1);
            const float Np = fmaf(r2.w, fmaf(ap, ap, hh), r0.w * ap);
            const float z2 = fmaxf(fmaf(r2.w, Np, 1.f), 0.f);
            const float rs2 = rsqrt_mufu(fmaxf(z2, kTiny));
            g = Np * rcp_mufu(1.f + z2 * rs2);
            const float c1 = 0.25f * rs1 * rs2 * fmaf(2.f * r2.w, ap, r0.w);
            const float ay = 2.f * c1 * r1.w;             // coefficient of y_perp
            const float bu = h * fmaf(rs2, r2.w, -ay);    // u coefficient after y_perp = y - h u
            gx = fmaf(ay, yx, fmaf(c1, r3.x, bu * r2.x));
            gy = fmaf(ay, yy, fmaf(c1, r3.y, bu * r2.y));
            gz = fmaf(ay, yz, fmaf(c1, r3.z, bu * r2.z));
            // lap m = 4k, |grad m|^2 = 4 s1^2 give lap a' = k / s1 and |grad a'| = 1;
            // then lap N' = 4K + (2K a' + 2 zeta) k / s1, |grad N'|^2 = 4 s2^2, so
            // lap g = (K + k (K a' + zeta) / s1) / s2
            if (LAP) lapg = fmaf(r1.w * fmaf(r2.w, ap, 0.5f * r0.w), rs1, r2.w) * rs2;
        }
        const float w = WEIGHTED ? ex2_mufu(fmaf(-L, d, A0)) * tile[4 * j + 3].w : ex2_mufu(fmaf(-L, d, A0));
        const float wg = w * g;
        const float wn = w * rd, wgn = wg * rd;
        acc[A_W] += w;
        acc[A_S] += wg;
        acc[A_GX] = fmaf(w, gx, acc[A_GX]);
        acc[A_GY] = fmaf(w, gy, acc[A_GY]);
        acc[A_GZ] = fmaf(w, gz, acc[A_GZ]);
        acc[A_NX] = fmaf(wn, dx, acc[A_NX]);
        acc[A_NY] = fmaf(wn, dy, acc[A_NY]);
        acc[A_NZ] = fmaf(wn, dz, acc[A_NZ]);
        acc[A_HX] = fmaf(wgn, dx, acc[A_HX]);
        acc[A_HY] = fmaf(wgn, dy, acc[A_HY]);
        acc[A_HZ] = fmaf(wgn, dz, acc[A_HZ]);
        acc[A_D] = fmaf(w, d, acc[A_D]);
        acc[A_GD] = fmaf(wg, d, acc[A_GD]);
        if (LAP) {
            const float wd = w * d, wgd = wg * d;
            acc[A_LG] = fmaf(w, lapg, acc[A_LG]);
            acc[A_UG] = fmaf(wn, fmaf(dx, gx, fmaf(dy, gy, dz * gz)), acc[A_UG]);
            acc[A_GR] = fmaf(wg, rd, acc[A_GR]);
            acc[A_R] = fmaf(w, rd, acc[A_R]);
            acc[A_DD] = fmaf(w, d2, acc[A_DD]);
            acc[A_DDG] = fmaf(wg, d2, acc[A_DDG]);
            acc[A_DUX] = fmaf(w, dx, acc[A_DUX]);
            acc[A_DUY] = fmaf(w, dy, acc[A_DUY]);
            acc[A_DUZ] = fmaf(w, dz, acc[A_DUZ]);
            acc[A_DHX] = fmaf(wg, dx, acc[A_DHX]);
            acc[A_DHY] = fmaf(wg, dy, acc[A_DHY]);
            acc[A_DHZ] = fmaf(wg, dz, acc[A_DHZ]);
            acc[A_DGX] = fmaf(wd, gx, acc[A_DGX]);
            acc[A_DGY] = fmaf(wd, gy, acc[A_DGY]);
            acc[A_DGZ] = fmaf(wd, gz, acc[A_DGZ]);
            (void)wgd;
        }
    }
}

// --------------------------------------------------------------------------
// The same tile two points at a time (the gradient without the Laplacian):
// the records come pair-interleaved (rec2: for points 2k, 2k+1 of a tile and
// each record float4 r_m, (r_m.x, r_m.x', r_m.y, r_m.y') then (r_m.z, r_m.z',
// r_m.w, r_m.w')), so every 128-bit shared load gives two .f32x2 operands and
// every FP32 step of the pair term runs for both points in one instruction;
// the special-function steps stay one per point.  acc2 holds the two points'
// partial sums side by side.  A pair's second point past the tile's `cnt`
// (a zero record) gets weight 0.
// --------------------------------------------------------------------------
__device__ __forceinline__ f32x2 f2_rsqrt_clamped(f32x2 v) {
    return f2_pack(rsqrt_mufu(fmaxf(f2_lo(v), kTiny)), rsqrt_mufu(fmaxf(f2_hi(v), kTiny)));
}

template <bool KAPPA, bool WEIGHTED>
__device__ __forceinline__ void grad_tile2(const ulonglong2* __restrict__ tile, int cnt, f32x2 X, f32x2 Y, f32x2 Z,
                                           f32x2 NL, f32x2 A0, f32x2 (&acc2)[A_LG]) {
    const f32x2 ONE = f2_splat(1.f), MONE = f2_splat(-1.f);
#pragma unroll 1
    for (int j = 0; j < cnt; j += 2) {
        const ulonglong2* r = tile + 4 * j;   // 8 x 16 B per pair of points
        const ulonglong2 a0 = r[0], b0 = r[1], a1 = r[2], b1 = r[3], a2 = r[4], b2 = r[5];
        const f32x2 DX = f2_sub(X, a0.x), DY = f2_sub(Y, a0.y), DZ = f2_sub(Z, b0.x);
        const f32x2 D2 = f2_fma(DX, DX, f2_fma(DY, DY, f2_mul(DZ, DZ)));
        const f32x2 RD = f2_rsqrt_clamped(D2);
        const f32x2 D = f2_mul(D2, RD);
        f32x2 G, GX, GY, GZ;
        if (!KAPPA) {
            // direct form (see grad_tile): g = sT (||(rho - R, h)|| - r), grad g = alpha v_perp + beta u
            const f32x2 VX = f2_sub(X, a1.x), VY = f2_sub(Y, a1.y), VZ = f2_sub(Z, b1.x);
            const f32x2 H = f2_fma(VX, a2.x, f2_fma(VY, a2.y, f2_mul(VZ, b2.x)));
            const f32x2 NH = f2_mul(H, MONE);
            const f32x2 PX = f2_fma(NH, a2.x, VX), PY = f2_fma(NH, a2.y, VY), PZ = f2_fma(NH, b2.x, VZ);
            const f32x2 RHO2 = f2_fma(PX, PX, f2_fma(PY, PY, f2_mul(PZ, PZ)));
            const f32x2 RR = f2_rsqrt_clamped(RHO2);
            const f32x2 E = f2_sub(f2_mul(RHO2, RR), b1.y);            // rho - R
            const f32x2 DT2 = f2_fma(E, E, f2_mul(H, H));
            const f32x2 RDT = f2_rsqrt_clamped(DT2);
            G = f2_fma(b0.y, f2_mul(DT2, RDT), b2.y);                  // sT D - sT r
            const f32x2 SR = f2_mul(b0.y, RDT);
            const f32x2 ALPHA = f2_mul(f2_mul(E, RR), SR), BETA = f2_mul(H, SR);
            GX = f2_fma(ALPHA, PX, f2_mul(BETA, a2.x));
            GY = f2_fma(ALPHA, PY, f2_mul(BETA, a2.y));
            GZ = f2_fma(ALPHA, PZ, f2_mul(BETA, b2.x));
        } else {
            // curvature form (see grad_tile)
            const ulonglong2 a3 = r[6], b3 = r[7];
            const f32x2 YX = f2_sub(X, a1.x), YY = f2_sub(Y, a1.y), YZ = f2_sub(Z, b1.x);
            const f32x2 H = f2_fma(YX, a2.x, f2_fma(YY, a2.y, f2_mul(YZ, b2.x)));
            const f32x2 HH = f2_mul(H, H);
            const f32x2 T2 = f2_sub(f2_fma(YX, YX, f2_fma(YY, YY, f2_mul(YZ, YZ))), HH);
            const f32x2 M = f2_fma(b1.y, T2, f2_fma(YX, a3.x, f2_fma(YY, a3.y, f2_mul(YZ, b3.x))));
            const f32x2 Z1 = f2_max0(f2_fma(b1.y, M, ONE));
            const f32x2 RS1 = f2_rsqrt_clamped(Z1);
            const f32x2 AP = f2_mul(M, f2_rcp(f2_fma(Z1, RS1, ONE)));
            const f32x2 NP = f2_fma(b2.y, f2_fma(AP, AP, HH), f2_mul(b0.y, AP));
            const f32x2 Z2 = f2_max0(f2_fma(b2.y, NP, ONE));
            const f32x2 RS2 = f2_rsqrt_clamped(Z2);
            G = f2_mul(NP, f2_rcp(f2_fma(Z2, RS2, ONE)));
            const f32x2 C1 = f2_mul(f2_mul(f2_splat(0.25f), f2_mul(RS1, RS2)),
                                    f2_fma(f2_add(b2.y, b2.y), AP, b0.y));
            const f32x2 AY = f2_mul(f2_add(C1, C1), b1.y);             // coefficient of y_perp
            const f32x2 BU = f2_mul(H, f2_sub(f2_mul(RS2, b2.y), AY)); // u coefficient after y_perp = y - h u
            GX = f2_fma(AY, YX, f2_fma(C1, a3.x, f2_mul(BU, a2.x)));
            GY = f2_fma(AY, YY, f2_fma(C1, a3.y, f2_mul(BU, a2.y)));
            GZ = f2_fma(AY, YZ, f2_fma(C1, b3.x, f2_mul(BU, b2.x)));
        }
        const f32x2 ARG = f2_fma(NL, D, A0);
        float w0 = ex2_mufu(f2_lo(ARG)), w1 = ex2_mufu(f2_hi(ARG));
        if (j + 1 >= cnt) w1 = 0.f;                                     // no second point
        f32x2 W = f2_pack(w0, w1);
        if (WEIGHTED) W = f2_mul(W, r[7].y);                            // (A, A') = r3.w of both
        const f32x2 WG = f2_mul(W, G), WN = f2_mul(W, RD), WGN = f2_mul(WG, RD);
        acc2[A_W] = f2_add(acc2[A_W], W);
        acc2[A_S] = f2_add(acc2[A_S], WG);
        acc2[A_GX] = f2_fma(W, GX, acc2[A_GX]);
        acc2[A_GY] = f2_fma(W, GY, acc2[A_GY]);
        acc2[A_GZ] = f2_fma(W, GZ, acc2[A_GZ]);
        acc2[A_NX] = f2_fma(WN, DX, acc2[A_NX]);
        acc2[A_NY] = f2_fma(WN, DY, acc2[A_NY]);
        acc2[A_NZ] = f2_fma(WN, DZ, acc2[A_NZ]);
        acc2[A_HX] = f2_fma(WGN, DX, acc2[A_HX]);
        acc2[A_HY] = f2_fma(WGN, DY, acc2[A_HY]);
        acc2[A_HZ] = f2_fma(WGN, DZ, acc2[A_HZ]);
        acc2[A_D] = f2_fma(W, D, acc2[A_D]);
        acc2[A_GD] = f2_fma(WG, D, acc2[A_GD]);
    }
}

// Pair-interleaved copy of the records (see grad_tile2), one thread per slot.
__global__ void k_pair_records(const float4* __restrict__ rec, int64_t slots, float* __restrict__ rec2) {
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= slots) return;
    const int64_t pair = s >> 1;   // tiles hold an even number of records, so pairs never straddle tiles
    const int half = (int)(s & 1);
    float* dst = rec2 + pair * 32;
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        const float4 v = rec[4 * s + m];
        dst[8 * m + half] = v.x;
        dst[8 * m + 2 + half] = v.y;
        dst[8 * m + 4 + half] = v.z;
        dst[8 * m + 6 + half] = v.w;
    }
}

// Per-query lambda and shift from the prepass partials; p_far for GLOBAL.
struct QueryLam {
    float L, A0, lam, dmax;
    float fx, fy, fz;
};

__device__ __forceinline__ QueryLam query_lambda(const QueryArgs& a, const float4* __restrict__ pre, int64_t qq) {
    QueryLam r;
    float2 d2 = a.d2[qq];
    int32_t far = a.far ? a.far[qq] : 0;
    for (int c = 1; c < a.pre_split; ++c) {
        const float2 v = a.d2[(size_t)c * a.q + qq];
        if (v.x > d2.x) {
            d2.x = v.x;
            if (a.far) far = a.far[(size_t)c * a.q + qq];
        }
        d2.y = fminf(d2.y, v.y);
    }
    const float dmin = sqrtf(fmaxf(d2.y, 0.f));
    r.dmax = sqrtf(fmaxf(d2.x, 0.f));
    r.lam = a.lam;
    r.fx = r.fy = r.fz = 0.f;
    if (a.mode == SDF_LAMBDA_GLOBAL) {
        r.lam = r.dmax > 0.f ? 2.f * a.C / r.dmax : 0.f;
        const float4 pf = pre[far];   // (-2 p', |p'|^2), p' = p - centre
        r.fx = fmaf(-0.5f, pf.x, a.cx);
        r.fy = fmaf(-0.5f, pf.y, a.cy);
        r.fz = fmaf(-0.5f, pf.z, a.cz);
    }
    r.L = r.lam * kLog2e;
    r.A0 = r.L * dmin;
    return r;
}

template <bool LAP>
__device__ __forceinline__ void finalize(const GradArgs& ga, int64_t qi, float x, float y, float z,
                                         const QueryLam& ql, const float (&acc)[NAcc<LAP>::value]) {
    const QueryArgs& a = ga.a;
    const float invW = 1.f / acc[A_W];
    const float phi = acc[A_S] * invW;
    const bool lam_x = a.mode == SDF_LAMBDA_GLOBAL && ql.dmax > 0.f;
    float glx = 0.f, gly = 0.f, glz = 0.f;
    if (lam_x) {
        const float s = -ql.lam / (ql.dmax * ql.dmax);
        glx = s * (x - ql.fx);
        gly = s * (y - ql.fy);
        glz = s * (z - ql.fz);
    }
    if (a.formula == SDF_FORMULA_LSE) {
        // the log-sum-exp distance d~ = (A0 - log2 W) / L (Eq. ConvolutionalDistanceFormula,
        // h = 1) and its gradient sum w n / W + ((sum w d / W - d~) / lambda) grad lambda:
        // the second term is d d~ / d lambda times the gradient of lambda_x
        const float dt = ql.L > 0.f ? (ql.A0 - log2f(acc[A_W])) / ql.L : 0.f;
        float gx = acc[A_NX] * invW, gy = acc[A_NY] * invW, gz = acc[A_NZ] * invW;
        if (lam_x) {
            const float c = fmaf(acc[A_D], invW, -dt) / ql.lam;
            gx = fmaf(c, glx, gx);
            gy = fmaf(c, gly, gy);
            gz = fmaf(c, glz, gz);
        }
        if (a.phi) a.phi[qi] = dt - a.offset;
        if (ga.grad) {
            ga.grad[3 * qi] = gx;
            ga.grad[3 * qi + 1] = gy;
            ga.grad[3 * qi + 2] = gz;
        }
        return;
    }
    const float cd = fmaf(-phi, acc[A_D], acc[A_GD]);   // sum w g d - phi sum w d
    // grad phi at constant lambda (App. D: A + phi B), then the lambda_x term
    const float fx = (acc[A_GX] - ql.lam * fmaf(-phi, acc[A_NX], acc[A_HX])) * invW;
    const float fy = (acc[A_GY] - ql.lam * fmaf(-phi, acc[A_NY], acc[A_HY])) * invW;
    const float fz = (acc[A_GZ] - ql.lam * fmaf(-phi, acc[A_NZ], acc[A_HZ])) * invW;
    const float gx = fmaf(-glx, cd * invW, fx), gy = fmaf(-gly, cd * invW, fy), gz = fmaf(-glz, cd * invW, fz);
    if (a.phi) a.phi[qi] = phi - a.offset;
    if (ga.grad) {
        ga.grad[3 * qi] = gx;
        ga.grad[3 * qi + 1] = gy;
        ga.grad[3 * qi + 2] = gz;
    }
    if (LAP) {
        // Laplacian at constant lambda (App. D, "Laplacian"), with the
        // lambda^2 terms cancelled analytically:
        //   lap_x F = [sum w lap g - 2 lambda (sum w <u, grad g> + sum w (g - F) / d)] / W
        //             + 2 <B, grad_x F>,   B = lambda sum w u / W
        const float bx = ql.lam * acc[A_NX] * invW, by = ql.lam * acc[A_NY] * invW, bz = ql.lam * acc[A_NZ] * invW;
        const float gr = fmaf(-phi, acc[A_R], acc[A_GR]);
        float lap = fmaf(-2.f * ql.lam, acc[A_UG] + gr, acc[A_LG]) * invW +
                    2.f * fmaf(bx, fx, fmaf(by, fy, bz * fz));
        if (lam_x) {
            // lambda_x = 2C / d_max(x) is harmonic (lap of 1/r is 0), so
            //   lap phi = lap_x F + 2 <grad_x F_lambda, grad lambda> + F_lambda_lambda |grad lambda|^2
            const float Fl = -cd * invW;
            const float md = acc[A_D] * invW;
            const float Fll = fmaf(-phi, acc[A_DD], acc[A_DDG]) * invW + 2.f * Fl * md;
            // grad_x F_lambda = [grad_x F M_d - (sum w g u - F sum w u) + lambda (sum w d g u - F sum w d u)
            //                    - sum w d grad g] / W + F_lambda B
            const float hx = fmaf(-phi, acc[A_NX], acc[A_HX]), hy = fmaf(-phi, acc[A_NY], acc[A_HY]),
                        hz = fmaf(-phi, acc[A_NZ], acc[A_HZ]);
            const float ex = fmaf(-phi, acc[A_DUX], acc[A_DHX]), ey = fmaf(-phi, acc[A_DUY], acc[A_DHY]),
                        ez = fmaf(-phi, acc[A_DUZ], acc[A_DHZ]);
            const float qx = fmaf(fx, acc[A_D], fmaf(ql.lam, ex, -hx - acc[A_DGX])) * invW + Fl * bx;
            const float qy = fmaf(fy, acc[A_D], fmaf(ql.lam, ey, -hy - acc[A_DGY])) * invW + Fl * by;
            const float qz = fmaf(fz, acc[A_D], fmaf(ql.lam, ez, -hz - acc[A_DGZ])) * invW + Fl * bz;
            const float gl2 = fmaf(glx, glx, fmaf(gly, gly, glz * glz));
            lap += 2.f * fmaf(qx, glx, fmaf(qy, gly, qz * glz)) + Fll * gl2;
        }
        ga.lap[qi] = lap;
    } else if (ga.saved) {
        float* s = ga.saved + 8 * qi;
        s[0] = x;
        s[1] = y;
        s[2] = z;
        s[3] = ql.L;
        s[4] = ql.A0;
        s[5] = acc[A_W];
        s[6] = phi;
        s[7] = 0.f;
    }
}

template <bool LAP, bool WEIGHTED>
__global__ void __launch_bounds__(GradGeom<LAP>::threads) __maxnreg__(LAP ? 112 : 96) k_fwd_grad(const float4* __restrict__ rec, int64_t n_direct,
                                                       int64_t n_kappa, int64_t tiles_direct, int64_t tiles_total,
                                                       int64_t tiles_per_chunk, GradArgs ga, int32_t* status) {
    extern __shared__ __align__(128) char smem[];
    __shared__ TileRing<kStages> ring;
    char* buf = smem;
    const QueryArgs& a = ga.a;
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int chunk = blockIdx.y;
    const int64_t t0 = (int64_t)chunk * tiles_per_chunk;
    const int64_t t1 = t0 + tiles_per_chunk < tiles_total ? t0 + tiles_per_chunk : tiles_total;
    const int64_t nt = t1 > t0 ? t1 - t0 : 0;
    constexpr int kWarps = GradGeom<LAP>::warps;
    if (threadIdx.x == 0) ring.init(kWarps);
    __syncthreads();
    if (warp == kWarps) {
        if (lane == 0)
            ring.produce(buf, reinterpret_cast<const char*>(rec + t0 * kTileRecs * 4), nt, kTileBytes, status);
        return;
    }
    const int64_t qi = (int64_t)blockIdx.x * (kWarps * 32) + threadIdx.x;
    const int64_t qq = qi < a.q ? qi : a.q - 1;
    const float x = a.x[3 * qq], y = a.x[3 * qq + 1], z = a.x[3 * qq + 2];
    const QueryLam ql = query_lambda(a, ga.pre, qq);
    constexpr int kAcc = NAcc<LAP>::value;
    float acc[kAcc];
#pragma unroll
    for (int k = 0; k < kAcc; ++k) acc[k] = 0.f;
    if (LAP) {
        // the Laplacian's 28 sums: one point at a time from the plain records
        float tacc[kAcc];
        for (int64_t t = 0; t < nt; ++t) {
            if (!ring.wait_full(t, status)) return;
            const float4* tile = reinterpret_cast<const float4*>(buf + (size_t)(t % kStages) * kTileBytes);
            const int64_t gt = t0 + t;
            const bool kappa = gt >= tiles_direct;
            const int64_t first = (kappa ? gt - tiles_direct : gt) * kTileRecs;
            const int64_t seg = kappa ? n_kappa : n_direct;
            const int cnt = (int)(seg - first < kTileRecs ? seg - first : kTileRecs);
#pragma unroll
            for (int k = 0; k < kAcc; ++k) tacc[k] = 0.f;
            if (kappa)
                grad_tile<true, LAP, WEIGHTED>(tile, cnt, x, y, z, ql.L, ql.A0, tacc);
            else
                grad_tile<false, LAP, WEIGHTED>(tile, cnt, x, y, z, ql.L, ql.A0, tacc);
#pragma unroll
            for (int k = 0; k < kAcc; ++k) acc[k] += tacc[k];
            ring.release(t, lane);
        }
    } else {
        // the gradient's 13 sums: two points at a time from the pair-interleaved records
        // (each half sums every other point; no per-tile blocking, to keep two CTAs per SM)
        const f32x2 X = f2_splat(x), Y = f2_splat(y), Z = f2_splat(z), NL = f2_splat(-ql.L), A0 = f2_splat(ql.A0);
        f32x2 acc2[A_LG];
#pragma unroll
        for (int k = 0; k < A_LG; ++k) acc2[k] = f2_splat(0.f);
        for (int64_t t = 0; t < nt; ++t) {
            if (!ring.wait_full(t, status)) return;
            const ulonglong2* tile = reinterpret_cast<const ulonglong2*>(buf + (size_t)(t % kStages) * kTileBytes);
            const int64_t gt = t0 + t;
            const bool kappa = gt >= tiles_direct;
            const int64_t first = (kappa ? gt - tiles_direct : gt) * kTileRecs;
            const int64_t seg = kappa ? n_kappa : n_direct;
            const int cnt = (int)(seg - first < kTileRecs ? seg - first : kTileRecs);
            if (kappa)
                grad_tile2<true, WEIGHTED>(tile, cnt, X, Y, Z, NL, A0, acc2);
            else
                grad_tile2<false, WEIGHTED>(tile, cnt, X, Y, Z, NL, A0, acc2);
            ring.release(t, lane);
        }
#pragma unroll
        for (int k = 0; k < A_LG; ++k) acc[k] = f2_lo(acc2[k]) + f2_hi(acc2[k]);
    }
    if (qi >= a.q) return;
    if (a.split == 1) {
        finalize<LAP>(ga, qi, x, y, z, ql, acc);
    } else {
        float* dst = ga.part + ((size_t)chunk * a.q + qi) * kAcc;
#pragma unroll
        for (int k = 0; k < kAcc; ++k) dst[k] = acc[k];
    }
}

template <bool LAP>
__global__ void k_merge_grad(GradArgs ga) {
    constexpr int kAcc = NAcc<LAP>::value;
    const QueryArgs& a = ga.a;
    const int64_t qi = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (qi >= a.q) return;
    float acc[kAcc];
#pragma unroll
    for (int k = 0; k < kAcc; ++k) acc[k] = 0.f;
    for (int c = 0; c < a.split; ++c) {
        const float* src = ga.part + ((size_t)c * a.q + qi) * kAcc;
#pragma unroll
        for (int k = 0; k < kAcc; ++k) acc[k] += src[k];
    }
    const QueryLam ql = query_lambda(a, ga.pre, qi);
    finalize<LAP>(ga, qi, a.x[3 * qi], a.x[3 * qi + 1], a.x[3 * qi + 2], ql, acc);
}

}  // namespace

sdf_status launch_query_grad(const Cloud& c, const float* d_x, int64_t q, float* d_phi, float* d_grad,
                             float* d_saved, const sdf_query_opts& o, cudaStream_t st, float* d_lap) {
    const bool lap = d_lap != nullptr;
    const int kAcc = lap ? NAcc<true>::value : NAcc<false>::value;
    const Plan p = make_plan(c, q, o.split_n, lap ? GradGeom<true>::warps * 32 : kGradQPerCta);
    GradArgs ga;
    QueryArgs& a = ga.a;
    a.x = d_x;
    a.q = q;
    a.phi = d_phi;
    a.split = p.split;
    a.mode = o.lambda_mode;
    a.C = o.C;
    a.lam = o.fixed_lambda;
    a.offset = o.offset;
    a.formula = o.formula;
    a.part = nullptr;
    a.d2 = nullptr;
    a.far = nullptr;
    a.cx = 0.5f * (c.aabb[0] + c.aabb[3]);
    a.cy = 0.5f * (c.aabb[1] + c.aabb[4]);
    a.cz = 0.5f * (c.aabb[2] + c.aabb[5]);
    a.cloud_radius = 0.5f * c.aabb_diag * (1.f + 1e-6f);
    ga.pre = c.pre;
    ga.grad = d_grad;
    ga.saved = d_saved;
    ga.lap = d_lap;
    ga.part = nullptr;
    auto oom = [&](cudaError_t e) {
        if (a.d2) cudaFreeAsync(a.d2, st);
        if (a.far) cudaFreeAsync(a.far, st);
        if (ga.part) cudaFreeAsync(ga.part, st);
        return e == cudaErrorMemoryAllocation ? set_error(SDF_ENOMEM, "sdf_query_grad: scratch")
                                              : cuda_error(e, "sdf_query_grad: scratch");
    };
    const bool warp_pre = use_warp_prepass(c, p, o), pruned = !warp_pre && use_pruned_prepass(c, p, o);
    a.pre_split = pruned || warp_pre ? 1 : p.split;
    cudaError_t e = cudaMallocAsync(&a.d2, (size_t)a.pre_split * q * sizeof(float2), st);
    if (e != cudaSuccess) return oom(e);
    if (o.lambda_mode == SDF_LAMBDA_GLOBAL) {
        e = cudaMallocAsync(&a.far, (size_t)a.pre_split * q * sizeof(int32_t), st);
        if (e != cudaSuccess) return oom(e);
    }
    if (p.split > 1) {
        e = cudaMallocAsync(&ga.part, (size_t)p.split * q * kAcc * sizeof(float), st);
        if (e != cudaSuccess) return oom(e);
    }
    const dim3 grid((unsigned)p.qblocks, (unsigned)p.split);
    const dim3 pre_grid((unsigned)p.pre_qblocks, (unsigned)p.split);
    {
        ProfRange pr(SDF_K_PREPASS, st);
        if (pruned)
            k_prepass_pruned<true><<<(unsigned)p.pre_qblocks, kPrunedThreads, 0, st>>>(c.pre, c.spheres, c.n,
                                                                                    c.n_spheres, a);
        else if (warp_pre)
            launch_prepass_warp(c, a, true, st);
        else if (o.lambda_mode == SDF_LAMBDA_GLOBAL)
            k_prepass<SDF_LAMBDA_GLOBAL, true><<<pre_grid, kThreads, kStages * kPreBytes, st>>>(
                c.pre, c.n, c.pre_tiles, p.pre_tiles_per_chunk, a, c.status);
        else
            k_prepass<SDF_LAMBDA_FIXED, false><<<pre_grid, kThreads, kStages * kPreBytes, st>>>(
                c.pre, c.n, c.pre_tiles, p.pre_tiles_per_chunk, a, c.status);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        ProfRange pr(SDF_K_FWD_GRAD, st);
        auto kern = lap ? (c.weighted ? k_fwd_grad<true, true> : k_fwd_grad<true, false>)
                        : (c.weighted ? k_fwd_grad<false, true> : k_fwd_grad<false, false>);
        // the gradient takes the pair-interleaved copy, the Laplacian the plain records
        kern<<<grid, lap ? GradGeom<true>::threads : GradGeom<false>::threads, kStages * kTileBytes, st>>>(
            lap ? c.rec : c.rec2, c.n_direct, c.n_kappa, c.tiles_direct, c.tiles_direct + c.tiles_kappa,
            p.tiles_per_chunk, ga, c.status);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && p.split > 1) {
        ProfRange pr(SDF_K_MERGE, st);
        (lap ? k_merge_grad<true> : k_merge_grad<false>)<<<(unsigned)((q + 255) / 256), 256, 0, st>>>(ga);
        e = cudaGetLastError();
    }
    cudaFreeAsync(a.d2, st);
    if (a.far) cudaFreeAsync(a.far, st);
    if (ga.part) cudaFreeAsync(ga.part, st);
    return e == cudaSuccess ? SDF_OK : cuda_error(e, "sdf_query_grad: launch");
}

sdf_status build_pair_records(Cloud& c, cudaStream_t st) {
    const int64_t slots = (c.tiles_direct + c.tiles_kappa) * kTileRecs;
    if (slots == 0) return SDF_OK;
    cudaError_t e = cudaMalloc(&c.rec2, (size_t)slots * 4 * sizeof(float4));
    if (e != cudaSuccess)
        return e == cudaErrorMemoryAllocation ? set_error(SDF_ENOMEM, "sdf_build: paired records")
                                              : cuda_error(e, "sdf_build: paired records");
    k_pair_records<<<(unsigned)((slots + 255) / 256), 256, 0, st>>>(c.rec, slots, reinterpret_cast<float*>(c.rec2));
    e = cudaGetLastError();
    return e == cudaSuccess ? SDF_OK : cuda_error(e, "sdf_build: k_pair_records");
}

}  // namespace ptsdf
