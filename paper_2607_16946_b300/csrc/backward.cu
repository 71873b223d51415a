// sdf_backward_params: dL/da for L = sum_q G_q phi(x_q).
//
// The weights w_qi = exp(-lambda_q (|x_q - p_i| - d_min,q)) do not depend on
// the coefficients a_i, so
//   dL/da_i = sum_q (G_q / W_q) w_qi  d g_i(x_q) / d a_i
//           = sum_theta [ sum_q (G_q / W_q) w_qi d g_i(x_q) / d theta ] d theta / d a_i,
// where theta is the packed torus record of point i.  The inner sum runs in a
// point-major kernel (one record per thread, the queries' saved statistics
// streamed through the shared-memory ring); the outer product with the fit's
// Jacobian d theta / d a runs once per point in double precision with
// forward-mode dual numbers through the same fit as sdf_build.
//
//   direct record theta = (c, u, R, r):
//     dg/dc = -(alpha v_perp + beta u),  dg/du = beta v - h alpha v_perp,
//     dg/dR = -sT e / D,  dg/dr = -sT
//   with v = x - c, h = <v, u>, v_perp = v - h u, e = |v_perp| - R,
//   D = ||(e, h)||, alpha = sT e / (|v_perp| D), beta = sT h / D.
//   kappa record theta = (q, u, m* = 2 zeta n*, k = |kappa_min|, K = -kappa_max):
//     dg/dq = -grad_x g,  dg/du = bu y,  dg/dm* = c1 y,
//     dg/dk = c1 (t^2 - a'^2),  dg/dK = (a'^2 + h^2 - g^2) / (2 s2)
//   with the quantities of the curvature form (see grad.cu).
#include <cuda_runtime.h>

#include <cmath>

#include "device_common.cuh"
#include "f32x2_ops.cuh"
#include "fit_math.cuh"
#include "internal.h"

namespace ptsdf {

namespace {

constexpr int kThreads = (kConsumerWarps + 1) * 32;
constexpr int kPointsPerCta = kConsumerWarps * 32;     // one record per consumer thread
constexpr int kQTile = 64;                             // queries per streamed tile
constexpr uint32_t kQTileBytes = kQTile * 6 * sizeof(float);   // 32 pairs x 3 float4
constexpr int kNAcc = 11;
constexpr float kTiny = 1e-30f;

// The queries' streamed records, two queries side by side: for queries 2k and
// 2k + 1, (x, x', y, y'), (z, z', L, L'), (A0, A0', G / W, G' / W'), so that
// every 128-bit shared load gives two .f32x2 operands.  Padding queries have
// coefficient 0.
__global__ void k_bwd_prep(const float* __restrict__ saved, const float* __restrict__ G, int64_t q,
                           int64_t q_padded, float* __restrict__ qrec) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= q_padded) return;
    float v[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};   // x, y, z, L, A0, G / W
    if (j < q) {
        const float* s = saved + 8 * j;
        v[0] = s[0];
        v[1] = s[1];
        v[2] = s[2];
        v[3] = s[3];
        v[4] = s[4];
        v[5] = G[j] / s[5];
    }
    float* dst = qrec + (j >> 1) * 12 + (j & 1);
#pragma unroll
    for (int k = 0; k < 6; ++k) dst[2 * k] = v[k];
}

__device__ __forceinline__ f32x2 f2_rsqrt_clamped(f32x2 v) {
    return f2_pack(rsqrt_mufu(fmaxf(f2_lo(v), kTiny)), rsqrt_mufu(fmaxf(f2_hi(v), kTiny)));
}

// The record of this thread's point as pairs (both halves the same value).
struct Rec2 {
    f32x2 p[3], c[3], u[3], m[3];   // r0.xyz, r1.xyz, r2.xyz, r3.xyz
    f32x2 s0, s1, s2, s3;           // r0.w, r1.w, r2.w, r3.w
};

__device__ __forceinline__ Rec2 rec2_of(const float4& r0, const float4& r1, const float4& r2, const float4& r3) {
    Rec2 R;
    R.p[0] = f2_splat(r0.x); R.p[1] = f2_splat(r0.y); R.p[2] = f2_splat(r0.z);
    R.c[0] = f2_splat(r1.x); R.c[1] = f2_splat(r1.y); R.c[2] = f2_splat(r1.z);
    R.u[0] = f2_splat(r2.x); R.u[1] = f2_splat(r2.y); R.u[2] = f2_splat(r2.z);
    R.m[0] = f2_splat(r3.x); R.m[1] = f2_splat(r3.y); R.m[2] = f2_splat(r3.z);
    R.s0 = f2_splat(r0.w); R.s1 = f2_splat(r1.w); R.s2 = f2_splat(r2.w); R.s3 = f2_splat(r3.w);
    return R;
}

// The sums of bwd_tile for two queries at a time (one per half of every
// pair), the FP32 arithmetic as .f32x2, one special-function step per query.
template <bool KAPPA, bool WEIGHTED>
__device__ __forceinline__ void bwd_tile2(const ulonglong2* __restrict__ tile, const Rec2& R,
                                          f32x2 (&acc)[kNAcc]) {
    const f32x2 ONE = f2_splat(1.f), MONE = f2_splat(-1.f);
#pragma unroll 1
    for (int j = 0; j < kQTile / 2; ++j) {
        const ulonglong2 qa = tile[3 * j], qb = tile[3 * j + 1], qc = tile[3 * j + 2];
        const f32x2 X = qa.x, Y = qa.y, Z = qb.x;
        const f32x2 DX = f2_sub(X, R.p[0]), DY = f2_sub(Y, R.p[1]), DZ = f2_sub(Z, R.p[2]);
        const f32x2 D2 = f2_fma(DX, DX, f2_fma(DY, DY, f2_mul(DZ, DZ)));
        const f32x2 D = f2_pack(sqrt_mufu(f2_lo(D2)), sqrt_mufu(f2_hi(D2)));
        const f32x2 ARG = f2_sub(qc.x, f2_mul(qb.y, D));                    // A0 - L d
        f32x2 CW = f2_mul(qc.y, f2_pack(ex2_mufu(f2_lo(ARG)), ex2_mufu(f2_hi(ARG))));   // (G/W) w
        if (WEIGHTED) CW = f2_mul(CW, R.s3);
        if (!KAPPA) {
            const f32x2 VX = f2_sub(X, R.c[0]), VY = f2_sub(Y, R.c[1]), VZ = f2_sub(Z, R.c[2]);
            const f32x2 H = f2_fma(VX, R.u[0], f2_fma(VY, R.u[1], f2_mul(VZ, R.u[2])));
            const f32x2 NH = f2_mul(H, MONE);
            const f32x2 PX = f2_fma(NH, R.u[0], VX), PY = f2_fma(NH, R.u[1], VY), PZ = f2_fma(NH, R.u[2], VZ);
            const f32x2 RHO2 = f2_fma(PX, PX, f2_fma(PY, PY, f2_mul(PZ, PZ)));
            const f32x2 RR = f2_rsqrt_clamped(RHO2);
            const f32x2 E = f2_sub(f2_mul(RHO2, RR), R.s1);
            const f32x2 RD = f2_rsqrt_clamped(f2_fma(E, E, f2_mul(H, H)));
            const f32x2 SR = f2_mul(R.s0, RD);
            const f32x2 CA = f2_mul(CW, f2_mul(f2_mul(E, RR), SR)), CB = f2_mul(CW, f2_mul(H, SR));
            const f32x2 NCA = f2_mul(CA, MONE), NCB = f2_mul(CB, MONE), NCHA = f2_mul(NH, CA);
            acc[0] = f2_fma(NCA, PX, f2_fma(NCB, R.u[0], acc[0]));
            acc[1] = f2_fma(NCA, PY, f2_fma(NCB, R.u[1], acc[1]));
            acc[2] = f2_fma(NCA, PZ, f2_fma(NCB, R.u[2], acc[2]));
            acc[3] = f2_fma(CB, VX, f2_fma(NCHA, PX, acc[3]));
            acc[4] = f2_fma(CB, VY, f2_fma(NCHA, PY, acc[4]));
            acc[5] = f2_fma(CB, VZ, f2_fma(NCHA, PZ, acc[5]));
            acc[6] = f2_fma(f2_mul(CW, MONE), f2_mul(E, SR), acc[6]);
            acc[7] = f2_add(acc[7], CW);                                      // times -sT at the end
        } else {
            const f32x2 YX = f2_sub(X, R.c[0]), YY = f2_sub(Y, R.c[1]), YZ = f2_sub(Z, R.c[2]);
            const f32x2 H = f2_fma(YX, R.u[0], f2_fma(YY, R.u[1], f2_mul(YZ, R.u[2])));
            const f32x2 HH = f2_mul(H, H);
            const f32x2 T2 = f2_sub(f2_fma(YX, YX, f2_fma(YY, YY, f2_mul(YZ, YZ))), HH);
            const f32x2 M = f2_fma(R.s1, T2, f2_fma(YX, R.m[0], f2_fma(YY, R.m[1], f2_mul(YZ, R.m[2]))));
            const f32x2 Z1 = f2_max0(f2_fma(R.s1, M, ONE));
            const f32x2 RS1 = f2_rsqrt_clamped(Z1);
            const f32x2 AP = f2_mul(M, f2_rcp(f2_fma(Z1, RS1, ONE)));
            const f32x2 AA = f2_mul(AP, AP);
            const f32x2 NP = f2_fma(R.s2, f2_add(AA, HH), f2_mul(R.s0, AP));
            const f32x2 Z2 = f2_max0(f2_fma(R.s2, NP, ONE));
            const f32x2 RS2 = f2_rsqrt_clamped(Z2);
            const f32x2 G = f2_mul(NP, f2_rcp(f2_fma(Z2, RS2, ONE)));
            const f32x2 C1 = f2_mul(f2_mul(f2_splat(0.25f), f2_mul(RS1, RS2)), f2_fma(f2_add(R.s2, R.s2), AP, R.s0));
            const f32x2 AY = f2_mul(f2_add(C1, C1), R.s1);
            const f32x2 BU = f2_mul(H, f2_sub(f2_mul(RS2, R.s2), AY));
            const f32x2 CAY = f2_mul(CW, AY), CC1 = f2_mul(CW, C1), CBU = f2_mul(CW, BU);
            const f32x2 NCAY = f2_mul(CAY, MONE), NCC1 = f2_mul(CC1, MONE), NCBU = f2_mul(CBU, MONE);
            // dg/dq = -(ay y + c1 m* + bu u)
            acc[0] = f2_fma(NCAY, YX, f2_fma(NCC1, R.m[0], f2_fma(NCBU, R.u[0], acc[0])));
            acc[1] = f2_fma(NCAY, YY, f2_fma(NCC1, R.m[1], f2_fma(NCBU, R.u[1], acc[1])));
            acc[2] = f2_fma(NCAY, YZ, f2_fma(NCC1, R.m[2], f2_fma(NCBU, R.u[2], acc[2])));
            acc[3] = f2_fma(CBU, YX, acc[3]);                                 // dg/du = bu y
            acc[4] = f2_fma(CBU, YY, acc[4]);
            acc[5] = f2_fma(CBU, YZ, acc[5]);
            acc[6] = f2_fma(CC1, YX, acc[6]);                                 // dg/dm* = c1 y
            acc[7] = f2_fma(CC1, YY, acc[7]);
            acc[8] = f2_fma(CC1, YZ, acc[8]);
            acc[9] = f2_fma(CC1, f2_sub(T2, AA), acc[9]);                     // dg/dk
            acc[10] = f2_fma(f2_mul(f2_splat(0.5f), f2_mul(CW, RS2)),        // dg/dK
                             f2_sub(f2_add(AA, HH), f2_mul(G, G)), acc[10]);
        }
    }
}

// WEIGHTED: the weight is multiplied by this point's weight A_i (r3.w).
template <bool KAPPA, bool WEIGHTED>
__device__ __forceinline__ void bwd_tile(const float4* __restrict__ tile, const float4& r0, const float4& r1,
                                         const float4& r2, const float4& r3, float (&acc)[kNAcc]) {
#pragma unroll 1
    for (int j = 0; j < kQTile; ++j) {
        const float4 qa = tile[2 * j], qb = tile[2 * j + 1];
        const float x = qa.x, y = qa.y, z = qa.z;
        const float dx = x - r0.x, dy = y - r0.y, dz = z - r0.z;
        const float d = sqrt_mufu(fmaf(dx, dx, fmaf(dy, dy, dz * dz)));
        const float cw = qb.y * (WEIGHTED ? ex2_mufu(fmaf(-qa.w, d, qb.x)) * r3.w
                                          : ex2_mufu(fmaf(-qa.w, d, qb.x)));   // (G/W) w
        if (!KAPPA) {
            const float vx = x - r1.x, vy = y - r1.y, vz = z - r1.z;
            const float h = fmaf(vx, r2.x, fmaf(vy, r2.y, vz * r2.z));
            const float px = fmaf(-h, r2.x, vx), py = fmaf(-h, r2.y, vy), pz = fmaf(-h, r2.z, vz);
            const float rho2 = fmaf(px, px, fmaf(py, py, pz * pz));
            const float rr = rsqrt_mufu(fmaxf(rho2, kTiny));
            const float e = fmaf(rho2, rr, -r1.w);
            const float rD = rsqrt_mufu(fmaxf(fmaf(e, e, h * h), kTiny));
            const float sr = r0.w * rD;
            const float ca = cw * (e * rr * sr), cb = cw * (h * sr), cha = h * ca;
            acc[0] = fmaf(-ca, px, fmaf(-cb, r2.x, acc[0]));
            acc[1] = fmaf(-ca, py, fmaf(-cb, r2.y, acc[1]));
            acc[2] = fmaf(-ca, pz, fmaf(-cb, r2.z, acc[2]));
            acc[3] = fmaf(cb, vx, fmaf(-cha, px, acc[3]));
            acc[4] = fmaf(cb, vy, fmaf(-cha, py, acc[4]));
            acc[5] = fmaf(cb, vz, fmaf(-cha, pz, acc[5]));
            acc[6] = fmaf(-cw, e * sr, acc[6]);
            acc[7] += cw;                                  // times -sT at the end
        } else {
            const float yx = x - r1.x, yy = y - r1.y, yz = z - r1.z;
            const float h = fmaf(yx, r2.x, fmaf(yy, r2.y, yz * r2.z));
            const float hh = h * h;
            const float t2 = fmaf(yx, yx, fmaf(yy, yy, yz * yz)) - hh;
            const float m = fmaf(r1.w, t2, fmaf(yx, r3.x, fmaf(yy, r3.y, yz * r3.z)));
            const float z1 = fmaxf(fmaf(r1.w, m, 1.f), 0.f);
            const float rs1 = rsqrt_mufu(fmaxf(z1, kTiny));
            const float ap = m * rcp_mufu(1.f + z1 * rs1);
            const float aa = ap * ap;
            const float Np = fmaf(r2.w, aa + hh, r0.w * ap);
            const float z2 = fmaxf(fmaf(r2.w, Np, 1.f), 0.f);
            const float rs2 = rsqrt_mufu(fmaxf(z2, kTiny));
            const float g = Np * rcp_mufu(1.f + z2 * rs2);
            const float c1 = 0.25f * rs1 * rs2 * fmaf(2.f * r2.w, ap, r0.w);
            const float ay = 2.f * c1 * r1.w;
            const float bu = h * fmaf(rs2, r2.w, -ay);
            const float cay = cw * ay, cc1 = cw * c1, cbu = cw * bu;
            // dg/dq = -(ay y + c1 m* + bu u)
            acc[0] = fmaf(-cay, yx, fmaf(-cc1, r3.x, fmaf(-cbu, r2.x, acc[0])));
            acc[1] = fmaf(-cay, yy, fmaf(-cc1, r3.y, fmaf(-cbu, r2.y, acc[1])));
            acc[2] = fmaf(-cay, yz, fmaf(-cc1, r3.z, fmaf(-cbu, r2.z, acc[2])));
            acc[3] = fmaf(cbu, yx, acc[3]);               // dg/du = bu y
            acc[4] = fmaf(cbu, yy, acc[4]);
            acc[5] = fmaf(cbu, yz, acc[5]);
            acc[6] = fmaf(cc1, yx, acc[6]);               // dg/dm* = c1 y
            acc[7] = fmaf(cc1, yy, acc[7]);
            acc[8] = fmaf(cc1, yz, acc[8]);
            acc[9] = fmaf(cc1, t2 - aa, acc[9]);          // dg/dk
            acc[10] = fmaf(0.5f * cw * rs2, aa + hh - g * g, acc[10]);   // dg/dK
        }
    }
}

template <bool WEIGHTED>
__global__ void __launch_bounds__(kThreads) k_bwd_params(const float4* __restrict__ rec, int64_t slots,
                                                         int64_t direct_slots, const float* __restrict__ qrec,
                                                         int64_t qtiles, int64_t qtiles_per_chunk,
                                                         float* __restrict__ part, int32_t* status) {
    extern __shared__ __align__(128) char smem[];
    __shared__ TileRing<kStages> ring;
    char* buf = smem;
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int chunk = blockIdx.y;
    const int64_t t0 = (int64_t)chunk * qtiles_per_chunk;
    const int64_t t1 = t0 + qtiles_per_chunk < qtiles ? t0 + qtiles_per_chunk : qtiles;
    const int64_t nt = t1 > t0 ? t1 - t0 : 0;
    if (threadIdx.x == 0) ring.init(kConsumerWarps);
    __syncthreads();
    if (warp == kConsumerWarps) {
        if (lane == 0)
            ring.produce(buf, reinterpret_cast<const char*>(qrec) + (size_t)t0 * kQTileBytes, nt, kQTileBytes, status);
        return;
    }
    const int64_t slot = (int64_t)blockIdx.x * kPointsPerCta + threadIdx.x;
    const int64_t sl = slot < slots ? slot : slots - 1;
    const float4 r0 = rec[4 * sl], r1 = rec[4 * sl + 1], r2 = rec[4 * sl + 2], r3 = rec[4 * sl + 3];
    // each warp holds one 32-record tile, all of one form
    const bool kappa = ((int64_t)blockIdx.x * kPointsPerCta + warp * 32) >= direct_slots;
    const Rec2 R = rec2_of(r0, r1, r2, r3);
    // two queries' sums side by side (each half sums every other query)
    f32x2 acc2[kNAcc];
#pragma unroll
    for (int k = 0; k < kNAcc; ++k) acc2[k] = f2_splat(0.f);
    for (int64_t t = 0; t < nt; ++t) {
        if (!ring.wait_full(t, status)) return;
        const ulonglong2* tile = reinterpret_cast<const ulonglong2*>(buf + (size_t)(t % kStages) * kQTileBytes);
        if (kappa)
            bwd_tile2<true, WEIGHTED>(tile, R, acc2);
        else
            bwd_tile2<false, WEIGHTED>(tile, R, acc2);
        ring.release(t, lane);
    }
    float acc[kNAcc];
#pragma unroll
    for (int k = 0; k < kNAcc; ++k) acc[k] = f2_lo(acc2[k]) + f2_hi(acc2[k]);
    if (slot < slots) {
        float* dst = part + ((size_t)chunk * slots + slot) * kNAcc;
#pragma unroll
        for (int k = 0; k < kNAcc; ++k) dst[k] = acc[k];
    }
}

// Per point: sum the chunk partials, then chain through the fit (double
// precision duals) into the six coefficients, written in the original order.
__global__ void k_bwd_chain(const float* __restrict__ part, int nchunks, int64_t slots, int64_t direct_slots,
                            const int32_t* __restrict__ perm, const float4* __restrict__ rec,
                            const float* __restrict__ P, const float* __restrict__ Nrm, const float* __restrict__ A6,
                            float* __restrict__ out) {
    const int64_t slot = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (slot >= slots) return;
    const int32_t i = perm[slot];
    if (i < 0) return;
    double acc[kNAcc];
    for (int k = 0; k < kNAcc; ++k) acc[k] = 0.0;
    for (int c = 0; c < nchunks; ++c) {
        const float* s = part + ((size_t)c * slots + slot) * kNAcc;
        for (int k = 0; k < kNAcc; ++k) acc[k] += (double)s[k];
    }
    double p[3], n[3];
    Dual6 a[6];
    for (int k = 0; k < 3; ++k) {
        p[k] = P[3 * i + k];
        n[k] = Nrm[3 * i + k];
    }
    const double len = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
    for (int k = 0; k < 3; ++k) n[k] /= len;
    for (int k = 0; k < 6; ++k) {
        a[k] = dconst((double)A6[6 * i + k]);
        a[k].d[k] = 1.0;
    }
    FitPoint<Dual6> f;
    fit_point<Dual6>(p, n, a, f);
    double g6[6] = {0, 0, 0, 0, 0, 0};
    auto add = [&](const Dual6& th, double coef) {
        for (int k = 0; k < 6; ++k) g6[k] += coef * th.d[k];
    };
    if (slot < direct_slots) {
        const double sT = -sgn_convex(f.kmax.v);
        const Dual6 r = 1.0 / fabsT(f.kmax);
        const Dual6 R = 1.0 / fabsT(f.kmin) - (sgn_convex(f.kmin.v) * sgn_convex(f.kmax.v)) * r;
        for (int k = 0; k < 3; ++k) {
            add(f.q[k] + f.nstar[k] / f.kmin, acc[k]);   // centre c
            add(f.u[k], acc[3 + k]);
        }
        add(R, acc[6]);
        add(r, -sT * acc[7]);
    } else {
        const double zeta = -sgn_convex(f.kmin.v);
        for (int k = 0; k < 3; ++k) {
            add(f.q[k], acc[k]);
            add(f.u[k], acc[3 + k]);
            add(f.nstar[k] * (2.0 * zeta), acc[6 + k]);
        }
        add(fabsT(f.kmin), acc[9]);
        add(-f.kmax, acc[10]);
    }
    for (int k = 0; k < 6; ++k) out[6 * (int64_t)i + k] = (float)g6[k];
    (void)rec;
}

}  // namespace

sdf_status launch_backward_params(const Cloud& c, int64_t q, const float* d_saved, const float* d_grad_phi,
                                  float* d_grad_params, const sdf_query_opts& o, cudaStream_t st) {
    (void)o;
    const int64_t slots = (c.tiles_direct + c.tiles_kappa) * kTileRecs;
    const int64_t direct_slots = c.tiles_direct * kTileRecs;
    const int64_t qtiles = (q + kQTile - 1) / kQTile;
    const int64_t pblocks = (slots + kPointsPerCta - 1) / kPointsPerCta;
    // split the queries until there are about two waves of 3 CTAs per SM
    int64_t nchunks = 1;
    const int64_t target = 2LL * 3 * c.num_sms;
    if (pblocks < target) nchunks = (target + pblocks - 1) / pblocks;
    const int64_t max_chunks = qtiles / 4 > 0 ? qtiles / 4 : 1;
    if (nchunks > max_chunks) nchunks = max_chunks;
    if (nchunks > 64) nchunks = 64;
    const int64_t per = (qtiles + nchunks - 1) / nchunks;
    nchunks = (qtiles + per - 1) / per;

    float* qrec = nullptr;
    float* part = nullptr;
    cudaError_t e = cudaMallocAsync(&qrec, (size_t)qtiles * kQTileBytes, st);
    if (e == cudaSuccess) e = cudaMallocAsync(&part, (size_t)nchunks * slots * kNAcc * sizeof(float), st);
    if (e != cudaSuccess) {
        if (qrec) cudaFreeAsync(qrec, st);
        return e == cudaErrorMemoryAllocation ? set_error(SDF_ENOMEM, "sdf_backward_params: scratch")
                                              : cuda_error(e, "sdf_backward_params: scratch");
    }
    {
        ProfRange pr(SDF_K_BWD, st);
        const int64_t qp = qtiles * kQTile;
        k_bwd_prep<<<(unsigned)((qp + 255) / 256), 256, 0, st>>>(d_saved, d_grad_phi, q, qp, qrec);
        e = cudaGetLastError();
        if (e == cudaSuccess) {
            (c.weighted ? k_bwd_params<true> : k_bwd_params<false>)<<<dim3((unsigned)pblocks, (unsigned)nchunks),
                                                                     kThreads, kStages * kQTileBytes, st>>>(
                c.rec, slots, direct_slots, qrec, qtiles, per, part, c.status);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) {
            k_bwd_chain<<<(unsigned)((slots + 127) / 128), 128, 0, st>>>(part, (int)nchunks, slots, direct_slots,
                                                                         c.perm, c.rec, c.src_points,
                                                                         c.src_normals, c.src_params, d_grad_params);
            e = cudaGetLastError();
        }
    }
    cudaFreeAsync(qrec, st);
    cudaFreeAsync(part, st);
    return e == cudaSuccess ? SDF_OK : cuda_error(e, "sdf_backward_params: launch");
}

}  // namespace ptsdf
