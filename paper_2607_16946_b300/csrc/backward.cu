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
#include "fit_math.cuh"
#include "internal.h"

namespace ptsdf {

namespace {

constexpr int kThreads = (kConsumerWarps + 1) * 32;
constexpr int kPointsPerCta = kConsumerWarps * 32;     // one record per consumer thread
constexpr int kQTile = 64;                             // queries per streamed tile
constexpr uint32_t kQTileBytes = kQTile * 8 * sizeof(float);
constexpr int kNAcc = 11;
constexpr float kTiny = 1e-30f;

// qrec[j] = {x, y, z, L, A0, G / W, 0, 0}; padding rows have coefficient 0.
__global__ void k_bwd_prep(const float* __restrict__ saved, const float* __restrict__ G, int64_t q,
                           int64_t q_padded, float4* __restrict__ qrec) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= q_padded) return;
    if (j < q) {
        const float* s = saved + 8 * j;
        qrec[2 * j] = make_float4(s[0], s[1], s[2], s[3]);
        qrec[2 * j + 1] = make_float4(s[4], G[j] / s[5], 0.f, 0.f);
    } else {
        qrec[2 * j] = make_float4(0.f, 0.f, 0.f, 0.f);
        qrec[2 * j + 1] = make_float4(0.f, 0.f, 0.f, 0.f);
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
                                                         int64_t direct_slots, const float4* __restrict__ qrec,
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
            ring.produce(buf, reinterpret_cast<const char*>(qrec + t0 * kQTile * 2), nt, kQTileBytes, status);
        return;
    }
    const int64_t slot = (int64_t)blockIdx.x * kPointsPerCta + threadIdx.x;
    const int64_t sl = slot < slots ? slot : slots - 1;
    const float4 r0 = rec[4 * sl], r1 = rec[4 * sl + 1], r2 = rec[4 * sl + 2], r3 = rec[4 * sl + 3];
    // each warp holds one 32-record tile, all of one form
    const bool kappa = ((int64_t)blockIdx.x * kPointsPerCta + warp * 32) >= direct_slots;
    float acc[kNAcc], tacc[kNAcc];
#pragma unroll
    for (int k = 0; k < kNAcc; ++k) acc[k] = 0.f;
    for (int64_t t = 0; t < nt; ++t) {
        if (!ring.wait_full(t, status)) return;
        const float4* tile = reinterpret_cast<const float4*>(buf + (size_t)(t % kStages) * kQTileBytes);
#pragma unroll
        for (int k = 0; k < kNAcc; ++k) tacc[k] = 0.f;
        if (kappa)
            bwd_tile<true, WEIGHTED>(tile, r0, r1, r2, r3, tacc);
        else
            bwd_tile<false, WEIGHTED>(tile, r0, r1, r2, r3, tacc);
#pragma unroll
        for (int k = 0; k < kNAcc; ++k) acc[k] += tacc[k];
        ring.release(t, lane);
    }
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

    float4* qrec = nullptr;
    float* part = nullptr;
    cudaError_t e = cudaMallocAsync(&qrec, (size_t)qtiles * kQTile * 2 * sizeof(float4), st);
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
