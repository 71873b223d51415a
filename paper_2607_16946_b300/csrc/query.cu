// Query kernels: phi(x) for every query against every point (Sec. 4.2,
// Eqs. BasicFormulaShifted and RelationshipBetweenLambdaAndRadius; torus SDF
// of Eq. SingleTorusSDF).
//
//   k_prepass  per query, over a chunk of points: max_i and min_i of
//              |x - p_i|^2 (d_max gives lambda_x, d_min the exponent shift).
//   k_fwd      per query, over a chunk of tiles: W = sum_i w_i,
//              S = sum_i w_i g_i.  Writes phi = S / W - offset when the
//              points are not split, else the (W, S) partials.
//   k_merge    sums the partials of every chunk in chunk order.
//
// Geometry of both pair kernels: a CTA holds kQueriesPerCta = 512 queries in
// registers (8 consumer warps x 32 lanes x 2 queries) and streams the point
// data through a 4-stage shared-memory ring filled by bulk (TMA) copies from
// a 9th, producer warp.  All lanes of a warp read the same record (a
// shared-memory broadcast), so per point every lane does 2 independent pair
// evaluations.
//
// Exponent shift: the ratio S / W does not depend on the shift.  The paper
// shifts by sigma_x = d_max / 2, which bounds the smallest weight by e^-C but
// lets near points weigh up to e^C: for C near 87 a few such terms overflow an
// FP32 sum.  The kernels shift by d_min instead, w_i = exp2(-L (d_i - d_min)),
// L = lambda_x log2 e, so every weight is at most 1 (the nearest point's is 1),
// W >= 1 and nothing overflows for any C; weights far below the nearest one
// underflow to 0 without changing phi at FP32 precision.  All chunks of a
// split query share the same d_min, so their partial sums add directly.
//
// The prepass works in coordinates centred on the cloud's bounding box, so
// |x - p|^2 = |x'|^2 + |p'|^2 - 2 <x', p'> keeps its relative accuracy for
// clouds away from the origin.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>
#include <string>

#include "query_common.cuh"
#include "f32x2_ops.cuh"
#include "prepass_warp.cuh"

#ifndef PTSDF_FWD_PAIRS
#define PTSDF_FWD_PAIRS 1   // k_fwd: two points per .f32x2 step over the pair-interleaved records (0: scalar)
#endif
#ifndef PTSDF_FWD_PAIR_BLOCKS
#define PTSDF_FWD_PAIR_BLOCKS 3   // resident CTAs per SM the packed k_fwd is compiled for
#endif

namespace ptsdf {

using namespace qk;

namespace {

struct QState {
    float x, y, z;     // query
    float L, A0;       // exponent = A0 - L d
    float W, S;        // totals
    float w, s;        // tile partials
};

// Weights of two queries at once.  SDF_F32: two FP32 exp2 (one MUFU each).
// SDF_F16X2 / SDF_BF16X2: the two exponents are packed into one 32-bit
// register of half / bfloat16 values and evaluated by one packed exp2 (the
// only packed-half MUFU operation of sm_103a besides tanh), then widened back
// to FP32 for the FP32 accumulation.
template <int PREC>
__device__ __forceinline__ void weights2(float a0, float a1, float& w0, float& w1) {
    if (PREC == SDF_F16X2) {
        asm("{\n\t.reg .b32 t;\n\t.reg .f16 lo, hi;\n\t"
            "cvt.rn.f16x2.f32 t, %2, %3;\n\t"
            "ex2.approx.f16x2 t, t;\n\t"
            "mov.b32 {lo, hi}, t;\n\t"
            "cvt.f32.f16 %0, hi;\n\t"
            "cvt.f32.f16 %1, lo;\n\t}"
            : "=f"(w0), "=f"(w1)
            : "f"(a0), "f"(a1));
    } else if (PREC == SDF_BF16X2) {
        uint32_t t;
        asm("{\n\t.reg .b32 u;\n\t"
            "cvt.rn.bf16x2.f32 u, %1, %2;\n\t"
            "ex2.approx.ftz.bf16x2 %0, u;\n\t}"
            : "=r"(t)
            : "f"(a0), "f"(a1));
        w0 = __uint_as_float(t & 0xffff0000u);    // high half: a0
        w1 = __uint_as_float(t << 16);            // low half: a1
    } else {
        w0 = ex2_mufu(a0);
        w1 = ex2_mufu(a1);
    }
}

// WEIGHTED: every weight is multiplied by the point's weight A_i (record r3.w),
// after the exponential, so that the packed-half exponentials keep their
// arguments near 0 for the points that matter.
template <bool KAPPA, int PREC, bool WEIGHTED, bool FLAT = false>
__device__ __forceinline__ void pair_tile(const float4* __restrict__ tile, int cnt, QState (&qs)[kQueriesPerThread]) {
    static_assert(kQueriesPerThread % 2 == 0, "queries are paired for the packed weights");
#pragma unroll kUnrollPts
    for (int j = 0; j < cnt; ++j) {
        const float4 r0 = tile[4 * j], r1 = tile[4 * j + 1], r2 = tile[4 * j + 2];
        float4 r3 = make_float4(0.f, 0.f, 0.f, 0.f);
        if (KAPPA || WEIGHTED) r3 = tile[4 * j + 3];
#pragma unroll
        for (int k = 0; k < kQueriesPerThread; k += 2) {
            float arg[2], g[2];
#pragma unroll
            for (int m = 0; m < 2; ++m) {
                const QState& s = qs[k + m];
                const float dx = s.x - r0.x, dy = s.y - r0.y, dz = s.z - r0.z;
                const float d = sqrt_mufu(fmaf(dx, dx, fmaf(dy, dy, dz * dz)));
                g[m] = !KAPPA ? g_direct(s.x, s.y, s.z, r1, r2, r0.w)
                              : FLAT ? g_kappa_flat(s.x, s.y, s.z, r0, r1, r2, r3) : g_kappa(s.x, s.y, s.z, r0, r1, r2, r3);
                arg[m] = fmaf(-s.L, d, s.A0);
            }
            float w0, w1;
            weights2<PREC>(arg[0], arg[1], w0, w1);
            if (WEIGHTED) {
                w0 *= r3.w;
                w1 *= r3.w;
            }
            qs[k].w += w0;
            qs[k].s = fmaf(w0, g[0], qs[k].s);
            qs[k + 1].w += w1;
            qs[k + 1].s = fmaf(w1, g[1], qs[k + 1].s);
        }
    }
}

// The same tile two points at a time, over the pair-interleaved records
// (Cloud::rec2: for points 2k, 2k+1 each record float4 r_m is stored as
// (r_m.x, r_m.x', r_m.y, r_m.y') (r_m.z, r_m.z', r_m.w, r_m.w')): every 128-bit
// shared load gives two .f32x2 operands, and every FP32 step of a pair runs
// for both points in one instruction against the lane's query broadcast into
// both halves (the special-function steps stay one per point).  The pair
// arithmetic is that of pair_tile, operation for operation; a pair's second
// point past the tile's `cnt` (a zero record) gets weight 0.
struct QPair {
    f32x2 X, Y, Z, NL, A0;   // the query and its exponent, in both halves
    f32x2 w, s;              // tile partials of the two points' halves
};

template <bool KAPPA, int PREC, bool WEIGHTED, bool FLAT = false>
__device__ __forceinline__ void pair_tile2(const ulonglong2* __restrict__ tile, int cnt,
                                           QPair (&qp)[kQueriesPerThread]) {
    const f32x2 ONE = f2_splat(1.f);
#pragma unroll 1
    for (int j = 0; j < cnt; j += 2) {
        const ulonglong2* r = tile + 4 * j;   // 8 x 16 B per pair of points
        const ulonglong2 a0 = r[0], b0 = r[1], a1 = r[2], b1 = r[3], a2 = r[4], b2 = r[5];
        ulonglong2 a3 = make_ulonglong2(0ull, 0ull), b3 = a3;
        if (KAPPA || WEIGHTED) {
            a3 = r[6];
            b3 = r[7];
        }
        const bool second = j + 1 < cnt;
#pragma unroll
        for (int k = 0; k < kQueriesPerThread; ++k) {
            QPair& q = qp[k];
            const f32x2 DX = f2_sub(q.X, a0.x), DY = f2_sub(q.Y, a0.y), DZ = f2_sub(q.Z, b0.x);
            const f32x2 D = f2_sqrt(f2_fma(DX, DX, f2_fma(DY, DY, f2_mul(DZ, DZ))));
            f32x2 G;
            if (!KAPPA) {
                // g_direct: v = x - c, h = <v, u>, w = v - h u, rho = |w|, D = |(rho - R, h)|
                const f32x2 VX = f2_sub(q.X, a1.x), VY = f2_sub(q.Y, a1.y), VZ = f2_sub(q.Z, b1.x);
                const f32x2 H = f2_fma(VX, a2.x, f2_fma(VY, a2.y, f2_mul(VZ, b2.x)));
                const f32x2 NH = f2_sub(f2_splat(0.f), H);
                const f32x2 WX = f2_fma(NH, a2.x, VX), WY = f2_fma(NH, a2.y, VY), WZ = f2_fma(NH, b2.x, VZ);
                const f32x2 RHO = f2_sqrt(f2_fma(WX, WX, f2_fma(WY, WY, f2_mul(WZ, WZ))));
                const f32x2 E = f2_sub(RHO, b1.y);
                G = f2_fma(b0.y, f2_sqrt(f2_fma(E, E, f2_mul(H, H))), b2.y);
            } else {
                // g_kappa / g_kappa_flat
                const f32x2 YX = f2_sub(q.X, a1.x), YY = f2_sub(q.Y, a1.y), YZ = f2_sub(q.Z, b1.x);
                const f32x2 H = f2_fma(YX, a2.x, f2_fma(YY, a2.y, f2_mul(YZ, b2.x)));
                const f32x2 HH = f2_mul(H, H);
                const f32x2 YN = f2_fma(YX, a3.x, f2_fma(YY, a3.y, f2_mul(YZ, b3.x)));
                f32x2 AP;
                if (FLAT) {
                    AP = f2_mul(f2_splat(0.5f), YN);
                } else {
                    const f32x2 T2 = f2_sub(f2_fma(YX, YX, f2_fma(YY, YY, f2_mul(YZ, YZ))), HH);
                    const f32x2 M = f2_fma(b1.y, T2, YN);
                    const f32x2 S1 = f2_sqrt(f2_max0(f2_fma(b1.y, M, ONE)));
                    AP = f2_mul(M, f2_rcp(f2_add(ONE, S1)));
                }
                const f32x2 NP = f2_fma(b2.y, f2_fma(AP, AP, HH), f2_mul(b0.y, AP));
                const f32x2 S2 = f2_sqrt(f2_max0(f2_fma(b2.y, NP, ONE)));
                G = f2_mul(NP, f2_rcp(f2_add(ONE, S2)));
            }
            const f32x2 ARG = f2_fma(q.NL, D, q.A0);
            float w0, w1;
            weights2<PREC>(f2_lo(ARG), f2_hi(ARG), w0, w1);
            if (!second) w1 = 0.f;                                      // no second point
            f32x2 W = f2_pack(w0, w1);
            if (WEIGHTED) W = f2_mul(W, b3.y);                          // (A, A') = r3.w of both
            q.w = f2_add(q.w, W);
            q.s = f2_fma(W, G, q.s);
        }
    }
}

// --------------------------------------------------------------------------
// Forward pass
// --------------------------------------------------------------------------
template <int PREC, bool WEIGHTED>
__global__ void __launch_bounds__(kThreads, PTSDF_FWD_PAIRS ? PTSDF_FWD_PAIR_BLOCKS : kFwdMinBlocks) k_fwd(const float4* __restrict__ rec, int64_t n_direct, int64_t n_kappa,
                                                  int64_t tiles_direct, int64_t tiles_total, int64_t tiles_per_chunk,
                                                  QueryArgs a, int32_t* status, int64_t n_kappa_flat) {
    extern __shared__ __align__(128) char smem[];
    __shared__ TileRing<kStages> ring;
    char* buf = smem;
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int chunk = blockIdx.y;
    const int64_t t0 = a.tile_base + (int64_t)chunk * tiles_per_chunk;
    const int64_t t1 = t0 + tiles_per_chunk < tiles_total ? t0 + tiles_per_chunk : tiles_total;
    const int64_t nt = t1 > t0 ? t1 - t0 : 0;
    if (threadIdx.x == 0) ring.init(kConsumerWarps);
    __syncthreads();
    if (warp == kConsumerWarps) {
        if (lane == 0)
            ring.produce(buf, reinterpret_cast<const char*>(rec + t0 * kTileRecs * 4), nt, kTileBytes, status);
        return;
    }
#if PTSDF_FWD_PAIRS
    QPair qp[kQueriesPerThread];
    float Wt[kQueriesPerThread], St[kQueriesPerThread];
#endif
    QState qs[kQueriesPerThread];
    int64_t qi[kQueriesPerThread];
#pragma unroll
    for (int k = 0; k < kQueriesPerThread; ++k) {
        qi[k] = (int64_t)blockIdx.x * kQueriesPerCta + k * (kConsumerWarps * 32) + threadIdx.x;
        const int64_t qq = qi[k] < a.q ? qi[k] : a.q - 1;
        qs[k].x = a.x[3 * qq];
        qs[k].y = a.x[3 * qq + 1];
        qs[k].z = a.x[3 * qq + 2];
        // exponent A0 - L d = -lambda_x (d - d_min) log2(e)
        query_screening(a.d2, a.pre_split, a.q, qq, a.mode, a.C, a.lam, qs[k].L, qs[k].A0);
        qs[k].W = qs[k].S = 0.f;
#if PTSDF_FWD_PAIRS
        qp[k].X = f2_splat(qs[k].x);
        qp[k].Y = f2_splat(qs[k].y);
        qp[k].Z = f2_splat(qs[k].z);
        qp[k].NL = f2_splat(-qs[k].L);
        qp[k].A0 = f2_splat(qs[k].A0);
        Wt[k] = St[k] = 0.f;
#endif
    }
    for (int64_t t = 0; t < nt; ++t) {
        if (!ring.wait_full(t, status)) return;
        const float4* tile = reinterpret_cast<const float4*>(buf + (size_t)(t % kStages) * kTileBytes);
        const int64_t gt = t0 + t;
        const bool kappa = gt >= tiles_direct;
        const int64_t first = (kappa ? gt - tiles_direct : gt) * kTileRecs;
        const int64_t seg = kappa ? n_kappa : n_direct;
        const int cnt = (int)(seg - first < kTileRecs ? seg - first : kTileRecs);
#if PTSDF_FWD_PAIRS
        const ulonglong2* tile2 = reinterpret_cast<const ulonglong2*>(tile);
#pragma unroll
        for (int k = 0; k < kQueriesPerThread; ++k) qp[k].w = qp[k].s = f2_splat(0.f);
        if (kappa && first + kTileRecs <= n_kappa_flat)   // every record of the tile has kappa_min = 0
            pair_tile2<true, PREC, WEIGHTED, true>(tile2, cnt, qp);
        else if (kappa)
            pair_tile2<true, PREC, WEIGHTED>(tile2, cnt, qp);
        else
            pair_tile2<false, PREC, WEIGHTED>(tile2, cnt, qp);
        // blocked summation, the two halves of a tile's partials first
#pragma unroll
        for (int k = 0; k < kQueriesPerThread; ++k) {
            Wt[k] += f2_lo(qp[k].w) + f2_hi(qp[k].w);
            St[k] += f2_lo(qp[k].s) + f2_hi(qp[k].s);
        }
#else
#pragma unroll
        for (int k = 0; k < kQueriesPerThread; ++k) qs[k].w = qs[k].s = 0.f;
        if (kappa && first + kTileRecs <= n_kappa_flat)   // every record of the tile has kappa_min = 0
            pair_tile<true, PREC, WEIGHTED, true>(tile, cnt, qs);
        else if (kappa)
            pair_tile<true, PREC, WEIGHTED>(tile, cnt, qs);
        else
            pair_tile<false, PREC, WEIGHTED>(tile, cnt, qs);
        // blocked summation: tile partials are added to the totals once per
        // tile, which keeps the FP32 rounding of long sums small
#pragma unroll
        for (int k = 0; k < kQueriesPerThread; ++k) {
            qs[k].W += qs[k].w;
            qs[k].S += qs[k].s;
        }
#endif
        ring.release(t, lane);
    }
#if PTSDF_FWD_PAIRS
#pragma unroll
    for (int k = 0; k < kQueriesPerThread; ++k) {
        qs[k].W = Wt[k];
        qs[k].S = St[k];
    }
#endif
#pragma unroll
    for (int k = 0; k < kQueriesPerThread; ++k) {
        if (qi[k] >= a.q) continue;
        if (a.split == 1)
            a.phi[qi[k]] = finish_sums(qs[k].W, qs[k].S, a.formula, qs[k].L, qs[k].A0, a.offset);
        else
            a.part[(size_t)(a.part_base + chunk) * a.q + qi[k]] = make_float2(qs[k].W, qs[k].S);
    }
}

using FwdKernel = decltype(&k_fwd<SDF_F32, false>);

// the records k_fwd reads: pair-interleaved for the packed pair loop
const float4* fwd_records(const Cloud& c) { return PTSDF_FWD_PAIRS ? c.rec2 : c.rec; }

FwdKernel fwd_kernel(int precision, bool weighted) {
    if (weighted)
        return precision == SDF_F16X2 ? k_fwd<SDF_F16X2, true> : precision == SDF_BF16X2 ? k_fwd<SDF_BF16X2, true>
                                                                                         : k_fwd<SDF_F32, true>;
    return precision == SDF_F16X2 ? k_fwd<SDF_F16X2, false> : precision == SDF_BF16X2 ? k_fwd<SDF_BF16X2, false>
                                                                                       : k_fwd<SDF_F32, false>;
}

}  // namespace

// Point chunks of `tiles` tiles for `qblocks` query blocks: enough CTAs to
// reach `target`, at least 4 tiles per chunk, at most 64 chunks (or exactly
// `split_override` chunks when it is positive, capped at one tile each).
void chunk_tiles(int64_t qblocks, int64_t tiles, int64_t target, int split_override, int64_t& tiles_per_chunk,
                 int& nchunks) {
    int64_t split = 1;
    if (split_override > 0) {
        split = split_override;
    } else {
        if (qblocks < target) split = (target + qblocks - 1) / qblocks;
        const int64_t max_split = tiles / 4 > 0 ? tiles / 4 : 1;
        if (split > max_split) split = max_split;
        if (split > 64) split = 64;
    }
    if (split > tiles) split = tiles;
    if (split < 1) split = 1;
    tiles_per_chunk = (tiles + split - 1) / split;
    nchunks = (int)((tiles + tiles_per_chunk - 1) / tiles_per_chunk);
}

Plan make_plan(const Cloud& c, int64_t q, int split_override, int queries_per_cta) {
    Plan p;
    p.q = q;
    p.qblocks = (q + queries_per_cta - 1) / queries_per_cta;
    p.pre_qblocks = (q + kQueriesPerCta - 1) / kQueriesPerCta;
    // aim for at least two waves of the resident CTAs per SM
    chunk_tiles(p.qblocks, c.tiles_direct + c.tiles_kappa, 2LL * kFwdMinBlocks * c.num_sms, split_override,
                p.tiles_per_chunk, p.split);
    p.pre_tiles_per_chunk = (c.pre_tiles + p.split - 1) / p.split;
    return p;
}

bool use_tensor_engine(const Cloud& c, const sdf_query_opts& o) {
    return o.engine != SDF_ENGINE_ALU && o.precision == SDF_F32 && c.btiles != nullptr && tc_tiles_end(c) > 0;
}

namespace {

// Launch plan of the tensor-core engine: the direct tiles on the direct
// instance of k_fwd_tc in nd chunks, the whole kappa_min = 0 tiles
// [tiles_direct, flat_end) on the flat instance in nf chunks, the other
// curvature-form tiles [flat_end, tc_end) on the general one in nk chunks,
// any others on k_fwd in na chunks; with more than one chunk in all, each
// writes (W, S) partial rows in that order and k_merge sums them in row order.
struct TcPlan {
    int64_t tc_end = 0, flat_end = 0, tpc_d = 0, tpc_f = 0, tpc_k = 0, tpc_a = 0;
    int nd = 0, nf = 0, nk = 0, na = 0;
    int parts() const { return nd + nf + nk + na; }
};

TcPlan tc_plan(const Cloud& c, int64_t q, int split_n, int64_t alu_qblocks) {
    TcPlan t;
    t.tc_end = tc_tiles_end(c);
    t.flat_end = tc_flat_end(c);
    const int64_t qb = tc_query_blocks(q), target = 2LL * c.num_sms;   // one CTA per SM, two waves
    if (c.tiles_direct > 0) chunk_tiles(qb, c.tiles_direct, target, split_n, t.tpc_d, t.nd);
    if (t.flat_end > c.tiles_direct) chunk_tiles(qb, t.flat_end - c.tiles_direct, target, split_n, t.tpc_f, t.nf);
    if (t.tc_end > t.flat_end) chunk_tiles(qb, t.tc_end - t.flat_end, target, split_n, t.tpc_k, t.nk);
    const int64_t tiles = c.tiles_direct + c.tiles_kappa;
    if (tiles > t.tc_end)
        chunk_tiles(alu_qblocks, tiles - t.tc_end, 2LL * kFwdMinBlocks * c.num_sms, split_n, t.tpc_a, t.na);
    return t;
}

}  // namespace

int query_partials(const Cloud& c, int64_t q, const sdf_query_opts& o) {
    const Plan p = make_plan(c, q, o.split_n);
    if (!use_tensor_engine(c, o)) return p.split;
    return tc_plan(c, q, o.split_n, p.qblocks).parts();
}

sdf_status launch_query(const Cloud& c, const float* d_x, int64_t q, float* d_phi, const sdf_query_opts& o,
                        cudaStream_t st) {
    if (o.lambda_mode == SDF_LAMBDA_RADIUS) return launch_radius_query(c, d_x, q, d_phi, o, st);
    if (o.formula == SDF_FORMULA_SSPD || o.formula == SDF_FORMULA_SHC) return launch_plane_query(c, d_x, q, d_phi, o, st);
    const Plan p = make_plan(c, q, o.split_n);
    // Tensor-core engine: see TcPlan
    const bool tc = use_tensor_engine(c, o);
    const TcPlan tp = tc ? tc_plan(c, q, o.split_n, p.qblocks) : TcPlan();
    const int nparts = tc ? tp.parts() : p.split;
    QueryArgs a;
    a.x = d_x;
    a.q = q;
    a.phi = d_phi;
    a.split = nparts;
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
    // the pruned prepass keeps one query block per CTA with no point split, so
    // it is used once there are enough query blocks to fill the GPU
    const bool warp_pre = use_warp_prepass(c, p, o), pruned = !warp_pre && use_pruned_prepass(c, p, o);
    a.pre_split = pruned || warp_pre ? 1 : p.split;
    cudaError_t e = cudaMallocAsync(&a.d2, (size_t)a.pre_split * q * sizeof(float2), st);
    if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? set_error(SDF_ENOMEM, "sdf_query: scratch")
                                                                : cuda_error(e, "sdf_query: scratch");
    if (nparts > 1) {
        e = cudaMallocAsync(&a.part, (size_t)nparts * q * sizeof(float2), st);
        if (e != cudaSuccess) {
            cudaFreeAsync(a.d2, st);
            return e == cudaErrorMemoryAllocation ? set_error(SDF_ENOMEM, "sdf_query: scratch")
                                                  : cuda_error(e, "sdf_query: scratch");
        }
    }
    const dim3 grid((unsigned)p.qblocks, (unsigned)p.split);
    const dim3 pre_grid((unsigned)p.pre_qblocks, (unsigned)p.split);
    {
        ProfRange pr(SDF_K_PREPASS, st);
        if (pruned)
            k_prepass_pruned<false><<<(unsigned)p.pre_qblocks, kPrunedThreads, 0, st>>>(c.pre, c.spheres, c.n,
                                                                                     c.n_spheres, a);
        else if (warp_pre)
            launch_prepass_warp(c, a, false, st);
        else if (o.lambda_mode == SDF_LAMBDA_GLOBAL)
            k_prepass<SDF_LAMBDA_GLOBAL><<<pre_grid, kThreads, kStages * kPreBytes, st>>>(
                c.pre, c.n, c.pre_tiles, p.pre_tiles_per_chunk, a, c.status);
        else
            k_prepass<SDF_LAMBDA_FIXED><<<pre_grid, kThreads, kStages * kPreBytes, st>>>(
                c.pre, c.n, c.pre_tiles, p.pre_tiles_per_chunk, a, c.status);
        e = cudaGetLastError();
    }
    sdf_status s = SDF_OK;
    if (e == cudaSuccess && !tc) {
        ProfRange pr(SDF_K_FWD, st);
        const FwdKernel kern = fwd_kernel(o.precision, c.weighted);
        kern<<<grid, kThreads, kStages * kTileBytes, st>>>(fwd_records(c), c.n_direct, c.n_kappa, c.tiles_direct,
                                                          c.tiles_direct + c.tiles_kappa, p.tiles_per_chunk, a,
                                                          c.status, c.n_kappa_flat);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && tc) {
        {
            TcQuery tq;
            tq.x = a.x;
            tq.q = q;
            tq.phi = a.phi;
            tq.part = a.part;
            tq.d2 = a.d2;
            tq.cx = a.cx;
            tq.cy = a.cy;
            tq.cz = a.cz;
            tq.pre_split = a.pre_split;
            tq.mode = a.mode;
            tq.C = a.C;
            tq.lam = a.lam;
            tq.offset = a.offset;
            tq.formula = a.formula;
            tq.part_base = 0;
            if (tp.nd > 0) {   // one profiled range per launch
                ProfRange pr(SDF_K_FWD_TC, st);
                s = launch_fwd_tc(c, tq, 0, c.tiles_direct, tp.tpc_d, tp.nd, nparts == 1, st);
            }
            tq.part_base = tp.nd;
            if (s == SDF_OK && tp.nf > 0) {
                ProfRange pr(SDF_K_FWD_TC, st);
                s = launch_fwd_tc(c, tq, c.tiles_direct, tp.flat_end, tp.tpc_f, tp.nf, nparts == 1, st);
            }
            tq.part_base = tp.nd + tp.nf;
            if (s == SDF_OK && tp.nk > 0) {
                ProfRange pr(SDF_K_FWD_TC, st);
                s = launch_fwd_tc(c, tq, tp.flat_end, tp.tc_end, tp.tpc_k, tp.nk, nparts == 1, st);
            }
        }
        if (s == SDF_OK && tp.na > 0) {
            ProfRange pr(SDF_K_FWD, st);
            QueryArgs ak = a;
            ak.tile_base = tp.tc_end;
            ak.part_base = tp.nd + tp.nf + tp.nk;
            fwd_kernel(SDF_F32, c.weighted)<<<dim3((unsigned)p.qblocks, (unsigned)tp.na), kThreads,
                                               kStages * kTileBytes, st>>>(
                fwd_records(c), c.n_direct, c.n_kappa, c.tiles_direct, c.tiles_direct + c.tiles_kappa, tp.tpc_a, ak,
                c.status, c.n_kappa_flat);
            e = cudaGetLastError();
        }
    }
    if (e == cudaSuccess && s == SDF_OK && nparts > 1) {
        ProfRange pr(SDF_K_MERGE, st);
        k_merge<<<(unsigned)((q + 255) / 256), 256, 0, st>>>(a);
        e = cudaGetLastError();
    }
    cudaFreeAsync(a.d2, st);
    if (a.part) cudaFreeAsync(a.part, st);
    if (s != SDF_OK) return s;
    return e == cudaSuccess ? SDF_OK : cuda_error(e, "sdf_query: launch");
}

}  // namespace ptsdf

// ---------------------------------------------------------------------------
// sdf_query_noalloc: sdf_query for callers that must not allocate device
// memory while they run.  Its scratch (the prepass partials and, for split
// point chunks, the (W, S) partials) lives in one fixed file-scope device
// array instead of the stream-ordered allocator.
// ---------------------------------------------------------------------------
namespace ptsdf {

namespace {

constexpr size_t kNoAllocScratchBytes = 8u << 20;   // 8 MiB per device, held until the process exits

// The scratch array.  Host code must not use this symbol as a pointer (it is a
// host-side stand-in); the device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device, looked up once
// per device (the first call on a device does this lookup).
sdf_status noalloc_scratch(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_error(e, "sdf_query_noalloc: cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) return set_error(SDF_EINVAL, "sdf_query_noalloc: device id out of range");
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_error(e, "sdf_query_noalloc: cudaGetSymbolAddress");
        g_noalloc_ptr[dev] = p;
    }
    *out = g_noalloc_ptr[dev];
    return SDF_OK;
}

size_t round256(size_t b) { return (b + 255) & ~(size_t)255; }

}  // namespace

}  // namespace ptsdf

extern "C" sdf_status sdf_query_noalloc(sdf_cloud cloud, const float* d_x, int64_t q, float* d_phi,
                                        const sdf_query_opts* opts, void* stream) {
    using namespace ptsdf;
    if (q < 0) return set_error(SDF_EINVAL, "sdf_query_noalloc: q < 0");
    sdf_query_opts o;
    sdf_opts_default(&o);
    if (opts) o = *opts;
    // the options sdf_query accepts, checked the same way, then what this
    // entry point leaves out
    sdf_status s = check_opts(o, "sdf_query_noalloc");
    if (s != SDF_OK) return s;
    if (o.lambda_mode == SDF_LAMBDA_RADIUS)
        return set_error(SDF_EINVAL, "sdf_query_noalloc: GLOBAL or FIXED lambda only");
    if (o.precision != SDF_F32) return set_error(SDF_EINVAL, "sdf_query_noalloc: FP32 only");
    if (o.engine == SDF_ENGINE_TENSOR)
        return set_error(SDF_EINVAL, "sdf_query_noalloc: only the FP32-unit engine is available here");
    if (o.formula == SDF_FORMULA_SSPD || o.formula == SDF_FORMULA_SHC)
        return set_error(SDF_EINVAL, "sdf_query_noalloc: the blend and the log-sum-exp distance only");
    if (!cloud) return set_error(SDF_EINVAL, "sdf_query_noalloc: cloud is NULL");
    if (q == 0) return SDF_OK;
    if (!d_x || !d_phi) return set_error(SDF_EINVAL, "sdf_query_noalloc: NULL buffer");
    // one float2 per query for the prepass is the least this path needs
    if ((size_t)q * sizeof(float2) > kNoAllocScratchBytes)
        return set_error(SDF_EINVAL, "sdf_query_noalloc: q = " + std::to_string(q) + " exceeds the maximum of " +
                                         std::to_string(kNoAllocScratchBytes / sizeof(float2)) +
                                         " queries per call (8 MiB of fixed scratch); split the batch");
    const Cloud& c = *reinterpret_cast<const Cloud*>(cloud);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    void* scratch = nullptr;
    s = noalloc_scratch(&scratch);
    if (s != SDF_OK) return s;
    Plan p = make_plan(c, q, o.split_n);
    // the split partials must fit too: d2 (split x q float2) + (W, S) (split x q float2)
    const int64_t tiles = c.tiles_direct + c.tiles_kappa;
    int64_t split = p.split;
    while (split > 1 && round256((size_t)split * q * sizeof(float2)) + (size_t)split * q * sizeof(float2) >
                            kNoAllocScratchBytes)
        --split;
    if (split != p.split) {
        p.tiles_per_chunk = (tiles + split - 1) / split;
        split = (tiles + p.tiles_per_chunk - 1) / p.tiles_per_chunk;
        p.split = (int)split;
        p.pre_tiles_per_chunk = (c.pre_tiles + split - 1) / split;
    }
    QueryArgs a;
    a.x = d_x;
    a.q = q;
    a.phi = d_phi;
    a.split = p.split;
    a.mode = o.lambda_mode;
    a.C = o.C;
    a.lam = o.fixed_lambda;
    a.offset = o.offset;
    a.formula = o.formula;
    a.far = nullptr;
    a.pre_split = p.split;
    a.cx = 0.5f * (c.aabb[0] + c.aabb[3]);
    a.cy = 0.5f * (c.aabb[1] + c.aabb[4]);
    a.cz = 0.5f * (c.aabb[2] + c.aabb[5]);
    a.cloud_radius = 0.5f * c.aabb_diag * (1.f + 1e-6f);
    // every scratch entry is written before it is read, so nothing is cleared
    char* base = static_cast<char*>(scratch);
    a.d2 = reinterpret_cast<float2*>(base);
    a.part = p.split > 1 ? reinterpret_cast<float2*>(base + round256((size_t)p.split * q * sizeof(float2))) : nullptr;
    const dim3 grid((unsigned)p.qblocks, (unsigned)p.split);
    const dim3 pre_grid((unsigned)p.pre_qblocks, (unsigned)p.split);
    if (o.lambda_mode == SDF_LAMBDA_GLOBAL)
        k_prepass<SDF_LAMBDA_GLOBAL><<<pre_grid, kThreads, kStages * kPreBytes, st>>>(
            c.pre, c.n, c.pre_tiles, p.pre_tiles_per_chunk, a, c.status);
    else
        k_prepass<SDF_LAMBDA_FIXED><<<pre_grid, kThreads, kStages * kPreBytes, st>>>(
            c.pre, c.n, c.pre_tiles, p.pre_tiles_per_chunk, a, c.status);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) {
        fwd_kernel(SDF_F32, c.weighted)<<<grid, kThreads, kStages * kTileBytes, st>>>(fwd_records(c), c.n_direct, c.n_kappa, c.tiles_direct,
                                                           c.tiles_direct + c.tiles_kappa, p.tiles_per_chunk, a,
                                                           c.status, c.n_kappa_flat);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && p.split > 1) {
        k_merge<<<(unsigned)((q + 255) / 256), 256, 0, st>>>(a);
        e = cudaGetLastError();
    }
    return e == cudaSuccess ? SDF_OK : cuda_error(e, "sdf_query_noalloc: launch");
}
