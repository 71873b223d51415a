// Tensor-core pair loop (FP32 result) for both torus record forms.
//
// Every per-pair quantity of the torus SDF (Eq. SingleTorusSDF) and of the
// weights (Eq. BasicFormulaShifted) that depends on both the query and the
// point is an inner product of a per-query and a per-point feature vector.
// In coordinates x'' = (x - centre) / s (centre of the cloud's bounding box,
// s a power of two at least its diagonal), with f(x) = (x'', |x''|^2, 1):
//
// direct form, (u, e1, e2) an orthonormal frame of the torus axis u:
//   d^2 = |x - p|^2     = f . (-2 p'', 1, |p''|^2)
//   h   = <x - c, u>    = f . (u, 0, -<c'', u>)
//   a   = <x - c, e1>   = f . (e1, 0, -<c'', e1>)
//   b   = <x - c, e2>   = f . (e2, 0, -<c'', e2>)
// so that rho^2 = a^2 + b^2 is the squared distance to the axis without the
// cancellation of |x - c|^2 - h^2 near the axis; the constants R, -sT r and
// sT come out through the constant feature.
//
// curvature form (Sec. 4.1, the form without 1/kappa), y = x - q:
//   d^2, h = <y, u>, |y|^2 = f . (-2 q'', 1, |q''|^2),
//   m0 = <y, 2 zeta n*> = f . (2 zeta n*, 0, -<q'', 2 zeta n*>)
// and the constants |kappa_min| s, -kappa_max s, 2 zeta.
//
// Seven quantities either way: one 128 x 224 x 32 product on the tensor
// cores (two tcgen05 MMAs of K = 16) gives them for 128 queries and a
// 32-point tile.  Tiles never mix the two forms (the record segments are
// padded to whole tiles), and the kernel is compiled once per formula (direct;
// whole kappa_min = 0 tiles; the other curvature-form tiles), one launch per
// range, so that no epilogue carries a per-tile choice.
//
// Per-point weights A (sdf_build_weighted) ride in the direct form's B tiles:
// -sT r and sT are scaled by A, so the epilogue's w (sT D - sT r) is A w g and
// W takes w |A sT| = A w (a separate instance of the direct loop).
//
// Precision: every feature and coefficient is split into three f16 parts
// (v = v_hi + v_mid + v_lo for FP32 inputs), and K holds the six cross
// products hi.hi, hi.mid, mid.hi, hi.lo, mid.mid, lo.hi.  The dropped terms
// are below 2^-30 of the products, but the smallest part of a value below 1
// is an f16 subnormal, an absolute floor of about 2^-25 per product (units of
// s or s^2); with the FP32 rounding of the accumulation the quantities carry
// absolute errors of order 1e-7 s^2 (d^2) and 1e-7 s |x - c| (h, a, b).
// Queries farther than 32 s from the centre, where |x''|^2 would leave the
// range these splits are sized for, take the formula of their tile's form
// from the FP32 record for every pair.
//
// A tile whose constants leave that range (|value| > 2^15, e.g. a tube radius
// below s / 2^15) is flagged at build time and every pair of it takes the
// FP32 record formula.
//
// The epilogue finishes each pair on the FP32 units.  Direct form:
// rho = sqrt(a^2 + b^2), D = sqrt((rho - R)^2 + h^2), g = sT D - sT r (three
// square roots with d).  Curvature form: the two half-angle steps of the
// record formula (kappa_min = 0 tiles skip the first, which is then exact
// without a root; the other tiles take the two steps over one denominator),
// three roots and one reciprocal with d, or two and one.  Then w = exp2(-L (d - d_min)), W += w, S += w g.  The packed
// epilogues keep W and S as .f32x2 running sums (one per point parity of a
// step) for the lane's whole share of the tiles and add the two halves once
// at the end: on the dense grid this saves the four scalar adds per batch
// (1,452.9 -> 1,442.8 ms per 256^3 step) and lowers the error against the
// oracle (max 6.6e-7 -> 4.7e-7 of the diagonal on 8,192 nodes), two shorter
// chains of additions instead of one.  The sums finish into the blend S / W
// or the log-sum-exp distance (finish_sums).
//
// Warps: 0 producer (bulk copies of B tiles into an 8-stage ring), 1 MMA
// issuer and TMEM owner (two 224-column accumulators), 2..17 epilogue in two
// sets of eight that take alternate tiles (set 0 the even tiles in
// accumulator 0, set 1 the odd ones in accumulator 1), so the two sets run
// out of phase and their square-root bursts do not meet on the MUFU queue.
// In a set, two warps per TMEM lane quadrant each take 16 of the tile's 32
// points (two batches of 8) for their 32 query rows.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "query_common.cuh"
#include "tc_common.cuh"

namespace ptsdf {

using namespace qk;

namespace {

static_assert(kTileRecs == 32, "the tensor-core path packs 32-point tiles");

constexpr int kTcM = 128;                             // queries per CTA (MMA M)
constexpr int kTcQuant = 7;                           // direct: d^2, h, a, b, R, -sT r, sT
                                                      // kappa: d^2, h, |y|^2, m0, |kmin| s, -kmax s, 2 zeta
constexpr int kTcN = kTcQuant * kTileRecs;            // 224 (MMA N)
constexpr uint32_t kTcSubA = kTcM * 32;               // one K = 16 sub-tile of A (4 KB)
constexpr uint32_t kTcSubB = kTcN * 32;               // one K = 16 sub-tile of B (7 KB)
constexpr uint32_t kBTileBytes = 2 * kTcSubB;         // K = 32
#ifndef PTSDF_TC_KAPPA2
#define PTSDF_TC_KAPPA2 1   // curvature-form epilogue: .f32x2 arithmetic and d on the FMA pipe (0: scalar)
#endif
#ifndef PTSDF_TC_ACC2
#define PTSDF_TC_ACC2 1     // the packed epilogues add into .f32x2 sums kept across batches and tiles (0: into W, S per batch)
#endif
#ifndef PTSDF_TC_ONE_RCP
#define PTSDF_TC_ONE_RCP 1  // general curvature-form pairs: one reciprocal instead of two (0: the record formula's two)
#endif
#ifndef PTSDF_TC_FLAT_LD
#define PTSDF_TC_FLAT_LD 1  // flat tiles load only the five quantities their formula reads (0: all seven)
#endif
#ifndef PTSDF_TC_STAGES
#define PTSDF_TC_STAGES 8
#endif
constexpr int kTcStages = PTSDF_TC_STAGES;
constexpr int kEpiGroups = 4;                         // epilogue warps per TMEM lane quadrant
constexpr int kEpiWarps = 4 * kEpiGroups;
constexpr int kEpiSets = 2;                           // sets of epilogue warps taking alternate tiles
constexpr int kSetWarps = kEpiWarps / kEpiSets;
constexpr int kPtsPerWarp = 8;                        // points per TMEM batch (one column group)
constexpr int kGroupsPerWarp = kTileRecs / kPtsPerWarp / (kEpiGroups / kEpiSets);   // 2 batches
constexpr int kVals = kTcQuant * kPtsPerWarp;         // 56 accumulator columns per epilogue warp
constexpr int kTcThreads = (2 + kEpiWarps) * 32;
constexpr uint32_t kTmemCols = 512;                   // two accumulators of kTcN columns
constexpr uint32_t kBufCols = 256;
constexpr float kFarSq = 1024.f;                      // |x''|^2 beyond which a query is exact-only
constexpr double kMaxCoef = 32768.0;                  // largest B coefficient the f16 split takes
enum TileForm { kFormDirect = 0, kFormKappa = 1, kFormFlat = 2 };
constexpr uint32_t kTcIdesc = tc::idesc_f16_f32(kTcM, kTcN);
// dynamic shared memory: A, the ring, the group partial sums; padded so that
// two CTAs never share an SM (each holds all 512 TMEM columns)
constexpr size_t kTcSmemUsed = 2 * kTcSubA + (size_t)kTcStages * kBTileBytes + (kEpiGroups - 1) * kTcM * 8;
constexpr size_t kTcSmemBytes = kTcSmemUsed > 118 * 1024 ? kTcSmemUsed : 118 * 1024;

// B row of quantity k of point j: each epilogue warp's 8 points x 7
// quantities are 56 consecutive accumulator columns
__host__ __device__ constexpr int brow(int j, int k) {
    return (j / kPtsPerWarp) * kVals + k * kPtsPerWarp + (j % kPtsPerWarp);
}

// Which part of the split each K slot holds (0 hi, 1 mid, 2 lo; -1 zero).
// A: [hi hi mid 0 | hi mid lo 0], B: [hi mid hi 0 | lo mid hi 0], 5 slots per
// segment: the products are hi.hi + hi.mid + mid.hi + hi.lo + mid.mid + lo.hi.
__host__ __device__ constexpr int a_part(int m) {
    return (m % 16 == 15) ? -1 : (m < 16 ? ((m % 16) / 5 == 2 ? 1 : 0) : (m % 16) / 5);
}
__host__ __device__ constexpr int b_part(int m) {
    return (m % 16 == 15) ? -1 : (m < 16 ? ((m % 16) / 5 == 1 ? 1 : 0) : 2 - (m % 16) / 5);
}
static_assert(kTcN % 16 == 0 && kTcN <= 256 && kTcN <= (int)kBufCols, "MMA N for M = 128");
static_assert(a_part(0) == 0 && a_part(5) == 0 && a_part(10) == 1 && a_part(16) == 0 && a_part(21) == 1 &&
                  a_part(26) == 2 && a_part(31) == -1,
              "A slot layout");
static_assert(b_part(0) == 0 && b_part(5) == 1 && b_part(10) == 0 && b_part(16) == 2 && b_part(21) == 1 &&
                  b_part(26) == 0 && b_part(15) == -1,
              "B slot layout");

// byte offset of K slot m of `row` in a two-sub-tile operand
__host__ __device__ inline uint32_t slot_offset(int row, int m, uint32_t sub_bytes) {
    return (uint32_t)(m / 16) * sub_bytes + tc::canon_offset(row, m % 16);
}

// One thread per record slot of every tile (both segments).  Padding slots
// get all-zero rows (their pairs are masked in the epilogue).  A tile with a
// coefficient outside the split's range gets its exact flag set.
__global__ void k_build_btiles(const float4* __restrict__ rec, int64_t n_direct, int64_t tiles_direct,
                               int64_t n_kappa, int64_t tiles_total, double cx, double cy, double cz, double inv_s,
                               uint8_t* __restrict__ bt, int32_t* __restrict__ exact) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= tiles_total * kTileRecs) return;
    const int64_t t = i / kTileRecs;
    const int j = (int)(i % kTileRecs);
    const bool kappa = t >= tiles_direct;
    const bool valid = kappa ? i - tiles_direct * kTileRecs < n_kappa : i < n_direct;
    double b[kTcQuant][5];
    for (int k = 0; k < kTcQuant; ++k)
        for (int m = 0; m < 5; ++m) b[k][m] = 0.0;
    if (valid && !kappa) {
        const float4 r0 = rec[4 * i], r1 = rec[4 * i + 1], r2 = rec[4 * i + 2];
        const double p[3] = {((double)r0.x - cx) * inv_s, ((double)r0.y - cy) * inv_s, ((double)r0.z - cz) * inv_s};
        const double c[3] = {((double)r1.x - cx) * inv_s, ((double)r1.y - cy) * inv_s, ((double)r1.z - cz) * inv_s};
        const double u[3] = {r2.x, r2.y, r2.z};
        // e1, e2: an orthonormal basis of the plane normal to u
        const double un = sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
        const double w[3] = {u[0] / un, u[1] / un, u[2] / un};
        const int ax = (fabs(w[0]) <= fabs(w[1]) && fabs(w[0]) <= fabs(w[2])) ? 0 : (fabs(w[1]) <= fabs(w[2]) ? 1 : 2);
        double t[3] = {0.0, 0.0, 0.0};
        t[ax] = 1.0;
        double e1[3] = {w[1] * t[2] - w[2] * t[1], w[2] * t[0] - w[0] * t[2], w[0] * t[1] - w[1] * t[0]};
        const double e1n = sqrt(e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2]);
        for (int m = 0; m < 3; ++m) e1[m] /= e1n;
        const double e2[3] = {w[1] * e1[2] - w[2] * e1[1], w[2] * e1[0] - w[0] * e1[2], w[0] * e1[1] - w[1] * e1[0]};
        for (int m = 0; m < 3; ++m) {
            b[0][m] = -2.0 * p[m];
            b[1][m] = u[m];
            b[2][m] = e1[m];
            b[3][m] = e2[m];
        }
        b[0][3] = 1.0;
        b[0][4] = p[0] * p[0] + p[1] * p[1] + p[2] * p[2];
        b[1][4] = -(c[0] * u[0] + c[1] * u[1] + c[2] * u[2]);
        b[2][4] = -(c[0] * e1[0] + c[1] * e1[1] + c[2] * e1[2]);
        b[3][4] = -(c[0] * e2[0] + c[1] * e2[1] + c[2] * e2[2]);
        b[4][4] = (double)r1.w * inv_s;   // R
        // -sT r and sT times the point's weight A (r3.w; 1 without weights):
        // the epilogue's w (sT D - sT r) is then A w g, and |A sT| = A
        const double A = rec[4 * i + 3].w;
        b[5][4] = A * (double)r2.w * inv_s;   // -A sT r
        b[6][4] = A * (double)r0.w;           // A sT
    } else if (valid) {
        // {p, 2 zeta}{q, |kmin|}{u, -kmax}{2 zeta n*, 0}
        const float4 r0 = rec[4 * i], r1 = rec[4 * i + 1], r2 = rec[4 * i + 2], r3 = rec[4 * i + 3];
        const double p[3] = {((double)r0.x - cx) * inv_s, ((double)r0.y - cy) * inv_s, ((double)r0.z - cz) * inv_s};
        const double q[3] = {((double)r1.x - cx) * inv_s, ((double)r1.y - cy) * inv_s, ((double)r1.z - cz) * inv_s};
        const double u[3] = {r2.x, r2.y, r2.z};
        const double zn[3] = {r3.x, r3.y, r3.z};
        for (int m = 0; m < 3; ++m) {
            b[0][m] = -2.0 * p[m];
            b[1][m] = u[m];
            b[2][m] = -2.0 * q[m];
            b[3][m] = zn[m];
        }
        b[0][3] = 1.0;
        b[0][4] = p[0] * p[0] + p[1] * p[1] + p[2] * p[2];
        b[1][4] = -(q[0] * u[0] + q[1] * u[1] + q[2] * u[2]);
        b[2][3] = 1.0;
        b[2][4] = q[0] * q[0] + q[1] * q[1] + q[2] * q[2];
        b[3][4] = -(q[0] * zn[0] + q[1] * zn[1] + q[2] * zn[2]);
        b[4][4] = (double)r1.w / inv_s;   // |kappa_min| in units of 1/s
        b[5][4] = (double)r2.w / inv_s;   // -kappa_max
        b[6][4] = r0.w;                   // 2 zeta
    }
    bool in_range = true;
    for (int k = 0; k < kTcQuant; ++k)
        for (int m = 0; m < 5; ++m) in_range = in_range && fabs(b[k][m]) <= kMaxCoef;
    if (!in_range) {
        atomicOr(exact + t, 1);
        for (int k = 0; k < kTcQuant; ++k)
            for (int m = 0; m < 5; ++m) b[k][m] = 0.0;
    }
    uint8_t* tile = bt + (size_t)t * kBTileBytes;
    for (int k = 0; k < kTcQuant; ++k) {
        const int row = brow(j, k);
        __half part[3][5];
        for (int m = 0; m < 5; ++m) {
            const double v = b[k][m];
            part[0][m] = __double2half(v);
            const double r1 = v - (double)__half2float(part[0][m]);
            part[1][m] = __double2half(r1);
            part[2][m] = __double2half(r1 - (double)__half2float(part[1][m]));
        }
        for (int m = 0; m < 32; ++m) {
            const int pt = b_part(m);
            *reinterpret_cast<__half*>(tile + slot_offset(row, m, kTcSubB)) =
                pt < 0 ? __float2half(0.f) : part[pt][(m % 16) % 5];
        }
    }
}

struct TcArgs {
    TcQuery a;
    const uint8_t* btiles;
    const int32_t* tile_exact;   // per tile: 1 when its pairs must take the record formula
    const float4* rec;
    int64_t tiles_begin, tiles_end, tiles_per_chunk;   // tiles [begin, end) in chunks
    // tile classes (tiles < 2^26): [0, tiles_direct) direct, of which the
    // first direct_full are full; then the kappa-form tiles, kappa_full of
    // them full; *_rem points in the partial last tile of each segment
    int32_t tiles_direct, direct_full, kappa_full, direct_rem, kappa_rem;
    float s, inv_s;          // coordinate scale of the B tiles (a power of two) and its inverse
    int direct_out;          // 1: write phi; 0: write (W, S) at partial row part_base + chunk
};

__device__ __forceinline__ float sqrt_abs_mufu(float x) { return sqrt_mufu(fabsf(x)); }

// torus distance of one curvature-form pair from the accumulator quantities
// q1..q6 (units of s): h, |y|^2, m0, |kmin|, -kmax, 2 zeta
template <int FORM>
__device__ __forceinline__ float g_from_quantities(float q1, float q2, float q3, float q4, float q5, float q6) {
    static_assert(FORM != kFormDirect, "direct-form pairs go through tile_pairs_direct2");
    const float hh = q1 * q1;
    float ap;
    if (FORM == kFormFlat) {
        ap = 0.5f * q3;
    } else {
        const float m = fmaf(q4, q2 - hh, q3);
        const float s1 = sqrt_mufu(fmaxf(fmaf(q4, m, 1.f), 0.f));
        ap = m * rcp_mufu(1.f + s1);
    }
    const float Np = fmaf(q5, fmaf(ap, ap, hh), q6 * ap);
    const float s2 = sqrt_mufu(fmaxf(fmaf(q5, Np, 1.f), 0.f));
    return Np * rcp_mufu(1.f + s2);
}

// The direct form's share, two points at a time: the FP32 arithmetic of a
// lane's two pairs as .f32x2, and the square root of d^2 (which only sets
// the weight) on the FMA pipe (sqrt2_newton, two Newton steps: 4.7e-6
// relative), so that the special-function unit does 2 sqrt + 1 exp2 per pair
// (20 of its cycles per 32 pairs instead of 28).  On the dense grid this
// runs 3.8% faster than a scalar epilogue with three MUFU square roots
// (1,091 against 1,051 Gpairs/s per step); a third Newton step, or fitted
// constants for the two, cost more issue slots or registers than they save,
// and so did keeping the MUFU root for one pair in two or in four (1,072 and
// 1,064).  FMA-pipe work per pair: 17 FP32 operations (8 of them the square
// root); ALU: the clamp and the integer estimate.
template <bool WEIGHTED>
__device__ __forceinline__ void tile_pairs_direct2(const float (&v)[kVals], float Ls, float A0, f32x2& tw, f32x2& ts) {
    const f32x2 NLs = f2_pack(-Ls, -Ls), A0v = f2_pack(A0, A0);
#pragma unroll
    for (int i = 0; i < kPtsPerWarp; i += 2) {
        // q1 h, q2 a, q3 b, q4 R, q5 -sT r, q6 sT of points i and i + 1
        const f32x2 h = f2_pack(v[8 + i], v[9 + i]), a = f2_pack(v[16 + i], v[17 + i]);
        const f32x2 b = f2_pack(v[24 + i], v[25 + i]), R = f2_pack(v[32 + i], v[33 + i]);
        const f32x2 nsr = f2_pack(v[40 + i], v[41 + i]), sT = f2_pack(v[48 + i], v[49 + i]);
        const f32x2 rr = f2_fma(a, a, f2_mul(b, b));
        const f32x2 e = f2_sub(f2_pack(sqrt_mufu(f2_lo(rr)), sqrt_mufu(f2_hi(rr))), R);
        const f32x2 ee = f2_fma(e, e, f2_mul(h, h));
        const f32x2 g = f2_fma(sT, f2_pack(sqrt_mufu(f2_lo(ee)), sqrt_mufu(f2_hi(ee))), nsr);
        // |d^2|: the products may round a zero distance slightly negative
        const f32x2 d = sqrt2_newton(fabsf(v[i]), fabsf(v[i + 1]));
        const f32x2 arg = f2_fma(NLs, d, A0v);
        const f32x2 w = f2_pack(ex2_mufu(f2_lo(arg)), ex2_mufu(f2_hi(arg)));
        tw = WEIGHTED ? f2_fma(w, f2_pack(fabsf(v[48 + i]), fabsf(v[49 + i])), tw) : f2_add(tw, w);
        ts = f2_fma(w, g, ts);
    }
}

// The curvature forms' share, two points at a time: the half-angle steps'
// FP32 arithmetic as .f32x2 (the MUFU roots and reciprocals stay scalar) and
// d on the FMA pipe as in the direct form, so that a flat pair costs the
// special-function unit 1 sqrt + 1 rcp + 1 exp2 (20 cycles per 32 pairs
// instead of 28) and a curved one, with its two half-angle steps over one
// denominator, 2 sqrt + 1 rcp + 1 exp2 (28 instead of 44).
template <int FORM>
__device__ __forceinline__ void tile_pairs_kappa2(const float (&v)[kVals], float Ls, float A0, f32x2& tw, f32x2& ts) {
    const f32x2 NLs = f2_pack(-Ls, -Ls), A0v = f2_pack(A0, A0), ONE = f2_pack(1.f, 1.f);
#pragma unroll
    for (int i = 0; i < kPtsPerWarp; i += 2) {
        // q1 h, q2 |y|^2, q3 m0, q4 |kmin|, q5 -kmax, q6 2 zeta of points i and i + 1
        const f32x2 h = f2_pack(v[8 + i], v[9 + i]), m0 = f2_pack(v[24 + i], v[25 + i]);
        const f32x2 nkM = f2_pack(v[40 + i], v[41 + i]), z2 = f2_pack(v[48 + i], v[49 + i]);
        const f32x2 hh = f2_mul(h, h);
        f32x2 g;
        if (FORM != kFormFlat && PTSDF_TC_ONE_RCP) {
            // The general formula with one reciprocal: with D1 = 1 + sqrt(1 + k m),
            // a' = m / D1 and Nn = N' D1^2 = kM (m^2 + h^2 D1^2) + 2 zeta m D1 (kM the
            // record's -kappa_max), 1 + kM N' = (D1^2 + kM Nn) / D1^2, so
            // g = N' / (1 + sqrt(1 + kM N')) = Nn / (D1 (D1 + sqrt(D1^2 + kM Nn))).
            // D1 >= 1 keeps the denominator >= 1, and the clamp of the second
            // root's argument at 0 is the same as the general formula's.
            const f32x2 yy = f2_pack(v[16 + i], v[17 + i]), k = f2_pack(v[32 + i], v[33 + i]);
            const f32x2 m = f2_fma(k, f2_sub(yy, hh), m0);
            const f32x2 t1 = f2_fma(k, m, ONE);
            const f32x2 D1 = f2_add(ONE, f2_pack(sqrt_mufu(fmaxf(f2_lo(t1), 0.f)), sqrt_mufu(fmaxf(f2_hi(t1), 0.f))));
            const f32x2 D1sq = f2_mul(D1, D1);
            const f32x2 Nn = f2_fma(nkM, f2_fma(m, m, f2_mul(hh, D1sq)), f2_mul(z2, f2_mul(m, D1)));
            const f32x2 u = f2_fma(nkM, Nn, D1sq);
            const f32x2 den = f2_mul(D1, f2_add(D1, f2_pack(sqrt_mufu(fmaxf(f2_lo(u), 0.f)),
                                                            sqrt_mufu(fmaxf(f2_hi(u), 0.f)))));
            g = f2_mul(Nn, f2_pack(rcp_mufu(f2_lo(den)), rcp_mufu(f2_hi(den))));
        } else {
            f32x2 ap;
            if (FORM == kFormFlat) {
                ap = f2_mul(m0, f2_pack(0.5f, 0.5f));
            } else {
                const f32x2 yy = f2_pack(v[16 + i], v[17 + i]), k = f2_pack(v[32 + i], v[33 + i]);
                const f32x2 m = f2_fma(k, f2_sub(yy, hh), m0);
                const f32x2 t1 = f2_fma(k, m, ONE);
                const f32x2 den1 =
                    f2_add(ONE, f2_pack(sqrt_mufu(fmaxf(f2_lo(t1), 0.f)), sqrt_mufu(fmaxf(f2_hi(t1), 0.f))));
                ap = f2_mul(m, f2_pack(rcp_mufu(f2_lo(den1)), rcp_mufu(f2_hi(den1))));
            }
            const f32x2 Np = f2_fma(nkM, f2_fma(ap, ap, hh), f2_mul(z2, ap));
            const f32x2 t2 = f2_fma(nkM, Np, ONE);
            const f32x2 den2 =
                f2_add(ONE, f2_pack(sqrt_mufu(fmaxf(f2_lo(t2), 0.f)), sqrt_mufu(fmaxf(f2_hi(t2), 0.f))));
            g = f2_mul(Np, f2_pack(rcp_mufu(f2_lo(den2)), rcp_mufu(f2_hi(den2))));
        }
        // |d^2|: the products may round a zero distance slightly negative
        const f32x2 d = sqrt2_newton(fabsf(v[i]), fabsf(v[i + 1]));
        const f32x2 arg = f2_fma(NLs, d, A0v);
        const f32x2 w = f2_pack(ex2_mufu(f2_lo(arg)), ex2_mufu(f2_hi(arg)));
        tw = f2_add(tw, w);
        ts = f2_fma(w, g, ts);
    }
}

// One epilogue warp's share of a full tile from the accumulator: 8 pairs per
// lane; v[k * 8 + i] is quantity k of point i.  WEIGHTED (direct form only):
// quantity 6 is A sT, so W takes w |A sT| = A w (S takes A w g through the
// scaled constants of g).
// W2, S2: the packed epilogues' running .f32x2 sums (PTSDF_TC_ACC2); else
// each batch's packed sums are added into W, S.
template <int FORM, bool WEIGHTED = false>
__device__ __forceinline__ void tile_pairs(const float (&v)[kVals], float Ls, float A0, float& W, float& S,
                                           f32x2& W2, f32x2& S2) {
    constexpr bool kPacked = FORM == kFormDirect || (PTSDF_TC_KAPPA2 && !WEIGHTED);
    if constexpr (kPacked) {
        f32x2 tw = f2_pack(0.f, 0.f), ts = tw;
        f32x2& aw = PTSDF_TC_ACC2 ? W2 : tw;
        f32x2& as = PTSDF_TC_ACC2 ? S2 : ts;
        if constexpr (FORM == kFormDirect)
            tile_pairs_direct2<WEIGHTED>(v, Ls, A0, aw, as);
        else
            tile_pairs_kappa2<FORM>(v, Ls, A0, aw, as);
        if (!PTSDF_TC_ACC2) {
            W += f2_lo(tw) + f2_hi(tw);
            S += f2_lo(ts) + f2_hi(ts);
        }
    } else {
        float tw = 0.f, ts = 0.f;
#pragma unroll
        for (int i = 0; i < kPtsPerWarp; ++i) {
            const float g = g_from_quantities<FORM>(v[8 + i], v[16 + i], v[24 + i], v[32 + i], v[40 + i], v[48 + i]);
            // |d^2|: the products may round a zero distance slightly negative
            const float d = sqrt_abs_mufu(v[i]);
            const float w = ex2_mufu(fmaf(-Ls, d, A0));
            tw = WEIGHTED ? fmaf(w, fabsf(v[48 + i]), tw) : tw + w;
            ts = fmaf(w, g, ts);
        }
        W += tw;
        S += ts;
    }
}

// The same share from the FP32 records (the formula of the tile's form, in
// world units, rescaled to units of s): for far queries, for flagged tiles
// and for the partial last tile of a segment (only `valid` points exist).
// WEIGHTED: each weight times the point's A (r3.w).
template <int FORM, bool WEIGHTED = false>
__device__ __forceinline__ void record_pairs(int valid, float x, float y, float z, float inv_s,
                                             const float4* __restrict__ rec, int64_t slot0, float Ls, float A0,
                                             float& W, float& S) {
    float tw = 0.f, ts = 0.f;
#pragma unroll 1
    for (int i = 0; i < valid; ++i) {
        const float4* r = rec + 4 * (slot0 + i);
        const float4 r0 = __ldg(r), r1 = __ldg(r + 1), r2 = __ldg(r + 2);
        float g;
        if (FORM == kFormDirect) {
            g = g_direct(x, y, z, r1, r2, r0.w);
        } else {
            const float4 r3 = __ldg(r + 3);
            g = FORM == kFormFlat ? g_kappa_flat(x, y, z, r0, r1, r2, r3) : g_kappa(x, y, z, r0, r1, r2, r3);
        }
        g *= inv_s;
        const float dx = x - r0.x, dy = y - r0.y, dz = z - r0.z;
        const float d = sqrt_mufu(fmaf(dx, dx, fmaf(dy, dy, dz * dz))) * inv_s;
        float w = ex2_mufu(fmaf(-Ls, d, A0));
        if (WEIGHTED) w *= __ldg(r + 3).w;
        tw += w;
        ts = fmaf(w, g, ts);
    }
    W += tw;
    S += ts;
}

// 18 warps: five share one SM sub-partition's 16K registers, so at most 96
// registers per thread (allocated in multiples of 8)
// FORMS: the one formula of the launch's tiles.  kFormDirect: direct-form
// tiles, never flagged without weights (their coefficients are bounded by
// the 8-diagonal radius rule).  kFormFlat: whole curvature-form tiles whose
// points all have kappa_min = 0.  kFormKappa: the other curvature-form tiles
// (the general formula, exact for kappa_min = 0 too, so the tile at the
// flat boundary may mix them).  Curvature-form tiles may be flagged.
// WEIGHTED (direct segment of a weighted cloud): the B tiles carry A sT, and
// tiles whose scaled constants left the f16 split's range are flagged too.
template <int FORMS, bool WEIGHTED>
__global__ void __maxnreg__(96) k_fwd_tc(TcArgs ta, int32_t* status) {
    constexpr bool KAPPA = FORMS != kFormDirect;
    extern __shared__ __align__(1024) uint8_t smem[];
    uint8_t* sA = smem;                                                         // 2 sub-tiles
    uint8_t* sB = smem + 2 * kTcSubA;                                           // kTcStages tiles
    float2* sComb = reinterpret_cast<float2*>(sB + (size_t)kTcStages * kBTileBytes);   // [kEpiGroups - 1][kTcM]
    __shared__ __align__(8) uint64_t bfull[kTcStages], bempty[kTcStages], tfull[2], tempty[2];
    __shared__ uint32_t tmem_base;
    __shared__ int abort_flag;
    const TcQuery& a = ta.a;
    const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
    const int chunk = blockIdx.y;
    const int64_t t0 = ta.tiles_begin + (int64_t)chunk * ta.tiles_per_chunk;
    const int64_t t1 = t0 + ta.tiles_per_chunk < ta.tiles_end ? t0 + ta.tiles_per_chunk : ta.tiles_end;
    const int64_t nt = t1 > t0 ? t1 - t0 : 0;

    if (tid == 0) {
        for (int s = 0; s < kTcStages; ++s) {
            mbar_init(&bfull[s], 1);
            mbar_init(&bempty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&tfull[b], 1);
            mbar_init(&tempty[b], kSetWarps);
        }
        abort_flag = 0;
        fence_mbar_init();
    }
    if (warp == 1) tc::tmem_alloc(&tmem_base, kTmemCols);

    // epilogue threads: one query row each; combine group 0 also writes the A row
    const int quad = warp & 3;            // TMEM lane quadrant this warp may access
    const int eset = (warp - 2) >> 3;     // tile parity this warp takes
    const int half = ((warp - 2) >> 2) & 1;   // which 16 points of each tile
    const int group = eset * 2 + half;    // which partial sums it contributes to the row
    const int row = quad * 32 + lane;
    const int64_t qi = (int64_t)blockIdx.x * kTcM + row;
    float x = 0.f, y = 0.f, z = 0.f, Ls = 0.f, A0 = 0.f;
    bool exact_lane = false;
    if (warp >= 2) {
        const int64_t qq = qi < a.q ? qi : a.q - 1;
        x = a.x[3 * qq];
        y = a.x[3 * qq + 1];
        z = a.x[3 * qq + 2];
        float L;            // exponent A0 - L d = -lambda_x (d - d_min) log2(e), d in world units
        query_screening(a.d2, a.pre_split, a.q, qq, a.mode, a.C, a.lam, L, A0);
        Ls = L * ta.s;      // the same per unit of d'' = d / s
        const float xs = (x - a.cx) * ta.inv_s, ys = (y - a.cy) * ta.inv_s, zs = (z - a.cz) * ta.inv_s;
        const float xx = fmaf(xs, xs, fmaf(ys, ys, zs * zs));
        exact_lane = !(xx <= kFarSq) && xx == xx;   // far (or infinite); NaN queries stay NaN
        if (group == 0) {
            const float f[5] = {xs, ys, zs, xx, 1.f};
            __half part[3][5];
#pragma unroll
            for (int m = 0; m < 5; ++m) {
                const float fv = exact_lane ? 0.f : f[m];
                part[0][m] = __float2half_rn(fv);
                const float r1 = fv - __half2float(part[0][m]);
                part[1][m] = __float2half_rn(r1);
                part[2][m] = __float2half_rn(r1 - __half2float(part[1][m]));
            }
#pragma unroll
            for (int m = 0; m < 32; ++m) {
                const int pt = a_part(m);
                *reinterpret_cast<__half*>(sA + slot_offset(row, m, kTcSubA)) =
                    pt < 0 ? __float2half(0.f) : part[pt][(m % 16) % 5];
            }
            tc::fence_proxy_async_smem();
        }
    }
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tbase = tmem_base;

    if (warp == 0) {
        // ---- producer: B tiles through the shared-memory ring ----
        if (lane == 0) {
            int64_t issued = 0;
            for (int64_t t = 0; t < nt; ++t) {
                const int s = (int)(t % kTcStages);
                if (t >= kTcStages &&
                    !mbar_wait_bounded(&bempty[s], (uint32_t)(((t / kTcStages) - 1) & 1), &abort_flag, status))
                    break;
                mbar_arrive_expect_tx(&bfull[s], kBTileBytes);
                bulk_g2s(sB + (size_t)s * kBTileBytes, ta.btiles + (size_t)(t0 + t) * kBTileBytes, kBTileBytes,
                         &bfull[s]);
                issued = t + 1;
            }
            if (*(volatile int*)&abort_flag) {   // copies in flight land before the CTA ends
                for (int64_t t = (issued > kTcStages ? issued - kTcStages : 0); t < issued; ++t) {
                    const uint64_t tw = global_ns();
                    while (!mbar_try_wait(&bfull[t % kTcStages], (uint32_t)((t / kTcStages) & 1)))
                        if (global_ns() - tw > kWaitLimitNs) break;
                }
            }
        }
    } else if (warp == 1) {
        // ---- MMA issuer ----
        if (lane == 0) {
            const uint32_t sa = smem_u32(sA);
            const uint64_t adesc0 = tc::smem_desc(sa), adesc1 = tc::smem_desc(sa + kTcSubA);
            int64_t issued = 0;
            for (int64_t t = 0; t < nt; ++t) {
                const int s = (int)(t % kTcStages);
                const int b = (int)(t & 1);
                if (!mbar_wait_bounded(&bfull[s], (uint32_t)((t / kTcStages) & 1), &abort_flag, status)) break;
                if (t >= 2 && !mbar_wait_bounded(&tempty[b], (uint32_t)(((t >> 1) - 1) & 1), &abort_flag, status))
                    break;
                tc::fence_after_sync();
                const uint32_t d = tbase + (uint32_t)b * kBufCols;
                const uint32_t sb = smem_u32(sB + (size_t)s * kBTileBytes);
                tc::mma_f16(d, adesc0, tc::smem_desc(sb), kTcIdesc, 0u);
                tc::mma_f16(d, adesc1, tc::smem_desc(sb + kTcSubB), kTcIdesc, 1u);
                tc::commit(&tfull[b]);
                tc::commit(&bempty[s]);
                issued = t + 1;
            }
            if (issued > 0) {   // the last MMA completes before TMEM is released
                const uint64_t tw = global_ns();
                while (!mbar_try_wait(&tfull[(issued - 1) & 1], (uint32_t)(((issued - 1) >> 1) & 1)))
                    if (global_ns() - tw > kWaitLimitNs) break;
            }
        }
    } else {
        // ---- epilogue ----
        float W = 0.f, S = 0.f;
        f32x2 W2 = f2_pack(0.f, 0.f), S2 = W2;
        const uint32_t lane_addr = tbase + ((uint32_t)(quad * 32) << 16);
        const int ntiles = (int)nt;
        const int b = eset;   // this set's accumulator
        const int32_t* flags = ta.tile_exact + t0;
        // the next tile's exact flag is fetched one tile ahead
        int32_t flag_next = (KAPPA || WEIGHTED) && eset < ntiles ? __ldg(flags + eset) : 0;
        for (int t = eset; t < ntiles; t += kEpiSets) {
            const bool flagged = (KAPPA || WEIGHTED) && flag_next != 0;
            if ((KAPPA || WEIGHTED) && t + kEpiSets < ntiles) flag_next = __ldg(flags + t + kEpiSets);
            // warp-uniform: the TMEM loads below are .sync.aligned
            const bool ok = mbar_wait_bounded(&tfull[b], (uint32_t)(t >> 1) & 1u, &abort_flag, status);
            if (!__all_sync(0xffffffffu, ok)) break;
            tc::fence_after_sync();
            const int gt = (int)t0 + t;
            const int rel = KAPPA ? gt - ta.tiles_direct : gt;   // tile within its segment
            const bool partial = rel >= (KAPPA ? ta.kappa_full : ta.direct_full);
            // pairs from the records: far lanes, flagged and partial tiles
            const bool lane_rec = exact_lane || flagged || partial;
#pragma unroll 1
            for (int gb = 0; gb < kGroupsPerWarp; ++gb) {
                const int cg = half * kGroupsPerWarp + gb;   // column group: 8 points x 7 quantities
                float v[kVals];
                const uint32_t ta_addr = lane_addr + (uint32_t)b * kBufCols + (uint32_t)(cg * kVals);
                if constexpr (FORMS == kFormFlat && PTSDF_TC_FLAT_LD) {
                    // the flat formula reads d^2, h, m0, -kmax s and 2 zeta
                    // (quantities 0, 1, 3, 5, 6): |y|^2 and |kmin| s stay in TMEM
                    tc::tmem_ld16(ta_addr, v, 0);
                    tc::tmem_ld8(ta_addr + 24, v, 24);
                    tc::tmem_ld16(ta_addr + 40, v, 40);
                    tc::tmem_wait_ld();
#pragma unroll
                    for (int i = 0; i < kVals; ++i)
                        if (i < 16 || (i >= 24 && i < 32) || i >= 40) asm volatile("" : "+f"(v[i]));
                } else {
                    tc::tmem_ld16(ta_addr, v, 0);
                    tc::tmem_ld16(ta_addr + 16, v, 16);
                    tc::tmem_ld16(ta_addr + 32, v, 32);
                    tc::tmem_ld8(ta_addr + 48, v, 48);
                    tc::tmem_wait_ld_values(v);
                }
                if (gb == kGroupsPerWarp - 1) {   // the accumulator is read: the next MMA may overwrite it
                    tc::fence_before_sync();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&tempty[b]);
                }
                if (!lane_rec) {
                    tile_pairs<FORMS, WEIGHTED>(v, Ls, A0, W, S, W2, S2);
                } else {
                    int valid = kPtsPerWarp;
                    if (partial) {
                        const int left = (KAPPA ? ta.kappa_rem : ta.direct_rem) - cg * kPtsPerWarp;
                        valid = left < 0 ? 0 : left > kPtsPerWarp ? kPtsPerWarp : left;
                    }
                    const int64_t slot0 = (int64_t)gt * kTileRecs + cg * kPtsPerWarp;
                    record_pairs<FORMS, WEIGHTED>(valid, x, y, z, ta.inv_s, ta.rec, slot0, Ls, A0, W, S);
                }
            }
        }
        if (PTSDF_TC_ACC2) {
            W += f2_lo(W2) + f2_hi(W2);
            S += f2_lo(S2) + f2_hi(S2);
        }
        S *= ta.s;   // back to world units
        // combine the four groups of each query row (named barrier of the epilogue warps)
        if (group > 0) sComb[(group - 1) * kTcM + row] = make_float2(W, S);
        asm volatile("bar.sync 1, %0;" ::"r"(kEpiWarps * 32) : "memory");
        if (group == 0 && qi < a.q) {
#pragma unroll
            for (int gq = 0; gq < kEpiGroups - 1; ++gq) {
                const float2 o = sComb[gq * kTcM + row];
                W += o.x;
                S += o.y;
            }
            if (ta.direct_out)   // Ls / s = L, the exponent's lambda log2(e) per world unit
                a.phi[qi] = finish_sums(W, S, a.formula, Ls * ta.inv_s, A0, a.offset);
            else
                a.part[(size_t)(a.part_base + chunk) * a.q + qi] = make_float2(W, S);
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 1) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tbase, kTmemCols);
    }
}

}  // namespace

float tc_scale_for(float aabb_diag) {
    int e = 0;
    std::frexp(std::max((double)aabb_diag, 0x1p-60), &e);   // diag = m 2^e, m in [0.5, 1)
    e = std::min(std::max(e, -60), 60);
    return (float)std::ldexp(1.0, e);
}

sdf_status build_btiles(Cloud& c, cudaStream_t st) {
    c.tc_scale = tc_scale_for(c.aabb_diag);
    const int64_t tiles = c.tiles_direct + c.tiles_kappa;
    if (tiles == 0) return SDF_OK;
    cudaError_t e = cudaMalloc(&c.btiles, (size_t)tiles * kBTileBytes);
    if (e == cudaSuccess) e = cudaMalloc(&c.btile_exact, (size_t)tiles * sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMemsetAsync(c.btile_exact, 0, (size_t)tiles * sizeof(int32_t), st);
    if (e != cudaSuccess) {
        cudaFree(c.btiles);
        cudaFree(c.btile_exact);
        c.btiles = nullptr;
        c.btile_exact = nullptr;
        return e == cudaErrorMemoryAllocation ? set_error(SDF_ENOMEM, "sdf_build: tensor-core tiles")
                                              : cuda_error(e, "sdf_build: tensor-core tiles");
    }
    const int64_t slots = tiles * kTileRecs;
    k_build_btiles<<<(unsigned)((slots + 127) / 128), 128, 0, st>>>(
        c.rec, c.n_direct, c.tiles_direct, c.n_kappa, tiles, 0.5 * ((double)c.aabb[0] + c.aabb[3]),
        0.5 * ((double)c.aabb[1] + c.aabb[4]), 0.5 * ((double)c.aabb[2] + c.aabb[5]), 1.0 / (double)c.tc_scale,
        c.btiles, c.btile_exact);
    e = cudaGetLastError();
    return e == cudaSuccess ? SDF_OK : cuda_error(e, "sdf_build: k_build_btiles launch");
}

int64_t tc_flat_end(const Cloud& c) {
    const int64_t end = tc_tiles_end(c), flat = c.tiles_direct + c.n_kappa_flat / kTileRecs;
    return flat < end ? flat : end;
}

int64_t tc_tiles_end(const Cloud& c) {
    if (c.weighted) return c.tiles_direct;   // weighted curvature-form tiles take the FP32 units
    if (PTSDF_TC_KAPPA) return c.tiles_direct + c.tiles_kappa;
    return c.tiles_direct + c.n_kappa_flat / kTileRecs;
}

int64_t tc_query_blocks(int64_t q) { return (q + kTcM - 1) / kTcM; }

sdf_status launch_fwd_tc(const Cloud& c, const TcQuery& a, int64_t tiles_begin, int64_t tiles_end,
                         int64_t tiles_per_chunk, int nchunks, int direct_out, cudaStream_t st) {
    // the range's one formula: direct tiles, whole kappa_min = 0 tiles, or the rest
    const int64_t flat_end = tc_flat_end(c);
    int forms;
    if (tiles_end <= c.tiles_direct)
        forms = kFormDirect;
    else if (tiles_begin >= c.tiles_direct && tiles_end <= flat_end)
        forms = kFormFlat;
    else if (tiles_begin >= flat_end)
        forms = kFormKappa;
    else
        forms = -1;
    if (tiles_begin >= tiles_end || forms < 0 || (forms != kFormDirect && c.weighted))
        return set_error(SDF_EINVAL, "sdf_query: tensor-core tile range straddles the record forms");
    static bool attr_done[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_error(e, "sdf_query: cudaGetDevice");
    if (dev < 0 || dev >= 64) return set_error(SDF_EINVAL, "sdf_query: device id out of range");
    if (!attr_done[dev]) {
        const void* kernels[4] = {(const void*)k_fwd_tc<kFormDirect, false>, (const void*)k_fwd_tc<kFormDirect, true>,
                                  (const void*)k_fwd_tc<kFormFlat, false>, (const void*)k_fwd_tc<kFormKappa, false>};
        for (int k = 0; k < 4 && e == cudaSuccess; ++k)
            e = cudaFuncSetAttribute(kernels[k], cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcSmemBytes);
        if (e != cudaSuccess) return cuda_error(e, "sdf_query: k_fwd_tc shared-memory attribute");
        attr_done[dev] = true;
    }
    TcArgs ta;
    ta.a = a;
    ta.btiles = c.btiles;
    ta.tile_exact = c.btile_exact;
    ta.rec = c.rec;
    ta.tiles_begin = tiles_begin;
    ta.tiles_end = tiles_end;
    ta.tiles_direct = (int32_t)c.tiles_direct;
    ta.direct_full = (int32_t)(c.n_direct / kTileRecs);
    ta.kappa_full = (int32_t)(c.n_kappa / kTileRecs);
    ta.direct_rem = (int32_t)(c.n_direct % kTileRecs);
    ta.kappa_rem = (int32_t)(c.n_kappa % kTileRecs);
    ta.tiles_per_chunk = tiles_per_chunk;
    ta.s = c.tc_scale;
    ta.inv_s = 1.f / c.tc_scale;
    ta.direct_out = direct_out;
    const dim3 grid((unsigned)tc_query_blocks(a.q), (unsigned)nchunks);
    if (forms == kFormFlat)
        k_fwd_tc<kFormFlat, false><<<grid, kTcThreads, kTcSmemBytes, st>>>(ta, c.status);
    else if (forms == kFormKappa)
        k_fwd_tc<kFormKappa, false><<<grid, kTcThreads, kTcSmemBytes, st>>>(ta, c.status);
    else if (c.weighted)
        k_fwd_tc<kFormDirect, true><<<grid, kTcThreads, kTcSmemBytes, st>>>(ta, c.status);
    else
        k_fwd_tc<kFormDirect, false><<<grid, kTcThreads, kTcSmemBytes, st>>>(ta, c.status);
    e = cudaGetLastError();
    return e == cudaSuccess ? SDF_OK : cuda_error(e, "sdf_query: k_fwd_tc launch");
}

}  // namespace ptsdf
