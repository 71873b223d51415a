// The paper's two convolutional baselines (Sec. 5, "Signed distance
// accuracy"), evaluated for every (query, point) pair on the blend's
// screening (lambda_x = C / sigma_x per query, or a fixed lambda):
//
//   phi_SSPD  Eq. SmoothedSignedPlanarDistance: the self-normalised blend of
//             the signed distances <x - p_i, n_i> to the points' tangent
//             planes, W = sum A_i w_i, S = sum A_i w_i <x - p_i, n_i>;
//   phi_SHC   Eq. ScreenedWindingNumber: the signed Hopf-Cole distance of the
//             screened double-layer sum, S = sum A_i w_i (lambda d_i + 1)
//             <x - p_i, n_i> / d_i^3 (2 pi times the paper's w with the d_min
//             shift), finished as sign(S) (d_min - ln(|S| / 2 pi) / lambda).
//
// with w_i = exp2(A0 - L d_i) = exp(-lambda (d_i - d_min)) as in the blend
// (every weight <= 1).  The same prepass gives d_max (lambda_x) and d_min.
//
// Geometry as the FP32-unit blend loop k_fwd: 8 consumer warps with 2 queries
// per lane and a producer warp streaming 4 KB tiles of 64 plane records
// through a 4-stage shared-memory ring by bulk copies.  A lane's two queries
// are held as pairs (x0, x1), ... and every product runs as one .f32x2
// instruction for both; each point's record stores its values twice,
// (px, px, py, py), (pz, pz, A, A), (nx, nx, ny, ny), (nz, nz, 0, 0), so a
// 128-bit shared-memory load yields ready pairs.  Per pair: SSPD 1 sqrt + 1
// exp2 on the special-function unit and 6.5 packed FP32 instructions; SHC
// 1 rsqrt + 1 exp2 and 9 (d = d^2 rsqrt(d^2), 1/d^3 = rsqrt(d^2)^3).
#include <cuda_runtime.h>

#include "query_common.cuh"
#include "prepass_warp.cuh"

namespace ptsdf {

using namespace qk;

namespace {

constexpr uint32_t kPlaneRecBytes = 4 * sizeof(float4);
constexpr uint32_t kPlaneTileBytes = kPlaneTile * kPlaneRecBytes;   // 4 KB
constexpr int kPlaneMinBlocks = 4;                                  // resident CTAs per SM
constexpr float kLn2 = 0.6931471805599453f;

// One plane record per point (input order), padded to whole tiles with zeros;
// the normal is normalised here (sdf_build has already refused zero and
// non-finite normals), A_i is the point's weight (1 without weights).
__global__ void k_plane_records(const float* __restrict__ P, const float* __restrict__ N,
                                const float* __restrict__ Wt, int64_t n, int64_t slots, float4* __restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= slots) return;
    float4 r0 = make_float4(0.f, 0.f, 0.f, 0.f), r1 = r0, r2 = r0, r3 = r0;
    if (i < n) {
        const float px = P[3 * i], py = P[3 * i + 1], pz = P[3 * i + 2];
        float nx = N[3 * i], ny = N[3 * i + 1], nz = N[3 * i + 2];
        const float inv = 1.f / sqrtf(nx * nx + ny * ny + nz * nz);
        nx *= inv;
        ny *= inv;
        nz *= inv;
        const float A = Wt ? Wt[i] : 1.f;
        r0 = make_float4(px, px, py, py);
        r1 = make_float4(pz, pz, A, A);
        r2 = make_float4(nx, nx, ny, ny);
        r3 = make_float4(nz, nz, 0.f, 0.f);
    }
    out[4 * i] = r0;
    out[4 * i + 1] = r1;
    out[4 * i + 2] = r2;
    out[4 * i + 3] = r3;
}

template <bool SHC, bool WEIGHTED>
__global__ void __launch_bounds__(kThreads, kPlaneMinBlocks)
    k_fwd_plane(const float4* __restrict__ prec, int64_t n, int64_t tiles_total, int64_t tiles_per_chunk,
                QueryArgs a, int32_t* status) {
    static_assert(kQueriesPerThread == 2, "a lane's two queries form the packed pairs");
    extern __shared__ __align__(128) char smem[];
    __shared__ TileRing<kStages> ring;
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int chunk = blockIdx.y;
    const int64_t t0 = (int64_t)chunk * tiles_per_chunk;
    const int64_t t1 = t0 + tiles_per_chunk < tiles_total ? t0 + tiles_per_chunk : tiles_total;
    const int64_t nt = t1 > t0 ? t1 - t0 : 0;
    if (threadIdx.x == 0) ring.init(kConsumerWarps);
    __syncthreads();
    if (warp == kConsumerWarps) {
        if (lane == 0)
            ring.produce(smem, reinterpret_cast<const char*>(prec) + (size_t)t0 * kPlaneTileBytes, nt,
                         kPlaneTileBytes, status);
        return;
    }
    int64_t qi[2];
    float xs[2][3], L[2], A0[2];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        qi[k] = (int64_t)blockIdx.x * kQueriesPerCta + k * (kConsumerWarps * 32) + threadIdx.x;
        const int64_t qq = qi[k] < a.q ? qi[k] : a.q - 1;
        xs[k][0] = a.x[3 * qq];
        xs[k][1] = a.x[3 * qq + 1];
        xs[k][2] = a.x[3 * qq + 2];
        query_screening(a.d2, a.pre_split, a.q, qq, a.mode, a.C, a.lam, L[k], A0[k]);
    }
    const f32x2 X = f2_pack(xs[0][0], xs[1][0]), Y = f2_pack(xs[0][1], xs[1][1]), Z = f2_pack(xs[0][2], xs[1][2]);
    const f32x2 NL = f2_pack(-L[0], -L[1]), A0v = f2_pack(A0[0], A0[1]);
    const f32x2 LAM = f2_pack(L[0] * kLn2, L[1] * kLn2), ONE = f2_pack(1.f, 1.f), ZERO = f2_pack(0.f, 0.f);
    f32x2 Wt = ZERO, St = ZERO;
    for (int64_t t = 0; t < nt; ++t) {
        if (!ring.wait_full(t, status)) return;
        const ulonglong2* tile = reinterpret_cast<const ulonglong2*>(smem + (size_t)(t % kStages) * kPlaneTileBytes);
        const int64_t first = (t0 + t) * kPlaneTile;
        const int cnt = (int)(n - first < kPlaneTile ? n - first : kPlaneTile);
        f32x2 w = ZERO, s = ZERO;
#pragma unroll 2
        for (int j = 0; j < cnt; ++j) {
            const ulonglong2 r0 = tile[4 * j], r1 = tile[4 * j + 1], r2 = tile[4 * j + 2], r3 = tile[4 * j + 3];
            const f32x2 DX = f2_sub(X, r0.x), DY = f2_sub(Y, r0.y), DZ = f2_sub(Z, r1.x);
            const f32x2 D2 = f2_fma(DZ, DZ, f2_fma(DY, DY, f2_mul(DX, DX)));
            const f32x2 G = f2_fma(DZ, r3.x, f2_fma(DY, r2.y, f2_mul(DX, r2.x)));   // <x - p, n>
            if (!SHC) {
                const f32x2 D = f2_pack(sqrt_mufu(f2_lo(D2)), sqrt_mufu(f2_hi(D2)));
                const f32x2 ARG = f2_fma(NL, D, A0v);
                f32x2 E = f2_pack(ex2_mufu(f2_lo(ARG)), ex2_mufu(f2_hi(ARG)));
                if (WEIGHTED) E = f2_mul(E, r1.y);
                w = f2_add(w, E);
                s = f2_fma(E, G, s);
            } else {
                // d = 0 (a point at the query) adds nothing: there G = 0 and
                // the clamp keeps 1/d^3 finite (1e36)
                const float d2l = fmaxf(f2_lo(D2), 1e-24f), d2h = fmaxf(f2_hi(D2), 1e-24f);
                const f32x2 R = f2_pack(rsqrt_mufu(d2l), rsqrt_mufu(d2h));
                const f32x2 D = f2_mul(f2_pack(d2l, d2h), R);
                const f32x2 ARG = f2_fma(NL, D, A0v);
                f32x2 E = f2_pack(ex2_mufu(f2_lo(ARG)), ex2_mufu(f2_hi(ARG)));
                if (WEIGHTED) E = f2_mul(E, r1.y);
                const f32x2 K = f2_fma(LAM, D, ONE);                  // lambda d + 1
                const f32x2 R3 = f2_mul(f2_mul(R, R), R);              // 1 / d^3
                s = f2_fma(f2_mul(f2_mul(E, K), G), R3, s);
            }
        }
        // blocked summation, as in k_fwd
        Wt = f2_add(Wt, w);
        St = f2_add(St, s);
        ring.release(t, lane);
    }
    const float Wq[2] = {f2_lo(Wt), f2_hi(Wt)}, Sq[2] = {f2_lo(St), f2_hi(St)};
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        if (qi[k] >= a.q) continue;
        if (a.split == 1)
            a.phi[qi[k]] = finish_sums(Wq[k], Sq[k], a.formula, L[k], A0[k], a.offset);
        else
            a.part[(size_t)(a.part_base + chunk) * a.q + qi[k]] = make_float2(Wq[k], Sq[k]);
    }
}

using PlaneKernel = decltype(&k_fwd_plane<false, false>);

PlaneKernel plane_kernel(bool shc, bool weighted) {
    if (shc) return weighted ? k_fwd_plane<true, true> : k_fwd_plane<true, false>;
    return weighted ? k_fwd_plane<false, true> : k_fwd_plane<false, false>;
}

}  // namespace

sdf_status build_plane_records(Cloud& c, const float* d_weights, cudaStream_t st) {
    c.plane_tiles = (c.n + kPlaneTile - 1) / kPlaneTile;
    const int64_t slots = c.plane_tiles * kPlaneTile;
    cudaError_t e = cudaMalloc(&c.prec, (size_t)slots * kPlaneRecBytes);
    if (e != cudaSuccess)
        return e == cudaErrorMemoryAllocation ? set_error(SDF_ENOMEM, "sdf_build: plane records")
                                              : cuda_error(e, "sdf_build: plane records");
    k_plane_records<<<(unsigned)((slots + 255) / 256), 256, 0, st>>>(c.src_points, c.src_normals, d_weights, c.n,
                                                                     slots, c.prec);
    e = cudaGetLastError();
    return e == cudaSuccess ? SDF_OK : cuda_error(e, "sdf_build: k_plane_records");
}

sdf_status launch_plane_query(const Cloud& c, const float* d_x, int64_t q, float* d_phi, const sdf_query_opts& o,
                              cudaStream_t st) {
    Plan p = make_plan(c, q, o.split_n);
    // point chunks over the plane tiles: at least two waves of the resident CTAs
    chunk_tiles(p.qblocks, c.plane_tiles, 2LL * kPlaneMinBlocks * c.num_sms, o.split_n, p.tiles_per_chunk, p.split);
    p.pre_tiles_per_chunk = (c.pre_tiles + p.split - 1) / p.split;
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
    a.part = nullptr;
    a.d2 = nullptr;
    a.far = nullptr;
    a.cx = 0.5f * (c.aabb[0] + c.aabb[3]);
    a.cy = 0.5f * (c.aabb[1] + c.aabb[4]);
    a.cz = 0.5f * (c.aabb[2] + c.aabb[5]);
    a.cloud_radius = 0.5f * c.aabb_diag * (1.f + 1e-6f);
    const bool warp_pre = use_warp_prepass(c, p, o), pruned = !warp_pre && use_pruned_prepass(c, p, o);
    a.pre_split = pruned || warp_pre ? 1 : p.split;
    cudaError_t e = cudaMallocAsync(&a.d2, (size_t)a.pre_split * q * sizeof(float2), st);
    if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? set_error(SDF_ENOMEM, "sdf_query: scratch")
                                                                : cuda_error(e, "sdf_query: scratch");
    if (p.split > 1) {
        e = cudaMallocAsync(&a.part, (size_t)p.split * q * sizeof(float2), st);
        if (e != cudaSuccess) {
            cudaFreeAsync(a.d2, st);
            return e == cudaErrorMemoryAllocation ? set_error(SDF_ENOMEM, "sdf_query: scratch")
                                                  : cuda_error(e, "sdf_query: scratch");
        }
    }
    {
        ProfRange pr(SDF_K_PREPASS, st);
        const dim3 pre_grid((unsigned)p.pre_qblocks, (unsigned)p.split);
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
    if (e == cudaSuccess) {
        ProfRange pr(SDF_K_PLANE, st);
        plane_kernel(o.formula == SDF_FORMULA_SHC, c.weighted)<<<dim3((unsigned)p.qblocks, (unsigned)p.split),
                                                                  kThreads, kStages * kPlaneTileBytes, st>>>(
            c.prec, c.n, c.plane_tiles, p.tiles_per_chunk, a, c.status);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && p.split > 1) {
        ProfRange pr(SDF_K_MERGE, st);
        k_merge<<<(unsigned)((q + 255) / 256), 256, 0, st>>>(a);
        e = cudaGetLastError();
    }
    cudaFreeAsync(a.d2, st);
    if (a.part) cudaFreeAsync(a.part, st);
    return e == cudaSuccess ? SDF_OK : cuda_error(e, "sdf_query: plane-baseline launch");
}

}  // namespace ptsdf
