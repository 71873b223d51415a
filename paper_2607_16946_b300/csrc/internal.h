// Internal declarations shared by the translation units of libptsdf.so.
// Not part of the public ABI (that is include/ptsdf.h).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>

#include "ptsdf.h"

namespace ptsdf {

// ---------------------------------------------------------------------------
// Packed cloud layout in HBM
// ---------------------------------------------------------------------------
// Every point becomes one 64-byte record (4 x float4) in one of two forms.
// Records are partitioned: all direct-form records first, padded to a whole
// tile, then all kappa-form records, padded to a whole tile.  A tile is
// kTileRecs records = kTileRecs * 64 bytes, the unit of one bulk (TMA) copy.
//
//  direct (radius) form, Eq. SingleTorusSDF with its centre and radii:
//    r0 = (p.x, p.y, p.z, sT)      sT = sign(T_i) = -sgn(kappa_max)
//    r1 = (c.x, c.y, c.z, R)
//    r2 = (u.x, u.y, u.z, -sT r)
//    r3 = 0
//  curvature (kappa) form, the same SDF rewritten around Q*(0,0) so that it
//  stays accurate when R or r is huge (near-flat points):
//    r0 = (p.x, p.y, p.z, 2 zeta)  zeta = -sgn(kappa_min)
//    r1 = (q.x, q.y, q.z, k)       q = Q*(0,0), k = |kappa_min|
//    r2 = (u.x, u.y, u.z, -kappa_max)
//    r3 = (2 zeta n*.x, 2 zeta n*.y, 2 zeta n*.z, 0)
// with sgn(0) := -1 (a zero curvature counts as convex).
//
// A second array holds, per point, float4(-2 p', |p'|^2) with
// p' = p - (bounding-box centre), for the d_max / d_min prepass.  It is
// ordered along a Morton (Z-order) curve of p and padded to kPreTile; every
// kSphereTile consecutive entries have a bounding sphere (centre p'_c,
// radius), used to skip tiles that cannot hold a query's farthest or nearest
// point.
// Tuning constants can be overridden at compile time (-DPTSDF_TILE_RECS=...,
// -DPTSDF_QPT=..., -DPTSDF_STAGES=...) to build variants for a sweep.
#ifndef PTSDF_TILE_RECS
#define PTSDF_TILE_RECS 32
#endif
#ifndef PTSDF_QPT
#define PTSDF_QPT 2
#endif
#ifndef PTSDF_STAGES
#define PTSDF_STAGES 4
#endif
#ifndef PTSDF_UNROLL
#define PTSDF_UNROLL 2
#endif
#ifndef PTSDF_TC_KAPPA
#define PTSDF_TC_KAPPA 1
#endif
#ifndef PTSDF_FWD_MINB
#define PTSDF_FWD_MINB 4
#endif
constexpr int kTileRecs = PTSDF_TILE_RECS;   // records per main-loop tile (32 x 64 B = 2 KB)
constexpr int kRecFloats = 16;
constexpr int kPreTile = 256;        // points per prepass tile (4 KB)
constexpr int kSphereTile = 64;      // points per bounding sphere of the pruned prepass
constexpr int kPlaneTile = 64;       // points per tile of the baselines' plane records (4 KB)

struct Cloud {
    int device = 0;
    int64_t n = 0;                   // points
    int64_t n_direct = 0, n_kappa = 0;
    int64_t n_kappa_flat = 0;        // kappa-form points with kappa_min = 0, first in the kappa segment
    bool weighted = false;           // built with per-point weights (record r3.w; 1 otherwise)
    int64_t tiles_direct = 0, tiles_kappa = 0;
    int64_t pre_tiles = 0;
    float aabb_diag = 0.f;
    float aabb[6] = {0, 0, 0, 0, 0, 0};
    float4* rec = nullptr;           // (tiles_direct + tiles_kappa) * kTileRecs * 4 float4
    float4* rec2 = nullptr;          // the same records pair-interleaved for the packed gradient loop
    float4* pre = nullptr;           // pre_tiles * kPreTile float4
    float4* spheres = nullptr;       // n_spheres x (centre', radius), then the group spheres (sphere_index.h)
    int64_t n_spheres = 0;
    int32_t* perm = nullptr;         // record slot -> original point index (-1 for padding)
    float* src_points = nullptr;     // copies of the inputs (N x 3, N x 3, N x 6), kept for
    float* src_normals = nullptr;    // the parameter gradient's chain through the fit
    float* src_params = nullptr;
    int32_t* status = nullptr;       // device status word (SDF_DEV_* bits)
    uint8_t* btiles = nullptr;       // (tiles_direct + tiles_kappa) x 14 KB split-f16 operands of the
                                     // tensor-core loop, both segments
    int32_t* btile_exact = nullptr;  // per tile: 1 when a coefficient leaves the f16 split's range
    float4* prec = nullptr;          // plane records of the baselines: per point (px,px,py,py) (pz,pz,A,A)
                                     // (nx,nx,ny,ny) (nz,nz,0,0), input order, plane_tiles x kPlaneTile points
    int64_t plane_tiles = 0;
    float4* mrec = nullptr;          // n x 4 float4 records in the prepass (Morton) order, r3.w = 1 for kappa
    int32_t* mperm = nullptr;        // input index of each Morton position
    float tc_scale = 1.f;            // their coordinate scale (a power of two >= the AABB diagonal)
    int num_sms = 148;
};

// thread-local error message
sdf_status set_error(sdf_status st, const std::string& msg);
sdf_status cuda_error(cudaError_t e, const char* what);
// the option checks every query-type entry point shares (api.cu); fn names the
// caller in the message
sdf_status check_opts(const sdf_query_opts& o, const char* fn);

// launch planning shared by the query kernels
struct Plan {
    int64_t q = 0;
    int64_t qblocks = 0;             // query blocks of the main kernel
    int64_t pre_qblocks = 0;         // query blocks of the prepass (kQueriesPerCta)
    int split = 1;                   // point chunks
    int64_t tiles_per_chunk = 0;     // main-loop tiles per chunk
    int64_t pre_tiles_per_chunk = 0; // prepass tiles per chunk
};

constexpr int kConsumerWarps = 8;
constexpr int kQueriesPerThread = PTSDF_QPT;
constexpr int kQueriesPerCta = kConsumerWarps * 32 * kQueriesPerThread;   // 512
constexpr int kStages = PTSDF_STAGES;
constexpr int kUnrollPts = PTSDF_UNROLL;      // points per unrolled step of the pair loop
constexpr int kFwdMinBlocks = PTSDF_FWD_MINB; // resident CTAs per SM the pair loop is compiled for

// queries_per_cta: queries one CTA of the main kernel holds (the prepass
// always uses kQueriesPerCta).
Plan make_plan(const Cloud& c, int64_t q, int split_override, int queries_per_cta = kQueriesPerCta);
void chunk_tiles(int64_t qblocks, int64_t tiles, int64_t target, int split_override, int64_t& tiles_per_chunk,
                 int& nchunks);
// whether sdf_query runs the direct-form tiles on the tensor cores, and how
// many (W, S) partial rows it then writes (1: none)
bool use_tensor_engine(const Cloud& c, const sdf_query_opts& o);
int query_partials(const Cloud& c, int64_t q, const sdf_query_opts& o);

// Brackets one kernel launch with CUDA events while sdf_profile is enabled.
class ProfRange {
  public:
    ProfRange(int kernel, cudaStream_t st);
    ~ProfRange();
    ProfRange(const ProfRange&) = delete;
    ProfRange& operator=(const ProfRange&) = delete;

  private:
    cudaStream_t st_;
    int idx_;
};

// kernels' host launchers (query.cu)
// tensor-core pair loop over the direct-form tiles (query_tc.cu)
struct TcQuery {
    const float* x = nullptr;      // Q x 3
    int64_t q = 0;
    float* phi = nullptr;          // written when direct_out
    float2* part = nullptr;        // else (W, S) at partial row part_base + chunk
    const float2* d2 = nullptr;    // pre_split x Q prepass partials
    float cx = 0.f, cy = 0.f, cz = 0.f;
    int pre_split = 1;
    int mode = SDF_LAMBDA_GLOBAL;
    float C = 64.f, lam = 0.f, offset = 0.f;
    int part_base = 0;
    int formula = SDF_FORMULA_BLEND;
};
sdf_status build_btiles(Cloud& c, cudaStream_t st);
// The tensor-core loop takes tiles [0, tc_tiles_end(c)): every tile, or
// (PTSDF_TC_KAPPA=0) the direct tiles and the whole kappa_min = 0 tiles,
// leaving the other kappa tiles to k_fwd; for a weighted cloud only the
// direct tiles.
int64_t tc_tiles_end(const Cloud& c);
// End of the whole kappa_min = 0 tiles that follow the direct segment
// (<= tc_tiles_end): the flat-formula instance takes [tiles_direct, that).
int64_t tc_flat_end(const Cloud& c);
int64_t tc_query_blocks(int64_t q);
// tiles [tiles_begin, tiles_end) of one segment (direct, or curvature form)
sdf_status launch_fwd_tc(const Cloud& c, const TcQuery& a, int64_t tiles_begin, int64_t tiles_end,
                         int64_t tiles_per_chunk, int nchunks, int direct_out, cudaStream_t st);

// radius-limited evaluation (radius.cu): the fallback neighbour count of Sec. 4.2
constexpr int kRadiusFallbackK = 32;
// the k (<= 64) nearest other points of every point, as input indices (n x k,
// input order), and the mean of their distances (D of the lambda heuristic)
sdf_status launch_knn_indices(const Cloud& c, int k, int32_t* d_idx, double* mean_dist, cudaStream_t st);
sdf_status launch_radius_query(const Cloud& c, const float* d_x, int64_t q, float* d_phi, const sdf_query_opts& o,
                               cudaStream_t st);

sdf_status launch_query(const Cloud& c, const float* d_x, int64_t q, float* d_phi,
                        const sdf_query_opts& o, cudaStream_t st);
// the two convolutional baselines, phi_SSPD and phi_SHC (baselines.cu)
sdf_status launch_plane_query(const Cloud& c, const float* d_x, int64_t q, float* d_phi, const sdf_query_opts& o,
                              cudaStream_t st);
sdf_status build_plane_records(Cloud& c, const float* d_weights, cudaStream_t st);
// grad.cu: the pair-interleaved records of the gradient loop (from c.rec)
sdf_status build_pair_records(Cloud& c, cudaStream_t st);
// trace.cu
sdf_status launch_trace(const Cloud& c, const float* d_org, const float* d_dir, int64_t nrays, int32_t max_steps,
                        float eps, float t_max, float* d_t_hit, int32_t* d_steps, float* d_normals,
                        const sdf_query_opts& o, cudaStream_t st);
// backward.cu
sdf_status launch_backward_params(const Cloud& c, int64_t q, const float* d_saved, const float* d_grad_phi,
                                  float* d_grad_params, const sdf_query_opts& o, cudaStream_t st);
// grad.cu
// d_lap non-null: also the Laplacian (and d_grad may be null)
sdf_status launch_query_grad(const Cloud& c, const float* d_x, int64_t q, float* d_phi, float* d_grad,
                             float* d_saved, const sdf_query_opts& o, cudaStream_t st, float* d_lap = nullptr);

}  // namespace ptsdf
