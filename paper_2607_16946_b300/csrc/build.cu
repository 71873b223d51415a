// sdf_build: one torus per point from six coefficients (Sec. 4.1, App. C),
// packed into the two record forms of the query kernels.
//
//   1. k_aabb       one CTA: axis-aligned bounding box of the points.
//   2. k_fit        one thread per point, double precision: frame, fundamental
//                   forms, curvatures, principal direction, n*, Q*(0,0), axis,
//                   sign, and the record in the direct or the kappa form.
//   3. k_partition  one CTA: stable partition of the records into the two
//                   segments, each padded to whole tiles; the prepass array
//                   and the slot -> point permutation.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <utility>
#include <vector>

#include "device_common.cuh"
#include "fit_math.cuh"
#include "sphere_index.h"
#include "internal.h"

namespace ptsdf {

namespace {

constexpr int kAabbThreads = 1024;
constexpr int kPartThreads = 1024;

__global__ void k_aabb(const float* __restrict__ pts, int64_t n, float* __restrict__ box) {
    __shared__ float red[6][kAabbThreads / 32];
    float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        for (int k = 0; k < 3; ++k) {
            const float v = pts[3 * i + k];
            lo[k] = fminf(lo[k], v);
            hi[k] = fmaxf(hi[k], v);
        }
    }
    for (int off = 16; off > 0; off >>= 1) {
        for (int k = 0; k < 3; ++k) {
            lo[k] = fminf(lo[k], __shfl_xor_sync(0xffffffffu, lo[k], off));
            hi[k] = fmaxf(hi[k], __shfl_xor_sync(0xffffffffu, hi[k], off));
        }
    }
    const int w = threadIdx.x / 32, lane = threadIdx.x % 32;
    if (lane == 0) {
        for (int k = 0; k < 3; ++k) {
            red[k][w] = lo[k];
            red[3 + k][w] = hi[k];
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 0; k < 3; ++k) {
            float a = INFINITY, b = -INFINITY;
            for (int j = 0; j < (int)(blockDim.x / 32); ++j) {
                a = fminf(a, red[k][j]);
                b = fmaxf(b, red[3 + k][j]);
            }
            box[k] = a;
            box[3 + k] = b;
        }
    }
}

// One point: returns the record (16 floats) and its kind (0 direct, 1 kappa,
// 2 kappa with kappa_min = 0); sets *bad for a zero / non-finite normal,
// non-finite input or a weight outside [2^-64, 2^64].  Both record forms
// carry the point's weight A_i in their last float (1 without weights),
// which the pair loops multiply onto w_i.
__global__ void k_fit(const float* __restrict__ P, const float* __restrict__ Nrm, const float* __restrict__ A6,
                      const float* __restrict__ Wt, int64_t n, double thr, float* __restrict__ rec_tmp,
                      int8_t* __restrict__ kind, int32_t* __restrict__ status) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double p[3], nv[3], a[6];
    bool finite = true;
    for (int k = 0; k < 3; ++k) {
        p[k] = P[3 * i + k];
        nv[k] = Nrm[3 * i + k];
        finite = finite && isfinite(p[k]) && isfinite(nv[k]);
    }
    for (int k = 0; k < 6; ++k) {
        a[k] = A6[6 * i + k];
        finite = finite && isfinite(a[k]);
    }
    float wa = 1.f;
    if (Wt) {
        wa = Wt[i];
        finite = finite && wa >= 0x1p-64f && wa <= 0x1p64f;   // keeps every sum inside FP32's range
    }
    const double len = sqrt(nv[0] * nv[0] + nv[1] * nv[1] + nv[2] * nv[2]);
    float* out = rec_tmp + (size_t)i * kRecFloats;
    if (!finite || !(len > 0.0) || !isfinite(len)) {
        atomicOr(status, (int32_t)SDF_DEV_BAD_INPUT);
        for (int k = 0; k < kRecFloats; ++k) out[k] = 0.f;
        kind[i] = 0;
        return;
    }
    for (int k = 0; k < 3; ++k) nv[k] /= len;
    FitPoint<double> f;
    fit_point<double>(p, nv, a, f);
    const double kmin = f.kmin, kmax = f.kmax;
    const double* q = f.q;
    const double* nstar = f.nstar;
    const double* u = f.u;

    const double sT = -sgn_convex(kmax);          // Eq. TorusSigns
    const bool direct = (kmin != 0.0) && (1.0 / fabs(kmin) <= thr) && (1.0 / fabs(kmax) <= thr);
    if (direct) {
        const double r = 1.0 / fabs(kmax);
        const double R = 1.0 / fabs(kmin) - sgn_convex(kmin) * sgn_convex(kmax) * r;
        double c[3];
        for (int k = 0; k < 3; ++k) c[k] = q[k] + nstar[k] / kmin;   // signed kappa_min
        out[0] = (float)p[0]; out[1] = (float)p[1]; out[2] = (float)p[2]; out[3] = (float)sT;
        out[4] = (float)c[0]; out[5] = (float)c[1]; out[6] = (float)c[2]; out[7] = (float)R;
        out[8] = (float)u[0]; out[9] = (float)u[1]; out[10] = (float)u[2]; out[11] = (float)(-sT * r);
        out[12] = 0.f; out[13] = 0.f; out[14] = 0.f; out[15] = wa;
        kind[i] = 0;
    } else {
        const double zeta = -sgn_convex(kmin);
        out[0] = (float)p[0]; out[1] = (float)p[1]; out[2] = (float)p[2]; out[3] = (float)(2.0 * zeta);
        out[4] = (float)q[0]; out[5] = (float)q[1]; out[6] = (float)q[2]; out[7] = (float)fabs(kmin);
        out[8] = (float)u[0]; out[9] = (float)u[1]; out[10] = (float)u[2]; out[11] = (float)(-kmax);
        out[12] = (float)(2.0 * zeta * nstar[0]); out[13] = (float)(2.0 * zeta * nstar[1]);
        out[14] = (float)(2.0 * zeta * nstar[2]); out[15] = wa;
        kind[i] = out[7] == 0.f ? 2 : 1;   // 2: kappa_min = 0 (cylinders, planes): the shorter formula
    }
}

// Block-wide exclusive scan of one int per thread; returns the prefix and
// writes the block total to *total.
__device__ int block_exclusive_scan(int v, int* warp_sums, int* total) {
    const int lane = threadIdx.x % 32, w = threadIdx.x / 32, nw = blockDim.x / 32;
    int x = v;
    for (int off = 1; off < 32; off <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, off);
        if (lane >= off) x += y;
    }
    if (lane == 31) warp_sums[w] = x;
    __syncthreads();
    if (w == 0) {
        int s = lane < nw ? warp_sums[lane] : 0;
        for (int off = 1; off < 32; off <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, s, off);
            if (lane >= off) s += y;
        }
        if (lane < nw) warp_sums[lane] = s;   // inclusive over warps
    }
    __syncthreads();
    const int base = w > 0 ? warp_sums[w - 1] : 0;
    *total = warp_sums[nw - 1];
    __syncthreads();
    return base + x - v;
}

// counts[0] direct, counts[1] kappa form, counts[2] of those with kappa_min = 0
__global__ void k_count(const int8_t* __restrict__ kind, int64_t n, int64_t* __restrict__ counts) {
    __shared__ int ws[32];
    int64_t nk = 0, nf = 0;
    for (int64_t base = 0; base < n; base += blockDim.x) {
        const int64_t i = base + threadIdx.x;
        int tot;
        block_exclusive_scan((i < n && kind[i]) ? 1 : 0, ws, &tot);
        nk += tot;
        block_exclusive_scan((i < n && kind[i] == 2) ? 1 : 0, ws, &tot);
        nf += tot;
    }
    if (threadIdx.x == 0) {
        counts[0] = n - nk;
        counts[1] = nk;
        counts[2] = nf;
    }
}

// Order of the records: direct form | kappa form with kappa_min = 0 |
// the other kappa-form records, each in input order.
__global__ void k_partition(const float4* __restrict__ rec_tmp, const int8_t* __restrict__ kind,
                            const float* __restrict__ P, int64_t n, int64_t n_direct, int64_t n_flat,
                            int64_t tiles_direct, float cx, float cy, float cz, float4* __restrict__ rec,
                            float4* __restrict__ pre, int32_t* __restrict__ perm) {
    __shared__ int ws[32];
    int64_t pos_d = 0, pos_f = 0, pos_k = 0;
    for (int64_t base = 0; base < n; base += blockDim.x) {
        const int64_t i = base + threadIdx.x;
        const bool valid = i < n;
        const int kd = valid ? (int)kind[i] : 0;
        int tot_k, tot_d, tot_f;
        const int ek = block_exclusive_scan(valid && kd == 1 ? 1 : 0, ws, &tot_k);
        const int ef = block_exclusive_scan(valid && kd == 2 ? 1 : 0, ws, &tot_f);
        const int ed = block_exclusive_scan(valid && kd == 0 ? 1 : 0, ws, &tot_d);
        const int isk = kd != 0;
        if (valid) {
            const int64_t kpos = kd == 2 ? pos_f + ef : n_flat + pos_k + ek;   // within the kappa segment
            const int64_t slot = isk ? tiles_direct * kTileRecs + kpos : pos_d + ed;
            const int64_t cpos = isk ? n_direct + kpos : pos_d + ed;
            for (int k = 0; k < 4; ++k) rec[slot * 4 + k] = rec_tmp[i * 4 + k];
            perm[slot] = (int32_t)i;
            const float px = P[3 * i] - cx, py = P[3 * i + 1] - cy, pz = P[3 * i + 2] - cz;
            pre[cpos] = make_float4(-2.f * px, -2.f * py, -2.f * pz, px * px + py * py + pz * pz);
        }
        pos_d += tot_d;
        pos_f += tot_f;
        pos_k += tot_k;
    }
}

// Records in the Morton order of the prepass array (compact position order[m]:
// direct points first, then kappa-form ones), for the radius-limited
// evaluation and the k-nearest searches.  The form is read back from r0.w:
// sT = +-1 in the direct form, 2 zeta = +-2 in the kappa form.
__global__ void k_gather_morton(const float4* __restrict__ rec, const int32_t* __restrict__ order,
                                const int32_t* __restrict__ perm, int64_t n, int64_t n_direct, int64_t tiles_direct,
                                float4* __restrict__ mrec, int32_t* __restrict__ mperm) {
    const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= n) return;
    const int64_t cpos = order[m];
    const bool kappa = cpos >= n_direct;
    const int64_t slot = kappa ? tiles_direct * kTileRecs + (cpos - n_direct) : cpos;
    for (int k = 0; k < 4; ++k) mrec[4 * m + k] = rec[4 * slot + k];
    mperm[m] = perm[slot];
}

__global__ void k_fill_perm(int32_t* perm, int64_t m) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < m) perm[i] = -1;
}

}  // namespace

}  // namespace ptsdf

using namespace ptsdf;

namespace {

// Spreads the low 10 bits of v to every third bit.
uint32_t spread3(uint32_t v) {
    v &= 0x3ffu;
    v = (v | (v << 16)) & 0x030000ffu;
    v = (v | (v << 8)) & 0x0300f00fu;
    v = (v | (v << 4)) & 0x030c30c3u;
    v = (v | (v << 2)) & 0x09249249u;
    return v;
}

// Orders the prepass entries (-2 p', |p'|^2) along a 30-bit Morton curve of p'
// and returns one bounding sphere (centre p'_c, radius) per kSphereTile
// consecutive entries, followed by one group sphere per kGroupSpheres
// consecutive spheres.  Radii are inflated by 1e-5 of the AABB diagonal plus a
// relative 1e-6 so that FP32 rounding of the query-to-centre distance never
// excludes a tile that holds an extreme point.
void morton_order_and_spheres(const std::vector<float4>& in, const float* box, float diag,
                              std::vector<float4>& out, std::vector<float4>& spheres,
                              std::vector<int32_t>& order) {
    const size_t n = in.size();
    const double half[3] = {0.5 * (box[3] - box[0]), 0.5 * (box[4] - box[1]), 0.5 * (box[5] - box[2])};
    std::vector<std::pair<uint32_t, uint32_t>> key(n);
    for (size_t i = 0; i < n; ++i) {
        const double p[3] = {-0.5 * in[i].x, -0.5 * in[i].y, -0.5 * in[i].z};
        uint32_t cell[3];
        for (int k = 0; k < 3; ++k) {
            const double u = half[k] > 0.0 ? (p[k] + half[k]) / (2.0 * half[k]) : 0.5;
            const double cl = u < 0.0 ? 0.0 : (u > 1.0 ? 1.0 : u);
            cell[k] = (uint32_t)(cl * 1023.0);
        }
        key[i] = {spread3(cell[0]) | (spread3(cell[1]) << 1) | (spread3(cell[2]) << 2), (uint32_t)i};
    }
    std::sort(key.begin(), key.end());
    out.resize(n);
    order.resize(n);
    for (size_t i = 0; i < n; ++i) {
        out[i] = in[key[i].second];
        order[i] = (int32_t)key[i].second;
    }
    const size_t ns = (n + kSphereTile - 1) / kSphereTile;
    spheres.resize(ns);
    for (size_t t = 0; t < ns; ++t) {
        const size_t a = t * kSphereTile, b = std::min(n, a + kSphereTile);
        double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
        for (size_t i = a; i < b; ++i) {
            const double p[3] = {-0.5 * out[i].x, -0.5 * out[i].y, -0.5 * out[i].z};
            for (int k = 0; k < 3; ++k) {
                lo[k] = std::min(lo[k], p[k]);
                hi[k] = std::max(hi[k], p[k]);
            }
        }
        const double cc[3] = {0.5 * (lo[0] + hi[0]), 0.5 * (lo[1] + hi[1]), 0.5 * (lo[2] + hi[2])};
        double r2 = 0.0, cn = 0.0;
        for (size_t i = a; i < b; ++i) {
            const double p[3] = {-0.5 * out[i].x, -0.5 * out[i].y, -0.5 * out[i].z};
            const double d2 = (p[0] - cc[0]) * (p[0] - cc[0]) + (p[1] - cc[1]) * (p[1] - cc[1]) +
                              (p[2] - cc[2]) * (p[2] - cc[2]);
            r2 = std::max(r2, d2);
        }
        cn = std::sqrt(cc[0] * cc[0] + cc[1] * cc[1] + cc[2] * cc[2]);
        const double r = std::sqrt(r2) + 1e-5 * diag + 1e-6 * (cn + diag);
        spheres[t] = make_float4((float)cc[0], (float)cc[1], (float)cc[2], (float)r);
    }
    // Group spheres, from the FP32 centres and radii the kernels read: centre
    // of the members' boxes (rounded to FP32 first), radius max |c_t - C| + r_t
    // in double, inflated by a relative 1e-5 (the FP32 rounding of the radius
    // and of both centre distances a kernel compares) and 1e-6 of |C| + diag.
    const size_t ng = (size_t)group_count((int64_t)ns);
    spheres.resize(ns + ng);
    for (size_t g = 0; g < ng; ++g) {
        const size_t a = g * kGroupSpheres, b = std::min(ns, a + kGroupSpheres);
        double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
        for (size_t t = a; t < b; ++t) {
            const float4 s = spheres[t];
            const double c[3] = {s.x, s.y, s.z};
            for (int k = 0; k < 3; ++k) {
                lo[k] = std::min(lo[k], c[k] - s.w);
                hi[k] = std::max(hi[k], c[k] + s.w);
            }
        }
        const float cf[3] = {(float)(0.5 * (lo[0] + hi[0])), (float)(0.5 * (lo[1] + hi[1])),
                             (float)(0.5 * (lo[2] + hi[2]))};
        double rg = 0.0;
        for (size_t t = a; t < b; ++t) {
            const float4 s = spheres[t];
            const double dx = (double)s.x - cf[0], dy = (double)s.y - cf[1], dz = (double)s.z - cf[2];
            rg = std::max(rg, std::sqrt(dx * dx + dy * dy + dz * dz) + (double)s.w);
        }
        const double cn = std::sqrt((double)cf[0] * cf[0] + (double)cf[1] * cf[1] + (double)cf[2] * cf[2]);
        spheres[ns + g] = make_float4(cf[0], cf[1], cf[2], (float)(rg * (1.0 + 1e-5) + 1e-6 * (cn + diag)));
    }
}

void free_cloud(Cloud* c) {
    if (!c) return;
    cudaFree(c->rec);
    cudaFree(c->pre);
    cudaFree(c->spheres);
    cudaFree(c->perm);
    cudaFree(c->src_points);
    cudaFree(c->src_normals);
    cudaFree(c->src_params);
    cudaFree(c->status);
    cudaFree(c->btiles);
    cudaFree(c->btile_exact);
    cudaFree(c->mrec);
    cudaFree(c->mperm);
    cudaFree(c->prec);
    cudaFree(c->rec2);
    delete c;
}

// The build from device inputs.  d_rec_in / d_kind_in (n x 16 floats and n
// kinds, input order, as k_fit writes them): the fitted records of an
// export, used instead of fitting again; NULL: fit.
sdf_status build_impl(const float* d_points, const float* d_normals, const float* d_params, const float* d_weights,
                      int64_t n, cudaStream_t st, sdf_cloud* out, const float* d_rec_in, const int8_t* d_kind_in) {
    Cloud* c = new Cloud();
    c->n = n;
    c->weighted = d_weights != nullptr;
    cudaError_t e = cudaGetDevice(&c->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device);
    if (e != cudaSuccess) {
        delete c;
        return cuda_error(e, "sdf_build: device query");
    }
    float* box = nullptr;
    float* rec_tmp = nullptr;
    int8_t* kind = nullptr;
    int64_t* counts = nullptr;
    auto fail = [&](cudaError_t err, const char* what) {
        cudaStreamSynchronize(st);
        cudaFree(box);
        cudaFree(rec_tmp);
        cudaFree(kind);
        cudaFree(counts);
        free_cloud(c);
        return err == cudaErrorMemoryAllocation ? set_error(SDF_ENOMEM, what) : cuda_error(err, what);
    };
#define PTSDF_TRY(call, what)                  \
    do {                                       \
        cudaError_t _e = (call);               \
        if (_e != cudaSuccess) return fail(_e, what); \
    } while (0)
    PTSDF_TRY(cudaMalloc(&c->status, sizeof(int32_t)), "sdf_build: status alloc");
    PTSDF_TRY(cudaMemsetAsync(c->status, 0, sizeof(int32_t), st), "sdf_build: status init");
    PTSDF_TRY(cudaMalloc(&box, 6 * sizeof(float)), "sdf_build: box alloc");
    PTSDF_TRY(cudaMalloc(&rec_tmp, (size_t)n * kRecFloats * sizeof(float)), "sdf_build: temp alloc");
    PTSDF_TRY(cudaMalloc(&kind, (size_t)n), "sdf_build: temp alloc");
    PTSDF_TRY(cudaMalloc(&counts, 3 * sizeof(int64_t)), "sdf_build: temp alloc");
    PTSDF_TRY(cudaMalloc(&c->src_points, (size_t)n * 3 * sizeof(float)), "sdf_build: copy alloc");
    PTSDF_TRY(cudaMalloc(&c->src_normals, (size_t)n * 3 * sizeof(float)), "sdf_build: copy alloc");
    PTSDF_TRY(cudaMalloc(&c->src_params, (size_t)n * 6 * sizeof(float)), "sdf_build: copy alloc");
    PTSDF_TRY(cudaMemcpyAsync(c->src_points, d_points, (size_t)n * 3 * sizeof(float), cudaMemcpyDeviceToDevice, st),
              "sdf_build: copy points");
    PTSDF_TRY(cudaMemcpyAsync(c->src_normals, d_normals, (size_t)n * 3 * sizeof(float), cudaMemcpyDeviceToDevice, st),
              "sdf_build: copy normals");
    PTSDF_TRY(cudaMemcpyAsync(c->src_params, d_params, (size_t)n * 6 * sizeof(float), cudaMemcpyDeviceToDevice, st),
              "sdf_build: copy params");

    k_aabb<<<1, kAabbThreads, 0, st>>>(c->src_points, n, box);
    PTSDF_TRY(cudaGetLastError(), "sdf_build: k_aabb launch");
    PTSDF_TRY(cudaMemcpyAsync(c->aabb, box, 6 * sizeof(float), cudaMemcpyDeviceToHost, st), "sdf_build: box copy");
    PTSDF_TRY(cudaStreamSynchronize(st), "sdf_build: sync");
    const double dx = c->aabb[3] - c->aabb[0], dy = c->aabb[4] - c->aabb[1], dz = c->aabb[5] - c->aabb[2];
    c->aabb_diag = (float)std::sqrt(dx * dx + dy * dy + dz * dz);
    // radii up to 8 AABB diagonals keep the direct form's FP32 cancellation
    // (about 3 ulp of the radius) below 1e-5 of the diagonal; larger ones, and
    // zero curvatures, use the kappa form
    const double thr = 8.0 * std::fmax((double)c->aabb_diag, 1e-6);

    if (d_rec_in) {
        PTSDF_TRY(cudaMemcpyAsync(rec_tmp, d_rec_in, (size_t)n * kRecFloats * sizeof(float), cudaMemcpyDeviceToDevice,
                                  st),
                  "sdf_import: records");
        PTSDF_TRY(cudaMemcpyAsync(kind, d_kind_in, (size_t)n, cudaMemcpyDeviceToDevice, st), "sdf_import: kinds");
    } else {
        const int fit_threads = 128;
        k_fit<<<(unsigned)((n + fit_threads - 1) / fit_threads), fit_threads, 0, st>>>(
            c->src_points, c->src_normals, c->src_params, d_weights, n, thr, rec_tmp, kind, c->status);
        PTSDF_TRY(cudaGetLastError(), "sdf_build: k_fit launch");
    }
    k_count<<<1, kPartThreads, 0, st>>>(kind, n, counts);
    PTSDF_TRY(cudaGetLastError(), "sdf_build: k_count launch");
    int64_t hcounts[3];
    int32_t hstatus = 0;
    PTSDF_TRY(cudaMemcpyAsync(hcounts, counts, sizeof(hcounts), cudaMemcpyDeviceToHost, st), "sdf_build: counts");
    PTSDF_TRY(cudaMemcpyAsync(&hstatus, c->status, sizeof(int32_t), cudaMemcpyDeviceToHost, st), "sdf_build: status");
    PTSDF_TRY(cudaStreamSynchronize(st), "sdf_build: sync");
    if (hstatus & SDF_DEV_BAD_INPUT) {
        fail(cudaSuccess, "");
        return set_error(SDF_EINVAL, "sdf_build: zero or non-finite normal, non-finite point / coefficient, or a "
                                     "weight outside [2^-64, 2^64]");
    }
    c->n_direct = hcounts[0];
    c->n_kappa_flat = hcounts[2];
    c->n_kappa = hcounts[1];
    c->tiles_direct = (c->n_direct + kTileRecs - 1) / kTileRecs;
    c->tiles_kappa = (c->n_kappa + kTileRecs - 1) / kTileRecs;
    c->pre_tiles = (n + kPreTile - 1) / kPreTile;
    const int64_t slots = (c->tiles_direct + c->tiles_kappa) * kTileRecs;
    PTSDF_TRY(cudaMalloc(&c->rec, (size_t)slots * 4 * sizeof(float4)), "sdf_build: record alloc");
    PTSDF_TRY(cudaMemsetAsync(c->rec, 0, (size_t)slots * 4 * sizeof(float4), st), "sdf_build: record init");
    PTSDF_TRY(cudaMalloc(&c->pre, (size_t)c->pre_tiles * kPreTile * sizeof(float4)), "sdf_build: prepass alloc");
    PTSDF_TRY(cudaMemsetAsync(c->pre, 0, (size_t)c->pre_tiles * kPreTile * sizeof(float4), st),
              "sdf_build: prepass init");
    PTSDF_TRY(cudaMalloc(&c->perm, (size_t)slots * sizeof(int32_t)), "sdf_build: perm alloc");
    k_fill_perm<<<(unsigned)((slots + 255) / 256), 256, 0, st>>>(c->perm, slots);
    PTSDF_TRY(cudaGetLastError(), "sdf_build: k_fill_perm launch");
    k_partition<<<1, kPartThreads, 0, st>>>(reinterpret_cast<const float4*>(rec_tmp), kind, c->src_points, n,
                                            c->n_direct, c->n_kappa_flat, c->tiles_direct,
                                            0.5f * (c->aabb[0] + c->aabb[3]),
                                            0.5f * (c->aabb[1] + c->aabb[4]), 0.5f * (c->aabb[2] + c->aabb[5]),
                                            c->rec, c->pre, c->perm);
    PTSDF_TRY(cudaGetLastError(), "sdf_build: k_partition launch");
    {
        sdf_status bs = build_btiles(*c, st);
        if (bs == SDF_OK) bs = build_plane_records(*c, d_weights, st);   // the SSPD / SHC baselines
        if (bs == SDF_OK) bs = build_pair_records(*c, st);               // the packed gradient loop
        if (bs != SDF_OK) {
            const std::string msg = sdf_last_error();
            fail(cudaSuccess, "");
            return set_error(bs, msg);
        }
    }
    PTSDF_TRY(cudaStreamSynchronize(st), "sdf_build: sync");
    {
        // Morton order of the prepass array and one bounding sphere per
        // kSphereTile points (host side: O(N log N) once per cloud)
        std::vector<float4> hp((size_t)n);
        PTSDF_TRY(cudaMemcpy(hp.data(), c->pre, (size_t)n * sizeof(float4), cudaMemcpyDeviceToHost),
                  "sdf_build: prepass download");
        std::vector<float4> sorted;
        std::vector<float4> spheres;
        std::vector<int32_t> order;
        morton_order_and_spheres(hp, c->aabb, c->aabb_diag, sorted, spheres, order);
        c->n_spheres = (n + kSphereTile - 1) / kSphereTile;   // the group spheres follow them
        PTSDF_TRY(cudaMemcpy(c->pre, sorted.data(), (size_t)n * sizeof(float4), cudaMemcpyHostToDevice),
                  "sdf_build: prepass upload");
        PTSDF_TRY(cudaMalloc(&c->spheres, spheres.size() * sizeof(float4)), "sdf_build: sphere alloc");
        PTSDF_TRY(cudaMemcpy(c->spheres, spheres.data(), spheres.size() * sizeof(float4), cudaMemcpyHostToDevice),
                  "sdf_build: sphere upload");
        int32_t* d_order = nullptr;
        PTSDF_TRY(cudaMalloc(&d_order, (size_t)n * sizeof(int32_t)), "sdf_build: order alloc");
        cudaError_t oe = cudaMemcpy(d_order, order.data(), (size_t)n * sizeof(int32_t), cudaMemcpyHostToDevice);
        if (oe == cudaSuccess) oe = cudaMalloc(&c->mrec, (size_t)n * 4 * sizeof(float4));
        if (oe == cudaSuccess) oe = cudaMalloc(&c->mperm, (size_t)n * sizeof(int32_t));
        if (oe == cudaSuccess) {
            k_gather_morton<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(c->rec, d_order, c->perm, n, c->n_direct,
                                                                       c->tiles_direct, c->mrec, c->mperm);
            oe = cudaGetLastError();
        }
        if (oe == cudaSuccess) oe = cudaStreamSynchronize(st);
        cudaFree(d_order);
        PTSDF_TRY(oe, "sdf_build: Morton-ordered records");
    }
#undef PTSDF_TRY
    cudaFree(box);
    cudaFree(rec_tmp);
    cudaFree(kind);
    cudaFree(counts);
    *out = reinterpret_cast<sdf_cloud>(c);
    return SDF_OK;
}

// Checkpoint layout (host byte order): the header, then the points (n x 3),
// normals (n x 3), coefficients (n x 6) and, for a weighted cloud, weights (n)
// as float; the fitted records (n x 16 float, input order) and their kinds
// (n bytes).
struct ExportHeader {
    char magic[8];        // "PTSDFCK\0"
    uint32_t version;     // 1
    uint32_t weighted;    // 0 or 1
    int64_t n;
};
constexpr char kExportMagic[8] = {'P', 'T', 'S', 'D', 'F', 'C', 'K', 0};

int64_t export_bytes(int64_t n, bool weighted) {
    return (int64_t)sizeof(ExportHeader) + n * (int64_t)((12 + (weighted ? 1 : 0) + kRecFloats) * sizeof(float)) + n;
}

}  // namespace

extern "C" sdf_status sdf_build(const float* d_points, const float* d_normals, const float* d_params, int64_t n,
                                void* stream, sdf_cloud* out) {
    return sdf_build_weighted(d_points, d_normals, d_params, nullptr, n, stream, out);
}

extern "C" sdf_status sdf_build_weighted(const float* d_points, const float* d_normals, const float* d_params,
                                         const float* d_weights, int64_t n, void* stream, sdf_cloud* out) {
    if (!out) return set_error(SDF_EINVAL, "sdf_build: out is NULL");
    *out = nullptr;
    if (n < 1 || n > 0x7fffffffLL) return set_error(SDF_EINVAL, "sdf_build: n must be in [1, 2^31-1]");
    if (!d_points || !d_normals || !d_params) return set_error(SDF_EINVAL, "sdf_build: NULL input pointer");
    return build_impl(d_points, d_normals, d_params, d_weights, n, static_cast<cudaStream_t>(stream), out, nullptr,
                      nullptr);
}

extern "C" sdf_status sdf_export(sdf_cloud cloud, void* buf, int64_t cap, int64_t* size) {
    if (!cloud || !size) return set_error(SDF_EINVAL, "sdf_export: cloud or size is NULL");
    const Cloud* c = reinterpret_cast<const Cloud*>(cloud);
    const int64_t n = c->n, need = export_bytes(n, c->weighted);
    *size = need;
    if (!buf) return SDF_OK;
    if (cap < need) return set_error(SDF_EINVAL, "sdf_export: buffer smaller than the size sdf_export reports");
    char* out = static_cast<char*>(buf);
    ExportHeader h{};
    std::memcpy(h.magic, kExportMagic, sizeof(h.magic));
    h.version = 1;
    h.weighted = c->weighted ? 1u : 0u;
    h.n = n;
    std::memcpy(out, &h, sizeof(h));
    char* p = out + sizeof(h);
    // the inputs, then the records fitted from them again (k_fit is deterministic)
    float* d_w = nullptr;
    float* d_rec = nullptr;
    int8_t* d_kind = nullptr;
    int32_t* d_status = nullptr;
    cudaError_t e = cudaMemcpy(p, c->src_points, (size_t)n * 3 * sizeof(float), cudaMemcpyDeviceToHost);
    p += n * 3 * sizeof(float);
    if (e == cudaSuccess) e = cudaMemcpy(p, c->src_normals, (size_t)n * 3 * sizeof(float), cudaMemcpyDeviceToHost);
    p += n * 3 * sizeof(float);
    if (e == cudaSuccess) e = cudaMemcpy(p, c->src_params, (size_t)n * 6 * sizeof(float), cudaMemcpyDeviceToHost);
    p += n * 6 * sizeof(float);
    if (e == cudaSuccess && c->weighted) {
        // A_i sits in the plane records, (pz, pz, A, A) at float4 4 i + 1, input order
        e = cudaMalloc(&d_w, (size_t)n * sizeof(float));
        if (e == cudaSuccess)
            e = cudaMemcpy2D(d_w, sizeof(float), reinterpret_cast<const char*>(c->prec) + sizeof(float4) + 2 * sizeof(float),
                             4 * sizeof(float4), sizeof(float), (size_t)n, cudaMemcpyDeviceToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(p, d_w, (size_t)n * sizeof(float), cudaMemcpyDeviceToHost);
        p += n * sizeof(float);
    }
    if (e == cudaSuccess) e = cudaMalloc(&d_rec, (size_t)n * kRecFloats * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&d_kind, (size_t)n);
    if (e == cudaSuccess) e = cudaMalloc(&d_status, sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMemset(d_status, 0, sizeof(int32_t));
    if (e == cudaSuccess) {
        const double thr = 8.0 * std::fmax((double)c->aabb_diag, 1e-6);
        k_fit<<<(unsigned)((n + 127) / 128), 128>>>(c->src_points, c->src_normals, c->src_params, d_w, n, thr, d_rec,
                                                     d_kind, d_status);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(p, d_rec, (size_t)n * kRecFloats * sizeof(float), cudaMemcpyDeviceToHost);
    p += n * kRecFloats * sizeof(float);
    if (e == cudaSuccess) e = cudaMemcpy(p, d_kind, (size_t)n, cudaMemcpyDeviceToHost);
    cudaFree(d_w);
    cudaFree(d_rec);
    cudaFree(d_kind);
    cudaFree(d_status);
    return e == cudaSuccess ? SDF_OK : cuda_error(e, "sdf_export");
}

extern "C" sdf_status sdf_import(const void* buf, int64_t size, void* stream, sdf_cloud* out) {
    if (!buf || !out) return set_error(SDF_EINVAL, "sdf_import: buf or out is NULL");
    *out = nullptr;
    ExportHeader h{};
    if (size < (int64_t)sizeof(h)) return set_error(SDF_EINVAL, "sdf_import: buffer shorter than the header");
    std::memcpy(&h, buf, sizeof(h));
    if (std::memcmp(h.magic, kExportMagic, sizeof(h.magic)) != 0 || h.version != 1 || h.weighted > 1)
        return set_error(SDF_EINVAL, "sdf_import: not an sdf_export buffer of version 1");
    if (h.n < 1 || h.n > 0x7fffffffLL || size != export_bytes(h.n, h.weighted != 0))
        return set_error(SDF_EINVAL, "sdf_import: the buffer's size does not match its header");
    const int64_t n = h.n;
    const bool weighted = h.weighted != 0;
    const int64_t inputs = n * (12 + (weighted ? 1 : 0));
    const char* p = static_cast<const char*>(buf) + sizeof(h);
    float* d_in = nullptr;      // points, normals, coefficients, weights, records
    int8_t* d_kind = nullptr;
    cudaError_t e = cudaMalloc(&d_in, (size_t)(inputs + n * kRecFloats) * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&d_kind, (size_t)n);
    if (e == cudaSuccess)
        e = cudaMemcpy(d_in, p, (size_t)(inputs + n * kRecFloats) * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(d_kind, p + (inputs + n * kRecFloats) * sizeof(float), (size_t)n, cudaMemcpyHostToDevice);
    sdf_status s;
    if (e != cudaSuccess) {
        s = e == cudaErrorMemoryAllocation ? set_error(SDF_ENOMEM, "sdf_import: staging") : cuda_error(e, "sdf_import");
    } else {
        s = build_impl(d_in, d_in + 3 * n, d_in + 6 * n, weighted ? d_in + 12 * n : nullptr, n,
                       static_cast<cudaStream_t>(stream), out, d_in + inputs, d_kind);
    }
    cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
    cudaFree(d_in);
    cudaFree(d_kind);
    return s;
}

extern "C" sdf_status sdf_destroy(sdf_cloud cloud) {
    if (!cloud) return SDF_OK;
    Cloud* c = reinterpret_cast<Cloud*>(cloud);
    cudaDeviceSynchronize();
    free_cloud(c);
    return SDF_OK;
}

extern "C" sdf_status sdf_cloud_info(sdf_cloud cloud, int64_t* n, float* aabb_diag, int64_t* n_direct,
                                     int64_t* n_kappa) {
    if (!cloud) return set_error(SDF_EINVAL, "sdf_cloud_info: cloud is NULL");
    const Cloud* c = reinterpret_cast<const Cloud*>(cloud);
    if (n) *n = c->n;
    if (aabb_diag) *aabb_diag = c->aabb_diag;
    if (n_direct) *n_direct = c->n_direct;
    if (n_kappa) *n_kappa = c->n_kappa;
    return SDF_OK;
}

extern "C" sdf_status sdf_cloud_forms(sdf_cloud cloud, int64_t* n_kappa_flat, int64_t* exact_tiles) {
    if (!cloud) return set_error(SDF_EINVAL, "sdf_cloud_forms: cloud is NULL");
    const Cloud* c = reinterpret_cast<const Cloud*>(cloud);
    if (n_kappa_flat) *n_kappa_flat = c->n_kappa_flat;
    if (exact_tiles) {
        const int64_t tiles = c->btile_exact ? c->tiles_direct + c->tiles_kappa : 0;
        std::vector<int32_t> h((size_t)tiles);
        if (tiles > 0) {
            const cudaError_t e = cudaMemcpy(h.data(), c->btile_exact, (size_t)tiles * sizeof(int32_t),
                                             cudaMemcpyDeviceToHost);
            if (e != cudaSuccess) return cuda_error(e, "sdf_cloud_forms: read tile flags");
        }
        int64_t k = 0;
        for (int32_t v : h) k += v != 0;
        *exact_tiles = k;
    }
    return SDF_OK;
}
