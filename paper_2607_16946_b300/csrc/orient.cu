// Orientation repair of inconsistently oriented clouds (Sec. 6, "Orienting
// inconsistently oriented point clouds").
//
// One iteration, every point deciding from the same cloud:
//   1. build the cloud from the current (points, normals, coefficients) and
//      evaluate grad phi at every point of the cloud (sdf_query_grad's loop);
//   2. for point i, n~_i = sum over its k nearest other points j of
//      exp(-M_i(p_i - p_j)) grad phi(p_j) with
//      M_i(r) = sqrt(kmin^2 <r, v_min>^2 + kmax^2 <r, v_max>^2 + eps^2 <r, n_i>^2),
//      the principal curvatures and directions of point i's fit (v_max is the
//      torus axis u, v_min = u x n*);
//   3. flip n_i where <n_i, n~_i> < 0, and re-express its quadratic patch in
//      the frame of -n_i, so that its torus stays the same torus with the
//      opposite sign (the paper re-runs its network instead, which is absent).
// Repeat until nothing flips.  The k nearest are found once (the points do
// not move), with the Morton-ordered spheres of the cloud.
#include <cuda_runtime.h>

#include <cmath>

#include "fit_math.cuh"
#include "internal.h"

namespace ptsdf {

namespace {

constexpr int kOrientThreads = 128;

__device__ __forceinline__ void cross3(const double a[3], const double b[3], double c[3]) {
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

__device__ __forceinline__ double dot3d(const double a[3], const double b[3]) {
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

__device__ __forceinline__ void unit_normal(const float* __restrict__ N, int64_t i, double n[3]) {
    n[0] = N[3 * i];
    n[1] = N[3 * i + 1];
    n[2] = N[3 * i + 2];
    const double l = sqrt(dot3d(n, n));
    for (int k = 0; k < 3; ++k) n[k] /= l;
}

__global__ void k_orient_score(const float* __restrict__ P, const float* __restrict__ N, const float* __restrict__ A,
                               const int32_t* __restrict__ nbr, int k, const float* __restrict__ grad, double eps,
                               int64_t n, uint8_t* __restrict__ flip, int32_t* __restrict__ count) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double p[3] = {P[3 * i], P[3 * i + 1], P[3 * i + 2]};
    double nu[3];
    unit_normal(N, i, nu);
    double a[6];
    for (int m = 0; m < 6; ++m) a[m] = A[6 * i + m];
    FitPoint<double> f;
    fit_point<double>(p, nu, a, f);
    double vmin[3];
    cross3(f.u, f.nstar, vmin);
    double nt[3] = {0.0, 0.0, 0.0};
    for (int j = 0; j < k; ++j) {
        const int32_t q = nbr[i * k + j];
        if (q < 0) continue;
        const double r[3] = {p[0] - P[3 * (int64_t)q], p[1] - P[3 * (int64_t)q + 1], p[2] - P[3 * (int64_t)q + 2]};
        const double e1 = f.kmin * dot3d(r, vmin), e2 = f.kmax * dot3d(r, f.u), e3 = eps * dot3d(r, nu);
        const double w = exp(-sqrt(e1 * e1 + e2 * e2 + e3 * e3));
        for (int m = 0; m < 3; ++m) nt[m] += w * (double)grad[3 * (int64_t)q + m];
    }
    const bool fl = dot3d(nu, nt) < 0.0;
    flip[i] = fl ? 1 : 0;
    if (fl) atomicAdd(count, 1);
}

// n -> -n; the coefficients of the same patch over the frame of -n:
// (s, t) = M (s', t'), f' = -f o M.
__global__ void k_orient_apply(float* __restrict__ N, float* __restrict__ A, const uint8_t* __restrict__ flip,
                               int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || !flip[i]) return;
    double nu[3];
    unit_normal(N, i, nu);
    const double nm[3] = {-nu[0], -nu[1], -nu[2]};
    double s[3], t[3], s2[3], t2[3];
    duff_frame(nu, s, t);
    duff_frame(nm, s2, t2);
    const double m11 = dot3d(s2, s), m12 = dot3d(t2, s), m21 = dot3d(s2, t), m22 = dot3d(t2, t);
    const double a00 = A[6 * i], a01 = A[6 * i + 1], a10 = A[6 * i + 2], a11 = A[6 * i + 3], a02 = A[6 * i + 4],
                 a20 = A[6 * i + 5];
    // linear part a10 s + a01 t; quadratic form H = [[a20, a11/2], [a11/2, a02]] -> M^T H M
    const double l1 = a10 * m11 + a01 * m21, l2 = a10 * m12 + a01 * m22;
    const double h12 = 0.5 * a11;
    const double c11 = a20 * m11 + h12 * m21, c12 = a20 * m12 + h12 * m22;   // (H M) row 1
    const double c21 = h12 * m11 + a02 * m21, c22 = h12 * m12 + a02 * m22;   // (H M) row 2
    const double H11 = m11 * c11 + m21 * c21, H12 = m11 * c12 + m21 * c22, H22 = m12 * c12 + m22 * c22;
    A[6 * i] = (float)(-a00);
    A[6 * i + 1] = (float)(-l2);
    A[6 * i + 2] = (float)(-l1);
    A[6 * i + 3] = (float)(-2.0 * H12);
    A[6 * i + 4] = (float)(-H22);
    A[6 * i + 5] = (float)(-H11);
    for (int m = 0; m < 3; ++m) N[3 * i + m] = -N[3 * i + m];
}

}  // namespace

}  // namespace ptsdf

using namespace ptsdf;

extern "C" sdf_status sdf_orient(const float* d_points, float* d_normals, float* d_params, int64_t n, int32_t k,
                                 int32_t max_iter, const sdf_query_opts* opts, int32_t* flips, int32_t* iterations,
                                 void* stream) {
    if (!d_points || !d_normals || !d_params || !flips || !iterations)
        return set_error(SDF_EINVAL, "sdf_orient: NULL argument");
    if (n < 2 || n > 0x7fffffffLL) return set_error(SDF_EINVAL, "sdf_orient: n must be in [2, 2^31-1]");
    if (k < 1 || k > 64) return set_error(SDF_EINVAL, "sdf_orient: k must be in [1, 64]");
    if (max_iter < 1) return set_error(SDF_EINVAL, "sdf_orient: max_iter must be >= 1");
    sdf_query_opts o;
    sdf_opts_default(&o);
    if (opts) o = *opts;
    if ((o.lambda_mode != SDF_LAMBDA_GLOBAL && o.lambda_mode != SDF_LAMBDA_FIXED) || o.precision != SDF_F32 ||
        !(o.C > 0.f) || (o.lambda_mode == SDF_LAMBDA_FIXED && !(o.fixed_lambda >= 0.f)))
        return set_error(SDF_EINVAL, "sdf_orient: GLOBAL or FIXED lambda, FP32");
    o.offset = 0.f;
    o.engine = SDF_ENGINE_ALU;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    *iterations = 0;
    int32_t *nbr = nullptr, *cnt = nullptr;
    float *grad = nullptr, *phi = nullptr;
    uint8_t* flip = nullptr;
    cudaError_t e = cudaMallocAsync(&nbr, (size_t)n * k * sizeof(int32_t), st);
    if (e == cudaSuccess) e = cudaMallocAsync(&grad, (size_t)n * 3 * sizeof(float), st);
    if (e == cudaSuccess) e = cudaMallocAsync(&phi, (size_t)n * sizeof(float), st);
    if (e == cudaSuccess) e = cudaMallocAsync(&flip, (size_t)n, st);
    if (e == cudaSuccess) e = cudaMallocAsync(&cnt, sizeof(int32_t), st);
    sdf_status s = e == cudaSuccess ? SDF_OK : cuda_error(e, "sdf_orient: scratch");
    double eps = 0.0;
    const unsigned blocks = (unsigned)((n + kOrientThreads - 1) / kOrientThreads);
    for (int it = 0; s == SDF_OK && it < max_iter; ++it) {
        sdf_cloud cl = nullptr;
        s = sdf_build(d_points, d_normals, d_params, n, stream, &cl);
        if (s != SDF_OK) break;
        const Cloud& c = *reinterpret_cast<const Cloud*>(cl);
        if (it == 0) {
            double D = 0.0;
            s = launch_knn_indices(c, k, nbr, &D, st);
            eps = D > 0.0 ? 1.0 / D : 0.0;
        }
        if (s == SDF_OK) s = launch_query_grad(c, d_points, n, phi, grad, nullptr, o, st);
        int32_t h = 0;
        if (s == SDF_OK) {
            e = cudaMemsetAsync(cnt, 0, sizeof(int32_t), st);
            if (e == cudaSuccess) {
                k_orient_score<<<blocks, kOrientThreads, 0, st>>>(d_points, d_normals, d_params, nbr, k, grad, eps, n,
                                                                  flip, cnt);
                e = cudaGetLastError();
            }
            if (e == cudaSuccess) e = cudaMemcpyAsync(&h, cnt, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
            if (e != cudaSuccess) s = cuda_error(e, "sdf_orient: score");
        }
        sdf_destroy(cl);
        if (s != SDF_OK) break;
        flips[it] = h;
        *iterations = it + 1;
        if (h == 0) break;
        k_orient_apply<<<blocks, kOrientThreads, 0, st>>>(d_normals, d_params, flip, n);
        e = cudaGetLastError();
        if (e != cudaSuccess) s = cuda_error(e, "sdf_orient: apply");
    }
    cudaFreeAsync(nbr, st);
    cudaFreeAsync(grad, st);
    cudaFreeAsync(phi, st);
    cudaFreeAsync(flip, st);
    cudaFreeAsync(cnt, st);
    cudaStreamSynchronize(st);
    return s;
}
