// C-ABI entry points of libptsdf.so that are not tied to one kernel family:
// options, argument checks, the host-buffer query, the device status word and
// error reporting.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <string>

#include "internal.h"

namespace ptsdf {

namespace {
thread_local std::string g_last_error;
}

sdf_status set_error(sdf_status st, const std::string& msg) {
    g_last_error = msg;
    return st;
}

sdf_status cuda_error(cudaError_t e, const char* what) {
    return set_error(SDF_ECUDA, std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")");
}

static_assert(sizeof(sdf_query_opts) == 32, "sdf_query_opts layout");
static_assert(sizeof(sdf_request) == 88, "sdf_request layout");

sdf_status check_opts(const sdf_query_opts& o, const char* fn) {
    if (o.lambda_mode != SDF_LAMBDA_GLOBAL && o.lambda_mode != SDF_LAMBDA_FIXED && o.lambda_mode != SDF_LAMBDA_RADIUS)
        return set_error(SDF_EINVAL, std::string(fn) + ": unknown lambda_mode");
    if (o.lambda_mode == SDF_LAMBDA_RADIUS) {
        if (!(o.fixed_lambda > 0.f) || !std::isfinite(o.fixed_lambda))
            return set_error(SDF_EINVAL, std::string(fn) + ": SDF_LAMBDA_RADIUS needs fixed_lambda > 0");
        if (o.precision != SDF_F32 || o.engine == SDF_ENGINE_TENSOR)
            return set_error(SDF_EINVAL, std::string(fn) + ": SDF_LAMBDA_RADIUS runs in FP32 on the FP32 units");
    }
    if (o.precision != SDF_F32 && o.precision != SDF_F16X2 && o.precision != SDF_BF16X2)
        return set_error(SDF_EINVAL, std::string(fn) + ": unknown precision");
    if (!(o.C > 0.f) || !std::isfinite(o.C)) return set_error(SDF_EINVAL, std::string(fn) + ": C must be > 0");
    if (o.lambda_mode == SDF_LAMBDA_FIXED && (!(o.fixed_lambda >= 0.f) || !std::isfinite(o.fixed_lambda)))
        return set_error(SDF_EINVAL, std::string(fn) + ": fixed_lambda must be >= 0");
    if (!std::isfinite(o.offset)) return set_error(SDF_EINVAL, std::string(fn) + ": offset must be finite");
    if (o.split_n < 0) return set_error(SDF_EINVAL, std::string(fn) + ": split_n must be >= 0");
    if (o.engine != SDF_ENGINE_AUTO && o.engine != SDF_ENGINE_ALU && o.engine != SDF_ENGINE_TENSOR)
        return set_error(SDF_EINVAL, std::string(fn) + ": unknown engine");
    if (o.engine == SDF_ENGINE_TENSOR && o.precision != SDF_F32)
        return set_error(SDF_EINVAL, std::string(fn) + ": the tensor-core engine computes in FP32 only");
    if (o.formula != SDF_FORMULA_BLEND && o.formula != SDF_FORMULA_LSE && o.formula != SDF_FORMULA_SSPD &&
        o.formula != SDF_FORMULA_SHC)
        return set_error(SDF_EINVAL, std::string(fn) + ": unknown formula");
    if (o.formula == SDF_FORMULA_LSE && o.lambda_mode == SDF_LAMBDA_FIXED && !(o.fixed_lambda > 0.f))
        return set_error(SDF_EINVAL, std::string(fn) + ": the log-sum-exp distance needs fixed_lambda > 0");
    if (o.formula == SDF_FORMULA_SSPD || o.formula == SDF_FORMULA_SHC) {
        if (o.lambda_mode == SDF_LAMBDA_RADIUS || o.precision != SDF_F32 || o.engine == SDF_ENGINE_TENSOR)
            return set_error(SDF_EINVAL, std::string(fn) + ": the SSPD and SHC baselines run in FP32 on the FP32 "
                                                            "units, with GLOBAL or FIXED lambda");
        if (o.formula == SDF_FORMULA_SHC && o.lambda_mode == SDF_LAMBDA_FIXED && !(o.fixed_lambda > 0.f))
            return set_error(SDF_EINVAL, std::string(fn) + ": the signed Hopf-Cole distance needs fixed_lambda > 0");
    }
    return SDF_OK;
}

// The gradient-type calls evaluate the blend only.
sdf_status blend_only(const sdf_query_opts& o, const char* fn) {
    return o.formula == SDF_FORMULA_BLEND
               ? SDF_OK
               : set_error(SDF_EINVAL, std::string(fn) + ": the log-sum-exp distance and the SSPD and SHC "
                                                         "baselines are for sdf_query only");
}

// Booleans of two phi arrays (Sec. 6): union min, intersection max, difference max(a, -b)
__global__ void k_combine(int op, const float* __restrict__ a, const float* __restrict__ b, int64_t q,
                          float* __restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= q) return;
    const float x = a[i], y = b[i];
    out[i] = op == SDF_UNION ? fminf(x, y) : op == SDF_INTERSECT ? fmaxf(x, y) : fmaxf(x, -y);
}

sdf_query_opts resolve_opts(const sdf_query_opts* o) {
    sdf_query_opts r;
    sdf_opts_default(&r);
    return o ? *o : r;
}

// One Newton step onto the `level` set of phi (Sec. 6, "Morphological
// operations": sampling a level set): x -= (phi - level) grad / |grad|^2,
// except where |phi - level| <= tol or the gradient vanishes.
__global__ void k_level_step(float* __restrict__ x, const float* __restrict__ phi, const float* __restrict__ grad,
                             int64_t q, float level, float tol) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= q) return;
    const float r = phi[i] - level;
    const float gx = grad[3 * i], gy = grad[3 * i + 1], gz = grad[3 * i + 2];
    const float g2 = fmaf(gx, gx, fmaf(gy, gy, gz * gz));
    if (!(fabsf(r) > tol) || !(g2 > 1e-30f)) return;
    const float f = r / g2;
    x[3 * i] -= f * gx;
    x[3 * i + 1] -= f * gy;
    x[3 * i + 2] -= f * gz;
}

// Normals grad / |grad| in place, residual phi - level in place.
__global__ void k_level_finish(float* __restrict__ phi, float* __restrict__ grad, int64_t q, float level) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= q) return;
    phi[i] -= level;
    const float gx = grad[3 * i], gy = grad[3 * i + 1], gz = grad[3 * i + 2];
    const float inv = rsqrtf(fmaxf(fmaf(gx, gx, fmaf(gy, gy, gz * gz)), 1e-30f));
    grad[3 * i] = gx * inv;
    grad[3 * i + 1] = gy * inv;
    grad[3 * i + 2] = gz * inv;
}

}  // namespace ptsdf

using namespace ptsdf;

extern "C" sdf_status sdf_opts_default(sdf_query_opts* o) {
    if (!o) return set_error(SDF_EINVAL, "sdf_opts_default: NULL");
    o->lambda_mode = SDF_LAMBDA_GLOBAL;
    o->precision = SDF_F32;
    o->C = 64.f;
    o->fixed_lambda = 0.f;
    o->offset = 0.f;
    o->split_n = 0;
    o->engine = SDF_ENGINE_AUTO;
    o->formula = SDF_FORMULA_BLEND;
    return SDF_OK;
}

extern "C" sdf_status sdf_query(sdf_cloud cloud, const float* d_x, int64_t q, float* d_phi,
                                const sdf_query_opts* opts, void* stream) {
    if (!cloud) return set_error(SDF_EINVAL, "sdf_query: cloud is NULL");
    if (q < 0) return set_error(SDF_EINVAL, "sdf_query: q < 0");
    const sdf_query_opts o = resolve_opts(opts);
    const sdf_status s = check_opts(o, "sdf_query");
    if (s != SDF_OK) return s;
    if (q == 0) return SDF_OK;
    if (!d_x || !d_phi) return set_error(SDF_EINVAL, "sdf_query: NULL buffer");
    return launch_query(*reinterpret_cast<const Cloud*>(cloud), d_x, q, d_phi, o,
                        static_cast<cudaStream_t>(stream));
}

extern "C" sdf_status sdf_query_grad(sdf_cloud cloud, const float* d_x, int64_t q, float* d_phi, float* d_grad,
                                     float* d_saved, const sdf_query_opts* opts, void* stream) {
    if (!cloud) return set_error(SDF_EINVAL, "sdf_query_grad: cloud is NULL");
    if (q < 0) return set_error(SDF_EINVAL, "sdf_query_grad: q < 0");
    const sdf_query_opts o = resolve_opts(opts);
    sdf_status s = check_opts(o, "sdf_query_grad");
    if (s != SDF_OK) return s;
    if (o.formula == SDF_FORMULA_SSPD || o.formula == SDF_FORMULA_SHC)
        return set_error(SDF_EINVAL, "sdf_query_grad: no gradient of the SSPD and SHC baselines");
    if (o.formula == SDF_FORMULA_LSE && d_saved)
        return set_error(SDF_EINVAL, "sdf_query_grad: no saved statistics for the log-sum-exp distance "
                                     "(they serve the blend's parameter gradient)");
    if (o.precision != SDF_F32) return set_error(SDF_EINVAL, "sdf_query_grad: gradients are computed in FP32 only");
    if (o.lambda_mode == SDF_LAMBDA_RADIUS)
        return set_error(SDF_EINVAL, "sdf_query_grad: no gradient for SDF_LAMBDA_RADIUS");
    if (o.engine == SDF_ENGINE_TENSOR)
        return set_error(SDF_EINVAL, "sdf_query_grad: gradients use the FP32 units (no tensor-core engine)");
    if (q == 0) return SDF_OK;
    if (!d_x || !d_phi || !d_grad) return set_error(SDF_EINVAL, "sdf_query_grad: NULL buffer");
    return launch_query_grad(*reinterpret_cast<const Cloud*>(cloud), d_x, q, d_phi, d_grad, d_saved, o,
                             static_cast<cudaStream_t>(stream));
}

extern "C" sdf_status sdf_project_level_set(sdf_cloud cloud, const float* d_x0, int64_t q, float level,
                                            int32_t max_iter, float tol, float* d_x, float* d_normals,
                                            float* d_residual, const sdf_query_opts* opts, void* stream) {
    if (!cloud) return set_error(SDF_EINVAL, "sdf_project_level_set: cloud is NULL");
    if (q < 0) return set_error(SDF_EINVAL, "sdf_project_level_set: q < 0");
    if (max_iter < 0 || max_iter > 100) return set_error(SDF_EINVAL, "sdf_project_level_set: max_iter in [0, 100]");
    if (!std::isfinite(level) || !(tol >= 0.f) || !std::isfinite(tol))
        return set_error(SDF_EINVAL, "sdf_project_level_set: level finite, tol finite and >= 0");
    sdf_query_opts o = resolve_opts(opts);
    sdf_status s = check_opts(o, "sdf_project_level_set");
    if (s == SDF_OK) s = blend_only(o, "sdf_project_level_set");
    if (s != SDF_OK) return s;
    if (o.precision != SDF_F32 || o.lambda_mode == SDF_LAMBDA_RADIUS || o.engine == SDF_ENGINE_TENSOR)
        return set_error(SDF_EINVAL, "sdf_project_level_set: the gradient's options (FP32, GLOBAL or FIXED lambda)");
    if (q == 0) return SDF_OK;
    if (!d_x0 || !d_x || !d_normals || !d_residual) return set_error(SDF_EINVAL, "sdf_project_level_set: NULL buffer");
    o.offset = 0.f;   // the level plays the offset's part
    const Cloud& c = *reinterpret_cast<const Cloud*>(cloud);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaSuccess;
    if (d_x != d_x0) e = cudaMemcpyAsync(d_x, d_x0, (size_t)q * 3 * sizeof(float), cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return cuda_error(e, "sdf_project_level_set: copy");
    const unsigned blocks = (unsigned)((q + 255) / 256);
    // phi and grad phi land in the residual and normal outputs, which serve as scratch
    for (int it = 0; it <= max_iter; ++it) {
        s = launch_query_grad(c, d_x, q, d_residual, d_normals, nullptr, o, st);
        if (s != SDF_OK) return s;
        if (it == max_iter) break;
        ptsdf::k_level_step<<<blocks, 256, 0, st>>>(d_x, d_residual, d_normals, q, level, tol);
        e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_error(e, "sdf_project_level_set: k_level_step");
    }
    ptsdf::k_level_finish<<<blocks, 256, 0, st>>>(d_residual, d_normals, q, level);
    e = cudaGetLastError();
    return e == cudaSuccess ? SDF_OK : cuda_error(e, "sdf_project_level_set: k_level_finish");
}

extern "C" sdf_status sdf_query_laplacian(sdf_cloud cloud, const float* d_x, int64_t q, float* d_phi, float* d_grad,
                                          float* d_lap, const sdf_query_opts* opts, void* stream) {
    if (!cloud) return set_error(SDF_EINVAL, "sdf_query_laplacian: cloud is NULL");
    if (q < 0) return set_error(SDF_EINVAL, "sdf_query_laplacian: q < 0");
    const sdf_query_opts o = resolve_opts(opts);
    sdf_status s = check_opts(o, "sdf_query_laplacian");
    if (s == SDF_OK) s = blend_only(o, "sdf_query_laplacian");
    if (s != SDF_OK) return s;
    if (o.precision != SDF_F32 || o.engine == SDF_ENGINE_TENSOR)
        return set_error(SDF_EINVAL, "sdf_query_laplacian: FP32 on the FP32 units only");
    if (o.lambda_mode == SDF_LAMBDA_RADIUS)
        return set_error(SDF_EINVAL, "sdf_query_laplacian: not defined for SDF_LAMBDA_RADIUS");
    if (q == 0) return SDF_OK;
    if (!d_x || !d_lap) return set_error(SDF_EINVAL, "sdf_query_laplacian: NULL buffer");
    return launch_query_grad(*reinterpret_cast<const Cloud*>(cloud), d_x, q, d_phi, d_grad, nullptr, o,
                             static_cast<cudaStream_t>(stream), d_lap);
}

extern "C" sdf_status sdf_backward_params(sdf_cloud cloud, const float* d_x, int64_t q, const float* d_saved,
                                          const float* d_grad_phi, float* d_grad_params,
                                          const sdf_query_opts* opts, void* stream) {
    if (!cloud) return set_error(SDF_EINVAL, "sdf_backward_params: cloud is NULL");
    if (q < 0) return set_error(SDF_EINVAL, "sdf_backward_params: q < 0");
    if (!d_grad_params) return set_error(SDF_EINVAL, "sdf_backward_params: NULL output");
    const sdf_query_opts o = resolve_opts(opts);
    sdf_status s = check_opts(o, "sdf_backward_params");
    if (s == SDF_OK) s = blend_only(o, "sdf_backward_params");
    if (s != SDF_OK) return s;
    if (o.precision != SDF_F32)
        return set_error(SDF_EINVAL, "sdf_backward_params: gradients are computed in FP32 only");
    if (o.lambda_mode == SDF_LAMBDA_RADIUS)
        return set_error(SDF_EINVAL, "sdf_backward_params: no gradient for SDF_LAMBDA_RADIUS");
    if (o.engine == SDF_ENGINE_TENSOR)
        return set_error(SDF_EINVAL, "sdf_backward_params: gradients use the FP32 units (no tensor-core engine)");
    const Cloud& c = *reinterpret_cast<const Cloud*>(cloud);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (q == 0) {
        const cudaError_t e = cudaMemsetAsync(d_grad_params, 0, (size_t)c.n * 6 * sizeof(float), st);
        return e == cudaSuccess ? SDF_OK : cuda_error(e, "sdf_backward_params: clear");
    }
    if (!d_x || !d_saved || !d_grad_phi) return set_error(SDF_EINVAL, "sdf_backward_params: NULL buffer");
    return launch_backward_params(c, q, d_saved, d_grad_phi, d_grad_params, o, st);
}

extern "C" sdf_status sdf_trace(sdf_cloud cloud, const float* d_origins, const float* d_dirs, int64_t nrays,
                                int32_t max_steps, float eps, float t_max, float* d_t_hit, int32_t* d_steps,
                                float* d_normals, const sdf_query_opts* opts, void* stream) {
    if (!cloud) return set_error(SDF_EINVAL, "sdf_trace: cloud is NULL");
    if (nrays < 0 || nrays > 0x7fffffffLL) return set_error(SDF_EINVAL, "sdf_trace: nrays out of range");
    if (max_steps < 1 || !(eps > 0.f) || !(t_max > 0.f) || !std::isfinite(t_max))
        return set_error(SDF_EINVAL, "sdf_trace: need max_steps >= 1, eps > 0, finite t_max > 0");
    const sdf_query_opts o = resolve_opts(opts);
    sdf_status s = check_opts(o, "sdf_trace");
    if (s == SDF_OK) s = blend_only(o, "sdf_trace");
    if (s != SDF_OK) return s;
    if (nrays == 0) return SDF_OK;
    if (!d_origins || !d_dirs || !d_t_hit || !d_steps) return set_error(SDF_EINVAL, "sdf_trace: NULL buffer");
    return launch_trace(*reinterpret_cast<const Cloud*>(cloud), d_origins, d_dirs, nrays, max_steps, eps, t_max,
                        d_t_hit, d_steps, d_normals, o, static_cast<cudaStream_t>(stream));
}

extern "C" sdf_status sdf_combine(int32_t op, const float* d_a, const float* d_b, int64_t q, float* d_out,
                                  void* stream) {
    if (op != SDF_UNION && op != SDF_INTERSECT && op != SDF_DIFFERENCE)
        return set_error(SDF_EINVAL, "sdf_combine: unknown op");
    if (q < 0) return set_error(SDF_EINVAL, "sdf_combine: q < 0");
    if (q == 0) return SDF_OK;
    if (!d_a || !d_b || !d_out) return set_error(SDF_EINVAL, "sdf_combine: NULL buffer");
    ptsdf::k_combine<<<(unsigned)((q + 255) / 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(op, d_a, d_b, q, d_out);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? SDF_OK : cuda_error(e, "sdf_combine");
}

extern "C" sdf_status sdf_query_host(sdf_cloud cloud, const float* h_x, int64_t q, float* h_phi,
                                     const sdf_query_opts* opts, void* stream) {
    if (!cloud) return set_error(SDF_EINVAL, "sdf_query_host: cloud is NULL");
    if (q < 0) return set_error(SDF_EINVAL, "sdf_query_host: q < 0");
    const sdf_query_opts o = resolve_opts(opts);
    sdf_status s = check_opts(o, "sdf_query_host");
    if (s != SDF_OK) return s;
    if (q == 0) return SDF_OK;
    if (!h_x || !h_phi) return set_error(SDF_EINVAL, "sdf_query_host: NULL buffer");
    const Cloud& c = *reinterpret_cast<const Cloud*>(cloud);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // chunks of up to 2^26 queries (768 MB of positions) bound the staging memory
    const int64_t chunk = q < (1LL << 26) ? q : (1LL << 26);
    float* dx = nullptr;
    float* dphi = nullptr;
    cudaError_t e = cudaMallocAsync(&dx, (size_t)chunk * 3 * sizeof(float), st);
    if (e == cudaSuccess) e = cudaMallocAsync(&dphi, (size_t)chunk * sizeof(float), st);
    if (e != cudaSuccess) {
        if (dx) cudaFreeAsync(dx, st);
        cudaStreamSynchronize(st);
        return e == cudaErrorMemoryAllocation ? set_error(SDF_ENOMEM, "sdf_query_host: staging")
                                              : cuda_error(e, "sdf_query_host: staging");
    }
    for (int64_t q0 = 0; q0 < q && s == SDF_OK; q0 += chunk) {
        const int64_t m = q - q0 < chunk ? q - q0 : chunk;
        e = cudaMemcpyAsync(dx, h_x + 3 * q0, (size_t)m * 3 * sizeof(float), cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) {
            s = cuda_error(e, "sdf_query_host: copy in");
            break;
        }
        s = launch_query(c, dx, m, dphi, o, st);
        if (s != SDF_OK) break;
        e = cudaMemcpyAsync(h_phi + q0, dphi, (size_t)m * sizeof(float), cudaMemcpyDeviceToHost, st);
        if (e != cudaSuccess) s = cuda_error(e, "sdf_query_host: copy out");
    }
    cudaFreeAsync(dx, st);
    cudaFreeAsync(dphi, st);
    e = cudaStreamSynchronize(st);
    if (s == SDF_OK && e != cudaSuccess) s = cuda_error(e, "sdf_query_host: sync");
    return s;
}

extern "C" sdf_status sdf_device_status(sdf_cloud cloud, void* stream, int32_t* code) {
    if (!cloud || !code) return set_error(SDF_EINVAL, "sdf_device_status: NULL argument");
    const Cloud& c = *reinterpret_cast<const Cloud*>(cloud);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int32_t v = 0;
    cudaError_t e = cudaMemcpyAsync(&v, c.status, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(c.status, 0, sizeof(int32_t), st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_error(e, "sdf_device_status");
    *code = v;
    return v ? set_error(SDF_EDEVICE, "a kernel reported a fault (status bits " + std::to_string(v) + ")") : SDF_OK;
}

extern "C" const char* sdf_last_error(void) { return g_last_error.c_str(); }

extern "C" const char* sdf_version(void) { return "ptsdf 0.1 (sm_103a)"; }
