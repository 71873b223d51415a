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

sdf_status check_opts(const sdf_query_opts& o, const char* fn) {
    if (o.lambda_mode != SDF_LAMBDA_GLOBAL && o.lambda_mode != SDF_LAMBDA_FIXED)
        return set_error(SDF_EINVAL, std::string(fn) + ": unknown lambda_mode");
    if (o.precision != SDF_F32) return set_error(SDF_EINVAL, std::string(fn) + ": unsupported precision");
    if (!(o.C > 0.f) || !std::isfinite(o.C)) return set_error(SDF_EINVAL, std::string(fn) + ": C must be > 0");
    if (o.lambda_mode == SDF_LAMBDA_FIXED && (!(o.fixed_lambda >= 0.f) || !std::isfinite(o.fixed_lambda)))
        return set_error(SDF_EINVAL, std::string(fn) + ": fixed_lambda must be >= 0");
    if (!std::isfinite(o.offset)) return set_error(SDF_EINVAL, std::string(fn) + ": offset must be finite");
    if (o.split_n < 0) return set_error(SDF_EINVAL, std::string(fn) + ": split_n must be >= 0");
    return SDF_OK;
}

sdf_query_opts resolve_opts(const sdf_query_opts* o) {
    sdf_query_opts r;
    sdf_opts_default(&r);
    return o ? *o : r;
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
