// sdf_trace: sphere tracing of the level set phi = offset (Sec. 6, "Direct
// visualization of point cloud surfaces"; Hart 1996).
//
// Every ray starts at t = 0.  A step evaluates f = phi(o + t d) - offset for
// all rays still live, as one query batch through the same prepass and pair
// kernels as sdf_query.  A ray hits when f < eps (t_hit = t), otherwise
// advances t += f, and misses once t > t_max or after max_steps evaluations
// (t_hit = -1).  The live rays are compacted after each step, so the batch
// shrinks as rays finish.  Normals at the hits are grad phi / |grad phi| from
// sdf_query_grad's kernels.
#include <cuda_runtime.h>

#include <cmath>

#include "internal.h"

namespace ptsdf {

namespace {

__global__ void k_trace_init(int64_t nrays, int32_t* __restrict__ live, float* __restrict__ t,
                             float* __restrict__ t_hit, int32_t* __restrict__ steps) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nrays) return;
    live[i] = (int32_t)i;
    t[i] = 0.f;
    t_hit[i] = -1.f;
    steps[i] = 0;
}

// positions of the live rays, in live-list order
__global__ void k_trace_positions(const int32_t* __restrict__ live, const int32_t* __restrict__ nlive,
                                  const float* __restrict__ org, const float* __restrict__ dir,
                                  const float* __restrict__ t, float* __restrict__ xbuf) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= *nlive) return;
    const int32_t r = live[j];
    const float tr = t[r];
    xbuf[3 * j] = fmaf(tr, dir[3 * r], org[3 * r]);
    xbuf[3 * j + 1] = fmaf(tr, dir[3 * r + 1], org[3 * r + 1]);
    xbuf[3 * j + 2] = fmaf(tr, dir[3 * r + 2], org[3 * r + 2]);
}

// one step's decisions; survivors are appended to live_next
__global__ void k_trace_update(const int32_t* __restrict__ live, const int32_t* __restrict__ nlive,
                               const float* __restrict__ phi, float eps, float t_max, int32_t max_steps,
                               float* __restrict__ t, float* __restrict__ t_hit, int32_t* __restrict__ steps,
                               int32_t* __restrict__ live_next, int32_t* __restrict__ nlive_next,
                               int32_t* __restrict__ hits, int32_t* __restrict__ nhits) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= *nlive) return;
    const int32_t r = live[j];
    const float f = phi[j];            // phi - offset
    const int32_t k = steps[r] + 1;
    steps[r] = k;
    const float tr = t[r];
    if (f < eps) {
        t_hit[r] = tr;
        hits[atomicAdd(nhits, 1)] = r;
        return;
    }
    const float tn = tr + f;
    t[r] = tn;
    if (tn > t_max || k >= max_steps) return;   // miss: t_hit stays -1
    live_next[atomicAdd(nlive_next, 1)] = r;
}

__global__ void k_hit_positions(const int32_t* __restrict__ hits, int64_t nh, const float* __restrict__ org,
                                const float* __restrict__ dir, const float* __restrict__ t_hit,
                                float* __restrict__ xbuf) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= nh) return;
    const int32_t r = hits[j];
    const float tr = t_hit[r];
    for (int k = 0; k < 3; ++k) xbuf[3 * j + k] = fmaf(tr, dir[3 * r + k], org[3 * r + k]);
}

__global__ void k_scatter_normals(const int32_t* __restrict__ hits, int64_t nh, const float* __restrict__ grad,
                                  float* __restrict__ normals) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= nh) return;
    const int32_t r = hits[j];
    const float gx = grad[3 * j], gy = grad[3 * j + 1], gz = grad[3 * j + 2];
    const float l = sqrtf(gx * gx + gy * gy + gz * gz);
    const float s = l > 0.f ? 1.f / l : 0.f;
    normals[3 * r] = gx * s;
    normals[3 * r + 1] = gy * s;
    normals[3 * r + 2] = gz * s;
}

unsigned blocks_for(int64_t n) { return (unsigned)((n + 255) / 256 > 0 ? (n + 255) / 256 : 1); }

}  // namespace

sdf_status launch_trace(const Cloud& c, const float* d_org, const float* d_dir, int64_t nrays, int32_t max_steps,
                        float eps, float t_max, float* d_t_hit, int32_t* d_steps, float* d_normals,
                        const sdf_query_opts& o, cudaStream_t st) {
    int32_t* live[2] = {nullptr, nullptr};
    int32_t* hits = nullptr;
    int32_t* counters = nullptr;   // [nlive0, nlive1, nhits]
    float* t = nullptr;
    float* xbuf = nullptr;
    float* phi = nullptr;
    float* grad = nullptr;
    int32_t* hcount = nullptr;
    cudaError_t e = cudaSuccess;
    sdf_status s = SDF_OK;
    auto A = [&](void** p, size_t bytes) {
        if (e == cudaSuccess) e = cudaMallocAsync(p, bytes, st);
    };
    A((void**)&live[0], (size_t)nrays * 4);
    A((void**)&live[1], (size_t)nrays * 4);
    A((void**)&hits, (size_t)nrays * 4);
    A((void**)&counters, 3 * 4);
    A((void**)&t, (size_t)nrays * 4);
    A((void**)&xbuf, (size_t)nrays * 12);
    A((void**)&phi, (size_t)nrays * 4);
    if (d_normals) A((void**)&grad, (size_t)nrays * 12);
    if (e == cudaSuccess) e = cudaMallocHost(&hcount, 3 * sizeof(int32_t));
    if (e != cudaSuccess) {
        s = e == cudaErrorMemoryAllocation ? set_error(SDF_ENOMEM, "sdf_trace: scratch")
                                           : cuda_error(e, "sdf_trace: scratch");
    }
    int64_t n = nrays;
    int cur = 0;
    if (s == SDF_OK) {
        k_trace_init<<<blocks_for(nrays), 256, 0, st>>>(nrays, live[0], t, d_t_hit, d_steps);
        e = cudaMemsetAsync(counters, 0, 3 * 4, st);
        if (e == cudaSuccess) {
            const int32_t nr = (int32_t)nrays;
            e = cudaMemcpyAsync(counters, &nr, 4, cudaMemcpyHostToDevice, st);
        }
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) s = cuda_error(e, "sdf_trace: init");
    }
    for (int step = 0; s == SDF_OK && step < max_steps && n > 0; ++step) {
        const int nxt = cur ^ 1;
        k_trace_positions<<<blocks_for(n), 256, 0, st>>>(live[cur], counters + cur, d_org, d_dir, t, xbuf);
        s = launch_query(c, xbuf, n, phi, o, st);     // phi - offset of every live ray
        if (s != SDF_OK) break;
        e = cudaMemsetAsync(counters + nxt, 0, 4, st);
        if (e == cudaSuccess) {
            k_trace_update<<<blocks_for(n), 256, 0, st>>>(live[cur], counters + cur, phi, eps, t_max, max_steps, t,
                                                          d_t_hit, d_steps, live[nxt], counters + nxt, hits,
                                                          counters + 2);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaMemcpyAsync(hcount, counters, 3 * 4, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) {
            s = cuda_error(e, "sdf_trace: step");
            break;
        }
        cur = nxt;
        n = hcount[cur];
    }
    if (s == SDF_OK && d_normals) {
        e = cudaMemsetAsync(d_normals, 0, (size_t)nrays * 12, st);
        const int64_t nh = hcount[2];
        if (e == cudaSuccess && nh > 0) {
            k_hit_positions<<<blocks_for(nh), 256, 0, st>>>(hits, nh, d_org, d_dir, d_t_hit, xbuf);
            sdf_query_opts og = o;
            og.offset = 0.f;
            // radius-limited tracing takes its normals from the all-pairs blend with the same lambda
            if (og.lambda_mode == SDF_LAMBDA_RADIUS) og.lambda_mode = SDF_LAMBDA_FIXED;
            s = launch_query_grad(c, xbuf, nh, phi, grad, nullptr, og, st);
            if (s == SDF_OK) {
                k_scatter_normals<<<blocks_for(nh), 256, 0, st>>>(hits, nh, grad, d_normals);
                e = cudaGetLastError();
            }
        }
        if (s == SDF_OK && e != cudaSuccess) s = cuda_error(e, "sdf_trace: normals");
    }
    for (auto* p : {(void*)live[0], (void*)live[1], (void*)hits, (void*)counters, (void*)t, (void*)xbuf,
                    (void*)phi, (void*)grad})
        if (p) cudaFreeAsync(p, st);
    cudaStreamSynchronize(st);
    if (hcount) cudaFreeHost(hcount);
    return s;
}

}  // namespace ptsdf
