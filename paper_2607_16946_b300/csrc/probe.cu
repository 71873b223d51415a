// Throughput probe of the operations that bound the pair loops: the
// special-function unit's sqrt, rsqrt and exp2 (the approximate forms the
// kernels use) and FP32 FMA.  Each thread runs independent dependent chains
// of one operation; every SM holds the same number of CTAs, which record
// their SM and their clock64 cycle count, so the rates come out per SM and
// per SM clock without relying on a nominal clock.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "device_common.cuh"
#include "internal.h"

namespace ptsdf {

namespace {

constexpr int kProbeIter = 2048;
constexpr int kProbeChains = 8;
constexpr int kProbeThreads = 512;
constexpr int kProbeCtasPerSm = 4;

template <int OP>
__device__ __forceinline__ float probe_op(float a) {
    if (OP == 0) return sqrt_mufu(a);                 // a -> 1
    if (OP == 1) return rsqrt_mufu(a);                // stays in (0.5, 2)
    if (OP == 2) return ex2_mufu(-a);                 // stays in (0.5, 1]
    return fmaf(a, 0.999f, 0.001f);                   // -> 1
}

template <int OP>
__global__ void __launch_bounds__(kProbeThreads) k_probe(float* __restrict__ sink, long long* __restrict__ cycles,
                                                         int* __restrict__ smid) {
    float a[kProbeChains];
#pragma unroll
    for (int i = 0; i < kProbeChains; ++i) a[i] = 0.6f + 1e-4f * (float)((threadIdx.x + 7 * i) & 255);
    __syncthreads();
    const long long t0 = clock64();
    for (int it = 0; it < kProbeIter; ++it) {
#pragma unroll
        for (int i = 0; i < kProbeChains; ++i) a[i] = probe_op<OP>(a[i]);
    }
    __syncthreads();
    const long long t1 = clock64();
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < kProbeChains; ++i) s += a[i];
    sink[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
    if (threadIdx.x == 0) {
        cycles[blockIdx.x] = t1 - t0;
        unsigned id;
        asm volatile("mov.u32 %0, %%smid;" : "=r"(id));
        smid[blockIdx.x] = (int)id;
    }
}

// results per SM per clock: per SM, (its CTAs x results per CTA) / (the
// longest of its CTAs' cycle counts), averaged over the SMs that ran CTAs
double sm_rate(const std::vector<long long>& cyc, const std::vector<int>& sm) {
    const int max_sm = *std::max_element(sm.begin(), sm.end()) + 1;
    std::vector<long long> longest(max_sm, 0);
    std::vector<int> ctas(max_sm, 0);
    for (size_t b = 0; b < cyc.size(); ++b) {
        if (sm[b] < 0) continue;
        longest[sm[b]] = std::max(longest[sm[b]], cyc[b]);
        ctas[sm[b]] += 1;
    }
    const double per_cta = (double)kProbeThreads * kProbeChains * kProbeIter;
    double sum = 0.0;
    int used = 0;
    for (int s = 0; s < max_sm; ++s) {
        if (ctas[s] == 0 || longest[s] <= 0) continue;
        sum += ctas[s] * per_cta / (double)longest[s];
        ++used;
    }
    return used ? sum / used : 0.0;
}

}  // namespace

}  // namespace ptsdf

using namespace ptsdf;

extern "C" sdf_status sdf_probe_rates(double* rates) {
    if (!rates) return set_error(SDF_EINVAL, "sdf_probe_rates: NULL output");
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_error(e, "sdf_probe_rates: device query");
    const int blocks = sms * kProbeCtasPerSm;
    float* sink = nullptr;
    long long* cyc = nullptr;
    int* smid = nullptr;
    e = cudaMalloc(&sink, (size_t)blocks * kProbeThreads * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&cyc, (size_t)blocks * sizeof(long long));
    if (e == cudaSuccess) e = cudaMalloc(&smid, (size_t)blocks * sizeof(int));
    std::vector<long long> hc(blocks);
    std::vector<int> hs(blocks);
    using Kern = void (*)(float*, long long*, int*);
    const Kern kernels[4] = {k_probe<0>, k_probe<1>, k_probe<2>, k_probe<3>};
    for (int op = 0; op < 4 && e == cudaSuccess; ++op) {
        for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {   // the first run warms up
            kernels[op]<<<blocks, kProbeThreads>>>(sink, cyc, smid);
            e = cudaGetLastError();
            if (e == cudaSuccess) e = cudaDeviceSynchronize();
        }
        if (e == cudaSuccess) e = cudaMemcpy(hc.data(), cyc, blocks * sizeof(long long), cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) e = cudaMemcpy(hs.data(), smid, blocks * sizeof(int), cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) rates[op] = sm_rate(hc, hs);
    }
    cudaFree(sink);
    cudaFree(cyc);
    cudaFree(smid);
    return e == cudaSuccess ? SDF_OK : cuda_error(e, "sdf_probe_rates");
}
