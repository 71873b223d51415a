// Throughput probe of the operations that bound the pair loops: the
// special-function unit's sqrt, rsqrt, exp2 and reciprocal (the approximate
// forms the kernels use) and FP32 FMA, and the special-function work of one
// pair of each torus form as a whole (the mix the pair loops issue: direct
// 3 sqrt + 1 exp2; curvature form with kappa_min = 0, 2 sqrt + 1 rcp + 1
// exp2; other curvature form, 3 sqrt + 2 rcp + 1 exp2), one pair per chain
// step.  Each thread runs independent dependent chains
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
    if (OP == 4) return rcp_mufu(a) + 0.5f;           // -> 1.28 (a plain rcp chain folds to a copy)
    if (OP == 5) return ex2_mufu(-sqrt_mufu(sqrt_mufu(sqrt_mufu(a))));                         // in (0.5, 0.6)
    if (OP == 6) return ex2_mufu(-rcp_mufu(1.f + sqrt_mufu(sqrt_mufu(a))));                    // in (0.7, 0.8)
    if (OP == 7) return ex2_mufu(-rcp_mufu(1.f + sqrt_mufu(rcp_mufu(1.f + sqrt_mufu(sqrt_mufu(a))))));
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
    const Kern kernels[8] = {k_probe<0>, k_probe<1>, k_probe<2>, k_probe<3>,
                             k_probe<4>, k_probe<5>, k_probe<6>, k_probe<7>};
    for (int op = 0; op < 8 && e == cudaSuccess; ++op) {
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

// ---------------------------------------------------------------------------
// Self-test of the failure path: one thread waits, with a short limit, on an
// mbarrier phase that nothing will complete (no thread ever arrives), through
// the same bounded wait the pair loops use.  The wait must give up, record
// SDF_DEV_WAIT_TIMEOUT and return; nothing faults and nothing hangs.
// ---------------------------------------------------------------------------
namespace ptsdf {
namespace {

__global__ void k_wait_selftest(uint64_t limit_ns, int32_t* status, unsigned long long* waited_ns) {
    __shared__ __align__(8) uint64_t bar;
    __shared__ int abort_flag;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        abort_flag = 0;
        fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const uint64_t t0 = global_ns();
        const bool completed = mbar_wait_bounded_ns(&bar, 0u, &abort_flag, status, limit_ns);
        *waited_ns = global_ns() - t0;
        if (completed) atomicOr(status, 0x40000000);   // cannot happen: nothing arrives
    }
}

}  // namespace
}  // namespace ptsdf

extern "C" sdf_status sdf_selftest_wait_timeout(int32_t limit_us, int32_t* status_bits, double* waited_ms) {
    if (!status_bits || !waited_ms || limit_us < 1 || limit_us > 1000000)
        return set_error(SDF_EINVAL, "sdf_selftest_wait_timeout: limit_us in [1, 1e6] and non-NULL outputs");
    int32_t* d_status = nullptr;
    unsigned long long* d_waited = nullptr;
    cudaError_t e = cudaMalloc(&d_status, sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMalloc(&d_waited, sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemset(d_status, 0, sizeof(int32_t));
    if (e == cudaSuccess) {
        k_wait_selftest<<<1, 32>>>((uint64_t)limit_us * 1000ull, d_status, d_waited);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    unsigned long long w = 0;
    if (e == cudaSuccess) e = cudaMemcpy(status_bits, d_status, sizeof(int32_t), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(&w, d_waited, sizeof(w), cudaMemcpyDeviceToHost);
    cudaFree(d_status);
    cudaFree(d_waited);
    if (e != cudaSuccess) return cuda_error(e, "sdf_selftest_wait_timeout");
    *waited_ms = (double)w * 1e-6;
    return SDF_OK;
}
