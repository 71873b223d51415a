// Throughput probe of the operations that bound the pair loops: the
// special-function unit's sqrt, rsqrt, exp2 and reciprocal (the approximate
// forms the kernels use) and FP32 FMA, and the special-function work of one
// pair of each torus form as a whole (the mix the pair loops issue: direct
// 3 sqrt + 1 exp2; curvature form with kappa_min = 0, 2 sqrt + 1 rcp + 1
// exp2; other curvature form, 3 sqrt + 2 rcp + 1 exp2), one pair per chain
// step.  Each thread runs independent dependent chains of one operation;
// every SM holds the same number of CTAs, which record their SM, their
// clock64 cycle count and their %globaltimer start and end.  A rate is, per
// SM, the results of its CTAs over the union of their time windows (first
// start to last end), converted to SM clocks with the clock measured in the
// kernel (clock64 cycles over %globaltimer ns), averaged over the SMs: per SM
// clock, without relying on a nominal clock.  (Dividing by the longest
// single CTA's clock64 window instead overstates the rates by up to 14% on
// B300: the CTAs of an SM start and end at different times.)
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
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

// ns[2 b], ns[2 b + 1]: %globaltimer at the start and end of CTA b's timed
// loop (the same points as its clock64 reads), for the cross-checks of
// sdf_probe_timing.
template <int OP>
__global__ void __launch_bounds__(kProbeThreads) k_probe(float* __restrict__ sink, long long* __restrict__ cycles,
                                                         int* __restrict__ smid, unsigned long long* __restrict__ ns) {
    float a[kProbeChains];
#pragma unroll
    for (int i = 0; i < kProbeChains; ++i) a[i] = 0.6f + 1e-4f * (float)((threadIdx.x + 7 * i) & 255);
    __syncthreads();
    const uint64_t g0 = global_ns();
    const long long t0 = clock64();
    for (int it = 0; it < kProbeIter; ++it) {
#pragma unroll
        for (int i = 0; i < kProbeChains; ++i) a[i] = probe_op<OP>(a[i]);
    }
    __syncthreads();
    const long long t1 = clock64();
    const uint64_t g1 = global_ns();
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < kProbeChains; ++i) s += a[i];
    sink[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
    if (threadIdx.x == 0) {
        cycles[blockIdx.x] = t1 - t0;
        unsigned id;
        asm volatile("mov.u32 %0, %%smid;" : "=r"(id));
        smid[blockIdx.x] = (int)id;
        ns[2 * blockIdx.x] = g0;
        ns[2 * blockIdx.x + 1] = g1;
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

// The other readings of one probe launch (see sdf_probe_timing):
//  [1] per SM, its CTAs' results over the union of their %globaltimer windows
//      (first start to last end) times the SM clock measured in the kernel,
//      averaged over the SMs;
//  [2] all results over the launch's CUDA-event time and the SM count, per ns;
//  [3] the SM clock in GHz: clock64 cycles over %globaltimer ns, mean over CTAs.
void other_readings(const std::vector<long long>& cyc, const std::vector<int>& sm,
                    const std::vector<unsigned long long>& ns, double event_ms, int sms, double* out) {
    const int max_sm = *std::max_element(sm.begin(), sm.end()) + 1;
    std::vector<unsigned long long> first(max_sm, ~0ull), last(max_sm, 0ull);
    std::vector<int> ctas(max_sm, 0);
    double ghz_sum = 0.0;
    int ghz_n = 0;
    for (size_t b = 0; b < cyc.size(); ++b) {
        if (sm[b] < 0) continue;
        const unsigned long long g0 = ns[2 * b], g1 = ns[2 * b + 1];
        first[sm[b]] = std::min(first[sm[b]], g0);
        last[sm[b]] = std::max(last[sm[b]], g1);
        ctas[sm[b]] += 1;
        if (g1 > g0) {
            ghz_sum += (double)cyc[b] / (double)(g1 - g0);
            ++ghz_n;
        }
    }
    const double ghz = ghz_n ? ghz_sum / ghz_n : 0.0;
    const double per_cta = (double)kProbeThreads * kProbeChains * kProbeIter;
    double sum = 0.0;
    int used = 0;
    for (int s = 0; s < max_sm; ++s) {
        if (ctas[s] == 0 || last[s] <= first[s]) continue;
        sum += ctas[s] * per_cta / ((double)(last[s] - first[s]) * ghz);
        ++used;
    }
    out[1] = used && ghz > 0.0 ? sum / used : 0.0;
    out[2] = event_ms > 0.0 ? per_cta * (double)cyc.size() / (event_ms * 1e6) / sms : 0.0;
    out[3] = ghz;
}

}  // namespace

}  // namespace ptsdf

using namespace ptsdf;

extern "C" sdf_status sdf_probe_timing(int32_t op, double* out) {
    if (!out || op < 0 || op > 7) return set_error(SDF_EINVAL, "sdf_probe_timing: op in [0, 7] and non-NULL out");
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_error(e, "sdf_probe_timing: device query");
    const int blocks = sms * kProbeCtasPerSm;
    float* sink = nullptr;
    long long* cyc = nullptr;
    int* smid = nullptr;
    unsigned long long* ns = nullptr;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    e = cudaMalloc(&sink, (size_t)blocks * kProbeThreads * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&cyc, (size_t)blocks * sizeof(long long));
    if (e == cudaSuccess) e = cudaMalloc(&smid, (size_t)blocks * sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&ns, (size_t)blocks * 2 * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaEventCreate(&ev0);
    if (e == cudaSuccess) e = cudaEventCreate(&ev1);
    using Kern = void (*)(float*, long long*, int*, unsigned long long*);
    const Kern kernels[8] = {k_probe<0>, k_probe<1>, k_probe<2>, k_probe<3>,
                             k_probe<4>, k_probe<5>, k_probe<6>, k_probe<7>};
    float ms = 0.f;
    for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {   // the first run warms up
        e = cudaEventRecord(ev0);
        if (e == cudaSuccess) {
            kernels[op]<<<blocks, kProbeThreads>>>(sink, cyc, smid, ns);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaEventRecord(ev1);
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ev0, ev1);
    }
    std::vector<long long> hc(blocks);
    std::vector<int> hs(blocks);
    std::vector<unsigned long long> hn(2 * (size_t)blocks);
    if (e == cudaSuccess) e = cudaMemcpy(hc.data(), cyc, blocks * sizeof(long long), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(hs.data(), smid, blocks * sizeof(int), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess)
        e = cudaMemcpy(hn.data(), ns, 2 * (size_t)blocks * sizeof(unsigned long long), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) {
        out[0] = sm_rate(hc, hs);
        other_readings(hc, hs, hn, (double)ms, sms, out);
    }
    if (ev0) cudaEventDestroy(ev0);
    if (ev1) cudaEventDestroy(ev1);
    cudaFree(sink);
    cudaFree(cyc);
    cudaFree(smid);
    cudaFree(ns);
    return e == cudaSuccess ? SDF_OK : cuda_error(e, "sdf_probe_timing");
}

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
    unsigned long long* ns = nullptr;
    e = cudaMalloc(&sink, (size_t)blocks * kProbeThreads * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&cyc, (size_t)blocks * sizeof(long long));
    if (e == cudaSuccess) e = cudaMalloc(&smid, (size_t)blocks * sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&ns, (size_t)blocks * 2 * sizeof(unsigned long long));
    std::vector<long long> hc(blocks);
    std::vector<int> hs(blocks);
    std::vector<unsigned long long> hn(2 * (size_t)blocks);
    using Kern = void (*)(float*, long long*, int*, unsigned long long*);
    const Kern kernels[8] = {k_probe<0>, k_probe<1>, k_probe<2>, k_probe<3>,
                             k_probe<4>, k_probe<5>, k_probe<6>, k_probe<7>};
    for (int op = 0; op < 8 && e == cudaSuccess; ++op) {
        for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {   // the first run warms up
            kernels[op]<<<blocks, kProbeThreads>>>(sink, cyc, smid, ns);
            e = cudaGetLastError();
            if (e == cudaSuccess) e = cudaDeviceSynchronize();
        }
        if (e == cudaSuccess) e = cudaMemcpy(hc.data(), cyc, blocks * sizeof(long long), cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) e = cudaMemcpy(hs.data(), smid, blocks * sizeof(int), cudaMemcpyDeviceToHost);
        if (e == cudaSuccess)
            e = cudaMemcpy(hn.data(), ns, 2 * (size_t)blocks * sizeof(unsigned long long), cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) {
            double r[4] = {0, 0, 0, 0};
            other_readings(hc, hs, hn, 0.0, sms, r);
            rates[op] = r[1];
        }
    }
    cudaFree(sink);
    cudaFree(cyc);
    cudaFree(smid);
    cudaFree(ns);
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

// ---------------------------------------------------------------------------
// Accuracy of sqrt2_newton (the FMA-pipe square root of the tensor-core
// epilogue) against CUDA's correctly rounded sqrtf: every positive normal
// float whose bit pattern is a multiple of 64 (2^25 inputs from 1.2e-38 to
// 3.4e38), as relative errors; the largest is returned.
// ---------------------------------------------------------------------------
namespace ptsdf {
namespace {

__global__ void k_soft_sqrt_check(uint32_t n, unsigned int* worst_bits) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float x0 = __uint_as_float(0x00800000u + 128u * i), x1 = __uint_as_float(0x00800000u + 128u * i + 64u);
    const f32x2 r = sqrt2_newton(x0, x1);
    float e = 0.f;
    if (x0 >= 1e-30f) e = fmaxf(e, fabsf(f2_lo(r) - sqrtf(x0)) / sqrtf(x0));
    if (x1 >= 1e-30f) e = fmaxf(e, fabsf(f2_hi(r) - sqrtf(x1)) / sqrtf(x1));
    if (!(e == e)) e = 1.f;   // a NaN counts as a total miss
    atomicMax(worst_bits, __float_as_uint(e));
}

}  // namespace
}  // namespace ptsdf

extern "C" sdf_status sdf_selftest_soft_sqrt(double* max_rel_err) {
    if (!max_rel_err) return set_error(SDF_EINVAL, "sdf_selftest_soft_sqrt: NULL output");
    // normal floats 0x00800000 .. 0x7f7fffff, two per thread, 64 bit patterns apart
    const uint32_t n = (0x7f7fffffu - 0x00800000u) / 128u;
    unsigned int* d = nullptr;
    cudaError_t e = cudaMalloc(&d, sizeof(unsigned int));
    if (e == cudaSuccess) e = cudaMemset(d, 0, sizeof(unsigned int));
    if (e == cudaSuccess) {
        k_soft_sqrt_check<<<(n + 255) / 256, 256>>>(n, d);
        e = cudaGetLastError();
    }
    unsigned int h = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&h, d, sizeof(h), cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess) return cuda_error(e, "sdf_selftest_soft_sqrt");
    float f;
    std::memcpy(&f, &h, sizeof(f));
    *max_rel_err = (double)f;
    return SDF_OK;
}
