// Device-side helpers: approximate MUFU math, mbarriers, bulk (TMA) copies,
// and a bounded wait that reports a timeout through the device status word
// instead of hanging or trapping.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "ptsdf.h"

namespace ptsdf {

// --------------------------------------------------------------------------
// Approximate special functions (one MUFU instruction each).
// --------------------------------------------------------------------------
__device__ __forceinline__ float sqrt_mufu(float x) {
    float y;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float rsqrt_mufu(float x) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float rcp_mufu(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float ex2_mufu(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// --------------------------------------------------------------------------
// Pairs of FP32 values in one 64-bit register pair, with the sm_100+ .f32x2
// arithmetic: one instruction does the add / sub / mul / fma of both halves
// (round to nearest, as the scalar forms), halving the issue slots of code
// that does the same arithmetic for two queries.
// --------------------------------------------------------------------------
typedef unsigned long long f32x2;

__device__ __forceinline__ f32x2 f2_pack(float lo, float hi) {
    f32x2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ float f2_lo(f32x2 v) {
    float lo;
    asm("mov.b64 {%0, _}, %1;" : "=f"(lo) : "l"(v));
    return lo;
}
__device__ __forceinline__ float f2_hi(f32x2 v) {
    float hi;
    asm("mov.b64 {_, %0}, %1;" : "=f"(hi) : "l"(v));
    return hi;
}
__device__ __forceinline__ f32x2 f2_add(f32x2 a, f32x2 b) {
    f32x2 r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f32x2 f2_sub(f32x2 a, f32x2 b) {
    f32x2 r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f32x2 f2_mul(f32x2 a, f32x2 b) {
    f32x2 r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f32x2 f2_fma(f32x2 a, f32x2 b, f32x2 c) {
    f32x2 r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}

// sqrt(x0), sqrt(x1) for x >= 0 without the special-function unit (on the
// integer and FMA pipes, the latter as .f32x2): 1/sqrt(x) starts from the
// bit-level estimate of Lomont, "Fast Inverse Square Root" (2003): the
// integer 0x5f375a86 minus half of x's bit pattern, within 3.5% of 1/sqrt(x);
// then two Newton-Raphson steps for 1/y^2 = x, y <- y (c - x y^2 / 2), and
// sqrt(x) = x y.  With c = 3/2 each step squares the relative error and
// leaves y below 1/sqrt(x) (about -1.8e-3, then -4.7e-6).  Raising c by
// delta lifts a step's result by about delta times itself: c1 = 1.5009 and
// c2 = 1.5000006 centre the two error intervals (found by sweeping the
// constants over one period of the estimate), within 7.6e-7 relative, but
// the tensor-core pair loop compiled with them ran 1.2% slower (the two
// constants changed its register allocation), so 3/2 stays the default.
// x is clamped to >= 1e-30 (a zero comes out as 1e-15).
#ifndef PTSDF_SQRT_C1
#define PTSDF_SQRT_C1 1.5f   // the first step's constant (1.5009f: centred)
#endif
#ifndef PTSDF_SQRT_C2
#define PTSDF_SQRT_C2 1.5f   // the second step's (1.5000006f: centred)
#endif
__device__ __forceinline__ f32x2 sqrt2_newton(float x0, float x1) {
    x0 = fmaxf(x0, 1e-30f);
    x1 = fmaxf(x1, 1e-30f);
    const f32x2 X = f2_pack(x0, x1);
    const f32x2 NH = f2_mul(X, f2_pack(-0.5f, -0.5f));
    f32x2 Y = f2_pack(__int_as_float(0x5f375a86 - (__float_as_int(x0) >> 1)),
                      __int_as_float(0x5f375a86 - (__float_as_int(x1) >> 1)));
    Y = f2_mul(Y, f2_fma(NH, f2_mul(Y, Y), f2_pack(PTSDF_SQRT_C1, PTSDF_SQRT_C1)));
    Y = f2_mul(Y, f2_fma(NH, f2_mul(Y, Y), f2_pack(PTSDF_SQRT_C2, PTSDF_SQRT_C2)));
    return f2_mul(X, Y);
}

// --------------------------------------------------------------------------
// Shared-memory addresses, mbarriers and bulk copies (sm_90+ PTX).
// --------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// 1-D bulk copy global -> shared through the TMA unit, completing on `bar`.
// dst and src 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Any legitimate wait in these kernels lasts microseconds; after this long a
// wait gives up, records SDF_DEV_WAIT_TIMEOUT and the CTA winds down.
constexpr uint64_t kWaitLimitNs = 2000000000ull;

// Bounded wait on one mbarrier phase.  Returns false (and raises `abort` for
// the whole CTA) if the phase did not complete within limit_ns or another
// thread of the CTA already aborted; a timeout also sets SDF_DEV_WAIT_TIMEOUT
// in the device status word.
__device__ __forceinline__ bool mbar_wait_bounded_ns(uint64_t* bar, uint32_t parity, volatile int* abort,
                                                     int32_t* status, uint64_t limit_ns) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    while (true) {
        if (mbar_try_wait(bar, parity)) return true;
        if (*abort) return false;
        if (global_ns() - t0 > limit_ns) {
            *abort = 1;
            atomicOr(status, (int32_t)SDF_DEV_WAIT_TIMEOUT);
            return false;
        }
    }
}

__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, volatile int* abort,
                                                  int32_t* status) {
    return mbar_wait_bounded_ns(bar, parity, abort, status, kWaitLimitNs);
}

// --------------------------------------------------------------------------
// A ring of kStages tiles filled by one producer lane with bulk copies and
// drained by `consumers` warps (one mbarrier arrive per warp per tile).
// --------------------------------------------------------------------------
template <int STAGES>
struct TileRing {
    uint64_t full[STAGES];
    uint64_t empty[STAGES];
    int abort;

    __device__ void init(uint32_t consumer_warps) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], consumer_warps);
        }
        abort = 0;
        fence_mbar_init();
    }

    // Producer: copies tiles [0, ntiles) of `bytes` each from src into the
    // ring buffers `buf + s * bytes`.  On abort it waits (bounded) for the
    // copies it already issued, so none is in flight when the CTA exits.
    __device__ void produce(char* buf, const char* src, int64_t ntiles, uint32_t bytes, int32_t* status) {
        int64_t issued = 0;
        for (int64_t t = 0; t < ntiles; ++t) {
            const int s = (int)(t % STAGES);
            if (t >= STAGES) {
                if (!mbar_wait_bounded(&empty[s], (uint32_t)(((t / STAGES) - 1) & 1), &abort, status)) break;
            }
            mbar_arrive_expect_tx(&full[s], bytes);
            bulk_g2s(buf + (size_t)s * bytes, src + (size_t)t * bytes, bytes, &full[s]);
            issued = t + 1;
        }
        if (*(volatile int*)&abort) {
            for (int64_t t = (issued > STAGES ? issued - STAGES : 0); t < issued; ++t) {
                const int s = (int)(t % STAGES);
                const uint64_t t0 = global_ns();
                while (!mbar_try_wait(&full[s], (uint32_t)((t / STAGES) & 1))) {
                    if (global_ns() - t0 > kWaitLimitNs) break;
                }
            }
        }
    }

    __device__ bool wait_full(int64_t t, int32_t* status) {
        return mbar_wait_bounded(&full[t % STAGES], (uint32_t)((t / STAGES) & 1), &abort, status);
    }
    __device__ void release(int64_t t, int lane) {
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[t % STAGES]);
    }
};

}  // namespace ptsdf
