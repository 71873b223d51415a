// tcgen05 (5th-generation tensor core) helpers: TMEM allocation, MMA issue
// from shared-memory descriptors, commit to an mbarrier, TMEM loads and the
// ordering fences.  Operands use the K-major layout without swizzle: 8-row x
// 16-byte core matrices, LBO = byte distance between the two K core matrices
// of a row group, SBO = byte distance between consecutive row groups.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "device_common.cuh"

namespace ptsdf {
namespace tc {

constexpr uint32_t kLBO = 128;   // K = 16 halves: core matrices k = 0..7 and 8..15
constexpr uint32_t kSBO = 256;   // one row group of 8 rows = 2 core matrices

// byte offset of element (row, k) of a K = 16 f16 tile in the canonical layout
__host__ __device__ __forceinline__ uint32_t canon_offset(int row, int k) {
    return (uint32_t)((row >> 3) * kSBO + (k >> 3) * kLBO + (row & 7) * 16 + (k & 7) * 2);
}

// shared-memory matrix descriptor: start address, LBO, SBO (all >> 4),
// version 1 (bits 46-48), no base offset, no swizzle
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)(kLBO >> 4) << 16) | ((uint64_t)(kSBO >> 4) << 32) |
           (1ull << 46);
}

// instruction descriptor of kind::f16: D f32, A and B f16, both K-major
__host__ __device__ constexpr uint32_t idesc_f16_f32(int m, int n) {
    return (1u << 4) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ void tmem_alloc(uint32_t* smem_dst, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(smem_dst)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// D[tmem] = A[smem] * B[smem]^T, added to D when `accumulate` is nonzero
__device__ __forceinline__ void mma_f16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                        uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// arrive (once) on `bar` when every tcgen05 operation issued so far by this thread completes
__device__ __forceinline__ void commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Starts loading 8 consecutive 32-bit columns of this thread's TMEM lane into
// v[off..off+8); the values are valid only after tmem_wait_ld_values.
template <int NV>
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float (&v)[NV], int off) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=f"(v[off]), "=f"(v[off + 1]), "=f"(v[off + 2]), "=f"(v[off + 3]), "=f"(v[off + 4]),
                   "=f"(v[off + 5]), "=f"(v[off + 6]), "=f"(v[off + 7])
                 : "r"(taddr));
}

// Starts loading 16 consecutive 32-bit columns of this thread's TMEM lane
// into v[off..off+16).
template <int NV>
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[NV], int off) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=f"(v[off]), "=f"(v[off + 1]), "=f"(v[off + 2]), "=f"(v[off + 3]), "=f"(v[off + 4]), "=f"(v[off + 5]),
          "=f"(v[off + 6]), "=f"(v[off + 7]), "=f"(v[off + 8]), "=f"(v[off + 9]), "=f"(v[off + 10]),
          "=f"(v[off + 11]), "=f"(v[off + 12]), "=f"(v[off + 13]), "=f"(v[off + 14]), "=f"(v[off + 15])
        : "r"(taddr));
}

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Waits for outstanding TMEM loads, then ties the loaded registers to the
// wait so that no use of them is scheduled before it.
template <int NV>
__device__ __forceinline__ void tmem_wait_ld_values(float (&v)[NV]) {
    tmem_wait_ld();
#pragma unroll
    for (int i = 0; i < NV; ++i) asm volatile("" : "+f"(v[i]));
}

}  // namespace tc
}  // namespace ptsdf
