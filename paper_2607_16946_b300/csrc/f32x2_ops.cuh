// Helpers over the packed .f32x2 pairs of device_common.cuh shared by the
// FP32-unit pair loops: broadcasts, the clamp at zero and the MUFU
// reciprocal of both halves (the special-function steps stay one per value).
#pragma once

#include "device_common.cuh"

namespace ptsdf {

__device__ __forceinline__ f32x2 f2_splat(float v) { return f2_pack(v, v); }
__device__ __forceinline__ f32x2 f2_max0(f32x2 v) { return f2_pack(fmaxf(f2_lo(v), 0.f), fmaxf(f2_hi(v), 0.f)); }
__device__ __forceinline__ f32x2 f2_rcp(f32x2 v) { return f2_pack(rcp_mufu(f2_lo(v)), rcp_mufu(f2_hi(v))); }
__device__ __forceinline__ f32x2 f2_sqrt(f32x2 v) { return f2_pack(sqrt_mufu(f2_lo(v)), sqrt_mufu(f2_hi(v))); }

}  // namespace ptsdf
