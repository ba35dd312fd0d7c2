// Loads from the two storage precisions of P and Y: FP32, or BF16 (read
// into FP32; all arithmetic stays FP32, Z FP64).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstddef>

namespace tsgne {

typedef __nv_bfloat16 bf16;
typedef __nv_bfloat162 bf162;

__device__ __forceinline__ float2 ld_y(const float2* __restrict__ p, size_t i) { return p[i]; }
__device__ __forceinline__ float2 ld_y(const bf162* __restrict__ p, size_t i) { return __bfloat1622float2(p[i]); }
__device__ __forceinline__ float ld_p(const float* __restrict__ p, size_t e) { return p[e]; }
__device__ __forceinline__ float ld_p(const bf16* __restrict__ p, size_t e) { return __bfloat162float(p[e]); }

}  // namespace tsgne
