// Deterministic reductions: fixed-order trees, no floating-point atomics, so
// every result is bit-reproducible from run to run.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace tsgne {

// Sum of one double per thread over the CTA: xor butterfly in each warp, then
// warp 0 over the warp sums.  The result is valid in every lane of warp 0.
// Must be reached by every thread of the CTA.
__device__ __forceinline__ double block_sum_d(double v) {
  __shared__ double ws[32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if (lane == 0) ws[wid] = v;
  __syncthreads();
  double r = 0.0;
  if (wid == 0) {
    r = lane < nw ? ws[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
  }
  __syncthreads();
  return r;
}

// Called by every thread of every CTA after the CTA has written its partial
// result.  Returns true (uniformly within the CTA) in exactly one CTA: the
// last one to arrive, which also resets the counter for the next launch.
// The writes of all other CTAs are visible to it (fence / counter / fence).
__device__ __forceinline__ bool arrive_last(uint32_t* counter) {
  __shared__ bool last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const uint32_t total = gridDim.x * gridDim.y * gridDim.z;
    const uint32_t prev = atomicAdd(counter, 1u);
    last = (prev == total - 1u);
    if (last) atomicExch(counter, 0u);
  }
  __syncthreads();
  if (last) __threadfence();
  return last;
}

// Sum of parts[0..count) by one CTA in a fixed order (strided per thread, then
// block_sum_d).  L1 is bypassed so partials written by other CTAs are seen.
__device__ __forceinline__ double sum_partials(const double* parts, int count) {
  double s = 0.0;
  for (int k = threadIdx.x; k < count; k += blockDim.x) s += __ldcg(parts + k);
  return block_sum_d(s);
}

}  // namespace tsgne
