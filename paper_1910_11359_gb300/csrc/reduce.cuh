// Block reductions by warp shuffles: each warp reduces its 32 values with __shfl_xor_sync, the
// per-warp results meet in shared memory once, and warp 0 reduces those.  Fixed order, so the
// result does not depend on scheduling.  NT is the block size (a multiple of 32, at most 1024);
// every thread of the block must call, and every thread receives the result.
#pragma once
#include "common.cuh"

namespace ipeps {

template <int NT>
__device__ __forceinline__ double block_max(double v) {
  static_assert(NT % 32 == 0 && NT <= 1024, "block size");
  __shared__ double part[NT / 32];
  __shared__ double out;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) part[w] = v;
  __syncthreads();
  if (w == 0) {
    double x = lane < NT / 32 ? part[lane] : part[0];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x = fmax(x, __shfl_xor_sync(0xffffffffu, x, o));
    if (lane == 0) out = x;
  }
  __syncthreads();
  return out;
}

template <int NT>
__device__ __forceinline__ cplx block_sum(cplx v) {
  static_assert(NT % 32 == 0 && NT <= 1024, "block size");
  __shared__ cplx part[NT / 32];
  __shared__ cplx out;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
    v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
  }
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) part[w] = v;
  __syncthreads();
  if (w == 0) {
    cplx x = lane < NT / 32 ? part[lane] : cmk(0.0, 0.0);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      x.x += __shfl_xor_sync(0xffffffffu, x.x, o);
      x.y += __shfl_xor_sync(0xffffffffu, x.y, o);
    }
    if (lane == 0) out = x;
  }
  __syncthreads();
  return out;
}

}  // namespace ipeps
