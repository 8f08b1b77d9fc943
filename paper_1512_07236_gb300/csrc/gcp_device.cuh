// Device helpers shared by the kernels of libgcp.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

namespace gcp {

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_min(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Block-wide sum of NV doubles per thread (blockDim.x a multiple of 32,
// <= 1024).  Deterministic: fixed shuffle tree, then warps in order.
// Result valid in thread 0.  `sh` holds >= 32*NV doubles.
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV], double* sh) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) v[k] = warp_sum(v[k]);
  __syncthreads();
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) sh[warp * NV + k] = v[k];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      double s = 0.0;
      for (int w = 0; w < nw; ++w) s += sh[w * NV + k];
      v[k] = s;
    }
  }
  __syncthreads();
}

// Split a value of the shifted state into two 16-bit halves,
//   h = rn(v), l = rn(v - h),  v ~ h + l,
// where v is the FP32 value already multiplied by the global split scale
// (2^14).  Both halves are stored at their true weight so that all three
// products accumulate into one accumulator.  For fp16 the scale keeps
// every |v| >= 2^-3 in the normal range of the remainder l (fp16 normals
// start at 2^-14), so l carries 11 bits; smaller elements keep an absolute
// error below 2^-25 / 2^14.  |X| <= 1.5 keeps |v| below the fp16 maximum.
template <bool BF16>
struct Split;

template <>
struct Split<false> {
  using T = __half;
  __device__ __forceinline__ static void split(float v, T& h, T& l) {
    h = __float2half_rn(v);
    l = __float2half_rn(v - __half2float(h));
  }
};

template <>
struct Split<true> {
  using T = __nv_bfloat16;
  __device__ __forceinline__ static void split(float v, T& h, T& l) {
    h = __float2bfloat16_rn(v);
    l = __float2bfloat16_rn(v - __bfloat162float(h));
  }
};

}  // namespace gcp
