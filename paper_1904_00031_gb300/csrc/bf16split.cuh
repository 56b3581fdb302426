// BF16 hi + lo splits of FP32 / FP64 values (the tensor-core operand planes):
// hi = bf16(x), lo = bf16(x - hi), both round-to-nearest-even.
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

namespace nk {

__device__ __forceinline__ uint32_t bf16_bits(float x) {
  return (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(x));
}
__device__ __forceinline__ float bf16_val(uint32_t b) {
  return __bfloat162float(__ushort_as_bfloat16((unsigned short)b));
}
// hi = bf16(x), lo = bf16(x - hi)
__device__ __forceinline__ void split_bf16(float x, uint32_t& hi, uint32_t& lo) {
  hi = bf16_bits(x);
  lo = bf16_bits(x - bf16_val(hi));
}
// The same split of two values at once, packed (a in the low half): the paired
// conversions give bit for bit the results of two split_bf16 calls.
__device__ __forceinline__ void split_bf16x2(float a, float b, uint32_t& hi, uint32_t& lo) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  const float2 hf = __bfloat1622float2(h);
  const __nv_bfloat162 l = __floats2bfloat162_rn(a - hf.x, b - hf.y);
  hi = *reinterpret_cast<const uint32_t*>(&h);
  lo = *reinterpret_cast<const uint32_t*>(&l);
}
// FP64 input: rounded to FP32 first (one conversion; the FP64 pipe is slow on
// this GPU), which perturbs hi + lo by at most 2^-24 relative, far below the
// 2^-17 of the two-term split itself
__device__ __forceinline__ void split_bf16(double x, uint32_t& hi, uint32_t& lo) {
  split_bf16((float)x, hi, lo);
}

// Position of element (j, i, comp) of an augmented [rows][na] matrix (comp: 0 =
// Re, 1 = Im of a complex one) in its hi plane of [mt*128][na64] BF16 (the lo
// plane follows at + mt*128*na64): a tile of 128 plane rows holds Re and Im of 64
// rows of a complex matrix, or 128 rows of a real one.
__host__ __device__ __forceinline__ int64_t bplane_index(int j, int i, int comp, int cplx,
                                                         int na64) {
  const int row = cplx ? (j >> 6) * 128 + comp * 64 + (j & 63) : j;
  return (int64_t)row * na64 + i;
}

}  // namespace nk
