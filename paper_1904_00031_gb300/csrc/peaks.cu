// Measured ALU peaks of the current GPU: packed FP32 FMA throughput and the
// MUFU (special-function unit) throughput of ex2 / lg2 / sin.  These are the
// denominators of the roofline of the kernels bound by plain arithmetic
// (Metropolis, local energies), which no copy or GEMM measurement gives.
// Each thread runs 8 independent dependency chains so that latency is hidden.
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"
#include "internal.h"

namespace nk {

namespace {

constexpr int kPeakThreads = 256;
constexpr int kPeakChains = 8;

__device__ float g_peak_sink;

__global__ void __launch_bounds__(kPeakThreads) fma2_peak_kernel(int iters, float seed) {
  float2 x[kPeakChains];
  const float2 a = make_float2(0.999f, 0.998f), b = make_float2(1e-3f, 2e-3f);
#pragma unroll
  for (int c = 0; c < kPeakChains; ++c) x[c] = make_float2(seed + c, seed - c);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < kPeakChains; ++c) x[c] = __ffma2_rn(x[c], a, b);
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kPeakChains; ++c) s += x[c].x + x[c].y;
  if (s == 1234.5f) g_peak_sink = s;  // keeps the chains live
}

template <int OP>
__device__ __forceinline__ float mufu(float x) {
  float y;
  if (OP == 0) asm volatile("ex2.approx.f32 %0, %1;" : "=f"(y) : "f"(-x));  // x -> 2^-x
  if (OP == 1) asm volatile("lg2.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
  if (OP == 2) asm volatile("sin.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

template <int OP>
__global__ void __launch_bounds__(kPeakThreads) mufu_peak_kernel(int iters, float seed) {
  float x[kPeakChains];
#pragma unroll
  for (int c = 0; c < kPeakChains; ++c) x[c] = 1.5f + 0.1f * c + seed;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < kPeakChains; ++c) {
      if (OP == 1) x[c] = mufu<1>(x[c]) + 2.f;  // stays in [2, 4]
      else x[c] = mufu<OP>(x[c]);
    }
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kPeakChains; ++c) s += x[c];
  if (s == 1234.5f) g_peak_sink = s;
}

// Seconds of the fastest of `reps` timed launches (after one warm-up).
template <typename K>
double time_kernel(K kern, int blocks, int iters, cudaStream_t st, int reps, nk_status* err) {
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    *err = fail(NK_ERR_CUDA, "nk_measure_alu_peaks: cannot create events");
    return 0.0;
  }
  float best = 1e30f;
  for (int r = 0; r <= reps; ++r) {
    cudaEventRecord(e0, st);
    kern<<<blocks, kPeakThreads, 0, st>>>(iters, 0.25f);
    cudaEventRecord(e1, st);
    if (cudaEventSynchronize(e1) != cudaSuccess) {
      *err = fail(NK_ERR_CUDA, "nk_measure_alu_peaks: kernel failed");
      break;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (r > 0 && ms < best) best = ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (*err == NK_OK) *err = check_launch("nk_measure_alu_peaks");
  return best * 1e-3;
}

}  // namespace

nk_status measure_alu_peaks(double* out, cudaStream_t st) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return fail(NK_ERR_CUDA, "nk_measure_alu_peaks: no device");
  const int blocks = sms * 8;  // 8 CTAs of 256 threads per SM: 64 warps
  const double threads = (double)blocks * kPeakThreads;
  nk_status err = NK_OK;
  const int fit = 1 << 14, mit = 1 << 12;
  double t = time_kernel(fma2_peak_kernel, blocks, fit, st, 3, &err);
  if (err) return err;
  out[0] = threads * fit * kPeakChains * 4.0 / t;  // FFMA2: 2 lanes x 2 flop
  t = time_kernel(mufu_peak_kernel<0>, blocks, mit, st, 3, &err);
  if (err) return err;
  out[1] = threads * mit * kPeakChains / t;
  t = time_kernel(mufu_peak_kernel<1>, blocks, mit, st, 3, &err);
  if (err) return err;
  out[2] = threads * mit * kPeakChains / t;
  t = time_kernel(mufu_peak_kernel<2>, blocks, mit, st, 3, &err);
  if (err) return err;
  out[3] = threads * mit * kPeakChains / t;
  return NK_OK;
}

}  // namespace nk
