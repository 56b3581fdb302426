// FP32 CUDA-core contraction over the sites, row-reduced per sample:
//   U[s][j] = sum_{i <= n} sigma'[s][i] X[j][i],   sigma'[s][n] = 1,
// for a tile of 64 samples and every j-tile of 64 rows of X (complex or real),
// handing each finished 64 x 64 tile of U to an epilogue that folds it into a
// per-sample FP64 accumulator.  This is the "plain FP32" path of the theta
// contraction (theta = W sigma + b) and of the forward half of the SR matvec.
#pragma once

#include "common.cuh"

namespace nk {

constexpr int kSgBS = 64;  // samples per CTA
constexpr int kSgBJ = 64;  // rows of X per j-tile
constexpr int kSgBK = 16;  // sites per K chunk
constexpr int kSgThreads = 256;

template <bool CPLX>
struct SgTypes;
template <>
struct SgTypes<true> {
  using F = float2;
};
template <>
struct SgTypes<false> {
  using F = float;
};

// The CTA's sample tile is bx (blockIdx.x when bx < 0).
// Thread (tx, ty) = (tid % 16, tid / 16) owns samples s0 + 4 ty + p (p < 4) and
// rows j0 + tx + 16 q (q < 4).  Epi::tile(acc, s_base, j_base, part) folds the
// tile into part[p] (one complex-double partial per owned sample); after the
// last j-tile the 16 partials of a sample are summed over tx and
// Epi::finish(s, sum) is called by the thread with tx == 0.
// COMP: every 16-site chunk is summed in a fresh FP32 accumulator and added to
// the running sum with TwoSum (Knuth), its rounding error carried separately, so
// that the result is accurate to about one FP32 rounding instead of growing
// with the number of sites (used where theta itself is the output).
__device__ __forceinline__ void two_sum_acc(float& s, float& c, float x) {
  const float t = s + x;
  const float bp = t - s;
  c += (s - (t - bp)) + (x - bp);
  s = t;
}

template <bool CPLX, class Epi, bool COMP = false>
__device__ __forceinline__ void sgemm_rowreduce(const int8_t* __restrict__ sigma, int64_t ns,
                                                int n, const void* __restrict__ Xv, int rows,
                                                int ld, Epi& epi, int bx = -1) {
  using F = typename SgTypes<CPLX>::F;
  const F* X = reinterpret_cast<const F*>(Xv);
  __shared__ __align__(16) float Ss[kSgBK][kSgBS];
  __shared__ __align__(16) F Xs[kSgBK][kSgBJ];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int64_t s0 = (int64_t)(bx < 0 ? (int)blockIdx.x : bx) * kSgBS;
  const int K = n + 1;
  double2 part[4];
#pragma unroll
  for (int p = 0; p < 4; ++p) part[p] = make_double2(0.0, 0.0);

  for (int j0 = 0; j0 < rows; j0 += kSgBJ) {
    float acc_r[4][4], acc_i[4][4];
    float sr[COMP ? 4 : 1][4], si[COMP ? 4 : 1][4], cr[COMP ? 4 : 1][4], ci[COMP ? 4 : 1][4];
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        acc_r[p][q] = acc_i[p][q] = 0.f;
        if constexpr (COMP) sr[p][q] = si[p][q] = cr[p][q] = ci[p][q] = 0.f;
      }
    for (int k0 = 0; k0 < K; k0 += kSgBK) {
      // sigma' tile: 64 samples x 16 sites, 4 per thread
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        int e = tid + u * kSgThreads;  // 0..1023
        int ss = e >> 4, kk = e & 15;
        int64_t s = s0 + ss;
        int i = k0 + kk;
        float v = 0.f;
        if (s < ns) v = (i < n) ? (float)sigma[s * n + i] : (i == n ? 1.f : 0.f);
        Ss[kk][ss] = v;
      }
      // X tile: 64 rows x 16 sites, 4 per thread
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        int e = tid + u * kSgThreads;
        int jj = e >> 4, kk = e & 15;
        int j = j0 + jj, i = k0 + kk;
        F v;
        if constexpr (CPLX) v = make_float2(0.f, 0.f); else v = 0.f;
        if (j < rows && i < K) v = X[(int64_t)j * ld + i];
        Xs[kk][jj] = v;
      }
      __syncthreads();
#pragma unroll
      for (int kk = 0; kk < kSgBK; ++kk) {
        float4 a = *reinterpret_cast<const float4*>(&Ss[kk][ty * 4]);
        float av[4] = {a.x, a.y, a.z, a.w};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          F x = Xs[kk][tx + 16 * q];
#pragma unroll
          for (int p = 0; p < 4; ++p) {
            if constexpr (CPLX) {
              acc_r[p][q] = fmaf(av[p], x.x, acc_r[p][q]);
              acc_i[p][q] = fmaf(av[p], x.y, acc_i[p][q]);
            } else {
              acc_r[p][q] = fmaf(av[p], x, acc_r[p][q]);
            }
          }
        }
      }
      __syncthreads();
      if constexpr (COMP) {
#pragma unroll
        for (int p = 0; p < 4; ++p)
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            two_sum_acc(sr[p][q], cr[p][q], acc_r[p][q]);
            acc_r[p][q] = 0.f;
            if constexpr (CPLX) {
              two_sum_acc(si[p][q], ci[p][q], acc_i[p][q]);
              acc_i[p][q] = 0.f;
            }
          }
      }
    }
    if constexpr (COMP) {
#pragma unroll
      for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          acc_r[p][q] = sr[p][q] + cr[p][q];
          acc_i[p][q] = si[p][q] + ci[p][q];
        }
    }
    epi.tile(acc_r, acc_i, s0 + ty * 4, j0 + tx, part);
  }
  // reduce partials over the 16 threads (tx) sharing the samples: lanes
  // tid ^ 1, 2, 4, 8 are in the same warp
#pragma unroll
  for (int p = 0; p < 4; ++p) {
#pragma unroll
    for (int off = 8; off >= 1; off >>= 1) {
      part[p].x += __shfl_xor_sync(0xffffffffu, part[p].x, off);
      part[p].y += __shfl_xor_sync(0xffffffffu, part[p].y, off);
    }
  }
  if (tx == 0) {
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      int64_t s = s0 + ty * 4 + p;
      if (s < ns) epi.finish(s, part[p]);
    }
  }
}

}  // namespace nk
