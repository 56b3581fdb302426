// Shared device helpers of the nk library: complex arithmetic, Philox4x32-10,
// ln cosh / tanh in FP32, and the layout of the derived-parameter workspace.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "nk.h"

namespace nk {

// ------------------------------------------------------------------ sizes

constexpr int kWarp = 32;

__host__ __device__ inline int64_t round_up(int64_t x, int64_t a) { return (x + a - 1) / a * a; }
__host__ __device__ inline int ceil_div(int x, int a) { return (x + a - 1) / a; }

// Hidden-unit dimension padded to whole warps: lane l of a warp owns hidden
// units j = l + 32 q, q = 0 .. mp/32 - 1.  Padded entries hold W = 0, b = 0,
// cosh(2W) = 1, sinh(2W) = 0, so they contribute a ratio of exactly 1.
__host__ __device__ inline int padded_m(int m) { return (int)round_up(m, kWarp); }

// Byte offsets of the planes inside the derived workspace (all 256-B aligned).
//   a32  F32 [n]           b32  F32 [mp]
//   wt   F32 [n][mp]       W transposed: column i of W contiguous
//   tab  T2  [n][mp]       (cosh 2W_ji, sinh 2W_ji); T2 = float2 (real) or
//                          float4 (re A, im A, re B, im B) (complex)
//   xw   F32 [mp][n+1]     W | b row-major ("augmented" W, FP32), rows >= m zero
//   wbf  BF16 [2][mt*128][na64]  tensor-core operand planes of W | b (hi, lo),
//                          see tc_rows_per_tile below
struct WsLayout {
  int n, m, mp, cplx, na64, mt;
  size_t a32, b32, wt, tab, xw, wbf, total;
  __host__ __device__ WsLayout(int n_, int m_, int cplx_) : n(n_), m(m_), cplx(cplx_) {
    mp = padded_m(m);
    na64 = (int)round_up(n + 1, 64);
    mt = (m + (cplx ? 64 : 128) - 1) / (cplx ? 64 : 128);
    size_t f = cplx ? 8 : 4;  // bytes of one F32 element
    size_t off = 0;
    a32 = off;  off += round_up((int64_t)n * f, 256);
    b32 = off;  off += round_up((int64_t)mp * f, 256);
    wt = off;   off += round_up((int64_t)n * mp * f, 256);
    tab = off;  off += round_up((int64_t)n * mp * 2 * f, 256);
    xw = off;   off += round_up((int64_t)mp * (n + 1) * f, 256);
    wbf = off;  off += round_up((int64_t)2 * mt * 128 * na64 * 2, 256);
    total = off;
  }
};

// Tensor-core operand planes of a complex (or real) matrix X [rows][n+1]
// ("B planes"): BF16 [2][mt*128][na64], plane 0 = hi = bf16(X), plane 1 =
// lo = bf16(X - hi).  Tile jt covers 128 plane rows: for a complex X, rows
// 0..63 hold Re X[jt*64 + r] and rows 64..127 Im X[jt*64 + r]; for a real X,
// rows 0..127 hold X[jt*128 + r].  Entries beyond X are zero.
__host__ __device__ inline int tc_hidden_per_tile(int cplx) { return cplx ? 64 : 128; }

// ------------------------------------------------------------------ complex

struct cf {  // complex float
  float x, y;
};
__device__ __forceinline__ cf mk(float x, float y) { return cf{x, y}; }
__device__ __forceinline__ cf operator+(cf a, cf b) { return cf{a.x + b.x, a.y + b.y}; }
__device__ __forceinline__ cf operator-(cf a, cf b) { return cf{a.x - b.x, a.y - b.y}; }
__device__ __forceinline__ cf operator*(cf a, cf b) {
  return cf{fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x)};
}
__device__ __forceinline__ cf operator*(float s, cf a) { return cf{s * a.x, s * a.y}; }
__device__ __forceinline__ cf conj(cf a) { return cf{a.x, -a.y}; }

// ------------------------------------------------------------------ Philox4x32-10
// Salmon et al., SC'11.  Counter (c0..c3), key (k0, k1); ten rounds, key bumped
// by the Weyl constants between rounds.

struct u4 {
  uint32_t x, y, z, w;
};

__host__ __device__ __forceinline__ u4 philox4x32_10(u4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    uint64_t p0 = (uint64_t)0xD2511F53u * c.x;
    uint64_t p1 = (uint64_t)0xCD9E8D57u * c.z;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    c = u4{hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0};
  }
  return c;
}

constexpr uint32_t kTagSite = 0x53495445u;    // "SITE": proposal draw per group and step
constexpr uint32_t kTagAccept = 0x41434350u;  // "ACCP": accept uniform per chain and step

__host__ __device__ __forceinline__ u4 philox_stream(uint32_t index, uint64_t step, uint32_t tag,
                                                     uint64_t seed) {
  return philox4x32_10(u4{index, (uint32_t)step, (uint32_t)(step >> 32), tag}, (uint32_t)seed,
                       (uint32_t)(seed >> 32));
}

// floor(u * n / 2^32)
__host__ __device__ __forceinline__ int uniform_index(uint32_t u, int n) {
  return (int)(((uint64_t)u * (uint64_t)n) >> 32);
}
// 53-bit double in [0, 1) from 27 high bits of hi and 26 of lo
__host__ __device__ __forceinline__ double uniform53(uint32_t hi, uint32_t lo) {
  return ((double)(hi >> 5) * 67108864.0 + (double)(lo >> 6)) * (1.0 / 9007199254740992.0);
}

// ------------------------------------------------------------------ FP32 special functions

// ln cosh x = |x| + log1p(exp(-2|x|)) - ln 2
__device__ __forceinline__ float lncosh_f(float x) {
  float ax = fabsf(x);
  return ax + log1pf(expf(-2.f * ax)) - 0.69314718055994531f;
}

// ln cosh z for complex z = x + i y, s = sign(x):
//   s z + log1p(e^{-2 s z}) - ln 2,  e^{-2 s z} = e^{-2|x|} (cos 2y - i s sin 2y).
__device__ __forceinline__ cf lncosh_c(cf z) {
  float s = z.x >= 0.f ? 1.f : -1.f;
  float e = expf(-2.f * fabsf(z.x));
  float sn, cs;
  sincosf(2.f * z.y, &sn, &cs);
  float wr = e * cs, wi = -s * e * sn;
  float re = 0.5f * log1pf(fmaf(wr, 2.f, fmaf(wr, wr, wi * wi)));
  float im = atan2f(wi, 1.f + wr);
  return cf{s * z.x + re - 0.69314718055994531f, s * z.y + im};
}

// tanh x with absolute error ~1 ulp of 1 (all that the ratio formula needs).
__device__ __forceinline__ float tanh_f(float x) { return tanhf(x); }

// tanh z = (sinh x cosh x + i sin y cos y) / (sinh^2 x + cos^2 y): the usual
// denominator cosh 2x + cos 2y = 2 (sinh^2 x + cos^2 y) written without
// cancellation.  sinh x = e (2 + e) / (2 (1 + e)), e = expm1(x), is accurate at
// small x.  For |x| > 20, tanh z equals sign(x) to FP32 precision; x is clamped
// there so that nothing overflows.
__device__ __forceinline__ cf tanh_c(cf z) {
  float x = fminf(fmaxf(z.x, -20.f), 20.f);
  float em = expm1f(x);
  float sh = 0.5f * em * (2.f + em) / (1.f + em);
  float ch = sqrtf(fmaf(sh, sh, 1.f));
  float sn, cs;
  sincosf(z.y, &sn, &cs);
  float d = 1.f / fmaf(sh, sh, cs * cs);
  return cf{sh * ch * d, sn * cs * d};
}

}  // namespace nk
