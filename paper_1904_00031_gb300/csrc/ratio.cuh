// Amplitude ratios of an RBM for one- and two-spin moves, evaluated by a warp
// that holds t_j = tanh(theta_j) of one configuration in registers
// (lane l owns hidden units j = l + 32 q).
//
// For spins s_i (and s_k) flipped, theta' = theta - 2 s_i W_i (- 2 s_k W_k) and
//   psi(sigma')/psi(sigma) = exp(-2 s_i a_i (- 2 s_k a_k)) prod_j r_j,
//   r_j = cosh(theta_j - c_j)/cosh(theta_j) = cosh c_j - t_j sinh c_j,
// with c = 2 s_i W_i (+ 2 s_k W_k).  From the tables A = cosh 2W, B = sinh 2W:
//   one spin:  cosh c = A_i,                 sinh c = s_i B_i
//   two spins: cosh c = A_i A_k + s_i s_k B_i B_k,
//              sinh c = s_i B_i A_k + s_k A_i B_k.
#pragma once

#include "common.cuh"

namespace nk {

template <bool CPLX>
struct RatioTypes;
template <>
struct RatioTypes<true> {
  using F = float2;   // theta, W
  using T2 = float4;  // (A, B) complex
};
template <>
struct RatioTypes<false> {
  using F = float;
  using T2 = float2;
};

// Running product kept as mantissa * 2^expo so that products of thousands of
// factors neither overflow nor underflow.  Renormalised every 4 factors; each
// factor must lie in (2^-31, 2^31) in modulus (|Re W| < ~5 for the RBM ratios).
struct ScaledReal {
  float v;
  int e;
  __device__ __forceinline__ void init() { v = 1.f; e = 0; }
  __device__ __forceinline__ void renorm() {
    if (v == 0.f) return;
    int b = __float_as_int(v);
    int ex = ((b >> 23) & 0xff) - 127;
    v = __int_as_float((b & 0x807fffff) | (127 << 23));
    e += ex;
  }
  // log2 of the value
  __device__ __forceinline__ float log2v() const { return (float)e + __log2f(v); }
};

struct ScaledComplex {
  cf v;
  int e;
  __device__ __forceinline__ void init() { v = cf{1.f, 0.f}; e = 0; }
  __device__ __forceinline__ void renorm() {
    float mx = fmaxf(fabsf(v.x), fabsf(v.y));
    int ex = ((__float_as_int(mx) >> 23) & 0xff) - 127;
    if (mx == 0.f) ex = 0;
    float sc = __int_as_float((127 - ex) << 23);
    v = cf{v.x * sc, v.y * sc};
    e += ex;
  }
};

__device__ __forceinline__ void mul_scaled(ScaledComplex& a, const ScaledComplex& b) {
  a.v = a.v * b.v;
  a.e += b.e;
  a.renorm();
}

// cosh c, sinh c of a one-spin move from the table entry of site i
__device__ __forceinline__ void move_coef(float2 ab, float si, float& C, float& S) {
  C = ab.x;
  S = si * ab.y;
}
__device__ __forceinline__ void move_coef(float4 ab, float si, cf& C, cf& S) {
  C = cf{ab.x, ab.y};
  S = cf{si * ab.z, si * ab.w};
}
// two-spin move from the entries of sites i and k
__device__ __forceinline__ void move_coef2(float2 ai, float2 ak, float si, float sk, float& C,
                                           float& S) {
  float sik = si * sk;
  C = fmaf(sik * ai.y, ak.y, ai.x * ak.x);
  S = fmaf(si * ai.y, ak.x, sk * ai.x * ak.y);
}
__device__ __forceinline__ void move_coef2(float4 ai, float4 ak, float si, float sk, cf& C,
                                           cf& S) {
  cf Ai{ai.x, ai.y}, Bi{ai.z, ai.w}, Ak{ak.x, ak.y}, Bk{ak.z, ak.w};
  C = Ai * Ak + (si * sk) * (Bi * Bk);
  S = si * (Bi * Ak) + sk * (Ai * Bk);
}

}  // namespace nk
