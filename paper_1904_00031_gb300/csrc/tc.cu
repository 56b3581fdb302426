// Tensor-core contractions of the RBM path (tcgen05, BF16 hi + lo, FP32 in TMEM).
//
// sigma' = [sigma | 1] is exact in BF16.  The other operand X (W | b, or an SR
// direction) is split as X = hi + lo with hi = bf16(X), lo = bf16(X - hi), and
// every product is accumulated from both halves in FP32 (relative error of the
// split ~2^-17 per element).
//
// Forward (theta and the O x half of the SR matvec): one CTA owns 128
// configurations; their sigma' rows stay resident in shared memory as K-major
// 128-byte-swizzled tiles (TMA-loaded from a BF16 copy of sigma' in the SR
// forward; built by the CTA from the int8 samples for theta / ln psi), the B
// planes of X stream in by TMA through a 3-stage ring, one thread issues the
// MMAs (M = 128 configurations, N = 128 plane rows, K = n + 1 padded to 64)
// into one of two TMEM accumulators, and four epilogue warps fold each
// finished 128 x 128 tile (tcgen05.ld): ln cosh sums, theta / tanh(theta)
// stores, or the T'.U dot products of the SR forward, while the next tile's
// MMAs run.  The hidden tiles may be split over two CTAs.
//
// Adjoint (the O^H v half): one CTA owns 64 complex (128 real) parameter rows
// j and a range of samples (split-K).  Eight producer warps compute
// Z = conj(T'_sj) v_s for 64 samples at a time, split it into BF16 hi/lo and
// write it, swizzled, as the A operand; sigma'^T tiles (a BF16 plane built once
// per SR step) arrive by TMA; MMAs accumulate G[j][0..n] in TMEM (two halves of
// N <= 224); the epilogue writes FP32 partials that a fixed-order reduction
// (FP32 sum plus its TwoSum error term, one FP64 conversion) sums over the
// splits.
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <mutex>
#include <type_traits>

#include "bf16split.cuh"
#include "tc.cuh"
#include "status.cuh"
#include "umma.cuh"

namespace nk {

// ------------------------------------------------------------------ tensor maps

static PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
static std::once_flag g_encode_once;

static PFN_cuTensorMapEncodeTiled_v12000 encoder() {
  std::call_once(g_encode_once, [] {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    else
      cudaGetLastError();
  });
  return g_encode;
}

bool tc_make_map(CUtensorMap* map, const void* base, int64_t rows, int64_t cols,
                 int64_t row_stride_elems, int box_rows) {
  if (!encoder()) {
    fail(NK_ERR_UNSUPPORTED, "cuTensorMapEncodeTiled is not available from the driver");
    return false;
  }
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)row_stride_elems * 2};
  cuuint32_t box[2] = {64, (cuuint32_t)box_rows};
  cuuint32_t es[2] = {1, 1};
  CUresult r = g_encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims,
                        strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    fail(NK_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    return false;
  }
  return true;
}

bool make_map_f32(CUtensorMap* map, const void* base, int64_t rows, int64_t cols,
                  int64_t stride_bytes, int box_cols, int box_rows) {
  if (!encoder()) {
    fail(NK_ERR_UNSUPPORTED, "cuTensorMapEncodeTiled is not available from the driver");
    return false;
  }
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)stride_bytes};
  cuuint32_t box[2] = {(cuuint32_t)box_cols, (cuuint32_t)box_rows};
  cuuint32_t es[2] = {1, 1};
  CUresult r = g_encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(base), dims,
                        strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    fail(NK_ERR_CUDA, "cuTensorMapEncodeTiled (FP32) failed (%d)", (int)r);
    return false;
  }
  return true;
}

bool tc_supported_shape(int n, int m) { return n + 1 <= 448 && m >= 1; }

// BF16 hi/lo splits: bf16split.cuh


// ------------------------------------------------------------------ B planes

template <bool CPLX, bool FROM_RBM>
__device__ __forceinline__ void bplanes_body(int bx, int gx, const double* __restrict__ src,
                                             int src_rows, int ncols, int ld,
                                             const double* __restrict__ w,
                                             const double* __restrict__ b, int n, int mt,
                                             int na64, uint16_t* __restrict__ planes,
                                             const double* skip) {
  if (skip && *skip != 0.0) return;
  const int HJ = CPLX ? 64 : 128;
  const int64_t plane = (int64_t)mt * 128 * na64;
  for (int64_t e = bx * (int64_t)blockDim.x + threadIdx.x; e < plane;
       e += (int64_t)gx * blockDim.x) {
    const int row = (int)(e / na64), i = (int)(e % na64);
    const int jt = row >> 7, rr = row & 127;
    const int j = CPLX ? jt * HJ + (rr & 63) : jt * HJ + rr;
    const int comp = CPLX ? (rr >> 6) : 0;
    double x = 0.0;
    if (j < src_rows && i < ncols) {
      if (FROM_RBM) {
        const int k = CPLX ? 2 : 1;
        x = i < n ? w[((int64_t)j * n + i) * k + comp] : b[(int64_t)j * k + comp];
      } else {
        x = CPLX ? src[((int64_t)j * ld + i) * 2 + comp] : src[(int64_t)j * ld + i];
      }
    }
    uint32_t hi, lo;
    split_bf16(x, hi, lo);
    planes[e] = (uint16_t)hi;
    planes[plane + e] = (uint16_t)lo;
  }
}

template <bool CPLX, bool FROM_RBM>
__global__ void bplanes_kernel(const double* __restrict__ src, int src_rows, int ncols, int ld,
                               const double* __restrict__ w, const double* __restrict__ b, int n,
                               int mt, int na64, uint16_t* __restrict__ planes,
                               const double* skip) {
  bplanes_body<CPLX, FROM_RBM>(blockIdx.x, gridDim.x, src, src_rows, ncols, ld, w, b, n, mt,
                               na64, planes, skip);
}

nk_status launch_bplanes_from_f64(const void* src, int src_rows, int ncols, int ld, int cplx,
                                  int mt, int na64, void* planes, const double* skip,
                                  cudaStream_t st) {
  const int64_t tot = (int64_t)mt * 128 * na64;
  const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>((tot + 255) / 256, 152 * 8));
  if (cplx)
    bplanes_kernel<true, false><<<(unsigned)blocks, 256, 0, st>>>(
        (const double*)src, src_rows, ncols, ld, nullptr, nullptr, 0, mt, na64,
        (uint16_t*)planes, skip);
  else
    bplanes_kernel<false, false><<<(unsigned)blocks, 256, 0, st>>>(
        (const double*)src, src_rows, ncols, ld, nullptr, nullptr, 0, mt, na64,
        (uint16_t*)planes, skip);
  return check_launch("bplanes");
}

nk_status launch_bplanes_from_rbm(const nk_rbm* r, cudaStream_t st) {
  WsLayout L(r->n, r->m, r->is_complex);
  const int64_t tot = (int64_t)L.mt * 128 * L.na64;
  const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>((tot + 255) / 256, 152 * 8));
  uint16_t* planes = (uint16_t*)((char*)r->ws + L.wbf);
  if (r->is_complex)
    bplanes_kernel<true, true><<<(unsigned)blocks, 256, 0, st>>>(
        nullptr, r->m, r->n + 1, 0, r->w, r->b, r->n, L.mt, L.na64, planes, nullptr);
  else
    bplanes_kernel<false, true><<<(unsigned)blocks, 256, 0, st>>>(
        nullptr, r->m, r->n + 1, 0, r->w, r->b, r->n, L.mt, L.na64, planes, nullptr);
  return check_launch("nk_rbm_prepare(bf16 planes)");
}

// ------------------------------------------------------------------ sigma'^T

__device__ __forceinline__ void sigma_t_body(int bx, int gx, int i,
                                             const int8_t* __restrict__ sigma, int64_t ns, int n,
                                             int64_t ns8, uint16_t* __restrict__ out) {
  for (int64_t s = bx * (int64_t)blockDim.x + threadIdx.x; s < ns8;
       s += (int64_t)gx * blockDim.x) {
    uint16_t v = 0;
    if (s < ns) {
      if (i < n) v = sigma[s * n + i] > 0 ? 0x3F80 : 0xBF80;
      else if (i == n) v = 0x3F80;
    }
    out[(int64_t)i * ns8 + s] = v;
  }
}

__global__ void sigma_t_kernel(const int8_t* __restrict__ sigma, int64_t ns, int n, int na64,
                               int64_t ns8, uint16_t* __restrict__ out) {
  (void)na64;
  sigma_t_body(blockIdx.x, gridDim.x, blockIdx.y, sigma, ns, n, ns8, out);
}

nk_status launch_sigma_t(const int8_t* sigma, int64_t ns, int n, int na64, void* out,
                         cudaStream_t st) {
  const int64_t ns8 = round_up(ns, 8);
  dim3 grid((unsigned)std::max<int64_t>(1, std::min<int64_t>((ns8 + 255) / 256, 64)), na64);
  sigma_t_kernel<<<grid, 256, 0, st>>>(sigma, ns, n, na64, ns8, (uint16_t*)out);
  return check_launch("sigma_t");
}

// sigma' rows: thread per 16-B chunk of 8 BF16 values (coalesced stores)
__device__ __forceinline__ void sigma_rows_body(int bx, int gx, const int8_t* __restrict__ sigma,
                                                int64_t ns, int n, int na64,
                                                uint16_t* __restrict__ out) {
  const int cpr = na64 / 8;  // chunks per row
  const int64_t tot = ns * cpr;
  for (int64_t x = bx * (int64_t)blockDim.x + threadIdx.x; x < tot;
       x += (int64_t)gx * blockDim.x) {
    const int64_t s = x / cpr;
    const int i0 = (int)(x % cpr) * 8;
    uint32_t pk[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      uint32_t v[2];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int i = i0 + 2 * q + h;
        v[h] = i < n ? (sigma[s * n + i] > 0 ? 0x3F80u : 0xBF80u) : (i == n ? 0x3F80u : 0u);
      }
      pk[q] = v[0] | (v[1] << 16);
    }
    *reinterpret_cast<uint4*>(out + s * na64 + i0) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
  }
}

__global__ void sigma_rows_kernel(const int8_t* __restrict__ sigma, int64_t ns, int n, int na64,
                                  uint16_t* __restrict__ out) {
  sigma_rows_body(blockIdx.x, gridDim.x, sigma, ns, n, na64, out);
}

nk_status launch_sigma_rows(const int8_t* sigma, int64_t ns, int n, int na64, void* out,
                            cudaStream_t st) {
  const int64_t tot = ns * (na64 / 8);
  const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>((tot + 255) / 256, 152 * 8));
  sigma_rows_kernel<<<(unsigned)blocks, 256, 0, st>>>(sigma, ns, n, na64, (uint16_t*)out);
  return check_launch("sigma_rows");
}

// ------------------------------------------------------------------ forward

constexpr int kFwdStages = 3;
constexpr int kFwdThreads = 192;
constexpr uint32_t kStageB = 32768;  // hi + lo tiles of 128 rows x 128 B

__device__ __forceinline__ unsigned char* align1024(unsigned char* p) {
  return (unsigned char*)(((uintptr_t)p + 1023) & ~(uintptr_t)1023);
}

__device__ __forceinline__ uint32_t sig_bits(const int8_t* sigma, int64_t s, int64_t ns, int n,
                                             int i) {
  if (s >= ns) return 0;
  if (i < n) return sigma[s * n + i] > 0 ? 0x3F80u : 0xBF80u;
  return i == n ? 0x3F80u : 0u;
}

// STAGES: B-operand stages; PREFETCH: the next tile's T values are loaded into
// registers while its MMAs run (else each 16-unit chunk is loaded just before
// use, which needs far fewer registers); SIG_TMA: the sigma' sample tile is
// TMA-loaded from the BF16 rows of launch_sigma_rows (map `sgp`), else built
// from the int8 samples by the CTA.
template <bool CPLX, int STAGES, bool PREFETCH, bool SIG_TMA = false>
__device__ __forceinline__ void fwd_tc_body(const CUtensorMap* tbp, const FwdTcArgs& A, int bx,
                                            int seg, const CUtensorMap* sgp = nullptr) {
  if (A.skip && *A.skip != 0.0) return;
  extern __shared__ __align__(1024) unsigned char smraw[];
  unsigned char* sm = align1024(smraw);
  const int KC = A.na64 / 64;
  unsigned char* sA = sm;
  unsigned char* sB = sm + (size_t)KC * 16384;
  uint64_t* full = reinterpret_cast<uint64_t*>(sB + STAGES * kStageB);
  uint64_t* empty = full + STAGES;
  uint64_t* tfull = empty + STAGES;
  uint64_t* tempty = tfull + 2;
  uint64_t* afull = tempty + 2;
  uint32_t* slot = reinterpret_cast<uint32_t*>(afull + 1);
  // after the barriers (128 bytes): the epilogue warps' staging tiles, 4 KB each
  float4* epi_stage = reinterpret_cast<float4*>(reinterpret_cast<unsigned char*>(full) + 128);
  const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
  const int64_t s0 = (int64_t)bx * 128;

  if (tid == 0) {
    for (int st = 0; st < STAGES; ++st) {
      mbar_init(&full[st], 1);
      mbar_init(&empty[st], 1);
    }
    for (int k = 0; k < 2; ++k) {
      mbar_init(&tfull[k], 1);
      mbar_init(&tempty[k], 4);
    }
    mbar_init(afull, 1);
    mbar_fence_init();
  }
  if (w == 1) tmem_alloc(slot, 256);
  // resident sigma' tile: 128 rows x KC * 64 columns, 16-B chunks of 8 BF16
  for (int x = tid; x < (SIG_TMA ? 0 : 128 * KC * 8); x += blockDim.x) {
    const int r = x / (KC * 8), rem = x % (KC * 8), kc = rem >> 3, c = rem & 7;
    const int64_t s = s0 + r;
    const int i0 = kc * 64 + c * 8;
    uint32_t pk[4];
#pragma unroll
    for (int q = 0; q < 4; ++q)
      pk[q] = sig_bits(A.sigma, s, A.ns, A.n, i0 + 2 * q) |
              (sig_bits(A.sigma, s, A.ns, A.n, i0 + 2 * q + 1) << 16);
    *reinterpret_cast<uint4*>(sA + (size_t)kc * 16384 + sw128_offset(r, c * 8)) =
        make_uint4(pk[0], pk[1], pk[2], pk[3]);
  }
  fence_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t taddr = *slot;
  // hidden tiles of this CTA: all, or one half (seg) when the launch is split
  const int jt_begin = A.mt * seg / A.nseg, jt_end = A.mt * (seg + 1) / A.nseg;
  const int total_it = (jt_end - jt_begin) * KC;
  bool bad = false;

  if (w == 0) {
    if (lane == 0) {
      if (SIG_TMA && total_it > 0) {
        mbar_arrive_expect_tx(afull, (uint32_t)KC * 16384u);
        for (int kc = 0; kc < KC; ++kc)
          tma_load_2d(sA + (size_t)kc * 16384, sgp, kc * 64, (int)s0, afull);
      }
      for (int it = 0; it < total_it; ++it) {
        const int st = it % STAGES, u = it / STAGES, jt = jt_begin + it / KC,
                  kc = it % KC;
        if (u > 0 && !mbar_wait_bounded(&empty[st], (uint32_t)((u - 1) & 1))) {
          bad = true;
          break;
        }
        mbar_arrive_expect_tx(&full[st], kStageB);
        tma_load_2d(sB + (size_t)st * kStageB, tbp, kc * 64, jt * 128, &full[st]);
        tma_load_2d(sB + (size_t)st * kStageB + 16384, tbp, kc * 64, (A.mt + jt) * 128,
                    &full[st]);
      }
    }
  } else if (w == 1) {
    if (lane == 0) {
      const uint32_t idesc = idesc_bf16(128, 128);
      int it = 0;
      if (SIG_TMA && total_it > 0 && !mbar_wait_bounded(afull, 0u)) bad = true;
      for (int jt = jt_begin; jt < jt_end && !bad; ++jt) {
        const int acc = (jt - jt_begin) & 1, ua = (jt - jt_begin) >> 1;
        if (ua > 0 && !mbar_wait_bounded(&tempty[acc], (uint32_t)((ua - 1) & 1))) {
          bad = true;
          break;
        }
        tc_fence_after();
        const uint32_t d = taddr + (uint32_t)(acc * 128);
        for (int kc = 0; kc < KC; ++kc, ++it) {
          const int st = it % STAGES, u = it / STAGES;
          if (!mbar_wait_bounded(&full[st], (uint32_t)(u & 1))) {
            bad = true;
            break;
          }
          tc_fence_after();
#pragma unroll
          for (int kk = 0; kk < 4; ++kk) {
            const uint64_t ad = sdesc_sw128(smem_addr(sA + (size_t)kc * 16384 + kk * 32));
            const uint64_t bh = sdesc_sw128(smem_addr(sB + (size_t)st * kStageB + kk * 32));
            const uint64_t bl =
                sdesc_sw128(smem_addr(sB + (size_t)st * kStageB + 16384 + kk * 32));
            umma_bf16(d, ad, bh, idesc, (kc | kk) != 0);
            umma_bf16(d, ad, bl, idesc, 1u);
          }
          umma_commit(&empty[st]);
        }
        if (!bad) umma_commit(&tfull[acc]);
      }
    }
  } else {
    // epilogue warps 2..5: warp w reads TMEM lanes 32 (w % 4) .. + 31.  In SR
    // mode the T' values of the next tile are loaded into registers while the
    // MMAs of that tile run (all loads in flight at once).
    const int q = w & 3;
    const int row = 32 * q + lane;
    const int64_t s = s0 + row;
    const bool live = s < A.ns;
    const uint32_t lane_base = (uint32_t)(32 * q) << 16;
    constexpr int HJ = CPLX ? 64 : 128;
    using F = typename std::conditional<CPLX, float2, float>::type;
    const F* T = reinterpret_cast<const F*>(A.T);
    F tp[PREFETCH ? HJ : 1];
    // 16-byte loads when every row of T starts 16-B aligned (m even for complex,
    // m a multiple of 4 for real); the tile's tail and j = m are handled per element
    const bool vec = CPLX ? (A.m % 2 == 0) : (A.m % 4 == 0);
    // ln psi / theta mode with 16-B aligned rows: each 16-unit chunk of theta (and
    // tanh theta) goes through the warp's staging tile (32 rows, 16-B chunks
    // XOR-swizzled by row, so that neither side has bank conflicts) and out as
    // whole row segments: 4 rows of 128 B (complex) or 8 rows of 64 B (real) per
    // store instruction instead of one 8- or 4-byte value in each of 32 rows
    float4* stg = (A.mode == 1 && vec) ? epi_stage + q * 256 : nullptr;
    auto stage_store_c = [&](float4* sb, const float (&xr)[16], const float (&xi)[16], float2* dst,
                             int jc) {
#pragma unroll
      for (int k = 0; k < 8; ++k)
        sb[lane * 8 + (k ^ (lane & 7))] =
            make_float4(xr[2 * k], xi[2 * k], xr[2 * k + 1], xi[2 * k + 1]);
      __syncwarp();
#pragma unroll
      for (int it = 0; it < 8; ++it) {
        const int f = it * 32 + lane, r = f >> 3, k = f & 7;
        const float4 v = sb[r * 8 + (k ^ (r & 7))];
        const int64_t sr = s0 + 32 * q + r;
        const int j = jc + 2 * k;
        if (sr < A.ns && j < A.m) {
          float2* d = dst + sr * A.m + j;
          if (j + 1 < A.m) *reinterpret_cast<float4*>(d) = v;
          else *d = make_float2(v.x, v.y);
        }
      }
      __syncwarp();
    };
    auto stage_store_r = [&](float4* sb, const float (&x)[16], float* dst, int jc) {
#pragma unroll
      for (int k = 0; k < 4; ++k)
        sb[lane * 4 + (k ^ ((lane >> 1) & 3))] =
            make_float4(x[4 * k], x[4 * k + 1], x[4 * k + 2], x[4 * k + 3]);
      __syncwarp();
#pragma unroll
      for (int it = 0; it < 4; ++it) {
        const int f = it * 32 + lane, r = f >> 2, k = f & 3;
        const float4 v = sb[r * 4 + (k ^ ((r >> 1) & 3))];
        const int64_t sr = s0 + 32 * q + r;
        const int j = jc + 4 * k;
        if (sr < A.ns && j < A.m) {
          float* d = dst + sr * A.m + j;
          if (j + 3 < A.m) {
            *reinterpret_cast<float4*>(d) = v;
          } else {
            d[0] = v.x;
            if (j + 1 < A.m) d[1] = v.y;
            if (j + 2 < A.m) d[2] = v.z;
          }
        }
      }
      __syncwarp();
    };
    auto load_t = [&](int jt) {
      const int j0 = jt * HJ;
      if (vec && live && j0 + HJ <= A.m) {
        const float4* src = reinterpret_cast<const float4*>(T + s * A.m + j0);
        constexpr int NV = CPLX ? HJ / 2 : HJ / 4;
#pragma unroll
        for (int e = 0; e < NV; ++e) {
          const float4 x = src[e];
          if constexpr (CPLX) {
            tp[2 * e] = make_float2(x.x, x.y);
            tp[2 * e + 1] = make_float2(x.z, x.w);
          } else {
            tp[4 * e] = x.x;
            tp[4 * e + 1] = x.y;
            tp[4 * e + 2] = x.z;
            tp[4 * e + 3] = x.w;
          }
        }
        return;
      }
#pragma unroll
      for (int e = 0; e < HJ; ++e) {
        const int j = j0 + e;
        if constexpr (CPLX) {
          tp[e] = make_float2(0.f, 0.f);
          if (live && j < A.m) tp[e] = T[s * A.m + j];
          else if (j == A.m) tp[e] = make_float2(1.f, 0.f);
        } else {
          tp[e] = 0.f;
          if (live && j < A.m) tp[e] = T[s * A.m + j];
          else if (j == A.m) tp[e] = 1.f;
        }
      }
    };
    // one 16-unit chunk c of tile jt (the loads of the no-prefetch variant)
    auto load_chunk = [&](int jt, int c, F (&tc)[16]) {
      const int j0 = jt * HJ + c * 16;
      if (vec && live && j0 + 16 <= A.m) {
        const float4* src = reinterpret_cast<const float4*>(T + s * A.m + j0);
        constexpr int NV = CPLX ? 8 : 4;
#pragma unroll
        for (int e = 0; e < NV; ++e) {
          const float4 x = src[e];
          if constexpr (CPLX) {
            tc[2 * e] = make_float2(x.x, x.y);
            tc[2 * e + 1] = make_float2(x.z, x.w);
          } else {
            tc[4 * e] = x.x;
            tc[4 * e + 1] = x.y;
            tc[4 * e + 2] = x.z;
            tc[4 * e + 3] = x.w;
          }
        }
        return;
      }
#pragma unroll
      for (int e = 0; e < 16; ++e) {
        const int j = j0 + e;
        if constexpr (CPLX) {
          tc[e] = make_float2(0.f, 0.f);
          if (live && j < A.m) tc[e] = T[s * A.m + j];
          else if (j == A.m) tc[e] = make_float2(1.f, 0.f);
        } else {
          tc[e] = 0.f;
          if (live && j < A.m) tc[e] = T[s * A.m + j];
          else if (j == A.m) tc[e] = 1.f;
        }
      }
    };
    if (PREFETCH && A.mode == 0 && jt_end > jt_begin) load_t(jt_begin);
    double sr = 0.0, si = 0.0;
    for (int jt = jt_begin; jt < jt_end; ++jt) {
      const int acc = (jt - jt_begin) & 1;
      if (!mbar_wait_bounded(&tfull[acc], (uint32_t)(((jt - jt_begin) >> 1) & 1))) {
        bad = true;
        break;
      }
      tc_fence_after();
      const uint32_t tb0 = taddr + lane_base + (uint32_t)(acc * 128);
      const int j0 = jt * HJ;
      float pr = 0.f, pi = 0.f;
      if constexpr (CPLX) {
        float2* th = reinterpret_cast<float2*>(A.theta_out);
        float2* tt = reinterpret_cast<float2*>(A.t_out);
        // SR forward: the chunk loop unrolled (the prefetched T' values sit in a
        // register array indexed by chunk); ln psi / theta / tanh theta: one chunk
        // per loop trip, so that the transcendental epilogue is inlined once
        // instead of four times (the unrolled body overflowed the instruction
        // cache); the summation order is the same either way
        if (A.mode == 0) {
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            float2 tc[16];
            if (!PREFETCH) load_chunk(jt, c, tc);
            float ur[16], ui[16];
            tmem_ld16(tb0 + c * 16, ur);
            tmem_ld16(tb0 + 64 + c * 16, ui);
            tmem_ld_wait();
#pragma unroll
            for (int e = 0; e < 16; ++e) {
              const float2 t = PREFETCH ? tp[c * 16 + e] : tc[e];
              pr += t.x * ur[e] - t.y * ui[e];
              pi += t.x * ui[e] + t.y * ur[e];
            }
          }
        }
#pragma unroll 1
        for (int c = 0; c < (A.mode == 0 ? 0 : 4); ++c) {
          float ur[16], ui[16];
          tmem_ld16(tb0 + c * 16, ur);
          tmem_ld16(tb0 + 64 + c * 16, ui);
          tmem_ld_wait();
          {
            if (A.logpsi && live) {
#pragma unroll
              for (int e = 0; e < 16; ++e) {
                if (j0 + c * 16 + e < A.m) {
                  cf l = lncosh_c(cf{ur[e], ui[e]});
                  pr += l.x;
                  pi += l.y;
                }
              }
            }
            if (stg) {  // aligned rows: through the warp's staging tile
              if (th) stage_store_c(stg, ur, ui, th, j0 + c * 16);
              if (tt) {
                float vr[16], vi[16];
#pragma unroll
                for (int e = 0; e < 16; ++e) {
                  const cf t = tanh_c(cf{ur[e], ui[e]});
                  vr[e] = t.x;
                  vi[e] = t.y;
                }
                stage_store_c(stg, vr, vi, tt, j0 + c * 16);
              }
            } else if (live) {
#pragma unroll
              for (int e = 0; e < 16; ++e) {
                const int j = j0 + c * 16 + e;
                if (j < A.m) {
                  if (th) th[s * A.m + j] = make_float2(ur[e], ui[e]);
                  if (tt) {
                    cf t = tanh_c(cf{ur[e], ui[e]});
                    tt[s * A.m + j] = make_float2(t.x, t.y);
                  }
                }
              }
            }
          }
        }
      } else {
        float* th = reinterpret_cast<float*>(A.theta_out);
        float* tt = reinterpret_cast<float*>(A.t_out);
        if (A.mode == 0) {
#pragma unroll
          for (int c = 0; c < 8; ++c) {
            float tc[16];
            if (!PREFETCH) load_chunk(jt, c, tc);
            float u[16];
            tmem_ld16(tb0 + c * 16, u);
            tmem_ld_wait();
#pragma unroll
            for (int e = 0; e < 16; ++e) pr += (PREFETCH ? tp[c * 16 + e] : tc[e]) * u[e];
          }
        }
#pragma unroll 1
        for (int c = 0; c < (A.mode == 0 ? 0 : 8); ++c) {
          float u[16];
          tmem_ld16(tb0 + c * 16, u);
          tmem_ld_wait();
          {
            if (A.logpsi && live) {
#pragma unroll
              for (int e = 0; e < 16; ++e)
                if (j0 + c * 16 + e < A.m) pr += lncosh_f(u[e]);
            }
            if (stg) {  // aligned rows: through the warp's staging tile
              if (th) stage_store_r(stg, u, th, j0 + c * 16);
              if (tt) {
                float v[16];
#pragma unroll
                for (int e = 0; e < 16; ++e) v[e] = tanh_f(u[e]);
                stage_store_r(stg, v, tt, j0 + c * 16);
              }
            } else if (live) {
#pragma unroll
              for (int e = 0; e < 16; ++e) {
                const int j = j0 + c * 16 + e;
                if (j < A.m) {
                  if (th) th[s * A.m + j] = u[e];
                  if (tt) tt[s * A.m + j] = tanh_f(u[e]);
                }
              }
            }
          }
        }
      }
      sr += (double)pr;
      si += (double)pi;
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&tempty[acc]);
      if (PREFETCH && A.mode == 0 && jt + 1 < jt_end) load_t(jt + 1);
    }
    if (live && (A.mode == 0 || A.logpsi)) {
      if (bad) sr = si = __longlong_as_double(0x7ff8000000000000ll);  // NaN marks a timeout
      // split launches: two addends onto an exact zero (y, ln psi zeroed by the
      // launcher), so the sum does not depend on which half lands first
      double* yd = reinterpret_cast<double*>(A.mode == 0 ? A.y : (void*)A.logpsi);
      const int cs = CPLX || A.mode == 1 ? 2 : 1;  // doubles per sample
      if (A.mode == 0) {
        if (A.nseg == 1) {
          yd[cs * s] = sr;
          if (CPLX) yd[cs * s + 1] = si;
        } else {
          atomicAdd(&yd[cs * s], sr);
          if (CPLX) atomicAdd(&yd[cs * s + 1], si);
        }
      } else {
        double vr = 0.0, vi = 0.0;
        const int8_t* sg = A.sigma + s * A.n;
        for (int i = 0; i < (seg == 0 ? A.n : 0); ++i) {
          const double sv = (double)sg[i];
          if (CPLX) {
            vr += A.a[2 * i] * sv;
            vi += A.a[2 * i + 1] * sv;
          } else {
            vr += A.a[i] * sv;
          }
        }
        if (A.nseg == 1) {
          yd[2 * s] = sr + vr;
          yd[2 * s + 1] = si + vi;
        } else {
          atomicAdd(&yd[2 * s], sr + vr);
          atomicAdd(&yd[2 * s + 1], si + vi);
        }
      }
    }
    if (A.mode == 0 && A.mean_part) {
      // this CTA's partial of the centring mean sum_s w_s y_s, in a fixed order:
      // within each warp, then the four warps in lane-quarter order
      __shared__ double mp[4][2];
      double wr = 0.0, wi = 0.0;
      if (live) {
        const double wgt = A.weights ? A.weights[s] : 1.0 / (double)A.ns;
        wr = wgt * sr;
        wi = wgt * si;
      }
#pragma unroll
      for (int off = 16; off >= 1; off >>= 1) {
        wr += __shfl_xor_sync(0xffffffffu, wr, off);
        wi += __shfl_xor_sync(0xffffffffu, wi, off);
      }
      if (lane == 0) {
        mp[q][0] = wr;
        mp[q][1] = wi;
      }
      asm volatile("bar.sync 1, 128;" ::: "memory");  // the four epilogue warps
      if (q == 0 && lane == 0) {
        const int64_t pidx = (int64_t)seg * ((A.ns + 127) / 128) + bx;
        A.mean_part[pidx] = ((mp[0][0] + mp[1][0]) + mp[2][0]) + mp[3][0];
        A.mean_part[A.mean_stride + pidx] = ((mp[0][1] + mp[1][1]) + mp[2][1]) + mp[3][1];
      }
    }
  }
  if (bad) {
    if (A.err) atomicOr(A.err, 1);
    dev_status_set(1u << NK_ERR_TIMEOUT);
  }
  tc_fence_before();
  __syncthreads();
  if (w == 1) {
    tc_fence_after();
    tmem_dealloc(taddr, 256);
  }
}

template <bool CPLX, bool SIG_TMA>
__global__ void __launch_bounds__(kFwdThreads, 1)
    fwd_tc_kernel(const __grid_constant__ CUtensorMap tb, const __grid_constant__ CUtensorMap sg,
                  FwdTcArgs A) {
  fwd_tc_body<CPLX, kFwdStages, true, SIG_TMA>(&tb, A, blockIdx.x, blockIdx.y, &sg);
}

// Alignment slack, sigma' tile, stages, barriers and, for the ln psi / theta
// mode (mode 1), the epilogue warps' four 4 KB staging tiles: the SR forward
// (mode 0) does not reserve them, which keeps two CTAs per SM on small problems.
static size_t fwd_smem_bytes(int na64, int stages, bool staging) {
  return 1024 + (size_t)(na64 / 64) * 16384 + (size_t)stages * kStageB + 128 +
         (staging ? 4 * 4096 : 0);
}

// One CTA per SM: when the last wave would be far from full, split the hidden
// tiles into two halves (twice the CTAs) whose sums meet in the output.  (An
// SR forward that builds its sigma' tiles itself does not split: the extra
// builds cost more than the evener waves save.)
int fwd_tc_nseg(int64_t ns, int mt, int mode, bool sig_tma) {
  const int64_t blocks = (ns + 127) / 128;
  auto wave_eff = [](int64_t b) { return (double)b / (double)(((b + 151) / 152) * 152); };
  return ((mode == 1 || sig_tma) && mt >= 2 && wave_eff(2 * blocks) > wave_eff(blocks)) ? 2 : 1;
}

nk_status launch_fwd_tc(const FwdTcArgs& A, const void* planes, cudaStream_t st) {
  if (!tc_supported_shape(A.n, A.m))
    return fail(NK_ERR_UNSUPPORTED, "tensor-core path supports n + 1 <= 448 (n = %d)", A.n);
  CUtensorMap map, smap;
  if (!tc_make_map(&map, planes, 2LL * A.mt * 128, A.na64, A.na64, 128)) return NK_ERR_CUDA;
  const bool sig_tma = A.mode == 0 && A.sig_rows != nullptr;
  if (sig_tma) {
    if (!tc_make_map(&smap, A.sig_rows, A.ns, A.na64, A.na64, 128)) return NK_ERR_CUDA;
  } else {
    smap = map;  // unused
  }
  const size_t smem = fwd_smem_bytes(A.na64, kFwdStages, A.mode == 1);
  const int64_t blocks = (A.ns + 127) / 128;
  FwdTcArgs B = A;
  B.nseg = fwd_tc_nseg(A.ns, A.mt, A.mode, sig_tma);
  if (A.mode == 1 && A.nseg_req > 0) B.nseg = (A.nseg_req >= 2 && A.mt >= 2) ? 2 : 1;
  if (B.nseg == 2 && (A.mode == 0 || A.logpsi)) {
    void* out = A.mode == 0 ? A.y : (void*)A.logpsi;
    const size_t per = (A.mode == 1 || A.cplx) ? 16 : 8;
    if (cudaMemsetAsync(out, 0, (size_t)A.ns * per, st) != cudaSuccess)
      return fail(NK_ERR_CUDA, "fwd_tc: cudaMemsetAsync failed");
  }
  const dim3 grid((unsigned)blocks, (unsigned)B.nseg);
  auto go = [&](auto kern) -> nk_status {
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
      return fail(NK_ERR_CUDA, "fwd_tc: shared memory attribute");
    kern<<<grid, kFwdThreads, smem, st>>>(map, smap, B);
    return check_launch("fwd_tc");
  };
  if (A.cplx) return sig_tma ? go(fwd_tc_kernel<true, true>) : go(fwd_tc_kernel<true, false>);
  return sig_tma ? go(fwd_tc_kernel<false, true>) : go(fwd_tc_kernel<false, false>);
}

// Up to kFwdFuseMax theta / ln psi launches (mode 1) of one field in one launch:
// CTA b runs CTA b - start[k] of problem k, numbered as that problem's own
// launch (sample tile, hidden-tile half), with its own tensor map.
constexpr int kFwdFuseMax = 64;
struct FwdFuse {
  int n;
  int start[kFwdFuseMax + 1];
  int tiles[kFwdFuseMax];
  FwdTcArgs a[kFwdFuseMax];
  CUtensorMap map[kFwdFuseMax];
};

template <bool CPLX>
__global__ void __launch_bounds__(kFwdThreads, 1) fwd_tc_fused(const __grid_constant__ FwdFuse B) {
  int k = 0;
  while (k + 1 < B.n && (int)blockIdx.x >= B.start[k + 1]) ++k;
  const int b = (int)blockIdx.x - B.start[k], t = B.tiles[k];
  fwd_tc_body<CPLX, kFwdStages, true, false>(&B.map[k], B.a[k], b % t, b / t);
}

nk_status launch_fwd_tc_fused(const FwdTcArgs* args, const void* const* planes, int n,
                              cudaStream_t st) {
  for (int field = 0; field < 2; ++field) {
    for (int u0 = 0; u0 < n;) {
      FwdFuse* B = new FwdFuse;  // about 13 KB: kept off the stack
      B->n = 0;
      B->start[0] = 0;
      size_t smem = 0;
      int u = u0;
      nk_status e = NK_OK;
      for (; u < n && B->n < kFwdFuseMax && !e; ++u) {
        const FwdTcArgs& A = args[u];
        if (A.cplx != field || A.ns == 0) continue;
        if (!tc_supported_shape(A.n, A.m)) {
          e = fail(NK_ERR_UNSUPPORTED, "tensor-core path supports n + 1 <= 448 (n = %d)", A.n);
          break;
        }
        FwdTcArgs C = A;
        C.nseg = fwd_tc_nseg(A.ns, A.mt, A.mode, false);
        if (A.mode == 1 && A.nseg_req > 0) C.nseg = (A.nseg_req >= 2 && A.mt >= 2) ? 2 : 1;
        if (C.nseg == 2 && A.logpsi &&
            cudaMemsetAsync(A.logpsi, 0, (size_t)A.ns * 16, st) != cudaSuccess) {
          e = fail(NK_ERR_CUDA, "fwd_tc: cudaMemsetAsync failed");
          break;
        }
        if (!tc_make_map(&B->map[B->n], planes[u], 2LL * A.mt * 128, A.na64, A.na64, 128)) {
          e = NK_ERR_CUDA;
          break;
        }
        B->a[B->n] = C;
        B->tiles[B->n] = (int)((A.ns + 127) / 128);
        B->start[B->n + 1] = B->start[B->n] + B->tiles[B->n] * C.nseg;
        smem = std::max(smem, fwd_smem_bytes(A.na64, kFwdStages, A.mode == 1));
        ++B->n;
      }
      u0 = u;
      if (!e && B->n > 0) {
        auto kern = field ? fwd_tc_fused<true> : fwd_tc_fused<false>;
        if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess)
          e = fail(NK_ERR_CUDA, "fwd_tc_fused: shared memory attribute");
        else {
          kern<<<(unsigned)B->start[B->n], kFwdThreads, smem, st>>>(*B);
          e = check_launch("fwd_tc_fused");
        }
      }
      delete B;
      if (e) return e;
    }
  }
  return NK_OK;
}

// ------------------------------------------------------------------ adjoint

constexpr int kAdjProducerWarps = 8;
constexpr int kAdjThreads = 64 + 32 * kAdjProducerWarps;

template <bool CPLX>
__device__ __forceinline__ void adj_tc_body(const CUtensorMap* tsp, const AdjTcArgs& A,
                                            int64_t chunk, int bx, int by) {
  if (A.skip && *A.skip != 0.0) return;
  extern __shared__ __align__(1024) unsigned char smraw[];
  unsigned char* sm = align1024(smraw);
  const int NB = A.na64, NH = NB / 2;
  const uint32_t stage_bytes = 32768u + (uint32_t)NB * 128u;
  uint64_t* full = reinterpret_cast<uint64_t*>(sm + 2 * (size_t)stage_bytes);
  uint64_t* empty = full + 2;
  uint64_t* done = empty + 2;
  uint32_t* slot = reinterpret_cast<uint32_t*>(done + 1);
  const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
  const int HJ = CPLX ? 64 : 128;
  const int j0 = bx * HJ;
  const int z = by;
  const int64_t sb = (int64_t)z * chunk;
  const int64_t se = std::min<int64_t>(A.ns, sb + chunk);
  const int nit = se > sb ? (int)((se - sb + 63) / 64) : 0;
  const uint32_t ncols = NB <= 32 ? 32 : (NB <= 64 ? 64 : (NB <= 128 ? 128 : (NB <= 256 ? 256 : 512)));

  if (tid == 0) {
    for (int k = 0; k < 2; ++k) {
      mbar_init(&full[k], 1 + kAdjProducerWarps);
      mbar_init(&empty[k], 1);
    }
    mbar_init(done, 1);
    mbar_fence_init();
  }
  if (w == 1) tmem_alloc(slot, ncols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t taddr = *slot;
  bool bad = false;

  if (w == 0) {
    if (lane == 0) {
      for (int it = 0; it < nit; ++it) {
        const int st = it & 1, u = it >> 1;
        if (u > 0 && !mbar_wait_bounded(&empty[st], (uint32_t)((u - 1) & 1))) {
          bad = true;
          break;
        }
        unsigned char* B = sm + (size_t)st * stage_bytes + 32768;
        mbar_arrive_expect_tx(&full[st], (uint32_t)NB * 128u);
        tma_load_2d(B, tsp, (int)(sb + (int64_t)it * 64), 0, &full[st]);
        tma_load_2d(B + (size_t)NH * 128, tsp, (int)(sb + (int64_t)it * 64), NH, &full[st]);
      }
    }
  } else if (w == 1) {
    if (lane == 0) {
      const uint32_t idesc = idesc_bf16(128, NH);
      for (int it = 0; it < nit; ++it) {
        const int st = it & 1;
        if (!mbar_wait_bounded(&full[st], (uint32_t)((it >> 1) & 1))) {
          bad = true;
          break;
        }
        tc_fence_after();
        unsigned char* S = sm + (size_t)st * stage_bytes;
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
          const uint64_t ah = sdesc_sw128(smem_addr(S + kk * 32));
          const uint64_t al = sdesc_sw128(smem_addr(S + 16384 + kk * 32));
          const uint64_t b0 = sdesc_sw128(smem_addr(S + 32768 + kk * 32));
          const uint64_t b1 = sdesc_sw128(smem_addr(S + 32768 + (size_t)NH * 128 + kk * 32));
          const uint32_t first = (it | kk) == 0;
          umma_bf16(taddr, ah, b0, idesc, !first);
          umma_bf16(taddr, al, b0, idesc, 1u);
          umma_bf16(taddr + (uint32_t)NH, ah, b1, idesc, !first);
          umma_bf16(taddr + (uint32_t)NH, al, b1, idesc, 1u);
        }
        umma_commit(&empty[st]);
      }
      umma_commit(done);
    }
  } else {
    // producers: Z = conj(T'_sj) v_s as BF16 hi/lo, K-major swizzled A tiles.
    // Complex: thread (jp, qs) of the eight producer warps owns parameter rows
    // j0 + 2 jp, j0 + 2 jp + 1 and samples 8 qs .. 8 qs + 7 of each 64-sample
    // stage, loading both T values of a sample with one 16-byte load (a warp
    // reads 512 contiguous bytes per sample); real: thread (jq, qs) owns rows
    // j0 + 4 jq .. + 3.  The next stage's T values are loaded into registers
    // before the thread waits for its buffer; v_s reaches the warp by shuffles.
    const int pt = tid - 64;
    __shared__ double cmean[2];              // the centring mean (A.y mode)
    const double invn = 1.0 / (double)A.ns;
    constexpr int JPT = CPLX ? 2 : 4;        // parameter rows per thread
    const int jb = (pt & 31) * JPT;          // first local row
    const int qs = pt >> 5;                  // sample quarter of the stage
    const bool vec = (A.m % JPT) == 0;
    using F = typename std::conditional<CPLX, float2, float>::type;
    const F* T = reinterpret_cast<const F*>(A.T);
    constexpr int SPT = 64 / kAdjProducerWarps;  // samples per thread and stage
    F tq[SPT][JPT];
    float vq0 = 0.f, vq1 = 0.f;  // v of sample (lane % SPT) of this thread's slice
    auto load_stage = [&](int it) {
      const int64_t kb = sb + (int64_t)it * 64 + qs * SPT;
#pragma unroll
      for (int e = 0; e < SPT; ++e) {
        const int64_t smp = kb + e;
        const int j = j0 + jb;
        if (vec && smp < se && j + JPT <= A.m) {
          const float4 x = *reinterpret_cast<const float4*>(T + smp * A.m + j);
          if constexpr (CPLX) {
            tq[e][0] = make_float2(x.x, x.y);
            tq[e][1] = make_float2(x.z, x.w);
          } else {
            tq[e][0] = x.x;
            tq[e][1] = x.y;
            tq[e][2] = x.z;
            tq[e][3] = x.w;
          }
        } else {
#pragma unroll
          for (int u = 0; u < JPT; ++u) {
            const int jj = j + u;
            if constexpr (CPLX) {
              tq[e][u] = make_float2(0.f, 0.f);
              if (smp < se && jj < A.m) tq[e][u] = T[smp * A.m + jj];
              else if (smp < se && jj == A.m) tq[e][u] = make_float2(1.f, 0.f);
            } else {
              tq[e][u] = 0.f;
              if (smp < se && jj < A.m) tq[e][u] = T[smp * A.m + jj];
              else if (smp < se && jj == A.m) tq[e][u] = 1.f;
            }
          }
        }
      }
      const int64_t smp = kb + (lane % SPT);
      if (A.y) {
        // centred on the fly: v = w (y - mean)
        double vr = 0.0, vi = 0.0;
        if (smp < se) {
          const double wgt = A.weights ? A.weights[smp] : invn;
          if constexpr (CPLX) {
            const double2 yv = reinterpret_cast<const double2*>(A.y)[smp];
            vr = wgt * (yv.x - cmean[0]);
            vi = wgt * (yv.y - cmean[1]);
          } else {
            vr = wgt * (reinterpret_cast<const double*>(A.y)[smp] - cmean[0]);
          }
        }
        vq0 = (float)vr;
        vq1 = (float)vi;
      } else if constexpr (CPLX) {
        const double2 vd = smp < se ? reinterpret_cast<const double2*>(A.v)[smp]
                                    : make_double2(0.0, 0.0);
        vq0 = (float)vd.x;
        vq1 = (float)vd.y;
      } else {
        vq0 = smp < se ? (float)reinterpret_cast<const double*>(A.v)[smp] : 0.f;
      }
    };
    if (A.y) {
      // the centring mean, summed by the first producer warp in the centring
      // kernel's order (lane-strided partial sums, then a butterfly)
      if (pt < 32) {
        double r = 0.0, i = 0.0;
        for (int u = pt; u < A.mean_parts; u += 32) {
          r += A.mean_part[u];
          i += A.mean_part[A.mean_stride + u];
        }
#pragma unroll
        for (int off = 16; off >= 1; off >>= 1) {
          r += __shfl_xor_sync(0xffffffffu, r, off);
          i += __shfl_xor_sync(0xffffffffu, i, off);
        }
        if (pt == 0) {
          cmean[0] = r;
          cmean[1] = i;
        }
      }
      asm volatile("bar.sync 2, %0;" ::"r"(32 * kAdjProducerWarps) : "memory");  // producers
    }
    if (nit > 0) load_stage(0);
    for (int it = 0; it < nit && !bad; ++it) {
      const int st = it & 1, u = it >> 1;
      if (u > 0 && !mbar_wait_bounded(&empty[st], (uint32_t)((u - 1) & 1))) {
        bad = true;
        break;
      }
      unsigned char* Ahi = sm + (size_t)st * stage_bytes;
      unsigned char* Alo = Ahi + 16384;
#pragma unroll
      for (int cc = 0; cc < SPT / 8; ++cc) {
        const int kl = qs * SPT + cc * 8;
        // v of the chunk's 8 samples, fetched once for all of the thread's rows
        float vr8[8], vi8[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          vr8[e] = __shfl_sync(0xffffffffu, vq0, cc * 8 + e);
          vi8[e] = CPLX ? __shfl_sync(0xffffffffu, vq1, cc * 8 + e) : 0.f;
        }
#pragma unroll
        for (int u2 = 0; u2 < JPT; ++u2) {
          uint32_t hr[4], lr[4], hi_[4], li[4];
#pragma unroll
          for (int e2 = 0; e2 < 4; ++e2) {
            float zr[2], zi[2];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
              const int e = cc * 8 + 2 * e2 + h;
              const float vr = vr8[2 * e2 + h], vi = vi8[2 * e2 + h];
              if constexpr (CPLX) {
                const float2 t = tq[e][u2];
                zr[h] = t.x * vr + t.y * vi;  // conj(t) v
                zi[h] = t.x * vi - t.y * vr;
              } else {
                zr[h] = tq[e][u2] * vr;
                zi[h] = 0.f;
                (void)vi;
              }
            }
            split_bf16x2(zr[0], zr[1], hr[e2], lr[e2]);
            if constexpr (CPLX) split_bf16x2(zi[0], zi[1], hi_[e2], li[e2]);
          }
          const int row = jb + u2;
          *reinterpret_cast<uint4*>(Ahi + sw128_offset(row, kl)) = make_uint4(hr[0], hr[1], hr[2], hr[3]);
          *reinterpret_cast<uint4*>(Alo + sw128_offset(row, kl)) = make_uint4(lr[0], lr[1], lr[2], lr[3]);
          if constexpr (CPLX) {
            *reinterpret_cast<uint4*>(Ahi + sw128_offset(64 + row, kl)) =
                make_uint4(hi_[0], hi_[1], hi_[2], hi_[3]);
            *reinterpret_cast<uint4*>(Alo + sw128_offset(64 + row, kl)) =
                make_uint4(li[0], li[1], li[2], li[3]);
          }
        }
      }
      fence_async_smem();
      __syncwarp();
      if (lane == 0) mbar_arrive(&full[st]);
      if (it + 1 < nit) load_stage(it + 1);
    }
    // epilogue (warps 2..5, one per TMEM lane quarter): partial sums of this split
    if (!bad && !mbar_wait_bounded(done, 0u)) bad = true;
    tc_fence_after();
    const int q = w & 3, row = 32 * q + lane;
    const int jo = CPLX ? j0 + (row & 63) : j0 + row;
    const int comp = CPLX ? (row >> 6) : 0;
    const int ma = A.m + 1, na = A.n + 1;
    float* part = reinterpret_cast<float*>(A.part);
    for (int col = 0; col < (w < 6 ? NB : 0); col += 16) {
      float v[16];
      tmem_ld16(taddr + ((uint32_t)(32 * q) << 16) + (uint32_t)col, v);
      tmem_ld_wait();
      if (jo < ma) {
#pragma unroll
        for (int e = 0; e < 16; ++e) {
          const int i = col + e;
          if (i < na) {
            const float x = (nit > 0 && !bad) ? v[e] : (bad ? __int_as_float(0x7fc00000) : 0.f);
            const int64_t idx = ((int64_t)z * ma + jo) * na + i;
            if (CPLX) part[2 * idx + comp] = x;
            else part[idx] = x;
          }
        }
      }
    }
  }
  if (bad) {
    if (A.err) atomicOr(A.err, 1);
    dev_status_set(1u << NK_ERR_TIMEOUT);
  }
  tc_fence_before();
  __syncthreads();
  if (w == 1) {
    tc_fence_after();
    tmem_dealloc(taddr, ncols);
  }
}

template <bool CPLX>
__global__ void __launch_bounds__(kAdjThreads, 1)
    adj_tc_kernel(const __grid_constant__ CUtensorMap ts_map, AdjTcArgs A, int64_t chunk) {
  adj_tc_body<CPLX>(&ts_map, A, chunk, blockIdx.x, blockIdx.y);
}

int adj_tc_splits(int n, int m, int cplx, int64_t ns) {
  (void)n;
  const int HJ = cplx ? 64 : 128;
  const int tiles = (m + 1 + HJ - 1) / HJ;
  // at most two full waves of one CTA per SM (a third, nearly empty wave
  // would cost as much as a full one)
  int64_t sp = std::max(1, (2 * 152) / tiles);
  sp = std::min<int64_t>(sp, std::max<int64_t>(1, (ns + 63) / 64));
  return (int)std::max<int64_t>(1, std::min<int64_t>(sp, 64));
}

nk_status launch_adj_tc(const AdjTcArgs& A, const void* sigma_t, cudaStream_t st) {
  if (!tc_supported_shape(A.n, A.m))
    return fail(NK_ERR_UNSUPPORTED, "tensor-core path supports n + 1 <= 448 (n = %d)", A.n);
  const int64_t ns8 = round_up(A.ns, 8);
  CUtensorMap map;
  if (!tc_make_map(&map, sigma_t, A.na64, ns8, ns8, A.na64 / 2)) return NK_ERR_CUDA;
  const int HJ = A.cplx ? 64 : 128;
  const int tiles = (A.m + 1 + HJ - 1) / HJ;
  int64_t chunk = (A.ns + A.splits - 1) / A.splits;
  chunk = round_up(std::max<int64_t>(chunk, 1), 64);
  const size_t smem = 1024 + 2 * (32768 + (size_t)A.na64 * 128) + 64;
  dim3 grid(tiles, A.splits);
  if (A.cplx) {
    if (cudaFuncSetAttribute(adj_tc_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem) != cudaSuccess)
      return fail(NK_ERR_CUDA, "adj_tc: shared memory attribute");
    adj_tc_kernel<true><<<grid, kAdjThreads, smem, st>>>(map, A, chunk);
  } else {
    if (cudaFuncSetAttribute(adj_tc_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem) != cudaSuccess)
      return fail(NK_ERR_CUDA, "adj_tc: shared memory attribute");
    adj_tc_kernel<false><<<grid, kAdjThreads, smem, st>>>(map, A, chunk);
  }
  return check_launch("adj_tc");
}

// ------------------------------------------------------------------ batches

// The tensor maps of a batch live in global memory (written before the launch);
// make them visible to the TMA unit's tensor-map reads.
__device__ __forceinline__ void tensormap_acquire(const CUtensorMap* m) {
  asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(m) : "memory");
}

// Batched forward: two B stages and no T prefetch, so that two CTAs fit on an
// SM (the problems of a batch are small: many short CTAs).
constexpr int kFwdBatchStages = 2;
__global__ void __launch_bounds__(kFwdThreads, 2) fwd_tc_batch(const __grid_constant__ FwdBatch P) {
  const int z = blockIdx.z;
  const int t = P.tiles[z];
  if ((int)blockIdx.x >= t * P.a[z].nseg) return;
  if (threadIdx.x == 0) {
    tensormap_acquire(P.map[z]);
    tensormap_acquire(P.smap[z]);
  }
  const int bx = (int)blockIdx.x % t, seg = (int)blockIdx.x / t;
  if (P.a[z].cplx)
    fwd_tc_body<true, kFwdBatchStages, false, true>(P.map[z], P.a[z], bx, seg, P.smap[z]);
  else
    fwd_tc_body<false, kFwdBatchStages, false, true>(P.map[z], P.a[z], bx, seg, P.smap[z]);
}

// Batched adjoint: two CTAs per SM (96 registers per thread).
__global__ void __launch_bounds__(kAdjThreads, 2) adj_tc_batch(const __grid_constant__ AdjBatch P) {
  const int z = blockIdx.z;
  if ((int)blockIdx.x >= P.tiles[z] || (int)blockIdx.y >= P.splits[z]) return;
  if (threadIdx.x == 0) tensormap_acquire(P.map[z]);
  if (P.a[z].cplx)
    adj_tc_body<true>(P.map[z], P.a[z], P.chunk[z], blockIdx.x, blockIdx.y);
  else
    adj_tc_body<false>(P.map[z], P.a[z], P.chunk[z], blockIdx.x, blockIdx.y);
}

__global__ void sigma_t_batch(const SrDesc* __restrict__ D) {
  const SrDesc& d = D[blockIdx.z];
  const int64_t nbx = (d.ns8 + 255) / 256;
  const int nb = (int)(nbx < 1 ? 1 : (nbx > 64 ? 64 : nbx));
  if ((int)blockIdx.y >= d.na64 || (int)blockIdx.x >= nb) return;
  sigma_t_body(blockIdx.x, nb, blockIdx.y, d.sigma, d.ns, d.n, d.ns8,
               reinterpret_cast<uint16_t*>(d.sigt));
}

// blocks of an elementwise kernel over `elems` (the single-problem launches' count)
__device__ __host__ __forceinline__ int elem_blocks(int64_t elems) {
  const int64_t b = (elems + 255) / 256;
  return (int)(b < 1 ? 1 : (b > 152 * 8 ? 152 * 8 : b));
}

__global__ void bplanes_p_batch(const SrDesc* __restrict__ D) {
  const SrDesc& d = D[blockIdx.y];
  const int nb = elem_blocks((int64_t)d.mt1 * 128 * d.na64);
  if ((int)blockIdx.x >= nb) return;
  if (d.fwd_nseg == 2 && *d.done == 0.0) {
    // the two halves of the forward add their sums onto zero
    double* y = reinterpret_cast<double*>(d.y);
    const int64_t len = d.ns * (d.cplx ? 2 : 1);
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < len;
         e += (int64_t)nb * blockDim.x)
      y[e] = 0.0;
  }
  if (d.cplx)
    bplanes_body<true, false>(blockIdx.x, nb, reinterpret_cast<const double*>(d.p),
                              d.m + 1, d.n + 1, d.n + 1, nullptr, nullptr, 0, d.mt1, d.na64,
                              reinterpret_cast<uint16_t*>(d.xbf), d.done);
  else
    bplanes_body<false, false>(blockIdx.x, nb, reinterpret_cast<const double*>(d.p),
                               d.m + 1, d.n + 1, d.n + 1, nullptr, nullptr, 0, d.mt1, d.na64,
                               reinterpret_cast<uint16_t*>(d.xbf), d.done);
}

__global__ void bplanes_rbm_batch(const SrDesc* __restrict__ D) {
  const SrDesc& d = D[blockIdx.y];
  const int nb = elem_blocks((int64_t)d.wmt * 128 * d.wna64);
  if ((int)blockIdx.x >= nb) return;
  if (d.cplx)
    bplanes_body<true, true>(blockIdx.x, nb, nullptr, d.m, d.n + 1, 0, d.w, d.b, d.n,
                             d.wmt, d.wna64, reinterpret_cast<uint16_t*>(d.ws + d.ws_wbf),
                             nullptr);
  else
    bplanes_body<false, true>(blockIdx.x, nb, nullptr, d.m, d.n + 1, 0, d.w, d.b, d.n,
                              d.wmt, d.wna64, reinterpret_cast<uint16_t*>(d.ws + d.ws_wbf),
                              nullptr);
}

static unsigned vec_blocks(int64_t elems) {
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>((elems + 255) / 256, 152 * 8));
}

nk_status launch_fwd_tc_batch(const FwdBatch& P, int G, int max_tiles, int max_na64,
                              cudaStream_t st) {
  bool staging = false;  // the SR forwards run mode 0; any ln psi item needs the tiles
  for (int z = 0; z < G; ++z) staging = staging || P.a[z].mode == 1;
  const size_t smem = fwd_smem_bytes(max_na64, kFwdBatchStages, staging);
  if (cudaFuncSetAttribute(fwd_tc_batch, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem) != cudaSuccess)
    return fail(NK_ERR_CUDA, "fwd_tc_batch: shared memory attribute");
  fwd_tc_batch<<<dim3((unsigned)max_tiles, 1, (unsigned)G), kFwdThreads, smem, st>>>(P);
  return check_launch("fwd_tc_batch");
}

nk_status launch_adj_tc_batch(const AdjBatch& P, int G, int max_tiles, int max_splits,
                              int max_na64, cudaStream_t st) {
  const size_t smem = 1024 + 2 * (32768 + (size_t)max_na64 * 128) + 64;
  if (cudaFuncSetAttribute(adj_tc_batch, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem) != cudaSuccess)
    return fail(NK_ERR_CUDA, "adj_tc_batch: shared memory attribute");
  adj_tc_batch<<<dim3((unsigned)max_tiles, (unsigned)max_splits, (unsigned)G), kAdjThreads, smem,
                 st>>>(P);
  return check_launch("adj_tc_batch");
}

nk_status launch_sigma_t_batch(const SrDesc* D, int G, int64_t max_ns8, int max_na64,
                               cudaStream_t st) {
  const dim3 grid((unsigned)std::max<int64_t>(1, std::min<int64_t>((max_ns8 + 255) / 256, 64)),
                  (unsigned)max_na64, (unsigned)G);
  sigma_t_batch<<<grid, 256, 0, st>>>(D);
  return check_launch("sigma_t_batch");
}

__global__ void sigma_rows_batch(const SrDesc* __restrict__ D) {
  const SrDesc& d = D[blockIdx.y];
  const int nb = elem_blocks(d.ns * (d.na64 / 8));
  if ((int)blockIdx.x >= nb) return;
  sigma_rows_body(blockIdx.x, nb, d.sigma, d.ns, d.n, d.na64, reinterpret_cast<uint16_t*>(d.sigr));
}

nk_status launch_sigma_rows_batch(const SrDesc* D, int G, int64_t max_elems, cudaStream_t st) {
  sigma_rows_batch<<<dim3(vec_blocks(max_elems), (unsigned)G), 256, 0, st>>>(D);
  return check_launch("sigma_rows_batch");
}

nk_status launch_bplanes_p_batch(const SrDesc* D, int G, int64_t max_elems, cudaStream_t st) {
  bplanes_p_batch<<<dim3(vec_blocks(max_elems), (unsigned)G), 256, 0, st>>>(D);
  return check_launch("bplanes_p_batch");
}

nk_status launch_bplanes_rbm_batch(const SrDesc* D, int G, int64_t max_elems, cudaStream_t st) {
  bplanes_rbm_batch<<<dim3(vec_blocks(max_elems), (unsigned)G), 256, 0, st>>>(D);
  return check_launch("bplanes_rbm_batch");
}

NK_STATUS_COLLECTOR(collect_status_tc)

}  // namespace nk
