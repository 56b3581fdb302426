// K2: Metropolis sampling of |psi|^2 (Eq. 4; Sec. 2.2.5), single-spin flips or
// nearest-neighbour exchanges (MetropolisExchange of the VMC listing, Sec. 3.1).
//
// One or two warps run one chain; a CTA runs one proposal group, whose chains
// all propose the same site (bond) at a step.  Per proposal the ratio needs, for
// every hidden unit j, the table column (cosh c_j, sinh c_j / s_i) of the move
// and, on acceptance, its theta increment W_i (- W_k).  Each step's row (table
// block, increments and a header with a_i - a_k, built per call) reaches shared
// memory by one 1-D TMA bulk copy into a ring of slots, issued by the warp that
// releases the slot last, so the warps read every table value from shared
// memory once per chain.  (metro_group.cuh holds the other form: one CTA per
// group with the hidden units split over its threads.)
//
// Per chain: sigma lives in shared memory, theta in tensor memory (per-thread
// TMEM columns), t = tanh(theta) in registers.  With C = cosh c and
// D = sinh c / s_i, the factor of hidden unit j is r_j = C_j - s_i t_j D_j.  Real
// RBMs read (C, D) and multiply r_j.  Complex RBMs need only |r_j|^2 for the
// accept test and read, per unit, the expanded form
//   |r|^2 = |C|^2 + |t|^2 |D|^2 - 2 s_i Re(t conj(C) D),
// from per-call tables (|C|^2, |D|^2, conj(C) D) laid out so that one 16-byte
// load gives a thread two of its units, evaluated with packed FP32 pair
// instructions.  An accepted move updates theta += -2 s_i W_i (- 2 s_k W_k) and
// t by the tanh addition formula t' = (t C - s_i D) / r, for complex RBMs from
// the same tables: t' = (t |C|^2 + conj(t) |D|^2 - s_i (|t|^2 conj(E) + E)) / |r|^2
// with E = conj(C) D.  t is recomputed exactly from theta after every sweep.
// Philox draws are made 32 steps at a time, one step per lane (the rows and
// sites of the next block ahead of use), and broadcast by shuffles.
#include "common.cuh"
#include "internal.h"
#include "ratio.cuh"
#include "tma.cuh"
#include "status.cuh"
#include "umma.cuh"

namespace nk {

struct MetroArgs {
  int n, m, mp, nc, G, move, nb, n_discard, n_samples;
  int ring;             // slots of the shared-memory table ring (2 .. kMaxRing)
  uint64_t seed, counter;
  const uint64_t* counter_dev;  // if set, the counter is read from here
  const int32_t* bond_i;
  const int32_t* bond_k;
  int8_t* sigma;        // [nc][n]
  int8_t* samples;      // [nc * n_samples][n]
  uint64_t* n_acc;      // [nc] or null
  const double* a;      // master a (F64)
  const void* cd;       // [rows] rows per site (flip) or bond: real_row_stride(mp) or
                        // cplx_row_stride(NU, WPC, mp) bytes (table block, theta
                        // increments, header); group kernel: group_row_bytes(m2p)
  const void* wd;       // unused
  const void* wt;       // [n][mp] F    : W transposed (initial theta)
  const void* b32;      // [mp] F
  // parallel tempering (0 / null: plain sampling): chain c is replica c % pt_R
  // of its ladder, sampling |psi|^(2 beta) with beta = 1 - (c % pt_R) / pt_R
  int pt_R = 0;
  double* lval = nullptr;  // [nc] 2 Re ln psi of each chain's final state, or null
  int acc_add = 0;         // n_acc[c] += accepted (else =)
  int m2p = 0;             // group kernel: unit pairs per table row (threads x pairs)
};

// The step's uniform as a float, from the bits uniform53 takes: within 2^-23
// relative of uniform53(hi, lo) (hi >> 5 is exact below 2^24, rounded once above),
// far inside the accept test's 1e-5 margin; FP64 is kept for near-ties.
__device__ __forceinline__ float uniform53_f(uint32_t hi, uint32_t lo) {
  return __fmaf_rn((float)(hi >> 5), 0x1p-27f, (float)(lo >> 6) * 0x1p-53f);
}

// Accept test U < exp(two_re), decided in FP64.  A float pre-test on
// u32 ~ U with a 1e-5 relative margin settles all but near-ties (the per-step
// path then has no FP64 instruction, which is slow on this GPU); a near-tie
// fetches the bits of the step's U from its lane and compares in FP64.
// Warp-uniform: every lane holds the same two_re and u32.
__device__ __forceinline__ bool accept_test(float u32, float two_re, uint32_t my_uh, uint32_t my_ul,
                                            int src_lane) {
  if (two_re >= 0.f) return true;
  float e32 = __expf(two_re);
  if (u32 < e32 * (1.f - 1e-5f) - 1e-37f) return true;
  if (u32 > e32 * (1.f + 1e-5f) + 1e-37f) return false;
  const uint32_t hi = __shfl_sync(0xffffffffu, my_uh, src_lane);
  const uint32_t lo = __shfl_sync(0xffffffffu, my_ul, src_lane);
  return uniform53(hi, lo) < exp((double)two_re);
}

// A lane's share of log2 prod_j |r_j|^2, made finite before it is summed with
// the other lanes'.  The expanded |r|^2 = |C|^2 + |t|^2 |D|^2 - 2 s Re(t E)
// loses its relative accuracy when |t| is large (theta near a zero of cosh) and
// can round to zero or below for a move whose true |r|^2 is tiny: log2 is then
// -inf or NaN.  Both become -1e30 (the move's ratio underflows to zero and it is
// rejected, as it is in exact arithmetic up to a U below ~1e-30), +inf becomes
// +1e30 (accepted), so that the sums stay finite and a NaN partial can only mean
// a wait that gave up.
__device__ __forceinline__ float clamp_log2(float x) { return fminf(fmaxf(x, -1e30f), 1e30f); }

__device__ __forceinline__ int move_row(const MetroArgs& A, uint64_t ctr, uint32_t g, int step) {
  u4 us = philox_stream(g, ctr + (uint64_t)step, kTagSite, A.seed);
  return uniform_index(us.x, A.move == NK_MOVE_FLIP ? A.n : A.nb);
}

// Thread (chain cw, half h, lane l) of a CTA owns hidden units
// j = 32 (h + WPC q) + l, q < E: WPC warps share a chain and split its hidden
// units; their partial log-products meet in shared memory across a named
// barrier of the pair.  The columns of step t sit in ring slot t % R (R up to
// kMaxRing, as many as shared memory holds).  The warps are not in lockstep:
// each waits for its slot to be filled (full barrier) and releases it when done
// (one count per warp in shared memory); the warp whose release completes the
// count issues the slot's next copy (the step R on) at once, so chains may run
// up to R - 1 steps apart and absorb the uneven work of accepted, rejected and
// null proposals.  A row is one copy: the table block, the theta increments
// and a 16-byte header holding a_i (- a_k) as a float.  theta is kept in tensor
// memory (per-thread TMEM columns, loaded and stored with tcgen05.ld /
// tcgen05.st), which leaves shared memory to the ring.
constexpr int kMaxRing = 8;

// Complex tables: a thread (half h, lane l) owns units j = 32 (h + WPC q) + l,
// q < NU, taken in pairs (2 qp, 2 qp + 1).  A row holds one 1024-byte block per
// (qp, h), in the order qp * WPC + h: 32 float4 (|C|^2 of the pair, |D|^2 of
// the pair), then 32 float4 (Re E of the pair, -Im E of the pair), E = conj(C) D,
// followed by the row's theta increments [mp] float2 (W_i for a flip, W_i - W_k
// for an exchange), so that one bulk copy brings a step's whole slot (a CTA's
// bulk copies complete one after another, a few hundred cycles each).
// Units beyond m hold C = 1, D = 0 (a factor of exactly 1).
__host__ __device__ constexpr size_t cplx_row_bytes(int nu, int wpc) {
  return (size_t)512 * nu * wpc;
}
constexpr int kRowHdr = 16;  // row header: a_i (- a_k) as a float, then padding
__host__ __device__ constexpr size_t cplx_row_stride(int nu, int wpc, int mp) {
  return cplx_row_bytes(nu, wpc) + (size_t)mp * 8 + kRowHdr;
}
// Real rows: [mp] (cosh c, sinh c / s_i), [mp] increments, header.
__host__ __device__ constexpr size_t real_row_stride(int mp) { return (size_t)mp * 12 + kRowHdr; }

__device__ __forceinline__ float2 f2fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 f2mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 f2add(float2 a, float2 b) { return __fadd2_rn(a, b); }

// tanh addition update of two units' t after an accepted move with s_i = si,
// from the unit pair's table values (|C|^2, |D|^2 as c2, d2; Re E, -Im E as
// ex, ney):  Re t' = (t_x (|C|^2 + |D|^2) - s Re E (|t|^2 + 1)) / |r|^2,
//            Im t' = (t_y (|C|^2 - |D|^2) - s Im E (1 - |t|^2)) / |r|^2.
__device__ __forceinline__ void t_add_pair(float2& tx, float2& ty, float2 c2, float2 d2, float2 ex,
                                           float2 ney, float si) {
  const float2 m2s = make_float2(-2.f * si, -2.f * si);
  const float2 ns2 = make_float2(-si, -si), s2 = make_float2(si, si);
  const float2 one = make_float2(1.f, 1.f), mone = make_float2(-1.f, -1.f);
  const float2 tt = f2fma(tx, tx, f2mul(ty, ty));
  const float2 e = f2fma(tx, ex, f2mul(ty, ney));
  const float2 r2 = f2fma(m2s, e, f2fma(tt, d2, c2));
  const float2 inv = make_float2(__fdividef(1.f, r2.x), __fdividef(1.f, r2.y));
  const float2 nx = f2fma(ns2, f2mul(ex, f2add(tt, one)), f2mul(tx, f2add(c2, d2)));
  const float2 ny = f2fma(s2, f2mul(ney, f2fma(tt, mone, one)), f2mul(ty, f2fma(d2, mone, c2)));
  tx = f2mul(nx, inv);
  ty = f2mul(ny, inv);
}

__device__ __forceinline__ void pair_sync(int id, int nthreads) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

constexpr int kThetaChunk = 13;  // TMEM columns per load / wait / store round trip

// Real RBMs, accepted move: theta += m2s * increment for this thread's units
// (TMEM column q = theta of unit q), in chunks of kThetaChunk columns.  The
// stores are not waited for here: the wait comes before the next read of theta
// (the next accepted move, the end-of-sweep refresh, the kernel's end), so that
// their latency overlaps the steps in between.
template <int WPC, int TC, int C0>
__device__ __forceinline__ void theta_add(uint32_t tm, const float* wdc, float m2s, int h, int lane,
                                          int mp) {
  if constexpr (C0 == 0) tmem_st_wait();  // the previous update's stores
  if constexpr (C0 < TC) {
    constexpr int N = (TC - C0) < kThetaChunk ? (TC - C0) : kThetaChunk;
    float v[N];
    tmem_ld_cols<N>(tm + C0, v);
    tmem_ld_wait();
#pragma unroll
    for (int e = 0; e < N; ++e) {
      const int j = 32 * (h + WPC * (C0 + e)) + lane;
      if (j < mp) v[e] = fmaf(m2s, wdc[j], v[e]);
    }
    tmem_st_cols<N>(tm + C0, v);
    theta_add<WPC, TC, C0 + kThetaChunk>(tm, wdc, m2s, h, lane, mp);
  }
}

// Complex RBMs, accepted move: for unit pairs Q0, Q0 + 1, Q0 + 2 (columns
// 4 Q0 .. 4 Q0 + 11), load theta, run tupd(qp) for those pairs (the t update,
// which does not read theta) while the load is in flight, then add m2s times
// the increments and store; then the next three pairs.
template <int Q0, int EP, int WPC, typename Fn>
__device__ __forceinline__ void theta_t_update(uint32_t tm, const float2* wdc, float m2s, int h,
                                               int lane, int mp, Fn&& tupd) {
  if constexpr (Q0 < EP) {
    constexpr int NQ = (EP - Q0) < 3 ? (EP - Q0) : 3;
    float th[4 * NQ];
    tmem_ld_cols<4 * NQ>(tm + 4 * Q0, th);
#pragma unroll
    for (int qp = Q0; qp < Q0 + NQ; ++qp) tupd(qp);
    tmem_ld_wait();
#pragma unroll
    for (int e = 0; e < 4 * NQ; ++e) {
      const int col = 4 * Q0 + e;
      const int j = 32 * (h + WPC * (col / 2)) + lane;
      if (j < mp) th[e] = fmaf(m2s, (col & 1) ? wdc[j].y : wdc[j].x, th[e]);
    }
    tmem_st_cols<4 * NQ>(tm + 4 * Q0, th);
    theta_t_update<Q0 + NQ, EP, WPC>(tm, wdc, m2s, h, lane, mp, tupd);
  }
}

// Read this thread's theta from TMEM in chunks of 16 columns and hand each unit
// (index q, value) to f.
template <bool CPLX, int TC, int C0, typename Fn>
__device__ __forceinline__ void theta_each(uint32_t tm, Fn&& f) {
  if constexpr (C0 < TC) {
    constexpr int N = (TC - C0) < 16 ? (TC - C0) : 16;
    float v[N];
    tmem_ld_cols<N>(tm + C0, v);
    tmem_ld_wait();
    if constexpr (CPLX) {
#pragma unroll
      for (int e = 0; e < N; e += 2) f((C0 + e) / 2, make_float2(v[e], v[e + 1]));
    } else {
#pragma unroll
      for (int e = 0; e < N; ++e) f(C0 + e, v[e]);
    }
    theta_each<CPLX, TC, C0 + 16>(tm, f);
  }
}

// NU hidden units per thread (even for complex RBMs), WPC warps per chain.
template <bool CPLX, int NU, int WPC>
__device__ __forceinline__ void metropolis_body(const MetroArgs& A, const int bx) {
  using F = typename RatioTypes<CPLX>::F;
  using T2 = typename RatioTypes<CPLX>::T2;
  constexpr int E = NU;
  constexpr int EP = (NU + 1) / 2;
  extern __shared__ __align__(128) unsigned char smem[];
  const int mp = A.mp, n = A.n, G = A.G, R = A.ring;
  const size_t cd_row = CPLX ? cplx_row_bytes(NU, WPC) : (size_t)mp * sizeof(T2);
  const size_t slot_bytes = cd_row + (size_t)mp * sizeof(F) + kRowHdr;  // one row
  // ring slot k: the move's row: table block (cd_row bytes), increments [mp] F, header
  float* part = reinterpret_cast<float*>(smem + (size_t)R * slot_bytes);            // [2][G][WPC]
  uint64_t* full = reinterpret_cast<uint64_t*>(part + round_up(2 * G * WPC, 2));    // [kMaxRing]
  uint64_t* empty = full + kMaxRing;                                                 // [kMaxRing]
  uint32_t* tslot = reinterpret_cast<uint32_t*>(empty + kMaxRing);                  // TMEM base
  int8_t* sgall = reinterpret_cast<int8_t*>(tslot + 4);                              // [G*WPC][n16]
  const int n16 = (int)round_up(n, 16);
  const uint64_t ctr = A.counter_dev ? *A.counter_dev : A.counter;

  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int cw = w / WPC, h = w % WPC;
  const int c = bx * G + cw;
  const int chains_here = min(G, A.nc - bx * G);
  const bool active = (cw < G) && (c < A.nc);
  const uint32_t g = (uint32_t)bx;
  int8_t* sg = sgall + (size_t)(active ? w : 0) * n16;  // one copy per warp
  const F* wt = reinterpret_cast<const F*>(A.wt);
  const F* b32 = reinterpret_cast<const F*>(A.b32);
  auto jof = [&](int q) { return 32 * (h + WPC * q) + lane; };

  if (tid == 0) {
    for (int k = 0; k < R; ++k) {
      mbar_init(&full[k], 1);
      reinterpret_cast<int*>(empty)[k] = 0;              // releases of slot k
      reinterpret_cast<int*>(empty)[kMaxRing + k] = 0;   // copies issued into slot k
    }
    mbar_fence_init();
  }
  if (active)
    for (int i = lane; i < n; i += 32) sg[i] = A.sigma[(int64_t)c * n + i];
  // theta lives in tensor memory: thread (warp w, lane l) owns TMEM lane
  // 32 (w % 4) + l, columns (w / 4) * TC .. + TC - 1 (its units' theta)
  constexpr int TC = CPLX ? 2 * NU : NU;
  const uint32_t tcols_total = (uint32_t)(((blockDim.x / 32 + 3) / 4) * TC);
  const uint32_t tcols = tcols_total <= 32 ? 32 : tcols_total <= 64 ? 64 : tcols_total <= 128 ? 128
                         : tcols_total <= 256 ? 256 : 512;
  if (w == 0) tmem_alloc(tslot, tcols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_th = *tslot + ((uint32_t)(32 * (w & 3)) << 16) + (uint32_t)((w >> 2) * TC);

  // theta = W sigma + b: rows of W^T staged through the (not yet used) ring
  float t[CPLX ? 1 : E];             // real: t of unit q
  float2 tx[CPLX ? EP : 1], ty[CPLX ? EP : 1];  // complex: Re t, Im t of units (2 qp, 2 qp + 1)
  auto set_t = [&](int q, F x, bool valid) {
    if constexpr (CPLX) {
      cf tt = valid ? tanh_c(cf{x.x, x.y}) : cf{0.f, 0.f};
      if (q & 1) {
        tx[q >> 1].y = tt.x;
        ty[q >> 1].y = tt.y;
      } else {
        tx[q >> 1].x = tt.x;
        ty[q >> 1].x = tt.y;
      }
    } else {
      t[q] = valid ? tanh_f(x) : 0.f;
    }
  };
  {
    F* stg = reinterpret_cast<F*>(smem);
    const int KC = (int)(((size_t)R * slot_bytes) / ((size_t)mp * sizeof(F)));
    F acc[E];
#pragma unroll
    for (int q = 0; q < E; ++q) {
      if constexpr (CPLX) acc[q] = make_float2(0.f, 0.f); else acc[q] = 0.f;
      if (jof(q) < mp) acc[q] = b32[jof(q)];
    }
    for (int i0 = 0; i0 < n; i0 += KC) {
      const int kc = min(KC, n - i0);
      for (int x = tid; x < kc * mp; x += blockDim.x) stg[x] = wt[(int64_t)i0 * mp + x];
      __syncthreads();
      if (active) {
        for (int kk = 0; kk < kc; ++kk) {
          const float si = (float)sg[i0 + kk];
#pragma unroll
          for (int q = 0; q < E; ++q) {
            if (jof(q) < mp) {
              F wv = stg[kk * mp + jof(q)];
              if constexpr (CPLX) {
                acc[q].x = fmaf(si, wv.x, acc[q].x);
                acc[q].y = fmaf(si, wv.y, acc[q].y);
              } else {
                acc[q] = fmaf(si, wv, acc[q]);
              }
            }
          }
        }
      }
      __syncthreads();
    }
#pragma unroll
    for (int q = 0; q < E; ++q) set_t(q, acc[q], jof(q) < mp);
    if (active) {
      tmem_st_cols<TC>(tmem_th, reinterpret_cast<const float*>(acc));
      tmem_st_wait();
    }
  }
  __syncthreads();
  // inactive warps skip the steps (no CTA-wide barrier until the end)
  const int total = active ? (A.n_discard + A.n_samples) * n : 0;
  const uint32_t cd_bytes = (uint32_t)cd_row, wd_bytes = (uint32_t)(mp * sizeof(F));
  const uint32_t row_bytes = (uint32_t)slot_bytes;  // table block, increments, header
  const unsigned char* rows = reinterpret_cast<const unsigned char*>(A.cd);
  // per slot: releases of its current step, copies issued into it
  int* rel = reinterpret_cast<int*>(empty);
  int* iss = rel + kMaxRing;
  const int nwarps = chains_here * WPC;  // every active warp releases every step's slot
  auto issue = [&](int step, int row) {   // one thread
    const int k = step % R;
    ++iss[k];
    mbar_arrive_expect_tx(&full[k], row_bytes);
    bulk_g2s(smem + (size_t)k * slot_bytes, rows + (int64_t)row * slot_bytes, row_bytes, &full[k]);
  };
  // inverse temperature of this chain (exactly 1 without tempering, so that the
  // accept test below is unchanged bit for bit)
  const float beta = A.pt_R > 0 ? 1.f - (float)(c % A.pt_R) / (float)A.pt_R : 1.f;
  if (tid == 0) {
    // the staging writes above (generic proxy) before the copies (async proxy)
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    for (int s = 0; s < R && s < total; ++s) issue(s, move_row(A, ctr, g, s));
  }

  uint64_t nacc = 0;
  bool timed_out = false;  // a bounded wait gave up: finish the loop without work
  int nn = 0;              // non-null steps so far (identical in the warps of a chain)
  int sweep_pos = 0, sweep_no = 0;  // step within the sweep, sweeps completed
  int kslot = 0;          // ring slot of the current step (step % R)
  uint32_t kphase = 0u;   // phase of its full barrier ((step / R) & 1)
  // per lane, drawn one 32-step block ahead: the row (site or bond) of step
  // (block start + lane) and of the next block's step (for refills), the sites of
  // the move (their loads land during the block before they are used), and the
  // accept draw of step (block start + lane) as a float for the test and as bits
  // (FP64 only on near-ties)
  int row_cur = 0, row_nxt = 0, my_i = 0, my_k = -1, nx_i = 0, nx_k = -1;
  uint32_t my_uh = 0u, my_ul = 0u;
  float my_u32 = 0.f;
  auto sites_of = [&](int row, int& si_, int& sk_) {
    if (A.move == NK_MOVE_FLIP) {
      si_ = row;
      sk_ = -1;
    } else {
      si_ = A.bond_i[row];
      sk_ = A.bond_k[row];
    }
  };
  for (int step = 0; step < total; ++step) {
    const int q32 = step & 31;
    if (q32 == 0) {
      if (step == 0) {
        row_nxt = move_row(A, ctr, g, lane);
        sites_of(row_nxt, nx_i, nx_k);
      }
      row_cur = row_nxt;
      my_i = nx_i;
      my_k = nx_k;
      row_nxt = move_row(A, ctr, g, step + 32 + lane);
      sites_of(row_nxt, nx_i, nx_k);
      const u4 ua = philox_stream((uint32_t)c, ctr + (uint64_t)(step + lane), kTagAccept, A.seed);
      my_uh = ua.x;
      my_ul = ua.y;
      my_u32 = uniform53_f(ua.x, ua.y);
    }
    const int i = __shfl_sync(0xffffffffu, my_i, q32);
    const int kk2 = __shfl_sync(0xffffffffu, my_k, q32);
    const float u32 = __shfl_sync(0xffffffffu, my_u32, q32);
    const int k = kslot;
    const T2* cd = reinterpret_cast<const T2*>(smem + (size_t)k * slot_bytes);
    const F* wdc = reinterpret_cast<const F*>(smem + (size_t)k * slot_bytes + cd_bytes);
    const float si = (float)sg[i];
    const bool null_move = (kk2 >= 0) && (sg[kk2] == sg[i]);
    // every warp observes every phase of the slot's barrier, in order, so that
    // no barrier is ever more than one phase ahead of a waiting warp
    if (!timed_out) {
      const bool ok = mbar_wait_bounded(&full[k], kphase);
      timed_out = __any_sync(0xffffffffu, !ok);  // warp-uniform
    }
    if (!null_move) {
      float l2 = 0.f;
      if (!timed_out) {
        if constexpr (CPLX) {
          // four packed running products of |r|^2; with at most 16 pairs each
          // lane collects at most 4 factors, so no renormalisation is needed
          // for factors in (2^-31, 2^31)
          const float4* row4 = reinterpret_cast<const float4*>(smem + (size_t)k * slot_bytes);
          const float2 m2s = make_float2(-2.f * si, -2.f * si);
          float2 Pp[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) Pp[u] = make_float2(1.f, 1.f);
#pragma unroll
          for (int qp = 0; qp < EP; ++qp) {
            const float4 q0 = row4[(qp * WPC + h) * 64 + lane];
            const float4 q1 = row4[(qp * WPC + h) * 64 + 32 + lane];
            const float2 c2 = make_float2(q0.x, q0.y), d2 = make_float2(q0.z, q0.w);
            const float2 ex = make_float2(q1.x, q1.y), ney = make_float2(q1.z, q1.w);
            const float2 tt = f2fma(tx[qp], tx[qp], f2mul(ty[qp], ty[qp]));
            const float2 e = f2fma(tx[qp], ex, f2mul(ty[qp], ney));  // Re(t E)
            Pp[qp & 3] = f2mul(Pp[qp & 3], f2fma(m2s, e, f2fma(tt, d2, c2)));
          }
          l2 = 0.f;
#pragma unroll
          for (int u = 0; u < (EP < 4 ? EP : 4); ++u) l2 += __log2f(Pp[u].x) + __log2f(Pp[u].y);
        } else {
        // four independent running products, renormalised every 8 factors each
        ScaledReal P[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) P[u].init();
#pragma unroll
        for (int q = 0; q < E; ++q) {
          if (jof(q) < mp) {
            const T2 v = cd[jof(q)];
            P[q & 3].v *= fmaf(-si * t[q], v.y, v.x);
          }
          if ((q & 31) == 31) {
#pragma unroll
            for (int u = 0; u < 4; ++u) P[u].renorm();
          }
        }
        l2 = P[0].log2v() + P[1].log2v() + P[2].log2v() + P[3].log2v();
        }
        l2 = clamp_log2(l2);
#pragma unroll
        for (int off = 16; off >= 1; off >>= 1) l2 += __shfl_xor_sync(0xffffffffu, l2, off);
      }
      if (WPC > 1) {
        // partial buffer indexed by the non-null step count: a warp's next write
        // to it comes after the partner has passed the next pair barrier.  A
        // timed-out warp contributes NaN, so both warps of the chain see it and
        // take the same (no-op) decision, keeping their sigma copies identical.
        float* pslot = part + (nn & 1) * G * WPC;
        if (lane == 0) pslot[cw * WPC + h] = timed_out ? __int_as_float(0x7fc00000) : l2;
        pair_sync(1 + cw, 32 * WPC);
        l2 = 0.f;
#pragma unroll
        for (int hh = 0; hh < WPC; ++hh) l2 += pslot[cw * WPC + hh];
        if (isnan(l2)) timed_out = true;
      }
      ++nn;
      // visible term -2 s_i a_i (- 2 s_k a_k) = -2 s_i (a_i - a_k) (s_k = -s_i),
      // in FP32 like the hidden-unit product; a_i (- a_k) from the row's header
      const float da = *reinterpret_cast<const float*>(smem + (size_t)k * slot_bytes + cd_bytes +
                                                       wd_bytes);
      const float two_re = (CPLX ? 1.f : 2.f) * 0.69314718055994531f * l2 - 4.f * si * da;
      if (!timed_out && accept_test(u32, beta * two_re, my_uh, my_ul, q32)) {
        ++nacc;
        if constexpr (CPLX) {
          // theta's columns of three unit pairs at a time are read before those
          // pairs' t is updated, so that the tensor-memory loads complete under
          // the tanh-addition arithmetic
          const float4* row4 = reinterpret_cast<const float4*>(smem + (size_t)k * slot_bytes);
          tmem_st_wait();  // the previous update's stores
          theta_t_update<0, EP, WPC>(tmem_th, wdc, -2.f * si, h, lane, mp, [&](int qp) {
            const float4 q0 = row4[(qp * WPC + h) * 64 + lane];
            const float4 q1 = row4[(qp * WPC + h) * 64 + 32 + lane];
            t_add_pair(tx[qp], ty[qp], make_float2(q0.x, q0.y), make_float2(q0.z, q0.w),
                       make_float2(q1.x, q1.y), make_float2(q1.z, q1.w), si);
          });
        } else {
#pragma unroll
          for (int q = 0; q < E; ++q) {
            const int j = jof(q);
            if (j < mp) {
              const T2 v = cd[j];
              const float r = fmaf(-si * t[q], v.y, v.x);
              t[q] = __fdividef(fmaf(t[q], v.x, -si * v.y), r);
            }
          }
          theta_add<WPC, TC, 0>(tmem_th, wdc, -2.f * si, h, lane, mp);
        }
        __syncwarp();
        if (lane == 0) {
          sg[i] = (int8_t)(-sg[i]);
          if (kk2 >= 0) sg[kk2] = (int8_t)(-sg[kk2]);
        }
      }
    }
    // release slot k; the last warp to release it refills it with the step R on
    // (its row drawn by this warp's lanes), so that no copy waits for a
    // particular warp to come round
    __syncwarp();
    bool last = false;
    if (lane == 0) {
      __threadfence_block();  // this warp's reads of the slot before the release
      last = atomicAdd(&rel[k], 1) == nwarps - 1;
      if (last) atomicExch(&rel[k], 0);
    }
    last = __shfl_sync(0xffffffffu, (int)last, 0) != 0;
    if (last && !timed_out && step + R < total) {
      const int tq = q32 + R;  // the refill's offset from this block's start (< 64)
      const int rc = __shfl_sync(0xffffffffu, row_cur, tq & 31);
      const int rn = __shfl_sync(0xffffffffu, row_nxt, tq & 31);
      if (lane == 0) {
        __threadfence_block();
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        issue(step + R, tq < 32 ? rc : rn);
      }
    }
    if (++sweep_pos == n) {  // the last step of a sweep
      sweep_pos = 0;
      const int sweep = sweep_no++;
      if (sweep >= A.n_discard && h == 0) {
        int8_t* out = A.samples + ((int64_t)c * A.n_samples + (sweep - A.n_discard)) * n;
        for (int ii = lane; ii < n; ii += 32) out[ii] = sg[ii];
      }
      // exact refresh of t from theta (this thread's own entries)
      tmem_st_wait();
      theta_each<CPLX, TC, 0>(tmem_th, [&](int q, F x) {
        if (jof(q) < mp) set_t(q, x, true);
      });
    }
    if (++kslot == R) {
      kslot = 0;
      kphase ^= 1u;
    }
  }
  tmem_st_wait();  // the last update's stores, before the columns are freed
  if (A.lval && active) {
    // 2 Re ln psi of the final state: Re ln cosh of this thread's units from
    // theta in tensor memory (FP32 each, summed in FP64), reduced over the
    // chain's lanes and warps; the visible term in FP64 from the master a
    double lr = 0.0;
    theta_each<CPLX, TC, 0>(tmem_th, [&](int q, F x) {
      if (jof(q) < A.m) {
        if constexpr (CPLX) lr += (double)lncosh_c(cf{x.x, x.y}).x;
        else lr += (double)lncosh_f(x);
      }
    });
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) lr += __shfl_xor_sync(0xffffffffu, lr, off);
    if (WPC > 1) {
      // the chain's own slots of the pair partials (both parity halves) carry
      // each warp's sum as hi + lo floats; the first barrier makes sure that
      // both warps have left the step loop, whose last reads used those slots
      pair_sync(1 + cw, 32 * WPC);
      if (lane == 0) {
        const float hi = (float)lr;
        part[cw * WPC + h] = hi;
        part[G * WPC + cw * WPC + h] = (float)(lr - (double)hi);
      }
      pair_sync(1 + cw, 32 * WPC);
      lr = 0.0;
      for (int hh = 0; hh < WPC; ++hh)
        lr += (double)part[cw * WPC + hh] + (double)part[G * WPC + cw * WPC + hh];
    }
    if (h == 0 && lane == 0) {
      double va = 0.0;
      for (int ii = 0; ii < n; ++ii) va += (CPLX ? A.a[2 * ii] : A.a[ii]) * (double)sg[ii];
      A.lval[c] = timed_out ? __longlong_as_double(0x7ff8000000000000ll) : 2.0 * (lr + va);
    }
  }
  if (timed_out && lane == 0) dev_status_set(1u << NK_ERR_TIMEOUT);
  if (active && h == 0) {
    for (int ii = lane; ii < n; ii += 32) A.sigma[(int64_t)c * n + ii] = sg[ii];
    if (A.n_acc && lane == 0) {
      if (timed_out) A.n_acc[c] = ~0ull;
      else if (A.acc_add) {
        if (A.n_acc[c] != ~0ull) A.n_acc[c] += nacc;  // a timeout marked earlier stays
      }
      else A.n_acc[c] = nacc;
    }
  }
  tc_fence_before();
  __syncthreads();
  if (tid == 0) {
    // copies still in flight (a timed-out run) land before the CTA exits: the
    // last copy issued into each slot
    const int* iss = reinterpret_cast<const int*>(empty) + kMaxRing;
    for (int k = 0; k < R; ++k)
      if (iss[k] > 0) mbar_wait_bounded(&full[k], (uint32_t)((iss[k] - 1) & 1), 1u << 20);
  }
  if (w == 0) {
    tc_fence_after();
    tmem_dealloc(*tslot, tcols);
  }
}

template <bool CPLX, int NU, int WPC>
__global__ void __launch_bounds__(512, 1) metropolis_kernel(MetroArgs A) {
  metropolis_body<CPLX, NU, WPC>(A, blockIdx.x);
}

// Up to kMetroBatch independent problems of one kernel template in one launch:
// CTA b runs block b - start[k] of problem k (start[k] <= b < start[k + 1]), with
// that problem's arguments, exactly as its own launch would.
constexpr int kMetroBatch = 64;
struct MetroBatch {
  int n;
  int start[kMetroBatch + 1];
  MetroArgs a[kMetroBatch];
};

template <bool CPLX, int NU, int WPC>
__global__ void __launch_bounds__(512, 1) metropolis_batch_kernel(const __grid_constant__ MetroBatch B) {
  int k = 0;
  while (k + 1 < B.n && (int)blockIdx.x >= B.start[k + 1]) ++k;
  metropolis_body<CPLX, NU, WPC>(B.a[k], (int)blockIdx.x - B.start[k]);
}

}  // namespace nk

#include "metro_group.cuh"

namespace nk {

// Rows of a real RBM (layout of real_row_stride), one per site (flips: the
// site's (cosh 2W_i, sinh 2W_i) and W_i) or bond (exchanges, s_k = -s_i:
// cosh c = A_i A_k - B_i B_k, sinh c / s_i = B_i A_k - A_i B_k, increment
// W_i - W_k), each with its header a_i (- a_k).  Element x of rows * mp.
__device__ __forceinline__ void real_rows_elem(int64_t x, bool pair, const float2* __restrict__ tab,
                                               const float* __restrict__ wt,
                                               const int32_t* __restrict__ bi,
                                               const int32_t* __restrict__ bk,
                                               const double* __restrict__ a, int mp,
                                               unsigned char* __restrict__ out) {
  const int r = (int)(x / mp), j = (int)(x % mp);
  unsigned char* base = out + (int64_t)r * real_row_stride(mp);
  float2* cd = reinterpret_cast<float2*>(base);
  float* wd = reinterpret_cast<float*>(base + (size_t)mp * 8);
  const int i = pair ? bi[r] : r;
  const float2 ti = tab[(int64_t)i * mp + j];
  if (pair) {
    const int k = bk[r];
    const float2 tk = tab[(int64_t)k * mp + j];
    cd[j] = make_float2(fmaf(-ti.y, tk.y, ti.x * tk.x), fmaf(-ti.x, tk.y, ti.y * tk.x));
    wd[j] = wt[(int64_t)i * mp + j] - wt[(int64_t)k * mp + j];
    if (j == 0) *reinterpret_cast<float*>(base + (size_t)mp * 12) = (float)(a[i] - a[k]);
  } else {
    cd[j] = ti;
    wd[j] = wt[(int64_t)i * mp + j];
    if (j == 0) *reinterpret_cast<float*>(base + (size_t)mp * 12) = (float)a[i];
  }
}

// Pair rows of a complex RBM (layout of cplx_row_stride): one per site (flips,
// C = A_i, D = B_i, increments W_i) or per bond (exchanges, s_k = -s_i:
// C = A_i A_k - B_i B_k, D = B_i A_k - A_i B_k, increments W_i - W_k), each with
// its header Re a_i (- Re a_k).  Element x of rows * (nu / 2) * wpc * 32.
__device__ __forceinline__ void cplx_rows_elem(int64_t x, bool pair, const float4* __restrict__ tab,
                                               const float2* __restrict__ wt,
                                               const int32_t* __restrict__ bi,
                                               const int32_t* __restrict__ bk,
                                               const double* __restrict__ a, int mp, int nu,
                                               int wpc, unsigned char* __restrict__ qout) {
  const int nblk = (nu / 2) * wpc;
  const int lane = (int)(x & 31);
  const int64_t rb = x >> 5;
  const int blk = (int)(rb % nblk), r = (int)(rb / nblk);
  const int qp = blk / wpc, h = blk % wpc;
  unsigned char* base = qout + (int64_t)r * cplx_row_stride(nu, wpc, mp);
  float2* wd = reinterpret_cast<float2*>(base + cplx_row_bytes(nu, wpc));
  if (blk == 0 && lane == 0)
    *reinterpret_cast<float*>(base + cplx_row_bytes(nu, wpc) + (size_t)mp * 8) =
        pair ? (float)(a[2 * bi[r]] - a[2 * bk[r]]) : (float)a[2 * r];
  float v[2][4];
#pragma unroll
  for (int u = 0; u < 2; ++u) {
    const int j = 32 * (h + wpc * (2 * qp + u)) + lane;
    cf C{1.f, 0.f}, D{0.f, 0.f};
    if (j < mp) {
      const int i = pair ? bi[r] : r;
      const float4 ti = tab[(int64_t)i * mp + j];
      const cf Ai{ti.x, ti.y}, Bi{ti.z, ti.w};
      if (pair) {
        const int k = bk[r];
        const float4 tk = tab[(int64_t)k * mp + j];
        const cf Ak{tk.x, tk.y}, Bk{tk.z, tk.w};
        C = Ai * Ak - Bi * Bk;
        D = Bi * Ak - Ai * Bk;
        const float2 wi = wt[(int64_t)i * mp + j], wk = wt[(int64_t)k * mp + j];
        wd[j] = make_float2(wi.x - wk.x, wi.y - wk.y);
      } else {
        C = Ai;
        D = Bi;
        wd[j] = wt[(int64_t)i * mp + j];
      }
    }
    const cf E = conj(C) * D;
    v[u][0] = fmaf(C.x, C.x, C.y * C.y);
    v[u][1] = fmaf(D.x, D.x, D.y * D.y);
    v[u][2] = E.x;
    v[u][3] = -E.y;
  }
  float4* row = reinterpret_cast<float4*>(base) + (int64_t)blk * 64;
  row[lane] = make_float4(v[0][0], v[1][0], v[0][1], v[1][1]);
  row[32 + lane] = make_float4(v[0][2], v[1][2], v[0][3], v[1][3]);
}


// The table builds of many problems in one launch: job k owns elements
// [start[k], start[k + 1]) of the concatenated index range.
enum { kTabNone = 0, kTabRealPair = 1, kTabCplxFlip = 2, kTabCplxPair = 3, kTabGroupFlip = 4,
       kTabGroupPair = 5, kTabRealFlip = 6 };
struct TableJob {
  int kind, mp, nu, wpc;
  const void* tab;
  const void* wt;
  const int32_t* bi;
  const int32_t* bk;
  void* out;
  void* wd;
  int m = 0, m2p = 0;  // group rows
  const double* a = nullptr;  // master visible biases (row headers)
};
struct TableBatch {
  int n;
  int64_t start[kMetroBatch + 1];
  TableJob j[kMetroBatch];
};

__global__ void tables_batch_kernel(const __grid_constant__ TableBatch B) {
  const int64_t total = B.start[B.n];
  for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < total;
       x += (int64_t)gridDim.x * blockDim.x) {
    int lo = 0, hi = B.n - 1;  // the job whose range holds x
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (B.start[mid] <= x) lo = mid; else hi = mid - 1;
    }
    const TableJob& J = B.j[lo];
    const int64_t e = x - B.start[lo];
    if (J.kind == kTabRealPair || J.kind == kTabRealFlip)
      real_rows_elem(e, J.kind == kTabRealPair, (const float2*)J.tab, (const float*)J.wt, J.bi,
                     J.bk, J.a, J.mp, (unsigned char*)J.out);
    else if (J.kind == kTabGroupFlip || J.kind == kTabGroupPair)
      group_rows_elem(e, J.kind == kTabGroupPair, (const float4*)J.tab, (const float2*)J.wt, J.bi,
                      J.bk, J.m, J.mp, J.m2p, (float4*)J.out);
    else
      cplx_rows_elem(e, J.kind == kTabCplxPair, (const float4*)J.tab, (const float2*)J.wt, J.bi,
                     J.bk, J.a, J.mp, J.nu, J.wpc, (unsigned char*)J.out);
  }
}

struct CounterBatch {
  int n;
  uint64_t* ctr[kMetroBatch];
  uint64_t delta[kMetroBatch];
};
__global__ void advance_counters_kernel(const __grid_constant__ CounterBatch B) {
  const int k = threadIdx.x;
  if (k < B.n) *B.ctr[k] += B.delta[k];
}

__global__ void advance_counter_kernel(uint64_t* ctr, uint64_t delta) { *ctr += delta; }

// ------------------------------------------------------------------ dispatch

// Hidden units per thread NU for WPC warps per chain: the smallest instantiated
// size >= mp / (32 WPC); complex RBMs need an even NU.  0 if m is too large.
static int metro_nu(int mp, int cplx, int wpc) {
  const int e = (mp + 32 * wpc - 1) / (32 * wpc);
  static const int real1[] = {1, 2, 4, 8, 16, 32, 64}, real2[] = {8, 13, 16, 25, 32};
  static const int cplx1[] = {2, 4, 8, 16, 32, 64}, cplx2[] = {8, 14, 16, 26, 32};
  const int* L = cplx ? (wpc == 1 ? cplx1 : cplx2) : (wpc == 1 ? real1 : real2);
  const int nl = cplx ? (wpc == 1 ? 6 : 5) : (wpc == 1 ? 7 : 5);
  for (int x = 0; x < nl; ++x)
    if (L[x] >= e) return L[x];
  return 0;
}

// two warps per chain from mp = 512 on, when the group fits in 512 threads
static int metro_wpc(int mp, int G) { return (mp >= 512 && G * 64 <= 512) ? 2 : 1; }

size_t metropolis_scratch_bytes(int n, int m, int cplx, int move, int nb) {
  const int mp = padded_m(m);
  const size_t f = cplx ? 8 : 4;
  if (!cplx) {
    (void)f;
    const int64_t rows = move == NK_MOVE_FLIP ? n : nb;
    return (size_t)round_up(rows * (int64_t)real_row_stride(mp), 256);
  }
  // the row layout depends on the warps per chain (group size): take the larger
  size_t row = 0;
  for (int wpc = 1; wpc <= 2; ++wpc) {
    if (wpc == 2 && mp < 512) continue;
    const int nu = metro_nu(mp, 1, wpc);
    if (nu) row = std::max(row, cplx_row_stride(nu, wpc, mp));
  }
  (void)f;
  const int64_t rows = move == NK_MOVE_FLIP ? n : nb;
  size_t bytes = (size_t)round_up((int64_t)(rows * row), 256);
  // or the group kernel's rows (any of its unit-pair choices)
  size_t grow = 0;
  for (int pp = 1; pp <= 3; ++pp)
    if (group_threads(m, pp) <= group_max_threads(pp))
      grow = std::max(grow, group_row_bytes(group_threads(m, pp) * pp));
  return std::max(bytes, (size_t)round_up((int64_t)rows * (int64_t)grow, 256));
}

// Launch functors for the kernel templates: one problem, or a batch of problems
// sharing a template (field, hidden units per lane, warps per chain, group size).
struct SingleLaunch {
  const MetroArgs& A;
  size_t smem;
  cudaStream_t st;
  template <bool CPLX, int NU, int WPC>
  nk_status go() const {
    auto kern = metropolis_kernel<CPLX, NU, WPC>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
      return fail(NK_ERR_CUDA, "nk_metropolis_sweep: cannot reserve %zu B shared memory", smem);
    const int blocks = (A.nc + A.G - 1) / A.G;
    kern<<<blocks, 32 * A.G * WPC, smem, st>>>(A);
    return check_launch("nk_metropolis_sweep");
  }
};

struct BatchLaunch {
  const MetroBatch& B;
  int G;
  size_t smem;
  cudaStream_t st;
  template <bool CPLX, int NU, int WPC>
  nk_status go() const {
    auto kern = metropolis_batch_kernel<CPLX, NU, WPC>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
      return fail(NK_ERR_CUDA, "nk_batch_sweep: cannot reserve %zu B shared memory", smem);
    kern<<<B.start[B.n], 32 * G * WPC, smem, st>>>(B);
    return check_launch("nk_batch_sweep");
  }
};

struct GroupSingleLaunch {
  const MetroArgs& A;
  int threads;
  size_t smem;
  cudaStream_t st;
  template <int PP>
  nk_status go() const {
    auto kern = metropolis_group_kernel<PP>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
      return fail(NK_ERR_CUDA, "nk_metropolis_sweep: cannot reserve %zu B shared memory", smem);
    const int blocks = (A.nc + A.G - 1) / A.G;
    kern<<<blocks, threads, smem, st>>>(A);
    return check_launch("nk_metropolis_sweep");
  }
};

struct GroupBatchLaunch {
  const MetroBatch& B;
  int threads;
  size_t smem;
  cudaStream_t st;
  template <int PP>
  nk_status go() const {
    auto kern = metropolis_group_batch_kernel<PP>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
      return fail(NK_ERR_CUDA, "nk_batch_sweep: cannot reserve %zu B shared memory", smem);
    kern<<<B.start[B.n], threads, smem, st>>>(B);
    return check_launch("nk_batch_sweep");
  }
};

template <class Fn>
static nk_status launch_group(int pp, const Fn& fn) {
  switch (pp) {
    case 1: return fn.template go<1>();
    case 2: return fn.template go<2>();
    case 3: return fn.template go<3>();
  }
  return fail(NK_ERR_SHAPE, "nk_metropolis_sweep: %d unit pairs per thread", pp);
}

template <bool CPLX, class Fn>
static nk_status launch_c(int nu, int wpc, int m, const Fn& fn) {
  if (wpc == 1) {
    if constexpr (CPLX) {
      switch (nu) {
        case 2: return fn.template go<true, 2, 1>();
        case 4: return fn.template go<true, 4, 1>();
        case 8: return fn.template go<true, 8, 1>();
        case 16: return fn.template go<true, 16, 1>();
        case 32: return fn.template go<true, 32, 1>();
        case 64: return fn.template go<true, 64, 1>();
      }
    } else {
      switch (nu) {
        case 1: return fn.template go<false, 1, 1>();
        case 2: return fn.template go<false, 2, 1>();
        case 4: return fn.template go<false, 4, 1>();
        case 8: return fn.template go<false, 8, 1>();
        case 16: return fn.template go<false, 16, 1>();
        case 32: return fn.template go<false, 32, 1>();
        case 64: return fn.template go<false, 64, 1>();
      }
    }
  } else {
    if constexpr (CPLX) {
      switch (nu) {
        case 8: return fn.template go<true, 8, 2>();
        case 14: return fn.template go<true, 14, 2>();
        case 16: return fn.template go<true, 16, 2>();
        case 26: return fn.template go<true, 26, 2>();
        case 32: return fn.template go<true, 32, 2>();
      }
    } else {
      switch (nu) {
        case 8: return fn.template go<false, 8, 2>();
        case 13: return fn.template go<false, 13, 2>();
        case 16: return fn.template go<false, 16, 2>();
        case 25: return fn.template go<false, 25, 2>();
        case 32: return fn.template go<false, 32, 2>();
      }
    }
  }
  return fail(NK_ERR_SHAPE, "nk_metropolis_sweep: m = %d exceeds the register-resident limit 2048",
              m);
}

// Everything one sweep call needs, checked and laid out, before anything is
// enqueued: the kernel arguments, its template and shared memory, the table
// build (if any) and the device-counter advance.
struct MetroPlan {
  MetroArgs A;
  bool cplx;
  int nu, wpc;
  int group_pp = 0;   // > 0: the group kernel with this many unit pairs per thread
  int threads = 0;    // its block size
  size_t smem;
  TableJob tj;
  int64_t tab_elems;
  uint64_t* ctr_dev;
  uint64_t advance;
};

static nk_status plan_metropolis(const nk_rbm* r, const nk_chains* ch, int move,
                                 const int32_t* bi, const int32_t* bk, int nb, int n_discard,
                                 int n_samples, int8_t* samples, uint64_t* n_acc, void* scratch,
                                 size_t scratch_bytes, const MetroPt* pt, MetroPlan* P) {
  WsLayout L(r->n, r->m, r->is_complex);
  MetroArgs& A = P->A;
  A = MetroArgs();
  if (pt) {
    A.pt_R = pt->R;
    A.lval = pt->lval;
    A.acc_add = pt->acc_add;
  }
  const bool skip_tables = pt && pt->skip_tables;
  A.n = r->n;
  A.m = r->m;
  A.mp = L.mp;
  A.nc = ch->nc;
  A.G = ch->group_size;
  A.move = move;
  A.nb = nb;
  A.n_discard = n_discard;
  A.n_samples = n_samples;
  A.seed = ch->seed;
  A.counter = ch->counter;
  A.counter_dev = ch->counter_dev;
  A.bond_i = bi;
  A.bond_k = bk;
  A.sigma = ch->sigma;
  A.samples = samples;
  A.n_acc = n_acc;
  A.a = r->a;
  const char* ws = (const char*)r->ws;
  A.wt = ws + L.wt;
  A.b32 = ws + L.b32;
  const bool cplx = r->is_complex != 0;
  // kernel: one CTA per proposal group (complex RBMs, group_size <= 8) or one
  // or two warps per chain
  const int choice = r->sampler;
  if (choice < 0 || choice > 4)
    return fail(NK_ERR_SHAPE, "nk_metropolis_sweep: sampler %d is not 0..4", choice);
  // built-in choice (measured on the 1D Heisenberg shapes, 16384 chains): the
  // group kernel with one unit pair per thread up to m = 256 (1.3 - 1.7x faster
  // at m = 80 - 160), warps per chain from m = 400 to 2048 (1.2 - 1.35x faster
  // there), the group kernel with three pairs per thread above 2048 (the only
  // one that holds t on chip there)
  int gpp = 0;
  if (cplx && A.G <= kGroupChains) {
    if (choice == 0)
      gpp = r->m <= 256 ? 1 : (r->m > 2048 ? 3 : 0);
    else if (choice >= 2)
      gpp = choice - 1;
  }
  if (gpp && group_threads(r->m, gpp) > group_max_threads(gpp)) gpp = 0;
  if (choice >= 2 && !gpp)
    return fail(NK_ERR_SHAPE,
                "nk_metropolis_sweep: sampler %d needs a complex RBM, group_size <= 8 and "
                "m <= %d",
                choice, 2 * (choice - 1) * group_max_threads(choice - 1));
  if (gpp) {
    const int T = group_threads(r->m, gpp), NW = T / 32;
    const int m2p = T * gpp;
    const size_t row = group_row_bytes(m2p);
    const size_t need = metropolis_scratch_bytes(r->n, r->m, 1, move, nb);
    if (!scratch || scratch_bytes < need)
      return fail(NK_ERR_SHAPE, "nk_metropolis_sweep: scratch of %zu B, need %zu B",
                  scratch_bytes, need);
    // ring depth: as many row slots as fit next to the partials, barriers and
    // the per-warp spin bytes (theta lives in tensor memory)
    const size_t rest = (size_t)64 * NW + 8 * kMaxRing + 16 + (size_t)NW * round_up(r->n, 16);
    const size_t cap = 227 * 1024;
    const int ring =
        rest + 2 * row > cap ? 0 : (int)std::min<size_t>(kMaxRing, (cap - rest) / row);
    if (ring < 2)
      return fail(NK_ERR_SHAPE,
                  "nk_metropolis_sweep: m = %d leaves room for fewer than two row slots in "
                  "227 KB of shared memory",
                  r->m);
    if ((int64_t)(n_discard + n_samples) * r->n > 0x7fffffff)
      return fail(NK_ERR_SHAPE, "nk_metropolis_sweep: too many proposals in one call");
    A.ring = ring;
    A.m2p = m2p;
    A.cd = scratch;
    A.wd = nullptr;
    P->cplx = true;
    P->nu = 0;
    P->wpc = 0;
    P->group_pp = gpp;
    P->threads = T;
    // tensor memory admits 512 / tcols CTAs per SM: ask for enough shared
    // memory that no more are resident (228 KB per SM, 1 KB reserved per CTA)
    const int tcw = 32 * gpp * ((NW + 3) / 4);
    const int tcols = tcw <= 32 ? 32 : tcw <= 64 ? 64 : tcw <= 128 ? 128 : tcw <= 256 ? 256 : 512;
    const size_t floor_smem = (size_t)233472 / (size_t)(512 / tcols + 1) + 1 - 1024;
    P->smem = std::max((size_t)ring * row + rest, floor_smem);
    P->ctr_dev = ch->counter_dev;
    P->advance = (uint64_t)(n_discard + n_samples) * r->n;
    const int rows = move == NK_MOVE_FLIP ? r->n : nb;
    TableJob& J = P->tj;
    J = TableJob{move == NK_MOVE_FLIP ? kTabGroupFlip : kTabGroupPair,
                 L.mp, 0, 0, ws + L.tab, ws + L.wt, bi, bk, scratch, nullptr, r->m, m2p};
    P->tab_elems = (int64_t)rows * m2p;
    if (skip_tables) {  // rows of an earlier launch of the same call
      J.kind = kTabNone;
      P->tab_elems = 0;
    }
    return NK_OK;
  }
  const size_t f = cplx ? 8 : 4;
  const int wpc = metro_wpc(L.mp, A.G);
  const int nu = metro_nu(L.mp, cplx, wpc);
  if (!nu)
    return fail(NK_ERR_SHAPE,
                "nk_metropolis_sweep: m = %d exceeds the register-resident limit 2048", r->m);
  const size_t cd_row = cplx ? cplx_row_bytes(nu, wpc) : (size_t)L.mp * 2 * f;
  const size_t need = metropolis_scratch_bytes(r->n, r->m, cplx, move, nb);
  if (need && (!scratch || scratch_bytes < need))
    return fail(NK_ERR_SHAPE, "nk_metropolis_sweep: scratch of %zu B, need %zu B", scratch_bytes,
                need);
  // ring depth: as many slots as fit next to the pair partials, barriers and
  // the per-warp sigma copies (theta lives in tensor memory)
  const size_t slot = cd_row + (size_t)L.mp * f + kRowHdr;
  const size_t rest = (size_t)round_up(2 * A.G * wpc, 2) * 4 + 2 * kMaxRing * 8 + 16 +
                      (size_t)A.G * wpc * round_up(r->n, 16);
  const size_t cap = 227 * 1024;
  const int ring = rest + 2 * slot > cap ? 0 : (int)std::min<size_t>(kMaxRing, (cap - rest) / slot);
  if (ring < 2)
    return fail(NK_ERR_SHAPE,
                "nk_metropolis_sweep: group_size %d with padded m %d leaves room for fewer "
                "than two table slots in 227 KB of shared memory",
                A.G, L.mp);
  A.ring = ring;
  if ((int64_t)(n_discard + n_samples) * r->n > 0x7fffffff)
    return fail(NK_ERR_SHAPE, "nk_metropolis_sweep: too many proposals in one call");
  P->cplx = cplx;
  P->nu = nu;
  P->wpc = wpc;
  P->smem = (size_t)ring * slot + rest;
  P->ctr_dev = ch->counter_dev;
  P->advance = (uint64_t)(n_discard + n_samples) * r->n;
  TableJob& J = P->tj;
  J = TableJob{kTabNone, L.mp, nu, wpc, ws + L.tab, ws + L.wt, bi, bk, scratch, nullptr};
  J.a = r->a;
  const int rows = move == NK_MOVE_FLIP ? r->n : nb;
  // rows of real_row_stride / cplx_row_stride bytes in the scratch: table block,
  // increments, header
  A.cd = scratch;
  A.wd = nullptr;
  if (!cplx) {
    J.kind = move == NK_MOVE_FLIP ? kTabRealFlip : kTabRealPair;
    P->tab_elems = (int64_t)rows * L.mp;
  } else {
    J.kind = move == NK_MOVE_FLIP ? kTabCplxFlip : kTabCplxPair;
    P->tab_elems = (int64_t)rows * (nu / 2) * wpc * 32;
  }
  if (skip_tables) {  // tables of an earlier launch of the same call
    J.kind = kTabNone;
    P->tab_elems = 0;
  }
  return NK_OK;
}

nk_status launch_metropolis(const nk_rbm* r, nk_chains* ch, int move, const int32_t* bi,
                            const int32_t* bk, int nb, int n_discard, int n_samples,
                            int8_t* samples, uint64_t* n_acc, void* scratch, size_t scratch_bytes,
                            cudaStream_t st, bool dry, const MetroPt* pt) {
  MetroPlan P;
  if (nk_status e = plan_metropolis(r, ch, move, bi, bk, nb, n_discard, n_samples, samples,
                                    n_acc, scratch, scratch_bytes, pt, &P))
    return e;
  if (dry) return NK_OK;  // every check passed; nothing is enqueued
  if (P.tj.kind != kTabNone && P.tab_elems > 0) {
    TableBatch TB;
    TB.n = 1;
    TB.start[0] = 0;
    TB.start[1] = P.tab_elems;
    TB.j[0] = P.tj;
    const int64_t blocks =
        std::max<int64_t>(1, std::min<int64_t>((P.tab_elems + 255) / 256, 152 * 16));
    tables_batch_kernel<<<(unsigned)blocks, 256, 0, st>>>(TB);
    if (nk_status e = check_launch("nk_metropolis_sweep(tables)")) return e;
  }
  nk_status e;
  if (P.group_pp) {
    GroupSingleLaunch LG{P.A, P.threads, P.smem, st};
    e = launch_group(P.group_pp, LG);
  } else {
    SingleLaunch L1{P.A, P.smem, st};
    e = P.cplx ? launch_c<true>(P.nu, P.wpc, r->m, L1) : launch_c<false>(P.nu, P.wpc, r->m, L1);
  }
  if (e == NK_OK && ch->counter_dev) {
    advance_counter_kernel<<<1, 1, 0, st>>>(ch->counter_dev, P.advance);
    e = check_launch("nk_metropolis_sweep(counter)");
  }
  return e;
}

// Fused sweeps of many problems: one launch of the table builds for all of
// them, one launch of the sweep kernel per group of problems that share its
// template (at most kMetroBatch per launch), one launch advancing every device
// counter.  Each problem runs the arithmetic of its own launch (same arguments,
// tables and ring depth), so the results are those of separate calls.
nk_status launch_metropolis_fused(const nk_sweep_item* items, const int* idx, int n,
                                  cudaStream_t st) {
  std::vector<MetroPlan> plans((size_t)n);
  for (int u = 0; u < n; ++u) {
    const nk_sweep_item& it = items[idx[u]];
    if (nk_status e = plan_metropolis(it.rbm, it.chains, it.move, it.bond_i, it.bond_k,
                                      it.n_bonds, it.n_discard, it.n_samples_per_chain,
                                      it.samples_out, it.n_accept_out, it.scratch,
                                      it.scratch_bytes, nullptr, &plans[u]))
      return e;
  }
  // table builds
  for (int u0 = 0; u0 < n; u0 += kMetroBatch) {
    TableBatch TB;
    TB.n = 0;
    TB.start[0] = 0;
    for (int u = u0; u < std::min(n, u0 + kMetroBatch); ++u) {
      if (plans[u].tj.kind == kTabNone || plans[u].tab_elems == 0) continue;
      TB.j[TB.n] = plans[u].tj;
      TB.start[TB.n + 1] = TB.start[TB.n] + plans[u].tab_elems;
      ++TB.n;
    }
    if (TB.n > 0) {
      const int64_t blocks =
          std::max<int64_t>(1, std::min<int64_t>((TB.start[TB.n] + 255) / 256, 152 * 16));
      tables_batch_kernel<<<(unsigned)blocks, 256, 0, st>>>(TB);
      if (nk_status e = check_launch("nk_batch_sweep(tables)")) return e;
    }
  }
  // sweeps, grouped by kernel template
  std::vector<bool> done((size_t)n, false);
  for (int u = 0; u < n; ++u) {
    if (done[u]) continue;
    const MetroPlan& P0 = plans[u];
    MetroBatch B;
    B.n = 0;
    B.start[0] = 0;
    size_t smem = 0;
    for (int v = u; v < n && B.n < kMetroBatch; ++v) {
      const MetroPlan& P = plans[v];
      if (done[v] || P.cplx != P0.cplx || P.nu != P0.nu || P.wpc != P0.wpc ||
          P.A.G != P0.A.G || P.group_pp != P0.group_pp || P.threads != P0.threads)
        continue;
      B.a[B.n] = P.A;
      B.start[B.n + 1] = B.start[B.n] + (P.A.nc + P.A.G - 1) / P.A.G;
      ++B.n;
      smem = std::max(smem, P.smem);
      done[v] = true;
    }
    nk_status e;
    if (P0.group_pp) {
      GroupBatchLaunch LB{B, P0.threads, smem, st};
      e = launch_group(P0.group_pp, LB);
    } else {
      BatchLaunch LB{B, P0.A.G, smem, st};
      e = P0.cplx ? launch_c<true>(P0.nu, P0.wpc, P0.A.m, LB)
                  : launch_c<false>(P0.nu, P0.wpc, P0.A.m, LB);
    }
    if (e) return e;  // problems of this template beyond kMetroBatch start later batches
  }
  // device counters
  for (int u0 = 0; u0 < n; u0 += kMetroBatch) {
    CounterBatch CB;
    CB.n = 0;
    for (int u = u0; u < std::min(n, u0 + kMetroBatch); ++u)
      if (plans[u].ctr_dev) {
        CB.ctr[CB.n] = plans[u].ctr_dev;
        CB.delta[CB.n] = plans[u].advance;
        ++CB.n;
      }
    if (CB.n > 0) {
      advance_counters_kernel<<<1, 64, 0, st>>>(CB);
      if (nk_status e = check_launch("nk_batch_sweep(counters)")) return e;
    }
  }
  return NK_OK;
}

NK_STATUS_COLLECTOR(collect_status_metropolis)

}  // namespace nk
