// K3: local energies E_loc(sigma) = sum_sigma' <sigma|H|sigma'> psi(sigma')/psi(sigma)
// (Eq. 5, Sec. 2.2.5) for a Hamiltonian of 1-local and 2-local terms, and K4:
// the factored log-derivatives T = tanh(theta) (Sec. 2.2.5: O_b = tanh theta,
// O_W = tanh theta (x) sigma, O_a = sigma).
//
// Every move's psi ratio is exp(visible) * prod_j (cosh c_j - t_j sinh c_j)
// (c = 2 s_i W_i (+ 2 s_k W_k), t = tanh theta) from the cosh/sinh(2W) tables,
// with each running product kept as mantissa * 2^e; matrix elements, visible
// factors and the sums over moves are FP64.
#include "common.cuh"
#include "internal.h"
#include "opdev.h"
#include "ratio.cuh"
#include "tc.cuh"
#include "status.cuh"
#include "umma.cuh"

#include <string.h>

#include <type_traits>

namespace nk {

struct ElocArgs {
  int n, m, mp, n_moves;
  int64_t ns;
  const int8_t* sigma;
  const void* theta;   // [ns][m] F
  const char* op;      // compiled operator
  const double* a;     // master a
  const double2* fac;  // [nm_pad][4] mel x exp(visible) per move and spin pattern (built per call)
  const void* tab;     // [n][mp] T2
  double* eloc;        // c128 [ns]
  void* t_out;         // [ns][m] F or null
  int nseg;            // 1, or 2: each configuration tile is split over two CTAs
                       // taking half of the move tiles each, whose sums are added
                       // into eloc (zeroed first) atomically
  int seg_fast;        // 1: the grid is (nseg, tiles), so the two halves of a
                       // configuration tile run back to back and share its theta /
                       // T rows in L2; 0: (tiles, nseg)
};

__device__ __forceinline__ int idx_of(int8_t s) { return s > 0 ? 0 : 1; }

// Tiled form: a CTA owns 64 configurations and walks the move list in tiles of
// 64 moves; every thread advances a 4 x 4 block of running products
// prod_j (cosh c_j - s_i t_j sinh c_j / s_i) held in registers, so each staged
// value is reused by 16 threads and the kernel is bound by the FP32 pipe.  The
// (cosh c, sinh c / s_i) columns of all moves are built once per call in the
// caller's scratch as a [m][moves] table (a two-spin move has cosh c =
// A_i A_k +/- B_i B_k, sinh c / s_i = B_i A_k +/- A_i B_k from the site tables;
// the sign is fixed per move by the alignment split at compilation); 16 x 64
// tiles of it arrive by 2-D TMA into a double buffer, one chunk ahead, while
// the t = tanh(theta) tile of the next chunk is loaded into registers.
constexpr int kEBS = 64;   // configurations per CTA
constexpr int kEBM = 64;   // moves per tile
constexpr int kEBK = 16;   // hidden units per chunk
constexpr int kETS = kEBS + 1;  // padded row of the t tile (conflict-free transposed stores)

// (cosh c_j, sinh c_j / s_i) of move mv: the two-spin form from the site tables
template <bool CPLX>
__device__ __forceinline__ typename RatioTypes<CPLX>::T2 move_column(const OpMove& M,
                                                                     const void* tabv, int mp,
                                                                     int j) {
  using T2 = typename RatioTypes<CPLX>::T2;
  const T2* tab = reinterpret_cast<const T2*>(tabv);
  const T2 ai = tab[(int64_t)M.i * mp + j];
  if (!M.two) return ai;
  const T2 ak = tab[(int64_t)M.k * mp + j];
  const float al = (float)M.align;
  if constexpr (CPLX) {
    cf Ai{ai.x, ai.y}, Bi{ai.z, ai.w}, Ak{ak.x, ak.y}, Bk{ak.z, ak.w};
    cf c = Ai * Ak + al * (Bi * Bk);
    cf d = Bi * Ak + al * (Ai * Bk);
    return make_float4(c.x, c.y, d.x, d.y);
  } else {
    return make_float2(fmaf(al * ai.y, ak.y, ai.x * ak.x), fmaf(al * ai.x, ak.y, ai.y * ak.x));
  }
}

// Real RBMs: table[j][mv] = (cosh c_j, sinh c_j / s_i) of move mv.
// Complex RBMs: row j holds, per tile of 64 moves, 32 slots for move pairs
// (a, b = a + 16) with a = (s mod 16) + 32 (s div 16): first the C plane,
// slot s = (Re C_a, Re C_b, Im C_a, Im C_b), then the D plane (same for
// D = sinh c / s_i), so that one 16-byte load gives a thread the operands of
// two moves as packed FP32 pairs.
// Element x of the table (complex: of mp * ntile * 32 slot pairs; real: of mp * nm_pad)
template <bool CPLX>
__device__ __forceinline__ void move_table_elem(int64_t x, const OpMove* __restrict__ mvs,
                                                const void* __restrict__ tabv, int mp, int nm,
                                                int nm_pad, void* outv) {
  if constexpr (CPLX) {
    float4* out = reinterpret_cast<float4*>(outv);
    const int ntile = nm_pad / kEBM;
    const int slot = (int)(x & 31);
    const int64_t jt = x >> 5;
    const int j = (int)(jt / ntile), mt = (int)(jt % ntile);
    const int a = mt * kEBM + (slot & 15) + 32 * (slot >> 4), b = a + 16;
    const float4 za = make_float4(0.f, 0.f, 0.f, 0.f);
    const float4 va = a < nm ? move_column<true>(mvs[a], tabv, mp, j) : za;
    const float4 vb = b < nm ? move_column<true>(mvs[b], tabv, mp, j) : za;
    float4* row = out + ((int64_t)j * ntile + mt) * 64;
    row[slot] = make_float4(va.x, vb.x, va.y, vb.y);
    row[32 + slot] = make_float4(va.z, vb.z, va.w, vb.w);
  } else {
    float2* out = reinterpret_cast<float2*>(outv);
    const int j = (int)(x / nm_pad), mv = (int)(x % nm_pad);
    out[x] = mv < nm ? move_column<false>(mvs[mv], tabv, mp, j) : make_float2(0.f, 0.f);
  }
}

__host__ __device__ inline int64_t move_table_elems(int cplx, int mp, int nm_pad) {
  return cplx ? (int64_t)mp * (nm_pad / kEBM) * 32 : (int64_t)mp * nm_pad;
}

// Byte offset of the factor table in the scratch: after the move table of
// mp x nm_pad entries (T2: 16 bytes complex, 8 real).
__host__ __device__ inline int64_t move_factor_offset(int cplx, int mp, int nm_pad) {
  return ((int64_t)mp * nm_pad * (cplx ? 16 : 8) + 255) / 256 * 256;
}

// Element y = 4 mv + x of the factor table: mel(x) exp(-2 s_i a_i (- 2 s_k a_k)) of
// move mv for the spin pattern x = 2 idx(s_i) + idx(s_k) (zero for a padding move
// or a zero matrix element), in FP64: the per-move constant of every ratio.
template <bool CPLX>
__device__ __forceinline__ void move_factor_elem(int64_t y, const OpMove* __restrict__ mvs,
                                                 const double* __restrict__ a, int nm,
                                                 double2* out) {
  const int mv = (int)(y >> 2), x = (int)(y & 3);
  double cr = 0.0, ci = 0.0;
  if (mv < nm) {
    const double mr = mvs[mv].mel[x][0], mi = mvs[mv].mel[x][1];
    if (mr != 0.0 || mi != 0.0) {
      const double si = (x >> 1) ? -1.0 : 1.0, sk = (x & 1) ? -1.0 : 1.0;
      const int i = mvs[mv].i, k = mvs[mv].k;
      double vr, vi;
      if (CPLX) {
        vr = -2.0 * si * a[2 * i];
        vi = -2.0 * si * a[2 * i + 1];
        if (mvs[mv].two) {
          vr += -2.0 * sk * a[2 * k];
          vi += -2.0 * sk * a[2 * k + 1];
        }
      } else {
        vr = -2.0 * si * a[i];
        vi = 0.0;
        if (mvs[mv].two) vr += -2.0 * sk * a[k];
      }
      const double ev = exp(vr), fr = ev * cos(vi), fi = ev * sin(vi);
      cr = mr * fr - mi * fi;
      ci = mr * fi + mi * fr;
    }
  }
  out[y] = make_double2(cr, ci);
}

// Element x of a call's tables: the move table, then the factor table.
template <bool CPLX>
__device__ __forceinline__ void move_job_elem(int64_t x, const OpMove* __restrict__ mvs,
                                              const void* __restrict__ tabv,
                                              const double* __restrict__ a, int mp, int nm,
                                              int nm_pad, void* outv) {
  const int64_t te = move_table_elems(CPLX, mp, nm_pad);
  if (x < te) {
    move_table_elem<CPLX>(x, mvs, tabv, mp, nm, nm_pad, outv);
  } else {
    double2* fac = reinterpret_cast<double2*>(reinterpret_cast<char*>(outv) +
                                              move_factor_offset(CPLX, mp, nm_pad));
    move_factor_elem<CPLX>(x - te, mvs, a, nm, fac);
  }
}

__host__ __device__ inline int64_t move_job_elems(int cplx, int mp, int nm_pad) {
  return move_table_elems(cplx, mp, nm_pad) + (int64_t)nm_pad * 4;
}

template <bool CPLX>
__global__ void move_tables_kernel(const char* __restrict__ op, const void* __restrict__ tabv,
                                   const double* __restrict__ a, int mp, int nm, int nm_pad,
                                   void* outv) {
  const OpDevHeader* H = reinterpret_cast<const OpDevHeader*>(op);
  const OpMove* mvs = reinterpret_cast<const OpMove*>(op + H->off_moves);
  const int64_t total = move_job_elems(CPLX, mp, nm_pad);
  for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < total;
       x += (int64_t)gridDim.x * blockDim.x)
    move_job_elem<CPLX>(x, mvs, tabv, a, mp, nm, nm_pad, outv);
}

// The move tables of many problems in one launch (job k owns elements
// [start[k], start[k + 1]) of the concatenated range; real and complex jobs mix).
constexpr int kMoveJobs = 64;
struct MoveTableJob {
  int cplx, mp, nm, nm_pad;
  const char* op;
  const void* tab;
  const double* a;
  void* out;
};
struct MoveTableBatch {
  int n;
  int64_t start[kMoveJobs + 1];
  MoveTableJob j[kMoveJobs];
};

__global__ void move_tables_batch_kernel(const __grid_constant__ MoveTableBatch B) {
  const int64_t total = B.start[B.n];
  for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < total;
       x += (int64_t)gridDim.x * blockDim.x) {
    int lo = 0, hi = B.n - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (B.start[mid] <= x) lo = mid; else hi = mid - 1;
    }
    const MoveTableJob& J = B.j[lo];
    const OpDevHeader* H = reinterpret_cast<const OpDevHeader*>(J.op);
    const OpMove* mvs = reinterpret_cast<const OpMove*>(J.op + H->off_moves);
    if (J.cplx)
      move_job_elem<true>(x - B.start[lo], mvs, J.tab, J.a, J.mp, J.nm, J.nm_pad, J.out);
    else
      move_job_elem<false>(x - B.start[lo], mvs, J.tab, J.a, J.mp, J.nm, J.nm_pad, J.out);
  }
}

// Packed FP32 pair arithmetic (two independent lanes per instruction).
__device__ __forceinline__ float2 f2fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 f2mul(float2 a, float2 b) { return __fmul2_rn(a, b); }

// Two running products (the lanes of a packed pair, complex: Re in x, Im in y)
// renormalised with one shared power of two, the exponent of the largest of
// their four parts: each is kept as mantissa * 2^e with the pair's e.  The
// smaller product keeps its full FP32 precision unless it is below 2^-126 of
// the larger, where its local-energy term is negligible against the larger one.
__device__ __forceinline__ void renorm_pair(float2& x, float2& y, int& e) {
  const float mx = fmaxf(fmaxf(fabsf(x.x), fabsf(x.y)), fmaxf(fabsf(y.x), fabsf(y.y)));
  int ex = ((__float_as_int(mx) >> 23) & 0xff) - 127;
  if (mx == 0.f) ex = 0;
  const float sc = __int_as_float((127 - ex) << 23);
  x = f2mul(x, make_float2(sc, sc));
  y = f2mul(y, make_float2(sc, sc));
  e += ex;
}

template <bool CPLX>
__device__ __forceinline__ void local_energy_body(const CUtensorMap* mtab, const ElocArgs& A,
                                                  const int tile_idx, const int seg) {
  using F = typename RatioTypes<CPLX>::F;
  using T2 = typename RatioTypes<CPLX>::T2;
  extern __shared__ __align__(128) unsigned char smraw[];
  // t tile entry: real t, or (Re t, Re t, Im t, Im t) as two packed pairs
  using TS = typename std::conditional<CPLX, float4, float>::type;
  T2* mvt = reinterpret_cast<T2*>(smraw);                                    // [2][BK][BM]
  TS* tS = reinterpret_cast<TS*>(smraw + 2 * kEBK * kEBM * sizeof(T2));      // [2][BK][BS+1]
  int* mvi = reinterpret_cast<int*>(reinterpret_cast<char*>(tS) +
                                    round_up(2 * kEBK * kETS * sizeof(TS), 16));
  int* mvk = mvi + kEBM;
  int* mvtwo = mvk + kEBM;
  double2* cvs = reinterpret_cast<double2*>(mvtwo + kEBM);                   // [BM][4]
  double2* eacc = cvs + 4 * kEBM;  // [4][256] per-thread partial E_loc (kept out of registers)
  uint64_t* mbar = reinterpret_cast<uint64_t*>(eacc + 4 * 256);              // [2]

  const int tid = threadIdx.x, ts = tid >> 4, tm = tid & 15;
  const int64_t s0 = (int64_t)tile_idx * kEBS;
  const int n = A.n, m = A.m, mp = A.mp;
  const OpDevHeader* H = reinterpret_cast<const OpDevHeader*>(A.op);
  const OpDSite* ds = reinterpret_cast<const OpDSite*>(A.op + H->off_dsite);
  const OpDBond* db = reinterpret_cast<const OpDBond*>(A.op + H->off_dbond);
  const OpMove* mvs = reinterpret_cast<const OpMove*>(A.op + H->off_moves);
  const F* th = reinterpret_cast<const F*>(A.theta);
  F* tout = reinterpret_cast<F*>(A.t_out);
  const int nm = A.n_moves;
  const bool quad = (H->flags & kOpQuadMoves) != 0;  // site-quad move layout
  const int ntile = (nm + kEBM - 1) / kEBM, nchunk = mp / kEBK;
  const int tile_begin = ntile * seg / A.nseg, tile_end = ntile * (seg + 1) / A.nseg;
  const int it_begin = tile_begin * nchunk, it_end = tile_end * nchunk;
  const uint32_t tile_bytes = kEBK * kEBM * sizeof(T2);

  if (tid == 0) {
    mbar_init(&mbar[0], 1);
    mbar_init(&mbar[1], 1);
    mbar_fence_init();
  }

  // diagonal part: the 16 threads of a configuration split the terms
  double er[4], ei[4];
#pragma unroll
  for (int p = 0; p < 4; ++p) {
    er[p] = ei[p] = 0.0;
    const int64_t s = s0 + ts * 4 + p;
    if (s < A.ns && seg == 0) {  // the diagonal belongs to the first segment
      const int8_t* sg = A.sigma + s * n;
      for (int u = tm; u < H->n_dsite; u += 16) {
        int x = idx_of(sg[ds[u].i]);
        er[p] += ds[u].d[x][0];
        ei[p] += ds[u].d[x][1];
      }
      for (int u = tm; u < H->n_dbond; u += 16) {
        int x = 2 * idx_of(sg[db[u].i]) + idx_of(sg[db[u].k]);
        er[p] += db[u].d[x][0];
        ei[p] += db[u].d[x][1];
      }
    }
    eacc[p * 256 + tid] = make_double2(er[p], ei[p]);
  }

  // Hidden-unit chunk of iteration it: each move tile walks the chunks in the
  // direction opposite to the previous one, so its first chunks are the ones the
  // CTA read last (still in L2) -- fewer DRAM re-reads of the t rows.
  auto chunk_of = [&](int it) {
    const int r = it % nchunk;
    return ((it / nchunk - tile_begin) & 1) ? nchunk - 1 - r : r;
  };
  // t tile of a chunk: thread covers (ss, kk) = (e >> 4, e & 15), e = tid + 256 u
  F tv[4];
  auto load_t = [&](int it) {
    const int kc = chunk_of(it), mt = it / nchunk;
    const bool reuse = tout && mt > tile_begin;  // t was written by this CTA at its first tile
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int e = tid + u * 256, ss = e >> 4, kk = e & 15;
      const int64_t s = s0 + ss;
      const int j = kc * kEBK + kk;
      if constexpr (CPLX) tv[u] = make_float2(0.f, 0.f); else tv[u] = 0.f;
      if (s < A.ns && j < m) tv[u] = reuse ? tout[s * m + j] : th[s * m + j];
    }
  };
  auto store_t = [&](int it, int buf) {
    const int kc = chunk_of(it), mt = it / nchunk;
    const bool reuse = tout && mt > tile_begin;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int e = tid + u * 256, ss = e >> 4, kk = e & 15;
      const int64_t s = s0 + ss;
      const int j = kc * kEBK + kk;
      F v = tv[u];
      if (!reuse && s < A.ns && j < m) {
        if constexpr (CPLX) {
          cf c = tanh_c(cf{v.x, v.y});
          v = make_float2(c.x, c.y);
        } else {
          v = tanh_f(v);
        }
        if (tout) tout[s * m + j] = v;
      }
      if constexpr (CPLX)
        tS[(buf * kEBK + kk) * kETS + ss] = make_float4(v.x, v.x, v.y, v.y);
      else
        tS[(buf * kEBK + kk) * kETS + ss] = v;
    }
  };

  __syncthreads();
  if (it_end > it_begin) {
    if (tid == 0) {
      mbar_arrive_expect_tx(&mbar[0], tile_bytes);
      tma_load_2d(mvt, mtab, tile_begin * kEBM * (CPLX ? 4 : 2), 0, &mbar[0]);
    }
    load_t(it_begin);
    store_t(it_begin, 0);
  }

  // running products: real, P[p][q]; complex, packed over the move pairs
  // (q = 2 qp, 2 qp + 1): Px/Py[p][qp] = (Re, Im) parts, shared exponent Pe[p][qp]
  ScaledReal P[4][4];
  float2 Px[4][2], Py[4][2];
  int Pe[4][4];         // real: unused; complex: Pe[p][qp] is the exponent of move pair qp
  float sgn[4][4];      // real: sigma_i of the configuration for each move
  float2 ns2[4][2];     // complex: -sigma_i packed over the move pairs
  bool bad = false;     // a bounded wait for a move-table chunk gave up
  __shared__ volatile int s_bad;
  if (tid == 0) s_bad = 0;
  __syncthreads();
  int it_stop = it_end; // first chunk not processed
  for (int it = it_begin; it < it_end; ++it) {
    const int b = (it - it_begin) & 1, kc = it % nchunk, mt = it / nchunk, mt0 = mt * kEBM;
    __syncthreads();  // chunk it-1 fully consumed; t tile of chunk it stored
    if (s_bad) {      // a wait timed out: all threads stop together
      it_stop = it;
      break;
    }
    if (kc == 0) {
      // new tile of moves: metadata and mel * exp(visible) per sign pattern
      if (tid < kEBM) {
        const int mv = mt0 + tid;
        mvi[tid] = mv < nm ? mvs[mv].i : 0;
        mvk[tid] = mv < nm ? mvs[mv].k : 0;
        mvtwo[tid] = mv < nm ? mvs[mv].two : -1;  // -1: padding move
      }
      // the tile's mel x exp(visible) factors, built once per call by the
      // move-table launch (tile mt0 .. mt0 + 63 lies inside the padded table)
      cvs[tid] = A.fac[(int64_t)mt0 * 4 + tid];
      __syncthreads();
#pragma unroll
      for (int p = 0; p < 4; ++p) {
        const int64_t s = s0 + ts * 4 + p;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const float sv = (s < A.ns) ? (float)A.sigma[s * n + mvi[tm + 16 * q]] : 1.f;
          if constexpr (CPLX) {
            Pe[p][q] = 0;
            if (q & 1) ns2[p][q >> 1].y = -sv; else ns2[p][q >> 1].x = -sv;
          } else {
            sgn[p][q] = sv;
            P[p][q].init();
          }
        }
        if constexpr (CPLX) {
#pragma unroll
          for (int qp = 0; qp < 2; ++qp) {
            Px[p][qp] = make_float2(1.f, 1.f);
            Py[p][qp] = make_float2(0.f, 0.f);
          }
        }
      }
    }
    if (tid == 0 && it + 1 < it_end) {
      const int it1 = it + 1;
      mbar_arrive_expect_tx(&mbar[b ^ 1], tile_bytes);
      tma_load_2d(mvt + (size_t)(b ^ 1) * kEBK * kEBM, mtab,
                      (it1 / nchunk) * kEBM * (CPLX ? 4 : 2), chunk_of(it1) * kEBK, &mbar[b ^ 1]);
    }
    if (it + 1 < it_end) load_t(it + 1);
    if (!mbar_wait_bounded(&mbar[b], (uint32_t)(((it - it_begin) >> 1) & 1))) {
      bad = true;
      s_bad = 1;
    }
    const T2* mv_b = mvt + (size_t)b * kEBK * kEBM;
    const TS* t_b = tS + (size_t)b * kEBK * kETS;
    // QUAD (site-quad move layout): the thread's four moves share s_i, so -s t
    // is formed once per configuration and hidden unit instead of per move
    auto chunk = [&](auto quad_tag) {
      constexpr bool QUAD = decltype(quad_tag)::value;
      if constexpr (CPLX) {
        // r = C - s t D for two moves at once: with ns = -s,
        // Re r = Re C + ns (Re t Re D - Im t Im D), Im r = Im C + ns (Re t Im D + Im t Re D),
        // then P *= r.
        const float4* mvc = reinterpret_cast<const float4*>(mv_b);
#pragma unroll
        for (int kk = 0; kk < kEBK; ++kk) {
          float4 t4[4], c4[2], d4[2];
#pragma unroll
          for (int p = 0; p < 4; ++p) t4[p] = t_b[kk * kETS + ts * 4 + p];
#pragma unroll
          for (int qp = 0; qp < 2; ++qp) {
            c4[qp] = mvc[kk * kEBM + tm + 16 * qp];
            d4[qp] = mvc[kk * kEBM + 32 + tm + 16 * qp];
          }
#pragma unroll
          for (int p = 0; p < 4; ++p) {
            const float2 tx = make_float2(t4[p].x, t4[p].y), ty = make_float2(t4[p].z, t4[p].w);
            const float2 nty = make_float2(-t4[p].z, -t4[p].w);
            // QUAD: (nux, nuy) = -s t, shared by both move pairs
            const float2 nux = QUAD ? f2mul(ns2[p][0], tx) : tx;
            const float2 nuy = QUAD ? f2mul(ns2[p][0], ty) : ty;
#pragma unroll
            for (int qp = 0; qp < 2; ++qp) {
              const float2 cx = make_float2(c4[qp].x, c4[qp].y), cy = make_float2(c4[qp].z, c4[qp].w);
              const float2 dx = make_float2(d4[qp].x, d4[qp].y), dy = make_float2(d4[qp].z, d4[qp].w);
              float2 rx, ry;
              if constexpr (QUAD) {
                rx = f2fma(nux, dx, f2fma(make_float2(-nuy.x, -nuy.y), dy, cx));
                ry = f2fma(nux, dy, f2fma(nuy, dx, cy));
              } else {
                const float2 tdx = f2fma(tx, dx, f2mul(nty, dy));
                const float2 tdy = f2fma(tx, dy, f2mul(ty, dx));
                rx = f2fma(ns2[p][qp], tdx, cx);
                ry = f2fma(ns2[p][qp], tdy, cy);
              }
              const float2 px = Px[p][qp], py = Py[p][qp];
              Px[p][qp] = f2fma(make_float2(-py.x, -py.y), ry, f2mul(px, rx));
              Py[p][qp] = f2fma(py, rx, f2mul(px, ry));
            }
          }
          if (kk == kEBK - 1) {  // once per chunk of 16 hidden units
#pragma unroll
            for (int p = 0; p < 4; ++p)
#pragma unroll
              for (int qp = 0; qp < 2; ++qp) renorm_pair(Px[p][qp], Py[p][qp], Pe[p][qp]);
          }
        }
      } else {
#pragma unroll
        for (int kk = 0; kk < kEBK; ++kk) {
          F t[4];
          T2 v[4];
#pragma unroll
          for (int p = 0; p < 4; ++p) t[p] = t_b[kk * kETS + ts * 4 + p];
#pragma unroll
          for (int q = 0; q < 4; ++q) v[q] = mv_b[kk * kEBM + tm + 16 * q];
#pragma unroll
          for (int p = 0; p < 4; ++p) {
            const float nst = -sgn[p][0] * t[p];  // QUAD: -s t of all four moves
#pragma unroll
            for (int q = 0; q < 4; ++q)
              P[p][q].v *= fmaf(QUAD ? nst : -sgn[p][q] * t[p], v[q].y, v[q].x);
          }
          if ((kk & 7) == 7) {
#pragma unroll
            for (int p = 0; p < 4; ++p)
#pragma unroll
              for (int q = 0; q < 4; ++q) P[p][q].renorm();
          }
        }
      }
    };
    if (quad) chunk(std::true_type{});
    else chunk(std::false_type{});
    if (it + 1 < it_end) store_t(it + 1, b ^ 1);
    if (kc == nchunk - 1) {
      // fold the tile's ratios into the local energies (FP64)
#pragma unroll
      for (int p = 0; p < 4; ++p) {
        const int64_t s = s0 + ts * 4 + p;
        if (s >= A.ns) continue;
        double2 acc = eacc[p * 256 + tid];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int mm = tm + 16 * q;
          if (mvtwo[mm] < 0) continue;
          const int x = 2 * idx_of(A.sigma[s * n + mvi[mm]]) + idx_of(A.sigma[s * n + mvk[mm]]);
          const double2 cv = cvs[mm * 4 + x];
          if (cv.x == 0.0 && cv.y == 0.0) continue;
          double pr, pi;
          if constexpr (CPLX) {
            const float2 px = Px[p][q >> 1], py = Py[p][q >> 1];
            pr = ldexp((double)((q & 1) ? px.y : px.x), Pe[p][q >> 1]);
            pi = ldexp((double)((q & 1) ? py.y : py.x), Pe[p][q >> 1]);
          } else {
            pr = ldexp((double)P[p][q].v, P[p][q].e);
            pi = 0.0;
          }
          acc.x += cv.x * pr - cv.y * pi;
          acc.y += cv.x * pi + cv.y * pr;
        }
        eacc[p * 256 + tid] = acc;
      }
    }
  }
  __syncthreads();
  bad = s_bad != 0;
  if (bad) {
    if (tid == 0) {
      // let the chunk copies still in flight (the one waited for and the next)
      // land before the CTA exits
      for (int c = it_stop - 1; c <= it_stop && c < it_end; ++c)
        if (c >= it_begin)
          mbar_wait_bounded(&mbar[(c - it_begin) & 1], (uint32_t)(((c - it_begin) >> 1) & 1),
                            1u << 20);
      dev_status_set(1u << NK_ERR_TIMEOUT);
    }
  }
  // the 16 threads of a configuration are lanes tid ^ 1, 2, 4, 8 of one warp
#pragma unroll
  for (int p = 0; p < 4; ++p) {
    er[p] = bad ? __longlong_as_double(0x7ff8000000000000ll) : eacc[p * 256 + tid].x;
    ei[p] = bad ? __longlong_as_double(0x7ff8000000000000ll) : eacc[p * 256 + tid].y;
#pragma unroll
    for (int off = 8; off >= 1; off >>= 1) {
      er[p] += __shfl_xor_sync(0xffffffffu, er[p], off);
      ei[p] += __shfl_xor_sync(0xffffffffu, ei[p], off);
    }
    const int64_t s = s0 + ts * 4 + p;
    if (tm == 0 && s < A.ns) {
      if (A.nseg == 1) {
        A.eloc[2 * s] = er[p];
        A.eloc[2 * s + 1] = ei[p];
      } else {
        // two addends onto an exact zero: 0 + x + y = 0 + y + x in IEEE
        // arithmetic, so the result does not depend on the order
        atomicAdd(&A.eloc[2 * s], er[p]);
        atomicAdd(&A.eloc[2 * s + 1], ei[p]);
      }
    }
  }
  // with no moves at all, t = tanh(theta) is still written
  if (nm == 0 && tout && seg == 0) {
    for (int e = tid; e < kEBS * m; e += blockDim.x) {
      const int64_t s = s0 + e / m;
      const int j = e % m;
      if (s >= A.ns) continue;
      if constexpr (CPLX) {
        F x = th[s * m + j];
        cf c = tanh_c(cf{x.x, x.y});
        tout[s * m + j] = make_float2(c.x, c.y);
      } else {
        tout[s * m + j] = tanh_f(th[s * m + j]);
      }
    }
  }
}

template <bool CPLX>
__global__ void __launch_bounds__(256, 2) local_energy_tiled(const __grid_constant__ CUtensorMap mtab,
                                                          ElocArgs A) {
  local_energy_body<CPLX>(&mtab, A, A.seg_fast ? blockIdx.y : blockIdx.x,
                          A.seg_fast ? blockIdx.x : blockIdx.y);
}

// Up to kElocBatch problems of one field in one launch: CTA b runs CTA
// b - start[k] of problem k, numbered as its own launch with the segment as
// the fast index (the two halves of a configuration tile back to back).
constexpr int kElocBatch = 64;
struct ElocBatch {
  int n;
  int start[kElocBatch + 1];
  ElocArgs a[kElocBatch];
  CUtensorMap map[kElocBatch];
};

template <bool CPLX>
__global__ void __launch_bounds__(256, 2) local_energy_batch(const __grid_constant__ ElocBatch B) {
  int k = 0;
  while (k + 1 < B.n && (int)blockIdx.x >= B.start[k + 1]) ++k;
  const int b = (int)blockIdx.x - B.start[k];
  const ElocArgs& A = B.a[k];
  local_energy_body<CPLX>(&B.map[k], A, b / A.nseg, b % A.nseg);
}

size_t local_energy_scratch_bytes(int m, int cplx, int n_moves) {
  const int64_t nm_pad = round_up(std::max(n_moves, 1), kEBM);
  // the move table, then the factor table (one double2 per move and spin pattern)
  return (size_t)(move_factor_offset(cplx, padded_m(m), (int)nm_pad) + nm_pad * 4 * 16);
}

// Everything one local-energy call needs, before anything is enqueued.
struct ElocPlan {
  ElocArgs A;
  CUtensorMap map;
  bool cplx;
  size_t smem;
  int64_t blocks;  // configuration tiles
  MoveTableJob job;
  int64_t tab_elems;
};

static nk_status plan_local_energy(const nk_rbm* r, const void* op_dev, int n_moves,
                                   const int8_t* sigma, const void* theta, int64_t ns,
                                   double* eloc, void* t_out, void* scratch, size_t scratch_bytes,
                                   ElocPlan* P) {
  WsLayout L(r->n, r->m, r->is_complex);
  const bool cplx = r->is_complex != 0;
  const size_t need = local_energy_scratch_bytes(r->m, cplx, n_moves);
  if (n_moves > 0 && (!scratch || scratch_bytes < need))
    return fail(NK_ERR_SHAPE, "nk_local_energy: scratch of %zu B, need %zu B", scratch_bytes, need);
  ElocArgs& A = P->A;
  A.n = r->n;
  A.m = r->m;
  A.mp = L.mp;
  A.ns = ns;
  A.n_moves = n_moves;
  A.sigma = sigma;
  A.theta = theta;
  A.op = (const char*)op_dev;
  A.a = r->a;
  A.tab = (const char*)r->ws + L.tab;
  A.eloc = eloc;
  A.t_out = t_out;
  P->cplx = cplx;
  const int nm_pad = (int)round_up(std::max(n_moves, 1), kEBM);
  memset(&P->map, 0, sizeof(P->map));
  P->job = MoveTableJob{cplx ? 1 : 0, L.mp, n_moves, nm_pad, A.op, A.tab, r->a, scratch};
  P->tab_elems = n_moves > 0 ? move_job_elems(cplx, L.mp, nm_pad) : 0;
  A.fac = n_moves > 0 ? reinterpret_cast<const double2*>(
                            (const char*)scratch + move_factor_offset(cplx, L.mp, nm_pad))
                      : nullptr;
  if (n_moves > 0) {
    const int fl = cplx ? 4 : 2;  // floats per table entry
    if (!make_map_f32(&P->map, scratch, L.mp, (int64_t)nm_pad * fl, (int64_t)nm_pad * fl * 4,
                      kEBM * fl, kEBK))
      return NK_ERR_CUDA;
  }
  const size_t t2 = cplx ? 16 : 8, f = cplx ? 16 : 4;  // table entry, t tile entry
  P->smem = 2 * kEBK * kEBM * t2 + round_up(2 * kEBK * kETS * f, 16) + 3 * kEBM * 4 +
            kEBM * 4 * 16 + 4 * 256 * 16 + 16;
  P->blocks = (ns + kEBS - 1) / kEBS;
  // two CTAs per SM: when the last wave of CTAs would be far from full, split
  // the move tiles into two halves (twice the CTAs) to even out the waves
  const int ntile = (n_moves + kEBM - 1) / kEBM;
  auto wave_eff = [&](int64_t b) {
    const int64_t slots = 2 * 152;
    return (double)b / (double)(((b + slots - 1) / slots) * slots);
  };
  A.nseg = (ntile >= 2 && wave_eff(2 * P->blocks) > wave_eff(P->blocks)) ? 2 : 1;
  if (r->eloc_segs > 0) A.nseg = (r->eloc_segs >= 2 && ntile >= 2) ? 2 : 1;  // tuned or set
  A.seg_fast = A.nseg == 2 && P->blocks <= 65535 ? 1 : 0;
  return NK_OK;
}

nk_status launch_local_energy(const nk_rbm* r, const void* op_dev, int n_moves,
                              const int8_t* sigma, const void* theta, int64_t ns, double* eloc,
                              void* t_out, void* scratch, size_t scratch_bytes, cudaStream_t st) {
  ElocPlan P;
  if (nk_status e = plan_local_energy(r, op_dev, n_moves, sigma, theta, ns, eloc, t_out, scratch,
                                      scratch_bytes, &P))
    return e;
  const ElocArgs& A = P.A;
  if (P.tab_elems > 0) {
    const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>((P.tab_elems + 255) / 256, 152 * 8));
    if (P.cplx)
      move_tables_kernel<true><<<(unsigned)blocks, 256, 0, st>>>(A.op, A.tab, A.a, A.mp, n_moves,
                                                                 P.job.nm_pad, scratch);
    else
      move_tables_kernel<false><<<(unsigned)blocks, 256, 0, st>>>(A.op, A.tab, A.a, A.mp,
                                                                  n_moves, P.job.nm_pad, scratch);
    if (nk_status e = check_launch("nk_local_energy(move tables)")) return e;
  }
  if (A.nseg == 2 &&
      cudaMemsetAsync(eloc, 0, (size_t)ns * 2 * sizeof(double), st) != cudaSuccess)
    return fail(NK_ERR_CUDA, "nk_local_energy: cudaMemsetAsync failed");
  const dim3 grid = A.seg_fast ? dim3((unsigned)A.nseg, (unsigned)P.blocks)
                               : dim3((unsigned)P.blocks, (unsigned)A.nseg);
  if (P.cplx) {
    if (cudaFuncSetAttribute(local_energy_tiled<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)P.smem) != cudaSuccess)
      return fail(NK_ERR_CUDA, "nk_local_energy: shared memory attribute");
    local_energy_tiled<true><<<grid, 256, P.smem, st>>>(P.map, A);
  } else {
    if (cudaFuncSetAttribute(local_energy_tiled<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)P.smem) != cudaSuccess)
      return fail(NK_ERR_CUDA, "nk_local_energy: shared memory attribute");
    local_energy_tiled<false><<<grid, 256, P.smem, st>>>(P.map, A);
  }
  return check_launch("nk_local_energy");
}

// Fused local energies of many problems: one move-table launch for all of them,
// one launch of the energy kernel per field (at most kElocBatch problems each).
// Every problem runs its own launch's arithmetic and move-tile split, so the
// results are those of separate calls.
nk_status launch_local_energy_fused(const nk_eloc_item* items, const int* idx, int n,
                                    cudaStream_t st) {
  std::vector<ElocPlan> plans((size_t)n);
  for (int u = 0; u < n; ++u) {
    const nk_eloc_item& it = items[idx[u]];
    if (nk_status e = plan_local_energy(it.rbm, it.op_dev, it.n_moves, it.sigma, it.theta, it.ns,
                                        it.eloc_out, it.t_out, it.scratch, it.scratch_bytes,
                                        &plans[u]))
      return e;
  }
  for (int u0 = 0; u0 < n; u0 += kMoveJobs) {
    MoveTableBatch TB;
    TB.n = 0;
    TB.start[0] = 0;
    for (int u = u0; u < std::min(n, u0 + kMoveJobs); ++u) {
      if (plans[u].tab_elems == 0) continue;
      TB.j[TB.n] = plans[u].job;
      TB.start[TB.n + 1] = TB.start[TB.n] + plans[u].tab_elems;
      ++TB.n;
    }
    if (TB.n > 0) {
      const int64_t blocks =
          std::max<int64_t>(1, std::min<int64_t>((TB.start[TB.n] + 255) / 256, 152 * 8));
      move_tables_batch_kernel<<<(unsigned)blocks, 256, 0, st>>>(TB);
      if (nk_status e = check_launch("nk_batch_local_energy(move tables)")) return e;
    }
  }
  for (int u = 0; u < n; ++u)
    if (plans[u].A.nseg == 2 &&
        cudaMemsetAsync(plans[u].A.eloc, 0, (size_t)plans[u].A.ns * 2 * sizeof(double), st) !=
            cudaSuccess)
      return fail(NK_ERR_CUDA, "nk_batch_local_energy: cudaMemsetAsync failed");
  for (int field = 0; field < 2; ++field) {
    const bool cplx = field == 1;
    for (int u0 = 0; u0 < n;) {
      ElocBatch* B = new ElocBatch;  // about 11 KB: kept off the stack
      B->n = 0;
      B->start[0] = 0;
      size_t smem = 0;
      int u = u0;
      for (; u < n && B->n < kElocBatch; ++u) {
        const ElocPlan& P = plans[u];
        if (P.cplx != cplx || P.blocks == 0) continue;
        B->a[B->n] = P.A;
        B->map[B->n] = P.map;
        B->start[B->n + 1] = B->start[B->n] + (int)(P.blocks * P.A.nseg);
        ++B->n;
        smem = std::max(smem, P.smem);
      }
      u0 = u;
      nk_status e = NK_OK;
      if (B->n > 0) {
        auto kern = cplx ? local_energy_batch<true> : local_energy_batch<false>;
        if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess)
          e = fail(NK_ERR_CUDA, "nk_batch_local_energy: shared memory attribute");
        else {
          kern<<<(unsigned)B->start[B->n], 256, smem, st>>>(*B);
          e = check_launch("nk_batch_local_energy");
        }
      }
      delete B;
      if (e) return e;
    }
  }
  return NK_OK;
}

// ------------------------------------------------------------------ K4 logderiv

template <bool CPLX>
__global__ void logderiv_kernel(int n, int m, int64_t ns, const int8_t* __restrict__ sigma,
                                const void* __restrict__ theta, int layout, void* out) {
  using F = typename RatioTypes<CPLX>::F;
  const F* th = reinterpret_cast<const F*>(theta);
  F* o = reinterpret_cast<F*>(out);
  const int64_t P = (int64_t)n + m + (int64_t)n * m;
  const int64_t total = layout == NK_LAYOUT_DENSE ? ns * P : ns * m;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    F v;
    if (layout != NK_LAYOUT_DENSE) {
      F x = th[e];
      if constexpr (CPLX) {
        cf tt = tanh_c(cf{x.x, x.y});
        v = make_float2(tt.x, tt.y);
      } else {
        v = tanh_f(x);
      }
    } else {
      int64_t s = e / P, k = e % P;
      if (k < n) {
        float sv = (float)sigma[s * n + k];
        if constexpr (CPLX) v = make_float2(sv, 0.f); else v = sv;
      } else {
        int64_t kk = k - n;
        int j = (int)(kk < m ? kk : (kk - m) / n);
        float mult = kk < m ? 1.f : (float)sigma[s * n + (kk - m) % n];
        F x = th[s * m + j];
        if constexpr (CPLX) {
          cf tt = tanh_c(cf{x.x, x.y});
          v = make_float2(mult * tt.x, mult * tt.y);
        } else {
          v = mult * tanh_f(x);
        }
      }
    }
    o[e] = v;
  }
}

nk_status launch_logderiv(const nk_rbm* r, const int8_t* sigma, const void* theta, int64_t ns,
                          int layout, void* o_out, cudaStream_t st) {
  int64_t P = (int64_t)r->n + r->m + (int64_t)r->n * r->m;
  int64_t total = layout == NK_LAYOUT_DENSE ? ns * P : ns * r->m;
  int64_t blocks = std::min<int64_t>((total + 255) / 256, 152 * 16);
  if (blocks < 1) blocks = 1;
  if (r->is_complex)
    logderiv_kernel<true><<<(unsigned)blocks, 256, 0, st>>>(r->n, r->m, ns, sigma, theta, layout,
                                                           o_out);
  else
    logderiv_kernel<false><<<(unsigned)blocks, 256, 0, st>>>(r->n, r->m, ns, sigma, theta, layout,
                                                            o_out);
  return check_launch("nk_logderiv");
}

NK_STATUS_COLLECTOR(collect_status_local_energy)

}  // namespace nk
