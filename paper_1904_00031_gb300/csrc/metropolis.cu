// K2: Metropolis sampling of |psi|^2 (Eq. 4; Sec. 2.2.5), single-spin flips or
// nearest-neighbour exchanges (MetropolisExchange of the VMC listing, Sec. 3.1).
//
// One warp runs one chain; a CTA runs one proposal group (all its chains draw
// the same site or bond at a step, so their table reads hit the same L1 lines).
// Per chain: sigma and theta live in shared memory, t = tanh(theta) in
// registers (lane l owns j = l + 32 q).  A proposal costs, per hidden unit, one
// table read and ~6 (real) / ~12 (complex) FMAs: |r_j|^2 with
// r_j = cosh c_j - t_j sinh c_j; the product over j is kept as mantissa * 2^e.
// Accepted moves update theta additively (theta -= 2 s W_i) and refresh
// t = tanh(theta) for the chain.  Philox draws are made 32 steps at a time, one
// step per lane, and broadcast by shuffles.
#include "common.cuh"
#include "internal.h"
#include "ratio.cuh"

namespace nk {

struct MetroArgs {
  int n, m, mp, nc, G, move, nb, n_discard, n_samples;
  uint64_t seed, counter;
  const int32_t* bond_i;
  const int32_t* bond_k;
  int8_t* sigma;        // [nc][n]
  int8_t* samples;      // [nc * n_samples][n]
  uint64_t* n_acc;      // [nc] or null
  const double* a;      // master a (F64)
  const void* tab;      // [n][mp] T2
  const void* wt;       // [n][mp] F
  const void* b32;      // [mp] F
};

// FP64 accept test U < exp(two_re).  A float pre-test with a 1e-5 relative
// margin settles all but near-ties; those get the double comparison.
__device__ __forceinline__ bool accept_test(double U, float two_re) {
  if (two_re >= 0.f) return true;
  float e32 = __expf(two_re);
  float u32 = (float)U;
  if (u32 < e32 * (1.f - 1e-5f) - 1e-37f) return true;
  if (u32 > e32 * (1.f + 1e-5f) + 1e-37f) return false;
  return U < exp((double)two_re);
}

template <bool CPLX, int E>
__global__ void __launch_bounds__(256) metropolis_kernel(MetroArgs A) {
  using F = typename RatioTypes<CPLX>::F;
  using T2 = typename RatioTypes<CPLX>::T2;
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int c = blockIdx.x * A.G + w;
  if (w >= A.G || c >= A.nc) return;
  const int n = A.n, mp = A.mp, e = mp >> 5;
  F* th = reinterpret_cast<F*>(smem) + (size_t)w * mp;
  int8_t* sg = reinterpret_cast<int8_t*>(smem + (size_t)A.G * mp * sizeof(F)) +
               (size_t)w * round_up(n, 16);
  const T2* tab = reinterpret_cast<const T2*>(A.tab);
  const F* wt = reinterpret_cast<const F*>(A.wt);
  const F* b32 = reinterpret_cast<const F*>(A.b32);

  for (int i = lane; i < n; i += 32) sg[i] = A.sigma[(int64_t)c * n + i];
  __syncwarp();
  // theta = W sigma + b (FP32), t = tanh(theta)
  F t[E];
#pragma unroll
  for (int q = 0; q < E; ++q) {
    if (q < e) {
      int j = lane + 32 * q;
      F acc = b32[j];
      for (int i = 0; i < n; ++i) {
        float si = (float)sg[i];
        F wv = wt[(int64_t)i * mp + j];
        if constexpr (CPLX) {
          acc.x = fmaf(si, wv.x, acc.x);
          acc.y = fmaf(si, wv.y, acc.y);
        } else {
          acc = fmaf(si, wv, acc);
        }
      }
      th[j] = acc;
      if constexpr (CPLX) {
        cf tt = tanh_c(cf{acc.x, acc.y});
        t[q] = make_float2(tt.x, tt.y);
      } else {
        t[q] = tanh_f(acc);
      }
    }
  }

  const int total = (A.n_discard + A.n_samples) * n;
  const uint32_t g = (uint32_t)blockIdx.x;
  uint64_t nacc = 0;
  int my_idx = 0;
  double my_u = 0.0;
  for (int step = 0; step < total; ++step) {
    const int q32 = step & 31;
    if (q32 == 0) {  // draws for steps step .. step + 31, one per lane
      uint64_t gs = A.counter + (uint64_t)(step + lane);
      u4 us = philox_stream(g, gs, kTagSite, A.seed);
      my_idx = uniform_index(us.x, A.move == NK_MOVE_FLIP ? n : A.nb);
      u4 ua = philox_stream((uint32_t)c, gs, kTagAccept, A.seed);
      my_u = uniform53(ua.x, ua.y);
    }
    const int idx = __shfl_sync(0xffffffffu, my_idx, q32);
    const double U = __shfl_sync(0xffffffffu, my_u, q32);
    int i, k = -1;
    float si, sk = 0.f;
    if (A.move == NK_MOVE_FLIP) {
      i = idx;
      si = (float)sg[i];
    } else {
      i = A.bond_i[idx];
      k = A.bond_k[idx];
      si = (float)sg[i];
      sk = (float)sg[k];
      if (si == sk) goto next;  // null move: rejected
    }
    {
      // log2 of prod_j |r_j|^2 (complex) or prod_j r_j (real), per lane
      const T2* ti = tab + (int64_t)i * mp;
      const T2* tk = tab + (int64_t)(k < 0 ? 0 : k) * mp;
      ScaledReal P;
      P.init();
#pragma unroll
      for (int q = 0; q < E; ++q) {
        if (q < e) {
          const int j = lane + 32 * q;
          if constexpr (CPLX) {
            cf C, S;
            if (k < 0) move_coef(ti[j], si, C, S);
            else move_coef2(ti[j], tk[j], si, sk, C, S);
            cf r = C - cf{t[q].x, t[q].y} * S;
            P.v *= fmaf(r.x, r.x, r.y * r.y);
          } else {
            float C, S;
            if (k < 0) move_coef(ti[j], si, C, S);
            else move_coef2(ti[j], tk[j], si, sk, C, S);
            P.v *= fmaf(-t[q], S, C);
          }
          if ((q & 3) == 3) P.renorm();
        }
      }
      float l2 = P.log2v();
#pragma unroll
      for (int off = 16; off >= 1; off >>= 1) l2 += __shfl_xor_sync(0xffffffffu, l2, off);
      // visible term: -2 s_i a_i - 2 s_k a_k (real part)
      double av = CPLX ? A.a[2 * i] : A.a[i];
      double vis = -2.0 * (double)si * av;
      if (k >= 0) vis += -2.0 * (double)sk * (CPLX ? A.a[2 * k] : A.a[k]);
      const float two_re = (CPLX ? 1.f : 2.f) * 0.69314718055994531f * l2 + 2.f * (float)vis;
      if (accept_test(U, two_re)) {
        ++nacc;
        const F* wi = wt + (int64_t)i * mp;
        const F* wk = wt + (int64_t)(k < 0 ? 0 : k) * mp;
#pragma unroll
        for (int q = 0; q < E; ++q) {
          if (q < e) {
            const int j = lane + 32 * q;
            F v = th[j];
            if constexpr (CPLX) {
              F d = wi[j];
              v.x = fmaf(-2.f * si, d.x, v.x);
              v.y = fmaf(-2.f * si, d.y, v.y);
              if (k >= 0) {
                F d2 = wk[j];
                v.x = fmaf(-2.f * sk, d2.x, v.x);
                v.y = fmaf(-2.f * sk, d2.y, v.y);
              }
              cf tt = tanh_c(cf{v.x, v.y});
              t[q] = make_float2(tt.x, tt.y);
            } else {
              v = fmaf(-2.f * si, wi[j], v);
              if (k >= 0) v = fmaf(-2.f * sk, wk[j], v);
              t[q] = tanh_f(v);
            }
            th[j] = v;
          }
        }
        __syncwarp();
        if (lane == 0) {
          sg[i] = (int8_t)(-sg[i]);
          if (k >= 0) sg[k] = (int8_t)(-sg[k]);
        }
        __syncwarp();
      }
    }
  next:
    if ((step + 1) % n == 0) {
      const int sweep = (step + 1) / n - 1;
      if (sweep >= A.n_discard) {
        int8_t* out = A.samples + ((int64_t)c * A.n_samples + (sweep - A.n_discard)) * n;
        for (int ii = lane; ii < n; ii += 32) out[ii] = sg[ii];
      }
    }
  }
  for (int ii = lane; ii < n; ii += 32) A.sigma[(int64_t)c * n + ii] = sg[ii];
  if (A.n_acc && lane == 0) A.n_acc[c] = nacc;
}

// ------------------------------------------------------------------ dispatch

template <bool CPLX, int E>
static nk_status launch_e(const MetroArgs& A, size_t smem, cudaStream_t st) {
  auto kern = metropolis_kernel<CPLX, E>;
  if (smem > 48 * 1024) {
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
      return fail(NK_ERR_CUDA, "nk_metropolis_sweep: cannot reserve %zu B shared memory", smem);
  }
  int blocks = (A.nc + A.G - 1) / A.G;
  kern<<<blocks, 32 * A.G, smem, st>>>(A);
  return check_launch("nk_metropolis_sweep");
}

template <bool CPLX>
static nk_status launch_c(const MetroArgs& A, size_t smem, cudaStream_t st) {
  int e = A.mp / 32;
  if (e <= 1) return launch_e<CPLX, 1>(A, smem, st);
  if (e <= 2) return launch_e<CPLX, 2>(A, smem, st);
  if (e <= 4) return launch_e<CPLX, 4>(A, smem, st);
  if (e <= 8) return launch_e<CPLX, 8>(A, smem, st);
  if (e <= 13) return launch_e<CPLX, 13>(A, smem, st);
  if (e <= 16) return launch_e<CPLX, 16>(A, smem, st);
  if (e <= 25) return launch_e<CPLX, 25>(A, smem, st);
  if (e <= 32) return launch_e<CPLX, 32>(A, smem, st);
  if (e <= 50) return launch_e<CPLX, 50>(A, smem, st);
  if (e <= 64) return launch_e<CPLX, 64>(A, smem, st);
  return fail(NK_ERR_SHAPE, "nk_metropolis_sweep: m = %d exceeds the register-resident limit 2048",
              A.m);
}

nk_status launch_metropolis(const nk_rbm* r, nk_chains* ch, int move, const int32_t* bi,
                            const int32_t* bk, int nb, int n_discard, int n_samples,
                            int8_t* samples, uint64_t* n_acc, cudaStream_t st) {
  WsLayout L(r->n, r->m, r->is_complex);
  MetroArgs A;
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
  A.bond_i = bi;
  A.bond_k = bk;
  A.sigma = ch->sigma;
  A.samples = samples;
  A.n_acc = n_acc;
  A.a = r->a;
  const char* ws = (const char*)r->ws;
  A.tab = ws + L.tab;
  A.wt = ws + L.wt;
  A.b32 = ws + L.b32;
  size_t f = r->is_complex ? 8 : 4;
  size_t smem = (size_t)A.G * (L.mp * f + round_up(r->n, 16));
  if (smem > 227 * 1024)
    return fail(NK_ERR_SHAPE,
                "nk_metropolis_sweep: group_size * (padded m * %zu + n) = %zu B exceeds 227 KB",
                f, smem);
  if ((int64_t)(n_discard + n_samples) * r->n > 0x7fffffff)
    return fail(NK_ERR_SHAPE, "nk_metropolis_sweep: too many proposals in one call");
  return r->is_complex ? launch_c<true>(A, smem, st) : launch_c<false>(A, smem, st);
}

}  // namespace nk
