// K3: local energies E_loc(sigma) = sum_sigma' <sigma|H|sigma'> psi(sigma')/psi(sigma)
// (Eq. 5, Sec. 2.2.5) for a Hamiltonian of 1-local and 2-local terms, and K4:
// the factored log-derivatives T = tanh(theta) (Sec. 2.2.5: O_b = tanh theta,
// O_W = tanh theta (x) sigma, O_a = sigma).
//
// One warp per configuration.  The warp loads theta, keeps t = tanh(theta) in
// registers (writing T out as a side product) and walks the compiled move
// list; every move's psi ratio is exp(visible) * prod_j (cosh c_j - t_j sinh c_j)
// from the cosh/sinh(2W) tables, with the product kept as mantissa * 2^e.  All
// warps of a CTA walk the same list, so the table columns of a move are read
// from L2 once per CTA.  Sums are FP64.
#include "common.cuh"
#include "internal.h"
#include "opdev.h"
#include "ratio.cuh"

namespace nk {

struct ElocArgs {
  int n, m, mp;
  int64_t ns;
  const int8_t* sigma;
  const void* theta;   // [ns][m] F
  const char* op;      // compiled operator
  const double* a;     // master a
  const void* tab;     // [n][mp] T2
  double* eloc;        // c128 [ns]
  void* t_out;         // [ns][m] F or null
};

__device__ __forceinline__ int idx_of(int8_t s) { return s > 0 ? 0 : 1; }

template <bool CPLX, int E>
__global__ void __launch_bounds__(256) local_energy_kernel(ElocArgs A) {
  using F = typename RatioTypes<CPLX>::F;
  using T2 = typename RatioTypes<CPLX>::T2;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t s = (int64_t)blockIdx.x * (blockDim.x >> 5) + w;
  if (s >= A.ns) return;
  const int n = A.n, m = A.m, mp = A.mp, e = mp >> 5;
  const int8_t* sg = A.sigma + s * n;
  const F* th = reinterpret_cast<const F*>(A.theta) + s * m;
  F* tout = reinterpret_cast<F*>(A.t_out);
  F t[E];
#pragma unroll
  for (int q = 0; q < E; ++q) {
    if (q < e) {
      const int j = lane + 32 * q;
      if constexpr (CPLX) {
        t[q] = make_float2(0.f, 0.f);
        if (j < m) {
          F v = th[j];
          cf tt = tanh_c(cf{v.x, v.y});
          t[q] = make_float2(tt.x, tt.y);
          if (tout) tout[s * m + j] = t[q];
        }
      } else {
        t[q] = 0.f;
        if (j < m) {
          t[q] = tanh_f(th[j]);
          if (tout) tout[s * m + j] = t[q];
        }
      }
    }
  }
  const OpDevHeader* H = reinterpret_cast<const OpDevHeader*>(A.op);
  const OpDSite* ds = reinterpret_cast<const OpDSite*>(A.op + H->off_dsite);
  const OpDBond* db = reinterpret_cast<const OpDBond*>(A.op + H->off_dbond);
  const OpMove* mv = reinterpret_cast<const OpMove*>(A.op + H->off_moves);
  // diagonal part, lanes split the terms
  double er = 0.0, ei = 0.0;
  for (int u = lane; u < H->n_dsite; u += 32) {
    int x = idx_of(sg[ds[u].i]);
    er += ds[u].d[x][0];
    ei += ds[u].d[x][1];
  }
  for (int u = lane; u < H->n_dbond; u += 32) {
    int x = 2 * idx_of(sg[db[u].i]) + idx_of(sg[db[u].k]);
    er += db[u].d[x][0];
    ei += db[u].d[x][1];
  }
#pragma unroll
  for (int off = 16; off >= 1; off >>= 1) {
    er += __shfl_xor_sync(0xffffffffu, er, off);
    ei += __shfl_xor_sync(0xffffffffu, ei, off);
  }
  const T2* tab = reinterpret_cast<const T2*>(A.tab);
  const int nm = H->n_moves;
  for (int u = 0; u < nm; ++u) {
    const int i = mv[u].i, k = mv[u].k, two = mv[u].two;
    const int8_t sik = sg[i], skk = sg[k];
    const int x = 2 * idx_of(sik) + idx_of(skk);
    const double mr = mv[u].mel[x][0], mi = mv[u].mel[x][1];
    if (mr == 0.0 && mi == 0.0) continue;  // warp-uniform
    const float si = (float)sik, sk = (float)skk;
    const T2* ti = tab + (int64_t)i * mp;
    const T2* tk = tab + (int64_t)k * mp;
    double pr, pi;  // prod_j r_j (complex double after the warp reduction)
    if constexpr (CPLX) {
      ScaledComplex P;
      P.init();
#pragma unroll
      for (int q = 0; q < E; ++q) {
        if (q < e) {
          const int j = lane + 32 * q;
          cf C, S;
          if (!two) move_coef(ti[j], si, C, S);
          else move_coef2(ti[j], tk[j], si, sk, C, S);
          P.v = P.v * (C - cf{t[q].x, t[q].y} * S);
          if ((q & 3) == 3) P.renorm();
        }
      }
      P.renorm();
#pragma unroll
      for (int off = 16; off >= 1; off >>= 1) {
        ScaledComplex o;
        o.v.x = __shfl_xor_sync(0xffffffffu, P.v.x, off);
        o.v.y = __shfl_xor_sync(0xffffffffu, P.v.y, off);
        o.e = __shfl_xor_sync(0xffffffffu, P.e, off);
        mul_scaled(P, o);
      }
      pr = ldexp((double)P.v.x, P.e);
      pi = ldexp((double)P.v.y, P.e);
    } else {
      ScaledReal P;
      P.init();
#pragma unroll
      for (int q = 0; q < E; ++q) {
        if (q < e) {
          const int j = lane + 32 * q;
          float C, S;
          if (!two) move_coef(ti[j], si, C, S);
          else move_coef2(ti[j], tk[j], si, sk, C, S);
          P.v *= fmaf(-t[q], S, C);
          if ((q & 3) == 3) P.renorm();
        }
      }
      P.renorm();
#pragma unroll
      for (int off = 16; off >= 1; off >>= 1) {
        float ov = __shfl_xor_sync(0xffffffffu, P.v, off);
        int oe = __shfl_xor_sync(0xffffffffu, P.e, off);
        P.v *= ov;
        P.e += oe;
        P.renorm();
      }
      pr = ldexp((double)P.v, P.e);
      pi = 0.0;
    }
    // visible factor exp(-2 s_i a_i (- 2 s_k a_k)), FP64
    double vr, vi;
    if constexpr (CPLX) {
      vr = -2.0 * si * A.a[2 * i];
      vi = -2.0 * si * A.a[2 * i + 1];
      if (two) {
        vr += -2.0 * sk * A.a[2 * k];
        vi += -2.0 * sk * A.a[2 * k + 1];
      }
    } else {
      vr = -2.0 * si * A.a[i];
      vi = 0.0;
      if (two) vr += -2.0 * sk * A.a[k];
    }
    double ev = exp(vr), c = cos(vi), sn = sin(vi);
    double fr = ev * c, fi = ev * sn;                   // exp(visible)
    double qr = fr * pr - fi * pi, qi = fr * pi + fi * pr;  // ratio psi'/psi
    er += mr * qr - mi * qi;
    ei += mr * qi + mi * qr;
  }
  if (lane == 0) {
    A.eloc[2 * s] = er;
    A.eloc[2 * s + 1] = ei;
  }
}

template <bool CPLX, int E>
static nk_status launch_e(const ElocArgs& A, cudaStream_t st) {
  const int warps = 8;
  int64_t blocks = (A.ns + warps - 1) / warps;
  local_energy_kernel<CPLX, E><<<(unsigned)blocks, 32 * warps, 0, st>>>(A);
  return check_launch("nk_local_energy");
}

template <bool CPLX>
static nk_status launch_c(const ElocArgs& A, cudaStream_t st) {
  int e = A.mp / 32;
  if (e <= 1) return launch_e<CPLX, 1>(A, st);
  if (e <= 2) return launch_e<CPLX, 2>(A, st);
  if (e <= 4) return launch_e<CPLX, 4>(A, st);
  if (e <= 8) return launch_e<CPLX, 8>(A, st);
  if (e <= 13) return launch_e<CPLX, 13>(A, st);
  if (e <= 16) return launch_e<CPLX, 16>(A, st);
  if (e <= 25) return launch_e<CPLX, 25>(A, st);
  if (e <= 32) return launch_e<CPLX, 32>(A, st);
  if (e <= 50) return launch_e<CPLX, 50>(A, st);
  if (e <= 64) return launch_e<CPLX, 64>(A, st);
  return fail(NK_ERR_SHAPE, "nk_local_energy: m = %d exceeds the register-resident limit 2048",
              A.m);
}

nk_status launch_local_energy(const nk_rbm* r, const void* op_dev, const int8_t* sigma,
                              const void* theta, int64_t ns, double* eloc, void* t_out,
                              cudaStream_t st) {
  WsLayout L(r->n, r->m, r->is_complex);
  ElocArgs A;
  A.n = r->n;
  A.m = r->m;
  A.mp = L.mp;
  A.ns = ns;
  A.sigma = sigma;
  A.theta = theta;
  A.op = (const char*)op_dev;
  A.a = r->a;
  A.tab = (const char*)r->ws + L.tab;
  A.eloc = eloc;
  A.t_out = t_out;
  return r->is_complex ? launch_c<true>(A, st) : launch_c<false>(A, st);
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

}  // namespace nk
