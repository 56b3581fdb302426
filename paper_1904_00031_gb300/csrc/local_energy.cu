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

// Tiled form: a CTA owns 64 configurations and walks the move list in tiles of
// 64 moves; per chunk of 16 hidden units it stages t = tanh(theta) of its
// configurations and (cosh c, sinh c / s_i) of the tile's moves in shared
// memory, and every thread advances a 4 x 4 block of running products
// prod_j (cosh c_j - s_i t_j sinh c_j / s_i) held in registers: each staged value
// is reused by 16 threads, so the kernel is bound by the FP32 pipe rather
// than by the memory system.  A two-spin move with cosh c = A_i A_k +/- B_i B_k,
// sinh c / s_i = B_i A_k +/- A_i B_k is built in the staging step from the
// site tables; the sign is fixed per move (alignment split at compilation).
constexpr int kEBS = 64;   // configurations per CTA
constexpr int kEBM = 64;   // moves per tile
constexpr int kEBK = 16;   // hidden units per chunk
constexpr int kERenorm = 8;

template <bool CPLX>
struct EScaled;
template <>
struct EScaled<true> {
  using S = ScaledComplex;
};
template <>
struct EScaled<false> {
  using S = ScaledReal;
};

template <bool CPLX>
__global__ void __launch_bounds__(256) local_energy_tiled(ElocArgs A) {
  using F = typename RatioTypes<CPLX>::F;
  using T2 = typename RatioTypes<CPLX>::T2;
  __shared__ __align__(16) F tS[kEBK][kEBS];
  __shared__ __align__(16) F Cs[kEBK][kEBM];
  __shared__ __align__(16) F Ds[kEBK][kEBM];
  __shared__ int mvi[kEBM], mvk[kEBM], mvtwo[kEBM], mval[kEBM];
  __shared__ double2 cvs[kEBM][4];  // mel(x) * exp(visible(x)) per sign pattern x

  const int tid = threadIdx.x, ts = tid >> 4, tm = tid & 15;
  const int64_t s0 = (int64_t)blockIdx.x * kEBS;
  const int n = A.n, m = A.m, mp = A.mp;
  const OpDevHeader* H = reinterpret_cast<const OpDevHeader*>(A.op);
  const OpDSite* ds = reinterpret_cast<const OpDSite*>(A.op + H->off_dsite);
  const OpDBond* db = reinterpret_cast<const OpDBond*>(A.op + H->off_dbond);
  const OpMove* mvs = reinterpret_cast<const OpMove*>(A.op + H->off_moves);
  const T2* tab = reinterpret_cast<const T2*>(A.tab);
  const F* th = reinterpret_cast<const F*>(A.theta);
  F* tout = reinterpret_cast<F*>(A.t_out);

  // diagonal part: the 16 threads of a configuration split the terms
  double er[4], ei[4];
#pragma unroll
  for (int p = 0; p < 4; ++p) {
    er[p] = ei[p] = 0.0;
    const int64_t s = s0 + ts * 4 + p;
    if (s >= A.ns) continue;
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

  const int nm = H->n_moves;
  for (int mt0 = 0; mt0 < nm; mt0 += kEBM) {
    __syncthreads();
    if (tid < kEBM) {
      const int mv = mt0 + tid;
      if (mv < nm) {
        mvi[tid] = mvs[mv].i;
        mvk[tid] = mvs[mv].k;
        mvtwo[tid] = mvs[mv].two;
        mval[tid] = mvs[mv].align;
      } else {
        mvi[tid] = 0;
        mvk[tid] = 0;
        mvtwo[tid] = -1;  // padding move: ratio 1, coefficient 0
        mval[tid] = 1;
      }
    }
    {
      const int mm = tid >> 2, x = tid & 3, mv = mt0 + mm;
      double cr = 0.0, ci = 0.0;
      if (mv < nm) {
        const double mr = mvs[mv].mel[x][0], mi = mvs[mv].mel[x][1];
        if (mr != 0.0 || mi != 0.0) {
          const double si = (x >> 1) ? -1.0 : 1.0, sk = (x & 1) ? -1.0 : 1.0;
          const int i = mvs[mv].i, k = mvs[mv].k;
          double vr, vi;
          if (CPLX) {
            vr = -2.0 * si * A.a[2 * i];
            vi = -2.0 * si * A.a[2 * i + 1];
            if (mvs[mv].two) {
              vr += -2.0 * sk * A.a[2 * k];
              vi += -2.0 * sk * A.a[2 * k + 1];
            }
          } else {
            vr = -2.0 * si * A.a[i];
            vi = 0.0;
            if (mvs[mv].two) vr += -2.0 * sk * A.a[k];
          }
          const double ev = exp(vr), fr = ev * cos(vi), fi = ev * sin(vi);
          cr = mr * fr - mi * fi;
          ci = mr * fi + mi * fr;
        }
      }
      cvs[mm][x] = make_double2(cr, ci);
    }
    __syncthreads();
    float sgn[4][4];
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      const int64_t s = s0 + ts * 4 + p;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int mm = tm + 16 * q;
        sgn[p][q] = (s < A.ns) ? (float)A.sigma[s * n + mvi[mm]] : 1.f;
      }
    }
    typename EScaled<CPLX>::S P[4][4];
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
      for (int q = 0; q < 4; ++q) P[p][q].init();

    for (int k0 = 0; k0 < mp; k0 += kEBK) {
      __syncthreads();
      // stage t = tanh(theta): 64 configurations x 16 hidden units
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int e = tid + u * 256, ss = e >> 4, kk = e & 15;
        const int64_t s = s0 + ss;
        const int j = k0 + kk;
        F tv;
        // after the first move tile, t is reread from this CTA's own output
        const bool reuse = tout && mt0 > 0;
        if constexpr (CPLX) {
          tv = make_float2(0.f, 0.f);
          if (s < A.ns && j < m) {
            if (reuse) {
              tv = tout[s * m + j];
            } else {
              F x = th[s * m + j];
              cf c = tanh_c(cf{x.x, x.y});
              tv = make_float2(c.x, c.y);
              if (tout) tout[s * m + j] = tv;
            }
          }
        } else {
          tv = 0.f;
          if (s < A.ns && j < m) {
            if (reuse) {
              tv = tout[s * m + j];
            } else {
              tv = tanh_f(th[s * m + j]);
              if (tout) tout[s * m + j] = tv;
            }
          }
        }
        tS[kk][ss] = tv;
      }
      // stage (cosh c, sinh c / s_i) of 64 moves x 16 hidden units
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int e = tid + u * 256, mm = e >> 4, kk = e & 15;
        const int j = k0 + kk;
        const int two = mvtwo[mm];
        F C, D;
        if constexpr (CPLX) {
          if (two < 0) {
            C = make_float2(1.f, 0.f);
            D = make_float2(0.f, 0.f);
          } else {
            const float4 ai = tab[(int64_t)mvi[mm] * mp + j];
            if (!two) {
              C = make_float2(ai.x, ai.y);
              D = make_float2(ai.z, ai.w);
            } else {
              const float4 ak = tab[(int64_t)mvk[mm] * mp + j];
              const float al = (float)mval[mm];
              cf Ai{ai.x, ai.y}, Bi{ai.z, ai.w}, Ak{ak.x, ak.y}, Bk{ak.z, ak.w};
              cf c = Ai * Ak + al * (Bi * Bk);
              cf d = Bi * Ak + al * (Ai * Bk);
              C = make_float2(c.x, c.y);
              D = make_float2(d.x, d.y);
            }
          }
        } else {
          if (two < 0) {
            C = 1.f;
            D = 0.f;
          } else {
            const float2 ai = tab[(int64_t)mvi[mm] * mp + j];
            if (!two) {
              C = ai.x;
              D = ai.y;
            } else {
              const float2 ak = tab[(int64_t)mvk[mm] * mp + j];
              const float al = (float)mval[mm];
              C = fmaf(al * ai.y, ak.y, ai.x * ak.x);
              D = fmaf(al * ai.x, ak.y, ai.y * ak.x);
            }
          }
        }
        Cs[kk][mm] = C;
        Ds[kk][mm] = D;
      }
      __syncthreads();
#pragma unroll
      for (int kk = 0; kk < kEBK; ++kk) {
        F t[4], C[4], D[4];
#pragma unroll
        for (int p = 0; p < 4; ++p) t[p] = tS[kk][ts * 4 + p];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          C[q] = Cs[kk][tm + 16 * q];
          D[q] = Ds[kk][tm + 16 * q];
        }
#pragma unroll
        for (int p = 0; p < 4; ++p) {
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            if constexpr (CPLX) {
              const float tdx = fmaf(t[p].x, D[q].x, -t[p].y * D[q].y);
              const float tdy = fmaf(t[p].x, D[q].y, t[p].y * D[q].x);
              const float rx = fmaf(-sgn[p][q], tdx, C[q].x);
              const float ry = fmaf(-sgn[p][q], tdy, C[q].y);
              P[p][q].v = P[p][q].v * cf{rx, ry};
            } else {
              P[p][q].v *= fmaf(-sgn[p][q] * t[p], D[q], C[q]);
            }
          }
        }
        if ((kk % kERenorm) == kERenorm - 1) {
#pragma unroll
          for (int p = 0; p < 4; ++p)
#pragma unroll
            for (int q = 0; q < 4; ++q) P[p][q].renorm();
        }
      }
    }
    // fold the tile's ratios into the local energies (FP64)
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      const int64_t s = s0 + ts * 4 + p;
      if (s >= A.ns) continue;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int mm = tm + 16 * q;
        if (mvtwo[mm] < 0) continue;
        const int x = 2 * idx_of(A.sigma[s * n + mvi[mm]]) + idx_of(A.sigma[s * n + mvk[mm]]);
        const double2 cv = cvs[mm][x];
        if (cv.x == 0.0 && cv.y == 0.0) continue;
        double pr, pi;
        if constexpr (CPLX) {
          pr = ldexp((double)P[p][q].v.x, P[p][q].e);
          pi = ldexp((double)P[p][q].v.y, P[p][q].e);
        } else {
          pr = ldexp((double)P[p][q].v, P[p][q].e);
          pi = 0.0;
        }
        er[p] += cv.x * pr - cv.y * pi;
        ei[p] += cv.x * pi + cv.y * pr;
      }
    }
  }
  // the 16 threads of a configuration are lanes tid ^ 1, 2, 4, 8 of one warp
#pragma unroll
  for (int p = 0; p < 4; ++p) {
#pragma unroll
    for (int off = 8; off >= 1; off >>= 1) {
      er[p] += __shfl_xor_sync(0xffffffffu, er[p], off);
      ei[p] += __shfl_xor_sync(0xffffffffu, ei[p], off);
    }
    const int64_t s = s0 + ts * 4 + p;
    if (tm == 0 && s < A.ns) {
      A.eloc[2 * s] = er[p];
      A.eloc[2 * s + 1] = ei[p];
    }
  }
  // with no moves at all, t = tanh(theta) is still written
  if (nm == 0 && tout) {
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
  const int64_t blocks = (ns + kEBS - 1) / kEBS;
  if (r->is_complex)
    local_energy_tiled<true><<<(unsigned)blocks, 256, 0, st>>>(A);
  else
    local_energy_tiled<false><<<(unsigned)blocks, 256, 0, st>>>(A);
  return check_launch("nk_local_energy");
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
