// K2, group-lockstep form for complex RBMs (Eq. 4; Sec. 2.2.5), included by
// metropolis.cu after MetroArgs, accept_test and move_row.
//
// All chains of a proposal group propose the same site (bond) at a step, so one
// table row serves the whole group.  Here one CTA runs one group of G <= 8
// chains and its threads split the hidden units instead of the chains: thread
// tid owns the unit pairs P = tid + T p (p < PP, T threads), units 2P and
// 2P + 1, and evaluates them for every chain of the group, with
// t = tanh(theta) of all G chains in registers.  The per-chain sums of
// log2 |r_j|^2 meet in one CTA barrier per step (a transposed butterfly inside
// each warp, then one partial per warp and chain in shared memory); every warp
// then reads the same partials in the same order and takes the same accept
// decisions, so no second barrier is needed.  A step's row (|C|^2, |D|^2,
// E = conj(C) D and the theta increment of every unit pair) arrives by one
// bulk copy into a ring of R shared-memory slots, issued R - 1 steps ahead.
// theta of the G chains lives in tensor memory; the spins in shared memory, one
// byte per site with bit c set when chain c has s_i = +1 (one copy per warp).
// The ratio, the tanh addition update and the theta increments are those of
// the chain-per-warp kernel (same table values, same operations per unit); only
// the order in which the per-unit logarithms are summed differs.
#pragma once

namespace nk {

constexpr int kGroupChains = 8;  // chains per CTA at most (one bit each)

// Group rows, per site (flips) or bond (exchanges): three blocks of m2p float4
// (m2p = unit pairs of the row, T PP):
//   [P]           (|C_a|^2, |C_b|^2, |D_a|^2, |D_b|^2),
//   [m2p + P]     (Re E_a, Re E_b, -Im E_a, -Im E_b),
//   [2 m2p + P]   theta increment (Re, Im of unit a, Re, Im of unit b):
//                 W_i (flip) or W_i - W_k (exchange),
// for units a = 2P, b = 2P + 1; units >= m hold C = 1, D = 0, increment 0.
__host__ __device__ constexpr size_t group_row_bytes(int m2p) { return (size_t)48 * m2p; }

// Element x of rows * m2p.
__device__ __forceinline__ void group_rows_elem(int64_t x, bool pair, const float4* __restrict__ tab,
                                                const float2* __restrict__ wt,
                                                const int32_t* __restrict__ bi,
                                                const int32_t* __restrict__ bk, int m, int mp,
                                                int m2p, float4* __restrict__ out) {
  const int P = (int)(x % m2p);
  const int64_t r = x / m2p;
  float v[2][4];
  float2 wv[2];
#pragma unroll
  for (int u = 0; u < 2; ++u) {
    const int j = 2 * P + u;
    cf C{1.f, 0.f}, D{0.f, 0.f};
    wv[u] = make_float2(0.f, 0.f);
    if (j < m) {
      const int i = pair ? bi[r] : (int)r;
      const float4 ti = tab[(int64_t)i * mp + j];
      const cf Ai{ti.x, ti.y}, Bi{ti.z, ti.w};
      const float2 wi = wt[(int64_t)i * mp + j];
      if (pair) {
        const int k = bk[r];
        const float4 tk = tab[(int64_t)k * mp + j];
        const cf Ak{tk.x, tk.y}, Bk{tk.z, tk.w};
        C = Ai * Ak - Bi * Bk;
        D = Bi * Ak - Ai * Bk;
        const float2 wk = wt[(int64_t)k * mp + j];
        wv[u] = make_float2(wi.x - wk.x, wi.y - wk.y);
      } else {
        C = Ai;
        D = Bi;
        wv[u] = wi;
      }
    }
    const cf E = conj(C) * D;
    v[u][0] = fmaf(C.x, C.x, C.y * C.y);
    v[u][1] = fmaf(D.x, D.x, D.y * D.y);
    v[u][2] = E.x;
    v[u][3] = -E.y;
  }
  float4* row = out + r * 3 * m2p;
  row[P] = make_float4(v[0][0], v[1][0], v[0][1], v[1][1]);
  row[m2p + P] = make_float4(v[0][2], v[1][2], v[0][3], v[1][3]);
  row[2 * m2p + P] = make_float4(wv[0].x, wv[0].y, wv[1].x, wv[1].y);
}

template <bool PAIR>
__global__ void group_rows_kernel(const float4* __restrict__ tab, const float2* __restrict__ wt,
                                  const int32_t* __restrict__ bi, const int32_t* __restrict__ bk,
                                  int rows, int m, int mp, int m2p, float4* __restrict__ out) {
  const int64_t total = (int64_t)rows * m2p;
  for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < total;
       x += (int64_t)gridDim.x * blockDim.x)
    group_rows_elem(x, PAIR, tab, wt, bi, bk, m, mp, m2p, out);
}

// The accept test of one lane (its own uniform; no shuffle), decided like
// accept_test: a float pre-test with a 1e-5 relative margin, FP64 on near-ties.
__device__ __forceinline__ bool accept_lane(float u32, float two_re, uint32_t uh, uint32_t ul) {
  if (two_re >= 0.f) return true;
  const float e32 = __expf(two_re);
  if (u32 < e32 * (1.f - 1e-5f) - 1e-37f) return true;
  if (u32 > e32 * (1.f + 1e-5f) + 1e-37f) return false;
  return uniform53(uh, ul) < exp((double)two_re);
}

// Threads of the group kernel with pp hidden-unit pairs per thread (a multiple
// of 32), and the most it is launched with (registers: t of 8 chains x 2 pp
// units stays resident).
__host__ inline int group_threads(int m, int pp) {
  const int pairs = (m + 1) / 2;
  return (int)round_up((pairs + pp - 1) / pp, 32);
}
__host__ __device__ constexpr int group_max_threads(int pp) { return pp >= 3 ? 384 : 512; }

template <int PP>
__device__ __forceinline__ void metropolis_group_body(const MetroArgs& A, const int bx) {
  extern __shared__ __align__(128) unsigned char smem[];
  constexpr unsigned FULL = 0xffffffffu;
  constexpr int TCW = kGroupChains * 4 * PP;  // TMEM columns per thread: chain, pair, Re/Im a, b
  const int n = A.n, R = A.ring, m2p = A.m2p;
  const int T = (int)blockDim.x, NW = T >> 5;
  const size_t row_bytes = group_row_bytes(m2p);
  float* part = reinterpret_cast<float*>(smem + (size_t)R * row_bytes);  // [2][NW][8]
  uint64_t* full = reinterpret_cast<uint64_t*>(part + 16 * NW);           // [kMaxRing]
  uint32_t* tslot = reinterpret_cast<uint32_t*>(full + kMaxRing);         // TMEM base
  uint8_t* sgall = reinterpret_cast<uint8_t*>(tslot + 4);                  // [NW][n16]
  const int n16 = (int)round_up(n, 16);
  const uint64_t ctr = A.counter_dev ? *A.counter_dev : A.counter;

  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int cl = lane >> 2;  // the chain this lane decides for
  const int c0 = bx * A.G;
  const int nch = min(A.G, A.nc - c0);
  const uint32_t cmask = (1u << nch) - 1u;
  uint8_t* sg = sgall + (size_t)w * n16;
  const float2* wt = reinterpret_cast<const float2*>(A.wt);
  const float2* b32 = reinterpret_cast<const float2*>(A.b32);

  if (tid == 0) {
    for (int k = 0; k < R; ++k) mbar_init(&full[k], 1);
    mbar_fence_init();
  }
  for (int i = lane; i < n; i += 32) {
    uint32_t bits = 0;
    for (int c = 0; c < nch; ++c) bits |= (uint32_t)(A.sigma[(int64_t)(c0 + c) * n + i] > 0) << c;
    sg[i] = (uint8_t)bits;
  }
  // theta in tensor memory: thread (warp w, lane l) owns TMEM lane 32 (w % 4) + l,
  // columns (w / 4) TCW + c 4 PP + 4 p + (0: Re a, 1: Im a, 2: Re b, 3: Im b)
  const uint32_t tcols_total = (uint32_t)(((NW + 3) / 4) * TCW);
  const uint32_t tcols = tcols_total <= 32 ? 32 : tcols_total <= 64 ? 64 : tcols_total <= 128 ? 128
                         : tcols_total <= 256 ? 256 : 512;
  if (w == 0) tmem_alloc(tslot, tcols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tm = *tslot + ((uint32_t)(32 * (w & 3)) << 16) + (uint32_t)((w >> 2) * TCW);

  // tx[c][p] = (Re t_a, Re t_b), ty[c][p] = (Im t_a, Im t_b) of chain c, pair p
  float2 tx[kGroupChains][PP], ty[kGroupChains][PP];
  auto refresh_t = [&](int c, const float (&th)[4 * PP]) {
#pragma unroll
    for (int p = 0; p < PP; ++p) {
      const cf ta = tanh_c(cf{th[4 * p], th[4 * p + 1]});
      const cf tb = tanh_c(cf{th[4 * p + 2], th[4 * p + 3]});
      tx[c][p] = make_float2(ta.x, tb.x);
      ty[c][p] = make_float2(ta.y, tb.y);
    }
  };
  {
    // theta = W sigma + b (FP32 fma per site in site order), rows of W^T staged
    // through the (not yet used) ring
    float2* stg = reinterpret_cast<float2*>(smem);
    const int mp = A.mp;
    const int KC = (int)(((size_t)R * row_bytes) / ((size_t)mp * sizeof(float2)));
#pragma unroll
    for (int p = 0; p < PP; ++p) {
      const int ja = 2 * (tid + T * p), jb = ja + 1;
      const float2 ba = ja < A.m ? b32[ja] : make_float2(0.f, 0.f);
      const float2 bb = jb < A.m ? b32[jb] : make_float2(0.f, 0.f);
#pragma unroll
      for (int c = 0; c < kGroupChains; ++c) {
        tx[c][p] = make_float2(ba.x, bb.x);
        ty[c][p] = make_float2(ba.y, bb.y);
      }
    }
    for (int i0 = 0; i0 < n; i0 += KC) {
      const int kc = min(KC, n - i0);
      for (int x = tid; x < kc * mp; x += T) stg[x] = wt[(int64_t)i0 * mp + x];
      __syncthreads();
      for (int kk = 0; kk < kc; ++kk) {
        const uint32_t bits = sg[i0 + kk];
#pragma unroll
        for (int p = 0; p < PP; ++p) {
          const int ja = 2 * (tid + T * p), jb = ja + 1;
          const float2 wa = ja < A.m ? stg[kk * mp + ja] : make_float2(0.f, 0.f);
          const float2 wb = jb < A.m ? stg[kk * mp + jb] : make_float2(0.f, 0.f);
          const float2 wre = make_float2(wa.x, wb.x), wim = make_float2(wa.y, wb.y);
#pragma unroll
          for (int c = 0; c < kGroupChains; ++c) {
            const float s = ((bits >> c) & 1u) ? 1.f : -1.f;
            const float2 s2 = make_float2(s, s);
            tx[c][p] = f2fma(s2, wre, tx[c][p]);
            ty[c][p] = f2fma(s2, wim, ty[c][p]);
          }
        }
      }
      __syncthreads();
    }
#pragma unroll
    for (int c = 0; c < kGroupChains; ++c) {
      float th[4 * PP];
#pragma unroll
      for (int p = 0; p < PP; ++p) {
        th[4 * p] = tx[c][p].x;
        th[4 * p + 1] = ty[c][p].x;
        th[4 * p + 2] = tx[c][p].y;
        th[4 * p + 3] = ty[c][p].y;
      }
      tmem_st_cols<4 * PP>(tm + c * 4 * PP, th);
      refresh_t(c, th);
    }
    tmem_st_wait();
    // the staging writes (generic proxy) before the ring's bulk copies (async proxy)
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  __syncthreads();

  const int total = (A.n_discard + A.n_samples) * n;
  const uint32_t rbytes = (uint32_t)row_bytes;
  const unsigned char* rows = reinterpret_cast<const unsigned char*>(A.cd);
  int issued = 0;  // steps whose rows have been requested (thread 0 only)
  auto issue = [&](int step) {
    const int k = step % R;
    const int row = move_row(A, ctr, (uint32_t)bx, step);
    mbar_arrive_expect_tx(&full[k], rbytes);
    bulk_g2s(smem + (size_t)k * row_bytes, rows + (int64_t)row * row_bytes, rbytes, &full[k]);
  };
  if (tid == 0)
    for (; issued < R && issued < total; ++issued) issue(issued);
  // inverse temperature of the chain this lane decides for (exactly 1 without
  // tempering)
  const float beta =
      A.pt_R > 0 ? 1.f - (float)((c0 + cl) % A.pt_R) / (float)A.pt_R : 1.f;

  bool bad = false;       // a bounded wait gave up (CTA-uniform after each step's barrier)
  uint32_t nacc = 0;      // accepted moves this lane decided (chain cl)
  int sweep_pos = 0, sweep_no = 0, kslot = 0;
  uint32_t kphase = 0u;
  int my_i = 0, my_k = -1;  // site draws of step (32-block + lane)
  float my_da = 0.f;
  uint32_t my_uh = 0u, my_ul = 0u;  // accept draw of chain cl, step (4-block + lane % 4)
  float my_u32 = 0.f;
  for (int step = 0; step < total; ++step) {
    const int q32 = step & 31;
    if (q32 == 0) {
      const uint64_t gs = ctr + (uint64_t)(step + lane);
      const u4 us = philox_stream((uint32_t)bx, gs, kTagSite, A.seed);
      const int idx = uniform_index(us.x, A.move == NK_MOVE_FLIP ? n : A.nb);
      if (A.move == NK_MOVE_FLIP) {
        my_i = idx;
        my_k = -1;
        my_da = (float)A.a[2 * idx];
      } else {
        my_i = A.bond_i[idx];
        my_k = A.bond_k[idx];
        my_da = (float)(A.a[2 * my_i] - A.a[2 * my_k]);
      }
    }
    if ((step & 3) == 0) {
      const uint64_t gs = ctr + (uint64_t)(step + (lane & 3));
      const u4 ua = philox_stream((uint32_t)(c0 + cl), gs, kTagAccept, A.seed);
      my_uh = ua.x;
      my_ul = ua.y;
      my_u32 = uniform53_f(ua.x, ua.y);
    }
    const int i = __shfl_sync(FULL, my_i, q32);
    const int kk2 = __shfl_sync(FULL, my_k, q32);
    const float da = __shfl_sync(FULL, my_da, q32);
    const uint32_t mi = sg[i];
    // chains whose proposal is not null (an exchange of equal spins is)
    const uint32_t nn = (kk2 >= 0 ? (mi ^ (uint32_t)sg[kk2]) : 0xffu) & cmask;
    const int k = kslot;
    if (!bad) {
      const bool ok = mbar_wait_bounded(&full[k], kphase);
      bad = __any_sync(FULL, !ok);
    }
    const float4* row4 = reinterpret_cast<const float4*>(smem + (size_t)k * row_bytes);
    float2 c2[PP], d2[PP], ex[PP], ney[PP];
#pragma unroll
    for (int p = 0; p < PP; ++p) {
      const float4 q0 = row4[tid + T * p];
      const float4 q1 = row4[m2p + tid + T * p];
      c2[p] = make_float2(q0.x, q0.y);
      d2[p] = make_float2(q0.z, q0.w);
      ex[p] = make_float2(q1.x, q1.y);
      ney[p] = make_float2(q1.z, q1.w);
    }
    // this thread's share of log2 prod_j |r_j|^2 for every chain; at most 2 PP
    // factors meet in one float (PP <= 2: one product of four factors in
    // (2^-31, 2^31) each)
    float v[kGroupChains];
#pragma unroll
    for (int c = 0; c < kGroupChains; ++c) {
      v[c] = 0.f;
      if (!bad && ((nn >> c) & 1u)) {
        const float si = ((mi >> c) & 1u) ? 1.f : -1.f;
        const float2 m2s = make_float2(-2.f * si, -2.f * si);
        float2 Pp = make_float2(1.f, 1.f);
#pragma unroll
        for (int p = 0; p < PP; ++p) {
          const float2 tt = f2fma(tx[c][p], tx[c][p], f2mul(ty[c][p], ty[c][p]));
          const float2 e = f2fma(tx[c][p], ex[p], f2mul(ty[c][p], ney[p]));  // Re(t E)
          Pp = f2mul(Pp, f2fma(m2s, e, f2fma(tt, d2[p], c2[p])));
        }
        v[c] = clamp_log2(PP <= 2 ? __log2f(Pp.x * Pp.y) : __log2f(Pp.x) + __log2f(Pp.y));
      }
    }
    // transposed butterfly: lane l ends with the warp's sum for chain l >> 2
    float y;
    {
      const bool b4 = (lane & 16) != 0, b3 = (lane & 8) != 0, b2 = (lane & 4) != 0;
      float w4[4], w2[2];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float send = b4 ? v[q] : v[q + 4];
        const float keep = b4 ? v[q + 4] : v[q];
        w4[q] = keep + __shfl_xor_sync(FULL, send, 16);
      }
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const float send = b3 ? w4[q] : w4[q + 2];
        const float keep = b3 ? w4[q + 2] : w4[q];
        w2[q] = keep + __shfl_xor_sync(FULL, send, 8);
      }
      const float send = b2 ? w2[0] : w2[1];
      const float keep = b2 ? w2[1] : w2[0];
      y = keep + __shfl_xor_sync(FULL, send, 4);
      y += __shfl_xor_sync(FULL, y, 1);
      y += __shfl_xor_sync(FULL, y, 2);
    }
    // one partial per warp and chain (double-buffered by step parity: a warp
    // writes this buffer again two steps on, after every warp has passed the
    // next barrier, i.e. has read it); a warp whose wait gave up writes NaN,
    // which no finite (clamped) partial can produce
    float* pp = part + (step & 1) * NW * kGroupChains;
    if ((lane & 3) == 0) pp[w * kGroupChains + cl] = bad ? __int_as_float(0x7fc00000) : y;
    __syncthreads();
    // every slot of step - 1 has been used by every warp: refill it
    if (tid == 0 && !bad && step >= 1 && issued < total && issued == step - 1 + R) {
      issue(issued);
      ++issued;
    }
    // the chain's total, summed in the same order by every warp
    float tot = 0.f;
    for (int w2 = lane & 3; w2 < NW; w2 += 4) tot += pp[w2 * kGroupChains + cl];
    tot += __shfl_xor_sync(FULL, tot, 1);
    tot += __shfl_xor_sync(FULL, tot, 2);
    bad = __any_sync(FULL, tot != tot) || bad;
    uint32_t acc8 = 0;
    if (!bad) {
      bool acc = false;
      if ((lane & 3) == (step & 3) && ((nn >> cl) & 1u)) {
        const float si = ((mi >> cl) & 1u) ? 1.f : -1.f;
        // visible term -2 s_i (a_i - a_k), in FP32 like the hidden-unit product
        const float two_re = 0.69314718055994531f * tot - 4.f * si * da;
        acc = accept_lane(my_u32, beta * two_re, my_uh, my_ul);
      }
      const uint32_t bal = __ballot_sync(FULL, acc) >> (step & 3);
#pragma unroll
      for (int c = 0; c < kGroupChains; ++c) acc8 |= ((bal >> (4 * c)) & 1u) << c;
      nacc += acc ? 1u : 0u;
    }
    if (acc8) {
      const float4* wd4 = row4 + 2 * m2p;
      float4 wdp[PP];
#pragma unroll
      for (int p = 0; p < PP; ++p) wdp[p] = wd4[tid + T * p];
#pragma unroll
      for (int c = 0; c < kGroupChains; ++c) {
        if ((acc8 >> c) & 1u) {
          const float si = ((mi >> c) & 1u) ? 1.f : -1.f;
          tmem_st_wait();  // earlier stores to these columns
          float th[4 * PP];
          tmem_ld_cols<4 * PP>(tm + c * 4 * PP, th);
#pragma unroll
          for (int p = 0; p < PP; ++p) t_add_pair(tx[c][p], ty[c][p], c2[p], d2[p], ex[p], ney[p], si);
          tmem_ld_wait();
          const float m2s = -2.f * si;
#pragma unroll
          for (int p = 0; p < PP; ++p) {
            th[4 * p] = fmaf(m2s, wdp[p].x, th[4 * p]);
            th[4 * p + 1] = fmaf(m2s, wdp[p].y, th[4 * p + 1]);
            th[4 * p + 2] = fmaf(m2s, wdp[p].z, th[4 * p + 2]);
            th[4 * p + 3] = fmaf(m2s, wdp[p].w, th[4 * p + 3]);
          }
          tmem_st_cols<4 * PP>(tm + c * 4 * PP, th);
        }
      }
      __syncwarp();
      if (lane == 0) {
        sg[i] = (uint8_t)(mi ^ acc8);
        if (kk2 >= 0) sg[kk2] = (uint8_t)(sg[kk2] ^ acc8);
      }
    }
    __syncwarp();
    if (++sweep_pos == n) {  // the last step of a sweep
      sweep_pos = 0;
      const int sweep = sweep_no++;
      if (!bad && sweep >= A.n_discard) {
        for (int ii = tid; ii < n; ii += T) {
          const uint32_t bits = sg[ii];
          for (int c = 0; c < nch; ++c)
            A.samples[((int64_t)(c0 + c) * A.n_samples + (sweep - A.n_discard)) * n + ii] =
                ((bits >> c) & 1u) ? (int8_t)1 : (int8_t)-1;
        }
      }
      if (!bad) {
        // exact refresh of t from theta
        tmem_st_wait();
#pragma unroll
        for (int c = 0; c < kGroupChains; ++c) {
          float th[4 * PP];
          tmem_ld_cols<4 * PP>(tm + c * 4 * PP, th);
          tmem_ld_wait();
          refresh_t(c, th);
        }
      }
    }
    if (++kslot == R) {
      kslot = 0;
      kphase ^= 1u;
    }
    if (bad) break;  // uniform: every warp saw the same partials
  }
  tmem_st_wait();
  if (A.lval) {
    // 2 Re ln psi of every chain's final state: Re ln cosh of this thread's
    // units (FP32 each, summed in FP64), reduced over the CTA in a fixed order;
    // the visible term in FP64 from the master a
    double lr[kGroupChains];
#pragma unroll
    for (int c = 0; c < kGroupChains; ++c) {
      lr[c] = 0.0;
      float th[4 * PP];
      tmem_ld_cols<4 * PP>(tm + c * 4 * PP, th);
      tmem_ld_wait();
#pragma unroll
      for (int p = 0; p < PP; ++p) {
        const int ja = 2 * (tid + T * p);
        if (ja < A.m) lr[c] += (double)lncosh_c(cf{th[4 * p], th[4 * p + 1]}).x;
        if (ja + 1 < A.m) lr[c] += (double)lncosh_c(cf{th[4 * p + 2], th[4 * p + 3]}).x;
      }
#pragma unroll
      for (int off = 16; off >= 1; off >>= 1) lr[c] += __shfl_xor_sync(FULL, lr[c], off);
    }
    __syncthreads();  // every warp has read its last partials
    double* dp = reinterpret_cast<double*>(part);  // [NW][8], the partials' bytes
#pragma unroll
    for (int c = 0; c < kGroupChains; ++c)
      if (lane == c) dp[w * kGroupChains + c] = lr[c];
    __syncthreads();
    if (w == 0 && lane < nch) {
      double s = 0.0;
      for (int w2 = 0; w2 < NW; ++w2) s += dp[w2 * kGroupChains + lane];
      double va = 0.0;
      for (int ii = 0; ii < n; ++ii) va += A.a[2 * ii] * (((sg[ii] >> lane) & 1u) ? 1.0 : -1.0);
      A.lval[c0 + lane] = bad ? __longlong_as_double(0x7ff8000000000000ll) : 2.0 * (s + va);
    }
  }
  if (bad && lane == 0) dev_status_set(1u << NK_ERR_TIMEOUT);
  if (bad && tid == 0) {
    // let the copies still in flight land before the CTA exits: the last
    // issued step of each slot
    for (int k = 0; k < R; ++k) {
      int last = -1;
      for (int s = issued - 1; s >= 0 && s >= issued - R; --s)
        if (s % R == k) last = s;
      if (last >= 0) mbar_wait_bounded(&full[k], (uint32_t)((last / R) & 1), 1u << 20);
    }
  }
  if (w == 0) {
    for (int ii = lane; ii < n; ii += 32) {
      const uint32_t bits = sg[ii];
      for (int c = 0; c < nch; ++c)
        A.sigma[(int64_t)(c0 + c) * n + ii] = ((bits >> c) & 1u) ? (int8_t)1 : (int8_t)-1;
    }
    uint32_t cnt = nacc;
    cnt += __shfl_xor_sync(FULL, cnt, 1);
    cnt += __shfl_xor_sync(FULL, cnt, 2);
    if (A.n_acc && (lane & 3) == 0 && cl < nch) {
      const int c = c0 + cl;
      if (bad) A.n_acc[c] = ~0ull;
      else if (A.acc_add) {
        if (A.n_acc[c] != ~0ull) A.n_acc[c] += cnt;  // a timeout marked earlier stays
      } else {
        A.n_acc[c] = cnt;
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (w == 0) {
    tc_fence_after();
    tmem_dealloc(*tslot, tcols);
  }
}

template <int PP>
__global__ void __launch_bounds__(group_max_threads(PP), 1) metropolis_group_kernel(MetroArgs A) {
  metropolis_group_body<PP>(A, blockIdx.x);
}

template <int PP>
__global__ void __launch_bounds__(group_max_threads(PP), 1) metropolis_group_batch_kernel(
    const __grid_constant__ MetroBatch B) {
  int k = 0;
  while (k + 1 < B.n && (int)blockIdx.x >= B.start[k + 1]) ++k;
  metropolis_group_body<PP>(B.a[k], (int)blockIdx.x - B.start[k]);
}

}  // namespace nk
