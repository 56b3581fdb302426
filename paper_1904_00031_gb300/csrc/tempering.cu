// Parallel tempering (replica exchange), the sampler option Sec. 2.2.5 names to
// improve sampling.  Readings (the paper gives none of the details): each chain
// is a ladder of R replicas at beta_r = 1 - r / R, replica r sampling
// |psi|^(2 beta_r); replicas are numbered chain-major (c R + r) and each runs the
// Metropolis sweep of metropolis.cu at its own beta (its proposal group and
// Philox streams by replica number); after every sweep, neighbouring replicas
// (r, r + 1) exchange states, over the pairs starting at r = 0 on even sweeps
// and at r = 1 on odd ones, iff U < exp((beta_r - beta_(r+1)) (L_(r+1) - L_r)),
// L = 2 Re ln psi, with U from Philox stream (replica c R + r, sweep, SWAP); only
// the beta = 1 replica is recorded, one sample per sweep after the burn-in.
//
// One sweep is two launches: the Metropolis kernel over all replicas (one
// sweep, accept counts accumulated, 2 Re ln psi of every final state written
// from theta in tensor memory), then pt_exchange_kernel, one warp per ladder,
// which decides the exchanges in FP64, swaps the replicas' states and L values,
// and records the beta = 1 replica.  The sweep number of an exchange is
// floor(counter / n) with counter the chains' proposal counter before the sweep.
#include "common.cuh"
#include "internal.h"

namespace nk {

namespace {

constexpr uint32_t kTagSwap = 0x53574150u;  // "SWAP": exchange uniform per replica and sweep
constexpr int kPtWarps = 4;                 // ladders (warps) per block

__global__ void __launch_bounds__(32 * kPtWarps)
    pt_exchange_kernel(int8_t* __restrict__ sigma, double* __restrict__ lval, int n, int nlad,
                       int R, uint64_t seed, const uint64_t* ctr_dev, uint64_t ctr_host,
                       int8_t* __restrict__ samples, int n_samples, int record,
                       uint64_t* __restrict__ n_swap) {
  const int lane = threadIdx.x & 31;
  const int lad = blockIdx.x * kPtWarps + (threadIdx.x >> 5);
  if (lad >= nlad) return;
  // the counter after this sweep's Metropolis launch, which advanced it by n
  const uint64_t after = ctr_dev ? *ctr_dev : ctr_host;
  const uint64_t sweep = after / (uint64_t)n - 1;
  const int64_t base = (int64_t)lad * R;
  for (int r = (int)(sweep & 1); r + 1 < R; r += 2) {
    const int64_t lo = base + r, hi = lo + 1;
    const u4 u = philox_stream((uint32_t)lo, sweep, kTagSwap, seed);
    const double U = uniform53(u.x, u.y);
    const double br = 1.0 - (double)r / (double)R, bs = 1.0 - (double)(r + 1) / (double)R;
    const double ll = lval[lo], lh = lval[hi];
    const bool ok = U < exp((br - bs) * (lh - ll));
    if (ok) {  // warp-uniform: every lane computed the same decision
      int8_t* a = sigma + lo * n;
      int8_t* b = sigma + hi * n;
      for (int i = lane; i < n; i += 32) {
        const int8_t t = a[i];
        a[i] = b[i];
        b[i] = t;
      }
      if (lane == 0) {
        lval[lo] = lh;
        lval[hi] = ll;
        if (n_swap) n_swap[(int64_t)lad * (R - 1) + r] += 1;
      }
    }
    __syncwarp();
  }
  if (record >= 0) {
    const int8_t* src = sigma + base * n;
    int8_t* dst = samples + ((int64_t)lad * n_samples + record) * n;
    for (int i = lane; i < n; i += 32) dst[i] = src[i];
  }
}

size_t align256(size_t b) { return (b + 255) / 256 * 256; }

}  // namespace

size_t pt_scratch_bytes(int n, int m, int cplx, int move, int nb, int nc) {
  return align256(metropolis_scratch_bytes(n, m, cplx, move, nb)) +
         align256((size_t)std::max(nc, 1) * sizeof(double));
}

nk_status run_pt_sweep(const nk_rbm* r, nk_chains* ch, int R, int move, const int32_t* bi,
                       const int32_t* bk, int nb, int n_discard, int n_samples, int8_t* samples,
                       uint64_t* n_acc, uint64_t* n_swap, void* scratch, size_t scratch_bytes,
                       cudaStream_t st, bool dry) {
  const size_t mbytes = align256(metropolis_scratch_bytes(r->n, r->m, r->is_complex, move, nb));
  const size_t need = pt_scratch_bytes(r->n, r->m, r->is_complex, move, nb, ch->nc);
  if (!scratch || scratch_bytes < need)
    return fail(NK_ERR_SHAPE, "nk_pt_sweep: scratch of %zu B, need %zu B", scratch_bytes, need);
  double* lval = reinterpret_cast<double*>((char*)scratch + mbytes);
  MetroPt pt;
  pt.R = R;
  pt.lval = lval;
  pt.acc_add = 1;
  // every argument and shape check of the Metropolis launch, nothing enqueued
  if (nk_status e = launch_metropolis(r, ch, move, bi, bk, nb, 1, 0, nullptr, n_acc, scratch,
                                      mbytes, st, true, &pt))
    return e;
  if (dry) return NK_OK;
  const int nlad = ch->nc / R;
  if (n_acc && cudaMemsetAsync(n_acc, 0, (size_t)ch->nc * sizeof(uint64_t), st) != cudaSuccess)
    return fail(NK_ERR_CUDA, "nk_pt_sweep: cudaMemsetAsync failed");
  if (n_swap && R > 1 &&
      cudaMemsetAsync(n_swap, 0, (size_t)nlad * (R - 1) * sizeof(uint64_t), st) != cudaSuccess)
    return fail(NK_ERR_CUDA, "nk_pt_sweep: cudaMemsetAsync failed");
  const int sweeps = n_discard + n_samples;
  const unsigned blocks = (unsigned)((nlad + kPtWarps - 1) / kPtWarps);
  for (int k = 0; k < sweeps; ++k) {
    pt.skip_tables = k > 0;
    nk_status e = launch_metropolis(r, ch, move, bi, bk, nb, 1, 0, nullptr, n_acc, scratch,
                                    mbytes, st, false, &pt);
    if (e) return e;
    ch->counter += (uint64_t)r->n;  // the host counter (the device one advanced itself)
    pt_exchange_kernel<<<blocks, 32 * kPtWarps, 0, st>>>(
        ch->sigma, lval, r->n, nlad, R, ch->seed, ch->counter_dev, ch->counter, samples,
        n_samples, k >= n_discard ? k - n_discard : -1, n_swap);
    if ((e = check_launch("nk_pt_sweep(exchange)"))) return e;
  }
  return NK_OK;
}

}  // namespace nk
