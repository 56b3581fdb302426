// Internal declarations shared by the nk library's translation units.
#pragma once

#include <vector>

#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "nk.h"

namespace nk {

// Record an error message for nk_last_error() and return `s`.
nk_status fail(nk_status s, const char* fmt, ...);
// NK_ERR_CUDA with the pending launch error, or NK_OK.
nk_status check_launch(const char* where);

nk_status launch_prepare(const nk_rbm* r, cudaStream_t st);

// Device status words (status.cuh): OR each translation unit's word into *out
// (device int32) and clear it.
nk_status collect_status_tc(int32_t* out, cudaStream_t st);
nk_status collect_status_metropolis(int32_t* out, cudaStream_t st);
nk_status collect_status_local_energy(int32_t* out, cudaStream_t st);
nk_status collect_status_api(int32_t* out, cudaStream_t st);

// FP32 FMA FLOP/s and MUFU ex2 / lg2 / sin op/s of the current GPU (host out[4]).
nk_status measure_alu_peaks(double* out, cudaStream_t st);

// theta = W sigma + b and ln psi; theta_out may be null.
// logpsi may be null (then only theta_out and / or t_out = tanh(theta) are written).
nk_status launch_logpsi_fp32(const nk_rbm* r, const int8_t* sigma, int64_t ns, double* logpsi,
                             void* theta_out, cudaStream_t st, void* t_out = nullptr);
nk_status launch_logpsi_bf16(const nk_rbm* r, const int8_t* sigma, int64_t ns, double* logpsi,
                             void* theta_out, cudaStream_t st, void* t_out = nullptr);
// The theta / ln psi calls of items[idx[0..n)] fused: one launch per field.
nk_status launch_logpsi_fp32_fused(const nk_logpsi_item* items, const int* idx, int n,
                                   cudaStream_t st);
nk_status launch_logpsi_bf16_fused(const nk_logpsi_item* items, const int* idx, int n,
                                   cudaStream_t st);

// Parallel-tempering options of a Metropolis launch: chain c is replica c % R of
// its ladder (beta = 1 - (c % R) / R); lval (if set) receives 2 Re ln psi of every
// chain's final state; acc_add adds to n_acc instead of overwriting it;
// skip_tables reuses the move tables an earlier launch of the same call built.
struct MetroPt {
  int R = 0;
  double* lval = nullptr;
  int acc_add = 0;
  int skip_tables = 0;
};
nk_status launch_metropolis(const nk_rbm* r, nk_chains* ch, int move, const int32_t* bi,
                            const int32_t* bk, int nb, int n_discard, int n_samples,
                            int8_t* samples, uint64_t* n_acc, void* scratch, size_t scratch_bytes,
                            cudaStream_t st, bool dry = false, const MetroPt* pt = nullptr);
size_t metropolis_scratch_bytes(int n, int m, int cplx, int move, int nb);
// The sweeps of items[idx[0..n)] fused into one table launch, one sweep launch per
// kernel template and one counter launch (items already checked).
nk_status launch_metropolis_fused(const nk_sweep_item* items, const int* idx, int n,
                                  cudaStream_t st);

nk_status launch_local_energy(const nk_rbm* r, const void* op_dev, int n_moves,
                              const int8_t* sigma, const void* theta, int64_t ns, double* eloc,
                              void* t_out, void* scratch, size_t scratch_bytes, cudaStream_t st);
size_t local_energy_scratch_bytes(int m, int cplx, int n_moves);
// The local energies of items[idx[0..n)] fused into one move-table launch and one
// energy launch per field (items already checked).
nk_status launch_local_energy_fused(const nk_eloc_item* items, const int* idx, int n,
                                    cudaStream_t st);
nk_status launch_logderiv(const nk_rbm* r, const int8_t* sigma, const void* theta, int64_t ns,
                          int layout, void* o_out, cudaStream_t st);

// ------------------------------------------------------------------ SR
// The SR algebra runs on "augmented" matrices: T' = [T | 1] (ns x (m+1)) and
// sigma' = [sigma | 1] (ns x (n+1)); a parameter-space vector is held as an
// (m+1) x (n+1) row-major array X' with X'[j][i] = x_W[j][i], X'[j][n] = x_b[j],
// X'[m][i] = x_a[i], X'[m][n] = 0.  Then O_s . x = sum_j T'_sj (X' sigma'_s)_j and
// sum_s conj(O_s) v_s = T'^H diag(v) sigma'.
struct SrLayout {
  int n, m, cplx;
  int64_t ns;
  int ma, na;        // m + 1, n + 1
  int64_t pa;        // ma * na
  int splits;        // split-K capacity of the partial buffer (2 x the heuristics)
  int splits_fp32, splits_tc;  // heuristic split-K counts
  int na64, mt1;      // tensor-core path: n + 1 padded to 64; tiles of the m + 1 rows
  int64_t ns8;        // ns rounded up to 8
  size_t x, r, p, ap, xf, part, y, v, red, scal, sigt, sigr, xbf, total;
  SrLayout(int n_, int m_, int cplx_, int64_t ns_);
};

size_t sr_scratch_bytes(int n, int m, int cplx, int64_t ns);
size_t backward_scratch_bytes(int n, int m, int cplx, int64_t ns);
nk_status run_sr_step(nk_rbm* r, const int8_t* sigma, const void* t, const double* eloc,
                      const double* weights, int64_t ns, int n_chains, double diag_shift,
                      double lr, int n_cg, double cg_rtol, int prec, void* scratch,
                      size_t scratch_bytes, double* info, cudaStream_t st);
int sr_choose_splits(const SrLayout& L, int prec, int requested);
// Symmetric RBM (tied parameters over a permutation group, nk_sr_step_symm).
// Tables in one device buffer: perm [n_perm][n], tie [pa] (untied augmented
// element -> tied element or -1), fold CSR off [pa_t + 1] / idx [pa - 1].
struct SymmTables {
  int n, alpha, n_perm;
  int64_t pa, pa_t;  // (m + 1)(n + 1) with m = alpha n_perm; (alpha + 1)(n + 1)
  size_t perm, tie, off, idx, total;
  SymmTables(int n_, int alpha_, int n_perm_);
};
nk_status symm_build_tables(const int32_t* perm, int n, int alpha, int n_perm,
                            std::vector<int32_t>* out);
size_t sr_symm_scratch_bytes(int n, int alpha, int n_perm, int cplx, int64_t ns);
nk_status run_symm_expand(const nk_rbm_symm* s, nk_rbm* r, cudaStream_t st);
nk_status run_sr_step_symm(nk_rbm_symm* s, nk_rbm* r, const int8_t* sigma, const void* t,
                           const double* eloc, const double* weights, int64_t ns,
                           int n_chains, double diag_shift, double lr, int n_cg,
                           double cg_rtol, int prec, void* scratch, size_t scratch_bytes,
                           double* info, cudaStream_t st);
nk_status run_sr_tune(nk_rbm* r, const int8_t* sigma, const void* t, int64_t ns, int prec,
                      void* scratch, size_t scratch_bytes, cudaStream_t st);
// SR batches (nk_sr_step_batch)
nk_status sr_batch_check(const nk_sr_batch_item* items, int n_inst, int prec);
size_t sr_batch_desc_bytes(int n_inst);
nk_status sr_batch_describe(const nk_sr_batch_item* items, int n_inst, int prec, void* host,
                            size_t bytes);
nk_status run_sr_step_batch(const nk_sr_batch_item* items, int n_inst, const void* desc_dev,
                            double eps, double lr, int n_cg, double rtol, int prec,
                            cudaStream_t st);
nk_status run_backward(const nk_rbm* r, const int8_t* sigma, int64_t ns, const double* g,
                       double* grad, int prec, void* scratch, size_t scratch_bytes,
                       cudaStream_t st);
// Parallel tempering (tempering.cu)
size_t pt_scratch_bytes(int n, int m, int cplx, int move, int nb, int nc);
nk_status run_pt_sweep(const nk_rbm* r, nk_chains* ch, int R, int move, const int32_t* bi,
                       const int32_t* bk, int nb, int n_discard, int n_samples, int8_t* samples,
                       uint64_t* n_acc, uint64_t* n_swap, void* scratch, size_t scratch_bytes,
                       cudaStream_t st, bool dry);
// Feed-forward ln cosh networks (ffnn.cu)
nk_status check_ffnn(const nk_ffnn* f, const char* who);
size_t ffnn_scratch_bytes(const nk_ffnn* f, int64_t ns);
nk_status run_ffnn_logpsi(const nk_ffnn* f, const int8_t* sigma, int64_t ns, double* logpsi,
                          void* scratch, size_t bytes, cudaStream_t st);
nk_status run_ffnn_backward(const nk_ffnn* f, const int8_t* sigma, int64_t ns, const double* g,
                            double* grad, void* scratch, size_t bytes, cudaStream_t st);
// Supervised learning (Eq. 1 loss, its gradient, AdaMax): supervised.cu
size_t supervised_scratch_bytes(int n, int m, int cplx, int64_t ns);
nk_status run_supervised_step(nk_rbm* r, const int8_t* sigma, const double* log_target,
                              const double* weights, int64_t ns, int prec, double lr,
                              double beta1, double beta2, int step, double* moments,
                              double* grad_out, void* scratch, size_t scratch_bytes,
                              double* info, cudaStream_t st);

}  // namespace nk
