// Tensor-core (tcgen05, BF16 hi + lo split, FP32 accumulation in TMEM)
// contractions of the RBM path.  Declarations shared by logpsi, SR and backward.
#pragma once

#include <cuda.h>

#include "common.cuh"
#include "internal.h"

namespace nk {

// Encode a 2-D BF16 tensor map (row-major [rows][cols], 128-byte swizzle,
// box = 64 columns x box_rows rows).  Returns false (and sets the error
// message) if the driver entry point is unavailable or rejects the map.
bool tc_make_map(CUtensorMap* map, const void* base, int64_t rows, int64_t cols,
                 int64_t row_stride_elems, int box_rows);

// Encode a 2-D FP32 tensor map without swizzle: row-major [rows][cols] with a
// row stride of stride_bytes, box = box_cols x box_rows.
bool make_map_f32(CUtensorMap* map, const void* base, int64_t rows, int64_t cols,
                  int64_t stride_bytes, int box_cols, int box_rows);

// Build B planes (see WsLayout) from an FP64 augmented matrix src [src_rows][ld]
// (double or interleaved complex), only columns < ncols used.
nk_status launch_bplanes_from_f64(const void* src, int src_rows, int ncols, int ld, int cplx,
                                  int mt, int na64, void* planes, const double* skip_flag,
                                  cudaStream_t st);
// Build the B planes of W | b from the master parameters.
nk_status launch_bplanes_from_rbm(const nk_rbm* r, cudaStream_t st);

// sigma' transposed, BF16 [na64][ns8]: sigma'[s][i] = sigma (i < n), 1 (i = n),
// 0 beyond; ns8 = ns rounded up to 8.
// sigma' rows as BF16 [ns][na64]: sigma_i (i < n), 1 (i = n), 0 beyond; the A
// operand of the SR forward, TMA-loaded per 128-sample tile.
nk_status launch_sigma_rows(const int8_t* sigma, int64_t ns, int n, int na64, void* out,
                            cudaStream_t st);
nk_status launch_sigma_t(const int8_t* sigma, int64_t ns, int n, int na64, void* out,
                         cudaStream_t st);

// Forward contraction with a fused epilogue, for 128 configurations per CTA:
//   U[s][j] = sum_i sigma'[s][i] X[j][i]  (X given as B planes)
// mode 0 (SR):     y_s = sum_j T'_sj U_sj,  T' = [T | 1]    -> y (F64 [ns])
// mode 1 (logpsi): ln psi_s = a . sigma_s + sum_j ln cosh U_sj -> logpsi (c128),
//                  theta_out[s][j] = U_sj (optional)
struct FwdTcArgs {
  const int8_t* sigma;
  int64_t ns;
  int n, m, cplx, mode, mt, na64, rows;  // rows = hidden rows of X (m or m + 1)
  const void* T;          // mode 0
  void* y;                // mode 0: F64 [ns]
  const double* a;        // mode 1: master a
  double* logpsi;         // mode 1 (may be null: no ln cosh, theta / tanh theta only)
  void* theta_out;        // mode 1 (may be null)
  void* t_out = nullptr;  // mode 1: tanh(theta) [ns][m] (may be null)
  const double* skip;     // if non-null and *skip != 0, the kernel returns at once
  int* err;               // set on a timed-out wait (may be null)
  int nseg = 1;           // set by launch_fwd_tc: 1, or 2 halves of the hidden tiles
  int nseg_req = 0;       // 1 or 2 to override the heuristic (mode 1), 0 = heuristic
  const void* sig_rows = nullptr;  // mode 0: sigma' as BF16 [ns][na64] (launch_sigma_rows);
                                   // the sample tiles are then TMA-loaded, else built
  // mode 0, optional: per-CTA partial sums of w_s y_s (the centring mean of the
  // SR forward) at mean_part[seg * tiles + tile] (Re) and mean_part[mean_stride +
  // same] (Im); w_s = weights[s], or 1 / ns when weights is NULL
  double* mean_part = nullptr;
  int64_t mean_stride = 0;
  const double* weights = nullptr;
};
nk_status launch_fwd_tc(const FwdTcArgs& A, const void* planes, cudaStream_t st);
// Many mode-1 (theta / ln psi) launches fused: one launch per field.
nk_status launch_fwd_tc_fused(const FwdTcArgs* args, const void* const* planes, int n,
                              cudaStream_t st);
// Hidden-tile halves (1 or 2) launch_fwd_tc uses for ns samples and mt hidden
// tiles: 2 when twice the CTAs fill their last wave better (ln psi, and the SR
// forward with TMA-loaded sigma' tiles).
int fwd_tc_nseg(int64_t ns, int mt, int mode, bool sig_tma);

// Adjoint contraction: part[z][j][i] = sum_{s in split z} conj(T'_sj) v_s sigma'_si
// (FP32 partials, complex interleaved for a complex RBM), j < m + 1, i < n + 1.
struct AdjTcArgs {
  const void* T;
  const void* v;          // F64 [ns]
  int64_t ns;
  int n, m, cplx, na64, splits;
  void* part;
  const double* skip;
  int* err;
  // optional, instead of v: v_s = w_s (y_s - mean) formed while loading, with
  // mean = the fixed-order sum of mean_parts partials at mean_part (Re) and
  // mean_part + mean_stride (Im), w_s = weights[s] or 1 / ns (the centring of
  // the SR forward's output, same formula and order as the centring kernel)
  const void* y = nullptr;
  const double* mean_part = nullptr;
  int64_t mean_stride = 0;
  int mean_parts = 0;
  const double* weights = nullptr;
};
nk_status launch_adj_tc(const AdjTcArgs& A, const void* sigma_t, cudaStream_t st);

int adj_tc_splits(int n, int m, int cplx, int64_t ns);
bool tc_supported_shape(int n, int m);

// ------------------------------------------------------------------ batches
// One SR problem of a batch advanced by nk_sr_step_batch: everything the
// batched kernels read, in device memory (blockIdx.z or blockIdx.y selects the
// problem); TMA reads the two tensor maps from here.
struct alignas(128) SrDesc {
  CUtensorMap fwd_map;    // B planes of the CG direction (xbf)
  CUtensorMap adj_map;    // sigma'^T (sigt)
  CUtensorMap sig_map;    // sigma' rows (sigr), the forward's A operand
  const double* done;     // scal + SC_DONE: the CG has converged
  int splits;
  int nb_pa, nb_ns;       // blocks of the CG vector kernels over parameters / samples
  int cplx;               // 1: complex RBM
  int fwd_nseg;           // hidden-tile halves of the forward (fwd_tc_nseg); 2: y zeroed first
  int ctr_parts;          // > 0: the forward writes that many centring partials (no
                          // separate partial pass); 0: center_partial computes them
  int n, m, n_chains, na64, mt1, mp, wmt, wna64;  // wmt, wna64: B planes of W | b
  int64_t ns, pa, corner, ns8;
  const int8_t* sigma;
  const void* T;
  const double* eloc;
  const double* weights;
  double* a;
  double* b;
  double* w;
  char* ws;
  size_t ws_a32, ws_b32, ws_wt, ws_tab, ws_xw, ws_wbf;
  char* x;
  char* r;
  char* p;
  char* ap;
  char* part;
  char* y;
  char* v;
  char* sigt;
  char* sigr;
  char* xbf;
  double* red;
  double* scal;
  double* info;
};

// Per-launch arguments of the batched tensor-core contractions, passed as
// kernel parameters (the kernels read their problem's fields from the constant
// bank, as the single-problem kernels do); up to kBatchMax problems per launch.
constexpr int kBatchMax = 64;
struct FwdBatch {
  FwdTcArgs a[kBatchMax];
  const CUtensorMap* map[kBatchMax];   // in the problem's SrDesc (global memory)
  const CUtensorMap* smap[kBatchMax];  // sigma' rows map, also in the SrDesc
  int tiles[kBatchMax];                // sample tiles (CTAs per hidden-tile half)
};
struct AdjBatch {
  AdjTcArgs a[kBatchMax];
  const CUtensorMap* map[kBatchMax];
  int64_t chunk[kBatchMax];
  int tiles[kBatchMax], splits[kBatchMax];
};

// Batched launches over G problems (complex and real ones branch on their
// field); the max_* arguments bound the grid, and every problem's CTAs beyond
// its own sizes return at once.
nk_status launch_fwd_tc_batch(const FwdBatch& P, int G, int max_tiles, int max_na64,
                              cudaStream_t st);
nk_status launch_adj_tc_batch(const AdjBatch& P, int G, int max_tiles, int max_splits,
                              int max_na64, cudaStream_t st);
nk_status launch_sigma_t_batch(const SrDesc* D, int G, int64_t max_ns8, int max_na64,
                               cudaStream_t st);
// B planes of the CG direction p (skipped once converged), or of W | b
nk_status launch_bplanes_p_batch(const SrDesc* D, int G, int64_t max_elems, cudaStream_t st);
nk_status launch_sigma_rows_batch(const SrDesc* D, int G, int64_t max_elems, cudaStream_t st);
nk_status launch_bplanes_rbm_batch(const SrDesc* D, int G, int64_t max_elems, cudaStream_t st);
// the derived planes of every problem's RBM (prepare.cu)
nk_status launch_prepare_batch(const SrDesc* D, int G, int64_t max_work, int64_t max_minb,
                               cudaStream_t st);

}  // namespace nk
