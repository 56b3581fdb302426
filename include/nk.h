/*
 * nk.h -- C ABI of the GB300 (sm_103a) RBM variational Monte Carlo + stochastic
 * reconfiguration hot path, after NetKet (Carleo et al., arXiv:1904.00031).
 *
 * Conventions (apply to every entry point unless stated otherwise)
 * ---------------------------------------------------------------
 * - Pointers are DEVICE pointers, allocated and owned by the caller.  The
 *   library never allocates or frees device memory and never synchronises the
 *   stream inside a call (nk_operator_upload and nk_symm_upload are the
 *   exceptions and say so).
 * - Calls are asynchronous on `stream` (a cudaStream_t; NULL = legacy default
 *   stream).  Argument errors are detected on the host and returned
 *   synchronously, with nothing enqueued.  A kernel launch failure returns
 *   NK_ERR_CUDA.  nk_last_error() gives a message for the calling thread.
 * - Spin configurations sigma in {+1,-1}^N are int8, row-major [rows][n].
 *   +1 is spin up.  The local basis index of a spin is idx(+1)=0, idx(-1)=1.
 * - Complex numbers are interleaved (re, im): "c128" = 2 doubles, "c64" = 2
 *   floats.  "F32" below means float for a real RBM and c64 for a complex one;
 *   "F64" means double / c128 likewise.
 * - RBM (Sec. 2.2.2, RbmSpin): ln psi(sigma) = sum_i a_i sigma_i
 *   + sum_j ln cosh(theta_j), theta = W sigma + b, W row-major [m][n].  No
 *   constant M ln 2 is added.
 * - Parameter vectors (gradients, SR directions) are ordered (a, b, W
 *   row-major), length P = n + m + n*m, F64.
 */
#ifndef NK_H
#define NK_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t nk_status;
#define NK_OK 0
#define NK_ERR_INVALID_ARG 1   /* NULL pointer, negative size, unknown enum   */
#define NK_ERR_SHAPE 2         /* sizes outside the supported range            */
#define NK_ERR_CUDA 3          /* a CUDA runtime call or launch failed         */
#define NK_ERR_NOT_CONVERGED 4 /* (info flag) CG stopped at n_cg above cg_rtol */
#define NK_ERR_NONFINITE 5     /* (info flag) NaN/Inf met in E_loc or CG       */
#define NK_ERR_TIMEOUT 6       /* a bounded device-side wait gave up           */
#define NK_ERR_UNSUPPORTED 7   /* valid request this library does not implement */

/* Arithmetic of the dense contractions (theta GEMM, SR matvec, backward). */
#define NK_PREC_FP32 0   /* FP32 FMA on the CUDA cores ("plain FP32 path")          */
#define NK_PREC_BF16X2 1 /* tensor cores (tcgen05), operand split into BF16 hi + lo,
                            sigma exact in BF16, FP32 accumulation in TMEM        */

#define NK_MOVE_FLIP 0     /* single-spin flip at a uniformly random site          */
#define NK_MOVE_EXCHANGE 1 /* swap of the two spins of a uniformly random bond     */

#define NK_LAYOUT_FACTORED 0 /* O as T = tanh(theta) F32 [ns][m]; O_a = sigma,
                                O_W = T (x) sigma are implied                       */
#define NK_LAYOUT_DENSE 1    /* O as F32 [ns][P]                                    */

/* Size limits of this library. */
#define NK_MAX_N 4096      /* sites                                               */
#define NK_MAX_M 8192      /* hidden units (kernels hold tanh(theta) in registers) */
#define NK_MAX_GROUP 32    /* chains sharing one proposal stream (one CTA)         */

/* An RBM: FP64 master parameters plus the FP32 planes derived from them. */
typedef struct nk_rbm {
  int32_t n;          /* visible units (sites), 1..NK_MAX_N                         */
  int32_t m;          /* hidden units, 1..NK_MAX_M                                  */
  int32_t is_complex; /* 0: parameters in R, 1: in C                                */
  int32_t sr_splits;  /* split-K count of the adjoint contraction of nk_sr_step and
                         nk_rbm_logpsi_backward; 0 = built-in heuristic.  Set by
                         nk_sr_tune (or by hand); clamped to the scratch capacity */
  int32_t eloc_segs;  /* nk_local_energy: CTAs per configuration tile, each taking a
                         share of the move tiles (1 or 2); 0 = built-in heuristic.
                         Set by nk_tune_shapes (or by hand)                       */
  int32_t theta_segs; /* tensor-core ln psi / theta: CTAs per sample tile, each
                         taking a share of the hidden tiles (1 or 2); 0 = built-in
                         heuristic.  Set by nk_tune_shapes (or by hand)           */
  int32_t sampler;    /* nk_metropolis_sweep kernel: 0 = built-in choice; 1 = one
                         or two warps per chain; 2, 3, 4 = one CTA per proposal
                         group (complex RBMs, group_size <= 8, m <= 1024, 2048,
                         2304) with k - 1 hidden-unit pairs per thread, k this
                         value.  Built-in: 2 for complex RBMs with m <= 256 and
                         group_size <= 8, 4 for m > 2048, else 1             */
  double* a;          /* F64 [n]    (device)                                        */
  double* b;          /* F64 [m]    (device)                                        */
  double* w;          /* F64 [m][n] (device, row-major)                             */
  void* ws;           /* derived planes, nk_rbm_workspace_bytes() bytes, 256-B
                         aligned (device); filled by nk_rbm_prepare              */
  size_t ws_bytes;
} nk_rbm;

/* Persistent Markov chains. */
typedef struct nk_chains {
  int32_t nc;         /* number of chains                                           */
  int32_t group_size; /* chains per proposal group, 1..NK_MAX_GROUP                 */
  int8_t* sigma;      /* int8 [nc][n] current states (device, updated in place)     */
  uint64_t seed;      /* Philox4x32-10 key                                          */
  uint64_t counter;   /* proposals made so far by each chain (host; advanced by
                         nk_metropolis_sweep)                                      */
  uint64_t* counter_dev; /* optional device copy of the counter: if not NULL the
                         sweep reads the counter from it and advances it on the
                         device, so that replays of a captured CUDA graph draw
                         fresh random numbers; `counter` is then not used       */
} nk_chains;

/* A Hamiltonian as 1-local site terms and 2-local bond terms (GraphOperator,
 * Sec. 2.2.1).  HOST memory.  Site term t acts on site_idx[t] with the 2x2 c128
 * matrix site_mat[t][idx(s)][idx(s')] = <s|O|s'>; bond term t acts on
 * (bond_i[t], bond_k[t]) with the 4x4 c128 matrix bond_mat[t][r][c], r,c =
 * 2*idx(s_i) + idx(s_k). */
typedef struct nk_operator {
  int32_t n;
  int32_t n_site_terms;
  const int32_t* site_idx; /* [n_site_terms]          */
  const double* site_mat;  /* [n_site_terms][2][2][2] */
  int32_t n_bond_terms;
  int32_t reserved;
  const int32_t* bond_i;   /* [n_bond_terms]          */
  const int32_t* bond_k;   /* [n_bond_terms]          */
  const double* bond_mat;  /* [n_bond_terms][4][4][2] */
} nk_operator;

/* Layout of the nk_sr_step info block (device, NK_INFO_LEN doubles). */
#define NK_INFO_E_RE 0     /* Re <E_loc>                                     */
#define NK_INFO_E_IM 1     /* Im <E_loc>                                     */
#define NK_INFO_VAR 2      /* <|E_loc - <E_loc>|^2>                          */
#define NK_INFO_ERR 3      /* error bar from block means (0 with weights)    */
#define NK_INFO_CG_ITERS 4 /* CG iterations run                              */
#define NK_INFO_CG_RESID 5 /* final ||r|| / ||F||                            */
#define NK_INFO_F_NORM 6   /* ||F||                                          */
#define NK_INFO_FLAGS 7    /* bit (1<<NK_ERR_NOT_CONVERGED), (1<<NK_ERR_NONFINITE) */
#define NK_INFO_LEN 8

/* ---------------------------------------------------------------- library */

/* Human-readable name of a status code (static string). */
const char* nk_status_string(nk_status s);
/* Message describing the last error returned to the calling thread. */
const char* nk_last_error(void);
/* 1 if the library was compiled for sm_103a and a device of that kind is
 * current; 0 otherwise (no error is raised). */
int32_t nk_device_supported(void);

/* Device-side status (the paper has no counterpart: failure reporting of this
 * library).  Every wait of a kernel on an mbarrier (a bulk copy or a producer /
 * consumer hand-off) gives up after a bounded number of polls; the kernel then
 * finishes without hanging, marks its own outputs (NaN ln psi / E_loc / SR info,
 * UINT64_MAX accept counts) and sets bit (1 << NK_ERR_TIMEOUT) in a device
 * status word.  nk_query_status enqueues on `stream`: *flags (device int32,
 * caller-owned) = OR of the status bits set since the previous query, and
 * clears them.  Read *flags after the stream has passed the call.  Returns
 * NK_ERR_INVALID_ARG for a NULL flags pointer, NK_ERR_CUDA on a launch failure. */
nk_status nk_query_status(int32_t* flags, void* stream);

/* Measured ALU peaks of the current GPU (the paper has no counterpart: the
 * roofline denominators of the kernels bound by plain arithmetic).  HOST
 * out[4] = { packed FP32 FMA FLOP/s, MUFU ex2 op/s, MUFU lg2 op/s, MUFU sin
 * op/s }, each the best of 3 timed launches (8 CTAs of 256 threads per SM, 8
 * independent chains per thread).  Runs on its own stream and SYNCHRONISES it
 * (about 0.1 s).  NK_ERR_INVALID_ARG for NULL out, NK_ERR_CUDA on failure. */
nk_status nk_measure_alu_peaks(double* out);

/* Exercise the timeout path: one thread waits for an mbarrier phase that
 * nothing completes and gives up after `polls` polls (1 .. 2^20), setting
 * (1 << NK_ERR_TIMEOUT) in the status word read by nk_query_status.  For tests
 * of the failure reporting; it touches no caller memory. */
nk_status nk_debug_bounded_wait(uint32_t polls, void* stream);

/* ---------------------------------------------------------------- RBM */

/* Bytes of the derived-plane workspace of an (n, m, is_complex) RBM. */
size_t nk_rbm_workspace_bytes(int32_t n, int32_t m, int32_t is_complex);

/* Refresh the derived planes from the FP64 master (a, b, W): FP32 copies of
 * a, b and W^T, the tables cosh(2 W), sinh(2 W) used by the amplitude-ratio
 * kernels, and the BF16 hi/lo planes of the tensor-core path.  Must be called
 * after any change of the master parameters (nk_sr_step calls it itself). */
nk_status nk_rbm_prepare(const nk_rbm* rbm, void* stream);

/* ln psi(sigma) for ns configurations (Sec. 2.2.2).
 *   sigma      int8 [ns][n]
 *   prec       NK_PREC_FP32 or NK_PREC_BF16X2 (theta = W sigma + b contraction)
 *   logpsi_out c128 [ns], or NULL to compute theta only (no ln cosh; the local
 *              energies of a VMC iteration need theta, not ln psi)
 *   theta_out  F32 [ns][m] theta of every configuration, or NULL
 * At least one of logpsi_out and theta_out must be given.  ns = 0 is a no-op. */
nk_status nk_rbm_logpsi(const nk_rbm* rbm, const int8_t* sigma, int64_t ns, int32_t prec,
                        double* logpsi_out, void* theta_out, void* stream);

/* ---------------------------------------------------------------- sampling */

/* Scratch bytes nk_metropolis_sweep needs: one move row per site (flips) or
 * bond (exchanges), built at the start of every call: the move's table block,
 * its theta increments and a 16-byte header (a_i - a_k), sized for the larger
 * of the two sampler kernels' row layouts (nk_rbm.sampler).  Never 0. */
size_t nk_metropolis_scratch_bytes(int32_t n, int32_t m, int32_t is_complex, int32_t move,
                                   int32_t n_bonds);

/* Metropolis sampling of |psi|^2 (Eq. 4; Sec. 2.2.5), single-spin-flip or
 * nearest-neighbour exchange moves (the MetropolisExchange of the VMC listing,
 * Sec. 3.1).  Every chain runs n_discard + n_samples_per_chain sweeps of n
 * proposals and records its state after each of the last n_samples_per_chain
 * sweeps.  The proposal of step t for the chains of group g = c / group_size is
 * drawn from Philox4x32-10 stream (g, t, "SITE"); the accept uniform of chain c
 * from (c, t, "ACCP") (key = seed).  An exchange of two equal spins is a null
 * move and is rejected.  Accept iff U < exp(2 Re(ln psi' - ln psi)): the
 * log-ratio is formed in FP32 (per-unit factors, their running products and
 * logs) and compared with U in FP32, or in FP64 when the two are within 1e-5
 * (relative) of a tie; decisions agree with an FP64 evaluation except where
 * |ln U - 2 Re(ln psi' - ln psi)| is below the FP32 error of the log-ratio (none
 * of the decisions with a margin of 1e-4 or more differed in the parity tests,
 * up to m = 1600).  For complex RBMs a factor |r_j|^2 that rounds to zero or
 * below in FP32 makes the move's ratio zero (rejected).
 *   bond_i, bond_k  int32 [n_bonds] exchange bonds (ignored for FLIP; may be NULL)
 *   samples_out     int8 [nc * n_samples_per_chain][n], chain-major
 *                   (row c * n_samples_per_chain + s)
 *   n_accept_out    uint64 [nc] accepted proposals per chain in this call, or NULL.
 *                   UINT64_MAX marks a chain whose CTA gave up waiting for a
 *                   row copy (bounded wait; the call's results are then invalid)
 *   scratch         nk_metropolis_scratch_bytes(...) bytes, 256-B aligned
 *                   (move rows built at the start of the call); required
 * chains->sigma is updated in place and chains->counter advanced by
 * (n_discard + n_samples_per_chain) * n on success. */
nk_status nk_metropolis_sweep(const nk_rbm* rbm, nk_chains* chains, int32_t move,
                              const int32_t* bond_i, const int32_t* bond_k, int32_t n_bonds,
                              int32_t n_discard, int32_t n_samples_per_chain,
                              int8_t* samples_out, uint64_t* n_accept_out, void* scratch,
                              size_t scratch_bytes, void* stream);

/* Scratch bytes nk_pt_sweep needs: the move tables of nk_metropolis_sweep and
 * one double per replica (nc = chains->nc counts replicas). */
size_t nk_pt_scratch_bytes(int32_t n, int32_t m, int32_t is_complex, int32_t move,
                           int32_t n_bonds, int32_t nc);

/* Parallel tempering (replica exchange; the sampler option of Sec. 2.2.5).
 * chains holds nc = n_ladders * n_replicas replicas, chain-major: replica
 * c * R + r (R = n_replicas) of ladder c samples |psi|^(2 beta_r) with
 * beta_r = 1 - r / R, by the Metropolis sweep of nk_metropolis_sweep (its
 * proposal group and Philox streams indexed by replica number) with the accept
 * test U < exp(beta_r 2 Re(ln psi' - ln psi)).  After every sweep, neighbouring
 * replicas (r, r + 1), over the pairs starting at r = 0 when the sweep number
 * is even and at r = 1 when it is odd, exchange states iff
 * U < exp((beta_r - beta_(r+1)) (L_(r+1) - L_r)), L = 2 Re ln psi (decided in
 * FP64 from L formed at the end of the sweep: FP32 ln cosh per unit, summed in
 * FP64), U from Philox stream (c * R + r, sweep, "SWAP").  The sweep number is
 * floor(counter / n) with counter the chains' proposal counter before that
 * sweep.  After each of the last n_samples_per_chain sweeps the beta = 1
 * replica of every ladder is recorded.  R = 1 is nk_metropolis_sweep.
 *   samples_out   int8 [n_ladders * n_samples_per_chain][n], ladder-major
 *   n_accept_out  uint64 [nc] accepted proposals per replica in this call, or NULL
 *   n_swap_out    uint64 [n_ladders][R - 1] accepted exchanges per pair in this
 *                 call, or NULL
 *   scratch       nk_pt_scratch_bytes(n, m, is_complex, move, n_bonds, nc) bytes,
 *                 256-B aligned
 * Two launches per sweep (the sweep, the exchanges).  chains->sigma holds the
 * replicas' states after the call; chains->counter advances by
 * (n_discard + n_samples_per_chain) * n. */
nk_status nk_pt_sweep(const nk_rbm* rbm, nk_chains* chains, int32_t n_replicas, int32_t move,
                      const int32_t* bond_i, const int32_t* bond_k, int32_t n_bonds,
                      int32_t n_discard, int32_t n_samples_per_chain, int8_t* samples_out,
                      uint64_t* n_accept_out, uint64_t* n_swap_out, void* scratch,
                      size_t scratch_bytes, void* stream);

/* ---------------------------------------------------------------- operators */

/* Bytes of the compiled device form of a host operator description. */
size_t nk_operator_bytes(const nk_operator* op);
/* Compile the operator (merge terms into diagonal tables and a list of
 * distinct one- and two-spin moves with sigma-dependent matrix elements) and
 * copy it to `dev` (nk_operator_bytes(op) bytes).  Unlike the other calls this
 * one SYNCHRONISES `stream` before returning (it stages through host memory). */
nk_status nk_operator_upload(const nk_operator* op, void* dev, size_t bytes, void* stream);

/* ---------------------------------------------------------------- estimators */

/* Number of distinct moves (one- and two-spin flips with nonzero elements)
 * of the compiled operator; host only. */
int32_t nk_operator_moves(const nk_operator* op);

/* Scratch bytes nk_local_energy needs for an operator with n_moves moves. */
size_t nk_local_energy_scratch_bytes(int32_t m, int32_t is_complex, int32_t n_moves);

/* Local energies E_loc(sigma) = sum_sigma' <sigma|H|sigma'> psi(sigma')/psi(sigma)
 * (Eq. 5, Sec. 2.2.5), with every psi ratio from the exact theta update.
 *   op_dev   compiled operator (nk_operator_upload); n_moves = nk_operator_moves(op)
 *   sigma    int8 [ns][n];   theta F32 [ns][m] (from nk_rbm_logpsi)
 *   eloc_out c128 [ns]
 *   t_out    F32 [ns][m] tanh(theta) (the factored log-derivatives), or NULL
 *   scratch  nk_local_energy_scratch_bytes(m, is_complex, n_moves) bytes, 256-B
 *            aligned (built by the call: the per-move ratio tables, and per move and
 *            spin pattern the FP64 factor mel x exp(-2 s_i a_i - 2 s_k a_k)) */
nk_status nk_local_energy(const nk_rbm* rbm, const void* op_dev, int32_t n_moves,
                          const int8_t* sigma, const void* theta, int64_t ns, double* eloc_out,
                          void* t_out, void* scratch, size_t scratch_bytes, void* stream);

/* Log-derivatives O_k = d ln psi / d alpha_k (Sec. 2.2.5, analytic for the RBM):
 * O_a = sigma, O_b = tanh(theta), O_W = tanh(theta) (x) sigma.
 *   layout NK_LAYOUT_FACTORED: o_out = T F32 [ns][m]
 *          NK_LAYOUT_DENSE:    o_out = O F32 [ns][P] */
nk_status nk_logderiv(const nk_rbm* rbm, const int8_t* sigma, const void* theta, int64_t ns,
                      int32_t layout, void* o_out, void* stream);

/* ---------------------------------------------------------------- SR */

/* Scratch bytes nk_sr_step / nk_rbm_logpsi_backward need for ns samples. */
size_t nk_sr_scratch_bytes(int32_t n, int32_t m, int32_t is_complex, int64_t ns);

/* One stochastic-reconfiguration step (Sec. 2.2.5; SGD rule Eq. 2):
 *   <X> = sum_s w_s X_s, w = weights (double [ns]) or 1/ns when NULL,
 *   F = <O^* E_loc> - <O^*><E_loc>,
 *   (S + diag_shift I) delta = F with S x = <O^* (O x)> - <O^*>(<O> x), S never
 *   formed: conjugate gradient from x0 = 0, n_cg iterations unless
 *   ||r|| <= cg_rtol ||F|| first (decided on the device, no host sync),
 *   then alpha <- alpha - lr delta in the FP64 master and nk_rbm_prepare.
 * Real RBMs use Re S and Re F.  n_chains (>= 0, dividing ns) is the number of
 * equal blocks of consecutive samples that are independent of one another, for
 * the error bar NK_INFO_ERR (from the block means): with chain-major samples,
 * the number of proposal groups (nk_chains.nc / nk_chains.group_size), since the
 * chains of one group share their proposals; 0 or 1 gives no error bar.  CG
 * vectors and all reductions are FP64; the O and O^H contractions run at `prec`.
 *   t        F32 [ns][m] tanh(theta) (nk_local_energy t_out or nk_logderiv)
 *   eloc     c128 [ns]
 *   info_out double [NK_INFO_LEN] (device)
 *   scratch  nk_sr_scratch_bytes(n, m, is_complex, ns) bytes, 256-B aligned */
nk_status nk_sr_step(nk_rbm* rbm, const int8_t* sigma, const void* t, const double* eloc,
                     const double* weights, int64_t ns, int32_t n_chains, double diag_shift,
                     double lr, int32_t n_cg, double cg_rtol, int32_t prec, void* scratch,
                     size_t scratch_bytes, double* info_out, void* stream);

/* Size of the built-in scratch array used by nk_sr_step_noalloc (16 MiB). */
#define NK_SR_NOALLOC_MAX_BYTES (16u << 20)

/* nk_sr_step for callers that cannot allocate device memory (a framework that
 * owns the allocator and forbids raw cudaMalloc, a plugin handed only a stream
 * and its tensors, a loop that must not block on allocation).  The paper has
 * no counterpart: this is a deployment variant of the SR step above, with the
 * same arguments minus the scratch, and the same results.
 *   Scratch comes from one static device array of NK_SR_NOALLOC_MAX_BYTES in
 *   the library image, present on every GPU that loads the library until exit.
 *   Problems needing more (nk_sr_scratch_bytes(n, m, is_complex, ns) above the
 *   limit) return NK_ERR_SHAPE with nothing enqueued.
 *   The first call on a device looks up the array's device address
 *   (cudaGetSymbolAddress) with that device current; make it before any
 *   stream capture.  The address is cached per device ordinal for the primary
 *   context (the runtime's): after cudaDeviceReset, or from another context
 *   made current by the driver API, the cached address is stale; do not call
 *   this entry point there.  All calls share the array: calls that overlap on the GPU
 *   race and must be serialised by the caller.  No memory is allocated or
 *   freed. */
nk_status nk_sr_step_noalloc(nk_rbm* rbm, const int8_t* sigma, const void* t, const double* eloc,
                             const double* weights, int64_t ns, int32_t n_chains,
                             double diag_shift, double lr, int32_t n_cg, double cg_rtol,
                             int32_t prec, double* info_out, void* stream);

/* Autotuner of the SR contractions: times the adjoint contraction (the O^H
 * half of every CG iteration) for a few split-K counts on the given samples
 * and stores the fastest in rbm->sr_splits.  Arguments as for nk_sr_step.
 * Unlike the other calls this one SYNCHRONISES `stream` (it measures with
 * CUDA events) and must not be called while a stream is being captured. */
nk_status nk_sr_tune(nk_rbm* rbm, const int8_t* sigma, const void* t, int64_t ns, int32_t prec,
                     void* scratch, size_t scratch_bytes, void* stream);

/* ------------------------------------------------------ supervised learning */

/* Scratch bytes nk_supervised_step needs for ns samples. */
size_t nk_supervised_scratch_bytes(int32_t n, int32_t m, int32_t is_complex, int64_t ns);

/* One step of supervised learning of a target wavefunction (Sec. 2.2.3): the
 * negative log overlap of Eq. 1, L = -log(|<tar|psi>|^2 / (<tar|tar><psi|psi>)),
 * estimated from samples sigma_s of |tar|^2 as L = -log(|<R>|^2 / <|R|^2>) with
 * R_s = psi(sigma_s) / tar(sigma_s) and <X> = sum_s w_s X_s / sum_s w_s; its
 * gradient 2 dL/d conj(alpha) = sum_s conj(O_sk) g_s with
 * g_s = 2 w_s (|R_s|^2 / <|R|^2> - conj(R_s) / conj(<R>)) / sum w (the analytic
 * log-derivatives O of Sec. 2.2.5; for real parameters its real part, which is
 * dL/dalpha); then, if `moments` is given, one AdaMax update (the optimiser
 * list of Sec. 2.2.3; Kingma and Ba, Algorithm 2) of the FP64 master and
 * nk_rbm_prepare.  AdaMax treats the real and imaginary parts of a complex
 * parameter as two real parameters, in the master layout a | b | W:
 *   m <- beta1 m + (1 - beta1) g, u <- max(beta2 u, |g|),
 *   x <- x - lr / (1 - beta1^step) m / u   (a component with u = 0 does not move).
 *   sigma       int8 [ns][n] samples of |tar|^2
 *   log_target  c128 [ns] ln tar(sigma_s) (any branch of the complex log)
 *   weights     F64 [ns] sample weights, or NULL (equal weights)
 *   prec        contraction precision of ln psi and of the gradient
 *   lr, beta1, beta2, step  AdaMax step size, moment decays, 1-based step count
 *   moments     F64 [2][Pr] (m then u), Pr = P (real) or 2 P (complex), zeroed
 *               by the caller before step 1; NULL: loss and gradient only
 *   grad_out    F64 [P] or c128 [P] gradient (a | b | W order), or NULL
 *   scratch     nk_supervised_scratch_bytes(n, m, is_complex, ns) bytes, 256-B
 *               aligned
 *   info_out    double [4] (device) or NULL: L, the overlap |<R>|^2 / <|R|^2>
 *               (= exp(-L)), the shift c of the ratios R = exp(ln psi - ln tar - c)
 *               (c = max Re, which keeps them finite; L and g do not depend on it),
 *               flags (bit 1 << NK_ERR_NONFINITE).
 * Reductions run in a fixed order: a step is bitwise reproducible. */
nk_status nk_supervised_step(nk_rbm* rbm, const int8_t* sigma, const double* log_target,
                             const double* weights, int64_t ns, int32_t prec, double lr,
                             double beta1, double beta2, int32_t step, double* moments,
                             double* grad_out, void* scratch, size_t scratch_bytes,
                             double* info_out, void* stream);

/* ----------------------------------------------- feed-forward ln cosh networks */

/* A multi-layer feed-forward network (Sec. 2.2.2, FFNN machines): dense layers
 * h_l = W_l x_(l-1) + b_l, each followed by the ln cosh activation
 * x_l = ln cosh(h_l), x_0 = sigma, and a sum output ln psi = sum_j x_(L, j).  The
 * one-layer network is the RBM without visible bias; deeper ones generalise
 * it.  Real or complex (holomorphic) parameters. */
typedef struct nk_ffnn {
  int32_t n_layers;       /* L, 1..8                                               */
  int32_t is_complex;
  const int32_t* widths;  /* HOST int32 [L + 1]: widths[0] = n (sites), widths[l] =
                             outputs of layer l (1..2^20)                          */
  double* params;         /* F64 (device) master parameters, layer by layer: W_l
                             row-major [w_l][w_(l-1)] then b_l [w_l]; complex
                             interleaved (re, im)                                  */
} nk_ffnn;

/* Scratch bytes nk_ffnn_logpsi / nk_ffnn_backward need for ns samples (the
 * pre-activations and activations of every layer, two backpropagation buffers
 * and the weight-gradient split partials); 0 for an invalid network. */
size_t nk_ffnn_scratch_bytes(const nk_ffnn* f, int64_t ns);

/* ln psi(sigma) of ns configurations: every dense layer a 64 x 64-tiled FP32
 * CUDA-core contraction reading the FP64 master parameters, ln cosh fused into
 * its epilogue, the output sum in FP64.
 *   sigma       int8 [ns][n];  logpsi_out  c128 [ns]
 *   scratch     nk_ffnn_scratch_bytes(f, ns) bytes, 256-B aligned */
nk_status nk_ffnn_logpsi(const nk_ffnn* f, const int8_t* sigma, int64_t ns, double* logpsi_out,
                         void* scratch, size_t scratch_bytes, void* stream);

/* Backward of ln psi: grad_k = sum_s conj(O_sk) g_s with O the holomorphic
 * log-derivatives (for real parameters sum_s O_sk Re g_s), by the chain rule
 * through the layers: e_L = conj(tanh h_L) g, e_(l-1) = conj(tanh h_(l-1))
 * (e_l conj(W_l)), grad W_l = e_l^T conj(x_(l-1)), grad b_l = sum_s e_l.  The
 * forward is recomputed into the scratch first; weight gradients are FP32
 * split partials summed in FP64 in a fixed order.
 *   g         c128 [ns];  grad_out  F64 [P] or c128 [P] in the parameter order */
nk_status nk_ffnn_backward(const nk_ffnn* f, const int8_t* sigma, int64_t ns, const double* g,
                           double* grad_out, void* scratch, size_t scratch_bytes, void* stream);

/* Autotuner of the tile shapes of the ln psi / theta contraction (tensor-core
 * path) and of the local energies: times each kernel with one and with two
 * CTAs per tile (the second CTA taking half of the hidden or move tiles; the
 * results agree to FP64 rounding of the two partial sums) on the given
 * samples and stores the faster counts in rbm->theta_segs and rbm->eloc_segs.
 * theta_tmp (F32 [ns][m]), eloc_tmp (c128 [ns]) and t_tmp (F32 [ns][m], or NULL;
 * given, the local energies are timed with their tanh(theta) output, as a VMC
 * iteration runs them) are overwritten; scratch as for nk_local_energy.  Unlike the other calls this one SYNCHRONISES `stream`
 * (it measures with CUDA events) and must not be called while a stream is
 * being captured.  (The paper has no counterpart: a tuning aid of this
 * library.) */
nk_status nk_tune_shapes(nk_rbm* rbm, const void* op_dev, int32_t n_moves, const int8_t* sigma,
                         int64_t ns, void* theta_tmp, double* eloc_tmp, void* t_tmp,
                         void* scratch, size_t scratch_bytes, void* stream);

/* ------------------------------------------- batches of independent instances */

/* Many independent RBMs (uneven n, m, field, sample counts) in one call each
 * for ln psi, sampling and local energies -- the multi-instance workload
 * (independent problems advanced together; the paper runs one problem per
 * process).  Each item holds the arguments of the single call; `stream` of an
 * item, if not NULL, overrides the call's stream (items on different streams
 * run concurrently, e.g. as parallel branches of a captured CUDA graph).
 * Every item passes all argument and shape checks of the single call before
 * anything is enqueued; on a failure the status names the first bad item (via
 * nk_last_error) and nothing is enqueued.  Results are identical to the single
 * calls.  Items with a stream of their own are launched per item, in item
 * order; all the others run fused on `stream`: one launch of each kernel for
 * every group of items that share its template (sampling: the move-row
 * builds of all items, one sweep launch per group of equal field, hidden units
 * per lane, warps per chain and group size -- for the one-CTA-per-group kernel
 * (nk_rbm.sampler) equal unit pairs per thread and block size -- one
 * device-counter launch; ln psi:
 * one launch per field; local energies: the move tables of all items, one
 * energy launch per field), each item running the arithmetic of its own call.
 * (With graph capture, the fused launches are single nodes.) */
typedef struct nk_logpsi_item {
  const nk_rbm* rbm;
  const int8_t* sigma;  /* int8 [ns][n] */
  int64_t ns;
  double* logpsi_out;   /* c128 [ns] */
  void* theta_out;      /* F32 [ns][m] or NULL */
  void* stream;
} nk_logpsi_item;
nk_status nk_batch_logpsi(const nk_logpsi_item* items, int32_t n_inst, int32_t prec,
                          void* stream);

typedef struct nk_sweep_item {
  const nk_rbm* rbm;
  nk_chains* chains;    /* counter advanced as by nk_metropolis_sweep */
  int32_t move;
  int32_t n_bonds;
  const int32_t* bond_i;
  const int32_t* bond_k;
  int32_t n_discard;
  int32_t n_samples_per_chain;
  int8_t* samples_out;
  uint64_t* n_accept_out;
  void* scratch;
  size_t scratch_bytes;
  void* stream;
} nk_sweep_item;
nk_status nk_batch_sweep(const nk_sweep_item* items, int32_t n_inst, void* stream);

typedef struct nk_eloc_item {
  const nk_rbm* rbm;
  const void* op_dev;   /* nk_operator_upload output */
  int32_t n_moves;
  int32_t reserved;
  const int8_t* sigma;
  const void* theta;
  int64_t ns;
  double* eloc_out;
  void* t_out;
  void* scratch;
  size_t scratch_bytes;
  void* stream;
} nk_eloc_item;
nk_status nk_batch_local_energy(const nk_eloc_item* items, int32_t n_inst, void* stream);

/* ---------------------------------------------------------------- SR batches */

/* One problem of an SR batch: the arguments nk_sr_step takes for one RBM.  The
 * RBMs of a batch are independent and may differ in n, m, field and ns. */
typedef struct nk_sr_batch_item {
  nk_rbm* rbm;            /* sr_splits > 0 fixes the problem's split-K count;
                             0 = a batch-wide default (about two waves of
                             adjoint CTAs over the whole batch)                  */
  const int8_t* sigma;    /* int8 [ns][n]                                      */
  const void* t;          /* F32 [ns][m] tanh(theta)                           */
  const double* eloc;     /* c128 [ns]                                         */
  const double* weights;  /* F64 [ns] or NULL (1/ns)                           */
  int64_t ns;
  int32_t n_chains;       /* blocks of the error bar, as for nk_sr_step        */
  int32_t reserved;       /* 0                                                 */
  void* scratch;          /* nk_sr_scratch_bytes(n, m, is_complex, ns) bytes,
                             256-B aligned (device), one per problem           */
  size_t scratch_bytes;
  double* info_out;       /* double [NK_INFO_LEN] (device)                     */
} nk_sr_batch_item;

/* Bytes of the descriptor array of a batch of n_inst problems. */
size_t nk_sr_batch_desc_bytes(int32_t n_inst);

/* Fill desc_host (nk_sr_batch_desc_bytes(n_inst) bytes of host memory) with the
 * device-side descriptors of the batch (every problem's sizes, device pointers
 * and tensor maps).  No CUDA work is enqueued; the caller copies the bytes into
 * device memory (256-B aligned) for nk_sr_step_batch, and describes the batch
 * again whenever an item's pointers, sizes or rbm->sr_splits change. */
nk_status nk_sr_batch_describe(const nk_sr_batch_item* items, int32_t n_inst, int32_t prec,
                               void* desc_host, size_t desc_bytes);

/* nk_sr_step (Sec. 2.2.5, Eq. 2) for every problem of a batch, with one launch
 * of each kernel per group of up to 64 problems (complex and real ones mixed)
 * instead of one launch per problem: many small RBMs fill the GPU together.
 * Each problem's arithmetic and reduction order are those of nk_sr_step with
 * the same split-K count, so the results are identical to n separate calls.
 * Tensor-core precision only (prec = NK_PREC_BF16X2; NK_ERR_UNSUPPORTED else).
 *   desc_dev  the bytes nk_sr_batch_describe wrote for these items, in device
 *             memory, 256-B aligned */
nk_status nk_sr_step_batch(const nk_sr_batch_item* items, int32_t n_inst,
                           const void* desc_dev, double diag_shift, double lr, int32_t n_cg,
                           double cg_rtol, int32_t prec, void* stream);

/* Scratch bytes nk_rbm_logpsi_backward needs for ns samples: one chunk of at
 * most 16384 samples (tanh(theta) of the chunk and the adjoint's buffers), so it
 * stops growing with ns beyond that. */
size_t nk_backward_scratch_bytes(int32_t n, int32_t m, int32_t is_complex, int64_t ns);

/* Backward of ln psi (the analytic derivatives of Sec. 2.2.5 contracted with
 * an upstream gradient): grad_k = sum_s conj(O_sk) g_s (PyTorch's convention
 * for a holomorphic function).  theta is recomputed from sigma chunk by chunk
 * (16384 samples at most), never stored for all ns: per chunk the theta
 * contraction writes tanh(theta) at `prec`, the adjoint contraction sums over
 * the chunk, and the chunk sums are added in FP64 in chunk order.
 *   g           c128 [ns]
 *   grad_out    F64 [P]
 *   scratch     nk_backward_scratch_bytes(n, m, is_complex, ns) bytes, 256-B
 *               aligned */
nk_status nk_rbm_logpsi_backward(const nk_rbm* rbm, const int8_t* sigma, int64_t ns,
                                 const double* g, double* grad_out, int32_t prec, void* scratch,
                                 size_t scratch_bytes, void* stream);

/* --------------------------------------------------- symmetric RBM (RbmSpinSymm) */
/* The RBM variant of Sec. 2.2.2 that carries lattice symmetries.  A group of
 * n_perm site permutations perm[g][i] (the image of site i under g) ties the
 * parameters: alpha feature families, one hidden unit (f, g) = f n_perm + g
 * per family and group element, with
 *   W[(f, g)][i] = Wt[f][perm[g][i]],  b[(f, g)] = bt[f],  a_i = at,
 * so psi(sigma o h) = psi(sigma) for every h of a group.  Amplitudes, sampling
 * and local energies run on the untied RBM this stands for (m = alpha n_perm,
 * written by nk_symm_expand); SR runs in the tied space (S_t = P^T S P,
 * F_t = P^T F, P the copy of a tied parameter into the untied ones it stands
 * for), with the untied contractions of nk_sr_step.  Tied parameter vectors
 * are ordered (at, bt, Wt row-major), length 1 + alpha + alpha n. */
typedef struct nk_rbm_symm {
  int32_t n;          /* sites                                                     */
  int32_t alpha;      /* feature families, >= 1                                    */
  int32_t n_perm;     /* permutations in the table, >= 1; alpha n_perm <= NK_MAX_M */
  int32_t is_complex;
  double* a;          /* F64 [1]          (device)                                 */
  double* b;          /* F64 [alpha]      (device)                                 */
  double* w;          /* F64 [alpha][n]   (device, row-major)                      */
  const void* tables; /* nk_symm_tables_bytes() bytes filled by nk_symm_upload     */
  size_t tables_bytes;
} nk_rbm_symm;

/* Bytes of the tie tables of a symmetric RBM (0 for sizes out of range). */
size_t nk_symm_tables_bytes(int32_t n, int32_t alpha, int32_t n_perm);

/* Builds the tie tables from the HOST permutation table perm [n_perm][n] into
 * HOST memory `host` (nk_symm_tables_bytes() bytes), for callers that stage the
 * copy themselves; no CUDA call.  Layout (int32, each section starting on a
 * 256-byte boundary, in this order), with m = alpha n_perm and the augmented
 * layouts of the SR vectors -- untied (m + 1) x (n + 1): W[j][i] at (j, i),
 * b_j at (j, n), a_i at (m, i); tied (alpha + 1) x (n + 1): Wt[f][i] at (f, i),
 * bt_f at (f, n), at at (alpha, 0):
 *   perm [n_perm][n]            the table as given
 *   tie  [(m + 1)(n + 1)]       untied element -> the tied element it copies, -1 for (m, n)
 *   off  [(alpha + 1)(n + 1) + 1], idx [(m + 1)(n + 1) - 1]
 *                               the untied elements of each tied one, ascending (CSR)
 * Errors as nk_symm_upload. */
nk_status nk_symm_build(const int32_t* perm, int32_t n, int32_t alpha, int32_t n_perm, void* host,
                        size_t bytes);

/* Builds the tie tables from the HOST permutation table perm [n_perm][n]
 * (each row a permutation of 0..n-1, else NK_ERR_INVALID_ARG) and copies them
 * into `dev` (device, 256-B aligned, nk_symm_tables_bytes() bytes).  Like
 * nk_operator_upload it synchronises `stream` before returning, so the host
 * table may be freed afterwards. */
nk_status nk_symm_upload(const int32_t* perm, int32_t n, int32_t alpha, int32_t n_perm,
                         void* dev, size_t bytes, void* stream);

/* Writes the untied parameters (a, b, W) of rbm from the tied ones and
 * prepares rbm's planes (nk_rbm_prepare).  rbm->n == s->n,
 * rbm->m == s->alpha * s->n_perm and the same is_complex, else NK_ERR_SHAPE. */
nk_status nk_symm_expand(const nk_rbm_symm* s, nk_rbm* rbm, void* stream);

/* Scratch bytes of nk_sr_step_symm. */
size_t nk_sr_symm_scratch_bytes(int32_t n, int32_t alpha, int32_t n_perm,
                                int32_t is_complex, int64_t ns);

/* One SR step of a symmetric RBM: the system (S_t + diag_shift I) delta = F_t
 * in the tied space by CG (every product S_t x expands x into the untied
 * layout, runs the untied O and O^H contractions of nk_sr_step at `prec`, and
 * folds the result back with fixed-order sums), then
 * theta_t <- theta_t - lr delta and nk_symm_expand into rbm.  sigma, t, eloc,
 * weights, info_out as for nk_sr_step, with t = tanh(theta) of the expanded
 * RBM; rbm must be s's expansion (nk_symm_expand).  Not available in batches. */
nk_status nk_sr_step_symm(nk_rbm_symm* s, nk_rbm* rbm, const int8_t* sigma, const void* t,
                          const double* eloc, const double* weights, int64_t ns,
                          int32_t n_chains, double diag_shift, double lr, int32_t n_cg,
                          double cg_rtol, int32_t prec, void* scratch, size_t scratch_bytes,
                          double* info_out, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* NK_H */
