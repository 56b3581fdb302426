// The C ABI (include/nk.h): argument validation, operator compilation and
// dispatch to the kernels.  No device memory is allocated here.
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <map>
#include <tuple>
#include <vector>

#include "common.cuh"
#include "internal.h"
#include "opdev.h"
#include "status.cuh"
#include "tc.cuh"
#include "tma.cuh"

namespace nk {

static thread_local char g_err[512] = "";

nk_status fail(nk_status s, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return s;
}

nk_status check_launch(const char* where) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(NK_ERR_CUDA, "%s: %s", where, cudaGetErrorString(e));
  return NK_OK;
}

static nk_status check_rbm(const nk_rbm* r, const char* who) {
  if (!r) return fail(NK_ERR_INVALID_ARG, "%s: rbm is NULL", who);
  if (r->n < 1 || r->n > NK_MAX_N || r->m < 1 || r->m > NK_MAX_M)
    return fail(NK_ERR_SHAPE, "%s: n = %d, m = %d outside [1, %d] x [1, %d]", who, r->n, r->m,
                NK_MAX_N, NK_MAX_M);
  if (r->is_complex != 0 && r->is_complex != 1)
    return fail(NK_ERR_INVALID_ARG, "%s: is_complex must be 0 or 1", who);
  if (!r->a || !r->b || !r->w || !r->ws)
    return fail(NK_ERR_INVALID_ARG, "%s: NULL parameter or workspace pointer", who);
  size_t need = WsLayout(r->n, r->m, r->is_complex).total;
  if (r->ws_bytes < need)
    return fail(NK_ERR_SHAPE, "%s: workspace of %zu B, need %zu B", who, r->ws_bytes, need);
  if (((uintptr_t)r->ws) & 255)
    return fail(NK_ERR_INVALID_ARG, "%s: workspace not 256-byte aligned", who);
  return NK_OK;
}

// ------------------------------------------------------------------ operator compilation

struct Compiled {
  std::vector<OpDSite> ds;
  std::vector<OpDBond> db;
  std::vector<OpMove> mv;
  int32_t flags = 0;  // OpDevHeader::flags
};

// Site-quad layout of the move list (kOpQuadMoves): the moves whose first spin
// is the same site are taken four at a time (a short last quad is completed by
// null moves of that site: all matrix elements zero), and within every tile of
// 64 moves, quad g of the tile occupies positions g, g + 16, g + 32, g + 48 --
// the four moves one thread of the local-energy tile evaluates, which then share
// the sign s_i of every configuration.  Used when it adds at most 1/16 null
// moves (e.g. a square lattice with nearest and next-nearest bonds: four moves
// per site); the move set and so the local energies are unchanged.
static bool quad_layout(std::vector<OpMove>& mv) {
  auto null_move = [](int site) {
    OpMove z;
    memset(&z, 0, sizeof(z));
    z.i = z.k = site;
    return z;
  };
  std::vector<OpMove> quads;  // 4 consecutive entries per quad
  size_t a = 0;
  while (a < mv.size()) {  // mv is ordered by first site
    size_t b = a;
    while (b < mv.size() && mv[b].i == mv[a].i) ++b;
    for (size_t c = a; c < b; c += 4)
      for (size_t u = 0; u < 4; ++u) quads.push_back(c + u < b ? mv[c + u] : null_move(mv[a].i));
    a = b;
  }
  const size_t nq = quads.size() / 4, nq16 = (nq + 15) / 16 * 16;
  if (mv.empty() || nq16 * 4 * 16 > mv.size() * 17) return false;
  for (size_t q = nq; q < nq16; ++q)
    for (int u = 0; u < 4; ++u) quads.push_back(null_move(0));
  std::vector<OpMove> out(nq16 * 4);
  for (size_t q = 0; q < nq16; ++q) {
    const size_t t = q / 16, g = q % 16;
    for (int u = 0; u < 4; ++u) out[64 * t + 16 * u + g] = quads[4 * q + u];
  }
  mv.swap(out);
  return true;
}

static bool nz(const double* c) { return c[0] != 0.0 || c[1] != 0.0; }

static nk_status compile_op(const nk_operator* op, Compiled& out) {
  if (!op) return fail(NK_ERR_INVALID_ARG, "operator is NULL");
  if (op->n < 1 || op->n > NK_MAX_N || op->n_site_terms < 0 || op->n_bond_terms < 0)
    return fail(NK_ERR_SHAPE, "operator: bad sizes");
  if ((op->n_site_terms && (!op->site_idx || !op->site_mat)) ||
      (op->n_bond_terms && (!op->bond_i || !op->bond_k || !op->bond_mat)))
    return fail(NK_ERR_INVALID_ARG, "operator: NULL table");
  // moves keyed by (i, k, two); mel indexed 2 idx(s_i) + idx(s_k)
  std::map<std::tuple<int, int, int>, OpMove> moves;
  auto add = [&](int i, int k, int two, int x, const double* v) {
    auto key = std::make_tuple(i, k, two);
    auto it = moves.find(key);
    if (it == moves.end()) {
      OpMove mvv;
      memset(&mvv, 0, sizeof(mvv));
      mvv.i = i;
      mvv.k = k;
      mvv.two = two;
      it = moves.emplace(key, mvv).first;
    }
    it->second.mel[x][0] += v[0];
    it->second.mel[x][1] += v[1];
  };
  for (int t = 0; t < op->n_site_terms; ++t) {
    int i = op->site_idx[t];
    if (i < 0 || i >= op->n) return fail(NK_ERR_SHAPE, "operator: site index %d out of range", i);
    const double* M = op->site_mat + 8 * t;  // [2][2][2]
    OpDSite d;
    memset(&d, 0, sizeof(d));
    d.i = i;
    for (int x = 0; x < 2; ++x) {
      d.d[x][0] = M[(x * 2 + x) * 2];
      d.d[x][1] = M[(x * 2 + x) * 2 + 1];
    }
    out.ds.push_back(d);
    // flip of site i: from idx 0 (up) -> element M[0][1]; from idx 1 -> M[1][0]
    if (nz(M + (0 * 2 + 1) * 2)) add(i, i, 0, 0, M + (0 * 2 + 1) * 2);
    if (nz(M + (1 * 2 + 0) * 2)) add(i, i, 0, 3, M + (1 * 2 + 0) * 2);
  }
  for (int t = 0; t < op->n_bond_terms; ++t) {
    int i = op->bond_i[t], k = op->bond_k[t];
    if (i < 0 || i >= op->n || k < 0 || k >= op->n || i == k)
      return fail(NK_ERR_SHAPE, "operator: bond (%d, %d) invalid", i, k);
    const double* M = op->bond_mat + 32 * t;  // [4][4][2]
    OpDBond d;
    memset(&d, 0, sizeof(d));
    d.i = i;
    d.k = k;
    for (int x = 0; x < 4; ++x) {
      d.d[x][0] = M[(x * 4 + x) * 2];
      d.d[x][1] = M[(x * 4 + x) * 2 + 1];
    }
    out.db.push_back(d);
    for (int row = 0; row < 4; ++row) {
      for (int col = 0; col < 4; ++col) {
        if (row == col) continue;
        const double* v = M + (row * 4 + col) * 2;
        if (!nz(v)) continue;
        int ri = row >> 1, rk = row & 1, ci = col >> 1, ck = col & 1;
        if (ri != ci && rk != ck) add(i, k, 1, row, v);
        else if (ri != ci) add(i, k, 0, 2 * ri + rk, v);      // flip i, context k
        else add(k, i, 0, 2 * rk + ri, v);                     // flip k, context i
      }
    }
  }
  for (auto& kv : moves) {
    const OpMove& m = kv.second;
    if (!m.two) {
      bool any = false;
      for (int x = 0; x < 4; ++x) any |= nz(m.mel[x]);
      if (any) out.mv.push_back(m);
      continue;
    }
    // split a two-spin move into its aligned (x = 0, 3) and anti-aligned
    // (x = 1, 2) parts: the ratio kernels use one (cosh c, sinh c) table per move
    for (int align = 1; align >= -1; align -= 2) {
      OpMove v = m;
      v.align = align;
      bool any = false;
      for (int x = 0; x < 4; ++x) {
        bool aligned = (x == 0 || x == 3);
        if (aligned != (align == 1)) v.mel[x][0] = v.mel[x][1] = 0.0;
        any |= nz(v.mel[x]);
      }
      if (any) out.mv.push_back(v);
    }
  }
  if (quad_layout(out.mv)) out.flags |= kOpQuadMoves;
  return NK_OK;
}

static size_t layout_sizes(const Compiled& c, int32_t* off_ds, int32_t* off_db, int32_t* off_mv) {
  size_t off = round_up(sizeof(OpDevHeader), 16);
  *off_ds = (int32_t)off;
  off += round_up(c.ds.size() * sizeof(OpDSite), 16);
  *off_db = (int32_t)off;
  off += round_up(c.db.size() * sizeof(OpDBond), 16);
  *off_mv = (int32_t)off;
  off += round_up(c.mv.size() * sizeof(OpMove), 16);
  return off;
}

// One thread waits for a phase of a fresh mbarrier that nothing completes,
// giving up after `polls` polls: exercises the timeout path of the bounded
// waits (the status bit and a context that stays usable) without a hang.
__global__ void bounded_wait_probe_kernel(uint32_t polls) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    mbar_fence_init();
    if (!mbar_wait_bounded(&bar, 0u, polls)) dev_status_set(1u << NK_ERR_TIMEOUT);
  }
}

NK_STATUS_COLLECTOR(collect_status_api)

}  // namespace nk

using namespace nk;

// Every item is checked (all argument and shape checks of the single call)
// before any is enqueued; then the items are launched in order, each on its own
// stream if it names one.
template <typename Item, typename Call>
static nk_status run_batch(const char* what, const Item* items, int32_t n_inst, void* stream,
                           Call call) {
  if (n_inst < 0 || (n_inst > 0 && !items))
    return fail(NK_ERR_INVALID_ARG, "%s: bad item array", what);
  char msg[512];
  for (int32_t k = 0; k < n_inst; ++k) {
    if (nk_status e = call(items[k], items[k].stream ? items[k].stream : stream, true)) {
      snprintf(msg, sizeof(msg), "%s", g_err);
      return fail(e, "%s item %d: %s", what, k, msg);
    }
  }
  for (int32_t k = 0; k < n_inst; ++k) {
    if (nk_status e = call(items[k], items[k].stream ? items[k].stream : stream, false)) {
      snprintf(msg, sizeof(msg), "%s", g_err);
      return fail(e, "%s item %d: %s", what, k, msg);
    }
  }
  return NK_OK;
}

// Mean time of `reps` launches of `fn` on `st` (CUDA events), after one warm-up launch.
template <typename Fn>
static nk_status time_launches(cudaStream_t st, int reps, Fn fn, float* ms) {
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    return fail(NK_ERR_CUDA, "nk_tune_shapes: cudaEventCreate failed");
  nk_status e = fn();
  if (!e && cudaEventRecord(e0, st) != cudaSuccess) e = fail(NK_ERR_CUDA, "event record failed");
  for (int k = 0; k < reps && !e; ++k) e = fn();
  if (!e && (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess))
    e = fail(NK_ERR_CUDA, "nk_tune_shapes: event synchronisation failed");
  float t = 0.f;
  if (!e) cudaEventElapsedTime(&t, e0, e1);
  *ms = t / (float)reps;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return e;
}

extern "C" {

const char* nk_status_string(nk_status s) {
  switch (s) {
    case NK_OK: return "ok";
    case NK_ERR_INVALID_ARG: return "invalid argument";
    case NK_ERR_SHAPE: return "unsupported shape";
    case NK_ERR_CUDA: return "CUDA error";
    case NK_ERR_NOT_CONVERGED: return "not converged";
    case NK_ERR_NONFINITE: return "non-finite value";
    case NK_ERR_TIMEOUT: return "device wait timed out";
    case NK_ERR_UNSUPPORTED: return "unsupported";
    default: return "unknown status";
  }
}

const char* nk_last_error(void) { return g_err; }

int32_t nk_device_supported(void) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  cudaDeviceProp p;
  if (cudaGetDeviceProperties(&p, dev) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return (p.major == 10 && p.minor == 3) ? 1 : 0;
}

size_t nk_rbm_workspace_bytes(int32_t n, int32_t m, int32_t is_complex) {
  if (n < 1 || m < 1) return 0;
  return WsLayout(n, m, is_complex ? 1 : 0).total;
}

nk_status nk_rbm_prepare(const nk_rbm* rbm, void* stream) {
  if (nk_status e = check_rbm(rbm, "nk_rbm_prepare")) return e;
  return launch_prepare(rbm, (cudaStream_t)stream);
}

static nk_status logpsi_call(const nk_rbm* rbm, const int8_t* sigma, int64_t ns, int32_t prec,
                             double* logpsi_out, void* theta_out, void* stream, bool dry) {
  if (nk_status e = check_rbm(rbm, "nk_rbm_logpsi")) return e;
  if (ns < 0) return fail(NK_ERR_INVALID_ARG, "nk_rbm_logpsi: ns < 0");
  if (prec != NK_PREC_FP32 && prec != NK_PREC_BF16X2)
    return fail(NK_ERR_INVALID_ARG, "nk_rbm_logpsi: unknown precision %d", prec);
  if (ns == 0) return NK_OK;
  if (!sigma || (!logpsi_out && !theta_out))
    return fail(NK_ERR_INVALID_ARG, "nk_rbm_logpsi: NULL pointer");
  if (prec == NK_PREC_BF16X2 && !tc_supported_shape(rbm->n, rbm->m))
    return fail(NK_ERR_UNSUPPORTED, "nk_rbm_logpsi: the tensor-core path supports n + 1 <= 448");
  if (dry) return NK_OK;
  if (prec == NK_PREC_FP32)
    return launch_logpsi_fp32(rbm, sigma, ns, logpsi_out, theta_out, (cudaStream_t)stream);
  return launch_logpsi_bf16(rbm, sigma, ns, logpsi_out, theta_out, (cudaStream_t)stream);
}

nk_status nk_rbm_logpsi(const nk_rbm* rbm, const int8_t* sigma, int64_t ns, int32_t prec,
                        double* logpsi_out, void* theta_out, void* stream) {
  return logpsi_call(rbm, sigma, ns, prec, logpsi_out, theta_out, stream, false);
}

size_t nk_metropolis_scratch_bytes(int32_t n, int32_t m, int32_t is_complex, int32_t move,
                                   int32_t n_bonds) {
  if (n < 1 || m < 1 || n_bonds < 0 || (move != NK_MOVE_EXCHANGE && move != NK_MOVE_FLIP))
    return 0;
  return metropolis_scratch_bytes(n, m, is_complex ? 1 : 0, move, n_bonds);
}

static nk_status sweep_call(const nk_rbm* rbm, nk_chains* chains, int32_t move,
                              const int32_t* bond_i, const int32_t* bond_k, int32_t n_bonds,
                              int32_t n_discard, int32_t n_samples_per_chain,
                              int8_t* samples_out, uint64_t* n_accept_out, void* scratch,
                              size_t scratch_bytes, void* stream, bool dry) {
  if (nk_status e = check_rbm(rbm, "nk_metropolis_sweep")) return e;
  if (!chains || !chains->sigma)
    return fail(NK_ERR_INVALID_ARG, "nk_metropolis_sweep: NULL chains");
  if (chains->nc < 0 || n_discard < 0 || n_samples_per_chain < 0)
    return fail(NK_ERR_INVALID_ARG, "nk_metropolis_sweep: negative size");
  if (chains->group_size < 1 || chains->group_size > NK_MAX_GROUP)
    return fail(NK_ERR_SHAPE, "nk_metropolis_sweep: group_size %d outside [1, %d]",
                chains->group_size, NK_MAX_GROUP);
  if (move != NK_MOVE_FLIP && move != NK_MOVE_EXCHANGE)
    return fail(NK_ERR_INVALID_ARG, "nk_metropolis_sweep: unknown move %d", move);
  if (move == NK_MOVE_EXCHANGE && (n_bonds < 1 || !bond_i || !bond_k))
    return fail(NK_ERR_INVALID_ARG, "nk_metropolis_sweep: exchange moves need a bond list");
  if (n_samples_per_chain > 0 && !samples_out)
    return fail(NK_ERR_INVALID_ARG, "nk_metropolis_sweep: NULL samples_out");
  if (scratch && (((uintptr_t)scratch) & 255))
    return fail(NK_ERR_INVALID_ARG, "nk_metropolis_sweep: scratch not 256-byte aligned");
  if (chains->nc == 0 || n_discard + n_samples_per_chain == 0) return NK_OK;
  nk_status e = launch_metropolis(rbm, chains, move, bond_i, bond_k, n_bonds, n_discard,
                                  n_samples_per_chain, samples_out, n_accept_out, scratch,
                                  scratch_bytes, (cudaStream_t)stream, dry);
  if (e == NK_OK && !dry) chains->counter += (uint64_t)(n_discard + n_samples_per_chain) * rbm->n;
  return e;
}

size_t nk_pt_scratch_bytes(int32_t n, int32_t m, int32_t is_complex, int32_t move,
                           int32_t n_bonds, int32_t nc) {
  if (n < 1 || m < 1 || nc < 0) return 0;
  return pt_scratch_bytes(n, m, is_complex ? 1 : 0, move, n_bonds, nc);
}

nk_status nk_pt_sweep(const nk_rbm* rbm, nk_chains* chains, int32_t n_replicas, int32_t move,
                      const int32_t* bond_i, const int32_t* bond_k, int32_t n_bonds,
                      int32_t n_discard, int32_t n_samples_per_chain, int8_t* samples_out,
                      uint64_t* n_accept_out, uint64_t* n_swap_out, void* scratch,
                      size_t scratch_bytes, void* stream) {
  if (nk_status e = check_rbm(rbm, "nk_pt_sweep")) return e;
  if (!chains || !chains->sigma) return fail(NK_ERR_INVALID_ARG, "nk_pt_sweep: NULL chains");
  if (n_replicas < 1) return fail(NK_ERR_INVALID_ARG, "nk_pt_sweep: n_replicas < 1");
  if (chains->nc < 0 || n_discard < 0 || n_samples_per_chain < 0)
    return fail(NK_ERR_INVALID_ARG, "nk_pt_sweep: negative size");
  if (chains->nc % n_replicas)
    return fail(NK_ERR_SHAPE, "nk_pt_sweep: nc = %d is not a multiple of n_replicas = %d",
                chains->nc, n_replicas);
  if (chains->group_size < 1 || chains->group_size > NK_MAX_GROUP)
    return fail(NK_ERR_SHAPE, "nk_pt_sweep: group_size %d outside [1, %d]", chains->group_size,
                NK_MAX_GROUP);
  if (move != NK_MOVE_FLIP && move != NK_MOVE_EXCHANGE)
    return fail(NK_ERR_INVALID_ARG, "nk_pt_sweep: unknown move %d", move);
  if (move == NK_MOVE_EXCHANGE && (n_bonds < 1 || !bond_i || !bond_k))
    return fail(NK_ERR_INVALID_ARG, "nk_pt_sweep: exchange moves need a bond list");
  if (n_samples_per_chain > 0 && !samples_out)
    return fail(NK_ERR_INVALID_ARG, "nk_pt_sweep: NULL samples_out");
  if (!scratch || (((uintptr_t)scratch) & 255))
    return fail(NK_ERR_INVALID_ARG, "nk_pt_sweep: scratch NULL or not 256-byte aligned");
  if (chains->nc == 0 || n_discard + n_samples_per_chain == 0) return NK_OK;
  if ((int64_t)(n_discard + n_samples_per_chain) * rbm->n > 0x7fffffff)
    return fail(NK_ERR_SHAPE, "nk_pt_sweep: too many proposals in one call");
  return run_pt_sweep(rbm, chains, n_replicas, move, bond_i, bond_k, n_bonds, n_discard,
                      n_samples_per_chain, samples_out, n_accept_out, n_swap_out, scratch,
                      scratch_bytes, (cudaStream_t)stream, false);
}

nk_status nk_metropolis_sweep(const nk_rbm* rbm, nk_chains* chains, int32_t move,
                              const int32_t* bond_i, const int32_t* bond_k, int32_t n_bonds,
                              int32_t n_discard, int32_t n_samples_per_chain,
                              int8_t* samples_out, uint64_t* n_accept_out, void* scratch,
                              size_t scratch_bytes, void* stream) {
  return sweep_call(rbm, chains, move, bond_i, bond_k, n_bonds, n_discard, n_samples_per_chain,
                    samples_out, n_accept_out, scratch, scratch_bytes, stream, false);
}

size_t nk_operator_bytes(const nk_operator* op) {
  Compiled c;
  if (compile_op(op, c) != NK_OK) return 0;
  int32_t a, b, d;
  return layout_sizes(c, &a, &b, &d);
}

nk_status nk_operator_upload(const nk_operator* op, void* dev, size_t bytes, void* stream) {
  Compiled c;
  if (nk_status e = compile_op(op, c)) return e;
  if (!dev) return fail(NK_ERR_INVALID_ARG, "nk_operator_upload: NULL destination");
  OpDevHeader h;
  memset(&h, 0, sizeof(h));
  h.n = op->n;
  h.n_dsite = (int32_t)c.ds.size();
  h.n_dbond = (int32_t)c.db.size();
  h.n_moves = (int32_t)c.mv.size();
  h.flags = c.flags;
  size_t total = layout_sizes(c, &h.off_dsite, &h.off_dbond, &h.off_moves);
  if (bytes < total)
    return fail(NK_ERR_SHAPE, "nk_operator_upload: %zu B given, %zu B needed", bytes, total);
  std::vector<char> buf(total, 0);
  memcpy(buf.data(), &h, sizeof(h));
  if (!c.ds.empty()) memcpy(buf.data() + h.off_dsite, c.ds.data(), c.ds.size() * sizeof(OpDSite));
  if (!c.db.empty()) memcpy(buf.data() + h.off_dbond, c.db.data(), c.db.size() * sizeof(OpDBond));
  if (!c.mv.empty()) memcpy(buf.data() + h.off_moves, c.mv.data(), c.mv.size() * sizeof(OpMove));
  cudaStream_t st = (cudaStream_t)stream;
  if (cudaMemcpyAsync(dev, buf.data(), total, cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return fail(NK_ERR_CUDA, "nk_operator_upload: %s", cudaGetErrorString(cudaGetLastError()));
  return NK_OK;
}

int32_t nk_operator_moves(const nk_operator* op) {
  Compiled c;
  if (compile_op(op, c) != NK_OK) return -1;
  return (int32_t)c.mv.size();
}

size_t nk_local_energy_scratch_bytes(int32_t m, int32_t is_complex, int32_t n_moves) {
  if (m < 1 || n_moves < 0) return 0;
  return local_energy_scratch_bytes(m, is_complex ? 1 : 0, n_moves);
}

static nk_status eloc_call(const nk_rbm* rbm, const void* op_dev, int32_t n_moves,
                          const int8_t* sigma, const void* theta, int64_t ns, double* eloc_out,
                          void* t_out, void* scratch, size_t scratch_bytes, void* stream,
                          bool dry) {
  if (nk_status e = check_rbm(rbm, "nk_local_energy")) return e;
  if (ns < 0 || n_moves < 0) return fail(NK_ERR_INVALID_ARG, "nk_local_energy: negative size");
  if (ns == 0) return NK_OK;
  if (!op_dev || !sigma || !theta || !eloc_out)
    return fail(NK_ERR_INVALID_ARG, "nk_local_energy: NULL pointer");
  if (scratch && (((uintptr_t)scratch) & 255))
    return fail(NK_ERR_INVALID_ARG, "nk_local_energy: scratch not 256-byte aligned");
  if (n_moves > 0) {
    const size_t need = local_energy_scratch_bytes(rbm->m, rbm->is_complex ? 1 : 0, n_moves);
    if (!scratch || scratch_bytes < need)
      return fail(NK_ERR_SHAPE, "nk_local_energy: scratch of %zu B, need %zu B", scratch_bytes,
                  need);
  }
  if (dry) return NK_OK;
  return launch_local_energy(rbm, op_dev, n_moves, sigma, theta, ns, eloc_out, t_out, scratch,
                             scratch_bytes, (cudaStream_t)stream);
}

nk_status nk_local_energy(const nk_rbm* rbm, const void* op_dev, int32_t n_moves,
                          const int8_t* sigma, const void* theta, int64_t ns, double* eloc_out,
                          void* t_out, void* scratch, size_t scratch_bytes, void* stream) {
  return eloc_call(rbm, op_dev, n_moves, sigma, theta, ns, eloc_out, t_out, scratch,
                   scratch_bytes, stream, false);
}

// ---------------------------------------------------------------- batches of instances

nk_status nk_batch_logpsi(const nk_logpsi_item* items, int32_t n_inst, int32_t prec,
                          void* stream) {
  auto call = [prec](const nk_logpsi_item& it, void* st, bool dry) {
    return logpsi_call(it.rbm, it.sigma, it.ns, prec, it.logpsi_out, it.theta_out, st, dry);
  };
  if (n_inst < 0 || (n_inst > 0 && !items))
    return fail(NK_ERR_INVALID_ARG, "nk_batch_logpsi: bad item array");
  char msg[512];
  for (int32_t k = 0; k < n_inst; ++k) {
    if (nk_status e = call(items[k], items[k].stream ? items[k].stream : stream, true)) {
      snprintf(msg, sizeof(msg), "%s", g_err);
      return fail(e, "nk_batch_logpsi item %d: %s", k, msg);
    }
  }
  // items on their own streams: one call each; the others fused on `stream`
  std::vector<int> fused;
  for (int32_t k = 0; k < n_inst; ++k) {
    const nk_logpsi_item& it = items[k];
    if (it.stream) {
      if (nk_status e = call(it, it.stream, false)) {
        snprintf(msg, sizeof(msg), "%s", g_err);
        return fail(e, "nk_batch_logpsi item %d: %s", k, msg);
      }
    } else if (it.ns > 0) {
      fused.push_back(k);
    }
  }
  if (fused.empty()) return NK_OK;
  return prec == NK_PREC_FP32
             ? launch_logpsi_fp32_fused(items, fused.data(), (int)fused.size(),
                                        (cudaStream_t)stream)
             : launch_logpsi_bf16_fused(items, fused.data(), (int)fused.size(),
                                        (cudaStream_t)stream);
}

nk_status nk_batch_sweep(const nk_sweep_item* items, int32_t n_inst, void* stream) {
  auto call = [](const nk_sweep_item& it, void* st, bool dry) {
    return sweep_call(it.rbm, it.chains, it.move, it.bond_i, it.bond_k, it.n_bonds,
                      it.n_discard, it.n_samples_per_chain, it.samples_out, it.n_accept_out,
                      it.scratch, it.scratch_bytes, st, dry);
  };
  if (n_inst < 0 || (n_inst > 0 && !items))
    return fail(NK_ERR_INVALID_ARG, "nk_batch_sweep: bad item array");
  char msg[512];
  for (int32_t k = 0; k < n_inst; ++k) {
    if (nk_status e = call(items[k], items[k].stream ? items[k].stream : stream, true)) {
      snprintf(msg, sizeof(msg), "%s", g_err);
      return fail(e, "nk_batch_sweep item %d: %s", k, msg);
    }
  }
  // items on their own streams: one call each; the others fused on `stream`
  std::vector<int> fused;
  for (int32_t k = 0; k < n_inst; ++k) {
    const nk_sweep_item& it = items[k];
    if (it.stream) {
      if (nk_status e = call(it, it.stream, false)) {
        snprintf(msg, sizeof(msg), "%s", g_err);
        return fail(e, "nk_batch_sweep item %d: %s", k, msg);
      }
    } else if (it.chains->nc > 0 && it.n_discard + it.n_samples_per_chain > 0) {
      fused.push_back(k);
    }
  }
  if (!fused.empty()) {
    if (nk_status e = launch_metropolis_fused(items, fused.data(), (int)fused.size(),
                                              (cudaStream_t)stream))
      return e;
    for (int k : fused)
      items[k].chains->counter +=
          (uint64_t)(items[k].n_discard + items[k].n_samples_per_chain) * items[k].rbm->n;
  }
  return NK_OK;
}

nk_status nk_batch_local_energy(const nk_eloc_item* items, int32_t n_inst, void* stream) {
  auto call = [](const nk_eloc_item& it, void* st, bool dry) {
    return eloc_call(it.rbm, it.op_dev, it.n_moves, it.sigma, it.theta, it.ns, it.eloc_out,
                     it.t_out, it.scratch, it.scratch_bytes, st, dry);
  };
  if (n_inst < 0 || (n_inst > 0 && !items))
    return fail(NK_ERR_INVALID_ARG, "nk_batch_local_energy: bad item array");
  char msg[512];
  for (int32_t k = 0; k < n_inst; ++k) {
    if (nk_status e = call(items[k], items[k].stream ? items[k].stream : stream, true)) {
      snprintf(msg, sizeof(msg), "%s", g_err);
      return fail(e, "nk_batch_local_energy item %d: %s", k, msg);
    }
  }
  // items on their own streams: one call each; the others fused on `stream`
  std::vector<int> fused;
  for (int32_t k = 0; k < n_inst; ++k) {
    const nk_eloc_item& it = items[k];
    if (it.stream) {
      if (nk_status e = call(it, it.stream, false)) {
        snprintf(msg, sizeof(msg), "%s", g_err);
        return fail(e, "nk_batch_local_energy item %d: %s", k, msg);
      }
    } else if (it.ns > 0) {
      fused.push_back(k);
    }
  }
  if (!fused.empty())
    return launch_local_energy_fused(items, fused.data(), (int)fused.size(),
                                     (cudaStream_t)stream);
  return NK_OK;
}

nk_status nk_logderiv(const nk_rbm* rbm, const int8_t* sigma, const void* theta, int64_t ns,
                      int32_t layout, void* o_out, void* stream) {
  if (nk_status e = check_rbm(rbm, "nk_logderiv")) return e;
  if (ns < 0) return fail(NK_ERR_INVALID_ARG, "nk_logderiv: ns < 0");
  if (layout != NK_LAYOUT_FACTORED && layout != NK_LAYOUT_DENSE)
    return fail(NK_ERR_INVALID_ARG, "nk_logderiv: unknown layout %d", layout);
  if (ns == 0) return NK_OK;
  if (!sigma || !theta || !o_out) return fail(NK_ERR_INVALID_ARG, "nk_logderiv: NULL pointer");
  return launch_logderiv(rbm, sigma, theta, ns, layout, o_out, (cudaStream_t)stream);
}

size_t nk_sr_scratch_bytes(int32_t n, int32_t m, int32_t is_complex, int64_t ns) {
  if (n < 1 || m < 1 || ns < 0) return 0;
  return sr_scratch_bytes(n, m, is_complex ? 1 : 0, ns);
}

size_t nk_backward_scratch_bytes(int32_t n, int32_t m, int32_t is_complex, int64_t ns) {
  if (n < 1 || m < 1 || ns < 0) return 0;
  return backward_scratch_bytes(n, m, is_complex ? 1 : 0, ns);
}

nk_status nk_sr_step(nk_rbm* rbm, const int8_t* sigma, const void* t, const double* eloc,
                     const double* weights, int64_t ns, int32_t n_chains, double diag_shift,
                     double lr, int32_t n_cg, double cg_rtol, int32_t prec, void* scratch,
                     size_t scratch_bytes, double* info_out, void* stream) {
  if (nk_status e = check_rbm(rbm, "nk_sr_step")) return e;
  if (ns < 1) return fail(NK_ERR_INVALID_ARG, "nk_sr_step: ns < 1");
  if (!sigma || !t || !eloc || !scratch || !info_out)
    return fail(NK_ERR_INVALID_ARG, "nk_sr_step: NULL pointer");
  if (n_cg < 0 || !(diag_shift >= 0.0) || !(cg_rtol >= 0.0))
    return fail(NK_ERR_INVALID_ARG, "nk_sr_step: negative n_cg, diag_shift or cg_rtol");
  if (n_chains < 0 || (n_chains > 0 && ns % n_chains))
    return fail(NK_ERR_SHAPE, "nk_sr_step: ns = %lld not a multiple of n_chains = %d",
                (long long)ns, n_chains);
  if (((uintptr_t)scratch) & 255)
    return fail(NK_ERR_INVALID_ARG, "nk_sr_step: scratch not 256-byte aligned");
  if (prec != NK_PREC_FP32 && prec != NK_PREC_BF16X2)
    return fail(NK_ERR_INVALID_ARG, "nk_sr_step: unknown precision %d", prec);
  if (prec == NK_PREC_BF16X2 && !tc_supported_shape(rbm->n, rbm->m))
    return fail(NK_ERR_UNSUPPORTED, "nk_sr_step: the tensor-core path supports n + 1 <= 448");
  return run_sr_step(rbm, sigma, t, eloc, weights, ns, n_chains, diag_shift, lr, n_cg, cg_rtol,
                     prec, scratch, scratch_bytes, info_out, (cudaStream_t)stream);
}

nk_status nk_sr_tune(nk_rbm* rbm, const int8_t* sigma, const void* t, int64_t ns, int32_t prec,
                     void* scratch, size_t scratch_bytes, void* stream) {
  if (nk_status e = check_rbm(rbm, "nk_sr_tune")) return e;
  if (ns < 1 || !sigma || !t || !scratch)
    return fail(NK_ERR_INVALID_ARG, "nk_sr_tune: bad arguments");
  if (((uintptr_t)scratch) & 255)
    return fail(NK_ERR_INVALID_ARG, "nk_sr_tune: scratch not 256-byte aligned");
  if (prec != NK_PREC_FP32 && prec != NK_PREC_BF16X2)
    return fail(NK_ERR_INVALID_ARG, "nk_sr_tune: unknown precision %d", prec);
  if (prec == NK_PREC_BF16X2 && !tc_supported_shape(rbm->n, rbm->m))
    return fail(NK_ERR_UNSUPPORTED, "nk_sr_tune: the tensor-core path supports n + 1 <= 448");
  return run_sr_tune(rbm, sigma, t, ns, prec, scratch, scratch_bytes, (cudaStream_t)stream);
}

static bool symm_sizes_ok(int32_t n, int32_t alpha, int32_t n_perm) {
  return n >= 1 && n <= NK_MAX_N && alpha >= 1 && n_perm >= 1 &&
         (int64_t)alpha * n_perm <= NK_MAX_M;
}

static nk_status check_symm(const nk_rbm_symm* s, const nk_rbm* r, const char* who) {
  if (!s) return fail(NK_ERR_INVALID_ARG, "%s: symmetric RBM is NULL", who);
  if (!symm_sizes_ok(s->n, s->alpha, s->n_perm))
    return fail(NK_ERR_SHAPE, "%s: n = %d, alpha = %d, n_perm = %d out of range", who, s->n,
                s->alpha, s->n_perm);
  if (s->is_complex != 0 && s->is_complex != 1)
    return fail(NK_ERR_INVALID_ARG, "%s: is_complex must be 0 or 1", who);
  if (!s->a || !s->b || !s->w || !s->tables)
    return fail(NK_ERR_INVALID_ARG, "%s: NULL tied parameter or table pointer", who);
  if (((uintptr_t)s->tables) & 255)
    return fail(NK_ERR_INVALID_ARG, "%s: tables not 256-byte aligned", who);
  const size_t need = SymmTables(s->n, s->alpha, s->n_perm).total;
  if (s->tables_bytes < need)
    return fail(NK_ERR_SHAPE, "%s: tables of %zu B, need %zu B", who, s->tables_bytes, need);
  if (nk_status e = check_rbm(r, who)) return e;
  if (r->n != s->n || (int64_t)r->m != (int64_t)s->alpha * s->n_perm ||
      r->is_complex != s->is_complex)
    return fail(NK_ERR_SHAPE, "%s: rbm (n = %d, m = %d) is not the expansion of the symmetric "
                "RBM (n = %d, alpha n_perm = %d)", who, r->n, r->m, s->n, s->alpha * s->n_perm);
  return NK_OK;
}

size_t nk_symm_tables_bytes(int32_t n, int32_t alpha, int32_t n_perm) {
  if (!symm_sizes_ok(n, alpha, n_perm)) return 0;
  return SymmTables(n, alpha, n_perm).total;
}

nk_status nk_symm_build(const int32_t* perm, int32_t n, int32_t alpha, int32_t n_perm, void* host,
                        size_t bytes) {
  if (!perm || !host) return fail(NK_ERR_INVALID_ARG, "nk_symm_build: NULL pointer");
  if (!symm_sizes_ok(n, alpha, n_perm))
    return fail(NK_ERR_SHAPE, "nk_symm_build: n = %d, alpha = %d, n_perm = %d out of range", n,
                alpha, n_perm);
  const size_t need = SymmTables(n, alpha, n_perm).total;
  if (bytes < need)
    return fail(NK_ERR_SHAPE, "nk_symm_build: %zu B given, %zu B needed", bytes, need);
  std::vector<int32_t> buf;
  if (nk_status e = symm_build_tables(perm, n, alpha, n_perm, &buf)) return e;
  memcpy(host, buf.data(), need);
  return NK_OK;
}

nk_status nk_symm_upload(const int32_t* perm, int32_t n, int32_t alpha, int32_t n_perm,
                         void* dev, size_t bytes, void* stream) {
  if (!perm || !dev) return fail(NK_ERR_INVALID_ARG, "nk_symm_upload: NULL pointer");
  if (!symm_sizes_ok(n, alpha, n_perm))
    return fail(NK_ERR_SHAPE, "nk_symm_upload: n = %d, alpha = %d, n_perm = %d out of range", n,
                alpha, n_perm);
  if (((uintptr_t)dev) & 255)
    return fail(NK_ERR_INVALID_ARG, "nk_symm_upload: dev not 256-byte aligned");
  const size_t need = SymmTables(n, alpha, n_perm).total;
  if (bytes < need)
    return fail(NK_ERR_SHAPE, "nk_symm_upload: %zu B given, %zu B needed", bytes, need);
  std::vector<int32_t> buf;
  if (nk_status e = symm_build_tables(perm, n, alpha, n_perm, &buf)) return e;
  cudaStream_t st = (cudaStream_t)stream;
  if (cudaMemcpyAsync(dev, buf.data(), need, cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return fail(NK_ERR_CUDA, "nk_symm_upload: %s", cudaGetErrorString(cudaGetLastError()));
  return NK_OK;
}

nk_status nk_symm_expand(const nk_rbm_symm* s, nk_rbm* rbm, void* stream) {
  if (nk_status e = check_symm(s, rbm, "nk_symm_expand")) return e;
  return run_symm_expand(s, rbm, (cudaStream_t)stream);
}

size_t nk_sr_symm_scratch_bytes(int32_t n, int32_t alpha, int32_t n_perm, int32_t is_complex,
                                int64_t ns) {
  if (!symm_sizes_ok(n, alpha, n_perm) || ns < 0) return 0;
  return sr_symm_scratch_bytes(n, alpha, n_perm, is_complex ? 1 : 0, ns);
}

nk_status nk_sr_step_symm(nk_rbm_symm* s, nk_rbm* rbm, const int8_t* sigma, const void* t,
                          const double* eloc, const double* weights, int64_t ns,
                          int32_t n_chains, double diag_shift, double lr, int32_t n_cg,
                          double cg_rtol, int32_t prec, void* scratch, size_t scratch_bytes,
                          double* info_out, void* stream) {
  const char* who = "nk_sr_step_symm";
  if (nk_status e = check_symm(s, rbm, who)) return e;
  if (ns < 1) return fail(NK_ERR_INVALID_ARG, "%s: ns < 1", who);
  if (!sigma || !t || !eloc || !scratch || !info_out)
    return fail(NK_ERR_INVALID_ARG, "%s: NULL pointer", who);
  if (n_cg < 0 || !(diag_shift >= 0.0) || !(cg_rtol >= 0.0))
    return fail(NK_ERR_INVALID_ARG, "%s: negative n_cg, diag_shift or cg_rtol", who);
  if (n_chains < 0 || (n_chains > 0 && ns % n_chains))
    return fail(NK_ERR_SHAPE, "%s: ns = %lld not a multiple of n_chains = %d", who,
                (long long)ns, n_chains);
  if (((uintptr_t)scratch) & 255)
    return fail(NK_ERR_INVALID_ARG, "%s: scratch not 256-byte aligned", who);
  if (prec != NK_PREC_FP32 && prec != NK_PREC_BF16X2)
    return fail(NK_ERR_INVALID_ARG, "%s: unknown precision %d", who, prec);
  if (prec == NK_PREC_BF16X2 && !tc_supported_shape(rbm->n, rbm->m))
    return fail(NK_ERR_UNSUPPORTED, "%s: the tensor-core path supports n + 1 <= 448", who);
  return run_sr_step_symm(s, rbm, sigma, t, eloc, weights, ns, n_chains, diag_shift, lr, n_cg,
                          cg_rtol, prec, scratch, scratch_bytes, info_out, (cudaStream_t)stream);
}

size_t nk_sr_batch_desc_bytes(int32_t n_inst) { return sr_batch_desc_bytes(n_inst); }

nk_status nk_sr_batch_describe(const nk_sr_batch_item* items, int32_t n_inst, int32_t prec,
                               void* desc_host, size_t desc_bytes) {
  return sr_batch_describe(items, n_inst, prec, desc_host, desc_bytes);
}

nk_status nk_sr_step_batch(const nk_sr_batch_item* items, int32_t n_inst,
                           const void* desc_dev, double diag_shift, double lr, int32_t n_cg,
                           double cg_rtol, int32_t prec, void* stream) {
  if (n_cg < 0 || !(diag_shift >= 0.0) || !(cg_rtol >= 0.0))
    return fail(NK_ERR_INVALID_ARG, "nk_sr_step_batch: negative n_cg, diag_shift or cg_rtol");
  return run_sr_step_batch(items, n_inst, desc_dev, diag_shift, lr, n_cg, cg_rtol, prec,
                           (cudaStream_t)stream);
}

nk_status nk_rbm_logpsi_backward(const nk_rbm* rbm, const int8_t* sigma, int64_t ns,
                                 const double* g, double* grad_out, int32_t prec, void* scratch,
                                 size_t scratch_bytes, void* stream) {
  if (nk_status e = check_rbm(rbm, "nk_rbm_logpsi_backward")) return e;
  if (ns < 1) return fail(NK_ERR_INVALID_ARG, "nk_rbm_logpsi_backward: ns < 1");
  if (!sigma || !g || !grad_out || !scratch)
    return fail(NK_ERR_INVALID_ARG, "nk_rbm_logpsi_backward: NULL pointer");
  if (((uintptr_t)scratch) & 255)
    return fail(NK_ERR_INVALID_ARG, "nk_rbm_logpsi_backward: scratch not 256-byte aligned");
  if (prec != NK_PREC_FP32 && prec != NK_PREC_BF16X2)
    return fail(NK_ERR_INVALID_ARG, "nk_rbm_logpsi_backward: unknown precision %d", prec);
  return run_backward(rbm, sigma, ns, g, grad_out, prec, scratch, scratch_bytes,
                      (cudaStream_t)stream);
}

size_t nk_ffnn_scratch_bytes(const nk_ffnn* f, int64_t ns) {
  if (check_ffnn(f, "nk_ffnn_scratch_bytes") || ns < 0) return 0;
  return ffnn_scratch_bytes(f, ns);
}

nk_status nk_ffnn_logpsi(const nk_ffnn* f, const int8_t* sigma, int64_t ns, double* logpsi_out,
                         void* scratch, size_t scratch_bytes, void* stream) {
  if (nk_status e = check_ffnn(f, "nk_ffnn_logpsi")) return e;
  if (ns < 0) return fail(NK_ERR_INVALID_ARG, "nk_ffnn_logpsi: ns < 0");
  if (ns == 0) return NK_OK;
  if (!sigma || !logpsi_out || !scratch)
    return fail(NK_ERR_INVALID_ARG, "nk_ffnn_logpsi: NULL pointer");
  if (((uintptr_t)scratch) & 255)
    return fail(NK_ERR_INVALID_ARG, "nk_ffnn_logpsi: scratch not 256-byte aligned");
  return run_ffnn_logpsi(f, sigma, ns, logpsi_out, scratch, scratch_bytes, (cudaStream_t)stream);
}

nk_status nk_ffnn_backward(const nk_ffnn* f, const int8_t* sigma, int64_t ns, const double* g,
                           double* grad_out, void* scratch, size_t scratch_bytes, void* stream) {
  if (nk_status e = check_ffnn(f, "nk_ffnn_backward")) return e;
  if (ns < 1) return fail(NK_ERR_INVALID_ARG, "nk_ffnn_backward: ns < 1");
  if (!sigma || !g || !grad_out || !scratch)
    return fail(NK_ERR_INVALID_ARG, "nk_ffnn_backward: NULL pointer");
  if (((uintptr_t)scratch) & 255)
    return fail(NK_ERR_INVALID_ARG, "nk_ffnn_backward: scratch not 256-byte aligned");
  return run_ffnn_backward(f, sigma, ns, g, grad_out, scratch, scratch_bytes,
                           (cudaStream_t)stream);
}

size_t nk_supervised_scratch_bytes(int32_t n, int32_t m, int32_t is_complex, int64_t ns) {
  if (n < 1 || m < 1 || ns < 1) return 0;
  return supervised_scratch_bytes(n, m, is_complex ? 1 : 0, ns);
}

nk_status nk_supervised_step(nk_rbm* rbm, const int8_t* sigma, const double* log_target,
                             const double* weights, int64_t ns, int32_t prec, double lr,
                             double beta1, double beta2, int32_t step, double* moments,
                             double* grad_out, void* scratch, size_t scratch_bytes,
                             double* info_out, void* stream) {
  if (nk_status e = check_rbm(rbm, "nk_supervised_step")) return e;
  if (ns < 1) return fail(NK_ERR_INVALID_ARG, "nk_supervised_step: ns < 1");
  if (!sigma || !log_target || !scratch)
    return fail(NK_ERR_INVALID_ARG, "nk_supervised_step: NULL pointer");
  if (((uintptr_t)scratch) & 255)
    return fail(NK_ERR_INVALID_ARG, "nk_supervised_step: scratch not 256-byte aligned");
  if (prec != NK_PREC_FP32 && prec != NK_PREC_BF16X2)
    return fail(NK_ERR_INVALID_ARG, "nk_supervised_step: unknown precision %d", prec);
  if (prec == NK_PREC_BF16X2 && !tc_supported_shape(rbm->n, rbm->m))
    return fail(NK_ERR_UNSUPPORTED, "nk_supervised_step: the tensor-core path supports n + 1 <= 448");
  if (moments && (step < 1 || !(lr >= 0.0) || !(beta1 >= 0.0 && beta1 < 1.0) ||
                  !(beta2 >= 0.0 && beta2 <= 1.0)))
    return fail(NK_ERR_INVALID_ARG,
                "nk_supervised_step: AdaMax needs step >= 1, lr >= 0, 0 <= beta1 < 1, "
                "0 <= beta2 <= 1");
  return run_supervised_step(rbm, sigma, log_target, weights, ns, prec, lr, beta1, beta2, step,
                             moments, grad_out, scratch, scratch_bytes, info_out,
                             (cudaStream_t)stream);
}

nk_status nk_tune_shapes(nk_rbm* rbm, const void* op_dev, int32_t n_moves, const int8_t* sigma,
                         int64_t ns, void* theta_tmp, double* eloc_tmp, void* t_tmp,
                         void* scratch, size_t scratch_bytes, void* stream) {
  if (nk_status e = check_rbm(rbm, "nk_tune_shapes")) return e;
  if (ns < 1 || n_moves < 0) return fail(NK_ERR_INVALID_ARG, "nk_tune_shapes: ns < 1");
  if (!op_dev || !sigma || !theta_tmp || !eloc_tmp)
    return fail(NK_ERR_INVALID_ARG, "nk_tune_shapes: NULL pointer");
  cudaStream_t st = (cudaStream_t)stream;
  const int reps = 3;
  nk_rbm r = *rbm;
  // theta (tensor-core path), one and two CTAs per sample tile
  if (tc_supported_shape(r.n, r.m)) {
    float best = 1e30f;
    int best_s = 0;
    for (int segs = 1; segs <= 2; ++segs) {
      r.theta_segs = segs;
      float ms = 0.f;
      if (nk_status e = time_launches(st, reps, [&] {
            return launch_logpsi_bf16(&r, sigma, ns, nullptr, theta_tmp, st);
          }, &ms))
        return e;
      if (ms < best) {
        best = ms;
        best_s = segs;
      }
    }
    rbm->theta_segs = best_s;
  }
  // local energies, one and two CTAs per configuration tile (theta from above)
  if (n_moves > 0) {
    const size_t need = local_energy_scratch_bytes(r.m, r.is_complex ? 1 : 0, n_moves);
    if (!scratch || scratch_bytes < need || (((uintptr_t)scratch) & 255))
      return fail(NK_ERR_SHAPE, "nk_tune_shapes: scratch of %zu B, need %zu B (256-B aligned)",
                  scratch_bytes, need);
    r.theta_segs = rbm->theta_segs;
    float best = 1e30f;
    int best_s = 0;
    for (int segs = 1; segs <= 2; ++segs) {
      r.eloc_segs = segs;
      float ms = 0.f;
      if (nk_status e = time_launches(st, reps, [&] {
            return launch_local_energy(&r, op_dev, n_moves, sigma, theta_tmp, ns, eloc_tmp,
                                       t_tmp, scratch, scratch_bytes, st);
          }, &ms))
        return e;
      if (ms < best) {
        best = ms;
        best_s = segs;
      }
    }
    rbm->eloc_segs = best_s;
  }
  return NK_OK;
}

nk_status nk_query_status(int32_t* flags, void* stream) {
  if (!flags) return fail(NK_ERR_INVALID_ARG, "nk_query_status: flags is NULL");
  cudaStream_t st = (cudaStream_t)stream;
  if (cudaMemsetAsync(flags, 0, sizeof(int32_t), st) != cudaSuccess)
    return fail(NK_ERR_CUDA, "nk_query_status: cudaMemsetAsync failed");
  if (nk_status e = collect_status_tc(flags, st)) return e;
  if (nk_status e = collect_status_metropolis(flags, st)) return e;
  if (nk_status e = collect_status_local_energy(flags, st)) return e;
  return collect_status_api(flags, st);
}

nk_status nk_measure_alu_peaks(double* out) {
  if (!out) return fail(NK_ERR_INVALID_ARG, "nk_measure_alu_peaks: out is NULL");
  cudaStream_t st;
  if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess)
    return fail(NK_ERR_CUDA, "nk_measure_alu_peaks: cannot create a stream");
  const nk_status e = measure_alu_peaks(out, st);
  cudaStreamDestroy(st);
  return e;
}

nk_status nk_debug_bounded_wait(uint32_t polls, void* stream) {
  if (polls < 1 || polls > (1u << 20))
    return fail(NK_ERR_INVALID_ARG, "nk_debug_bounded_wait: polls must be in [1, 2^20]");
  bounded_wait_probe_kernel<<<1, 32, 0, (cudaStream_t)stream>>>(polls);
  return check_launch("nk_debug_bounded_wait");
}

}  // extern "C"
