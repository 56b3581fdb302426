// Compiled device form of a Hamiltonian given as 1-local site terms and 2-local
// bond terms (GraphOperator, Sec. 2.2.1).  Built on the host by
// nk_operator_upload, read by the local-energy kernel.
//
// The local energy (Eq. 5) of a configuration is
//   E_loc = sum(diagonal elements) + sum over moves of mel(s_i, s_k) psi'/psi,
// where a move flips spin i, or spins i and k.  Terms that produce the same
// move are merged; mel is indexed by 2 idx(s_i) + idx(s_k) (for a move made by
// a site term, k = i).
#pragma once

#include <stdint.h>

namespace nk {

struct OpDevHeader {
  int32_t n;
  int32_t n_dsite, n_dbond, n_moves;
  int32_t off_dsite, off_dbond, off_moves;  // byte offsets from the header
  int32_t flags;                            // kOpQuadMoves
};

// The moves are laid out in site quads: in every tile of 64, positions g,
// g + 16, g + 32, g + 48 (g < 16) are moves with the same first spin i.
constexpr int32_t kOpQuadMoves = 1;

struct OpDSite {  // diagonal of a site term: d[idx(s_i)]
  int32_t i, reserved;
  double d[2][2];  // complex
};

struct OpDBond {  // diagonal of a bond term: d[2 idx(s_i) + idx(s_k)]
  int32_t i, k;
  double d[4][2];
};

struct OpMove {
  int32_t i, k;      // flipped spin i; context (or second flipped) spin k
  int32_t two;       // 1: spins i and k both flip
  int32_t align;     // two-spin moves: +1 if mel is nonzero only for s_i = s_k,
                     // -1 if only for s_i = -s_k (terms are split so that one holds)
  double mel[4][2];  // complex matrix element by 2 idx(s_i) + idx(s_k)
};

}  // namespace nk
