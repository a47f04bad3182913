// The top of the elimination tree as one dense operator (the W step's solve,
// Sec. 4 "Efficient Evaluation"; Algorithm 2, decompose(L)).
//
// Order the free columns as [B; T], T the columns of the supernodes on the top k
// levels of the elimination tree (closed under ancestors) and B the rest.  With
// L_FF = L L^T,
//     x_T = (L_TT L_TT^T)^-1 (b_T - L_TB L_BB^-1 b_B) = S^-1 t_T,
// S the Schur complement of the B block, so a solve is: the forward pass over the
// supernodes of B (which leaves t_T in the T rows of its running right-hand side),
// x_T = S^-1 t_T as one symmetric matrix-vector product, and the backward pass
// over B (which reads x_T at its structure rows).  The triangular passes over
// T read its factor twice, one level after the other, and these levels hold few
// large supernodes; S^-1 is read once, by all SMs at the same time.
//
// S^-1 = F^T F with F = L_TT^-1, computed on the device from the float blocks of
// the T supernodes after every decomposition of L: F comes from the forward pass
// over T applied to the identity (G = I; for each T supernode s in order,
// F_s = inv(L_ss) G_s and G_r -= (L_rs inv(L_ss)) G_s at its structure rows r),
// then the lower 64 x 64 tiles of F^T F.  The tiles are stored in float, packed
// row by row (tile (I, J), J <= I, at I (I + 1) / 2 + J, column-major, the
// diagonal tiles whole), zero past n_T.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "ffa_factor.h"

namespace ffa {

constexpr int kTiTile = 64;             // tile edge of S^-1
constexpr int kTiBlk = 2 * kTiTile;     // the product's work unit: a block of 2 x 2 tiles
constexpr int kTiMaxNodes = 16;         // T supernodes at most
constexpr int kTiMaxCols = 16384;       // n_T at most (packed tiles: 512 MB)
constexpr int kTiUnitRows = 2;          // the product's work unit: 2 rows of tiles ...
constexpr int kTiUnitCols = 4;          // ... times 4 columns of tiles

struct TopInvPlan {
  int levels = 0;                    // k (0: not used)
  int32_t nT = 0;                    // columns of T
  int32_t ldG = 0;                   // leading dimension of the setup work arrays (nT rounded up to 4)
  int32_t tiles = 0;                 // tile rows: ceil(nT / 64)
  int32_t nblk = 0;                  // block rows of the product: ceil(nT / 128)
  std::vector<int32_t> nodes;        // T supernodes in node order (children first)
  std::vector<int32_t> pos, lo;      // per T supernode: first T position, first T position of its T subtree
  std::vector<int64_t> rmap_off;     // per T supernode: its structure rows' T positions in rmap
  std::vector<int32_t> rmap;
  int64_t factor_bytes = 0;          // bytes the factor blocks of T occupy (ld x ncol floats each)
  int64_t tile_bytes = 0;            // bytes of the packed tiles of S^-1
};

// The top k levels of a factor's tree (levels >= n_levels - k); k = -1 picks the
// largest k < n_levels with at most kTiMaxNodes supernodes and kTiMaxCols columns
// whose packed S^-1 takes no more bytes than the factor blocks it replaces (each
// read twice per solve by the passes, S^-1 once), 0 if none.  An explicit k must
// leave a level below T and satisfy the same size limits.  Returns false with a
// message for an explicit k that cannot be used.
bool plan_top_inverse(const Factor& f, int k, TopInvPlan& P, std::string& err);

// T position of each eliminated column (-1 outside T)
std::vector<int32_t> top_positions(const Factor& f, const TopInvPlan& P);

// The product's work units (a, c), flattened: unit (a, c) covers the tiles (I, J)
// with I in [2a, 2a + 2), J in [4c, 4c + 4), J <= I < tiles; every lower tile lies
// in exactly one unit.
std::vector<int32_t> top_product_units(int32_t tiles);

}  // namespace ffa
