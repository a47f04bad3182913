// Numeric decomposition of the W-step operator on the device (Algorithm 2,
// decompose(L); Sec. 6, "Rescaling mu_i and Lambda": the penalties change, L is
// assembled and decomposed again).
//
// The ordering and the supernode structure come from the host analysis
// (ffa_factor.h); only the numbers are computed here, by the multifrontal method
// over the same elimination tree, level by level:
//   * every front F_s ((n_s + m_s) x (n_s + m_s), column-major, lower triangle
//     used) is zeroed, receives the entries of L_FF in its columns and then the
//     update matrices of its children (extend-add, one child after the other so
//     that no two writes meet);
//   * its first n_s columns are eliminated right-looking in panels of kDfTile
//     columns: the diagonal block is factored and inverted in shared memory, the
//     rows below it are multiplied by that inverse (transposed), the trailing
//     lower triangle is updated tile by tile;
//   * inv(L_ss) = X comes from the block forward substitution of L_ss X = I,
//     right-looking as well: X_pp = inv(L_pp), X_pj = -X_pp S_pj (j < p) with
//     S_qj = sum_{j<=k<q} L_qk X_kj; once block row p of X is known, every later
//     block row q adds L_qp X_pj to its S_qj (kept in place of X_qj, which starts
//     at zero), so that each step is one tile product per tile and all tiles of a
//     step run side by side;
//   * B_s = [inv(L_ss); L_rs inv(L_ss)] is written in float into the layout the
//     triangular passes read (column-major, leading dimension ld, zero above the
//     diagonal of inv(L_ss)), and the trailing part of F_s is the update matrix
//     its parent takes.
// Arithmetic in float or double (template T); the stored blocks are float either
// way.  The work of each launch is a list of items (two int32 each) built here on
// the host once per analysis; the geometry of an item is computed by the
// functions below, which the kernels and the host check of the plan share.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "ffa_factor.h"

#if defined(__CUDACC__)
#define FFA_HD __host__ __device__ __forceinline__
#else
#define FFA_HD inline
#endif

namespace ffa {

constexpr int kDfTile = 64;     // panel width and tile edge
constexpr int kDfEaCols = 8;    // update-matrix columns per extend-add item

struct DfNode {
  int64_t fr_off = 0;   // offset of the front (elements of T)
  int64_t li_off = 0;   // offset of inv(L_ss) (elements of T), n_s x n_s column-major
  int64_t blk_off = 0;  // offset of B_s in the float blocks
  int32_t N = 0;        // front order n_s + m_s
  int32_t ldF = 0;      // leading dimension of the front (N rounded up to 4)
  int32_t ns = 0;       // columns eliminated here
  int32_t ldL = 0;      // leading dimension of inv(L_ss) (n_s rounded up to 4)
  int32_t ld = 0;       // leading dimension of B_s
  int32_t parent = -1;
};

struct DfItem {
  int32_t node;
  int32_t code;
};

enum DfKind : int32_t {
  kDfExtendAdd = 0,   // item: child, first update-matrix column
  kDfDiag = 1,        // item: node (panel p of the launch)
  kDfSolve = 2,       // item: node, code >= 0 row tile below the panel, code < 0 block (p, -1-code) of inv(L_ss)
  kDfUpdate = 3,      // item: node, code >= 0 (I << 16) | J trailing tile, J <= I; code < 0
                      // -1-code = (q << 16) | j: S_qj += L_qp X_pj (q > p >= j)
  kDfBrs = 4,         // item: node, (A << 16) | J tile of L_rs inv(L_ss)
  kDfPack = 5         // item: node, block column J of inv(L_ss) into B_s
};

struct DfLaunch {
  int32_t kind = 0;
  int32_t p = 0;        // panel (diag, solve, update)
  int64_t off = 0;      // first item
  int64_t count = 0;    // items
};

struct DevFactorPlan {
  std::vector<DfNode> nodes;
  std::vector<int64_t> rel_off;   // per child: its extend-add map in rel
  std::vector<int32_t> rel;       // structure row of a child -> index in its parent's front
  std::vector<DfItem> items;
  std::vector<DfLaunch> prog;     // launches in order
  std::vector<int64_t> orig_dst;  // per ELL slot of L_FF: front element it sets, -1 none
  int64_t front_elems = 0, linv_elems = 0, block_floats = 0;
  int32_t max_panels = 0;
};

// Geometry of panel p of a node: columns [c0, c0 + w) of the front are
// eliminated, the trailing part starts at t0 = c0 + w.
struct DfPanel {
  int32_t c0, w, t0;
};
FFA_HD DfPanel df_panel(const DfNode& s, int p) {
  DfPanel g;
  g.c0 = p * kDfTile;
  g.w = s.ns - g.c0 < kDfTile ? s.ns - g.c0 : kDfTile;
  g.t0 = g.c0 + g.w;
  return g;
}
FFA_HD int32_t df_panels(const DfNode& s) { return (s.ns + kDfTile - 1) / kDfTile; }
FFA_HD int32_t df_tiles(int32_t rows) { return (rows + kDfTile - 1) / kDfTile; }
FFA_HD int32_t df_min(int32_t a, int32_t b) { return a < b ? a : b; }

// Host: the plan for an analyzed factor.  ell_col / ell_count describe the
// column-major ELL of L_FF in elimination order (ell_col[q * nF + c] the column of
// slot q of row c, the first ell_count[c] slots real).  Returns false with a
// message when a structure is inconsistent (a child row missing from its parent's
// front, an ELL entry outside its column's front) or a size overflows.
bool build_devfactor_plan(const Factor& f, int32_t width, const std::vector<int32_t>& ell_col,
                          const std::vector<int32_t>& ell_count, DevFactorPlan& P, std::string& err);

// Device assembly of L_FF and L_FC from new penalties (the same sums as the host
// assembly, in the same order): each ELL slot and each L_FC entry is a list of
// (element, local vertex j, local vertex l) terms mu_i g_j . g_l.
struct DevAssemblyPlan {
  std::vector<int64_t> ell_ptr;   // width * nF + 1
  std::vector<int32_t> ell_src;   // element << 4 | j << 2 | l
  std::vector<int64_t> fc_ptr;    // entries of L_FC + 1 (the order of the device CSR by row)
  std::vector<int32_t> fc_src;
  std::vector<int32_t> cf_src;    // L_CF entry -> its L_FC entry (the same value)
};

struct OperatorHost;
struct OperatorArrays;
bool build_assembly_plan(const OperatorHost& H, const Factor& f, const OperatorArrays& A,
                         const std::vector<int64_t>& Ap, DevAssemblyPlan& Q, std::string& err);

}  // namespace ffa
