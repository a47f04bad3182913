// The top of the elimination tree as one dense operator: choosing the levels and
// numbering their columns (ffa_topinv.h).  Host only.
#include <algorithm>
#include <climits>

#include "ffa_topinv.h"

namespace ffa {

namespace {

// T = the supernodes with columns on levels >= n_levels - k, numbered in node
// order; false (P unusable) when T is empty or over a size limit
bool top_levels(const Factor& f, int k, TopInvPlan& P) {
  P = TopInvPlan{};
  const int nn = (int)f.nodes.size();
  const int lmin = f.n_levels - k;
  int64_t nT = 0;
  std::vector<int32_t> lo_all(nn, INT_MAX);
  for (int s = 0; s < nn; ++s) {
    const Supernode& sn = f.nodes[s];
    if (sn.level < lmin) continue;
    if (sn.ncol > 0) {
      P.nodes.push_back(s);
      P.pos.push_back((int32_t)nT);
      lo_all[s] = std::min<int32_t>(lo_all[s], (int32_t)nT);
      nT += sn.ncol;
      P.factor_bytes += (int64_t)sn.ld * sn.ncol * 4;
    }
    // children come first, so lo_all[s] is final here
    if (sn.parent >= 0) lo_all[sn.parent] = std::min(lo_all[sn.parent], lo_all[s]);
  }
  if (P.nodes.empty() || (int)P.nodes.size() > kTiMaxNodes || nT > kTiMaxCols) return false;
  P.levels = k;
  P.nT = (int32_t)nT;
  P.ldG = (P.nT + 3) / 4 * 4;
  P.tiles = (P.nT + kTiTile - 1) / kTiTile;
  P.nblk = (P.nT + kTiBlk - 1) / kTiBlk;
  for (int32_t s : P.nodes) P.lo.push_back(lo_all[s]);
  P.tile_bytes = (int64_t)P.tiles * (P.tiles + 1) / 2 * kTiTile * kTiTile * 4;
  return true;
}

// structure rows of the T supernodes as T positions; false if one lies outside T
bool structure_map(const Factor& f, TopInvPlan& P) {
  const std::vector<int32_t> tpos = top_positions(f, P);
  P.rmap_off.assign(1, 0);
  for (int32_t s : P.nodes) {
    const Supernode& sn = f.nodes[s];
    for (int i = 0; i < sn.nrow; ++i) {
      const int32_t r = f.rows[sn.row_off + i];
      if (r < 0 || r >= (int32_t)tpos.size() || tpos[r] < 0) return false;
      P.rmap.push_back(tpos[r]);
    }
    P.rmap_off.push_back((int64_t)P.rmap.size());
  }
  return true;
}

}  // namespace

std::vector<int32_t> top_positions(const Factor& f, const TopInvPlan& P) {
  std::vector<int32_t> tpos(f.nF, -1);
  for (size_t q = 0; q < P.nodes.size(); ++q) {
    const Supernode& sn = f.nodes[P.nodes[q]];
    for (int c = 0; c < sn.ncol; ++c) tpos[sn.col0 + c] = P.pos[q] + c;
  }
  return tpos;
}

std::vector<int32_t> top_product_units(int32_t tiles) {
  std::vector<int32_t> u;
  const int nrow = (tiles + kTiUnitRows - 1) / kTiUnitRows;
  for (int a = 0; a < nrow; ++a) {
    const int last_col = std::min(tiles - 1, kTiUnitRows * a + kTiUnitRows - 1);   // J <= I
    for (int c = 0; c * kTiUnitCols <= last_col; ++c) {
      u.push_back(a);
      u.push_back(c);
    }
  }
  return u;
}

bool plan_top_inverse(const Factor& f, int k, TopInvPlan& P, std::string& err) {
  P = TopInvPlan{};
  if (k == 0) return true;
  if (k > 0) {
    if (k >= f.n_levels) {
      err = "top_inverse_levels must leave at least one level of the elimination tree below it";
      return false;
    }
    if (!top_levels(f, k, P)) {
      err = "top_inverse_levels: the top levels have more than " + std::to_string(kTiMaxNodes) +
            " supernodes or " + std::to_string(kTiMaxCols) + " columns";
      P = TopInvPlan{};
      return false;
    }
  } else {
    // automatic: the largest k whose S^-1 is no larger than the blocks it replaces
    int best = 0;
    TopInvPlan Q;
    for (int kk = 1; kk < f.n_levels; ++kk) {
      if (!top_levels(f, kk, Q)) break;
      if (Q.tile_bytes <= Q.factor_bytes) best = kk;
    }
    if (best == 0) return true;
    top_levels(f, best, P);
  }
  if (!structure_map(f, P)) {
    err = "internal: a structure row of a top supernode lies outside the top levels";
    P = TopInvPlan{};
    return false;
  }
  return true;
}

}  // namespace ffa
