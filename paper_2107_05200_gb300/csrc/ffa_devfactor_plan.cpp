// Host side of the device decomposition: the per-node layout of the fronts and
// of inv(L_ss), the extend-add maps, the scatter of L_FF into the fronts and the
// item lists of every launch (ffa_devfactor.h), and the term lists of the device
// assembly of L = sum_i mu_i G_i^T G_i (eq. solvinginw).
#include <algorithm>
#include <unordered_map>

#include "ffa_devfactor.h"
#include "ffa_operator_host.h"

namespace ffa {

bool build_devfactor_plan(const Factor& f, int32_t width, const std::vector<int32_t>& ell_col,
                          const std::vector<int32_t>& ell_count, DevFactorPlan& P, std::string& err) {
  P = DevFactorPlan();
  const int nn = (int)f.nodes.size();
  const int nF = f.nF;
  if ((int64_t)ell_col.size() != (int64_t)width * nF || (int)ell_count.size() != nF) {
    err = "device decomposition: ELL arrays do not match the factor";
    return false;
  }
  P.nodes.resize(nn);
  int64_t fr = 0, li = 0;
  int32_t max_level = 0;
  for (int s = 0; s < nn; ++s) {
    const Supernode& sn = f.nodes[s];
    DfNode& d = P.nodes[s];
    d.N = sn.ncol + sn.nrow;
    d.ldF = (d.N + 3) / 4 * 4;
    d.ns = sn.ncol;
    d.ldL = (d.ns + 3) / 4 * 4;
    d.ld = sn.ld;
    d.blk_off = sn.blk_off;
    d.parent = sn.parent;
    d.fr_off = fr;
    d.li_off = li;
    fr += (int64_t)d.ldF * d.N;
    li += (int64_t)d.ldL * d.ns;
    // tile indices are packed 16 bits each into an item
    if (df_tiles(d.N) >= (1 << 15)) {
      err = "device decomposition: a front of order " + std::to_string(d.N) + " is too large";
      return false;
    }
    P.block_floats = std::max<int64_t>(P.block_floats, sn.blk_off + (int64_t)sn.ld * sn.ncol);
    P.max_panels = std::max(P.max_panels, df_panels(d));
    max_level = std::max(max_level, sn.level);
  }
  P.front_elems = fr;
  P.linv_elems = li;

  // children in index order, and the extend-add map of each child
  std::vector<std::vector<int32_t>> children(nn);
  for (int s = 0; s < nn; ++s)
    if (f.nodes[s].parent >= 0) children[f.nodes[s].parent].push_back(s);
  P.rel_off.assign(nn, 0);
  for (int c = 0; c < nn; ++c) {
    const Supernode& cn = f.nodes[c];
    P.rel_off[c] = (int64_t)P.rel.size();
    if (cn.parent < 0 || cn.nrow == 0) continue;
    const Supernode& pn = f.nodes[cn.parent];
    const int32_t* pr = f.rows.data() + pn.row_off;
    for (int32_t a = 0; a < cn.nrow; ++a) {
      const int32_t r = f.rows[cn.row_off + a];
      int32_t local;
      if (r >= pn.col0 && r < pn.col0 + pn.ncol) {
        local = r - pn.col0;
      } else {
        const int32_t* it = std::lower_bound(pr, pr + pn.nrow, r);
        if (it == pr + pn.nrow || *it != r) {
          err = "device decomposition: structure row " + std::to_string(r) + " of supernode " + std::to_string(c) +
                " is not in its parent's front";
          return false;
        }
        local = pn.ncol + (int32_t)(it - pr);
      }
      if (a > 0 && local <= P.rel.back()) {
        err = "device decomposition: the extend-add map of supernode " + std::to_string(c) + " is not ascending";
        return false;
      }
      P.rel.push_back(local);
    }
  }

  // launches, level by level
  std::vector<std::vector<int32_t>> by_level(max_level + 1);
  for (int s = 0; s < nn; ++s) by_level[f.nodes[s].level].push_back(s);
  auto emit = [&](int32_t kind, int32_t p, int64_t first) {
    const int64_t count = (int64_t)P.items.size() - first;
    if (count > 0) {
      DfLaunch L;
      L.kind = kind;
      L.p = p;
      L.off = first;
      L.count = count;
      P.prog.push_back(L);
    }
  };
  for (int lev = 0; lev <= max_level; ++lev) {
    const std::vector<int32_t>& ls = by_level[lev];
    size_t max_children = 0;
    int32_t max_p = 0;
    for (int s : ls) {
      max_children = std::max(max_children, children[s].size());
      max_p = std::max(max_p, df_panels(P.nodes[s]));
    }
    for (size_t k = 0; k < max_children; ++k) {
      const int64_t first = (int64_t)P.items.size();
      for (int s : ls) {
        if (k >= children[s].size()) continue;
        const int c = children[s][k];
        for (int32_t b0 = 0; b0 < f.nodes[c].nrow; b0 += kDfEaCols) P.items.push_back({c, b0});
      }
      emit(kDfExtendAdd, 0, first);
    }
    for (int32_t p = 0; p < max_p; ++p) {
      int64_t first = (int64_t)P.items.size();
      for (int s : ls)
        if (df_panels(P.nodes[s]) > p) P.items.push_back({s, 0});
      emit(kDfDiag, p, first);
      first = (int64_t)P.items.size();
      for (int s : ls) {
        const DfNode& d = P.nodes[s];
        if (df_panels(d) <= p) continue;
        const DfPanel g = df_panel(d, p);
        for (int32_t t = 0; t < df_tiles(d.N - g.t0); ++t) P.items.push_back({s, t});
        for (int32_t j = 0; j < p; ++j) P.items.push_back({s, -1 - j});
      }
      emit(kDfSolve, p, first);
      first = (int64_t)P.items.size();
      for (int s : ls) {
        const DfNode& d = P.nodes[s];
        if (df_panels(d) <= p) continue;
        const DfPanel g = df_panel(d, p);
        const int32_t T = df_tiles(d.N - g.t0);
        for (int32_t I = 0; I < T; ++I)
          for (int32_t J = 0; J <= I; ++J) P.items.push_back({s, (I << 16) | J});
        // the sums of the later block rows of inv(L_ss) take block row p
        for (int32_t q = p + 1; q < df_panels(d); ++q)
          for (int32_t j = 0; j <= p; ++j) P.items.push_back({s, -1 - ((q << 16) | j)});
      }
      emit(kDfUpdate, p, first);
    }
    int64_t first = (int64_t)P.items.size();
    for (int s : ls) {
      const DfNode& d = P.nodes[s];
      const int32_t ms = d.N - d.ns;
      if (d.ns == 0 || ms == 0) continue;
      for (int32_t A = 0; A < df_tiles(ms); ++A)
        for (int32_t J = 0; J < df_tiles(d.ns); ++J) P.items.push_back({s, (A << 16) | J});
    }
    emit(kDfBrs, 0, first);
    first = (int64_t)P.items.size();
    for (int s : ls)
      for (int32_t J = 0; J < df_tiles(P.nodes[s].ns); ++J) P.items.push_back({s, J});
    emit(kDfPack, 0, first);
  }

  // entries of L_FF: slot q of row c (column r of the row, r >= c) sets the
  // front element (r, c) of the supernode owning column c
  std::vector<int32_t> node_of(nF, -1);
  for (int s = 0; s < nn; ++s)
    for (int32_t q = 0; q < f.nodes[s].ncol; ++q) node_of[f.nodes[s].col0 + q] = s;
  P.orig_dst.assign((size_t)width * nF, -1);
  for (int32_t c = 0; c < nF; ++c) {
    const int s = node_of[c];
    if (s < 0) {
      err = "device decomposition: column " + std::to_string(c) + " belongs to no supernode";
      return false;
    }
    const Supernode& sn = f.nodes[s];
    const DfNode& d = P.nodes[s];
    const int32_t* sr = f.rows.data() + sn.row_off;
    for (int32_t q = 0; q < ell_count[c]; ++q) {
      const int32_t r = ell_col[(size_t)q * nF + c];
      if (r < c) continue;
      int32_t lr;
      if (r < sn.col0 + sn.ncol) {
        lr = r - sn.col0;
      } else {
        const int32_t* it = std::lower_bound(sr, sr + sn.nrow, r);
        if (it == sr + sn.nrow || *it != r) {
          err = "device decomposition: entry (" + std::to_string(r) + ", " + std::to_string(c) +
                ") of L_FF is outside the front of supernode " + std::to_string(s);
          return false;
        }
        lr = sn.ncol + (int32_t)(it - sr);
      }
      P.orig_dst[(size_t)q * nF + c] = d.fr_off + (int64_t)(c - sn.col0) * d.ldF + lr;
    }
  }
  return true;
}

bool build_assembly_plan(const OperatorHost& H, const Factor& f, const OperatorArrays& A,
                         const std::vector<int64_t>& Ap, DevAssemblyPlan& Q, std::string& err) {
  Q = DevAssemblyPlan();
  const int d = H.d, nF = H.nF, width = A.width;
  if ((int64_t)H.m >= ((int64_t)1 << 27)) {
    err = "device assembly: more than 2^27 elements";
    return false;
  }
  const int64_t n_fc = A.fc_ptr.empty() ? 0 : A.fc_ptr.back();
  // pass 0 counts the terms of every slot, pass 1 writes them; both visit the
  // terms in the host assembly's order (incidences of the row's vertex, then the
  // element's vertices)
  std::vector<int64_t> ell_fill, fc_fill;
  Q.ell_ptr.assign((size_t)width * nF + 1, 0);
  Q.fc_ptr.assign((size_t)n_fc + 1, 0);
  std::unordered_map<int32_t, int32_t> slot_of;  // eliminated column -> ELL slot of the row
  std::unordered_map<int32_t, int64_t> fc_of;    // pin -> L_FC entry of the row
  for (int pass = 0; pass < 2; ++pass) {
    for (int32_t c = 0; c < nF; ++c) {
      const int32_t fr = f.perm[c];
      const int v = H.free_vertex[fr];
      const int32_t cnt = (int32_t)(Ap[fr + 1] - Ap[fr]);
      slot_of.clear();
      for (int32_t q = 0; q < cnt; ++q) slot_of[A.ell_col[(size_t)q * nF + c]] = q;
      fc_of.clear();
      for (int64_t k = A.fc_ptr[c]; k < A.fc_ptr[c + 1]; ++k) fc_of[A.fc_col[k]] = k;
      for (int64_t q = H.inc_ptr[v]; q < H.inc_ptr[v + 1]; ++q) {
        const int i = H.inc[q] / (d + 1), j = H.inc[q] % (d + 1);
        for (int l = 0; l <= d; ++l) {
          const int u = H.T[(int64_t)i * (d + 1) + l];
          const int32_t code = (i << 4) | (j << 2) | l;
          if (H.free_of[u] >= 0) {
            auto it = slot_of.find(f.iperm[H.free_of[u]]);
            if (it == slot_of.end()) {
              err = "device assembly: a neighbour is missing from the ELL row";
              return false;
            }
            const size_t slot = (size_t)it->second * nF + c;
            if (pass == 0) ++Q.ell_ptr[slot + 1];
            else Q.ell_src[ell_fill[slot]++] = code;
          } else {
            auto it = fc_of.find(H.v2pin[u]);
            if (it == fc_of.end()) {
              err = "device assembly: a pinned neighbour is missing from L_FC";
              return false;
            }
            if (pass == 0) ++Q.fc_ptr[it->second + 1];
            else Q.fc_src[fc_fill[it->second]++] = code;
          }
        }
      }
    }
    if (pass == 0) {
      for (size_t k = 1; k < Q.ell_ptr.size(); ++k) Q.ell_ptr[k] += Q.ell_ptr[k - 1];
      for (size_t k = 1; k < Q.fc_ptr.size(); ++k) Q.fc_ptr[k] += Q.fc_ptr[k - 1];
      Q.ell_src.assign((size_t)Q.ell_ptr.back(), 0);
      Q.fc_src.assign((size_t)Q.fc_ptr.back(), 0);
      ell_fill.assign(Q.ell_ptr.begin(), Q.ell_ptr.end() - 1);
      fc_fill.assign(Q.fc_ptr.begin(), Q.fc_ptr.end() - 1);
    }
  }
  // L_CF: the entries of L_FC regrouped by pin (operator_arrays' order)
  Q.cf_src.assign((size_t)n_fc, 0);
  std::vector<int64_t> fill(A.cf_ptr.begin(), A.cf_ptr.end() - 1);
  for (int32_t c = 0; c < nF; ++c)
    for (int64_t k = A.fc_ptr[c]; k < A.fc_ptr[c + 1]; ++k) Q.cf_src[fill[A.fc_col[k]]++] = (int32_t)k;
  return true;
}

}  // namespace ffa
