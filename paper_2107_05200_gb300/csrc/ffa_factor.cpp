// Nested-dissection ordering and multifrontal Cholesky of the W-step operator.
// See ffa_factor.h for the stored form.  Host code, run once per mesh and rho.
#include "ffa_factor.h"

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <functional>
#include <limits>
#include <exception>
#include <memory>
#include <mutex>
#include <thread>

namespace ffa {
namespace {

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

int resolve_threads(int req) {
  if (req > 0) return req;
  unsigned h = std::thread::hardware_concurrency();
  return h ? static_cast<int>(h) : 1;
}

// Dynamic-chunk parallel loop over [0, n).
void parallel_for(int64_t n, int threads, int64_t grain,
                  const std::function<void(int64_t, int64_t)>& fn) {
  if (n <= 0) return;
  if (threads <= 1 || n <= grain) {
    fn(0, n);
    return;
  }
  int t = static_cast<int>(std::min<int64_t>(threads, (n + grain - 1) / grain));
  std::atomic<int64_t> next(0);
  auto worker = [&]() {
    for (;;) {
      int64_t b = next.fetch_add(grain);
      if (b >= n) break;
      fn(b, std::min(n, b + grain));
    }
  };
  run_threads(t, [&](int) { worker(); });
}

// ---------------------------------------------------------------------------
// geometric nested dissection
// ---------------------------------------------------------------------------
struct TreeNode {
  std::vector<int32_t> verts;
  int child[2] = {-1, -1};
};

struct Dissection {
  const FactorInput& in;
  std::vector<int8_t> side;
  std::vector<TreeNode> tree;

  explicit Dissection(const FactorInput& i) : in(i), side(i.nF, 0) {}

  int leaf_node(std::vector<int32_t>& S) {
    int id = static_cast<int>(tree.size());
    tree.emplace_back();
    tree[id].verts = std::move(S);
    return id;
  }

  // Split S across the widest axis at the largest coordinate gap among the
  // middle ranks; the smaller one-sided boundary becomes the separator.
  int build(std::vector<int32_t>& S) {
    const size_t N = S.size();
    if (static_cast<int>(N) <= in.leaf_size) return leaf_node(S);
    double lo[3], hi[3];
    for (int a = 0; a < 3; ++a) {
      lo[a] = std::numeric_limits<double>::infinity();
      hi[a] = -lo[a];
    }
    for (int32_t v : S)
      for (int a = 0; a < 3; ++a) {
        double x = in.coords[3 * (int64_t)v + a];
        lo[a] = std::min(lo[a], x);
        hi[a] = std::max(hi[a], x);
      }
    int ax = 0;
    for (int a = 1; a < 3; ++a)
      if (hi[a] - lo[a] > hi[ax] - lo[ax]) ax = a;
    if (!(hi[ax] - lo[ax] > 0.0)) return leaf_node(S);

    std::vector<std::pair<double, int32_t>> key(N);
    for (size_t p = 0; p < N; ++p) key[p] = {in.coords[3 * (int64_t)S[p] + ax], S[p]};
    std::sort(key.begin(), key.end());
    size_t a = std::max<size_t>(1, N * 2 / 5), b = std::min<size_t>(N - 1, N * 3 / 5);
    size_t cut = N / 2;
    double best = -1.0;
    for (size_t p = a; p <= b; ++p) {
      double gap = key[p].first - key[p - 1].first;
      if (gap > best) {
        best = gap;
        cut = p;
      }
    }
    for (size_t p = 0; p < N; ++p) side[key[p].second] = (p < cut) ? 1 : 2;
    std::vector<int32_t> bl, br;
    for (size_t p = 0; p < N; ++p) {
      int32_t v = key[p].second;
      int8_t s = side[v], other = (s == 1) ? 2 : 1;
      for (int64_t k = in.Ap[v]; k < in.Ap[v + 1]; ++k)
        if (side[in.Ai[k]] == other) {
          (s == 1 ? bl : br).push_back(v);
          break;
        }
    }
    std::vector<int32_t>& sep = (bl.size() <= br.size()) ? bl : br;
    for (int32_t v : sep) side[v] = 3;
    std::vector<int32_t> L, R;
    L.reserve(cut);
    R.reserve(N - cut);
    for (size_t p = 0; p < N; ++p) {
      int32_t v = key[p].second;
      if (side[v] == 1) L.push_back(v);
      else if (side[v] == 2) R.push_back(v);
    }
    for (int32_t v : S) side[v] = 0;
    if (L.empty() && R.empty()) return leaf_node(S);
    std::vector<int32_t>().swap(S);
    int id = static_cast<int>(tree.size());
    tree.emplace_back();
    tree[id].verts = std::move(sep);
    int c0 = L.empty() ? -1 : build(L);
    int c1 = R.empty() ? -1 : build(R);
    tree[id].child[0] = c0;
    tree[id].child[1] = c1;
    return id;
  }
};

// Postorder numbering of the dissection tree into supernodes.  Of two children
// the shallower subtree is numbered first, so that a node's last child (the one
// whose columns end where the node's begin) is on its longest path to a leaf.
void number_tree(const std::vector<TreeNode>& tree, int t, Factor& f, std::vector<int>& tree2node) {
  // heights (children are created after their parent, so they have larger ids)
  std::vector<int> height(tree.size(), 0);
  for (int id = (int)tree.size() - 1; id >= 0; --id)
    for (int k = 0; k < 2; ++k)
      if (tree[id].child[k] >= 0) height[id] = std::max(height[id], height[tree[id].child[k]] + 1);
  auto ordered = [&](int id, int k) {
    const int a = tree[id].child[0], b = tree[id].child[1];
    const bool swap = a >= 0 && b >= 0 && height[a] > height[b];
    return tree[id].child[swap ? 1 - k : k];
  };
  // iterative postorder
  std::vector<std::pair<int, int>> st;  // (tree node, state)
  st.push_back({t, 0});
  while (!st.empty()) {
    auto& top = st.back();
    int id = top.first;
    if (top.second < 2) {
      int c = ordered(id, top.second++);
      if (c >= 0) st.push_back({c, 0});
      continue;
    }
    st.pop_back();
    Supernode sn;
    sn.col0 = static_cast<int32_t>(f.perm.size());
    sn.ncol = static_cast<int32_t>(tree[id].verts.size());
    for (int32_t v : tree[id].verts) f.perm.push_back(v);
    int lev = 0;
    bool has_child = false;
    int me = static_cast<int>(f.nodes.size());
    for (int k = 0; k < 2; ++k) {
      int c = tree[id].child[k];
      if (c < 0) continue;
      int cn = tree2node[c];
      f.nodes[cn].parent = me;
      lev = std::max(lev, f.nodes[cn].level + 1);
      has_child = true;
    }
    sn.level = has_child ? lev : 0;
    tree2node[id] = me;
    f.nodes.push_back(sn);
  }
}

// ---------------------------------------------------------------------------
// dense kernels on a front stored row-major (lower triangle used), ld = N
// ---------------------------------------------------------------------------
// Register tiles of the dense kernels: kMR rows times kNR columns of an update,
// the kNR columns contiguous in the packed operand so that the compiler's
// vectorizer keeps kMR x kNR independent accumulators (no reductions, so no
// reassociation and the same rounding whatever the target's vector width).
constexpr int kMR = 4, kNR = 8;

// acc[r][c] += sum_k a_r[k] * b[k * kNR + c], a_r the kMR rows of A (k contiguous)
inline void tile_rows(int64_t K, const double* const a[kMR], const double* b, double acc[kMR][kNR]) {
  for (int64_t k = 0; k < K; ++k) {
    const double* bk = b + k * kNR;
    for (int r = 0; r < kMR; ++r) {
      const double ar = a[r][k];
      for (int c = 0; c < kNR; ++c) acc[r][c] += ar * bk[c];
    }
  }
}

// acc[r][c] += sum_k a[k * kNR + r0 + r] * b[k * kNR + c]: both operands packed
inline void tile_packed(int64_t K, const double* a, const double* b, double acc[kMR][kNR]) {
  for (int64_t k = 0; k < K; ++k) {
    const double* ak = a + k * kNR;
    const double* bk = b + k * kNR;
    for (int r = 0; r < kMR; ++r) {
      const double ar = ak[r];
      for (int c = 0; c < kNR; ++c) acc[r][c] += ar * bk[c];
    }
  }
}

// Eliminate the first ns columns of the N x N front F; on return rows/cols
// [0, ns) hold L11, rows [ns, N) x cols [0, ns) hold L21 and the trailing lower
// triangle holds F22 - L21 L21^T.  Returns false if a pivot is not positive.
// Right-looking in panels of kPanel columns: the diagonal block is factored in
// place, the rows below it are packed kNR at a time (column k of the panel as kNR
// consecutive values), solved against the diagonal block in that form and
// written back, and the trailing lower triangle is updated tile by tile from the
// packed panel.
bool partial_cholesky(double* F, int N, int ns, int threads) {
  constexpr int kPanel = 96;
  std::vector<double> pack;
  for (int k0 = 0; k0 < ns; k0 += kPanel) {
    const int k1 = std::min(ns, k0 + kPanel);
    const int w = k1 - k0;
    // diagonal block, left-looking within the panel
    for (int k = k0; k < k1; ++k) {
      double* Fk = F + (int64_t)k * N;
      double dkk = Fk[k];
      for (int l = k0; l < k; ++l) dkk -= Fk[l] * Fk[l];
      if (!(dkk > 0.0) || !std::isfinite(dkk)) return false;
      dkk = std::sqrt(dkk);
      Fk[k] = dkk;
      for (int i = k + 1; i < k1; ++i) {
        double* Fi = F + (int64_t)i * N;
        double v = Fi[k];
        for (int l = k0; l < k; ++l) v -= Fi[l] * Fk[l];
        Fi[k] = v / dkk;
      }
    }
    const int64_t nrows = N - k1;
    if (nrows == 0) continue;
    const int64_t nblk = (nrows + kNR - 1) / kNR;
    pack.assign((size_t)nblk * w * kNR, 0.0);
    // rows below the panel: pack, solve X L11^T = F21 by columns, write back
    const int64_t tw = nrows * w * w;
    parallel_for(nblk, tw > (1 << 20) ? threads : 1, 4, [&](int64_t b, int64_t e) {
      for (int64_t blk = b; blk < e; ++blk) {
        double* P = pack.data() + blk * w * kNR;
        const int64_t r0 = blk * kNR;
        const int nr = (int)std::min<int64_t>(kNR, nrows - r0);
        for (int c = 0; c < nr; ++c) {
          const double* Fi = F + (k1 + r0 + c) * N + k0;
          for (int k = 0; k < w; ++k) P[k * kNR + c] = Fi[k];
        }
        for (int k = 0; k < w; ++k) {
          const double* Lk = F + (int64_t)(k0 + k) * N + k0;
          double v[kNR];
          for (int c = 0; c < kNR; ++c) v[c] = P[k * kNR + c];
          for (int l = 0; l < k; ++l) {
            const double lkl = Lk[l];
            for (int c = 0; c < kNR; ++c) v[c] -= P[l * kNR + c] * lkl;
          }
          const double dk = Lk[k];
          for (int c = 0; c < kNR; ++c) P[k * kNR + c] = v[c] / dk;
        }
        for (int c = 0; c < nr; ++c) {
          double* Fi = F + (k1 + r0 + c) * N + k0;
          for (int k = 0; k < w; ++k) Fi[k] = P[k * kNR + c];
        }
      }
    });
    // trailing update of the lower triangle: rows in tiles of kMR, columns in
    // tiles of kNR up to the diagonal
    const int64_t nrt = (nrows + kMR - 1) / kMR;
    const int64_t uw = nrows * nrows / 2 * w;
    parallel_for(nrt, uw > (1 << 20) ? threads : 1, 2, [&](int64_t b, int64_t e) {
      for (int64_t rt = b; rt < e; ++rt) {
        const int64_t i0 = rt * kMR;
        const double* a = pack.data() + (i0 / kNR) * w * kNR + (i0 % kNR);
        const int64_t jb_end = std::min<int64_t>(i0 + kMR - 1, nrows - 1) / kNR;
        for (int64_t jb = 0; jb <= jb_end; ++jb) {
          double acc[kMR][kNR] = {};
          tile_packed(w, a, pack.data() + jb * w * kNR, acc);
          for (int r = 0; r < kMR; ++r) {
            const int64_t i = i0 + r;
            if (i >= nrows) break;
            double* Fi = F + (k1 + i) * N + k1;
            for (int c = 0; c < kNR; ++c) {
              const int64_t j = jb * kNR + c;
              if (j > i) break;
              Fi[j] -= acc[r][c];
            }
          }
        }
      }
    });
  }
  return true;
}

// B = [inv(L11); L21 inv(L11)] (column-major, leading dimension N, zero above the
// diagonal of inv(L11); every entry of B is written) from the factored front F (row-major, L11 in rows/cols
// [0, ns), L21 in rows [ns, N)).  Columns go kNR at a time: the columns of
// inv(L11) by forward substitution of L11 X = I with the kNR right-hand sides
// side by side, then the rows of L21 times them kMR at a time.
void inverse_blocks(const double* F, int N, int ns, int threads, double* B) {
  const int ms = N - ns;
  const int64_t ncb = (ns + kNR - 1) / kNR;
  const int64_t work = (int64_t)ns * ns * (ns + ms);
  parallel_for(ncb, work > (1 << 21) ? threads : 1, 1, [&](int64_t b, int64_t e) {
    std::vector<double> X((size_t)ns * kNR);
    for (int64_t cb = b; cb < e; ++cb) {
      const int j0 = (int)(cb * kNR);
      const int nc = std::min(kNR, ns - j0);
      // rows [j0, ns) of columns j0 .. j0+kNR of inv(L11); rows above are zero.
      // Rows go kMR at a time: the part of the sum over rows already solved as
      // one tile, then the small triangle inside the row block in order.
      double* Xj = X.data() + (int64_t)j0 * kNR;
      for (int i0 = j0; i0 < ns; i0 += kMR) {
        const double* rows[kMR];
        for (int r = 0; r < kMR; ++r) rows[r] = F + (int64_t)std::min(i0 + r, ns - 1) * N + j0;
        double acc[kMR][kNR] = {};
        tile_rows(i0 - j0, rows, Xj, acc);
        for (int r = 0; r < kMR && i0 + r < ns; ++r) {
          const int i = i0 + r;
          const double* Li = F + (int64_t)i * N;
          double v[kNR];
          for (int c = 0; c < kNR; ++c) v[c] = ((i == j0 + c) ? 1.0 : 0.0) - acc[r][c];
          for (int k = i0; k < i; ++k) {
            const double lik = Li[k];
            const double* xk = X.data() + (int64_t)k * kNR;
            for (int c = 0; c < kNR; ++c) v[c] -= lik * xk[c];
          }
          const double di = Li[i];
          for (int c = 0; c < kNR; ++c) X[(int64_t)i * kNR + c] = v[c] / di;
        }
      }
      for (int c = 0; c < nc; ++c) {
        double* col = B + (int64_t)(j0 + c) * N;
        std::fill(col, col + j0 + c, 0.0);
        for (int i = j0 + c; i < ns; ++i) col[i] = X[(int64_t)i * kNR + c];
      }
      // rows of L21 inv(L11): sum over k >= j0 (inv(L11) is lower triangular)
      const int64_t K = ns - j0;
      for (int a0 = 0; a0 < ms; a0 += kMR) {
        const double* rows[kMR];
        for (int r = 0; r < kMR; ++r) rows[r] = F + (int64_t)(ns + std::min(a0 + r, ms - 1)) * N + j0;
        double acc[kMR][kNR] = {};
        tile_rows(K, rows, Xj, acc);
        for (int r = 0; r < kMR && a0 + r < ms; ++r)
          for (int c = 0; c < nc; ++c) B[(int64_t)(j0 + c) * N + ns + a0 + r] = acc[r][c];
      }
    }
  });
}

struct NumericWork {
  std::vector<int32_t> pos;
  explicit NumericWork(int nF) : pos(nF, -1) {}
};

// numeric multifrontal factorization into the blocks of an analyzed Factor
int numeric(const FactorInput& in, Factor& f, std::string& err, int threads) {
  const double t1 = now_s();
  const int nn = static_cast<int>(f.nodes.size());
  std::vector<std::vector<int32_t>> children(nn);
  for (int s = 0; s < nn; ++s)
    if (f.nodes[s].parent >= 0) children[f.nodes[s].parent].push_back(s);
  int64_t total = 0;
  for (auto& sn : f.nodes) total = std::max<int64_t>(total, sn.blk_off + (int64_t)sn.ld * sn.ncol);
  f.blocks.assign(total, 0.0f);
  if (in.keep_double) f.blocks64.assign(total, 0.0);
  std::vector<std::unique_ptr<double[]>> upd(nn);  // ms x ms, lower triangle used
  std::atomic<int> failed(-1);

  auto factor_node = [&](int s, NumericWork& wk, int dense_threads) {
    if (failed.load() >= 0) return;
    const Supernode& sn = f.nodes[s];
    const int ns = sn.ncol, ms = sn.nrow, N = ns + ms;
    const int32_t* R = f.rows.data() + sn.row_off;
    // the front, row-major; only its lower triangle is ever read, so only that is
    // zeroed (row by row, in parallel on the large fronts at the top of the tree)
    const int64_t big = (int64_t)N * N > (1 << 22) ? dense_threads : 1;
    std::unique_ptr<double[]> Fbuf(new double[(size_t)N * N]);
    double* F = Fbuf.get();
    parallel_for(N, big, 64, [&](int64_t b, int64_t e) {
      for (int64_t i = b; i < e; ++i) std::fill(F + i * N, F + i * N + i + 1, 0.0);
    });
    for (int q = 0; q < ns; ++q) wk.pos[sn.col0 + q] = q;
    for (int q = 0; q < ms; ++q) wk.pos[R[q]] = ns + q;
    // original entries (lower triangle of the front); each column is its own
    parallel_for(ns, big, 64, [&](int64_t b, int64_t e) {
      for (int64_t q = b; q < e; ++q) {
        const int32_t c = sn.col0 + (int32_t)q;
        const int32_t old = f.perm[c];
        for (int64_t k = in.Ap[old]; k < in.Ap[old + 1]; ++k) {
          const int32_t r = f.iperm[in.Ai[k]];
          if (r < c) continue;
          F[(int64_t)wk.pos[r] * N + q] += in.Ax[k];
        }
      }
    });
    // extend-add of the children's update matrices, child after child; the rows
    // of one child land on distinct rows of the front
    for (int ch : children[s]) {
      const Supernode& cn = f.nodes[ch];
      const int32_t* Rc = f.rows.data() + cn.row_off;
      const double* Uc = upd[ch].get();
      const int64_t cbig = (int64_t)cn.nrow * cn.nrow > (1 << 22) ? dense_threads : 1;
      parallel_for(cn.nrow, cbig, 32, [&](int64_t b0, int64_t e0) {
        for (int64_t a = b0; a < e0; ++a) {
          const int pa = wk.pos[Rc[a]];
          double* Fa = F + (int64_t)pa * N;
          const double* Ua = Uc + a * cn.nrow;
          for (int64_t b = 0; b <= a; ++b) Fa[wk.pos[Rc[b]]] += Ua[b];
        }
      });
      upd[ch].reset();
    }
    for (int q = 0; q < ns; ++q) wk.pos[sn.col0 + q] = -1;
    for (int q = 0; q < ms; ++q) wk.pos[R[q]] = -1;
    if (!partial_cholesky(F, N, ns, dense_threads)) {
      failed.store(s);
      return;
    }
    // update matrix for the parent
    if (ms > 0) {
      upd[s].reset(new double[(size_t)ms * ms]);
      double* U = upd[s].get();
      parallel_for(ms, (int64_t)ms * ms > (1 << 22) ? dense_threads : 1, 64, [&](int64_t b, int64_t e) {
        for (int64_t a = b; a < e; ++a) std::copy(F + (ns + a) * N + ns, F + (ns + a) * N + ns + a + 1, U + a * ms);
      });
    }
    if (ns == 0) return;
    // B_s = [inv(L11); L21 inv(L11)], column-major, leading dimension N
    std::unique_ptr<double[]> B(new double[(size_t)N * ns]);
    inverse_blocks(F, N, ns, dense_threads, B.get());
    parallel_for(ns, (int64_t)N * ns > (1 << 22) ? dense_threads : 1, 64, [&](int64_t b, int64_t e) {
      for (int64_t j = b; j < e; ++j) {
        float* dst = f.blocks.data() + sn.blk_off + j * sn.ld;
        const double* src = B.get() + j * N;
        for (int i = 0; i < N; ++i) dst[i] = static_cast<float>(src[i]);
        if (in.keep_double) std::copy(src, src + N, f.blocks64.begin() + sn.blk_off + j * sn.ld);
      }
    });
  };

  // independent subtrees go to a pool; the top of the tree runs with parallel dense kernels
  std::vector<int64_t> sub_work(nn, 0);
  for (int s = 0; s < nn; ++s) {
    const double ns = f.nodes[s].ncol, ms = f.nodes[s].nrow;
    sub_work[s] += (int64_t)(ns * ns * ns + ns * ns * ms + ns * ms * ms) + ns + ms + 1;
    if (f.nodes[s].parent >= 0) sub_work[f.nodes[s].parent] += sub_work[s];
  }
  std::vector<int> tasks, top;
  {
    std::vector<int> frontier;
    for (int s = 0; s < nn; ++s)
      if (f.nodes[s].parent < 0) frontier.push_back(s);
    std::vector<char> is_top(nn, 0);
    const size_t want = static_cast<size_t>(threads) * 4;
    while (!frontier.empty() && frontier.size() < want) {
      auto it = std::max_element(frontier.begin(), frontier.end(),
                                 [&](int a, int b) { return sub_work[a] < sub_work[b]; });
      int s = *it;
      if (children[s].empty()) break;
      frontier.erase(it);
      is_top[s] = 1;
      for (int ch : children[s]) frontier.push_back(ch);
    }
    tasks = frontier;
    std::sort(tasks.begin(), tasks.end(), [&](int a, int b) { return sub_work[a] > sub_work[b]; });
    for (int s = 0; s < nn; ++s)
      if (is_top[s]) top.push_back(s);  // ascending index = postorder
  }
  // subtree of a task root = contiguous postorder range ending at the root
  std::vector<int> first_desc(nn);
  for (int s = 0; s < nn; ++s) first_desc[s] = s;
  for (int s = 0; s < nn; ++s)
    if (f.nodes[s].parent >= 0)
      first_desc[f.nodes[s].parent] = std::min(first_desc[f.nodes[s].parent], first_desc[s]);
  {
    std::atomic<size_t> next(0);
    auto worker = [&]() {
      NumericWork wk(in.nF);
      for (;;) {
        size_t t = next.fetch_add(1);
        if (t >= tasks.size()) break;
        const int r = tasks[t];
        for (int s = first_desc[r]; s <= r; ++s) factor_node(s, wk, 1);
      }
    };
    const int tcount = std::max(1, std::min<int>(threads, (int)tasks.size()));
    run_threads(tcount, [&](int) { worker(); });
  }
  {
    NumericWork wk(in.nF);
    for (int s : top) factor_node(s, wk, threads);
  }
  if (failed.load() >= 0) {
    err = "the W-step matrix is not positive definite (pivot failure in supernode " +
          std::to_string(failed.load()) + ")";
    return 3;
  }
  f.t_factor = now_s() - t1;
  return 0;
}


}  // namespace

// ---------------------------------------------------------------------------
int build_factor(const FactorInput& in, Factor& f, std::string& err) {
  const double t0 = now_s();
  const int threads = resolve_threads(in.threads);
  if (in.nF <= 0) {
    err = "no free vertices";
    return 1;
  }
  f = Factor();
  f.nF = in.nF;

  // ---- ordering: one dissection per connected piece is not needed; the split
  // handles disconnected sets through empty separators.
  Dissection nd(in);
  std::vector<int32_t> all(in.nF);
  for (int32_t v = 0; v < in.nF; ++v) all[v] = v;
  int root_tree = nd.build(all);
  std::vector<int> tree2node(nd.tree.size(), -1);
  f.perm.reserve(in.nF);
  number_tree(nd.tree, root_tree, f, tree2node);
  if ((int)f.perm.size() != in.nF) {
    err = "nested dissection lost vertices";
    return 1;
  }
  f.iperm.assign(in.nF, -1);
  for (int32_t c = 0; c < in.nF; ++c) f.iperm[f.perm[c]] = c;
  const int nn = static_cast<int>(f.nodes.size());
  std::vector<std::vector<int32_t>> children(nn);
  for (int s = 0; s < nn; ++s)
    if (f.nodes[s].parent >= 0) children[f.nodes[s].parent].push_back(s);
  int maxlev = 0;
  for (auto& s : f.nodes) maxlev = std::max(maxlev, s.level);
  f.n_levels = maxlev + 1;

  // ---- symbolic: structure of every supernode
  {
    std::vector<int32_t> mark(in.nF, -1);
    std::vector<int32_t> tmp;
    for (int s = 0; s < nn; ++s) {
      Supernode& sn = f.nodes[s];
      const int32_t c1 = sn.col0 + sn.ncol;
      tmp.clear();
      for (int32_t c = sn.col0; c < c1; ++c) {
        int32_t old = f.perm[c];
        for (int64_t k = in.Ap[old]; k < in.Ap[old + 1]; ++k) {
          int32_t r = f.iperm[in.Ai[k]];
          if (r >= c1 && mark[r] != s) {
            mark[r] = s;
            tmp.push_back(r);
          }
        }
      }
      for (int ch : children[s]) {
        const Supernode& cn = f.nodes[ch];
        for (int64_t q = 0; q < cn.nrow; ++q) {
          int32_t r = f.rows[cn.row_off + q];
          if (r >= c1 && mark[r] != s) {
            mark[r] = s;
            tmp.push_back(r);
          }
        }
      }
      std::sort(tmp.begin(), tmp.end());
      sn.row_off = static_cast<int64_t>(f.rows.size());
      sn.nrow = static_cast<int32_t>(tmp.size());
      f.rows.insert(f.rows.end(), tmp.begin(), tmp.end());
    }
  }
  int64_t total = 0, flops = 0;
  for (auto& sn : f.nodes) {
    sn.ld = (sn.ncol + sn.nrow + 3) / 4 * 4;
    sn.blk_off = total;
    total += (int64_t)sn.ld * sn.ncol;
    const double ns = sn.ncol, ms = sn.nrow;
    // partial Cholesky + explicit inverse + M = L21 inv(L11), FMA = 2 flops
    flops += (int64_t)(ns * ns * ns / 3.0 + ns * ns * ms + ns * ms * ms + ns * ns * ns / 3.0 + ms * ns * ns);
  }
  f.flops = flops;
  const double t1 = now_s();
  f.t_analyze = t1 - t0;
  if (!in.numeric) return 0;
  return numeric(in, f, err, threads);
}

int refactor(const FactorInput& in, Factor& f, std::string& err) {
  if (in.nF != f.nF || f.nodes.empty()) {
    err = "refactor: the operator's pattern does not match the analyzed factor";
    return 1;
  }
  return numeric(in, f, err, resolve_threads(in.threads));
}

void host_solve(const Factor& f, const double* b, double* x, int nrhs) {
  const int64_t nF = f.nF;
  std::vector<double> y(nF * nrhs), z(nF * nrhs, 0.0), xs(nF * nrhs, 0.0);
  for (int64_t c = 0; c < nF; ++c)
    for (int k = 0; k < nrhs; ++k) y[c * nrhs + k] = b[(int64_t)f.perm[c] * nrhs + k];
  for (const Supernode& sn : f.nodes) {
    const int ns = sn.ncol, ms = sn.nrow, N = sn.ld;
    const double* B = f.blocks64.data() + sn.blk_off;
    const int32_t* R = f.rows.data() + sn.row_off;
    for (int j = 0; j < ns; ++j)
      for (int k = 0; k < nrhs; ++k) {
        const double fj = y[(int64_t)(sn.col0 + j) * nrhs + k];
        for (int i = j; i < ns; ++i) z[(int64_t)(sn.col0 + i) * nrhs + k] += B[(int64_t)j * N + i] * fj;
        for (int a = 0; a < ms; ++a) y[(int64_t)R[a] * nrhs + k] -= B[(int64_t)j * N + ns + a] * fj;
      }
  }
  for (auto it = f.nodes.rbegin(); it != f.nodes.rend(); ++it) {
    const Supernode& sn = *it;
    const int ns = sn.ncol, ms = sn.nrow, N = sn.ld;
    const double* B = f.blocks64.data() + sn.blk_off;
    const int32_t* R = f.rows.data() + sn.row_off;
    for (int j = 0; j < ns; ++j)
      for (int k = 0; k < nrhs; ++k) {
        double acc = 0.0;
        for (int i = j; i < ns; ++i) acc += B[(int64_t)j * N + i] * z[(int64_t)(sn.col0 + i) * nrhs + k];
        for (int a = 0; a < ms; ++a) acc -= B[(int64_t)j * N + ns + a] * xs[(int64_t)R[a] * nrhs + k];
        xs[(int64_t)(sn.col0 + j) * nrhs + k] = acc;
      }
  }
  for (int64_t c = 0; c < nF; ++c)
    for (int k = 0; k < nrhs; ++k) x[(int64_t)f.perm[c] * nrhs + k] = xs[c * nrhs + k];
}

void run_threads(int count, const std::function<void(int)>& worker) {
  std::exception_ptr first;
  std::mutex mu;
  auto guarded = [&](int i) {
    try {
      worker(i);
    } catch (...) {
      std::lock_guard<std::mutex> lock(mu);
      if (!first) first = std::current_exception();
    }
  };
  std::vector<std::thread> pool;
  try {
    pool.reserve(count > 1 ? count - 1 : 0);
    for (int i = 1; i < count; ++i) pool.emplace_back(guarded, i);
  } catch (...) {
    std::lock_guard<std::mutex> lock(mu);
    if (!first) first = std::current_exception();
  }
  guarded(0);
  for (auto& th : pool) th.join();
  if (first) std::rethrow_exception(first);
}

}  // namespace ffa
