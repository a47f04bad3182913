// Nested-dissection ordering and multifrontal Cholesky of the W-step operator.
// See ffa_factor.h for the stored form.  Host code, run once per mesh and rho.
#include "ffa_factor.h"

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <functional>
#include <limits>
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
  std::vector<std::thread> pool;
  pool.reserve(t - 1);
  for (int i = 1; i < t; ++i) pool.emplace_back(worker);
  worker();
  for (auto& th : pool) th.join();
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

// Postorder numbering of the dissection tree into supernodes.
void number_tree(const std::vector<TreeNode>& tree, int t, Factor& f, std::vector<int>& tree2node) {
  // iterative postorder
  std::vector<std::pair<int, int>> st;  // (tree node, state)
  st.push_back({t, 0});
  while (!st.empty()) {
    auto& top = st.back();
    int id = top.first;
    if (top.second < 2) {
      int c = tree[id].child[top.second++];
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
inline double dot(const double* a, const double* b, int n) {
  double s0 = 0, s1 = 0, s2 = 0, s3 = 0;
  int k = 0;
  for (; k + 4 <= n; k += 4) {
    s0 += a[k] * b[k];
    s1 += a[k + 1] * b[k + 1];
    s2 += a[k + 2] * b[k + 2];
    s3 += a[k + 3] * b[k + 3];
  }
  for (; k < n; ++k) s0 += a[k] * b[k];
  return (s0 + s1) + (s2 + s3);
}

// Eliminate the first ns columns of the N x N front F; on return rows/cols
// [0, ns) hold L11, rows [ns, N) x cols [0, ns) hold L21 and the trailing lower
// triangle holds F22 - L21 L21^T.  Returns false if a pivot is not positive.
bool partial_cholesky(double* F, int N, int ns, int threads) {
  const int NB = 64;
  for (int k0 = 0; k0 < ns; k0 += NB) {
    const int k1 = std::min(ns, k0 + NB);
    // diagonal block, left-looking within the panel
    for (int k = k0; k < k1; ++k) {
      double* Fk = F + (int64_t)k * N;
      double dkk = Fk[k] - dot(Fk + k0, Fk + k0, k - k0);
      if (!(dkk > 0.0) || !std::isfinite(dkk)) return false;
      dkk = std::sqrt(dkk);
      Fk[k] = dkk;
      for (int i = k + 1; i < k1; ++i) {
        double* Fi = F + (int64_t)i * N;
        Fi[k] = (Fi[k] - dot(Fi + k0, Fk + k0, k - k0)) / dkk;
      }
    }
    // rows below the panel: row-wise triangular solve against the panel
    const int64_t nrows = N - k1;
    const int64_t work = nrows * (k1 - k0) * (k1 - k0);
    parallel_for(nrows, work > (1 << 20) ? threads : 1, 64, [&](int64_t b, int64_t e) {
      for (int64_t r = b; r < e; ++r) {
        double* Fi = F + (k1 + r) * N;
        for (int k = k0; k < k1; ++k) {
          const double* Fk = F + (int64_t)k * N;
          Fi[k] = (Fi[k] - dot(Fi + k0, Fk + k0, k - k0)) / Fk[k];
        }
      }
    });
    // trailing update of the lower triangle below/right of the panel
    const int w = k1 - k0;
    const int64_t tw = nrows * nrows / 2 * w;
    parallel_for(nrows, tw > (1 << 20) ? threads : 1, 16, [&](int64_t b, int64_t e) {
      for (int64_t r = b; r < e; ++r) {
        const int64_t i = k1 + r;
        double* Fi = F + i * N;
        const double* ai = Fi + k0;
        int64_t j = k1;
        for (; j + 4 <= i + 1; j += 4) {
          const double* b0 = F + j * N + k0;
          const double* b1 = b0 + N;
          const double* b2 = b1 + N;
          const double* b3 = b2 + N;
          double s0 = 0, s1 = 0, s2 = 0, s3 = 0;
          for (int k = 0; k < w; ++k) {
            double x = ai[k];
            s0 += x * b0[k];
            s1 += x * b1[k];
            s2 += x * b2[k];
            s3 += x * b3[k];
          }
          Fi[j] -= s0;
          Fi[j + 1] -= s1;
          Fi[j + 2] -= s2;
          Fi[j + 3] -= s3;
        }
        for (; j <= i; ++j) Fi[j] -= dot(ai, F + j * N + k0, w);
      }
    });
  }
  return true;
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
  std::vector<std::vector<double>> upd(nn);
  std::atomic<int> failed(-1);

  auto factor_node = [&](int s, NumericWork& wk, int dense_threads) {
    if (failed.load() >= 0) return;
    const Supernode& sn = f.nodes[s];
    const int ns = sn.ncol, ms = sn.nrow, N = ns + ms;
    const int32_t* R = f.rows.data() + sn.row_off;
    std::vector<double> F((int64_t)N * N, 0.0);
    for (int q = 0; q < ns; ++q) wk.pos[sn.col0 + q] = q;
    for (int q = 0; q < ms; ++q) wk.pos[R[q]] = ns + q;
    // original entries (lower triangle of the front)
    for (int q = 0; q < ns; ++q) {
      const int32_t c = sn.col0 + q;
      const int32_t old = f.perm[c];
      for (int64_t k = in.Ap[old]; k < in.Ap[old + 1]; ++k) {
        const int32_t r = f.iperm[in.Ai[k]];
        if (r < c) continue;
        F[(int64_t)wk.pos[r] * N + q] += in.Ax[k];
      }
    }
    // extend-add of the children's update matrices
    for (int ch : children[s]) {
      const Supernode& cn = f.nodes[ch];
      const int32_t* Rc = f.rows.data() + cn.row_off;
      const std::vector<double>& Uc = upd[ch];
      for (int a = 0; a < cn.nrow; ++a) {
        const int pa = wk.pos[Rc[a]];
        double* Fa = F.data() + (int64_t)pa * N;
        const double* Ua = Uc.data() + (int64_t)a * cn.nrow;
        for (int b = 0; b <= a; ++b) Fa[wk.pos[Rc[b]]] += Ua[b];
      }
      std::vector<double>().swap(upd[ch]);
    }
    for (int q = 0; q < ns; ++q) wk.pos[sn.col0 + q] = -1;
    for (int q = 0; q < ms; ++q) wk.pos[R[q]] = -1;
    if (!partial_cholesky(F.data(), N, ns, dense_threads)) {
      failed.store(s);
      return;
    }
    // update matrix for the parent
    if (ms > 0) {
      std::vector<double>& U = upd[s];
      U.assign((int64_t)ms * ms, 0.0);
      for (int a = 0; a < ms; ++a)
        for (int b = 0; b <= a; ++b) U[(int64_t)a * ms + b] = F[(int64_t)(ns + a) * N + ns + b];
    }
    if (ns == 0) return;
    // B_s = [inv(L11); L21 inv(L11)], column-major, leading dimension N
    std::vector<double> B((int64_t)N * ns, 0.0);
    const int64_t inv_work = (int64_t)ns * ns * ns;
    parallel_for(ns, inv_work > (1 << 21) ? dense_threads : 1, 8, [&](int64_t b, int64_t e) {
      for (int64_t j = b; j < e; ++j) {
        double* x = B.data() + j * N;  // column j, rows [0, ns)
        x[j] = 1.0 / F[j * N + j];
        for (int64_t i = j + 1; i < ns; ++i) {
          const double* Li = F.data() + i * N;
          double sacc = 0.0;
          for (int64_t k = j; k < i; ++k) sacc += Li[k] * x[k];
          x[i] = -sacc / Li[i];
        }
      }
    });
    const int64_t m_work = (int64_t)ms * ns * ns;
    parallel_for(ms, m_work > (1 << 21) ? dense_threads : 1, 8, [&](int64_t b, int64_t e) {
      for (int64_t a = b; a < e; ++a) {
        const double* La = F.data() + (int64_t)(ns + a) * N;
        for (int j = 0; j < ns; ++j) {
          const double* col = B.data() + (int64_t)j * N;
          B[(int64_t)j * N + ns + a] = dot(La + j, col + j, ns - j);
        }
      }
    });
    for (int j = 0; j < ns; ++j) {
      float* dst = f.blocks.data() + sn.blk_off + (int64_t)j * sn.ld;
      const double* src = B.data() + (int64_t)j * N;
      for (int i = 0; i < N; ++i) dst[i] = static_cast<float>(src[i]);
      if (in.keep_double)
        std::copy(src, src + N, f.blocks64.begin() + sn.blk_off + (int64_t)j * sn.ld);
    }
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
    std::vector<std::thread> pool;
    const int tcount = std::max(1, std::min<int>(threads, (int)tasks.size()));
    for (int i = 1; i < tcount; ++i) pool.emplace_back(worker);
    worker();
    for (auto& th : pool) th.join();
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

}  // namespace ffa
