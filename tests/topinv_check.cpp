// Host check of the top-of-tree inverse (ffa_topinv.h) on the factors of grid
// Laplacians:
//   * the plan: T is the set of supernodes with columns on the top k levels, in
//     node order with contiguous positions; lo(s) is the first position of s's T
//     subtree; the structure rows map to their T positions; T is closed under
//     ancestors; the automatic choice satisfies its byte rule; the product's work
//     units cover every lower tile of S^-1 exactly once;
//   * the setup's arithmetic, emulated in double from the float blocks (G = I,
//     F_s = inv(L_ss) G_s, G_r -= (L_rs inv(L_ss)) G_s, S^-1 = F^T F over the lower
//     tiles): it equals the T block of the solution of L_FF X = [0; I] from a dense
//     Cholesky factorization of L_FF, which is S^-1 by block elimination, to float
//     rounding of the blocks.
// Prints "ok" and exits 0, or prints the first violation and exits 1.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdio>
#include <string>
#include <vector>

#include "../paper_2107_05200_gb300/csrc/ffa_factor.h"
#include "../paper_2107_05200_gb300/csrc/ffa_topinv.h"

using namespace ffa;

static int fail(const std::string& what) {
  std::printf("FAIL %s\n", what.c_str());
  return 1;
}

// 7-point (3D) or 5-point (2D) Laplacian of a grid with a positive shift
static void grid_laplacian(int nx, int ny, int nz, std::vector<int64_t>& Ap, std::vector<int32_t>& Ai,
                           std::vector<double>& Ax, std::vector<double>& xyz) {
  auto id = [&](int i, int j, int k) { return (k * ny + j) * nx + i; };
  Ap.assign(1, 0);
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        std::vector<std::pair<int, double>> row;
        const int nb[6][3] = {{-1, 0, 0}, {1, 0, 0}, {0, -1, 0}, {0, 1, 0}, {0, 0, -1}, {0, 0, 1}};
        for (auto& d : nb) {
          const int a = i + d[0], b = j + d[1], c = k + d[2];
          if (a < 0 || b < 0 || c < 0 || a >= nx || b >= ny || c >= nz) continue;
          row.push_back({id(a, b, c), -1.0});
        }
        row.push_back({id(i, j, k), (nz > 1 ? 6.0 : 4.0) + 0.05});
        std::sort(row.begin(), row.end());
        for (auto& e : row) {
          Ai.push_back(e.first);
          Ax.push_back(e.second);
        }
        Ap.push_back((int64_t)Ai.size());
        xyz.push_back(i);
        xyz.push_back(j);
        xyz.push_back(k);
      }
}

// the plan's structure against its definition
static bool check_plan(const Factor& f, int k, const TopInvPlan& P, std::string& err) {
  const int nn = (int)f.nodes.size();
  std::vector<int32_t> T;
  for (int s = 0; s < nn; ++s)
    if (f.nodes[s].ncol > 0 && f.nodes[s].level >= f.n_levels - k) T.push_back(s);
  if (P.levels != k || P.nodes != T) return err = "T is not the top-level supernodes in node order", false;
  std::vector<int> posof(nn, -1);
  int32_t next = 0;
  for (size_t q = 0; q < T.size(); ++q) {
    if (P.pos[q] != next) return err = "positions not contiguous in node order", false;
    posof[T[q]] = (int)q;
    next += f.nodes[T[q]].ncol;
  }
  if (P.nT != next) return err = "nT", false;
  for (size_t q = 0; q < T.size(); ++q) {
    const int s = T[q];
    for (int a = f.nodes[s].parent; a >= 0; a = f.nodes[a].parent)
      if (f.nodes[a].ncol > 0 && posof[a] < 0) return err = "T not closed under ancestors", false;
    int lo = INT_MAX;
    for (size_t u = 0; u < T.size(); ++u) {
      int a = T[u];
      while (a >= 0 && a != s) a = f.nodes[a].parent;
      if (a == s) lo = std::min(lo, P.pos[u]);
    }
    if (P.lo[q] != lo) return err = "lo", false;
    const Supernode& sn = f.nodes[s];
    if (P.rmap_off[q + 1] - P.rmap_off[q] != sn.nrow) return err = "rmap size", false;
    for (int i = 0; i < sn.nrow; ++i) {
      const int r = f.rows[sn.row_off + i];
      int owner = -1;
      for (size_t u = 0; u < T.size(); ++u) {
        const Supernode& t = f.nodes[T[u]];
        if (r >= t.col0 && r < t.col0 + t.ncol) owner = (int)u;
      }
      if (owner < 0) return err = "structure row outside T", false;
      if (P.rmap[P.rmap_off[q] + i] != P.pos[owner] + (r - f.nodes[T[owner]].col0)) return err = "rmap", false;
    }
  }
  const int64_t tiles = (P.nT + kTiTile - 1) / kTiTile;
  if (P.tile_bytes != tiles * (tiles + 1) / 2 * kTiTile * kTiTile * 4) return err = "tile bytes", false;
  return true;
}

// the setup's steps in double from the float blocks: S^-1 (nT x nT, full)
static std::vector<double> emulate(const Factor& f, const TopInvPlan& P) {
  const int n = P.nT;
  std::vector<double> G((size_t)n * n, 0.0), F((size_t)n * n, 0.0);   // column-major
  for (int p = 0; p < n; ++p) G[(size_t)p * n + p] = 1.0;
  for (size_t q = 0; q < P.nodes.size(); ++q) {
    const Supernode& sn = f.nodes[P.nodes[q]];
    const int ns = sn.ncol, pos = P.pos[q], lo = P.lo[q], c1 = pos + ns;
    const float* B = f.blocks.data() + sn.blk_off;
    for (int c = lo; c < c1; ++c) {
      for (int r = 0; r < ns; ++r) {
        double a = 0.0;
        for (int k = 0; k <= r; ++k) a += (double)B[(size_t)k * sn.ld + r] * G[(size_t)c * n + pos + k];
        F[(size_t)c * n + pos + r] = a;
      }
      for (int i = 0; i < sn.nrow; ++i) {
        double a = 0.0;
        for (int k = 0; k < ns; ++k) a += (double)B[(size_t)k * sn.ld + ns + i] * G[(size_t)c * n + pos + k];
        G[(size_t)c * n + P.rmap[P.rmap_off[q] + i]] -= a;
      }
    }
  }
  std::vector<double> S((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j <= i; ++j) {
      double a = 0.0;
      for (int k = i; k < n; ++k) a += F[(size_t)i * n + k] * F[(size_t)j * n + k];
      S[(size_t)j * n + i] = S[(size_t)i * n + j] = a;
    }
  return S;
}

// dense Cholesky of L_FF in the eliminated order, then the T block of L^-1 [0; I_T]
static std::vector<double> reference(const Factor& f, const TopInvPlan& P, const std::vector<int64_t>& Ap,
                                     const std::vector<int32_t>& Ai, const std::vector<double>& Ax) {
  const int N = f.nF;
  std::vector<double> A((size_t)N * N, 0.0);
  for (int i = 0; i < N; ++i)
    for (int64_t e = Ap[i]; e < Ap[i + 1]; ++e) A[(size_t)f.iperm[i] * N + f.iperm[Ai[e]]] = Ax[e];
  for (int j = 0; j < N; ++j) {   // lower Cholesky in place (row-major, L[i][j], i >= j)
    double d = A[(size_t)j * N + j];
    for (int k = 0; k < j; ++k) d -= A[(size_t)j * N + k] * A[(size_t)j * N + k];
    d = std::sqrt(d);
    A[(size_t)j * N + j] = d;
    for (int i = j + 1; i < N; ++i) {
      double a = A[(size_t)i * N + j];
      for (int k = 0; k < j; ++k) a -= A[(size_t)i * N + k] * A[(size_t)j * N + k];
      A[(size_t)i * N + j] = a / d;
    }
  }
  const std::vector<int32_t> tpos = top_positions(f, P);
  std::vector<int32_t> tcol(P.nT);
  for (int c = 0; c < N; ++c)
    if (tpos[c] >= 0) tcol[tpos[c]] = c;
  const int n = P.nT;
  std::vector<double> S((size_t)n * n), x(N);
  for (int j = 0; j < n; ++j) {
    std::fill(x.begin(), x.end(), 0.0);
    x[tcol[j]] = 1.0;
    for (int i = 0; i < N; ++i) {   // L y = b
      double a = x[i];
      for (int k = 0; k < i; ++k) a -= A[(size_t)i * N + k] * x[k];
      x[i] = a / A[(size_t)i * N + i];
    }
    for (int i = N - 1; i >= 0; --i) {   // L^T x = y
      double a = x[i];
      for (int k = i + 1; k < N; ++k) a -= A[(size_t)k * N + i] * x[k];
      x[i] = a / A[(size_t)i * N + i];
    }
    for (int p = 0; p < n; ++p) S[(size_t)j * n + p] = x[tcol[p]];
  }
  return S;
}

// every lower tile (J <= I < tiles) lies in exactly one work unit of the product
static bool check_units(int tiles, std::string& err) {
  const std::vector<int32_t> u = top_product_units(tiles);
  std::vector<int> hit((size_t)tiles * tiles, 0);
  for (size_t q = 0; q + 1 < u.size(); q += 2)
    for (int i = 0; i < kTiUnitRows; ++i)
      for (int j = 0; j < kTiUnitCols; ++j) {
        const int I = kTiUnitRows * u[q] + i, J = kTiUnitCols * u[q + 1] + j;
        if (I < tiles && J <= I) ++hit[(size_t)I * tiles + J];
      }
  for (int I = 0; I < tiles; ++I)
    for (int J = 0; J < tiles; ++J)
      if (hit[(size_t)I * tiles + J] != (J <= I ? 1 : 0)) return err = "work units at " + std::to_string(tiles) + " tiles", false;
  return true;
}

int main() {
  {
    std::string err;
    for (int tiles : {1, 2, 3, 4, 5, 7, 8, 9, 146, 147, 256})
      if (!check_units(tiles, err)) return fail(err);
  }
  struct Grid { int nx, ny, nz, leaf; };
  const Grid grids[] = {{6, 6, 6, 8}, {10, 9, 8, 16}, {30, 30, 1, 16}, {5, 4, 3, 4}};
  int checked = 0;
  for (const Grid& g : grids) {
    std::vector<int64_t> Ap;
    std::vector<int32_t> Ai;
    std::vector<double> Ax, xyz;
    grid_laplacian(g.nx, g.ny, g.nz, Ap, Ai, Ax, xyz);
    FactorInput in;
    in.nF = g.nx * g.ny * g.nz;
    in.Ap = Ap.data();
    in.Ai = Ai.data();
    in.Ax = Ax.data();
    in.coords = xyz.data();
    in.leaf_size = g.leaf;
    Factor f;
    std::string err;
    if (build_factor(in, f, err) != 0) return fail("factor: " + err);
    const std::string tag = "grid " + std::to_string(g.nx) + "x" + std::to_string(g.ny) + "x" + std::to_string(g.nz);
    // explicit k, the automatic choice, and the refusals
    std::vector<int> ks = {1, 2, 3, f.n_levels - 1, -1};
    for (int k : ks) {
      if (k == 0 || k >= f.n_levels) continue;
      TopInvPlan P;
      if (!plan_top_inverse(f, k, P, err)) {
        if (k > 0 && P.levels == 0 && err.find("top_inverse_levels") != std::string::npos) continue;   // over a limit
        return fail(tag + " k " + std::to_string(k) + ": " + err);
      }
      if (P.levels == 0) {
        if (k > 0) return fail(tag + " explicit k not planned");
        continue;
      }
      if (k < 0 && P.tile_bytes > P.factor_bytes) return fail(tag + " automatic choice breaks its byte rule");
      if (!check_plan(f, P.levels, P, err)) return fail(tag + " k " + std::to_string(P.levels) + ": " + err);
      const std::vector<double> S = emulate(f, P), R = reference(f, P, Ap, Ai, Ax);
      double md = 0.0, mr = 0.0;
      for (size_t i = 0; i < S.size(); ++i) {
        md = std::max(md, std::fabs(S[i] - R[i]));
        mr = std::max(mr, std::fabs(R[i]));
      }
      if (!(md <= 2e-5 * mr)) return fail(tag + " k " + std::to_string(P.levels) + ": S^-1 off by " + std::to_string(md / mr));
      ++checked;
    }
    TopInvPlan P;
    if (plan_top_inverse(f, f.n_levels, P, err) || P.levels != 0) return fail(tag + " k = levels accepted");
  }
  std::printf("ok %d plans\n", checked);
  return 0;
}
