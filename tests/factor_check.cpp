// Host check of the library's factorization of the fixed W-step operator
// (csrc/ffa_factor.cpp: nested-dissection order, multifrontal Cholesky, blocks
// B_s = [inv(L_ss); L_rs inv(L_ss)]) on SPD matrices with the sparsity of 2D and
// 3D meshes and random, also strongly graded, positive weights:
//   * perm and iperm are inverse permutations; every structure row lies below its
//     supernode and the structures are ascending; the blocks are 16-byte aligned;
//   * the double blocks solve A x = b to a normwise backward error below 1e-14;
//   * the float blocks are the double blocks rounded;
//   * threads do not change the factor (bitwise);
//   * refactor on new values equals a fresh factorization of them;
//   * an indefinite matrix is refused with code 3.
// Prints "ok" or the first failure.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <random>
#include <string>
#include <vector>

#include "../paper_2107_05200_gb300/csrc/ffa_factor.h"

using namespace ffa;

static int fails = 0;
#define CHECK(cond, ...)                    \
  do {                                      \
    if (!(cond)) {                          \
      if (!fails) std::printf(__VA_ARGS__); \
      ++fails;                              \
    }                                       \
  } while (0)

struct Sparse {
  int n = 0;
  std::vector<int64_t> Ap;
  std::vector<int32_t> Ai;
  std::vector<double> Ax;
  std::vector<double> xyz;
};

// weighted graph Laplacian of a grid (4-neighbour in 2D, 6-neighbour in 3D, plus
// one diagonal per cell so that the pattern resembles a triangulation), edge
// weights exp(N(0, spread)), plus shift * (weighted degree) on the diagonal
static Sparse grid_operator(int nx, int ny, int nz, double spread, double shift, std::mt19937_64& rng) {
  Sparse S;
  S.n = nx * ny * nz;
  auto id = [&](int i, int j, int k) { return (k * ny + j) * nx + i; };
  std::normal_distribution<double> N(0.0, spread);
  std::vector<std::vector<std::pair<int, double>>> adj(S.n);
  auto edge = [&](int a, int b) {
    const double w = std::exp(N(rng));
    adj[a].push_back({b, -w});
    adj[b].push_back({a, -w});
  };
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        const int v = id(i, j, k);
        if (i + 1 < nx) edge(v, id(i + 1, j, k));
        if (j + 1 < ny) edge(v, id(i, j + 1, k));
        if (k + 1 < nz) edge(v, id(i, j, k + 1));
        if (i + 1 < nx && j + 1 < ny) edge(v, id(i + 1, j + 1, k));
        S.xyz.push_back(i);
        S.xyz.push_back(j);
        S.xyz.push_back(k);
      }
  S.Ap.assign(1, 0);
  for (int v = 0; v < S.n; ++v) {
    double deg = 0.0;
    for (auto& e : adj[v]) deg -= e.second;
    auto row = adj[v];
    row.push_back({v, deg * (1.0 + shift)});
    std::sort(row.begin(), row.end());
    for (auto& e : row) {
      S.Ai.push_back(e.first);
      S.Ax.push_back(e.second);
    }
    S.Ap.push_back((int64_t)S.Ai.size());
  }
  return S;
}

static FactorInput input(const Sparse& S, int leaf, int threads) {
  FactorInput in;
  in.nF = S.n;
  in.Ap = S.Ap.data();
  in.Ai = S.Ai.data();
  in.Ax = S.Ax.data();
  in.coords = S.xyz.data();
  in.leaf_size = leaf;
  in.threads = threads;
  in.keep_double = true;
  return in;
}

static void check_structure(const Factor& f, const std::string& tag) {
  std::vector<int> seen(f.nF, 0);
  for (int c = 0; c < f.nF; ++c) {
    CHECK(f.perm[c] >= 0 && f.perm[c] < f.nF && f.iperm[f.perm[c]] == c, "%s: perm/iperm at %d\n", tag.c_str(), c);
    if (f.perm[c] >= 0 && f.perm[c] < f.nF) seen[f.perm[c]]++;
  }
  CHECK(std::all_of(seen.begin(), seen.end(), [](int s) { return s == 1; }), "%s: perm is not a permutation\n",
        tag.c_str());
  int64_t cols = 0;
  for (size_t s = 0; s < f.nodes.size(); ++s) {
    const Supernode& sn = f.nodes[s];
    cols += sn.ncol;
    CHECK(sn.ld % 4 == 0 && sn.ld >= sn.ncol + sn.nrow && sn.blk_off % 4 == 0, "%s: node %zu layout\n", tag.c_str(), s);
    for (int a = 0; a < sn.nrow; ++a) {
      const int32_t r = f.rows[sn.row_off + a];
      CHECK(r >= sn.col0 + sn.ncol && r < f.nF, "%s: node %zu structure row %d\n", tag.c_str(), s, r);
      if (a > 0) CHECK(r > f.rows[sn.row_off + a - 1], "%s: node %zu structure not ascending\n", tag.c_str(), s);
    }
    if (sn.parent >= 0) CHECK((size_t)sn.parent > s, "%s: node %zu parent before child\n", tag.c_str(), s);
  }
  CHECK(cols == f.nF, "%s: supernodes cover %lld of %d columns\n", tag.c_str(), (long long)cols, f.nF);
}

static double backward_error(const Sparse& S, const Factor& f, std::mt19937_64& rng) {
  const int nrhs = 3;
  std::normal_distribution<double> N(0.0, 1.0);
  std::vector<double> b((size_t)S.n * nrhs), x((size_t)S.n * nrhs);
  for (double& v : b) v = N(rng);
  host_solve(f, b.data(), x.data(), nrhs);
  double rmax = 0.0, anorm = 0.0, xmax = 0.0, bmax = 0.0;
  for (int i = 0; i < S.n; ++i) {
    double arow = 0.0;
    for (int64_t q = S.Ap[i]; q < S.Ap[i + 1]; ++q) arow += std::fabs(S.Ax[q]);
    anorm = std::max(anorm, arow);
    for (int k = 0; k < nrhs; ++k) {
      double r = -b[(size_t)i * nrhs + k];
      for (int64_t q = S.Ap[i]; q < S.Ap[i + 1]; ++q) r += S.Ax[q] * x[(size_t)S.Ai[q] * nrhs + k];
      rmax = std::max(rmax, std::fabs(r));
      xmax = std::max(xmax, std::fabs(x[(size_t)i * nrhs + k]));
      bmax = std::max(bmax, std::fabs(b[(size_t)i * nrhs + k]));
    }
  }
  return rmax / (anorm * xmax + bmax);
}

int main() {
  std::mt19937_64 rng(5);
  struct Case { int nx, ny, nz; double spread; int leaf; };
  // the last case is a larger 3D grid (fronts up to about 1300 rows)
  const Case cases[] = {{23, 17, 1, 0.5, 16}, {31, 29, 1, 3.0, 64}, {9, 8, 7, 0.5, 16}, {12, 11, 10, 3.0, 64},
                        {30, 29, 28, 1.0, 64}};
  for (const Case& cs : cases) {
    const std::string tag = std::to_string(cs.nx) + "x" + std::to_string(cs.ny) + "x" + std::to_string(cs.nz) +
                            " spread " + std::to_string(cs.spread);
    Sparse S = grid_operator(cs.nx, cs.ny, cs.nz, cs.spread, 1e-3, rng);
    Factor f1, f4;
    std::string err;
    CHECK(build_factor(input(S, cs.leaf, 1), f1, err) == 0, "%s: build (1 thread): %s\n", tag.c_str(), err.c_str());
    CHECK(build_factor(input(S, cs.leaf, 4), f4, err) == 0, "%s: build (4 threads): %s\n", tag.c_str(), err.c_str());
    if (fails) break;
    check_structure(f1, tag);
    const double be = backward_error(S, f1, rng);
    CHECK(be < 1e-14, "%s: backward error %g\n", tag.c_str(), be);
    CHECK(f1.blocks.size() == f1.blocks64.size(), "%s: block sizes\n", tag.c_str());
    for (size_t k = 0; k < f1.blocks.size() && k < f1.blocks64.size(); ++k)
      if (f1.blocks[k] != static_cast<float>(f1.blocks64[k])) {
        CHECK(false, "%s: float block %zu is not the rounded double\n", tag.c_str(), k);
        break;
      }
    CHECK(f1.perm == f4.perm && f1.blocks64 == f4.blocks64, "%s: threads changed the factor\n", tag.c_str());
    // new values on the same pattern: refactor == a fresh factorization
    Sparse S2 = S;
    std::uniform_real_distribution<double> U(0.5, 2.0);
    std::vector<double> scale(S.n);
    for (double& v : scale) v = U(rng);
    for (int i = 0; i < S.n; ++i)
      for (int64_t q = S2.Ap[i]; q < S2.Ap[i + 1]; ++q) S2.Ax[q] = S.Ax[q] * std::sqrt(scale[i] * scale[S.Ai[q]]);
    Factor fr = f1, fresh;
    CHECK(refactor(input(S2, cs.leaf, 4), fr, err) == 0, "%s: refactor: %s\n", tag.c_str(), err.c_str());
    CHECK(build_factor(input(S2, cs.leaf, 1), fresh, err) == 0, "%s: build of new values: %s\n", tag.c_str(),
          err.c_str());
    CHECK(fr.perm == fresh.perm && fr.blocks64 == fresh.blocks64, "%s: refactor differs from a fresh factor\n",
          tag.c_str());
    const double be2 = backward_error(S2, fr, rng);
    CHECK(be2 < 1e-14, "%s: backward error after refactor %g\n", tag.c_str(), be2);
    // indefinite: the diagonal lowered below the weighted degree
    Sparse S3 = S;
    for (int i = 0; i < S.n; ++i)
      for (int64_t q = S3.Ap[i]; q < S3.Ap[i + 1]; ++q)
        if (S3.Ai[q] == i) S3.Ax[q] *= 0.5;
    Factor fi;
    CHECK(build_factor(input(S3, cs.leaf, 1), fi, err) == 3, "%s: indefinite matrix not refused\n", tag.c_str());
  }
  if (!fails) std::printf("ok\n");
  return fails ? 1 : 0;
}
