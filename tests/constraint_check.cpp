// Host check of the library's constraint setup (csrc/ffa_constraint_host.cpp):
// the split of A into free and pinned parts, the inverse of the Schur complement
// and its refusal of dependent rows, and, on dense random problems, that the
// projection the GPU applies, X0 - Z S^-1 (A_F X0 - b') with Z = L^-1 A_F^T,
// S = A_F Z, equals the solution of the KKT system [L A_F^T; A_F 0] solved here
// by Gaussian elimination with partial pivoting.  Prints "ok" or the first failure.
#include <cmath>
#include <cstdio>
#include <random>
#include <vector>

#include "../paper_2107_05200_gb300/csrc/ffa_constraint_host.h"

using namespace ffa;

static int fails = 0;
#define CHECK(cond, ...)                    \
  do {                                      \
    if (!(cond)) {                          \
      if (!fails) std::printf(__VA_ARGS__); \
      ++fails;                              \
    }                                       \
  } while (0)

// x = M^-1 b for a dense n x n M (row-major), Gaussian elimination with partial pivoting
static std::vector<double> dense_solve(std::vector<double> M, std::vector<double> b, int n) {
  for (int k = 0; k < n; ++k) {
    int piv = k;
    for (int i = k + 1; i < n; ++i)
      if (std::fabs(M[(size_t)i * n + k]) > std::fabs(M[(size_t)piv * n + k])) piv = i;
    if (piv != k) {
      for (int j = 0; j < n; ++j) std::swap(M[(size_t)k * n + j], M[(size_t)piv * n + j]);
      std::swap(b[k], b[piv]);
    }
    for (int i = k + 1; i < n; ++i) {
      const double f = M[(size_t)i * n + k] / M[(size_t)k * n + k];
      for (int j = k; j < n; ++j) M[(size_t)i * n + j] -= f * M[(size_t)k * n + j];
      b[i] -= f * b[k];
    }
  }
  std::vector<double> x(n);
  for (int i = n - 1; i >= 0; --i) {
    double a = b[i];
    for (int j = i + 1; j < n; ++j) a -= M[(size_t)i * n + j] * x[j];
    x[i] = a / M[(size_t)i * n + i];
  }
  return x;
}

int main() {
  std::mt19937_64 rng(11);
  std::normal_distribution<double> N(0.0, 1.0);

  // 1. the split: 8 vertices, vertices 0 and 5 pinned (slots 1 and 0), the free
  //    ones eliminated in the order 7 3 1 6 2 4
  {
    const std::vector<int32_t> v2e = {-1, 2, 4, 1, 5, -1, 3, 0};
    const std::vector<int32_t> slot_of = {1, -1, -1, -1, -1, 0, -1, -1};
    // row 0: W3 + 2 W1 + W3 (a repeated column); row 1: W5 - W1 (its free column
    // equals row 0's last one, which must not merge across rows); row 2: W0 only;
    // row 3: empty
    const std::vector<int64_t> ptr = {0, 3, 5, 6, 6};
    const std::vector<int32_t> col = {3, 1, 3, 5, 1, 0};
    const std::vector<double> val = {1.0, 2.0, 1.0, 1.0, -1.0, 4.0};
    ConstraintSplit sp;
    split_constraints(4, ptr.data(), col.data(), val.data(), v2e, slot_of, sp);
    const std::vector<int64_t> want_ptr = {0, 2, 3, 3, 3};
    const std::vector<int32_t> want_col = {1, 2, 2};  // row 0: e(3) = 1, e(1) = 2; row 1: e(1) = 2
    const std::vector<double> want_val = {2.0, 2.0, -1.0};
    CHECK(sp.fptr == want_ptr, "split: row pointers\n");
    CHECK(sp.fcol == want_col, "split: columns\n");
    CHECK(sp.fval == want_val, "split: values\n");
    CHECK(sp.pin.size() == 2 && sp.pin[0].row == 1 && sp.pin[0].slot == 0 && sp.pin[0].val == 1.0 &&
              sp.pin[1].row == 2 && sp.pin[1].slot == 1 && sp.pin[1].val == 4.0,
          "split: pinned entries\n");
  }

  // 2. S^-1 of a random SPD S, and the refusals
  {
    const int c = 40;
    std::vector<double> B((size_t)c * c), S((size_t)c * c, 0.0), Sinv;
    for (double& x : B) x = N(rng);
    for (int i = 0; i < c; ++i)
      for (int j = 0; j < c; ++j) {
        double s = i == j ? 0.5 : 0.0;
        for (int k = 0; k < c; ++k) s += B[(size_t)i * c + k] * B[(size_t)j * c + k];
        S[(size_t)i * c + j] = s;
      }
    CHECK(schur_inverse(c, S, Sinv) == -1, "SPD S refused\n");
    double err = 0.0;
    for (int i = 0; i < c; ++i)
      for (int j = 0; j < c; ++j) {
        double s = 0.0;
        for (int k = 0; k < c; ++k) s += S[(size_t)i * c + k] * Sinv[(size_t)k * c + j];
        err = std::fmax(err, std::fabs(s - (i == j ? 1.0 : 0.0)));
      }
    CHECK(err < 1e-9, "S S^-1 - I = %g\n", err);
    // rows of A with row 3 = row 1 - 2 row 0: S = A A^T is singular from row 3 on
    const int r = 6, n = 10;
    std::vector<double> A((size_t)r * n), G((size_t)r * r);
    for (double& x : A) x = N(rng);
    for (int j = 0; j < n; ++j) A[(size_t)3 * n + j] = A[(size_t)1 * n + j] - 2.0 * A[j];
    for (int i = 0; i < r; ++i)
      for (int j = 0; j < r; ++j) {
        double s = 0.0;
        for (int k = 0; k < n; ++k) s += A[(size_t)i * n + k] * A[(size_t)j * n + k];
        G[(size_t)i * r + j] = s;
      }
    CHECK(schur_inverse(r, G, Sinv) == 3, "dependent row 3 not found\n");
    std::vector<double> Z2 = {1.0, 0.0, 0.0, 0.0};
    CHECK(schur_inverse(2, Z2, Sinv) == 1, "zero row 1 not refused\n");
  }

  // 3. the projection equals the KKT solution: L = B B^T + I (n x n), A_F (c x n),
  //    d right-hand-side columns
  for (int trial = 0; trial < 5; ++trial) {
    const int n = 30, c = 1 + trial * 2, d = 3;
    std::vector<double> B((size_t)n * n), L((size_t)n * n), A((size_t)c * n), rhs((size_t)n * d), bp((size_t)c * d);
    for (double& x : B) x = N(rng);
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        double s = i == j ? 1.0 : 0.0;
        for (int k = 0; k < n; ++k) s += B[(size_t)i * n + k] * B[(size_t)j * n + k];
        L[(size_t)i * n + j] = s;
      }
    for (double& x : A) x = N(rng);
    for (double& x : rhs) x = N(rng);
    for (double& x : bp) x = N(rng);
    // GPU formula: X0 = L^-1 rhs, Z = L^-1 A^T, S = A Z, X = X0 - Z S^-1 (A X0 - b')
    std::vector<double> X((size_t)n * d), Z((size_t)n * c), S((size_t)c * c, 0.0), Sinv;
    for (int k = 0; k < d; ++k) {
      std::vector<double> col(n);
      for (int i = 0; i < n; ++i) col[i] = rhs[(size_t)i * d + k];
      const std::vector<double> x = dense_solve(L, col, n);
      for (int i = 0; i < n; ++i) X[(size_t)i * d + k] = x[i];
    }
    for (int r = 0; r < c; ++r) {
      std::vector<double> col(n);
      for (int i = 0; i < n; ++i) col[i] = A[(size_t)r * n + i];
      const std::vector<double> z = dense_solve(L, col, n);
      for (int i = 0; i < n; ++i) Z[(size_t)i * c + r] = z[i];
    }
    for (int r = 0; r < c; ++r)
      for (int q = 0; q < c; ++q)
        for (int i = 0; i < n; ++i) S[(size_t)r * c + q] += A[(size_t)r * n + i] * Z[(size_t)i * c + q];
    CHECK(schur_inverse(c, S, Sinv) == -1, "projection trial %d: S refused\n", trial);
    for (int k = 0; k < d; ++k) {
      std::vector<double> t(c), nu(c, 0.0);
      for (int r = 0; r < c; ++r) {
        double s = -bp[(size_t)r * d + k];
        for (int i = 0; i < n; ++i) s += A[(size_t)r * n + i] * X[(size_t)i * d + k];
        t[r] = s;
      }
      for (int r = 0; r < c; ++r)
        for (int q = 0; q < c; ++q) nu[r] += Sinv[(size_t)r * c + q] * t[q];
      // KKT: [L A^T; A 0] [x; lambda] = [rhs; b']
      const int K = n + c;
      std::vector<double> M((size_t)K * K, 0.0), f(K);
      for (int i = 0; i < n; ++i) {
        for (int j = 0; j < n; ++j) M[(size_t)i * K + j] = L[(size_t)i * n + j];
        for (int r = 0; r < c; ++r) M[(size_t)i * K + n + r] = M[(size_t)(n + r) * K + i] = A[(size_t)r * n + i];
        f[i] = rhs[(size_t)i * d + k];
      }
      for (int r = 0; r < c; ++r) f[n + r] = bp[(size_t)r * d + k];
      const std::vector<double> sol = dense_solve(M, f, K);
      double err = 0.0, ref = 0.0;
      for (int i = 0; i < n; ++i) {
        double x = X[(size_t)i * d + k];
        for (int r = 0; r < c; ++r) x -= Z[(size_t)i * c + r] * nu[r];
        err = std::fmax(err, std::fabs(x - sol[i]));
        ref = std::fmax(ref, std::fabs(sol[i]));
      }
      CHECK(err <= 1e-10 * ref, "projection trial %d column %d: %g\n", trial, k, err / ref);
    }
  }

  if (!fails) std::printf("ok\n");
  return fails ? 1 : 0;
}
