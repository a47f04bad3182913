// Host check of the library's operator assembly (csrc/ffa_operator_host.cpp):
//   * element_geometry: an affine map's Jacobian is reproduced exactly (J = A^T,
//     column k the gradient of coordinate k) on triangles and tetrahedra, an
//     isometric copy of a planar triangle in R^3 has a rotation as its intrinsic
//     Jacobian, w is the area / volume, degenerate elements are refused;
//   * assemble_operator (one thread and, on the larger grid, several): L_FF is
//     symmetric with ascending columns, L 1 = 0 (rows of [L_FF L_FC] sum to zero),
//     and the quadratic form and the pin block equal sum_i mu_i |G_i x|^2 and
//     (G^T M G x)_F computed element by element;
//   * operator_arrays: the ELL rows in elimination order hold exactly the CSR row
//     of perm[c] (padding: own column, value 0), L_FC by elimination row, and L_CF
//     its transpose.
// Prints "ok" or the first failure.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <map>
#include <random>
#include <string>
#include <vector>

#include "../paper_2107_05200_gb300/csrc/ffa_factor.h"
#include "../paper_2107_05200_gb300/csrc/ffa_operator_host.h"

using namespace ffa;

static int fails = 0;
#define CHECK(cond, ...)                    \
  do {                                      \
    if (!(cond)) {                          \
      if (!fails) std::printf(__VA_ARGS__); \
      ++fails;                              \
    }                                       \
  } while (0)

// gradient of the hat function of local vertex j (0..d) from the stored 1..d
static void hat(const double g[3][3], int d, int j, double out[3]) {
  for (int a = 0; a < d; ++a) {
    if (j > 0) out[a] = g[j - 1][a];
    else {
      out[a] = 0.0;
      for (int jj = 0; jj < d; ++jj) out[a] -= g[jj][a];
    }
  }
}

static void check_geometry(std::mt19937_64& rng) {
  std::normal_distribution<double> N(0.0, 1.0);
  for (int d = 2; d <= 3; ++d)
    for (int trial = 0; trial < 50; ++trial) {
      std::vector<double> V((d + 1) * d);
      for (double& x : V) x = N(rng);
      const int32_t t[4] = {0, 1, 2, 3};
      double g[3][3], w;
      if (!element_geometry(d, d, V.data(), t, g, w)) {
        CHECK(false, "geometry refused a random element\n");
        continue;
      }
      double A[3][3], c[3];
      for (int k = 0; k < d; ++k) {
        c[k] = N(rng);
        for (int a = 0; a < d; ++a) A[k][a] = N(rng);
      }
      double J[3][3] = {{0}};
      for (int j = 0; j <= d; ++j) {
        double h[3], Wj[3];
        hat(g, d, j, h);
        for (int k = 0; k < d; ++k) {
          Wj[k] = c[k];
          for (int a = 0; a < d; ++a) Wj[k] += A[k][a] * V[j * d + a];
        }
        for (int a = 0; a < d; ++a)
          for (int k = 0; k < d; ++k) J[a][k] += h[a] * Wj[k];
      }
      for (int a = 0; a < d; ++a)
        for (int k = 0; k < d; ++k)
          CHECK(std::fabs(J[a][k] - A[k][a]) < 1e-9, "d=%d: affine Jacobian entry (%d,%d) off by %g\n", d, a, k,
                J[a][k] - A[k][a]);
      // measure: |(v1-v0) x (v2-v0)| / 2 or |det[v1-v0, v2-v0, v3-v0]| / 6
      double e[3][3];
      for (int j = 0; j < d; ++j)
        for (int a = 0; a < d; ++a) e[j][a] = V[(j + 1) * d + a] - V[a];
      const double meas = d == 2 ? std::fabs(e[0][0] * e[1][1] - e[0][1] * e[1][0]) / 2.0
                                 : std::fabs(e[0][0] * (e[1][1] * e[2][2] - e[1][2] * e[2][1]) -
                                             e[0][1] * (e[1][0] * e[2][2] - e[1][2] * e[2][0]) +
                                             e[0][2] * (e[1][0] * e[2][1] - e[1][1] * e[2][0])) / 6.0;
      CHECK(std::fabs(w - meas) <= 1e-12 * meas, "d=%d: measure %g vs %g\n", d, w, meas);
    }
  // a planar triangle p_j rotated and moved into R^3: the intrinsic Jacobian of
  // the map back to p_j is a rotation or a reflection, and w is its area
  for (int trial = 0; trial < 50; ++trial) {
    double p[3][2];
    for (auto& q : p)
      for (double& x : q) x = N(rng);
    double ax[3] = {N(rng), N(rng), N(rng)};
    const double nax = std::sqrt(ax[0] * ax[0] + ax[1] * ax[1] + ax[2] * ax[2]);
    for (double& x : ax) x /= nax;
    const double th = N(rng), co = std::cos(th), si = std::sin(th), C = 1 - co;
    const double R[3][3] = {{co + ax[0] * ax[0] * C, ax[0] * ax[1] * C - ax[2] * si, ax[0] * ax[2] * C + ax[1] * si},
                            {ax[1] * ax[0] * C + ax[2] * si, co + ax[1] * ax[1] * C, ax[1] * ax[2] * C - ax[0] * si},
                            {ax[2] * ax[0] * C - ax[1] * si, ax[2] * ax[1] * C + ax[0] * si, co + ax[2] * ax[2] * C}};
    std::vector<double> V(9);
    for (int j = 0; j < 3; ++j)
      for (int a = 0; a < 3; ++a) V[j * 3 + a] = R[a][0] * p[j][0] + R[a][1] * p[j][1] + 0.5 * a;
    const int32_t t[3] = {0, 1, 2};
    double g[3][3], w;
    CHECK(element_geometry(2, 3, V.data(), t, g, w), "surface triangle refused\n");
    double J[2][2] = {{0}};
    for (int j = 0; j < 3; ++j) {
      double h[3];
      hat(g, 2, j, h);
      for (int a = 0; a < 2; ++a)
        for (int k = 0; k < 2; ++k) J[a][k] += h[a] * p[j][k];
    }
    for (int a = 0; a < 2; ++a)
      for (int b = 0; b < 2; ++b) {
        const double s = J[0][a] * J[0][b] + J[1][a] * J[1][b];
        CHECK(std::fabs(s - (a == b ? 1.0 : 0.0)) < 1e-9, "surface Jacobian is not orthogonal\n");
      }
    const double area = 0.5 * std::fabs((p[1][0] - p[0][0]) * (p[2][1] - p[0][1]) - (p[1][1] - p[0][1]) * (p[2][0] - p[0][0]));
    CHECK(std::fabs(w - area) <= 1e-12 * area, "surface area %g vs %g\n", w, area);
  }
  // degenerate: collinear triangle, flat tetrahedron
  {
    const double V2[6] = {0, 0, 1, 1, 2, 2};
    const double V3[12] = {0, 0, 0, 1, 0, 0, 0, 1, 0, 1, 1, 0};
    const int32_t t[4] = {0, 1, 2, 3};
    double g[3][3], w;
    CHECK(!element_geometry(2, 2, V2, t, g, w), "collinear triangle accepted\n");
    CHECK(!element_geometry(3, 3, V3, t, g, w), "flat tetrahedron accepted\n");
  }
}

// a jittered nx x ny grid of triangles (two per cell), its left column pinned;
// grids above a few thousand free vertices are assembled by several threads
static void check_operator(std::mt19937_64& rng, int nx, int ny) {
  const int d = 2, n = nx * ny;
  std::uniform_real_distribution<double> J(-0.2, 0.2), M(0.5, 3.0);
  std::vector<double> V(n * 2);
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
      V[(j * nx + i) * 2] = i + J(rng);
      V[(j * nx + i) * 2 + 1] = j + J(rng);
    }
  std::vector<int32_t> T;
  for (int j = 0; j + 1 < ny; ++j)
    for (int i = 0; i + 1 < nx; ++i) {
      const int a = j * nx + i, b = a + 1, c = a + nx, e = c + 1;
      T.insert(T.end(), {a, b, e, a, e, c});
    }
  const int m = (int)T.size() / 3;
  OperatorHost H;
  H.n = n;
  H.m = m;
  H.d = d;
  H.g.resize((size_t)m * d * d);
  std::vector<double> mu(m);
  for (int i = 0; i < m; ++i) {
    double g[3][3], w;
    CHECK(element_geometry(d, d, V.data(), T.data() + 3 * i, g, w), "grid element refused\n");
    for (int j = 0; j < d; ++j)
      for (int a = 0; a < d; ++a) H.g[(size_t)i * d * d + j * d + a] = g[j][a];
    mu[i] = M(rng) * w;
  }
  H.T = T;
  H.v2pin.assign(n, -1);
  int n_pin = 0;
  for (int j = 0; j < ny; ++j) H.v2pin[j * nx] = n_pin++;
  H.n_pin = n_pin;
  H.free_of.assign(n, -1);
  for (int v = 0; v < n; ++v)
    if (H.v2pin[v] < 0) {
      H.free_of[v] = (int32_t)H.free_vertex.size();
      H.free_vertex.push_back(v);
    }
  const int nF = (int)H.free_vertex.size();
  H.nF = nF;
  H.inc_ptr.assign(n + 1, 0);
  for (int32_t v : T) H.inc_ptr[v + 1]++;
  for (int v = 0; v < n; ++v) H.inc_ptr[v + 1] += H.inc_ptr[v];
  H.inc.resize(H.inc_ptr[n]);
  {
    std::vector<int64_t> fill(H.inc_ptr.begin(), H.inc_ptr.end() - 1);
    for (int i = 0; i < m; ++i)
      for (int j = 0; j <= d; ++j) H.inc[fill[T[3 * i + j]]++] = i * 3 + j;
  }
  std::vector<int64_t> Ap, Cp;
  std::vector<int32_t> Ai, Ci;
  std::vector<double> Ax, Cx;
  assemble_operator(H, mu.data(), Ap, Ai, Ax, Cp, Ci, Cx);

  std::map<std::pair<int, int>, double> LFF;
  for (int f = 0; f < nF; ++f) {
    double sum = 0.0, scale = 0.0;
    for (int64_t q = Ap[f]; q < Ap[f + 1]; ++q) {
      if (q > Ap[f]) CHECK(Ai[q] > Ai[q - 1], "row %d columns not ascending\n", f);
      LFF[{f, Ai[q]}] = Ax[q];
      sum += Ax[q];
      scale = std::max(scale, std::fabs(Ax[q]));
    }
    for (int64_t q = Cp[f]; q < Cp[f + 1]; ++q) sum += Cx[q];
    CHECK(std::fabs(sum) <= 1e-12 * scale, "row %d of [L_FF L_FC] sums to %g\n", f, sum);
  }
  for (auto& e : LFF) {
    auto it = LFF.find({e.first.second, e.first.first});
    CHECK(it != LFF.end() && it->second == e.second, "L_FF not symmetric at (%d,%d)\n", e.first.first,
          e.first.second);
  }
  // x on the free vertices only: x^T L_FF x = sum_i mu_i |G_i x|^2; x on the pins
  // only: L_FC x_C = (G^T M G x)_F
  std::normal_distribution<double> N(0.0, 1.0);
  std::vector<double> xF(n, 0.0), xC(n, 0.0);
  for (int v = 0; v < n; ++v) (H.v2pin[v] < 0 ? xF : xC)[v] = N(rng);
  double quad_elem = 0.0;
  std::vector<double> GtMGx(n, 0.0);
  for (int i = 0; i < m; ++i) {
    double g[3][3];
    for (int j = 0; j < d; ++j)
      for (int a = 0; a < d; ++a) g[j][a] = H.g[(size_t)i * d * d + j * d + a];
    double gx[3] = {0, 0, 0}, gc[3] = {0, 0, 0};
    for (int j = 0; j <= d; ++j) {
      double h[3];
      hat(g, d, j, h);
      for (int a = 0; a < d; ++a) {
        gx[a] += h[a] * xF[T[3 * i + j]];
        gc[a] += h[a] * xC[T[3 * i + j]];
      }
    }
    for (int a = 0; a < d; ++a) quad_elem += mu[i] * gx[a] * gx[a];
    for (int j = 0; j <= d; ++j) {
      double h[3];
      hat(g, d, j, h);
      for (int a = 0; a < d; ++a) GtMGx[T[3 * i + j]] += mu[i] * h[a] * gc[a];
    }
  }
  double quad = 0.0;
  for (int f = 0; f < nF; ++f)
    for (int64_t q = Ap[f]; q < Ap[f + 1]; ++q) quad += xF[H.free_vertex[f]] * Ax[q] * xF[H.free_vertex[Ai[q]]];
  CHECK(std::fabs(quad - quad_elem) <= 1e-12 * quad_elem, "quadratic form %g vs %g\n", quad, quad_elem);
  std::vector<int> pin_vertex(n_pin);
  for (int v = 0; v < n; ++v)
    if (H.v2pin[v] >= 0) pin_vertex[H.v2pin[v]] = v;
  for (int f = 0; f < nF; ++f) {
    double s = 0.0;
    for (int64_t q = Cp[f]; q < Cp[f + 1]; ++q) s += Cx[q] * xC[pin_vertex[Ci[q]]];
    const double want = GtMGx[H.free_vertex[f]];
    CHECK(std::fabs(s - want) <= 1e-12 * (1.0 + std::fabs(want)), "L_FC x_C row %d: %g vs %g\n", f, s, want);
  }

  // device forms in elimination order
  H.coords.assign((size_t)nF * 3, 0.0);
  for (int f = 0; f < nF; ++f)
    for (int a = 0; a < 2; ++a) H.coords[(size_t)f * 3 + a] = V[H.free_vertex[f] * 2 + a];
  FactorInput in;
  in.nF = nF;
  in.Ap = Ap.data();
  in.Ai = Ai.data();
  in.Ax = Ax.data();
  in.coords = H.coords.data();
  in.leaf_size = 8;
  in.threads = 1;
  Factor fac;
  std::string err;
  CHECK(build_factor(in, fac, err) == 0, "factor: %s\n", err.c_str());
  OperatorArrays OA;
  operator_arrays(fac, nF, n_pin, Ap, Ai, Ax, Cp, Ci, Cx, OA);
  for (int c = 0; c < nF; ++c) {
    const int f = fac.perm[c];
    std::map<int, double> want, got;
    for (int64_t q = Ap[f]; q < Ap[f + 1]; ++q) want[fac.iperm[Ai[q]]] += Ax[q];
    for (int q = 0; q < OA.width; ++q) got[OA.ell_col[(size_t)q * nF + c]] += OA.ell_val[(size_t)q * nF + c];
    if (!want.count(c)) want[c] = 0.0;
    CHECK(got == want, "ELL row %d differs from the CSR row of vertex %d\n", c, f);
    std::vector<std::pair<int, double>> fc, cf;
    for (int64_t q = OA.fc_ptr[c]; q < OA.fc_ptr[c + 1]; ++q) fc.push_back({OA.fc_col[q], OA.fc_val[q]});
    for (int64_t q = Cp[f]; q < Cp[f + 1]; ++q) cf.push_back({Ci[q], Cx[q]});
    CHECK(fc == cf, "L_FC row %d differs\n", c);
  }
  for (int p = 0; p < n_pin; ++p)
    for (int64_t q = OA.cf_ptr[p]; q < OA.cf_ptr[p + 1]; ++q) {
      const int c = OA.cf_row[q];
      bool found = false;
      for (int64_t k = OA.fc_ptr[c]; k < OA.fc_ptr[c + 1]; ++k)
        found |= (OA.fc_col[k] == p && OA.fc_val[k] == OA.cf_val[q]);
      CHECK(found, "L_CF entry (%d,%d) has no L_FC counterpart\n", p, c);
    }
  CHECK(OA.cf_ptr[n_pin] == OA.fc_ptr[nF], "L_CF and L_FC sizes differ\n");
}

int main() {
  std::mt19937_64 rng(3);
  check_geometry(rng);
  check_operator(rng, 9, 7);
  check_operator(rng, 90, 80);
  if (!fails) std::printf("ok\n");
  return fails ? 1 : 0;
}
