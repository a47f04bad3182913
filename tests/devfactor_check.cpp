// Host check of the plan of the device decomposition (csrc/ffa_devfactor.h,
// csrc/ffa_devfactor_plan.cpp) and of the device assembly's term lists, without a
// GPU.  On tetrahedral and triangle meshes with pinned vertices:
//   * the launch program is run on the CPU in double with plain loops, item by
//     item in launch order, touching exactly the index ranges the kernels touch
//     (through the same geometry helpers), each access checked against its
//     node's front, its inv(L_ss) and its block (fronts and inverses start at
//     zero, as the device clears them);
//   * the blocks it writes equal the host multifrontal factor's double blocks
//     (relative 1e-10 per supernode), and every block entry is written once;
//   * the term lists reproduce the host assembly of L_FF, L_FC and L_CF for random
//     penalties (relative 1e-13).
// Prints "ok" or the first failure.
#include <cmath>
#include <cstdio>
#include <random>
#include <string>
#include <vector>

#include "../paper_2107_05200_gb300/csrc/ffa_devfactor.h"
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

struct Mesh {
  int d = 3, d_in = 3, n = 0;
  std::vector<double> V;
  std::vector<int32_t> T, pins;
};

// k^3 cells of the unit cube, six tetrahedra per cell around the v000-v111
// diagonal, jittered interior, bottom face pinned
static Mesh tet_cube(int k, std::mt19937_64& rng) {
  Mesh M;
  const int k1 = k + 1;
  M.n = k1 * k1 * k1;
  std::uniform_real_distribution<double> U(-0.2, 0.2);
  auto id = [&](int i, int j, int l) { return (l * k1 + j) * k1 + i; };
  for (int l = 0; l <= k; ++l)
    for (int j = 0; j <= k; ++j)
      for (int i = 0; i <= k; ++i) {
        const bool in = i > 0 && i < k && j > 0 && j < k && l > 0 && l < k;
        M.V.push_back((i + (in ? U(rng) : 0.0)) / k);
        M.V.push_back((j + (in ? U(rng) : 0.0)) / k);
        M.V.push_back((l + (in ? U(rng) : 0.0)) / k);
        if (l == 0) M.pins.push_back(id(i, j, l));
      }
  const int path[6][2] = {{0, 1}, {0, 2}, {1, 0}, {1, 2}, {2, 0}, {2, 1}};
  for (int l = 0; l < k; ++l)
    for (int j = 0; j < k; ++j)
      for (int i = 0; i < k; ++i)
        for (auto& pp : path) {
          int c[3] = {0, 0, 0};
          int32_t t[4];
          t[0] = id(i, j, l);
          c[pp[0]] = 1;
          t[1] = id(i + c[0], j + c[1], l + c[2]);
          c[pp[1]] = 1;
          t[2] = id(i + c[0], j + c[1], l + c[2]);
          t[3] = id(i + 1, j + 1, l + 1);
          // orient positively
          const double* v0 = &M.V[3 * t[0]];
          double e[3][3];
          for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) e[a][b] = M.V[3 * t[a + 1] + b] - v0[b];
          const double det = e[0][0] * (e[1][1] * e[2][2] - e[1][2] * e[2][1]) -
                             e[0][1] * (e[1][0] * e[2][2] - e[1][2] * e[2][0]) +
                             e[0][2] * (e[1][0] * e[2][1] - e[1][1] * e[2][0]);
          if (det < 0) std::swap(t[1], t[2]);
          M.T.insert(M.T.end(), t, t + 4);
        }
  return M;
}

// k x k grid of the unit square, two triangles per cell, two pinned corners
static Mesh tri_square(int k, std::mt19937_64& rng) {
  Mesh M;
  M.d = 2;
  M.d_in = 2;
  const int k1 = k + 1;
  M.n = k1 * k1;
  std::uniform_real_distribution<double> U(-0.2, 0.2);
  for (int j = 0; j <= k; ++j)
    for (int i = 0; i <= k; ++i) {
      const bool in = i > 0 && i < k && j > 0 && j < k;
      M.V.push_back((i + (in ? U(rng) : 0.0)) / k);
      M.V.push_back((j + (in ? U(rng) : 0.0)) / k);
    }
  for (int j = 0; j < k; ++j)
    for (int i = 0; i < k; ++i) {
      const int a = j * k1 + i, b = a + 1, c = a + k1, e = c + 1;
      const int32_t t0[3] = {a, b, e}, t1[3] = {a, e, c};
      M.T.insert(M.T.end(), t0, t0 + 3);
      M.T.insert(M.T.end(), t1, t1 + 3);
    }
  M.pins = {0, k};
  return M;
}

// the operator as the library's setup builds it
static OperatorHost operator_host(const Mesh& M, std::mt19937_64& rng, double spread) {
  OperatorHost H;
  const int d = M.d, m = (int)M.T.size() / (d + 1);
  H.n = M.n;
  H.m = m;
  H.d = d;
  H.n_pin = (int)M.pins.size();
  H.v2pin.assign(M.n, -1);
  for (int p = 0; p < H.n_pin; ++p) H.v2pin[M.pins[p]] = p;
  H.free_of.assign(M.n, -1);
  for (int v = 0; v < M.n; ++v)
    if (H.v2pin[v] < 0) {
      H.free_of[v] = (int32_t)H.free_vertex.size();
      H.free_vertex.push_back(v);
    }
  H.nF = (int)H.free_vertex.size();
  H.inc_ptr.assign(M.n + 1, 0);
  for (int32_t v : M.T) H.inc_ptr[v + 1]++;
  for (int v = 0; v < M.n; ++v) H.inc_ptr[v + 1] += H.inc_ptr[v];
  H.inc.resize(H.inc_ptr[M.n]);
  std::vector<int64_t> fill(H.inc_ptr.begin(), H.inc_ptr.end() - 1);
  for (int i = 0; i < m; ++i)
    for (int j = 0; j <= d; ++j) H.inc[fill[M.T[(int64_t)i * (d + 1) + j]]++] = i * (d + 1) + j;
  H.T = M.T;
  H.g.assign((size_t)m * d * d, 0.0);
  H.mu.assign(m, 0.0);
  std::normal_distribution<double> N(0.0, spread);
  for (int i = 0; i < m; ++i) {
    double g[3][3], w;
    if (!element_geometry(d, M.d_in, M.V.data(), M.T.data() + (int64_t)i * (d + 1), g, w)) {
      CHECK(false, "degenerate element %d\n", i);
      continue;
    }
    for (int j = 0; j < d; ++j)
      for (int a = 0; a < d; ++a) H.g[(int64_t)i * d * d + j * d + a] = g[j][a];
    H.mu[i] = w * std::exp(N(rng));
  }
  H.coords.assign((size_t)H.nF * 3, 0.0);
  for (int f = 0; f < H.nF; ++f)
    for (int a = 0; a < M.d_in; ++a) H.coords[(size_t)f * 3 + a] = M.V[(size_t)H.free_vertex[f] * M.d_in + a];
  return H;
}

// one launch program run on the CPU; fronts F and inverses Lv in double
struct Emu {
  const DevFactorPlan& P;
  std::vector<double> F, Lv, B;
  std::vector<int> written;
  explicit Emu(const DevFactorPlan& p)
      : P(p), F(p.front_elems, 0.0), Lv(p.linv_elems, 0.0),
        B(p.block_floats, 0.0), written(p.block_floats, 0) {}
  double& f(int s, int64_t r, int64_t c) {
    const DfNode& d = P.nodes[s];
    CHECK(r >= 0 && r < d.N && c >= 0 && c < d.N, "front access (%lld, %lld) outside node %d of order %d\n",
          (long long)r, (long long)c, s, d.N);
    return F[d.fr_off + c * d.ldF + r];
  }
  double& lv(int s, int64_t r, int64_t c) {
    const DfNode& d = P.nodes[s];
    CHECK(r >= 0 && r < d.ns && c >= 0 && c < d.ns, "inverse access (%lld, %lld) outside node %d with %d columns\n",
          (long long)r, (long long)c, s, d.ns);
    return Lv[d.li_off + c * d.ldL + r];
  }
  void blk(int s, int64_t r, int64_t c, double v) {
    const DfNode& d = P.nodes[s];
    CHECK(r >= 0 && r < d.N && c >= 0 && c < d.ns, "block write (%lld, %lld) outside node %d\n", (long long)r,
          (long long)c, s);
    const int64_t k = d.blk_off + c * d.ld + r;
    B[k] = v;
    written[k]++;
  }
  void run_item(const DfLaunch& L, const DfItem& it, const std::vector<int32_t>& rel_ok) {
    const int s = it.node;
    const DfNode& d = P.nodes[s];
    const int p = L.p;
    switch (L.kind) {
      case kDfExtendAdd: {
        const int par = d.parent;
        const int32_t ms = d.N - d.ns;
        const int32_t* rel = P.rel.data() + P.rel_off[s];
        CHECK(par >= 0 && rel_ok[s], "extend-add item of node %d without parent map\n", s);
        for (int32_t b = it.code; b < df_min(it.code + kDfEaCols, ms); ++b)
          for (int32_t a = b; a < ms; ++a) f(par, rel[a], rel[b]) += f(s, d.ns + a, d.ns + b);
        break;
      }
      case kDfDiag: {
        const DfPanel g = df_panel(d, p);
        for (int k = 0; k < g.w; ++k) {
          double& dk = f(s, g.c0 + k, g.c0 + k);
          CHECK(dk > 0, "pivot %g at node %d\n", dk, s);
          dk = std::sqrt(dk);
          for (int i = k + 1; i < g.w; ++i) f(s, g.c0 + i, g.c0 + k) /= dk;
          for (int j = k + 1; j < g.w; ++j)
            for (int i = j; i < g.w; ++i) f(s, g.c0 + i, g.c0 + j) -= f(s, g.c0 + i, g.c0 + k) * f(s, g.c0 + j, g.c0 + k);
        }
        for (int j = 0; j < g.w; ++j) {
          for (int i = 0; i < j; ++i) lv(s, g.c0 + i, g.c0 + j) = 0.0;
          lv(s, g.c0 + j, g.c0 + j) = 1.0 / f(s, g.c0 + j, g.c0 + j);
          for (int i = j + 1; i < g.w; ++i) {
            double sum = 0.0;
            for (int k = j; k < i; ++k) sum += f(s, g.c0 + i, g.c0 + k) * lv(s, g.c0 + k, g.c0 + j);
            lv(s, g.c0 + i, g.c0 + j) = -sum / f(s, g.c0 + i, g.c0 + i);
          }
        }
        break;
      }
      case kDfSolve: {
        const DfPanel g = df_panel(d, p);
        if (it.code >= 0) {
          const int32_t R0 = g.t0 + it.code * kDfTile, ra = df_min(kDfTile, d.N - R0);
          CHECK(ra > 0, "empty solve tile at node %d\n", s);
          std::vector<double> out((size_t)ra * g.w);
          for (int r = 0; r < ra; ++r)
            for (int k = 0; k < g.w; ++k) {
              double v = 0.0;
              for (int l = 0; l < g.w; ++l) v += f(s, R0 + r, g.c0 + l) * lv(s, g.c0 + k, g.c0 + l);
              out[(size_t)r * g.w + k] = v;
            }
          for (int r = 0; r < ra; ++r)
            for (int k = 0; k < g.w; ++k) f(s, R0 + r, g.c0 + k) = out[(size_t)r * g.w + k];
        } else {
          // X_pj = -X_pp S_pj in place of S_pj
          const int32_t j0 = (-1 - it.code) * kDfTile;
          CHECK(j0 + kDfTile <= g.c0, "inverse block column %d not left of panel %d\n", j0, p);
          std::vector<double> out((size_t)g.w * kDfTile, 0.0);
          for (int r = 0; r < g.w; ++r)
            for (int c = 0; c < kDfTile; ++c) {
              double v = 0.0;
              for (int q = 0; q < g.w; ++q) v += lv(s, g.c0 + r, g.c0 + q) * lv(s, g.c0 + q, j0 + c);
              out[(size_t)r * kDfTile + c] = -v;
            }
          for (int r = 0; r < g.w; ++r)
            for (int c = 0; c < kDfTile; ++c) lv(s, g.c0 + r, j0 + c) = out[(size_t)r * kDfTile + c];
        }
        break;
      }
      case kDfUpdate: {
        const DfPanel g = df_panel(d, p);
        if (it.code < 0) {
          // S_qj += L_qp X_pj
          const int32_t q = (-1 - it.code) >> 16, j = (-1 - it.code) & 0xffff;
          CHECK(q > p && j <= p && q < df_panels(d), "inverse update (%d, %d) at panel %d of node %d\n", q, j, p, s);
          const int32_t r0 = q * kDfTile, rq = df_min(kDfTile, d.ns - r0), j0 = j * kDfTile;
          const int32_t cb = j == p ? g.w : kDfTile;
          for (int r = 0; r < rq; ++r)
            for (int c = 0; c < cb; ++c) {
              double v = 0.0;
              for (int k = 0; k < g.w; ++k) v += f(s, r0 + r, g.c0 + k) * lv(s, g.c0 + k, j0 + c);
              lv(s, r0 + r, j0 + c) += v;
            }
          break;
        }
        const int32_t I = it.code >> 16, J = it.code & 0xffff;
        CHECK(J <= I, "update tile above the diagonal at node %d\n", s);
        const int32_t R0 = g.t0 + I * kDfTile, C0 = g.t0 + J * kDfTile;
        const int32_t ra = df_min(kDfTile, d.N - R0), cb = df_min(kDfTile, d.N - C0);
        for (int r = 0; r < ra; ++r)
          for (int c = 0; c < cb; ++c) {
            double v = 0.0;
            for (int k = 0; k < g.w; ++k) v += f(s, R0 + r, g.c0 + k) * f(s, C0 + c, g.c0 + k);
            f(s, R0 + r, C0 + c) -= v;
          }
        break;
      }
      case kDfBrs: {
        const int32_t A = it.code >> 16, J = it.code & 0xffff;
        const int32_t R0 = d.ns + A * kDfTile, col0 = J * kDfTile;
        const int32_t ra = df_min(kDfTile, d.N - R0), cb = df_min(kDfTile, d.ns - col0);
        for (int r = 0; r < ra; ++r)
          for (int c = 0; c < cb; ++c) {
            double v = 0.0;
            for (int k = col0; k < d.ns; ++k) v += f(s, R0 + r, k) * lv(s, k, col0 + c);
            blk(s, R0 + r, col0 + c, v);
          }
        break;
      }
      case kDfPack: {
        const int32_t col0 = it.code * kDfTile;
        for (int j = col0; j < df_min(d.ns, col0 + kDfTile); ++j)
          for (int i = 0; i < d.ns; ++i) blk(s, i, j, i >= j ? lv(s, i, j) : 0.0);
        break;
      }
      default:
        CHECK(false, "unknown launch kind %d\n", L.kind);
    }
  }
};

static void check_mesh(const Mesh& M, uint64_t seed, double spread, int leaf, const char* name) {
  std::mt19937_64 rng(seed);
  OperatorHost H = operator_host(M, rng, spread);
  std::vector<int64_t> Ap, Cp;
  std::vector<int32_t> Ai, Ci;
  std::vector<double> Ax, Cx;
  assemble_operator(H, H.mu.data(), Ap, Ai, Ax, Cp, Ci, Cx);
  FactorInput in;
  in.nF = H.nF;
  in.Ap = Ap.data();
  in.Ai = Ai.data();
  in.Ax = Ax.data();
  in.coords = H.coords.data();
  in.leaf_size = leaf;
  in.threads = 2;
  in.keep_double = true;
  Factor fac;
  std::string err;
  CHECK(build_factor(in, fac, err) == 0, "%s: factor failed: %s\n", name, err.c_str());
  if (fails) return;
  OperatorArrays OA;
  operator_arrays(fac, H.nF, H.n_pin, Ap, Ai, Ax, Cp, Ci, Cx, OA);
  std::vector<int32_t> cnt(H.nF);
  for (int c = 0; c < H.nF; ++c) cnt[c] = (int32_t)(Ap[fac.perm[c] + 1] - Ap[fac.perm[c]]);
  DevFactorPlan P;
  CHECK(build_devfactor_plan(fac, OA.width, OA.ell_col, cnt, P, err), "%s: plan failed: %s\n", name, err.c_str());
  if (fails) return;
  // fronts and inverses do not overlap
  for (size_t s = 0; s + 1 < P.nodes.size(); ++s) {
    CHECK(P.nodes[s].fr_off + (int64_t)P.nodes[s].ldF * P.nodes[s].N <= P.nodes[s + 1].fr_off, "%s: fronts overlap\n",
          name);
    CHECK(P.nodes[s].li_off + (int64_t)P.nodes[s].ldL * P.nodes[s].ns <= P.nodes[s + 1].li_off,
          "%s: inverses overlap\n", name);
  }
  std::vector<int32_t> rel_ok(P.nodes.size(), 0);
  for (size_t c = 0; c < P.nodes.size(); ++c) {
    const int64_t end = c + 1 < P.nodes.size() ? P.rel_off[c + 1] : (int64_t)P.rel.size();
    const int par = P.nodes[c].parent;
    rel_ok[c] = par >= 0 && end - P.rel_off[c] == P.nodes[c].N - P.nodes[c].ns;
    for (int64_t k = P.rel_off[c]; k < end && par >= 0; ++k)
      CHECK(P.rel[k] >= 0 && P.rel[k] < P.nodes[par].N, "%s: extend-add map out of range\n", name);
  }
  Emu E(P);
  for (size_t k = 0; k < P.orig_dst.size(); ++k)
    if (P.orig_dst[k] >= 0) {
      CHECK(P.orig_dst[k] < P.front_elems, "%s: scatter outside the fronts\n", name);
      E.F[P.orig_dst[k]] = OA.ell_val[k];
    }
  int64_t items = 0;
  for (const DfLaunch& L : P.prog) {
    CHECK(L.off >= 0 && L.off + L.count <= (int64_t)P.items.size(), "%s: launch items out of range\n", name);
    for (int64_t k = L.off; k < L.off + L.count && !fails; ++k) E.run_item(L, P.items[k], rel_ok);
    items += L.count;
    if (fails) return;
  }
  CHECK(items == (int64_t)P.items.size(), "%s: items not all launched\n", name);
  double worst = 0.0;
  for (size_t s = 0; s < fac.nodes.size(); ++s) {
    const Supernode& sn = fac.nodes[s];
    double mx = 0.0, md = 0.0;
    for (int j = 0; j < sn.ncol; ++j)
      for (int i = 0; i < sn.ncol + sn.nrow; ++i) {
        const int64_t k = sn.blk_off + (int64_t)j * sn.ld + i;
        mx = std::max(mx, std::fabs(fac.blocks64[k]));
        md = std::max(md, std::fabs(E.B[k] - fac.blocks64[k]));
        CHECK(E.written[k] == 1, "%s: block entry (%d, %d) of node %zu written %d times\n", name, i, j, s,
              E.written[k]);
      }
    if (mx > 0) worst = std::max(worst, md / mx);
  }
  CHECK(worst < 1e-10, "%s: device-program blocks differ from the host factor by %.3g\n", name, worst);
  std::printf("%s: %d free, %zu supernodes, %zu launches, %zu items, max panels %d, blocks rel. diff %.2e\n", name,
              H.nF, fac.nodes.size(), P.prog.size(), P.items.size(), P.max_panels, worst);

  // device assembly term lists against the host assembly, new penalties
  DevAssemblyPlan Q;
  CHECK(build_assembly_plan(H, fac, OA, Ap, Q, err), "%s: assembly plan failed: %s\n", name, err.c_str());
  if (fails) return;
  std::uniform_real_distribution<double> Um(0.5, 20.0);
  std::vector<double> mu2(H.m);
  for (int i = 0; i < H.m; ++i) mu2[i] = H.mu[i] * Um(rng);
  std::vector<int64_t> Ap2, Cp2;
  std::vector<int32_t> Ai2, Ci2;
  std::vector<double> Ax2, Cx2;
  assemble_operator(H, mu2.data(), Ap2, Ai2, Ax2, Cp2, Ci2, Cx2);
  OperatorArrays OB;
  operator_arrays(fac, H.nF, H.n_pin, Ap2, Ai2, Ax2, Cp2, Ci2, Cx2, OB);
  const int d = H.d;
  auto term = [&](int32_t code) {
    const int i = code >> 4, j = (code >> 2) & 3, l = code & 3;
    double gj[3], gl[3];
    for (int a = 0; a < d; ++a) {
      double s0 = 0.0;
      for (int jj = 0; jj < d; ++jj) s0 += H.g[(int64_t)i * d * d + jj * d + a];
      gj[a] = j > 0 ? H.g[(int64_t)i * d * d + (j - 1) * d + a] : -s0;
      gl[a] = l > 0 ? H.g[(int64_t)i * d * d + (l - 1) * d + a] : -s0;
    }
    double dv = 0.0;
    for (int a = 0; a < d; ++a) dv += gj[a] * gl[a];
    return mu2[i] * dv;
  };
  double wa = 0.0, scale = 0.0;
  for (size_t k = 0; k + 1 < Q.ell_ptr.size(); ++k) {
    double v = 0.0;
    for (int64_t t = Q.ell_ptr[k]; t < Q.ell_ptr[k + 1]; ++t) v += term(Q.ell_src[t]);
    scale = std::max(scale, std::fabs(OB.ell_val[k]));
    wa = std::max(wa, std::fabs(v - OB.ell_val[k]));
  }
  std::vector<double> fcv(Q.fc_ptr.size() - 1, 0.0);
  for (size_t k = 0; k + 1 < Q.fc_ptr.size(); ++k) {
    for (int64_t t = Q.fc_ptr[k]; t < Q.fc_ptr[k + 1]; ++t) fcv[k] += term(Q.fc_src[t]);
    wa = std::max(wa, std::fabs(fcv[k] - OB.fc_val[k]));
  }
  for (size_t k = 0; k < Q.cf_src.size(); ++k) wa = std::max(wa, std::fabs(fcv[Q.cf_src[k]] - OB.cf_val[k]));
  CHECK(OB.fc_val.size() == fcv.size() && OB.cf_val.size() == Q.cf_src.size(), "%s: L_FC sizes differ\n", name);
  CHECK(wa <= 1e-13 * scale, "%s: device assembly differs from the host assembly by %.3g (scale %.3g)\n", name, wa,
        scale);
}

int main() {
  std::mt19937_64 rng(7);
  check_mesh(tet_cube(5, rng), 11, 0.0, 16, "tet cube 5");
  check_mesh(tet_cube(9, rng), 12, 1.5, 16, "tet cube 9 graded");
  check_mesh(tet_cube(15, rng), 15, 1.0, 64, "tet cube 15");        // separators of 4 panels
  check_mesh(tet_cube(8, rng), 16, 0.5, 200, "tet cube 8 wide leaves");  // leaves of several panels
  check_mesh(tri_square(24, rng), 13, 0.0, 16, "triangles 24");
  check_mesh(tri_square(40, rng), 14, 2.0, 16, "triangles 40 graded");
  check_mesh(tri_square(150, rng), 17, 0.0, 64, "triangles 150");   // separators of 3 panels
  if (fails) {
    std::printf("%d failures\n", fails);
    return 1;
  }
  std::printf("ok\n");
  return 0;
}
