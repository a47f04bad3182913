#include "ffa_operator_host.h"

#include <algorithm>
#include <cmath>
#include <thread>
#include <utility>

namespace ffa {

bool element_geometry(int d, int d_in, const double* V, const int32_t* t, double g[3][3], double& w) {
  double E[3][3] = {{0}};
  const double* v0 = V + (int64_t)t[0] * d_in;
  if (d_in == d) {
    for (int j = 0; j < d; ++j) {
      const double* vj = V + (int64_t)t[j + 1] * d_in;
      for (int a = 0; a < d; ++a) E[j][a] = vj[a] - v0[a];
    }
  } else {
    const double* v1 = V + (int64_t)t[1] * 3;
    const double* v2 = V + (int64_t)t[2] * 3;
    double a[3] = {v1[0] - v0[0], v1[1] - v0[1], v1[2] - v0[2]};
    double b[3] = {v2[0] - v0[0], v2[1] - v0[1], v2[2] - v0[2]};
    const double la = std::sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
    double nrm[3] = {a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]};
    const double ln = std::sqrt(nrm[0] * nrm[0] + nrm[1] * nrm[1] + nrm[2] * nrm[2]);
    if (!(la > 0) || !(ln > 0)) return false;
    double e1[3] = {a[0] / la, a[1] / la, a[2] / la};
    for (double& c : nrm) c /= ln;
    double e2[3] = {nrm[1] * e1[2] - nrm[2] * e1[1], nrm[2] * e1[0] - nrm[0] * e1[2], nrm[0] * e1[1] - nrm[1] * e1[0]};
    E[0][0] = la;
    E[0][1] = 0.0;
    E[1][0] = b[0] * e1[0] + b[1] * e1[1] + b[2] * e1[2];
    E[1][1] = b[0] * e2[0] + b[1] * e2[1] + b[2] * e2[2];
  }
  double inv[3][3];
  double det;
  if (d == 2) {
    det = E[0][0] * E[1][1] - E[0][1] * E[1][0];
    if (!(std::fabs(det) > 0) || !std::isfinite(det)) return false;
    inv[0][0] = E[1][1] / det;
    inv[0][1] = -E[0][1] / det;
    inv[1][0] = -E[1][0] / det;
    inv[1][1] = E[0][0] / det;
    w = std::fabs(det) / 2.0;
  } else {
    const double c00 = E[1][1] * E[2][2] - E[1][2] * E[2][1];
    const double c01 = E[1][2] * E[2][0] - E[1][0] * E[2][2];
    const double c02 = E[1][0] * E[2][1] - E[1][1] * E[2][0];
    det = E[0][0] * c00 + E[0][1] * c01 + E[0][2] * c02;
    if (!(std::fabs(det) > 0) || !std::isfinite(det)) return false;
    inv[0][0] = c00 / det;
    inv[1][0] = c01 / det;
    inv[2][0] = c02 / det;
    inv[0][1] = (E[0][2] * E[2][1] - E[0][1] * E[2][2]) / det;
    inv[1][1] = (E[0][0] * E[2][2] - E[0][2] * E[2][0]) / det;
    inv[2][1] = (E[0][1] * E[2][0] - E[0][0] * E[2][1]) / det;
    inv[0][2] = (E[0][1] * E[1][2] - E[0][2] * E[1][1]) / det;
    inv[1][2] = (E[0][2] * E[1][0] - E[0][0] * E[1][2]) / det;
    inv[2][2] = (E[0][0] * E[1][1] - E[0][1] * E[1][0]) / det;
    w = std::fabs(det) / 6.0;
  }
  for (int j = 0; j < d; ++j)
    for (int a = 0; a < d; ++a) g[j][a] = inv[a][j];  // g_{j+1}[a] = (E^{-1})[a][j]
  return true;
}

void assemble_operator(const OperatorHost& H, const double* mu, std::vector<int64_t>& Ap, std::vector<int32_t>& Ai,
                       std::vector<double>& Ax, std::vector<int64_t>& Cp, std::vector<int32_t>& Ci,
                       std::vector<double>& Cx) {
  const int d = H.d, nF = H.nF;
  auto grad_of = [&](int i, int j, double out[3]) {  // hat gradient of local vertex j
    for (int a = 0; a < d; ++a) {
      if (j > 0) out[a] = H.g[(int64_t)i * d * d + (j - 1) * d + a];
      else {
        double sum = 0;
        for (int jj = 0; jj < d; ++jj) sum += H.g[(int64_t)i * d * d + jj * d + a];
        out[a] = -sum;
      }
    }
  };
  // Rows are independent: contiguous chunks of rows are assembled by separate
  // threads into their own arrays, then concatenated in row order, so the result
  // does not depend on the number of threads.
  struct Chunk {
    std::vector<int32_t> ai, ci;
    std::vector<double> ax, cx;
    std::vector<int32_t> na, nc;  // entries per row
  };
  const unsigned hw = std::thread::hardware_concurrency();
  const int nchunk = std::max(1, std::min<int>(hw ? (int)hw : 1, nF / 4096 + 1));
  std::vector<Chunk> chunks(nchunk);
  auto assemble_rows = [&](int ck) {
    Chunk& C = chunks[ck];
    const int f0 = (int)((int64_t)nF * ck / nchunk), f1 = (int)((int64_t)nF * (ck + 1) / nchunk);
    std::vector<int32_t> pos(H.n, -1), touched;
    std::vector<double> acc;
    std::vector<std::pair<int32_t, double>> fr, cr;
    for (int f = f0; f < f1; ++f) {
      const int v = H.free_vertex[f];
      touched.clear();
      acc.clear();
      for (int64_t q = H.inc_ptr[v]; q < H.inc_ptr[v + 1]; ++q) {
        const int i = H.inc[q] / (d + 1), j = H.inc[q] % (d + 1);
        double gj[3], gl[3];
        grad_of(i, j, gj);
        for (int l = 0; l <= d; ++l) {
          grad_of(i, l, gl);
          double dotv = 0;
          for (int a = 0; a < d; ++a) dotv += gj[a] * gl[a];
          const int u = H.T[(int64_t)i * (d + 1) + l];
          if (pos[u] < 0) {
            pos[u] = (int32_t)touched.size();
            touched.push_back(u);
            acc.push_back(0.0);
          }
          acc[pos[u]] += mu[i] * dotv;
        }
      }
      fr.clear();
      cr.clear();
      for (size_t k = 0; k < touched.size(); ++k) {
        const int u = touched[k];
        if (H.free_of[u] >= 0) fr.push_back({H.free_of[u], acc[k]});
        else cr.push_back({H.v2pin[u], acc[k]});
        pos[u] = -1;
      }
      std::sort(fr.begin(), fr.end());
      std::sort(cr.begin(), cr.end());
      for (auto& pr : fr) { C.ai.push_back(pr.first); C.ax.push_back(pr.second); }
      for (auto& pr : cr) { C.ci.push_back(pr.first); C.cx.push_back(pr.second); }
      C.na.push_back((int32_t)fr.size());
      C.nc.push_back((int32_t)cr.size());
    }
  };
  run_threads(nchunk, assemble_rows);
  Ap.assign(nF + 1, 0);
  Cp.assign(nF + 1, 0);
  Ai.clear(); Ax.clear(); Ci.clear(); Cx.clear();
  int f = 0;
  for (const Chunk& C : chunks) {
    Ai.insert(Ai.end(), C.ai.begin(), C.ai.end());
    Ax.insert(Ax.end(), C.ax.begin(), C.ax.end());
    Ci.insert(Ci.end(), C.ci.begin(), C.ci.end());
    Cx.insert(Cx.end(), C.cx.begin(), C.cx.end());
    for (size_t r = 0; r < C.na.size(); ++r, ++f) {
      Ap[f + 1] = Ap[f] + C.na[r];
      Cp[f + 1] = Cp[f] + C.nc[r];
    }
  }
}

void operator_arrays(const Factor& fac, int nF, int n_pin, const std::vector<int64_t>& Ap,
                     const std::vector<int32_t>& Ai, const std::vector<double>& Ax, const std::vector<int64_t>& Cp,
                     const std::vector<int32_t>& Ci, const std::vector<double>& Cx, OperatorArrays& A) {
  int width = 1;
  for (int f = 0; f < nF; ++f) width = std::max<int>(width, (int)(Ap[f + 1] - Ap[f]));
  A.width = width;
  A.ell_col.assign((size_t)width * nF, 0);
  A.ell_val.assign((size_t)width * nF, 0.0);
  A.fc_ptr.assign(nF + 1, 0);
  A.fc_col.clear();
  A.fc_val.clear();
  for (int c = 0; c < nF; ++c) {
    const int f = fac.perm[c];
    int q = 0;
    for (int64_t k = Ap[f]; k < Ap[f + 1]; ++k, ++q) {
      A.ell_col[(size_t)q * nF + c] = fac.iperm[Ai[k]];
      A.ell_val[(size_t)q * nF + c] = Ax[k];
    }
    for (; q < width; ++q) A.ell_col[(size_t)q * nF + c] = c;
    for (int64_t k = Cp[f]; k < Cp[f + 1]; ++k) {
      A.fc_col.push_back(Ci[k]);
      A.fc_val.push_back(Cx[k]);
    }
    A.fc_ptr[c + 1] = (int64_t)A.fc_col.size();
  }
  A.cf_ptr.assign(n_pin + 1, 0);
  for (int32_t p : A.fc_col) A.cf_ptr[p + 1]++;
  for (int p = 0; p < n_pin; ++p) A.cf_ptr[p + 1] += A.cf_ptr[p];
  A.cf_row.assign(A.fc_col.size(), 0);
  A.cf_val.assign(A.fc_col.size(), 0.0);
  std::vector<int64_t> fill(A.cf_ptr.begin(), A.cf_ptr.end() - 1);
  for (int c = 0; c < nF; ++c)
    for (int64_t q = A.fc_ptr[c]; q < A.fc_ptr[c + 1]; ++q) {
      const int64_t dst = fill[A.fc_col[q]]++;
      A.cf_row[dst] = c;
      A.cf_val[dst] = A.fc_val[q];
    }
}

}  // namespace ffa
