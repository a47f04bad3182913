#include "ffa_constraint_host.h"

#include <algorithm>
#include <cmath>
#include <utility>

namespace ffa {

void split_constraints(int c, const int64_t* ptr, const int32_t* col, const double* val,
                       const std::vector<int32_t>& v2e, const std::vector<int32_t>& slot_of, ConstraintSplit& out) {
  out.fptr.assign(c + 1, 0);
  out.fcol.clear();
  out.fval.clear();
  out.pin.clear();
  for (int r = 0; r < c; ++r) {
    std::vector<std::pair<int32_t, double>> row;
    for (int64_t q = ptr[r]; q < ptr[r + 1]; ++q) {
      const int v = col[q];
      if (v2e[v] >= 0) row.push_back({v2e[v], val[q]});
      else out.pin.push_back({r, slot_of[v], val[q]});
    }
    std::sort(row.begin(), row.end());
    for (size_t k = 0; k < row.size(); ++k) {
      if ((int64_t)out.fcol.size() > out.fptr[r] && out.fcol.back() == row[k].first) {
        out.fval.back() += row[k].second;
      } else {
        out.fcol.push_back(row[k].first);
        out.fval.push_back(row[k].second);
      }
    }
    out.fptr[r + 1] = (int64_t)out.fcol.size();
  }
}

int schur_inverse(int c, const std::vector<double>& S, std::vector<double>& Sinv) {
  // S = L L^T
  std::vector<double> Lc((size_t)c * c, 0.0);
  for (int i = 0; i < c; ++i)
    for (int j = 0; j <= i; ++j) {
      double a = 0.5 * (S[(size_t)i * c + j] + S[(size_t)j * c + i]);
      for (int k = 0; k < j; ++k) a -= Lc[(size_t)i * c + k] * Lc[(size_t)j * c + k];
      if (i == j) {
        if (!(a > 1e-10 * S[(size_t)i * c + i]) || !(S[(size_t)i * c + i] > 0.0)) return i;
        Lc[(size_t)i * c + i] = std::sqrt(a);
      } else {
        Lc[(size_t)i * c + j] = a / Lc[(size_t)j * c + j];
      }
    }
  // S^-1 column by column: L y = e_j, L^T x = y
  Sinv.assign((size_t)c * c, 0.0);
  std::vector<double> y(c);
  for (int j = 0; j < c; ++j) {
    for (int i = 0; i < c; ++i) {
      double a = i == j ? 1.0 : 0.0;
      for (int k = 0; k < i; ++k) a -= Lc[(size_t)i * c + k] * y[k];
      y[i] = a / Lc[(size_t)i * c + i];
    }
    for (int i = c - 1; i >= 0; --i) {
      double a = y[i];
      for (int k = i + 1; k < c; ++k) a -= Lc[(size_t)k * c + i] * Sinv[(size_t)k * c + j];
      Sinv[(size_t)i * c + j] = a / Lc[(size_t)i * c + i];
    }
  }
  return -1;
}

}  // namespace ffa
