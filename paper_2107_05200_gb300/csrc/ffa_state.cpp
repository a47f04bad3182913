#include "ffa_state.h"

#include <cmath>

namespace ffa {

namespace {

void quat_to_matrix(const double q[4], double* u) {
  const double w = q[0], x = q[1], y = q[2], z = q[3];
  u[0] = 1 - 2 * (y * y + z * z); u[1] = 2 * (x * y - z * w); u[2] = 2 * (x * z + y * w);
  u[3] = 2 * (x * y + z * w); u[4] = 1 - 2 * (x * x + z * z); u[5] = 2 * (y * z - x * w);
  u[6] = 2 * (x * z - y * w); u[7] = 2 * (y * z + x * w); u[8] = 1 - 2 * (x * x + y * y);
}

// Unit quaternion of a rotation matrix by Shepperd's method (S. W. Shepperd,
// "Quaternion from rotation matrix", J. Guidance and Control 1(3), 1978): the
// largest of 4w^2 = 1 + tr, 4x^2 = 1 + u00 - u11 - u22, ... is taken by a square
// root and the other three components follow from sums and differences of the
// off-diagonal pairs, so no division by a small number happens.
void matrix_to_quat(const double* u, double q[4]) {
  const double tr = u[0] + u[4] + u[8];
  double w, x, y, z;
  if (tr >= u[0] && tr >= u[4] && tr >= u[8]) {
    const double s = 2.0 * std::sqrt(1.0 + tr);
    w = 0.25 * s; x = (u[7] - u[5]) / s; y = (u[2] - u[6]) / s; z = (u[3] - u[1]) / s;
  } else if (u[0] >= u[4] && u[0] >= u[8]) {
    const double s = 2.0 * std::sqrt(1.0 + u[0] - u[4] - u[8]);
    w = (u[7] - u[5]) / s; x = 0.25 * s; y = (u[1] + u[3]) / s; z = (u[2] + u[6]) / s;
  } else if (u[4] >= u[8]) {
    const double s = 2.0 * std::sqrt(1.0 + u[4] - u[0] - u[8]);
    w = (u[2] - u[6]) / s; x = (u[1] + u[3]) / s; y = 0.25 * s; z = (u[5] + u[7]) / s;
  } else {
    const double s = 2.0 * std::sqrt(1.0 + u[8] - u[0] - u[4]);
    w = (u[3] - u[1]) / s; x = (u[2] + u[6]) / s; y = (u[5] + u[7]) / s; z = 0.25 * s;
  }
  const double nrm = std::sqrt(w * w + x * x + y * y + z * z);
  q[0] = w / nrm; q[1] = x / nrm; q[2] = y / nrm; q[3] = z / nrm;
}

bool is_rotation(int d, const double* u) {
  for (int a = 0; a < d; ++a)
    for (int b = 0; b < d; ++b) {
      double s = 0.0;
      for (int k = 0; k < d; ++k) s += u[k * d + a] * u[k * d + b];
      if (!(std::fabs(s - (a == b ? 1.0 : 0.0)) <= 1e-5)) return false;
    }
  const double det = d == 2 ? u[0] * u[3] - u[1] * u[2]
                            : u[0] * (u[4] * u[8] - u[5] * u[7]) - u[1] * (u[3] * u[8] - u[5] * u[6]) +
                                  u[2] * (u[3] * u[7] - u[4] * u[6]);
  return std::fabs(det - 1.0) <= 1e-5;
}

}  // namespace

void unpack_state(int d, int64_t m, const double* u, const double* p, const double* l, double* U, double* P,
                  double* Lam) {
  const int dd = d * d;
  for (int64_t i = 0; i < m; ++i) {
    double* Ui = U + i * dd;
    double* Pi = P + i * dd;
    double* Li = Lam + i * dd;
    if (d == 2) {
      const double c = u[i], s = u[m + i];
      Ui[0] = c; Ui[1] = -s; Ui[2] = s; Ui[3] = c;
      Pi[0] = p[i]; Pi[1] = Pi[2] = p[m + i]; Pi[3] = p[2 * m + i];
    } else {
      const double q[4] = {u[i], u[m + i], u[2 * m + i], u[3 * m + i]};
      quat_to_matrix(q, Ui);
      Pi[0] = p[i]; Pi[1] = Pi[3] = p[m + i]; Pi[2] = Pi[6] = p[2 * m + i];
      Pi[4] = p[3 * m + i]; Pi[5] = Pi[7] = p[4 * m + i]; Pi[8] = p[5 * m + i];
    }
    for (int q = 0; q < dd; ++q) Li[q] = l[q * m + i];
  }
}

bool pack_state(int d, int64_t m, const double* U, const double* P, const double* Lam, double* u, double* p, double* l,
                std::string& msg) {
  const int dd = d * d;
  for (int64_t i = 0; i < m; ++i) {
    const double* Ui = U + i * dd;
    const double* Pi = P + i * dd;
    const double* Li = Lam + i * dd;
    for (int q = 0; q < dd; ++q)
      if (!std::isfinite(Ui[q]) || !std::isfinite(Pi[q]) || !std::isfinite(Li[q])) {
        msg = "non-finite state entry at element " + std::to_string(i);
        return false;
      }
    if (!is_rotation(d, Ui)) {
      msg = "U of element " + std::to_string(i) + " is not a rotation";
      return false;
    }
    if (d == 2) {
      const double c = 0.5 * (Ui[0] + Ui[3]), s = 0.5 * (Ui[2] - Ui[1]);
      const double r = std::sqrt(c * c + s * s);
      u[i] = c / r;
      u[m + i] = s / r;
      p[i] = Pi[0];
      p[m + i] = 0.5 * (Pi[1] + Pi[2]);
      p[2 * m + i] = Pi[3];
    } else {
      double q[4];
      matrix_to_quat(Ui, q);
      for (int k = 0; k < 4; ++k) u[k * m + i] = q[k];
      p[i] = Pi[0];
      p[m + i] = 0.5 * (Pi[1] + Pi[3]);
      p[2 * m + i] = 0.5 * (Pi[2] + Pi[6]);
      p[3 * m + i] = Pi[4];
      p[4 * m + i] = 0.5 * (Pi[5] + Pi[7]);
      p[5 * m + i] = Pi[8];
    }
    for (int q = 0; q < dd; ++q) l[q * m + i] = Li[q];
  }
  return true;
}

}  // namespace ffa
