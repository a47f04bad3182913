// Host check of the library's state packing (csrc/ffa_state.cpp): the
// quaternion convention against a rotation written out by hand, round trips of
// random rotations through every branch of Shepperd's method, the layout of P
// and Lambda, the symmetrization of P, and the refusals.  Prints "ok" or the
// first failure.
#include <cmath>
#include <cstdio>
#include <random>
#include <string>
#include <vector>

#include "../paper_2107_05200_gb300/csrc/ffa_state.h"

using namespace ffa;

static int fails = 0;
#define CHECK(cond, ...)               \
  do {                                 \
    if (!(cond)) {                     \
      if (!fails) std::printf(__VA_ARGS__); \
      ++fails;                         \
    }                                  \
  } while (0)

// rotation by angle t about the unit axis a (Rodrigues' formula)
static void axis_angle(const double a[3], double t, double* u) {
  const double c = std::cos(t), s = std::sin(t), C = 1 - c;
  const double x = a[0], y = a[1], z = a[2];
  u[0] = c + x * x * C;     u[1] = x * y * C - z * s; u[2] = x * z * C + y * s;
  u[3] = y * x * C + z * s; u[4] = c + y * y * C;     u[5] = y * z * C - x * s;
  u[6] = z * x * C - y * s; u[7] = z * y * C + x * s; u[8] = c + z * z * C;
}

int main() {
  std::mt19937_64 rng(7);
  std::normal_distribution<double> N(0.0, 1.0);

  // 1. the quaternion (cos 45, 0, 0, sin 45) is the quarter turn about z: e_x -> e_y
  {
    const double h = std::sqrt(0.5);
    const double u[4] = {h, 0, 0, h}, p[6] = {1, 0, 0, 1, 0, 1}, l[9] = {0};
    double U[9], P[9], L[9];
    unpack_state(3, 1, u, p, l, U, P, L);
    const double want[9] = {0, -1, 0, 1, 0, 0, 0, 0, 1};
    for (int k = 0; k < 9; ++k) CHECK(std::fabs(U[k] - want[k]) < 1e-15, "quarter turn: U[%d] = %g\n", k, U[k]);
  }

  // 2. round trips in 3D: random axes and angles, and angles near pi about each
  //    coordinate axis (the three branches where the trace is not the largest)
  {
    std::vector<double> Us, Ps, Ls;
    auto add = [&](const double a[3], double t) {
      double u[9];
      axis_angle(a, t, u);
      Us.insert(Us.end(), u, u + 9);
      double B[9], P[9];
      for (double& b : B) b = N(rng);
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
          double s = i == j ? 1.0 : 0.0;
          for (int k = 0; k < 3; ++k) s += B[k * 3 + i] * B[k * 3 + j];
          P[i * 3 + j] = s;  // SPD
        }
      Ps.insert(Ps.end(), P, P + 9);
      for (int k = 0; k < 9; ++k) Ls.push_back(N(rng));
    };
    for (int r = 0; r < 200; ++r) {
      double a[3] = {N(rng), N(rng), N(rng)};
      const double n = std::sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
      for (double& x : a) x /= n;
      add(a, std::uniform_real_distribution<double>(-M_PI, M_PI)(rng));
    }
    const double ax[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
    for (int k = 0; k < 3; ++k) {
      add(ax[k], M_PI);
      add(ax[k], M_PI - 1e-3);
      add(ax[k], -M_PI + 1e-7);
    }
    const double id[3] = {0, 0, 1};
    add(id, 0.0);
    const int64_t m = (int64_t)Us.size() / 9;
    std::vector<double> u(4 * m), p(6 * m), l(9 * m), U(9 * m), P(9 * m), L(9 * m);
    std::string msg;
    CHECK(pack_state(3, m, Us.data(), Ps.data(), Ls.data(), u.data(), p.data(), l.data(), msg), "pack 3D: %s\n",
          msg.c_str());
    unpack_state(3, m, u.data(), p.data(), l.data(), U.data(), P.data(), L.data());
    for (int64_t i = 0; i < m; ++i) {
      double qn = 0.0;
      for (int k = 0; k < 4; ++k) qn += u[k * m + i] * u[k * m + i];
      CHECK(std::fabs(qn - 1.0) < 1e-14, "3D: |q| of element %lld\n", (long long)i);
      for (int k = 0; k < 9; ++k) {
        CHECK(std::fabs(U[i * 9 + k] - Us[i * 9 + k]) < 1e-14, "3D round trip U, element %lld entry %d\n", (long long)i, k);
        CHECK(P[i * 9 + k] == Ps[i * 9 + k], "3D round trip P, element %lld entry %d\n", (long long)i, k);
        CHECK(L[i * 9 + k] == Ls[i * 9 + k], "3D round trip Lambda, element %lld entry %d\n", (long long)i, k);
      }
      // the documented layout: P's upper triangle row by row, Lambda's (a*d + k)
      CHECK(p[4 * m + i] == Ps[i * 9 + 5] && p[2 * m + i] == Ps[i * 9 + 2], "3D P layout, element %lld\n", (long long)i);
      CHECK(l[5 * m + i] == Ls[i * 9 + 5] && l[7 * m + i] == Ls[i * 9 + 7], "3D Lambda layout, element %lld\n", (long long)i);
    }
  }

  // 3. round trips in 2D, and P symmetrized as the mean of its off-diagonal pair
  {
    const int64_t m = 100;
    std::vector<double> Us(4 * m), Ps(4 * m), Ls(4 * m), u(2 * m), p(3 * m), l(4 * m), U(4 * m), P(4 * m), L(4 * m);
    for (int64_t i = 0; i < m; ++i) {
      const double t = std::uniform_real_distribution<double>(-M_PI, M_PI)(rng);
      Us[4 * i] = std::cos(t); Us[4 * i + 1] = -std::sin(t); Us[4 * i + 2] = std::sin(t); Us[4 * i + 3] = std::cos(t);
      Ps[4 * i] = 2.0 + N(rng) * 0.1; Ps[4 * i + 1] = 0.3; Ps[4 * i + 2] = 0.5; Ps[4 * i + 3] = 1.5;
      for (int k = 0; k < 4; ++k) Ls[4 * i + k] = N(rng);
    }
    std::string msg;
    CHECK(pack_state(2, m, Us.data(), Ps.data(), Ls.data(), u.data(), p.data(), l.data(), msg), "pack 2D: %s\n",
          msg.c_str());
    unpack_state(2, m, u.data(), p.data(), l.data(), U.data(), P.data(), L.data());
    for (int64_t i = 0; i < m; ++i) {
      for (int k = 0; k < 4; ++k) {
        CHECK(std::fabs(U[4 * i + k] - Us[4 * i + k]) < 1e-15, "2D round trip U, element %lld\n", (long long)i);
        CHECK(L[4 * i + k] == Ls[4 * i + k], "2D round trip Lambda, element %lld\n", (long long)i);
      }
      CHECK(P[4 * i + 1] == 0.4 && P[4 * i + 2] == 0.4, "2D symmetrized P, element %lld\n", (long long)i);
      CHECK(P[4 * i] == Ps[4 * i] && P[4 * i + 3] == 1.5, "2D P diagonal, element %lld\n", (long long)i);
    }
  }

  // 4. refusals: a reflection, a scaled rotation, a non-finite Lambda
  {
    const double P[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1}, L0[9] = {0};
    double u[4], p[6], l[9];
    std::string msg;
    const double refl[9] = {1, 0, 0, 0, 1, 0, 0, 0, -1};
    CHECK(!pack_state(3, 1, refl, P, L0, u, p, l, msg) && msg.find("rotation") != std::string::npos,
          "a reflection was accepted\n");
    const double twice[9] = {2, 0, 0, 0, 2, 0, 0, 0, 2};
    CHECK(!pack_state(3, 1, twice, P, L0, u, p, l, msg), "a scaled rotation was accepted\n");
    const double I2[4] = {1, 0, 0, 1}, P2[4] = {1, 0, 0, 1};
    const double Lnan[4] = {0, NAN, 0, 0};
    CHECK(!pack_state(2, 1, I2, P2, Lnan, u, p, l, msg) && msg.find("non-finite") != std::string::npos,
          "a NaN in Lambda was accepted\n");
    const double refl2[4] = {1, 0, 0, -1};
    CHECK(!pack_state(2, 1, refl2, P2, P2, u, p, l, msg), "a 2D reflection was accepted\n");
  }

  if (!fails) std::printf("ok\n");
  return fails ? 1 : 0;
}
