// Register-resident per-element math for the local steps (paper Sec. 4 and the
// Supplemental "Solving the optimization in P / in U").  Templated on the scalar
// type: float for the FP32 local step, double for the FP64 one.
#pragma once

#include <cuda_runtime.h>
#include <math.h>

#include "ffa_internal.h"

namespace ffa {

template <typename R> struct Tr;
template <> struct Tr<float> {
  static __device__ __forceinline__ float sqrt_(float x) { return sqrtf(x); }
  static __device__ __forceinline__ float rsqrt_(float x) { return rsqrtf(x); }
  static __device__ __forceinline__ float cbrt_(float x) { return cbrtf(x); }
  static __device__ __forceinline__ float log_(float x) { return logf(x); }
  static __device__ __forceinline__ float abs_(float x) { return fabsf(x); }
  static __device__ __forceinline__ float tiny() { return 1e-30f; }
  static __device__ __forceinline__ float eps() { return 1.1920929e-07f; }
  // quotient for rotation angles only (c and s are then formed consistently from it)
  static __device__ __forceinline__ float fdiv(float a, float b) { return __fdividef(a, b); }
  // nearest rotation in closed form when the product of its eigenvalue gaps is at
  // least this fraction of |Q|^3 (error up to ~6 eps (1 + kappa) there, float)
  static __device__ __forceinline__ float rotation_gate() { return 0.8f; }
  static constexpr int jacobi_sweeps = 6;
  static constexpr int newton_iters = 24;
};
template <> struct Tr<double> {
  static __device__ __forceinline__ double sqrt_(double x) { return sqrt(x); }
  static __device__ __forceinline__ double rsqrt_(double x) { return rsqrt(x); }
  static __device__ __forceinline__ double cbrt_(double x) { return cbrt(x); }
  static __device__ __forceinline__ double log_(double x) { return log(x); }
  static __device__ __forceinline__ double abs_(double x) { return fabs(x); }
  static __device__ __forceinline__ double tiny() { return 1e-300; }
  static __device__ __forceinline__ double eps() { return 2.220446049250313e-16; }
  static __device__ __forceinline__ double fdiv(double a, double b) { return a / b; }
  // (double: its error grows like eps / gate^2, below 1.2e-13 at 0.1)
  static __device__ __forceinline__ double rotation_gate() { return 0.1; }
  static constexpr int jacobi_sweeps = 10;
  static constexpr int newton_iters = 48;
};

// Constants of the method, all in terms of the double machine epsilon 2^-52:
// eps_init = eps_m^(1/4) (SG) or eps_m^(1/8) (SD) for the polar initialization
// (eq. polardecompositionapplied) and the eigenvalue floor sqrt(eps_m) of the P step (Supplemental).
constexpr double kEpsInitSG = 1.220703125e-04;          // 2^-13
constexpr double kEpsInitSD = 1.104854345603981e-02;    // 2^-6.5
constexpr double kSqrtEpsM = 1.4901161193847656e-08;    // 2^-26

// ---------------------------------------------------------------------------
// scalar prox roots: the per-eigenvalue form of w grad f(P) + mu P = mu S
// ---------------------------------------------------------------------------

// Symmetric gradient: (w + mu) p^2 - mu q p - w = 0, positive root per eigenvalue
// (eq. solvesgwithquadraticformula).  Divided by (w + mu): p^2 - t q p - c = 0 with t = mu/(w+mu),
// c = w/(w+mu); for q < 0 the cancellation-free form 2c / (sqrt(disc) - t q).
template <typename R>
__device__ __forceinline__ R prox_root_sg(R q, R w, R mu) {
  const R inv = R(1) / (w + mu);
  const R t = mu * inv, c = w * inv;
  const R tq = t * q;
  const R sd = Tr<R>::sqrt_(tq * tq + R(4) * c);
  return (q >= R(0)) ? R(0.5) * (tq + sd) : (R(2) * c) / (sd - tq);
}

// Symmetric Dirichlet: (w + mu) p^4 - mu q p^3 - w = 0 (eq. peqfsdpluggedin per eigenvalue),
// i.e. g(p) = p^3 (p - a) - c with a = t q.  g is convex and increasing to the
// right of its unique positive root, so Newton started above the root decreases
// monotonically onto it.  Start: for a > 0 the root lies in (a, a + min(c^(1/4),
// c / a^3)]; for a <= 0 it lies in (0, min(c^(1/4), (c/|a|)^(1/3))].
template <typename R>
__device__ __forceinline__ R prox_root_sd(R q, R w, R mu) {
  const R inv = R(1) / (w + mu);
  const R a = mu * inv * q, c = w * inv;
  const R c4 = Tr<R>::sqrt_(Tr<R>::sqrt_(c));
  R p;
  if (a > R(0)) {
    const R a3 = a * a * a;
    p = a + fmin(c4, c / a3);
  } else if (a < R(0)) {
    p = fmin(c4, Tr<R>::cbrt_(c / (-a)));
  } else {
    return c4;
  }
#pragma unroll 1
  for (int it = 0; it < Tr<R>::newton_iters; ++it) {
    const R p2 = p * p;
    const R g = p2 * p * (p - a) - c;
    const R dg = p2 * (R(4) * p - R(3) * a);
    if (!(dg > R(0))) break;
    const R step = g / dg;
    p -= step;
    if (Tr<R>::abs_(step) <= R(2) * Tr<R>::eps() * p) break;
  }
  return p;
}

// Symmetric ARAP, phi(p) = ((p - 1)^2 + (1/p - 1)^2)/2: w phi'(p) + mu (p - q) = 0
// times p^3 is (w + mu) p^4 - (w + mu q) p^3 + w p - w = 0, i.e. g(p) = p^3 (p - a)
// + c (p - 1) with a = (w + mu q)/(w + mu), c = w/(w + mu).  g(0) = -c < 0 and the
// objective is strictly convex on p > 0, so the positive root is unique; it lies
// below max(1, a) (g(1) = 1 - a, g(a) = c (a - 1)), and for a < 0 also below
// (c/|a|)^(1/3) (g there is p^4 + c p > 0).  The root exceeds a/2, so g is convex
// and increasing to its right and Newton from the bound decreases monotonically
// onto it.
template <typename R>
__device__ __forceinline__ R prox_root_sa(R q, R w, R mu) {
  const R inv = R(1) / (w + mu);
  const R a = (w + mu * q) * inv, c = w * inv;
  R p = a >= R(1) ? a : R(1);
  if (a < R(0)) p = fmin(p, Tr<R>::cbrt_(c / (-a)));
#pragma unroll 1
  for (int it = 0; it < Tr<R>::newton_iters; ++it) {
    const R p2 = p * p;
    const R g = p2 * p * (p - a) + c * (p - R(1));
    const R dg = p2 * (R(4) * p - R(3) * a) + c;
    if (!(dg > R(0))) break;
    const R step = g / dg;
    p -= step;
    if (Tr<R>::abs_(step) <= R(2) * Tr<R>::eps() * p) break;
  }
  return p;
}

template <typename R, int ENERGY>
__device__ __forceinline__ R prox_root(R q, R w, R mu) {
  if constexpr (ENERGY == kEnSD) return prox_root_sd<R>(q, w, mu);
  else if constexpr (ENERGY == kEnSG) return prox_root_sg<R>(q, w, mu);
  else return prox_root_sa<R>(q, w, mu);
}

// EN = kEnSD / kEnSG / kEnSA: one energy for all elements; EN = kEnMixed: per
// element, en = that element's energy
template <typename R, int EN>
__device__ __forceinline__ R prox_root_en(R q, R w, R mu, int en) {
  if constexpr (EN == kEnMixed) {
    return en == kEnSD ? prox_root_sd<R>(q, w, mu) : (en == kEnSG ? prox_root_sg<R>(q, w, mu) : prox_root_sa<R>(q, w, mu));
  } else {
    return prox_root<R, EN>(q, w, mu);
  }
}

// f on an SPD matrix with eigenvalues p: SD (sum p^2 + sum p^-2)/2, SG sum p^2/2 - log p,
// SA sum ((p - 1)^2 + (1/p - 1)^2)/2.
template <typename R, int ENERGY, int D>
__device__ __forceinline__ R f_of_eigs(const R p[D]) {
  R s = 0;
#pragma unroll
  for (int j = 0; j < D; ++j) {
    if constexpr (ENERGY == kEnSD) {
      s += R(0.5) * (p[j] * p[j] + R(1) / (p[j] * p[j]));
    } else if constexpr (ENERGY == kEnSG) {
      s += R(0.5) * p[j] * p[j] - Tr<R>::log_(p[j]);
    } else {
      const R u = p[j] - R(1), v = R(1) / p[j] - R(1);
      s += R(0.5) * (u * u + v * v);
    }
  }
  return s;
}

template <typename R, int EN, int D>
__device__ __forceinline__ R f_of_eigs_en(const R p[D], int en) {
  if constexpr (EN == kEnMixed) {
    return en == kEnSD ? f_of_eigs<R, kEnSD, D>(p) : (en == kEnSG ? f_of_eigs<R, kEnSG, D>(p) : f_of_eigs<R, kEnSA, D>(p));
  } else {
    return f_of_eigs<R, EN, D>(p);
  }
}

// ---------------------------------------------------------------------------
// symmetric 3x3 eigen-decomposition by cyclic Jacobi rotations
// ---------------------------------------------------------------------------
template <typename R>
__device__ __forceinline__ void jacobi_rotate(R& app, R& aqq, R& apq, R& arp, R& arq, R V[3][3],
                                              int p, int q) {
  // already diagonal to working precision for this pair: nothing to rotate
  if (!(apq * apq > Tr<R>::eps() * Tr<R>::eps() * Tr<R>::abs_(app * aqq)) || apq == R(0)) return;
  const R theta = Tr<R>::fdiv(aqq - app, R(2) * apq);
  const R at = Tr<R>::abs_(theta);
  R t = Tr<R>::fdiv(R(1), at + Tr<R>::sqrt_(at * at + R(1)));
  if (at * Tr<R>::eps() > R(1)) t = R(0.5) / at;  // theta^2 would overflow
  t = (theta < R(0)) ? -t : t;
  const R c = Tr<R>::rsqrt_(t * t + R(1));
  const R s = t * c;
  app -= t * apq;
  aqq += t * apq;
  apq = R(0);
  const R rp = c * arp - s * arq;
  const R rq = s * arp + c * arq;
  arp = rp;
  arq = rq;
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    const R vp = V[r][p], vq = V[r][q];
    V[r][p] = c * vp - s * vq;
    V[r][q] = s * vp + c * vq;
  }
}

// In: symmetric (a00,a01,a02,a11,a12,a22).  Out: eigenvalues ev and eigenvectors
// in the columns of V (orthonormal, det +1).
template <typename R>
__device__ __forceinline__ void sym3_eig(R a00, R a01, R a02, R a11, R a12, R a22, R ev[3], R V[3][3]) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) V[i][j] = (i == j) ? R(1) : R(0);
  const R scale2 = a00 * a00 + a11 * a11 + a22 * a22 + R(2) * (a01 * a01 + a02 * a02 + a12 * a12);
#pragma unroll 1
  for (int sw = 0; sw < Tr<R>::jacobi_sweeps; ++sw) {
    const R off = a01 * a01 + a02 * a02 + a12 * a12;
    if (off <= Tr<R>::eps() * Tr<R>::eps() * scale2 || off <= Tr<R>::tiny()) break;
    jacobi_rotate<R>(a00, a11, a01, a02, a12, V, 0, 1);  // r = 2: (a20, a21)
    jacobi_rotate<R>(a00, a22, a02, a01, a12, V, 0, 2);  // r = 1: (a10, a12)
    jacobi_rotate<R>(a11, a22, a12, a01, a02, V, 1, 2);  // r = 0: (a01, a02)
  }
  ev[0] = a00;
  ev[1] = a11;
  ev[2] = a22;
}

// ---------------------------------------------------------------------------
// Eigenvalues of a symmetric 3x3 in closed form (the trigonometric solution of
// the characteristic cubic): with q = tr S / 3, B = S - q I, s = |B|_F / sqrt(6)
// and r = det(B / s) / 2 in [-1, 1], the eigenvalues are q + 2 s cos(phi + 2 pi
// k / 3), phi = acos(r) / 3; returned in descending order.  Near a repeated
// eigenvalue acos loses accuracy, which the matrix-function form below tolerates.
// ---------------------------------------------------------------------------
template <typename R>
__device__ __forceinline__ void sym3_eigvals(R a00, R a01, R a02, R a11, R a12, R a22, R lam[3]) {
  const R q = (a00 + a11 + a22) * R(1.0 / 3.0);
  const R b00 = a00 - q, b11 = a11 - q, b22 = a22 - q;
  const R off = a01 * a01 + a02 * a02 + a12 * a12;
  const R s2 = (b00 * b00 + b11 * b11 + b22 * b22 + R(2) * off) * R(1.0 / 6.0);
  if (!(s2 > Tr<R>::tiny())) {
    lam[0] = lam[1] = lam[2] = q;
    return;
  }
  const R sd = Tr<R>::sqrt_(s2);
  const R is = R(1) / sd;
  const R c00 = b00 * is, c11 = b11 * is, c22 = b22 * is, c01 = a01 * is, c02 = a02 * is, c12 = a12 * is;
  R r = R(0.5) * (c00 * (c11 * c22 - c12 * c12) - c01 * (c01 * c22 - c12 * c02) + c02 * (c01 * c12 - c11 * c02));
  r = fmin(fmax(r, R(-1)), R(1));
  const R phi = acos(r) * R(1.0 / 3.0);
  lam[0] = q + R(2) * sd * cos(phi);
  lam[2] = q + R(2) * sd * cos(phi + R(2.0943951023931957));   // + 2 pi / 3
  lam[1] = R(3) * q - lam[0] - lam[2];
}

// h[p1, p2], the divided difference of the inverse of the scalar prox map,
// q = h(p) = p + (w / mu) phi'(p) (w phi'(p) + mu (p - q) = 0, the per-eigenvalue
// form of eq. rootfindinginp), written without cancellation so that it also holds
// at p1 = p2 (then it is h'(p)): SD phi' = p - p^-3, SG phi' = p - 1/p, SA phi' =
// p - 1 - p^-3 + p^-2.  1 / h[p1, p2] is the divided difference of the prox map.
template <typename R, int EN>
__device__ __forceinline__ R prox_inverse_dd(R p1, R p2, R w, R mu, int en) {
  const int e = (EN == kEnMixed) ? en : EN;
  const R pp = p1 * p2;
  R dphi;
  if (e == kEnSG) {
    dphi = R(1) + R(1) / pp;
  } else {
    const R a = (p1 * p1 + pp + p2 * p2) / (pp * pp * pp);
    dphi = (e == kEnSD) ? R(1) + a : R(1) + a - (p1 + p2) / (pp * pp);
  }
  return R(1) + (w / mu) * dphi;
}

// ---------------------------------------------------------------------------
// The penalty bound of the paper's schedule (Lemma 1, Proposition 1, Sec. 6), in
// double.  gnorm2 = |grad f(P)|^2; B = sqrt(5 (1 + gnorm2)); C^L (SG) is the
// positive root of x^2 + B x - 1 (written as 2 / (B + sqrt(B^2 + 4)) to avoid
// cancellation), C^LG (SD) the positive root of x^4 + B x^3 - 1, which is
// increasing and convex on [0, 1] with value B >= 0 at 1, so Newton from 1 falls
// monotonically onto it; F = 1 + sqrt(d)/(C^L)^2 (SG) or 1 + 3 sqrt(d)/(C^LG)^4
// (SD), F^2 capped at eps_m^(-1/4); mu_min = (-w + sqrt(w^2 + 16 w^2 F^2)) / 2
// (gamma = 1, eps = 0).
// ---------------------------------------------------------------------------
template <int D>
__device__ __forceinline__ double penalty_mu_min(double gnorm2, double w, bool sg) {
  const double B = sqrt(5.0 * (1.0 + gnorm2));
  double F;
  if (sg) {
    const double C = 2.0 / (B + sqrt(B * B + 4.0));
    F = 1.0 + sqrt((double)D) / (C * C);
  } else {
    double x = 1.0;
#pragma unroll 1
    for (int it = 0; it < 200; ++it) {
      const double g = x * x * x * (x + B) - 1.0;
      const double dg = x * x * (4.0 * x + 3.0 * B);
      const double xn = x - g / dg;
      if (!(xn < x)) break;
      x = xn;
    }
    const double x2 = x * x;
    F = 1.0 + 3.0 * sqrt((double)D) / (x2 * x2);
  }
  F = fmin(F, sqrt(8192.0));   // F^2 <= eps_m^(-1/4) = 2^13
  return 0.5 * (-w + sqrt(w * w + 16.0 * w * w * F * F));
}

// ---------------------------------------------------------------------------
// signed 3x3 SVD: Q = U diag(s) V^T with U, V in SO(3), |s0| >= |s1| >= |s2|,
// s0, s1 >= 0 and sign(s2) = sign(det Q).  Jacobi on Q^T Q gives V; Givens QR
// of Q V gives U and the signed diagonal.
// ---------------------------------------------------------------------------
template <typename R>
__device__ __forceinline__ void givens_rows(R B[3][3], R U[3][3], int p, int q, int col) {
  const R a = B[p][col], b = B[q][col];
  const R r2 = a * a + b * b;
  R c = R(1), s = R(0);
  if (r2 > Tr<R>::tiny()) {
    const R ir = Tr<R>::rsqrt_(r2);
    c = a * ir;
    s = b * ir;
  }
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const R bp = B[p][k], bq = B[q][k];
    B[p][k] = c * bp + s * bq;
    B[q][k] = -s * bp + c * bq;
    const R up = U[k][p], uq = U[k][q];
    U[k][p] = c * up + s * uq;
    U[k][q] = -s * up + c * uq;
  }
}

template <typename R>
__device__ __forceinline__ void swap_cols_neg(R A[3][3], int i, int j) {
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    const R t = A[r][i];
    A[r][i] = A[r][j];
    A[r][j] = -t;
  }
}

template <typename R>
__device__ __forceinline__ void svd3_signed(const R Q[3][3], R U[3][3], R s[3], R V[3][3]) {
  R a00 = 0, a01 = 0, a02 = 0, a11 = 0, a12 = 0, a22 = 0;
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    a00 += Q[r][0] * Q[r][0];
    a01 += Q[r][0] * Q[r][1];
    a02 += Q[r][0] * Q[r][2];
    a11 += Q[r][1] * Q[r][1];
    a12 += Q[r][1] * Q[r][2];
    a22 += Q[r][2] * Q[r][2];
  }
  R ev[3];
  sym3_eig<R>(a00, a01, a02, a11, a12, a22, ev, V);
  R B[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) B[i][j] = Q[i][0] * V[0][j] + Q[i][1] * V[1][j] + Q[i][2] * V[2][j];
  R n0 = B[0][0] * B[0][0] + B[1][0] * B[1][0] + B[2][0] * B[2][0];
  R n1 = B[0][1] * B[0][1] + B[1][1] * B[1][1] + B[2][1] * B[2][1];
  R n2 = B[0][2] * B[0][2] + B[1][2] * B[1][2] + B[2][2] * B[2][2];
  if (n0 < n1) { swap_cols_neg<R>(B, 0, 1); swap_cols_neg<R>(V, 0, 1); R t = n0; n0 = n1; n1 = t; }
  if (n0 < n2) { swap_cols_neg<R>(B, 0, 2); swap_cols_neg<R>(V, 0, 2); R t = n0; n0 = n2; n2 = t; }
  if (n1 < n2) { swap_cols_neg<R>(B, 1, 2); swap_cols_neg<R>(V, 1, 2); R t = n1; n1 = n2; n2 = t; }
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) U[i][j] = (i == j) ? R(1) : R(0);
  givens_rows<R>(B, U, 0, 1, 0);
  givens_rows<R>(B, U, 0, 2, 0);
  givens_rows<R>(B, U, 1, 2, 1);
  s[0] = B[0][0];
  s[1] = B[1][1];
  s[2] = B[2][2];
}

// ---------------------------------------------------------------------------
// nearest rotation (SO(3) Procrustes, eq. optimizationinudecoupled) by one-sided
// Jacobi: plane rotations of the columns of B = Q V until they are orthogonal
// (no Q^T Q, so the condition number is not squared).  Then Q = [s_j u_j] V^T;
// with k the smallest column, u_k := u_{k+1} x u_{k+2} makes U a rotation and
// puts the sign of det Q on the smallest singular value, so R = U V^T is the
// rotation closest to Q.  cond returns (s_mid + s_min_signed) / s_max, the
// conditioning of R (R is ill-determined when it is tiny).
// ---------------------------------------------------------------------------
template <typename R>
__device__ __forceinline__ void onesided_rotate(R B[3][3], R V[3][3], int p, int q) {
  R al = 0, be = 0, ga = 0;
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    al = fma(B[r][p], B[r][p], al);
    be = fma(B[r][q], B[r][q], be);
    ga = fma(B[r][p], B[r][q], ga);
  }
  if (!(Tr<R>::abs_(ga) > Tr<R>::eps() * Tr<R>::sqrt_(al * be)) || ga == R(0)) return;
  const R zeta = Tr<R>::fdiv(be - al, R(2) * ga);
  const R az = Tr<R>::abs_(zeta);
  R t = Tr<R>::fdiv(R(1), az + Tr<R>::sqrt_(az * az + R(1)));
  if (az * Tr<R>::eps() > R(1)) t = R(0.5) / az;
  t = (zeta < R(0)) ? -t : t;
  const R c = Tr<R>::rsqrt_(t * t + R(1));
  const R sn = t * c;
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    const R bp = B[r][p], bq = B[r][q];
    B[r][p] = c * bp - sn * bq;
    B[r][q] = sn * bp + c * bq;
    const R vp = V[r][p], vq = V[r][q];
    V[r][p] = c * vp - sn * vq;
    V[r][q] = sn * vp + c * vq;
  }
}

// Full form: also returns V (columns = right singular vectors, det +1) and the
// signed singular values sig with Q = Rot V diag(sig) V^T (sig[k] < 0 when
// det Q < 0), which the adjoint of the rotation needs.
template <typename R>
__device__ __forceinline__ void polar3(const R Q[3][3], R Rot[3][3], R Vout[3][3], R sig[3], R& cond) {
  R B[3][3], V[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      B[i][j] = Q[i][j];
      V[i][j] = (i == j) ? R(1) : R(0);
    }
#pragma unroll 1
  for (int sw = 0; sw < Tr<R>::jacobi_sweeps; ++sw) {
    onesided_rotate<R>(B, V, 0, 1);
    onesided_rotate<R>(B, V, 0, 2);
    onesided_rotate<R>(B, V, 1, 2);
    // converged when every column pair is orthogonal to working precision
    R worst = 0;
#pragma unroll
    for (int pq = 0; pq < 3; ++pq) {
      const int p = pq == 2 ? 1 : 0, q = pq == 0 ? 1 : 2;
      R al = 0, be = 0, ga = 0;
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        al = fma(B[r][p], B[r][p], al);
        be = fma(B[r][q], B[r][q], be);
        ga = fma(B[r][p], B[r][q], ga);
      }
      worst = fmax(worst, ga * ga - R(16) * Tr<R>::eps() * Tr<R>::eps() * al * be);
    }
    if (!(worst > R(0))) break;
  }
  // Columns by norm: big, mid and the smallest k.  The columns are picked with
  // selects (no runtime index into a register array, which would put the arrays
  // in local memory).
  const R n0 = B[0][0] * B[0][0] + B[1][0] * B[1][0] + B[2][0] * B[2][0];
  const R n1 = B[0][1] * B[0][1] + B[1][1] * B[1][1] + B[2][1] * B[2][1];
  const R n2 = B[0][2] * B[0][2] + B[1][2] * B[1][2] + B[2][2] * B[2][2];
  const int k = (n0 <= n1 && n0 <= n2) ? 0 : ((n1 <= n2) ? 1 : 2);
  const int a = (k + 1) % 3, b = (k + 2) % 3;
  const R na = (a == 0) ? n0 : ((a == 1) ? n1 : n2);
  const R nb = (b == 0) ? n0 : ((b == 1) ? n1 : n2);
  const int big = na >= nb ? a : b, mid = na >= nb ? b : a;
  const R nbig = na >= nb ? na : nb, nmid = na >= nb ? nb : na;
  auto pick = [](int c, R x0, R x1, R x2) { return c == 0 ? x0 : (c == 1 ? x1 : x2); };
  R Bb[3], Bm[3], Bk[3], Vb[3], Vm[3], Vk[3];
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    Bb[r] = pick(big, B[r][0], B[r][1], B[r][2]);
    Bm[r] = pick(mid, B[r][0], B[r][1], B[r][2]);
    Bk[r] = pick(k, B[r][0], B[r][1], B[r][2]);
    Vb[r] = pick(big, V[r][0], V[r][1], V[r][2]);
    Vm[r] = pick(mid, V[r][0], V[r][1], V[r][2]);
    Vk[r] = pick(k, V[r][0], V[r][1], V[r][2]);
  }
  // u_big: normalized largest column (Q = 0: any rotation is optimal, take I)
  R ub[3], um[3], uk[3];
  if (nbig > Tr<R>::tiny()) {
    const R inv = Tr<R>::rsqrt_(nbig);
#pragma unroll
    for (int r = 0; r < 3; ++r) ub[r] = Bb[r] * inv;
  } else {
#pragma unroll
    for (int r = 0; r < 3; ++r) ub[r] = R(big == r);
  }
  // u_mid: middle column made orthogonal to u_big (rank-1 Q: any orthogonal unit vector)
  const R dp = Bm[0] * ub[0] + Bm[1] * ub[1] + Bm[2] * ub[2];
#pragma unroll
  for (int r = 0; r < 3; ++r) um[r] = Bm[r] - dp * ub[r];
  R nm = um[0] * um[0] + um[1] * um[1] + um[2] * um[2];
  if (!(nm > Tr<R>::eps() * Tr<R>::eps() * nbig) || !(nm > Tr<R>::tiny())) {
    // the coordinate axis least aligned with u_big, orthogonalized
    const int ax = (Tr<R>::abs_(ub[0]) <= Tr<R>::abs_(ub[1]) && Tr<R>::abs_(ub[0]) <= Tr<R>::abs_(ub[2])) ? 0
                   : (Tr<R>::abs_(ub[1]) <= Tr<R>::abs_(ub[2]) ? 1 : 2);
    const R uax = pick(ax, ub[0], ub[1], ub[2]);
#pragma unroll
    for (int r = 0; r < 3; ++r) um[r] = R(r == ax) - uax * ub[r];
    nm = um[0] * um[0] + um[1] * um[1] + um[2] * um[2];
  }
  const R invm = Tr<R>::rsqrt_(nm);
#pragma unroll
  for (int r = 0; r < 3; ++r) um[r] *= invm;
  // u_k = u_a x u_b (cyclic order keeps det U = +1): u_big x u_mid when big = a,
  // its negative otherwise
  const R sgn = (big == a) ? R(1) : R(-1);
  uk[0] = sgn * (ub[1] * um[2] - ub[2] * um[1]);
  uk[1] = sgn * (ub[2] * um[0] - ub[0] * um[2]);
  uk[2] = sgn * (ub[0] * um[1] - ub[1] * um[0]);
  // Rot = U V^T = u_big V_big^T + u_mid V_mid^T + u_k V_k^T
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) Rot[i][j] = ub[i] * Vb[j] + um[i] * Vm[j] + uk[i] * Vk[j];
  // signed singular values s_j = u_j . B_j (s_k < 0 when det Q < 0), in the
  // original column order
  const R sb = ub[0] * Bb[0] + ub[1] * Bb[1] + ub[2] * Bb[2];
  const R sm = um[0] * Bm[0] + um[1] * Bm[1] + um[2] * Bm[2];
  const R sk = uk[0] * Bk[0] + uk[1] * Bk[1] + uk[2] * Bk[2];
#pragma unroll
  for (int j = 0; j < 3; ++j) sig[j] = (j == big) ? sb : ((j == mid) ? sm : sk);
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) Vout[i][j] = V[i][j];
  const R smax = Tr<R>::sqrt_(nbig);
  cond = (smax > R(0)) ? (Tr<R>::sqrt_(nmid) + sk) / smax : R(1);
}

template <typename R>
__device__ __forceinline__ void nearest_rotation3(const R Q[3][3], R Rot[3][3], R& cond) {
  R V[3][3], sig[3];
  polar3<R>(Q, Rot, V, sig, cond);
}

// ---------------------------------------------------------------------------
// Nearest rotation as a unit quaternion (the float U step of the 3D local step).
// For R(q), q = (w, x, y, z) unit (the matrix of quat_to_rot below),
// tr(R(q)^T Q) = q^T K q with the symmetric, traceless 4x4
//   K = [ Q00+Q11+Q22  Q21-Q12      Q02-Q20      Q10-Q01     ]
//       [ Q21-Q12      Q00-Q11-Q22  Q01+Q10      Q02+Q20     ]
//       [ Q02-Q20      Q01+Q10     -Q00+Q11-Q22  Q12+Q21     ]
//       [ Q10-Q01      Q02+Q20      Q12+Q21     -Q00-Q11+Q22 ]
// (expand R(q) entry by entry), so the rotation maximizing tr(R^T Q) -- the one
// nearest to Q, eq. optimizationinudecoupled -- is the unit eigenvector of K's
// largest eigenvalue (Horn's closed-form absolute orientation, 1987).  That
// eigenvalue is the largest root of det(K - l I) = l^4 - 2|Q|^2 l^2 - 8 det(Q) l
// + det K (the power sums of K's eigenvalues are 0, 4|Q|^2 and 24 det Q).  All its
// roots are real, so Newton started above the largest root, at sqrt(3)|Q| (the
// sum of the singular values is at most that), falls monotonically onto it.  The
// eigenvector is the column of adj(K - l I) with the largest diagonal entry.
// adj(K - l I) = c v v^T with c the product of the gaps between l and the other
// three eigenvalues, so |column|^2 / |diagonal entry| = |c|; cond = |c| / |Q|^3 is
// about 8 (s_mid + s_min,signed) / s_max for a flat Q and 12 for a rotation.  In
// float the eigenvector is accurate to a few eps (1 + kappa) only while the gaps
// are large; for cond below about 1 the caller takes another method.
// ---------------------------------------------------------------------------
template <typename R>
__device__ __forceinline__ R det3(R a00, R a01, R a02, R a10, R a11, R a12, R a20, R a21, R a22) {
  return a00 * (a11 * a22 - a12 * a21) - a01 * (a10 * a22 - a12 * a20) + a02 * (a10 * a21 - a11 * a20);
}

template <typename R>
__device__ __forceinline__ void nearest_rotation3_quat(const R Q[3][3], R qv[4], R& cond) {
  R K[4][4];
  K[0][0] = Q[0][0] + Q[1][1] + Q[2][2];
  K[1][1] = Q[0][0] - Q[1][1] - Q[2][2];
  K[2][2] = -Q[0][0] + Q[1][1] - Q[2][2];
  K[3][3] = -Q[0][0] - Q[1][1] + Q[2][2];
  K[0][1] = K[1][0] = Q[2][1] - Q[1][2];
  K[0][2] = K[2][0] = Q[0][2] - Q[2][0];
  K[0][3] = K[3][0] = Q[1][0] - Q[0][1];
  K[1][2] = K[2][1] = Q[0][1] + Q[1][0];
  K[1][3] = K[3][1] = Q[0][2] + Q[2][0];
  K[2][3] = K[3][2] = Q[1][2] + Q[2][1];
  R n2 = 0;
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) n2 = fma(Q[a][b], Q[a][b], n2);
  if (!(n2 > Tr<R>::tiny())) {   // Q = 0: every rotation is optimal, take I
    qv[0] = R(1); qv[1] = qv[2] = qv[3] = R(0);
    cond = R(1);
    return;
  }
  const R dQ = det3<R>(Q[0][0], Q[0][1], Q[0][2], Q[1][0], Q[1][1], Q[1][2], Q[2][0], Q[2][1], Q[2][2]);
  // det K by 2x2 minors of the first two and the last two rows
  const R m01 = K[0][0] * K[1][1] - K[0][1] * K[1][0], m02 = K[0][0] * K[1][2] - K[0][2] * K[1][0];
  const R m03 = K[0][0] * K[1][3] - K[0][3] * K[1][0], m12 = K[0][1] * K[1][2] - K[0][2] * K[1][1];
  const R m13 = K[0][1] * K[1][3] - K[0][3] * K[1][1], m23 = K[0][2] * K[1][3] - K[0][3] * K[1][2];
  const R n01 = K[2][0] * K[3][1] - K[2][1] * K[3][0], n02 = K[2][0] * K[3][2] - K[2][2] * K[3][0];
  const R n03 = K[2][0] * K[3][3] - K[2][3] * K[3][0], n12 = K[2][1] * K[3][2] - K[2][2] * K[3][1];
  const R n13 = K[2][1] * K[3][3] - K[2][3] * K[3][1], n23 = K[2][2] * K[3][3] - K[2][3] * K[3][2];
  const R dK = m01 * n23 - m02 * n13 + m03 * n12 + m12 * n03 - m13 * n02 + m23 * n01;
  const R c2 = R(-2) * n2, c1 = R(-8) * dQ;
  R l = Tr<R>::sqrt_(R(3) * n2);
#pragma unroll 1
  for (int it = 0; it < 32; ++it) {
    const R l2 = l * l;
    const R p = (l2 + c2) * l2 + c1 * l + dK;
    const R dp = (R(4) * l2 + R(2) * c2) * l + c1;
    if (!(dp > R(0))) break;
    const R step = p / dp;
    l -= step;
    if (!(Tr<R>::abs_(step) > R(4) * Tr<R>::eps() * l)) break;
  }
  // adjugate of M = K - l I: the diagonal cofactors pick the best column
  R M[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) M[a][b] = K[a][b] - (a == b ? l : R(0));
  const R a0 = det3<R>(M[1][1], M[1][2], M[1][3], M[2][1], M[2][2], M[2][3], M[3][1], M[3][2], M[3][3]);
  const R a1 = det3<R>(M[0][0], M[0][2], M[0][3], M[2][0], M[2][2], M[2][3], M[3][0], M[3][2], M[3][3]);
  const R a2 = det3<R>(M[0][0], M[0][1], M[0][3], M[1][0], M[1][1], M[1][3], M[3][0], M[3][1], M[3][3]);
  const R a3 = det3<R>(M[0][0], M[0][1], M[0][2], M[1][0], M[1][1], M[1][2], M[2][0], M[2][1], M[2][2]);
  // the eigenvalue is the largest, so every diagonal cofactor is <= 0 (a product of
  // three non-positive gaps times v_j^2): take the largest in magnitude
  const R b0 = Tr<R>::abs_(a0), b1 = Tr<R>::abs_(a1), b2 = Tr<R>::abs_(a2), b3 = Tr<R>::abs_(a3);
  int j = 0;
  R best = b0;
  if (b1 > best) { best = b1; j = 1; }
  if (b2 > best) { best = b2; j = 2; }
  if (b3 > best) { best = b3; j = 3; }
  // column j of the adjugate: cofactors C_ij = (-1)^(i+j) det(M minus row i, column j);
  // M is symmetric, so column j equals row j of the cofactor matrix
  R v[4];
  {
    // rows other than j, in order
    const int r0 = j == 0 ? 1 : 0, r1 = j <= 1 ? 2 : 1, r2 = j <= 2 ? 3 : 2;
    R A[3][4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      A[0][c] = r0 == 0 ? M[0][c] : (r0 == 1 ? M[1][c] : M[2][c]);
      A[1][c] = r1 == 1 ? M[1][c] : (r1 == 2 ? M[2][c] : M[3][c]);
      A[2][c] = r2 == 2 ? M[2][c] : M[3][c];
    }
    // v_i = (-1)^(i+j) det(A minus column i)
    const R d0 = det3<R>(A[0][1], A[0][2], A[0][3], A[1][1], A[1][2], A[1][3], A[2][1], A[2][2], A[2][3]);
    const R d1 = det3<R>(A[0][0], A[0][2], A[0][3], A[1][0], A[1][2], A[1][3], A[2][0], A[2][2], A[2][3]);
    const R d2 = det3<R>(A[0][0], A[0][1], A[0][3], A[1][0], A[1][1], A[1][3], A[2][0], A[2][1], A[2][3]);
    const R d3 = det3<R>(A[0][0], A[0][1], A[0][2], A[1][0], A[1][1], A[1][2], A[2][0], A[2][1], A[2][2]);
    const R sj = (j & 1) ? R(-1) : R(1);
    v[0] = sj * d0;
    v[1] = -sj * d1;
    v[2] = sj * d2;
    v[3] = -sj * d3;
  }
  const R vn = v[0] * v[0] + v[1] * v[1] + v[2] * v[2] + v[3] * v[3];
  const R sc = n2 * Tr<R>::sqrt_(n2);
  cond = (best > R(0)) ? vn / (best * sc) : R(0);
  if (!(vn > Tr<R>::tiny())) {
    qv[0] = R(1); qv[1] = qv[2] = qv[3] = R(0);
    cond = R(0);
    return;
  }
  const R inv = Tr<R>::rsqrt_(vn);
#pragma unroll
  for (int k = 0; k < 4; ++k) qv[k] = v[k] * inv;
}

// ---------------------------------------------------------------------------
// rotations <-> compact storage
// ---------------------------------------------------------------------------
template <typename R>
__device__ __forceinline__ void rot_to_quat(const R M[3][3], R qv[4]) {  // (w, x, y, z)
  const R tr = M[0][0] + M[1][1] + M[2][2];
  R w, x, y, z;
  if (tr > R(0)) {
    const R s = Tr<R>::sqrt_(tr + R(1)) * R(2);
    w = R(0.25) * s; x = (M[2][1] - M[1][2]) / s; y = (M[0][2] - M[2][0]) / s; z = (M[1][0] - M[0][1]) / s;
  } else if (M[0][0] > M[1][1] && M[0][0] > M[2][2]) {
    const R s = Tr<R>::sqrt_(R(1) + M[0][0] - M[1][1] - M[2][2]) * R(2);
    w = (M[2][1] - M[1][2]) / s; x = R(0.25) * s; y = (M[0][1] + M[1][0]) / s; z = (M[0][2] + M[2][0]) / s;
  } else if (M[1][1] > M[2][2]) {
    const R s = Tr<R>::sqrt_(R(1) + M[1][1] - M[0][0] - M[2][2]) * R(2);
    w = (M[0][2] - M[2][0]) / s; x = (M[0][1] + M[1][0]) / s; y = R(0.25) * s; z = (M[1][2] + M[2][1]) / s;
  } else {
    const R s = Tr<R>::sqrt_(R(1) + M[2][2] - M[0][0] - M[1][1]) * R(2);
    w = (M[1][0] - M[0][1]) / s; x = (M[0][2] + M[2][0]) / s; y = (M[1][2] + M[2][1]) / s; z = R(0.25) * s;
  }
  const R nrm = Tr<R>::rsqrt_(w * w + x * x + y * y + z * z);
  qv[0] = w * nrm; qv[1] = x * nrm; qv[2] = y * nrm; qv[3] = z * nrm;
}

template <typename R>
__device__ __forceinline__ void quat_to_rot(const R qv[4], R M[3][3]) {
  const R w = qv[0], x = qv[1], y = qv[2], z = qv[3];
  M[0][0] = R(1) - R(2) * (y * y + z * z); M[0][1] = R(2) * (x * y - z * w); M[0][2] = R(2) * (x * z + y * w);
  M[1][0] = R(2) * (x * y + z * w); M[1][1] = R(1) - R(2) * (x * x + z * z); M[1][2] = R(2) * (y * z - x * w);
  M[2][0] = R(2) * (x * z - y * w); M[2][1] = R(2) * (y * z + x * w); M[2][2] = R(1) - R(2) * (x * x + y * y);
}

// ---------------------------------------------------------------------------
// double-float accumulation (two floats carry ~48 significant bits), used where
// sums of many float terms must keep double-level accuracy on the FP32 path.
// ---------------------------------------------------------------------------
struct FF {
  float hi, lo;
};
__device__ __forceinline__ FF ff_add(FF a, FF b) {
  const float s = a.hi + b.hi;
  const float bb = s - a.hi;
  float e = (a.hi - (s - bb)) + (b.hi - bb);
  e += a.lo + b.lo;
  const float hi = s + e;
  return FF{hi, e - (hi - s)};
}
__device__ __forceinline__ FF ff_addf(FF a, float b) { return ff_add(a, FF{b, 0.0f}); }

}  // namespace ffa
