// Reverse mode through unrolled iterations of Algorithm 1 (the paper has no
// differentiation; this is the adjoint of its W, U, P and Lambda steps).
//
// Iteration k maps state_{k-1} = (U, P, Lambda)^{k-1} to state_k:
//   W^k   = W step of r^k = mu (U^{k-1} P^{k-1} - Lambda^{k-1}) and the pins b
//           (eq. solvinginw), J = G W^k,
//   A     = J + Lambda^{k-1},  Q = A P^{k-1},  U^k = nearest rotation to Q
//           (eq. optimizationinudecoupled, h = 0),
//   S     = symm(U^k^T A),  P^k = prox(S) eigenvalue by eigenvalue
//           (eqs. optimizinginp/rootfindinginp),
//   Lambda^k = Lambda^{k-1} + J - U^k P^k (eq. lambdaupdate).
// The element kernel below applies, for one element and one iteration k, the
// vector-Jacobian products of these steps in reverse order.  The W step's
// adjoint is a solve with the same symmetric operator L_FF (done by the caller
// with the factor) whose solution xi enters the next element kernel through
// r_bar = mu G xi.
#include "ffa_internal.h"
#include "ffa_math.cuh"

namespace ffa {
namespace {

template <int D, typename R>
__device__ __forceinline__ void load_vertex_a(const void* rec, int v, R hi[D], R lo[D]) {
  if constexpr (sizeof(R) == 4) {
    const float4* r = reinterpret_cast<const float4*>(rec) + (int64_t)v * D;
    if constexpr (D == 3) {
      const float4 a = __ldg(r), b = __ldg(r + 1);
      hi[0] = a.x; hi[1] = a.y; hi[2] = a.z;
      lo[0] = b.x; lo[1] = b.y; lo[2] = b.z;
    } else {
      const float4 a = __ldg(r);
      hi[0] = a.x; hi[1] = a.y; lo[0] = a.z; lo[1] = a.w;
    }
  } else {
    const double2* r = reinterpret_cast<const double2*>(rec) + (int64_t)v * D;
    if constexpr (D == 3) {
      const double2 a = __ldg(r), b = __ldg(r + 1);
      hi[0] = a.x; hi[1] = a.y; hi[2] = b.x;
    } else {
      const double2 a = __ldg(r);
      hi[0] = a.x; hi[1] = a.y;
    }
#pragma unroll
    for (int k = 0; k < D; ++k) lo[k] = R(0);
  }
}

// derivative of the scalar prox root p(q): implicit differentiation of
// (w+mu) p^2 - mu q p - w = 0 (SG), (w+mu) p^4 - mu q p^3 - w = 0 (SD) or
// (w+mu) p^4 - (w + mu q) p^3 + w p - w = 0 (SA)
template <typename R, int EN>
__device__ __forceinline__ R prox_root_deriv(R p, R q, R w, R mu) {
  if constexpr (EN == kEnSD) return mu * p / (R(4) * (w + mu) * p - R(3) * mu * q);
  else if constexpr (EN == kEnSG) return mu * p / (R(2) * (w + mu) * p - mu * q);
  else return mu * p * p * p / ((R(4) * (w + mu) * p - R(3) * (w + mu * q)) * p * p + w);
}

template <int D, typename R, int EN>
__global__ void __launch_bounds__(128) k_adjoint_local(AdjointLaunch a) {
  const int i = blockIdx.x * 128 + threadIdx.x;
  if (i >= a.m) return;
  const int m = a.m;
  const R* gp = reinterpret_cast<const R*>(a.e.g);
  int vid[D + 1];
#pragma unroll
  for (int j = 0; j <= D; ++j) vid[j] = __ldg(a.e.idx + (int64_t)j * m + i);
  R g[D][D];
#pragma unroll
  for (int j = 0; j < D; ++j)
#pragma unroll
    for (int c = 0; c < D; ++c) g[j][c] = __ldg(gp + (int64_t)(j * D + c) * m + i);
  const R w = reinterpret_cast<const R*>(a.e.w)[i];
  const R mu = reinterpret_cast<const R*>(a.e.mu)[i];
  // ---- recompute the forward of iteration k for this element
  R J[D][D];
  {
    R h0[D], l0[D];
    load_vertex_a<D, R>(a.vrec, vid[0], h0, l0);
#pragma unroll
    for (int r = 0; r < D; ++r)
#pragma unroll
      for (int c = 0; c < D; ++c) J[r][c] = R(0);
#pragma unroll
    for (int j = 0; j < D; ++j) {
      R hj[D], lj[D];
      load_vertex_a<D, R>(a.vrec, vid[j + 1], hj, lj);
#pragma unroll
      for (int c = 0; c < D; ++c) {
        const R del = (hj[c] - h0[c]) + (lj[c] - l0[c]);
#pragma unroll
        for (int r = 0; r < D; ++r) J[r][c] = fma(g[j][r], del, J[r][c]);
      }
    }
  }
  const R* P0p = reinterpret_cast<const R*>(a.P_prev);
  const R* L0p = reinterpret_cast<const R*>(a.Lam_prev);
  R P0[D][D], L0[D][D], A[D][D];
  if constexpr (D == 2) {
    P0[0][0] = P0p[i]; P0[0][1] = P0[1][0] = P0p[(int64_t)m + i]; P0[1][1] = P0p[2 * (int64_t)m + i];
  } else {
    P0[0][0] = P0p[i]; P0[0][1] = P0[1][0] = P0p[(int64_t)m + i]; P0[0][2] = P0[2][0] = P0p[2 * (int64_t)m + i];
    P0[1][1] = P0p[3 * (int64_t)m + i]; P0[1][2] = P0[2][1] = P0p[4 * (int64_t)m + i]; P0[2][2] = P0p[5 * (int64_t)m + i];
  }
#pragma unroll
  for (int r = 0; r < D; ++r)
#pragma unroll
    for (int c = 0; c < D; ++c) {
      L0[r][c] = L0p[(int64_t)(r * D + c) * m + i];
      A[r][c] = J[r][c] + L0[r][c];
    }
  R Q[D][D];
#pragma unroll
  for (int r = 0; r < D; ++r)
#pragma unroll
    for (int c = 0; c < D; ++c) {
      R s = R(0);
#pragma unroll
      for (int l = 0; l < D; ++l) s = fma(A[r][l], P0[l][c], s);
      Q[r][c] = s;
    }
  // rotation and the pieces of its derivative
  R U[D][D], Vq[D][D], sg[D];
  bool tie = false;
  if constexpr (D == 2) {
    const R ca = Q[0][0] + Q[1][1], sa = Q[1][0] - Q[0][1];
    const R r2 = ca * ca + sa * sa;
    R c = R(1), s = R(0);
    if (r2 > R(0)) {
      const R ir = Tr<R>::rsqrt_(r2);
      c = ca * ir;
      s = sa * ir;
    } else {
      tie = true;
      const R* Up = reinterpret_cast<const R*>(a.U_prev);
      c = Up[i];
      s = Up[(int64_t)m + i];
    }
    U[0][0] = c; U[0][1] = -s; U[1][0] = s; U[1][1] = c;
    sg[0] = sg[1] = R(0.5) * Tr<R>::sqrt_(r2);  // only sg[0] + sg[1] = |(ca, sa)| is used
    Vq[0][0] = Vq[1][1] = R(1);
    Vq[0][1] = Vq[1][0] = R(0);
  } else {
    R cond;
    polar3<R>(Q, U, Vq, sg, cond);
  }
  R S[D][D];
#pragma unroll
  for (int r = 0; r < D; ++r)
#pragma unroll
    for (int c = 0; c < D; ++c) {
      R s = R(0);
#pragma unroll
      for (int l = 0; l < D; ++l) s = fma(U[l][r], A[l][c], s);
      S[r][c] = s;
    }
  R E[D][D], q[D], p[D];
  if constexpr (D == 2) {
    const R s00 = S[0][0], s11 = S[1][1], s01 = R(0.5) * (S[0][1] + S[1][0]);
    const R mean = R(0.5) * (s00 + s11), dl = R(0.5) * (s00 - s11);
    const R rr = Tr<R>::sqrt_(dl * dl + s01 * s01);
    q[0] = mean + rr;
    q[1] = mean - rr;
    // eigenvector of q0: (cos t, sin t) with (cos 2t, sin 2t) = (dl, s01)/rr
    R c2 = R(1), s2 = R(0);
    if (rr > R(0)) {
      c2 = dl / rr;
      s2 = s01 / rr;
    }
    const R ct = Tr<R>::sqrt_(fmax(R(0), R(0.5) * (R(1) + c2)));
    R st = Tr<R>::sqrt_(fmax(R(0), R(0.5) * (R(1) - c2)));
    st = (s2 < R(0)) ? -st : st;
    E[0][0] = ct; E[1][0] = st; E[0][1] = -st; E[1][1] = ct;
  } else {
    sym3_eig<R>(S[0][0], R(0.5) * (S[0][1] + S[1][0]), R(0.5) * (S[0][2] + S[2][0]), S[1][1],
                R(0.5) * (S[1][2] + S[2][1]), S[2][2], q, E);
  }
  bool floored = false;
  {
    R prod = R(1), sum = R(0);
#pragma unroll
    for (int j = 0; j < D; ++j) {
      p[j] = prox_root<R, EN>(q[j], w, mu);
      prod *= p[j];
      sum += p[j];
    }
    if (prod < R(kSqrtEpsM) || sum < R(kSqrtEpsM)) floored = true;
  }
  R dp[D];
#pragma unroll
  for (int j = 0; j < D; ++j) {
    if (floored && p[j] < R(kSqrtEpsM)) {
      p[j] = R(kSqrtEpsM);
      dp[j] = R(0);
    } else {
      dp[j] = prox_root_deriv<R, EN>(p[j], q[j], w, mu);
    }
  }
  R P[D][D];
#pragma unroll
  for (int r = 0; r < D; ++r)
#pragma unroll
    for (int c = 0; c < D; ++c) {
      R s = R(0);
#pragma unroll
      for (int j = 0; j < D; ++j) s = fma(E[r][j] * p[j], E[c][j], s);
      P[r][c] = s;
    }
  // ---- adjoints of state_k (from the later iterations), plus the W step of k+1:
  // r^{k+1} = mu (U^k P^k - Lambda^k), r_bar = mu G xi^{k+1}
  R* Pb = reinterpret_cast<R*>(a.Pbar);
  R* Lb = reinterpret_cast<R*>(a.Lbar);
  R Pbar[D][D], Lbar[D][D], Ubar[D][D];
#pragma unroll
  for (int r = 0; r < D; ++r)
#pragma unroll
    for (int c = 0; c < D; ++c) {
      Pbar[r][c] = Pb[(int64_t)(r * D + c) * m + i];
      Lbar[r][c] = Lb[(int64_t)(r * D + c) * m + i];
      Ubar[r][c] = R(0);
    }
  if (a.xi) {
    const R* xi = reinterpret_cast<const R*>(a.xi);
    R rb[D][D];
#pragma unroll
    for (int r = 0; r < D; ++r)
#pragma unroll
      for (int c = 0; c < D; ++c) rb[r][c] = R(0);
#pragma unroll
    for (int j = 0; j < D; ++j)
#pragma unroll
      for (int c = 0; c < D; ++c) {
        const R del = xi[(int64_t)vid[j + 1] * D + c] - xi[(int64_t)vid[0] * D + c];
#pragma unroll
        for (int r = 0; r < D; ++r) rb[r][c] = fma(g[j][r], del, rb[r][c]);
      }
#pragma unroll
    for (int r = 0; r < D; ++r)
#pragma unroll
      for (int c = 0; c < D; ++c) {
        rb[r][c] *= mu;
        Lbar[r][c] -= rb[r][c];
      }
#pragma unroll
    for (int r = 0; r < D; ++r)
#pragma unroll
      for (int c = 0; c < D; ++c) {
        R su = R(0), sp = R(0);
#pragma unroll
        for (int l = 0; l < D; ++l) {
          su = fma(rb[r][l], P[c][l], su);   // (r_bar P^T)[r][c]
          sp = fma(U[l][r], rb[l][c], sp);   // (U^T r_bar)[r][c]
        }
        Ubar[r][c] += su;
        Pbar[r][c] += sp;
      }
  }
  // ---- Lambda^k = Lambda^{k-1} + J - U P
  R Jbar[D][D], L0bar[D][D];
#pragma unroll
  for (int r = 0; r < D; ++r)
#pragma unroll
    for (int c = 0; c < D; ++c) {
      Jbar[r][c] = Lbar[r][c];
      L0bar[r][c] = Lbar[r][c];
    }
#pragma unroll
  for (int r = 0; r < D; ++r)
#pragma unroll
    for (int c = 0; c < D; ++c) {
      R su = R(0), sp = R(0);
#pragma unroll
      for (int l = 0; l < D; ++l) {
        su = fma(Lbar[r][l], P[c][l], su);
        sp = fma(U[l][r], Lbar[l][c], sp);
      }
      Ubar[r][c] -= su;
      Pbar[r][c] -= sp;
    }
  // ---- P = E diag(p(q)) E^T: S_bar = E (Gamma o (E^T sym(P_bar) E)) E^T
  R Sbar[D][D];
  {
    R Ps[D][D], Mb[D][D];
#pragma unroll
    for (int r = 0; r < D; ++r)
#pragma unroll
      for (int c = 0; c < D; ++c) Ps[r][c] = R(0.5) * (Pbar[r][c] + Pbar[c][r]);
#pragma unroll
    for (int r = 0; r < D; ++r)
#pragma unroll
      for (int c = 0; c < D; ++c) {
        R s = R(0);
#pragma unroll
        for (int l = 0; l < D; ++l)
#pragma unroll
          for (int n = 0; n < D; ++n) s = fma(E[l][r] * Ps[l][n], E[n][c], s);
        Mb[r][c] = s;
      }
#pragma unroll
    for (int r = 0; r < D; ++r)
#pragma unroll
      for (int c = 0; c < D; ++c) {
        R gam;
        if (r == c) {
          gam = dp[r];
        } else {
          // divided difference of the root; for close eigenvalues the trapezoid
          // average of p' (error O(dq^2)) replaces it.  The switch at
          // dq ~ eps^(1/3) balances the quotient's rounding error (eps / dq)
          // against the trapezoid error (dq^2).
          const R dq = q[r] - q[c];
          const R scale = fmax(Tr<R>::abs_(q[r]), Tr<R>::abs_(q[c])) + R(1);
          const R thr = (sizeof(R) == 4 ? R(4.9e-3) : R(6.1e-6)) * scale;   // eps^(1/3)
          gam = (Tr<R>::abs_(dq) > thr) ? (p[r] - p[c]) / dq : R(0.5) * (dp[r] + dp[c]);
        }
        Mb[r][c] *= gam;
      }
#pragma unroll
    for (int r = 0; r < D; ++r)
#pragma unroll
      for (int c = 0; c < D; ++c) {
        R s = R(0);
#pragma unroll
        for (int l = 0; l < D; ++l)
#pragma unroll
          for (int n = 0; n < D; ++n) s = fma(E[r][l] * Mb[l][n], E[c][n], s);
        Sbar[r][c] = s;
      }
  }
  // ---- S = symm(U^T A): U_bar += A S_bar, A_bar = U S_bar
  R Abar[D][D];
#pragma unroll
  for (int r = 0; r < D; ++r)
#pragma unroll
    for (int c = 0; c < D; ++c) {
      R su = R(0), sa = R(0);
#pragma unroll
      for (int l = 0; l < D; ++l) {
        su = fma(A[r][l], Sbar[l][c], su);
        sa = fma(U[r][l], Sbar[l][c], sa);
      }
      Ubar[r][c] += su;
      Abar[r][c] = sa;
    }
  // ---- U = polar(Q): Q_bar = U V N V^T, N_ij = (M_ij - M_ji)/(s_i + s_j), M = V^T U^T U_bar V
  R Qbar[D][D];
  if (tie) {
#pragma unroll
    for (int r = 0; r < D; ++r)
#pragma unroll
      for (int c = 0; c < D; ++c) Qbar[r][c] = R(0);
  } else {
    R T1[D][D], Mq[D][D], N[D][D];
#pragma unroll
    for (int r = 0; r < D; ++r)
#pragma unroll
      for (int c = 0; c < D; ++c) {
        R s = R(0);
#pragma unroll
        for (int l = 0; l < D; ++l) s = fma(U[l][r], Ubar[l][c], s);
        T1[r][c] = s;                       // U^T U_bar
      }
#pragma unroll
    for (int r = 0; r < D; ++r)
#pragma unroll
      for (int c = 0; c < D; ++c) {
        R s = R(0);
#pragma unroll
        for (int l = 0; l < D; ++l)
#pragma unroll
          for (int n = 0; n < D; ++n) s = fma(Vq[l][r] * T1[l][n], Vq[n][c], s);
        Mq[r][c] = s;
      }
    const R smax = fmax(Tr<R>::abs_(sg[0]), Tr<R>::abs_(sg[D - 1])) + Tr<R>::tiny();
#pragma unroll
    for (int r = 0; r < D; ++r)
#pragma unroll
      for (int c = 0; c < D; ++c) {
        if (r == c) {
          N[r][c] = R(0);
        } else {
          R den = sg[r] + sg[c];
          const R floor_ = R(1e-6) * smax;
          if (Tr<R>::abs_(den) < floor_) den = (den < R(0)) ? -floor_ : floor_;
          N[r][c] = (Mq[r][c] - Mq[c][r]) / den;
        }
      }
    R T2[D][D];
#pragma unroll
    for (int r = 0; r < D; ++r)
#pragma unroll
      for (int c = 0; c < D; ++c) {
        R s = R(0);
#pragma unroll
        for (int l = 0; l < D; ++l)
#pragma unroll
          for (int n = 0; n < D; ++n) s = fma(Vq[r][l] * N[l][n], Vq[c][n], s);
        T2[r][c] = s;                       // V N V^T
      }
#pragma unroll
    for (int r = 0; r < D; ++r)
#pragma unroll
      for (int c = 0; c < D; ++c) {
        R s = R(0);
#pragma unroll
        for (int l = 0; l < D; ++l) s = fma(U[r][l], T2[l][c], s);
        Qbar[r][c] = s;
      }
  }
  // ---- Q = A P^{k-1}: A_bar += Q_bar P^{k-1}; P_bar^{k-1} = A^T Q_bar
  R P0bar[D][D];
#pragma unroll
  for (int r = 0; r < D; ++r)
#pragma unroll
    for (int c = 0; c < D; ++c) {
      R sa = R(0), sp = R(0);
#pragma unroll
      for (int l = 0; l < D; ++l) {
        sa = fma(Qbar[r][l], P0[l][c], sa);
        sp = fma(A[l][r], Qbar[l][c], sp);
      }
      Abar[r][c] += sa;
      P0bar[r][c] = sp;
    }
  // ---- A = J + Lambda^{k-1}
#pragma unroll
  for (int r = 0; r < D; ++r)
#pragma unroll
    for (int c = 0; c < D; ++c) {
      Jbar[r][c] += Abar[r][c];
      L0bar[r][c] += Abar[r][c];
      Pb[(int64_t)(r * D + c) * m + i] = P0bar[r][c];
      Lb[(int64_t)(r * D + c) * m + i] = L0bar[r][c];
    }
  // ---- J = G W^k: per-vertex terms g_j . J_bar[:, c]
  R cj[D + 1][D];
#pragma unroll
  for (int c = 0; c < D; ++c) cj[0][c] = R(0);
#pragma unroll
  for (int j = 0; j < D; ++j)
#pragma unroll
    for (int c = 0; c < D; ++c) {
      R s = R(0);
#pragma unroll
      for (int r = 0; r < D; ++r) s = fma(g[j][r], Jbar[r][c], s);
      cj[j + 1][c] = s;
      cj[0][c] -= s;
    }
  R* out = reinterpret_cast<R*>(a.contribJ) + (int64_t)i * (D + 1) * D;
#pragma unroll
  for (int j = 0; j <= D; ++j)
#pragma unroll
    for (int c = 0; c < D; ++c) out[j * D + c] = cj[j][c];
}

// xi in original vertex order with zeros at the pinned vertices (Real)
template <typename R>
__global__ void k_xi_to_vertices(int n, int d, const int32_t* __restrict__ v2e, const double* __restrict__ xi_e,
                                 R* __restrict__ xi_v) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * d) return;
  const int v = t / d, c = t - v * d;
  const int e = v2e[v];
  xi_v[t] = (e >= 0) ? (R)xi_e[(int64_t)e * d + c] : R(0);
}

// b_adj (eliminated order) = W_bar at the free vertices; b_bar += W_bar at pins
__global__ void k_adj_rhs(int nF, int n_pin, int d, const int32_t* __restrict__ row_vertex,
                          const int32_t* __restrict__ pins, const double* __restrict__ Wbar,
                          double* __restrict__ b_adj, double* __restrict__ bbar) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < nF * d) {
    const int i = t / d, c = t - i * d;
    b_adj[t] = Wbar[(int64_t)row_vertex[i] * d + c];
  }
  if (t < n_pin * d) {
    const int p = t / d, c = t - p * d;
    bbar[t] += Wbar[(int64_t)pins[p] * d + c];
  }
}

// b_bar -= L_CF xi (the pins' share of the W step's constant term -L_FC b)
__global__ void k_adj_pins(int n_pin, int d, const int64_t* __restrict__ ptr, const int32_t* __restrict__ row,
                           const double* __restrict__ val, const double* __restrict__ xi, double* __restrict__ bbar) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n_pin * d) return;
  const int p = t / d, c = t - p * d;
  double s = 0.0;
  for (int64_t q = ptr[p]; q < ptr[p + 1]; ++q) s += val[q] * xi[(int64_t)row[q] * d + c];
  bbar[t] -= s;
}

}  // namespace

void launch_adjoint_local(const AdjointLaunch& a, cudaStream_t s) {
  if (a.energy == kEnMixed) return;  // mixed-energy (batched) contexts have no adjoint
  const int grid = (a.m + 127) / 128;
#define FFA_ADJ(D, R, EN) k_adjoint_local<D, R, EN><<<grid, 128, 0, s>>>(a)
  if (a.d == 2) {
    if (a.fp64) {
      if (a.energy == kEnSD) FFA_ADJ(2, double, kEnSD); else if (a.energy == kEnSG) FFA_ADJ(2, double, kEnSG);
      else FFA_ADJ(2, double, kEnSA);
    } else {
      if (a.energy == kEnSD) FFA_ADJ(2, float, kEnSD); else if (a.energy == kEnSG) FFA_ADJ(2, float, kEnSG);
      else FFA_ADJ(2, float, kEnSA);
    }
  } else {
    if (a.fp64) {
      if (a.energy == kEnSD) FFA_ADJ(3, double, kEnSD); else if (a.energy == kEnSG) FFA_ADJ(3, double, kEnSG);
      else FFA_ADJ(3, double, kEnSA);
    } else {
      if (a.energy == kEnSD) FFA_ADJ(3, float, kEnSD); else if (a.energy == kEnSG) FFA_ADJ(3, float, kEnSG);
      else FFA_ADJ(3, float, kEnSA);
    }
  }
#undef FFA_ADJ
}

void launch_xi_to_vertices(int n, int d, int fp64, const int32_t* v2e, const double* xi_e, void* xi_v,
                           cudaStream_t s) {
  const int grid = (n * d + 255) / 256;
  if (fp64) k_xi_to_vertices<double><<<grid, 256, 0, s>>>(n, d, v2e, xi_e, reinterpret_cast<double*>(xi_v));
  else k_xi_to_vertices<float><<<grid, 256, 0, s>>>(n, d, v2e, xi_e, reinterpret_cast<float*>(xi_v));
}

void launch_adj_rhs(int nF, int n_pin, int d, const int32_t* row_vertex, const int32_t* pins, const double* Wbar,
                    double* b_adj, double* bbar, cudaStream_t s) {
  const int nt = (nF > n_pin ? nF : n_pin) * d;
  k_adj_rhs<<<(nt + 255) / 256, 256, 0, s>>>(nF, n_pin, d, row_vertex, pins, Wbar, b_adj, bbar);
}

void launch_adj_pins(int n_pin, int d, const int64_t* ptr, const int32_t* row, const double* val, const double* xi,
                     double* bbar, cudaStream_t s) {
  k_adj_pins<<<(n_pin * d + 255) / 256, 256, 0, s>>>(n_pin, d, ptr, row, val, xi, bbar);
}

}  // namespace ffa
