// Per-element kernels: the fused local step (Jacobian assembly, U step, P step,
// multiplier update, right-hand-side terms and the error terms of
// eq. primaldualerror; paper Sec. 4), the polar initialization (Sec. 6,
// eqs. initialpolardecomposition/polardecompositionapplied) and the energy terms
// (eq. genericdeformationenergy with the defining functions of Sec. 7 and App. A).
// One thread per element; all per-element math stays in registers; element data
// are structure-of-arrays (coalesced).
#include "ffa_internal.h"
#include "ffa_math.cuh"

namespace ffa {
namespace {

// ---------------------------------------------------------------------------
// vertex records (written by the vertex-update kernel)
//   float, d=3: 3 float4 = (hi.xyz, dW.x) (lo.xyz, dW.y) (dW.z, -, -, -)
//   float, d=2: 2 float4 = (hi.xy, lo.xy) (dW.xy, -, -)
//   double, d=3: 3 double2 = (W.xy) (W.z, dW.x) (dW.yz)
//   double, d=2: 2 double2 = (W.xy) (dW.xy)
// hi + lo is W split into two floats, so differences of nearby vertices keep
// their relative accuracy in float arithmetic.
// ---------------------------------------------------------------------------
template <int D, typename R>
__device__ __forceinline__ void load_vertex(const void* rec, int v, R hi[D], R lo[D], R dw[D]) {
  if constexpr (sizeof(R) == 4) {
    const float4* r = reinterpret_cast<const float4*>(rec) + (int64_t)v * D;
    if constexpr (D == 3) {
      const float4 a = __ldg(r), b = __ldg(r + 1), c = __ldg(r + 2);
      hi[0] = a.x; hi[1] = a.y; hi[2] = a.z;
      lo[0] = b.x; lo[1] = b.y; lo[2] = b.z;
      dw[0] = a.w; dw[1] = b.w; dw[2] = c.x;
    } else {
      const float4 a = __ldg(r), b = __ldg(r + 1);
      hi[0] = a.x; hi[1] = a.y; lo[0] = a.z; lo[1] = a.w;
      dw[0] = b.x; dw[1] = b.y;
    }
  } else {
    const double2* r = reinterpret_cast<const double2*>(rec) + (int64_t)v * D;
    if constexpr (D == 3) {
      const double2 a = __ldg(r), b = __ldg(r + 1), c = __ldg(r + 2);
      hi[0] = a.x; hi[1] = a.y; hi[2] = b.x;
      dw[0] = b.y; dw[1] = c.x; dw[2] = c.y;
    } else {
      const double2 a = __ldg(r), b = __ldg(r + 1);
      hi[0] = a.x; hi[1] = a.y; dw[0] = b.x; dw[1] = b.y;
    }
#pragma unroll
    for (int k = 0; k < D; ++k) lo[k] = R(0);
  }
}

// J = G W and dJ = G (W - W_prev) of element i (Supplemental: column k of J is
// the gradient of target coordinate k), from the hat gradients of vertices 1..d.
template <int D, typename R>
__device__ __forceinline__ void element_jacobians(const int vid[D + 1], const R g[D][D], const void* vrec,
                                                  R J[D][D], R dJ[D][D]) {
  R h0[D], l0[D], d0[D];
  load_vertex<D, R>(vrec, vid[0], h0, l0, d0);
#pragma unroll
  for (int a = 0; a < D; ++a)
#pragma unroll
    for (int k = 0; k < D; ++k) { J[a][k] = R(0); dJ[a][k] = R(0); }
#pragma unroll
  for (int j = 0; j < D; ++j) {
    R hj[D], lj[D], dj[D];
    load_vertex<D, R>(vrec, vid[j + 1], hj, lj, dj);
#pragma unroll
    for (int k = 0; k < D; ++k) {
      const R del = (hj[k] - h0[k]) + (lj[k] - l0[k]);
      const R ddel = dj[k] - d0[k];
#pragma unroll
      for (int a = 0; a < D; ++a) {
        J[a][k] = fma(g[j][a], del, J[a][k]);
        dJ[a][k] = fma(g[j][a], ddel, dJ[a][k]);
      }
    }
  }
}

template <int D, typename R>
__device__ __forceinline__ void load_element(const ElemBufs& e, int m, int i, int vid[D + 1], R g[D][D],
                                             R& w, R& mu) {
  const R* gp = reinterpret_cast<const R*>(e.g);
#pragma unroll
  for (int j = 0; j <= D; ++j) vid[j] = __ldg(e.idx + (int64_t)j * m + i);
#pragma unroll
  for (int j = 0; j < D; ++j)
#pragma unroll
    for (int a = 0; a < D; ++a) g[j][a] = __ldg(gp + (int64_t)(j * D + a) * m + i);
  w = __ldg(reinterpret_cast<const R*>(e.w) + i);
  mu = __ldg(reinterpret_cast<const R*>(e.mu) + i);
}

// contributions g_j . X[:, k] for the d+1 element vertices (j = 0 is minus the sum)
template <int D, typename R>
__device__ __forceinline__ void store_terms(void* dst, int i, const R g[D][D], const R X[D][D]) {
  R c[D + 1][D];
#pragma unroll
  for (int k = 0; k < D; ++k) c[0][k] = R(0);
#pragma unroll
  for (int j = 0; j < D; ++j)
#pragma unroll
    for (int k = 0; k < D; ++k) {
      R s = R(0);
#pragma unroll
      for (int a = 0; a < D; ++a) s = fma(g[j][a], X[a][k], s);
      c[j + 1][k] = s;
      c[0][k] -= s;
    }
  R* out = reinterpret_cast<R*>(dst) + (int64_t)i * (D + 1) * D;
  constexpr int kBytes = (D + 1) * D * (int)sizeof(R);
  if constexpr (kBytes % 16 == 0) {
    // 16-byte stores: the element's terms start on a 16-byte boundary
    const R* f = &c[0][0];
#pragma unroll
    for (int q = 0; q < kBytes / 16; ++q) {
      if constexpr (sizeof(R) == 4)
        reinterpret_cast<float4*>(out)[q] = make_float4(f[4 * q], f[4 * q + 1], f[4 * q + 2], f[4 * q + 3]);
      else
        reinterpret_cast<double2*>(out)[q] = make_double2(f[2 * q], f[2 * q + 1]);
    }
  } else {
#pragma unroll
    for (int j = 0; j <= D; ++j)
#pragma unroll
      for (int k = 0; k < D; ++k) out[j * D + k] = c[j][k];
  }
}

// ---------------------------------------------------------------------------
// block reduction of NQ per-thread values into one double partial per block
// ---------------------------------------------------------------------------
template <typename R, int N>
__device__ __forceinline__ void block_reduce(R v[N], double* out) {
  __shared__ double red[8][N];   // up to 256 threads
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < N; ++q) {
    double tot;
    if constexpr (sizeof(R) == 4) {
      FF a{v[q], 0.0f};
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        FF b{__shfl_xor_sync(0xffffffffu, a.hi, o), __shfl_xor_sync(0xffffffffu, a.lo, o)};
        a = ff_add(a, b);
      }
      tot = (double)a.hi + (double)a.lo;
    } else {
      double a = v[q];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
      tot = a;
    }
    if (lane == 0) red[warp][q] = tot;
  }
  __syncthreads();
  if (threadIdx.x < N) {
    double s = 0.0;
#pragma unroll
    for (int wv = 0; wv < (int)(blockDim.x >> 5); ++wv) s += red[wv][threadIdx.x];
    out[(int64_t)blockIdx.x * N + threadIdx.x] = s;
  }
}

template <typename R>
__device__ __forceinline__ bool finite_(R x) { return isfinite(x); }

// Block sum of N per-thread values in a fixed order (warp shuffles, then the
// warps in index order; float values in double-float): the result in thread 0.
// Ends with a barrier, so it can be called again in a block-uniform loop.
template <typename R, int N>
__device__ __forceinline__ void block_sum_to0(const R v[N], double tot[N]) {
  __shared__ double red[8][N];   // up to 256 threads
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < N; ++q) {
    double t;
    if constexpr (sizeof(R) == 4) {
      FF a{v[q], 0.0f};
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        FF b{__shfl_xor_sync(0xffffffffu, a.hi, o), __shfl_xor_sync(0xffffffffu, a.lo, o)};
        a = ff_add(a, b);
      }
      t = (double)a.hi + (double)a.lo;
    } else {
      double a = v[q];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
      t = a;
    }
    if (lane == 0) red[warp][q] = t;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int q = 0; q < N; ++q) {
      double s = 0.0;
      for (int wv = 0; wv < (int)(blockDim.x >> 5); ++wv) s += red[wv][q];
      tot[q] = s;
    }
  }
  __syncthreads();
}

// batched meshes: per-mesh sums of the check quantities, deterministic.  The
// elements are sorted by mesh, so a block holds a run of meshes: each is summed
// over the block in a fixed order; a mesh wholly inside the block is written to
// mesh_acc (this block is its only contributor), the block's first and last
// meshes go to mesh_part, which launch_mesh_partials adds up in block order.
template <typename R>
__device__ __forceinline__ void mesh_block_sums(const R v[NQ], const ElemBufs& e, int m, int i) {
  const int64_t i0 = (int64_t)blockIdx.x * blockDim.x;
  const int64_t i1 = min((int64_t)m, i0 + blockDim.x);
  const int first = e.mesh_of[i0], last = e.mesh_of[i1 - 1];
  const int mine = (i < m) ? e.mesh_of[i] : -1;
  for (int k = first; k <= last; ++k) {   // block-uniform
    R w[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) w[q] = (mine == k) ? v[q] : R(0);
    double tot[NQ];
    block_sum_to0<R, NQ>(w, tot);
    if (threadIdx.x == 0) {
      double* dst = (k == first) ? e.mesh_part + ((int64_t)blockIdx.x * 2 + 0) * NQ
                  : (k == last) ? e.mesh_part + ((int64_t)blockIdx.x * 2 + 1) * NQ
                                : e.mesh_acc + (int64_t)k * (NQ + 1);
#pragma unroll
      for (int q = 0; q < NQ; ++q) dst[q] = tot[q];
    }
  }
}

// ---------------------------------------------------------------------------
// the fused local step
// ---------------------------------------------------------------------------
// float: 64 registers (4 blocks of 256 or 8 of 128 per SM).  The per-element math is issue
// bound, and the extra resident warps hide its latencies better than the spilled
// registers cost (measured 0.215 -> 0.167 ms on the 64^3-cell cube).
// local-step variants: the paper's (h = 0), the joint (U, P) prox (not the
// paper's scheme), and the paper's with the proximal U term h_i > 0
constexpr int kVarPaper = 0, kVarJoint = 1, kVarProx = 2;

template <int D, typename R, int EN, bool CHECK, int VAR>
__global__ void __launch_bounds__(256, sizeof(R) == 4 ? 4 : 1) k_local_step(ElemBufs e, int m, const void* __restrict__ vrec,
                                                    double* __restrict__ partials) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  R qv[NQ];
#pragma unroll
  for (int q = 0; q < NQ; ++q) qv[q] = R(0);
  if (i < m) {
    int vid[D + 1];
    R g[D][D], w, mu;
    load_element<D, R>(e, m, i, vid, g, w, mu);
    const int en = (EN == kEnMixed) ? (int)e.energy_of[i] : EN;
    R J[D][D], dJ[D][D];
    element_jacobians<D, R>(vid, g, vrec, J, dJ);
    R* Pp = reinterpret_cast<R*>(e.P);
    R* Lp = reinterpret_cast<R*>(e.Lam);
    R* Up = reinterpret_cast<R*>(e.U);
    R A[D][D], Lam[D][D], P[D][D];
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
      for (int k = 0; k < D; ++k) {
        Lam[a][k] = Lp[(int64_t)(a * D + k) * m + i];
        A[a][k] = J[a][k] + Lam[a][k];
      }
    if constexpr (D == 2) {
      P[0][0] = Pp[i]; P[0][1] = P[1][0] = Pp[(int64_t)m + i]; P[1][1] = Pp[2 * (int64_t)m + i];
    } else {
      P[0][0] = Pp[i]; P[0][1] = P[1][0] = Pp[(int64_t)m + i]; P[0][2] = P[2][0] = Pp[2 * (int64_t)m + i];
      P[1][1] = Pp[3 * (int64_t)m + i]; P[1][2] = P[2][1] = Pp[4 * (int64_t)m + i]; P[2][2] = Pp[5 * (int64_t)m + i];
    }
    // ---- U step: nearest rotation to Q = (J + Lambda) P + (h / mu) U^{k-1}
    // (eqs. rawoptimizationinudecoupled/optimizationinudecoupled; h = 0 unless VAR is kVarProx);
    // the joint (U, P) prox variant (not the paper's scheme) takes Q = J + Lambda:
    // for a rotation-invariant f the joint minimizer of w f(P) + mu/2 |U P - A|^2 is
    // the rotation nearest to A with P the prox of symm(U^T A)
    R Q[D][D], U[D][D];
    if constexpr (VAR == kVarJoint) {
#pragma unroll
      for (int a = 0; a < D; ++a)
#pragma unroll
        for (int k = 0; k < D; ++k) Q[a][k] = A[a][k];
    } else {
#pragma unroll
      for (int a = 0; a < D; ++a)
#pragma unroll
        for (int k = 0; k < D; ++k) {
          R s = R(0);
#pragma unroll
          for (int l = 0; l < D; ++l) s = fma(A[a][l], P[l][k], s);
          Q[a][k] = s;
        }
      if constexpr (VAR == kVarProx) {
        // + (h_i / mu_i) U^{k-1}, the stored rotation of the previous iteration
        const R hm = reinterpret_cast<const R*>(e.hmu)[i];
        R Uo[D][D];
        if constexpr (D == 2) {
          const R c = Up[i], sn = Up[(int64_t)m + i];
          Uo[0][0] = c; Uo[0][1] = -sn; Uo[1][0] = sn; Uo[1][1] = c;
        } else {
          R qt[4];
#pragma unroll
          for (int k = 0; k < 4; ++k) qt[k] = Up[(int64_t)k * m + i];
          quat_to_rot<R>(qt, Uo);
        }
#pragma unroll
        for (int a = 0; a < D; ++a)
#pragma unroll
          for (int k = 0; k < D; ++k) Q[a][k] = fma(hm, Uo[a][k], Q[a][k]);
      }
    }
    if constexpr (D == 2) {
      // maximize U(phi) . Q: (cos, sin) along (q00 + q11, q10 - q01); tie keeps U^{k-1}
      const R ca = Q[0][0] + Q[1][1], sa = Q[1][0] - Q[0][1];
      const R r2 = ca * ca + sa * sa;
      R c, s;
      if (r2 > R(0)) {
        const R ir = Tr<R>::rsqrt_(r2);
        c = ca * ir;
        s = sa * ir;
      } else {
        c = Up[i];
        s = Up[(int64_t)m + i];
      }
      U[0][0] = c; U[0][1] = -s; U[1][0] = s; U[1][1] = c;
      Up[i] = c;
      Up[(int64_t)m + i] = s;
    } else {
      R cond, qt[4];
      // the quaternion of the nearest rotation in closed form (the top eigenvector
      // of Horn's 4x4 matrix) when the product of the eigenvalue gaps is large
      // enough relative to |Q|^3 for the precision (float 0.8: s_mid +
      // s_min,signed above about 0.1 s_max; double 0.1), which is where the
      // closed-form eigenvector is accurate; otherwise one-sided Jacobi.
      nearest_rotation3_quat<R>(Q, qt, cond);
      if (cond >= Tr<R>::rotation_gate()) {
        quat_to_rot<R>(qt, U);
      } else if constexpr (sizeof(R) == 4) {
        // float: when even the Jacobi rotation is ill-determined (s_mid +
        // s_min,signed below 1e-5 s_max) Q itself carries float rounding, so double
        // cannot add accuracy there; those (near-)degenerate cases are redone in
        // double, so that the orthonormal frame is built from well-separated columns.
        nearest_rotation3<R>(Q, U, cond);
        if (cond < R(1e-5)) {
          double Qd[3][3], Ud[3][3], cd;
#pragma unroll
          for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int k = 0; k < 3; ++k) Qd[a][k] = (double)Q[a][k];
          nearest_rotation3<double>(Qd, Ud, cd);
#pragma unroll
          for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int k = 0; k < 3; ++k) U[a][k] = (R)Ud[a][k];
        }
        rot_to_quat<R>(U, qt);
      } else {
        nearest_rotation3<R>(Q, U, cond);
        rot_to_quat<R>(U, qt);
      }
#pragma unroll
      for (int k = 0; k < 4; ++k) Up[(int64_t)k * m + i] = qt[k];
    }
    // ---- P step: S = symm(U^T (J + Lambda)), per-eigenvalue prox root (eqs. optimizinginp/rootfindinginp)
    R S[D][D];
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
      for (int k = 0; k < D; ++k) {
        R s = R(0);
#pragma unroll
        for (int l = 0; l < D; ++l) s = fma(U[l][a], A[l][k], s);
        S[a][k] = s;
      }
    R p[D];
    if constexpr (D == 2) {
      const R s00 = S[0][0], s11 = S[1][1], s01 = R(0.5) * (S[0][1] + S[1][0]);
      const R mean = R(0.5) * (s00 + s11), dl = R(0.5) * (s00 - s11);
      const R rr = Tr<R>::sqrt_(dl * dl + s01 * s01);
      p[0] = prox_root_en<R, EN>(mean + rr, w, mu, en);
      p[1] = prox_root_en<R, EN>(mean - rr, w, mu, en);
      if (p[0] * p[1] < R(kSqrtEpsM) || p[0] + p[1] < R(kSqrtEpsM)) {
        p[0] = fmax(p[0], R(kSqrtEpsM));
        p[1] = fmax(p[1], R(kSqrtEpsM));
      }
      const R pm = R(0.5) * (p[0] + p[1]);
      const R dd = (rr > R(0)) ? (p[0] - p[1]) / (R(2) * rr) : R(0);
      P[0][0] = pm + dd * dl;
      P[1][1] = pm - dd * dl;
      P[0][1] = P[1][0] = dd * s01;
    } else {
      // the prox of the spectral function: P = f(S) with f the per-eigenvalue prox
      // map.  In float it is formed without eigenvectors: S's eigenvalues in closed
      // form (l1 >= l2 >= l3), the roots p_j = f(l_j), and the Newton form
      // P = p1 I + f[l1,l2] (S - l1 I) + f[l1,l2,l3] (S - l1 I)(S - l2 I) with the
      // first divided differences 1 / h[p_j, p_k] (cancellation-free, also for
      // equal eigenvalues).  Near a cluster the eigenvalues lose accuracy but the
      // interpolant evaluated at S does not: S - l1 I is then small.
      bool done = false;
      {
        R lam[3];
        sym3_eigvals<R>(S[0][0], R(0.5) * (S[0][1] + S[1][0]), R(0.5) * (S[0][2] + S[2][0]), S[1][1],
                        R(0.5) * (S[1][2] + S[2][1]), S[2][2], lam);
#pragma unroll
        for (int j = 0; j < 3; ++j) p[j] = prox_root_en<R, EN>(lam[j], w, mu, en);
        if (!(p[0] * p[1] * p[2] < R(kSqrtEpsM) || p[0] + p[1] + p[2] < R(kSqrtEpsM))) {
          const R d12 = R(1) / prox_inverse_dd<R, EN>(p[0], p[1], w, mu, en);
          const R d23 = R(1) / prox_inverse_dd<R, EN>(p[1], p[2], w, mu, en);
          const R g13 = lam[0] - lam[2];
          const R d123 = (g13 > R(0)) ? (d12 - d23) / g13 : R(0);
          R A1[3][3], A2[3][3];
#pragma unroll
          for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int k = 0; k < 3; ++k) {
              const R sym = R(0.5) * (S[a][k] + S[k][a]);
              A1[a][k] = sym - (a == k ? lam[0] : R(0));
              A2[a][k] = sym - (a == k ? lam[1] : R(0));
            }
#pragma unroll
          for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int k = a; k < 3; ++k) {
              const R quad = A1[a][0] * A2[0][k] + A1[a][1] * A2[1][k] + A1[a][2] * A2[2][k];
              const R v = (a == k ? p[0] : R(0)) + d12 * A1[a][k] + d123 * quad;
              P[a][k] = v;
              P[k][a] = v;
            }
          done = true;
        }
      }
      if (!done) {
        R ev[3], E[3][3];
        sym3_eig<R>(S[0][0], R(0.5) * (S[0][1] + S[1][0]), R(0.5) * (S[0][2] + S[2][0]), S[1][1],
                    R(0.5) * (S[1][2] + S[2][1]), S[2][2], ev, E);
#pragma unroll
        for (int j = 0; j < 3; ++j) p[j] = prox_root_en<R, EN>(ev[j], w, mu, en);
        if (p[0] * p[1] * p[2] < R(kSqrtEpsM) || p[0] + p[1] + p[2] < R(kSqrtEpsM)) {
#pragma unroll
          for (int j = 0; j < 3; ++j) p[j] = fmax(p[j], R(kSqrtEpsM));
        }
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
          for (int k = a; k < 3; ++k) {
            const R v = E[a][0] * p[0] * E[k][0] + E[a][1] * p[1] * E[k][1] + E[a][2] * p[2] * E[k][2];
            P[a][k] = v;
            P[k][a] = v;
          }
      }
    }
    // ---- multiplier update (eq. lambdaupdate) and the next right-hand-side terms (eq. solvinginw)
    // Lambda^k = (Lambda^{k-1} + J) - U P = A - U P: only A stays live through the
    // U and P steps (J and Lambda^{k-1} are kept for the check iterations alone)
    R UP[D][D], Rhs[D][D];
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
      for (int k = 0; k < D; ++k) {
        R s = R(0);
#pragma unroll
        for (int l = 0; l < D; ++l) s = fma(U[a][l], P[l][k], s);
        UP[a][k] = s;
        Lam[a][k] = A[a][k] - s;
        Rhs[a][k] = mu * (s - Lam[a][k]);
      }
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
      for (int k = 0; k < D; ++k) Lp[(int64_t)(a * D + k) * m + i] = Lam[a][k];
    if constexpr (D == 2) {
      Pp[i] = P[0][0]; Pp[(int64_t)m + i] = P[0][1]; Pp[2 * (int64_t)m + i] = P[1][1];
    } else {
      Pp[i] = P[0][0]; Pp[(int64_t)m + i] = P[0][1]; Pp[2 * (int64_t)m + i] = P[0][2];
      Pp[3 * (int64_t)m + i] = P[1][1]; Pp[4 * (int64_t)m + i] = P[1][2]; Pp[5 * (int64_t)m + i] = P[2][2];
    }
    // the hat gradients again (an L1 hit) rather than kept live through the steps
    R g2[D][D];
    {
      const R* gp = reinterpret_cast<const R*>(e.g);
#pragma unroll
      for (int j = 0; j < D; ++j)
#pragma unroll
        for (int a = 0; a < D; ++a) g2[j][a] = __ldg(gp + (int64_t)(j * D + a) * m + i);
    }
    store_terms<D, R>(e.contrib, i, g2, Rhs);
    if constexpr (CHECK) {
      store_terms<D, R>(e.contrib2, i, g2, Lam);
      R ep = 0, ed = 0, gw = 0, pp = 0;
#pragma unroll
      for (int a = 0; a < D; ++a)
#pragma unroll
        for (int k = 0; k < D; ++k) {
          const R rm = J[a][k] - UP[a][k];
          ep = fma(rm, rm, ep);
          ed = fma(dJ[a][k], dJ[a][k], ed);
          gw = fma(J[a][k], J[a][k], gw);
          pp = fma(P[a][k], P[a][k], pp);
        }
      R det;
      if constexpr (D == 2) det = J[0][0] * J[1][1] - J[0][1] * J[1][0];
      else
        det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) - J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
              J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
      qv[Q_EPRIM] = ep;
      qv[Q_EDUAL] = mu * mu * ed;
      qv[Q_GW] = gw;
      qv[Q_P] = pp;
      qv[Q_ENERGY] = w * f_of_eigs_en<R, EN, D>(p, en);
      qv[Q_FLIPS] = (det <= R(0)) ? R(1) : R(0);
      qv[Q_NONFINITE] = (finite_(ep) && finite_(pp) && finite_(gw)) ? R(0) : R(1);
    }
  }
  if constexpr (CHECK) {
    if (e.mesh_of) mesh_block_sums<R>(qv, e, m, i);
    else block_reduce<R, NQ>(qv, partials);
  }
}

// ---------------------------------------------------------------------------
// polar initialization (eqs. initialpolardecomposition/polardecompositionapplied): U0, P0 from the SVD of G W0, Lambda0 = 0
// ---------------------------------------------------------------------------
template <int D, typename R, int EN>
__global__ void __launch_bounds__(kLocalBlock) k_init_polar(ElemBufs e, int m, const void* __restrict__ vrec) {
  const int i = blockIdx.x * kLocalBlock + threadIdx.x;
  if (i >= m) return;
  int vid[D + 1];
  R g[D][D], w, mu;
  load_element<D, R>(e, m, i, vid, g, w, mu);
  R J[D][D], dJ[D][D];
  element_jacobians<D, R>(vid, g, vrec, J, dJ);
  const int en = (EN == kEnMixed) ? (int)e.energy_of[i] : EN;
  // the clamp of eq. polardecompositionapplied: SG's, or SD's for SD and SA (both grow like p^-2 at 0)
  const R eps = (en == kEnSG) ? R(kEpsInitSG) : R(kEpsInitSD);
  R U[D][D], P[D][D];
  R* Up = reinterpret_cast<R*>(e.U);
  if constexpr (D == 2) {
    const R det = J[0][0] * J[1][1] - J[0][1] * J[1][0];
    R c, s;
    if (det > R(0)) {
      // rotation maximizing tr(U^T J), then P = U^T J, singular values clamped
      const R ca = J[0][0] + J[1][1], sa = J[1][0] - J[0][1];
      const R ir = Tr<R>::rsqrt_(ca * ca + sa * sa);
      c = ca * ir;
      s = sa * ir;
      U[0][0] = c; U[0][1] = -s; U[1][0] = s; U[1][1] = c;
      R S[2][2];
#pragma unroll
      for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int k = 0; k < 2; ++k) S[a][k] = U[0][a] * J[0][k] + U[1][a] * J[1][k];
      const R s01 = R(0.5) * (S[0][1] + S[1][0]);
      const R mean = R(0.5) * (S[0][0] + S[1][1]), dl = R(0.5) * (S[0][0] - S[1][1]);
      const R rr = Tr<R>::sqrt_(dl * dl + s01 * s01);
      const R p0 = fmax(mean + rr, eps), p1 = fmax(mean - rr, eps);
      const R pm = R(0.5) * (p0 + p1), dd = (rr > R(0)) ? (p0 - p1) / (R(2) * rr) : R(0);
      P[0][0] = pm + dd * dl; P[1][1] = pm - dd * dl; P[0][1] = P[1][0] = dd * s01;
    } else {
      // polar factor is the reflection [[c, s], [s, -c]] maximizing tr(O^T J);
      // negating its last column gives the rotation (c, s); P0 = eps I
      const R ca = J[0][0] - J[1][1], sa = J[0][1] + J[1][0];
      const R r2 = ca * ca + sa * sa;
      if (r2 > R(0)) {
        const R ir = Tr<R>::rsqrt_(r2);
        c = ca * ir;
        s = sa * ir;
      } else {
        c = R(1);
        s = R(0);
      }
      U[0][0] = c; U[0][1] = -s; U[1][0] = s; U[1][1] = c;
      P[0][0] = eps; P[1][1] = eps; P[0][1] = P[1][0] = R(0);
    }
    Up[i] = c;
    Up[(int64_t)m + i] = s;
  } else {
    R Us[3][3], sv[3], Vs[3][3];
    svd3_signed<R>(J, Us, sv, Vs);
    const bool flipped = !(sv[2] > R(0));
    if (flipped && sv[2] < R(0)) {
      // polar factor U diag(1,1,-1) V^T, then its last column negated
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          const R o = Us[a][0] * Vs[k][0] + Us[a][1] * Vs[k][1] - Us[a][2] * Vs[k][2];
          U[a][k] = (k == 2) ? -o : o;
        }
    } else {
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int k = 0; k < 3; ++k) U[a][k] = Us[a][0] * Vs[k][0] + Us[a][1] * Vs[k][1] + Us[a][2] * Vs[k][2];
    }
    R sc[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) sc[j] = flipped ? eps : fmax(sv[j], eps);
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int k = 0; k < 3; ++k)
        P[a][k] = Vs[a][0] * sc[0] * Vs[k][0] + Vs[a][1] * sc[1] * Vs[k][1] + Vs[a][2] * sc[2] * Vs[k][2];
    R qt[4];
    rot_to_quat<R>(U, qt);
#pragma unroll
    for (int k = 0; k < 4; ++k) Up[(int64_t)k * m + i] = qt[k];
  }
  R* Pp = reinterpret_cast<R*>(e.P);
  R* Lp = reinterpret_cast<R*>(e.Lam);
  if constexpr (D == 2) {
    Pp[i] = P[0][0]; Pp[(int64_t)m + i] = P[0][1]; Pp[2 * (int64_t)m + i] = P[1][1];
  } else {
    Pp[i] = P[0][0]; Pp[(int64_t)m + i] = P[0][1]; Pp[2 * (int64_t)m + i] = P[0][2];
    Pp[3 * (int64_t)m + i] = P[1][1]; Pp[4 * (int64_t)m + i] = P[1][2]; Pp[5 * (int64_t)m + i] = P[2][2];
  }
  R Rhs[D][D];
#pragma unroll
  for (int a = 0; a < D; ++a)
#pragma unroll
    for (int k = 0; k < D; ++k) {
      Lp[(int64_t)(a * D + k) * m + i] = R(0);
      R s = R(0);
#pragma unroll
      for (int l = 0; l < D; ++l) s = fma(U[a][l], P[l][k], s);
      Rhs[a][k] = mu * s;
    }
  store_terms<D, R>(e.contrib, i, g, Rhs);
}

// ---------------------------------------------------------------------------
// energy terms at a given W: mode 0 -> partials (w f(J), flips); mode 1 -> the
// per-vertex terms of G^T (w grad f(J)) into contrib2 (eq. symmetricgradientdefininggrad / eq. symmetricdirichletdefininggrad)
// ---------------------------------------------------------------------------
template <int D, typename R, int EN, int MODE>
__global__ void __launch_bounds__(kLocalBlock) k_energy_terms(ElemBufs e, int m, const void* __restrict__ vrec,
                                                              double* __restrict__ partials) {
  const int i = blockIdx.x * kLocalBlock + threadIdx.x;
  R qv[NQ];
#pragma unroll
  for (int q = 0; q < NQ; ++q) qv[q] = R(0);
  if (i < m) {
    int vid[D + 1];
    R g[D][D], w, mu;
    load_element<D, R>(e, m, i, vid, g, w, mu);
    R J[D][D], dJ[D][D];
    element_jacobians<D, R>(vid, g, vrec, J, dJ);
    // inverse by the adjugate
    R Ji[D][D], det;
    if constexpr (D == 2) {
      det = J[0][0] * J[1][1] - J[0][1] * J[1][0];
      Ji[0][0] = J[1][1] / det; Ji[0][1] = -J[0][1] / det; Ji[1][0] = -J[1][0] / det; Ji[1][1] = J[0][0] / det;
    } else {
      const R c00 = J[1][1] * J[2][2] - J[1][2] * J[2][1];
      const R c01 = J[1][2] * J[2][0] - J[1][0] * J[2][2];
      const R c02 = J[1][0] * J[2][1] - J[1][1] * J[2][0];
      det = J[0][0] * c00 + J[0][1] * c01 + J[0][2] * c02;
      const R id = R(1) / det;
      Ji[0][0] = c00 * id; Ji[1][0] = c01 * id; Ji[2][0] = c02 * id;
      Ji[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) * id;
      Ji[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) * id;
      Ji[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) * id;
      Ji[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) * id;
      Ji[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) * id;
      Ji[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) * id;
    }
    const bool flipped = !(det > R(0));
    if constexpr (MODE == 0) {
      R fro = 0, fri = 0;
#pragma unroll
      for (int a = 0; a < D; ++a)
#pragma unroll
        for (int k = 0; k < D; ++k) {
          fro = fma(J[a][k], J[a][k], fro);
          fri = fma(Ji[a][k], Ji[a][k], fri);
        }
      const int en = (EN == kEnMixed) ? (int)e.energy_of[i] : EN;
      R f;
      if (en == kEnSD) {
        f = R(0.5) * (fro + fri);
      } else if (en == kEnSG) {
        f = R(0.5) * fro - Tr<R>::log_(det);
      } else {
        // SA: sum over the singular values s of ((s - 1)^2 + (1/s - 1)^2)/2, the s
        // from the eigenvalues of J^T J
        R s2[D];
        if constexpr (D == 2) {
          const R a = J[0][0] * J[0][0] + J[1][0] * J[1][0], b = J[0][1] * J[0][1] + J[1][1] * J[1][1];
          const R c = J[0][0] * J[0][1] + J[1][0] * J[1][1];
          const R h = R(0.5) * (a + b), dd = R(0.5) * (a - b);
          const R r = Tr<R>::sqrt_(dd * dd + c * c);
          s2[0] = h + r;
          s2[1] = h - r;
        } else {
          R C[3][3], V[3][3];
#pragma unroll
          for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int k = 0; k < 3; ++k) C[a][k] = J[0][a] * J[0][k] + J[1][a] * J[1][k] + J[2][a] * J[2][k];
          sym3_eig<R>(C[0][0], C[0][1], C[0][2], C[1][1], C[1][2], C[2][2], s2, V);
        }
        R sv[D];
#pragma unroll
        for (int k = 0; k < D; ++k) sv[k] = Tr<R>::sqrt_(fmax(s2[k], R(0)));
        f = f_of_eigs<R, kEnSA, D>(sv);
      }
      qv[Q_ENERGY] = flipped ? R(0) : w * f;
      qv[Q_FLIPS] = flipped ? R(1) : R(0);
    } else {
      // grad f_SG = J - J^-T ; grad f_SD = J - J^-T J^-1 J^-T ;
      // grad f_SA = J - R - J^-T J^-1 J^-T + J^-T J^-1 R, R the rotation of J
      // (U diag(phi'(s)) V^T with phi'(s) = s - 1 - s^-3 + s^-2 in matrix form)
      R Gr[D][D];
      const int en = (EN == kEnMixed) ? (int)e.energy_of[i] : EN;
      if (en == kEnSG) {
#pragma unroll
        for (int a = 0; a < D; ++a)
#pragma unroll
          for (int k = 0; k < D; ++k) Gr[a][k] = w * (J[a][k] - Ji[k][a]);
      } else {
        R T1[D][D];  // J^-T J^-1
#pragma unroll
        for (int a = 0; a < D; ++a)
#pragma unroll
          for (int k = 0; k < D; ++k) {
            R s = R(0);
#pragma unroll
            for (int l = 0; l < D; ++l) s = fma(Ji[l][a], Ji[l][k], s);
            T1[a][k] = s;
          }
        R Rt[D][D];   // the rotation of J (SA only)
        if (en == kEnSA && !flipped) {
          if constexpr (D == 2) {
            const R ca = J[0][0] + J[1][1], sa = J[1][0] - J[0][1];
            const R ir = Tr<R>::rsqrt_(ca * ca + sa * sa);
            Rt[0][0] = ca * ir; Rt[0][1] = -sa * ir; Rt[1][0] = sa * ir; Rt[1][1] = ca * ir;
          } else {
            R cond;
            nearest_rotation3<R>(J, Rt, cond);
          }
        }
#pragma unroll
        for (int a = 0; a < D; ++a)
#pragma unroll
          for (int k = 0; k < D; ++k) {
            R s = R(0);
#pragma unroll
            for (int l = 0; l < D; ++l) s = fma(T1[a][l], Ji[k][l], s);
            if (en == kEnSA && !flipped) {
              R t = R(0);
#pragma unroll
              for (int l = 0; l < D; ++l) t = fma(T1[a][l], Rt[l][k], t);
              s += Rt[a][k] - t;
            }
            Gr[a][k] = w * (J[a][k] - s);
          }
      }
      store_terms<D, R>(e.contrib2, i, g, Gr);
      qv[Q_FLIPS] = flipped ? R(1) : R(0);
    }
  }
  block_reduce<R, NQ>(qv, partials);
}

// ---------------------------------------------------------------------------
// W-step right-hand-side terms g_j . r_i, r_i = mu_i (U_i P_i - Lambda_i)
// (eq. solvinginw), from a stored state (used when a checkpoint is restored)
// ---------------------------------------------------------------------------
template <int D, typename R>
__global__ void __launch_bounds__(kLocalBlock) k_rhs_terms(ElemBufs e, int m) {
  const int i = blockIdx.x * kLocalBlock + threadIdx.x;
  if (i >= m) return;
  int vid[D + 1];
  R g[D][D], w, mu;
  load_element<D, R>(e, m, i, vid, g, w, mu);
  const R* Pp = reinterpret_cast<const R*>(e.P);
  const R* Lp = reinterpret_cast<const R*>(e.Lam);
  const R* Up = reinterpret_cast<const R*>(e.U);
  R P[D][D], U[D][D];
  if constexpr (D == 2) {
    P[0][0] = Pp[i]; P[0][1] = P[1][0] = Pp[(int64_t)m + i]; P[1][1] = Pp[2 * (int64_t)m + i];
    const R c = Up[i], s = Up[(int64_t)m + i];
    U[0][0] = c; U[0][1] = -s; U[1][0] = s; U[1][1] = c;
  } else {
    P[0][0] = Pp[i]; P[0][1] = P[1][0] = Pp[(int64_t)m + i]; P[0][2] = P[2][0] = Pp[2 * (int64_t)m + i];
    P[1][1] = Pp[3 * (int64_t)m + i]; P[1][2] = P[2][1] = Pp[4 * (int64_t)m + i]; P[2][2] = Pp[5 * (int64_t)m + i];
    R qt[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) qt[k] = Up[(int64_t)k * m + i];
    quat_to_rot<R>(qt, U);
  }
  R Rhs[D][D];
#pragma unroll
  for (int a = 0; a < D; ++a)
#pragma unroll
    for (int k = 0; k < D; ++k) {
      R s = R(0);
#pragma unroll
      for (int l = 0; l < D; ++l) s = fma(U[a][l], P[l][k], s);
      Rhs[a][k] = mu * (s - Lp[(int64_t)(a * D + k) * m + i]);
    }
  store_terms<D, R>(e.contrib, i, g, Rhs);
}

// ---------------------------------------------------------------------------
// The paper's penalty schedule (Algorithm 2; Sec. 6, "Rescaling mu_i and
// Lambda"), per element, in double: MODE 0 sets mu_i = max(mu_min,i(P_i), w_i)
// (after the polar initialization); MODE 1 rescales after an iteration: with
// e_prim_i = |J_i - U_i P_i| and e_dual_i = mu_i |J_i - J_i^prev| (eq.
// primaldualerror; an error below 2^-40 (1 + |J_i|), times mu_i for e_dual, counts
// as zero), mu_i is multiplied by rho/2 if e_prim_i > rho e_dual_i and
// divided by rho/2 if e_dual_i > rho e_prim_i, never below mu_min,i(P_i)/2, and the
// scaled multiplier is multiplied by mu_old/mu_new (mu_i Lambda_i is unchanged).
// mu64 holds the penalties in double (the host refactors L from it); e.mu gets
// the local step's precision.
// ---------------------------------------------------------------------------
template <int D, typename R, int EN, int MODE>
__global__ void __launch_bounds__(kLocalBlock) k_penalty(ElemBufs e, int m, const void* __restrict__ vrec,
                                                        double* __restrict__ mu64, double rho) {
  const int i = blockIdx.x * kLocalBlock + threadIdx.x;
  if (i >= m) return;
  const R* Pp = reinterpret_cast<const R*>(e.P);
  double P[D][D];
  if constexpr (D == 2) {
    P[0][0] = Pp[i]; P[0][1] = P[1][0] = Pp[(int64_t)m + i]; P[1][1] = Pp[2 * (int64_t)m + i];
  } else {
    P[0][0] = Pp[i]; P[0][1] = P[1][0] = Pp[(int64_t)m + i]; P[0][2] = P[2][0] = Pp[2 * (int64_t)m + i];
    P[1][1] = Pp[3 * (int64_t)m + i]; P[1][2] = P[2][1] = Pp[4 * (int64_t)m + i]; P[2][2] = Pp[5 * (int64_t)m + i];
  }
  // eigenvalues of P; |grad f(P)|^2 = sum (p - p^-3)^2 (SD) or sum (p - 1/p)^2 (SG)
  double ev[3];
  if constexpr (D == 2) {
    const double h = 0.5 * (P[0][0] + P[1][1]), dd = 0.5 * (P[0][0] - P[1][1]);
    const double r = sqrt(dd * dd + P[0][1] * P[0][1]);
    ev[0] = h + r;
    ev[1] = h - r;
  } else {
    double V[3][3];
    sym3_eig<double>(P[0][0], P[0][1], P[0][2], P[1][1], P[1][2], P[2][2], ev, V);
  }
  const bool sg = EN == 1;
  double gn2 = 0.0;
#pragma unroll
  for (int k = 0; k < D; ++k) {
    const double p = ev[k];
    const double gk = sg ? p - 1.0 / p : p - 1.0 / (p * p * p);
    gn2 += gk * gk;
  }
  const double w = (double)reinterpret_cast<const R*>(e.w)[i];
  const double mmin = penalty_mu_min<D>(gn2, w, sg);
  double mu_new;
  if constexpr (MODE == 0) {
    mu_new = fmax(mmin, w);
  } else {
    const double mu_old = mu64[i];
    int vid[D + 1];
    R g[D][D], wr, mur;
    load_element<D, R>(e, m, i, vid, g, wr, mur);
    R J[D][D], dJ[D][D];
    element_jacobians<D, R>(vid, g, vrec, J, dJ);
    const R* Up = reinterpret_cast<const R*>(e.U);
    double U[D][D];
    if constexpr (D == 2) {
      const double c = Up[i], sn = Up[(int64_t)m + i];
      U[0][0] = c; U[0][1] = -sn; U[1][0] = sn; U[1][1] = c;
    } else {
      double qt[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) qt[k] = Up[(int64_t)k * m + i];
      quat_to_rot<double>(qt, U);
    }
    double rp = 0.0, rd = 0.0, rj = 0.0;
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
      for (int k = 0; k < D; ++k) {
        double up = 0.0;
#pragma unroll
        for (int l = 0; l < D; ++l) up += U[a][l] * P[l][k];
        const double r = (double)J[a][k] - up;
        rp += r * r;
        rd += (double)dJ[a][k] * (double)dJ[a][k];
        rj += (double)J[a][k] * (double)J[a][k];
      }
    // an error below the rounding floor of the element counts as zero
    const double floor_e = 0x1p-40 * (1.0 + sqrt(rj));
    double ep = sqrt(rp), ed = mu_old * sqrt(rd);
    if (!(ep > floor_e)) ep = 0.0;
    if (!(ed > mu_old * floor_e)) ed = 0.0;
    mu_new = mu_old;
    if (ep > rho * ed) mu_new = mu_old * (0.5 * rho);
    else if (ed > rho * ep) mu_new = mu_old / (0.5 * rho);
    mu_new = fmax(mu_new, 0.5 * mmin);
    const double f = mu_old / mu_new;
    R* Lp = reinterpret_cast<R*>(e.Lam);
#pragma unroll
    for (int q = 0; q < D * D; ++q) Lp[(int64_t)q * m + i] = (R)((double)Lp[(int64_t)q * m + i] * f);
  }
  mu64[i] = mu_new;
  reinterpret_cast<R*>(e.mu)[i] = (R)mu_new;
}

// h_i / mu_i = 4 w_i^2 B_i^2 / mu_i^2 with B_i^2 = 5 (1 + |grad f(P_i)|^2): the
// proximal weight of eq. proximalfunctionu at the bound of Prop. 1 (gamma = 1,
// eps = 0, as Sec. 6 sets them), from the current P (after the polar
// initialization: P^0).  grad f(P) for symmetric P has the eigenvalues
// p - p^-3 (SD), p - 1/p (SG), p - 1 - p^-3 + p^-2 (SA).
template <int D, typename R, int EN>
__global__ void __launch_bounds__(kLocalBlock) k_prox_weight(ElemBufs e, int m) {
  const int i = blockIdx.x * kLocalBlock + threadIdx.x;
  if (i >= m) return;
  const R* Pp = reinterpret_cast<const R*>(e.P);
  double ev[3];
  if constexpr (D == 2) {
    const double p00 = Pp[i], p01 = Pp[(int64_t)m + i], p11 = Pp[2 * (int64_t)m + i];
    const double h = 0.5 * (p00 + p11), dd = 0.5 * (p00 - p11);
    const double r = sqrt(dd * dd + p01 * p01);
    ev[0] = h + r;
    ev[1] = h - r;
  } else {
    double V[3][3];
    sym3_eig<double>(Pp[i], Pp[(int64_t)m + i], Pp[2 * (int64_t)m + i], Pp[3 * (int64_t)m + i],
                     Pp[4 * (int64_t)m + i], Pp[5 * (int64_t)m + i], ev, V);
  }
  double gn2 = 0.0;
#pragma unroll
  for (int k = 0; k < D; ++k) {
    const double p = ev[k];
    double gk;
    if constexpr (EN == kEnSG) gk = p - 1.0 / p;
    else if constexpr (EN == kEnSD) gk = p - 1.0 / (p * p * p);
    else gk = p - 1.0 - 1.0 / (p * p * p) + 1.0 / (p * p);
    gn2 += gk * gk;
  }
  const double w = (double)reinterpret_cast<const R*>(e.w)[i];
  const double mu = (double)reinterpret_cast<const R*>(e.mu)[i];
  reinterpret_cast<R*>(e.hmu)[i] = (R)(4.0 * w * w * 5.0 * (1.0 + gn2) / (mu * mu));
}

template <int D, typename R, int EN>
void dispatch_local(const LocalLaunch& L, cudaStream_t s) {
  const int bs = L.block > 0 ? L.block : kLocalBlock;
  const int grid = (L.m + bs - 1) / bs;
  if (L.e.joint) {
    if (L.check) k_local_step<D, R, EN, true, kVarJoint><<<grid, bs, 0, s>>>(L.e, L.m, L.vrec, L.partials);
    else k_local_step<D, R, EN, false, kVarJoint><<<grid, bs, 0, s>>>(L.e, L.m, L.vrec, L.partials);
  } else if (L.e.hmu) {
    if constexpr (EN != kEnMixed) {
      if (L.check) k_local_step<D, R, EN, true, kVarProx><<<grid, bs, 0, s>>>(L.e, L.m, L.vrec, L.partials);
      else k_local_step<D, R, EN, false, kVarProx><<<grid, bs, 0, s>>>(L.e, L.m, L.vrec, L.partials);
    }
  } else {
    if (L.check) k_local_step<D, R, EN, true, kVarPaper><<<grid, bs, 0, s>>>(L.e, L.m, L.vrec, L.partials);
    else k_local_step<D, R, EN, false, kVarPaper><<<grid, bs, 0, s>>>(L.e, L.m, L.vrec, L.partials);
  }
}

}  // namespace

void launch_local_step(const LocalLaunch& L, cudaStream_t s) {
#define FFA_LS(D, R) \
  do { if (L.energy == kEnSD) dispatch_local<D, R, kEnSD>(L, s); else if (L.energy == kEnSG) dispatch_local<D, R, kEnSG>(L, s); \
       else if (L.energy == kEnSA) dispatch_local<D, R, kEnSA>(L, s); else dispatch_local<D, R, kEnMixed>(L, s); } while (0)
  if (L.d == 2) { if (L.fp64) FFA_LS(2, double); else FFA_LS(2, float); }
  else { if (L.fp64) FFA_LS(3, double); else FFA_LS(3, float); }
#undef FFA_LS
}

void launch_rhs_terms(const LocalLaunch& L, cudaStream_t s) {
  const int grid = (L.m + kLocalBlock - 1) / kLocalBlock;
  if (L.d == 2) {
    if (L.fp64) k_rhs_terms<2, double><<<grid, kLocalBlock, 0, s>>>(L.e, L.m);
    else k_rhs_terms<2, float><<<grid, kLocalBlock, 0, s>>>(L.e, L.m);
  } else {
    if (L.fp64) k_rhs_terms<3, double><<<grid, kLocalBlock, 0, s>>>(L.e, L.m);
    else k_rhs_terms<3, float><<<grid, kLocalBlock, 0, s>>>(L.e, L.m);
  }
}

void launch_penalty(const LocalLaunch& L, int mode, double* mu64, double rho, cudaStream_t s) {
  const int grid = (L.m + kLocalBlock - 1) / kLocalBlock;
#define FFA_PEN(D, R, EN)                                                                                   \
  do {                                                                                                      \
    if (mode == 0) k_penalty<D, R, EN, 0><<<grid, kLocalBlock, 0, s>>>(L.e, L.m, L.vrec, mu64, rho);        \
    else k_penalty<D, R, EN, 1><<<grid, kLocalBlock, 0, s>>>(L.e, L.m, L.vrec, mu64, rho);                  \
  } while (0)
#define FFA_PEN2(D, R) do { if (L.energy == 1) FFA_PEN(D, R, 1); else FFA_PEN(D, R, 0); } while (0)
  if (L.d == 2) { if (L.fp64) FFA_PEN2(2, double); else FFA_PEN2(2, float); }
  else { if (L.fp64) FFA_PEN2(3, double); else FFA_PEN2(3, float); }
#undef FFA_PEN2
#undef FFA_PEN
}

void launch_init_polar(const LocalLaunch& L, cudaStream_t s) {
  const int grid = (L.m + kLocalBlock - 1) / kLocalBlock;
#define FFA_INIT(D, R) \
  do { if (L.energy == kEnSD) k_init_polar<D, R, kEnSD><<<grid, kLocalBlock, 0, s>>>(L.e, L.m, L.vrec); \
       else if (L.energy == kEnSG) k_init_polar<D, R, kEnSG><<<grid, kLocalBlock, 0, s>>>(L.e, L.m, L.vrec); \
       else if (L.energy == kEnSA) k_init_polar<D, R, kEnSA><<<grid, kLocalBlock, 0, s>>>(L.e, L.m, L.vrec); \
       else k_init_polar<D, R, kEnMixed><<<grid, kLocalBlock, 0, s>>>(L.e, L.m, L.vrec); } while (0)
  if (L.d == 2) { if (L.fp64) FFA_INIT(2, double); else FFA_INIT(2, float); }
  else { if (L.fp64) FFA_INIT(3, double); else FFA_INIT(3, float); }
#undef FFA_INIT
}

void launch_prox_weight(const LocalLaunch& L, cudaStream_t s) {
  const int grid = (L.m + kLocalBlock - 1) / kLocalBlock;
#define FFA_PW(D, R) \
  do { if (L.energy == kEnSD) k_prox_weight<D, R, kEnSD><<<grid, kLocalBlock, 0, s>>>(L.e, L.m); \
       else if (L.energy == kEnSG) k_prox_weight<D, R, kEnSG><<<grid, kLocalBlock, 0, s>>>(L.e, L.m); \
       else if (L.energy == kEnSA) k_prox_weight<D, R, kEnSA><<<grid, kLocalBlock, 0, s>>>(L.e, L.m); } while (0)
  if (L.d == 2) { if (L.fp64) FFA_PW(2, double); else FFA_PW(2, float); }
  else { if (L.fp64) FFA_PW(3, double); else FFA_PW(3, float); }
#undef FFA_PW
}

void launch_energy_terms(const LocalLaunch& L, int mode, cudaStream_t s) {
  const int grid = (L.m + kLocalBlock - 1) / kLocalBlock;
#define FFA_EN(D, R, EN)                                                                           \
  do {                                                                                             \
    if (mode == 0) k_energy_terms<D, R, EN, 0><<<grid, kLocalBlock, 0, s>>>(L.e, L.m, L.vrec, L.partials); \
    else k_energy_terms<D, R, EN, 1><<<grid, kLocalBlock, 0, s>>>(L.e, L.m, L.vrec, L.partials);           \
  } while (0)
#define FFA_EN3(D, R) \
  do { if (L.energy == kEnSD) FFA_EN(D, R, kEnSD); else if (L.energy == kEnSG) FFA_EN(D, R, kEnSG); \
       else if (L.energy == kEnSA) FFA_EN(D, R, kEnSA); else FFA_EN(D, R, kEnMixed); } while (0)
  if (L.d == 2) { if (L.fp64) FFA_EN3(2, double); else FFA_EN3(2, float); }
  else { if (L.fp64) FFA_EN3(3, double); else FFA_EN3(3, float); }
#undef FFA_EN3
#undef FFA_EN
}

}  // namespace ffa
