// Device decomposition of the W-step operator (ffa_devfactor.h): the kernels of
// each launch kind and the driver that runs a plan's launch program, plus the
// device assembly of L = sum_i mu_i G_i^T G_i from new penalties.
//
// Every tile product runs on one block of 256 threads: a 64 x 64 output tile,
// each thread 4 x 4 outputs (rows 4 tx + i, columns 4 ty + j: its operands are one
// 16-byte shared load each per step of the sum, and the 16 threads of a half warp
// store 64 consecutive rows of one output column), operands staged in shared
// memory 32 steps of the sum at a time.  Rows and columns past the end of a front are
// read as zero and not written.  Divisions and square roots are IEEE (no
// approximate forms in this file).
#include <cuda_runtime.h>

#include "ffa_devfactor.h"
#include "ffa_devfactor_launch.h"

namespace ffa {
namespace {

constexpr int kT = kDfTile;
constexpr int kKc = 32;
constexpr int kThreads = 256;

// operand tiles in shared memory: 32 steps of the sum x 64 rows, rows padded to
// 68 elements so that every group of four starts on 16 bytes
constexpr int kLd = kT + 4;
template <typename T>
struct __align__(16) GemmSmem {
  T a[kKc][kLd];
  T b[kKc][kLd];
};

// four consecutive elements from shared memory (one 16-byte load for float, two
// for double)
__device__ __forceinline__ void ld4(const float* p, float (&v)[4]) {
  const float4 q = *reinterpret_cast<const float4*>(p);
  v[0] = q.x;
  v[1] = q.y;
  v[2] = q.z;
  v[3] = q.w;
}
__device__ __forceinline__ void ld4(const double* p, double (&v)[4]) {
  const double2 q0 = *reinterpret_cast<const double2*>(p);
  const double2 q1 = *reinterpret_cast<const double2*>(p + 2);
  v[0] = q0.x;
  v[1] = q0.y;
  v[2] = q1.x;
  v[3] = q1.y;
}

// acc[i][j] += sum_{k < K} A(4 tx + i, k) B(4 ty + j, k), where A(r, k) =
// A[k lda + r] for r < ra and B(c, k) = B[c ldb + k] (BK) or B[k ldb + c] (!BK)
// for c < cb.  Ends with a barrier, after which every read of A and B is done.
template <typename T, bool BK>
__device__ __forceinline__ void gemm_acc(T (&acc)[4][4], const T* A, int64_t lda, int ra, const T* B, int64_t ldb,
                                         int cb, int K, GemmSmem<T>& sm) {
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  for (int k0 = 0; k0 < K; k0 += kKc) {
    const int kc = min(kKc, K - k0);
    for (int e = tid; e < kKc * kT; e += kThreads) {
      const int k = e >> 6, r = e & 63;
      sm.a[k][r] = (k < kc && r < ra) ? A[(int64_t)(k0 + k) * lda + r] : T(0);
    }
    if (BK) {
      for (int e = tid; e < kKc * kT; e += kThreads) {
        const int c = e >> 5, k = e & 31;
        sm.b[k][c] = (k < kc && c < cb) ? B[(int64_t)c * ldb + k0 + k] : T(0);
      }
    } else {
      for (int e = tid; e < kKc * kT; e += kThreads) {
        const int k = e >> 6, c = e & 63;
        sm.b[k][c] = (k < kc && c < cb) ? B[(int64_t)(k0 + k) * ldb + c] : T(0);
      }
    }
    __syncthreads();
#pragma unroll 4
    for (int k = 0; k < kc; ++k) {
      T a[4], b[4];
      ld4(&sm.a[k][4 * tx], a);
      ld4(&sm.b[k][4 * ty], b);
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
}

template <typename T>
__device__ __forceinline__ void zero_acc(T (&acc)[4][4]) {
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = T(0);
}

// F = 0 is done by a memset; the entries of L_FF go to their front positions
template <typename T>
__global__ void k_df_scatter(const int64_t* __restrict__ dst, const double* __restrict__ val, int64_t n,
                             T* __restrict__ F) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const int64_t t = dst[k];
  if (t >= 0) F[t] = (T)val[k];
}

// child c's update matrix (the trailing part of its front) into its parent's
// front: columns code .. code + kDfEaCols, one warp per column
template <typename T>
__global__ void __launch_bounds__(kThreads) k_df_extend_add(const DfNode* __restrict__ nodes,
                                                            const DfItem* __restrict__ items,
                                                            const int64_t* __restrict__ rel_off,
                                                            const int32_t* __restrict__ rel, T* F) {
  const DfItem it = items[blockIdx.x];
  const DfNode c = nodes[it.node];
  const DfNode s = nodes[c.parent];
  const int32_t ms = c.N - c.ns;
  const int32_t b = it.code + (int)(threadIdx.x >> 5);
  if (b >= ms) return;
  const int32_t* rl = rel + rel_off[it.node];
  const int32_t rb = rl[b];
  const T* src = F + c.fr_off + (int64_t)(c.ns + b) * c.ldF + c.ns;
  T* dst = F + s.fr_off + (int64_t)rb * s.ldF;
  for (int32_t a = b + (int)(threadIdx.x & 31); a < ms; a += 32) dst[rl[a]] += src[a];
}

// diagonal block of panel p: Cholesky and inverse together, right-looking over
// the columns k in shared memory with the whole block: column k of L and row k of
// X = inv(L) are scaled by 1 / sqrt(pivot), then the trailing lower triangle takes
// -L_ik L_jk and the rows below k of X take -L_ik X_kj (X starts as the identity,
// so this is forward substitution of L X = I by columns).  Threads (tx, ty) cover
// column tx of rows k + 1 + ty, k + 5 + ty, ...
template <typename T>
__global__ void __launch_bounds__(kThreads) k_df_diag(const DfNode* __restrict__ nodes,
                                                      const DfItem* __restrict__ items, int p, T* __restrict__ F,
                                                      T* __restrict__ Lv, int32_t* __restrict__ err) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T(*D)[kT + 1] = reinterpret_cast<T(*)[kT + 1]>(smem_raw);
  T(*X)[kT + 1] = D + kT;
  const DfItem it = items[blockIdx.x];
  const DfNode d = nodes[it.node];
  const DfPanel g = df_panel(d, p);
  const int w = g.w, tid = threadIdx.x, tx = tid & 63, ty = tid >> 6;
  T* Fd = F + d.fr_off + (int64_t)g.c0 * d.ldF + g.c0;
  T* Ld = Lv + d.li_off + (int64_t)g.c0 * d.ldL + g.c0;
  for (int e = tid; e < kT * kT; e += kThreads) {
    const int i = e & 63, j = e >> 6;
    D[i][j] = (i < w && j < w && i >= j) ? Fd[(int64_t)j * d.ldF + i] : T(0);
    X[i][j] = i == j ? T(1) : T(0);
  }
  __syncthreads();
  for (int k = 0; k < w; ++k) {
    T pv = D[k][k];
    if (!(pv > T(0)) || !(pv < T(INFINITY))) {
      if (tid == 0) atomicExch(err, 1);
      pv = T(1);
    }
    const T dk = sqrt(pv), inv = T(1) / dk;
    if (tid < kT) {
      if (tid > k && tid < w) D[tid][k] *= inv;
    } else if (tid < 2 * kT) {
      const int j = tid - kT;
      if (j <= k) X[k][j] *= inv;
    }
    __syncthreads();
    for (int i = k + 1 + ty; i < w; i += kThreads / kT) {
      const T lik = D[i][k];
      if (tx <= k) X[i][tx] -= lik * X[k][tx];
      else if (tx <= i) D[i][tx] -= lik * D[tx][k];
    }
    if (tid == 0) D[k][k] = dk;
    __syncthreads();
  }
  for (int e = tid; e < kT * kT; e += kThreads) {
    const int i = e & 63, j = e >> 6;
    if (i < w && j < w) {
      if (i >= j) Fd[(int64_t)j * d.ldF + i] = D[i][j];
      Ld[(int64_t)j * d.ldL + i] = X[i][j];
    }
  }
}

// panel p: rows below the diagonal block times inv(L_pp)^T (code >= 0), or block
// (p, j) of inv(L_ss) from its sum, X_pj = -X_pp S_pj (code < 0), both in place
template <typename T>
__global__ void __launch_bounds__(kThreads) k_df_solve(const DfNode* __restrict__ nodes,
                                                       const DfItem* __restrict__ items, int p, T* F, T* Lv) {
  __shared__ GemmSmem<T> sm;
  const DfItem it = items[blockIdx.x];
  const DfNode d = nodes[it.node];
  const DfPanel g = df_panel(d, p);
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  T* Fs = F + d.fr_off;
  T* L = Lv + d.li_off;
  T acc[4][4];
  zero_acc(acc);
  if (it.code >= 0) {
    const int R0 = g.t0 + it.code * kT, ra = min(kT, d.N - R0);
    gemm_acc<T, false>(acc, Fs + (int64_t)g.c0 * d.ldF + R0, d.ldF, ra, L + (int64_t)g.c0 * d.ldL + g.c0, d.ldL,
                       g.w, g.w, sm);
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int r = 4 * tx + i, c = 4 * ty + j;
        if (r < ra && c < g.w) Fs[(int64_t)(g.c0 + c) * d.ldF + R0 + r] = acc[i][j];
      }
  } else {
    const int j0 = (-1 - it.code) * kT;
    gemm_acc<T, true>(acc, L + (int64_t)g.c0 * d.ldL + g.c0, d.ldL, g.w, L + (int64_t)j0 * d.ldL + g.c0, d.ldL,
                      kT, g.w, sm);
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int r = 4 * tx + i, c = 4 * ty + j;
        if (r < g.w) L[(int64_t)(j0 + c) * d.ldL + g.c0 + r] = -acc[i][j];
      }
  }
}

// panel p: trailing tiles F_IJ -= L_I L_J^T (code >= 0), or S_qj += L_qp X_pj
template <typename T>
__global__ void __launch_bounds__(kThreads) k_df_update(const DfNode* __restrict__ nodes,
                                                        const DfItem* __restrict__ items, int p, T* F, T* Lv) {
  __shared__ GemmSmem<T> sm;
  const DfItem it = items[blockIdx.x];
  const DfNode d = nodes[it.node];
  const DfPanel g = df_panel(d, p);
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  T* Fs = F + d.fr_off;
  T acc[4][4];
  zero_acc(acc);
  if (it.code >= 0) {
    const int I = it.code >> 16, J = it.code & 0xffff;
    const int R0 = g.t0 + I * kT, C0 = g.t0 + J * kT;
    const int ra = min(kT, d.N - R0), cb = min(kT, d.N - C0);
    gemm_acc<T, false>(acc, Fs + (int64_t)g.c0 * d.ldF + R0, d.ldF, ra, Fs + (int64_t)g.c0 * d.ldF + C0, d.ldF, cb,
                       g.w, sm);
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int r = 4 * tx + i, c = 4 * ty + j;
        if (r < ra && c < cb) Fs[(int64_t)(C0 + c) * d.ldF + R0 + r] -= acc[i][j];
      }
  } else {
    const int q = (-1 - it.code) >> 16, jb = (-1 - it.code) & 0xffff;
    const int r0 = q * kT, rq = min(kT, d.ns - r0), j0 = jb * kT;
    const int cb = jb == p ? g.w : kT;
    T* L = Lv + d.li_off;
    gemm_acc<T, true>(acc, Fs + (int64_t)g.c0 * d.ldF + r0, d.ldF, rq, L + (int64_t)j0 * d.ldL + g.c0, d.ldL, cb,
                      g.w, sm);
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int r = 4 * tx + i, c = 4 * ty + j;
        if (r < rq && c < cb) L[(int64_t)(j0 + c) * d.ldL + r0 + r] += acc[i][j];
      }
  }
}

// tile (A, J) of L_rs inv(L_ss) into B_s (float)
template <typename T>
__global__ void __launch_bounds__(kThreads) k_df_brs(const DfNode* __restrict__ nodes,
                                                     const DfItem* __restrict__ items, const T* __restrict__ F,
                                                     const T* __restrict__ Lv, float* __restrict__ blocks) {
  __shared__ GemmSmem<T> sm;
  const DfItem it = items[blockIdx.x];
  const DfNode d = nodes[it.node];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int A = it.code >> 16, J = it.code & 0xffff;
  const int R0 = d.ns + A * kT, col0 = J * kT;
  const int ra = min(kT, d.N - R0), cb = min(kT, d.ns - col0);
  const T* L = Lv + d.li_off;
  T acc[4][4];
  zero_acc(acc);
  gemm_acc<T, true>(acc, F + d.fr_off + (int64_t)col0 * d.ldF + R0, d.ldF, ra, L + (int64_t)col0 * d.ldL + col0,
                    d.ldL, cb, d.ns - col0, sm);
  float* B = blocks + d.blk_off;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int r = 4 * tx + i, c = 4 * ty + j;
      if (r < ra && c < cb) B[(int64_t)(col0 + c) * d.ld + R0 + r] = (float)acc[i][j];
    }
}

// block column J of inv(L_ss) into B_s (float), zero above the diagonal
template <typename T>
__global__ void __launch_bounds__(kThreads) k_df_pack(const DfNode* __restrict__ nodes,
                                                      const DfItem* __restrict__ items, const T* __restrict__ Lv,
                                                      float* __restrict__ blocks) {
  const DfItem it = items[blockIdx.x];
  const DfNode d = nodes[it.node];
  const int col0 = it.code * kT, ncol = min(kT, d.ns - col0);
  const T* L = Lv + d.li_off;
  float* B = blocks + d.blk_off;
  for (int c = threadIdx.x >> 5; c < ncol; c += kThreads / 32) {
    const int j = col0 + c;
    for (int i = threadIdx.x & 31; i < d.ns; i += 32)
      B[(int64_t)j * d.ld + i] = i >= j ? (float)L[(int64_t)j * d.ldL + i] : 0.0f;
  }
}

// sum_a g_j[a] g_l[a] of element i, g_0 = -(g_1 + ... + g_d)
template <int D>
__device__ __forceinline__ double grad_dot(const double* __restrict__ g, int i, int j, int l) {
  const double* gi = g + (int64_t)i * D * D;
  double dv = 0.0;
#pragma unroll
  for (int a = 0; a < D; ++a) {
    double s0 = 0.0;
#pragma unroll
    for (int jj = 0; jj < D; ++jj) s0 += gi[jj * D + a];
    const double gj = j > 0 ? gi[(j - 1) * D + a] : -s0;
    const double gl = l > 0 ? gi[(l - 1) * D + a] : -s0;
    dv += gj * gl;
  }
  return dv;
}

template <int D>
__global__ void k_df_assemble(const int64_t* __restrict__ ptr, const int32_t* __restrict__ src, int64_t n,
                              const double* __restrict__ g, const double* __restrict__ mu, double* __restrict__ out) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  double v = 0.0;
  for (int64_t t = ptr[k]; t < ptr[k + 1]; ++t) {
    const int32_t code = src[t];
    const int i = code >> 4;
    v += mu[i] * grad_dot<D>(g, i, (code >> 2) & 3, code & 3);
  }
  out[k] = v;
}

__global__ void k_df_gather(const int32_t* __restrict__ idx, int64_t n, const double* __restrict__ in,
                            double* __restrict__ out) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n) out[k] = in[idx[k]];
}

inline unsigned grid_of(int64_t n, int block) { return (unsigned)((n + block - 1) / block); }

template <typename T>
cudaError_t run_program(const DevFactorDev& D, const std::vector<DfLaunch>& prog, const double* ell_val,
                        float* blocks, cudaStream_t s) {
  T* F = static_cast<T*>(D.F);
  T* Lv = static_cast<T*>(D.Lv);
  const size_t diag_smem = 2 * kT * (kT + 1) * sizeof(T);
  cudaError_t e = cudaFuncSetAttribute(k_df_diag<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)diag_smem);
  if (e != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(F, 0, (size_t)D.front_elems * sizeof(T), s)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(Lv, 0, (size_t)D.linv_elems * sizeof(T), s)) != cudaSuccess) return e;
  if (D.n_slots > 0) k_df_scatter<T><<<grid_of(D.n_slots, 256), 256, 0, s>>>(D.orig_dst, ell_val, D.n_slots, F);
  for (const DfLaunch& L : prog) {
    const DfItem* it = D.items + L.off;
    const unsigned grid = (unsigned)L.count;
    switch (L.kind) {
      case kDfExtendAdd:
        k_df_extend_add<T><<<grid, kThreads, 0, s>>>(D.nodes, it, D.rel_off, D.rel, F);
        break;
      case kDfDiag:
        k_df_diag<T><<<grid, kThreads, diag_smem, s>>>(D.nodes, it, L.p, F, Lv, D.err);
        break;
      case kDfSolve:
        k_df_solve<T><<<grid, kThreads, 0, s>>>(D.nodes, it, L.p, F, Lv);
        break;
      case kDfUpdate:
        k_df_update<T><<<grid, kThreads, 0, s>>>(D.nodes, it, L.p, F, Lv);
        break;
      case kDfBrs:
        k_df_brs<T><<<grid, kThreads, 0, s>>>(D.nodes, it, F, Lv, blocks);
        break;
      case kDfPack:
        k_df_pack<T><<<grid, kThreads, 0, s>>>(D.nodes, it, Lv, blocks);
        break;
      default:
        return cudaErrorInvalidValue;
    }
  }
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_devfactor(const DevFactorDev& D, const std::vector<DfLaunch>& prog, const double* ell_val,
                             float* blocks, cudaStream_t s) {
  return D.fp64 ? run_program<double>(D, prog, ell_val, blocks, s) : run_program<float>(D, prog, ell_val, blocks, s);
}

cudaError_t launch_device_assembly(const DevAssemblyDev& A, int d, const double* mu, double* ell_val, double* fc_val,
                                   double* cf_val, cudaStream_t s) {
  if (A.n_ell > 0) {
    if (d == 2) k_df_assemble<2><<<grid_of(A.n_ell, 256), 256, 0, s>>>(A.ell_ptr, A.ell_src, A.n_ell, A.g, mu, ell_val);
    else k_df_assemble<3><<<grid_of(A.n_ell, 256), 256, 0, s>>>(A.ell_ptr, A.ell_src, A.n_ell, A.g, mu, ell_val);
  }
  if (A.n_fc > 0) {
    if (d == 2) k_df_assemble<2><<<grid_of(A.n_fc, 256), 256, 0, s>>>(A.fc_ptr, A.fc_src, A.n_fc, A.g, mu, fc_val);
    else k_df_assemble<3><<<grid_of(A.n_fc, 256), 256, 0, s>>>(A.fc_ptr, A.fc_src, A.n_fc, A.g, mu, fc_val);
    k_df_gather<<<grid_of(A.n_fc, 256), 256, 0, s>>>(A.cf_src, A.n_fc, fc_val, cf_val);
  }
  return cudaGetLastError();
}

}  // namespace ffa
