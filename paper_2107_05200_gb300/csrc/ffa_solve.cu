// Vertex-side kernels of the W step (eq. solvinginw): right-hand-side gather G^T r,
// the double-precision residual b - L_FF W_F, the float supernodal triangular
// solves that turn the residual into a correction (mixed-precision refinement),
// and the vertex update that publishes W for the next local step.  Also the
// reductions that evaluate the termination test of eqs. primaldualerror/primaldualthresholds.
#include <math.h>

#include <algorithm>

#include "ffa_internal.h"
#include "ffa_math.cuh"

namespace ffa {
namespace {

// ---------------------------------------------------------------------------
// vertex update: W_new from the eliminated-order solution (free vertices) or the
// pinned positions; writes W, optionally X, dW = W_new - W_old, and the records
// ---------------------------------------------------------------------------
template <int D, bool FP64>
__global__ void __launch_bounds__(kVertexBlock) k_vertex_update(VertexLaunch V) {
  const int v = blockIdx.x * kVertexBlock + threadIdx.x;
  if (v >= V.n) return;
  double wn[D], wo[D];
  const int e = V.v2e[v];
#pragma unroll
  for (int k = 0; k < D; ++k) wo[k] = V.W[(int64_t)v * D + k];
  if (V.W_in) {
#pragma unroll
    for (int k = 0; k < D; ++k) wn[k] = V.W_in[(int64_t)v * D + k];
    if (e < 0 && V.v2pin != nullptr) {
      const int p = V.v2pin[v];
#pragma unroll
      for (int k = 0; k < D; ++k) wn[k] = V.pin_pos[(int64_t)p * D + k];
    }
  } else if (e >= 0) {
#pragma unroll
    for (int k = 0; k < D; ++k) {
      double x = V.Wnew_free[(int64_t)e * D + k];
      if (V.corr) x += (double)V.corr[(int64_t)e * D + k];
      wn[k] = x;
    }
  } else {
    const int p = V.v2pin[v];
#pragma unroll
    for (int k = 0; k < D; ++k) wn[k] = V.pin_pos[(int64_t)p * D + k];
  }
  double dw[D];
#pragma unroll
  for (int k = 0; k < D; ++k) {
    dw[k] = V.write_dw ? wn[k] - wo[k] : 0.0;
    V.W[(int64_t)v * D + k] = wn[k];
    if (V.X && e >= 0) V.X[(int64_t)e * D + k] = wn[k];
  }
  if constexpr (FP64) {
    double2* r = reinterpret_cast<double2*>(V.vrec) + (int64_t)v * D;
    if constexpr (D == 3) {
      r[0] = make_double2(wn[0], wn[1]);
      r[1] = make_double2(wn[2], dw[0]);
      r[2] = make_double2(dw[1], dw[2]);
    } else {
      r[0] = make_double2(wn[0], wn[1]);
      r[1] = make_double2(dw[0], dw[1]);
    }
  } else {
    float hi[D], lo[D];
#pragma unroll
    for (int k = 0; k < D; ++k) {
      hi[k] = (float)wn[k];
      lo[k] = (float)(wn[k] - (double)hi[k]);
    }
    float4* r = reinterpret_cast<float4*>(V.vrec) + (int64_t)v * D;
    if constexpr (D == 3) {
      r[0] = make_float4(hi[0], hi[1], hi[2], (float)dw[0]);
      r[1] = make_float4(lo[0], lo[1], lo[2], (float)dw[1]);
      r[2] = make_float4((float)dw[2], 0.f, 0.f, 0.f);
    } else {
      r[0] = make_float4(hi[0], hi[1], lo[0], lo[1]);
      r[1] = make_float4((float)dw[0], (float)dw[1], 0.f, 0.f);
    }
  }
}

// ---------------------------------------------------------------------------
// gather of per-element vertex terms: out_row = sum over the incidences of the
// row's vertex (+ add_row); float terms are summed in double-float.  kGatherLanes
// consecutive lanes share a row, each taking every kGatherLanes-th incidence with
// its loads issued together, and the lane sums meet by shuffles, so a row costs a
// few dependent load latencies instead of one per incidence.
// ---------------------------------------------------------------------------
template <int D, bool FP64>
__global__ void __launch_bounds__(kVertexBlock) k_gather(GatherLaunch G) {
  const int t = blockIdx.x * kVertexBlock + threadIdx.x;
  const int row = t / kGatherLanes, sub = t % kGatherLanes;
  const bool active = row < G.rows;
  double outv[D];
  double sq = 0.0;
  int64_t q0 = 0, q1 = 0;
  if (active) {
    const int v = G.row_vertex ? G.row_vertex[row] : row;
    q0 = G.inc_ptr[v] + sub;
    q1 = G.inc_ptr[v + 1];
  }
  if constexpr (FP64) {
    const double* c = reinterpret_cast<const double*>(G.contrib);
    double acc[D];
#pragma unroll
    for (int k = 0; k < D; ++k) acc[k] = 0.0;
    int64_t q = q0;
    for (; q + 3 * kGatherLanes < q1; q += 4 * kGatherLanes) {
      int64_t base[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) base[u] = (int64_t)__ldg(G.inc + q + u * kGatherLanes) * D;
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int k = 0; k < D; ++k) acc[k] += __ldg(c + base[u] + k);
    }
    for (; q < q1; q += kGatherLanes) {
      const int64_t base = (int64_t)__ldg(G.inc + q) * D;
#pragma unroll
      for (int k = 0; k < D; ++k) acc[k] += __ldg(c + base + k);
    }
#pragma unroll
    for (int k = 0; k < D; ++k) {
      double a = acc[k];
#pragma unroll
      for (int o = 1; o < kGatherLanes; o <<= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
      outv[k] = a;
    }
  } else {
    const float* c = reinterpret_cast<const float*>(G.contrib);
    FF acc[D];
#pragma unroll
    for (int k = 0; k < D; ++k) acc[k] = FF{0.f, 0.f};
    int64_t q = q0;
    for (; q + 3 * kGatherLanes < q1; q += 4 * kGatherLanes) {
      int64_t base[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) base[u] = (int64_t)__ldg(G.inc + q + u * kGatherLanes) * D;
      float v[4][D];
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int k = 0; k < D; ++k) v[u][k] = __ldg(c + base[u] + k);
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int k = 0; k < D; ++k) acc[k] = ff_addf(acc[k], v[u][k]);
    }
    for (; q < q1; q += kGatherLanes) {
      const int64_t base = (int64_t)__ldg(G.inc + q) * D;
#pragma unroll
      for (int k = 0; k < D; ++k) acc[k] = ff_addf(acc[k], __ldg(c + base + k));
    }
#pragma unroll
    for (int k = 0; k < D; ++k) {
      FF a = acc[k];
#pragma unroll
      for (int o = 1; o < kGatherLanes; o <<= 1) {
        const FF b{__shfl_xor_sync(0xffffffffu, a.hi, o), __shfl_xor_sync(0xffffffffu, a.lo, o)};
        a = ff_add(a, b);
      }
      outv[k] = (double)a.hi + (double)a.lo;
    }
  }
  if (active && sub == 0) {
#pragma unroll
    for (int k = 0; k < D; ++k) {
      if (G.add) outv[k] += G.add[(int64_t)row * D + k];
      if (G.out) G.out[(int64_t)row * D + k] = outv[k];
      sq += outv[k] * outv[k];
    }
  }
  if (G.mesh_of) {
    // batched meshes (rows are the vertices, sorted by mesh): per-mesh sums of
    // squares in a fixed order; a mesh wholly inside the block is written to
    // mesh_acc, the block's first and last meshes to mesh_part (added up in block
    // order by launch_mesh_partials)
    constexpr int kRowsPerBlock = kVertexBlock / kGatherLanes;
    const int r0 = blockIdx.x * kRowsPerBlock;
    const int r1 = min(G.rows, r0 + kRowsPerBlock);
    const int first = G.mesh_of[r0], last = G.mesh_of[r1 - 1];
    const int mine = (active && sub == 0) ? G.mesh_of[row] : -1;
    __shared__ double red_m[kVertexBlock / 32];
    for (int k = first; k <= last; ++k) {   // block-uniform
      double w = (mine == k) ? sq : 0.0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
      if ((threadIdx.x & 31) == 0) red_m[threadIdx.x >> 5] = w;
      __syncthreads();
      if (threadIdx.x == 0) {
        double t = 0.0;
        for (int wv = 0; wv < kVertexBlock / 32; ++wv) t += red_m[wv];
        if (k == first) G.mesh_part[(int64_t)blockIdx.x * 2 + 0] = t;
        else if (k == last) G.mesh_part[(int64_t)blockIdx.x * 2 + 1] = t;
        else G.mesh_acc[(int64_t)k * (NQ + 1) + NQ] = t;
      }
      __syncthreads();
    }
  } else if (G.partials) {
    __shared__ double red[kVertexBlock / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = sq;
    __syncthreads();
    if (threadIdx.x == 0) {
      double s = 0.0;
      for (int w = 0; w < kVertexBlock / 32; ++w) s += red[w];
      G.partials[blockIdx.x] = s;
    }
  }
}

// ---------------------------------------------------------------------------
// residual y = float(b - L_FF X) in double (ELL, column-major, eliminated order)
// ---------------------------------------------------------------------------
template <int D>
__device__ __forceinline__ void residual_row(const int32_t* __restrict__ col, const double* __restrict__ val,
                                             int width, int nF, const double* __restrict__ X,
                                             const double* __restrict__ b, float* __restrict__ y, int i, double& rr,
                                             double& bb) {
  double acc[D];
#pragma unroll
  for (int k = 0; k < D; ++k) acc[k] = b[(int64_t)i * D + k];
  // the index and value loads of 4 entries go out together, then their X gathers
  int q = 0;
  for (; q + 4 <= width; q += 4) {
    int j[4];
    double a[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      j[u] = __ldg(col + (int64_t)(q + u) * nF + i);
      a[u] = __ldg(val + (int64_t)(q + u) * nF + i);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int k = 0; k < D; ++k) acc[k] = fma(-a[u], __ldg(X + (int64_t)j[u] * D + k), acc[k]);
  }
  for (; q < width; ++q) {
    const int j = __ldg(col + (int64_t)q * nF + i);
    const double a = __ldg(val + (int64_t)q * nF + i);
#pragma unroll
    for (int k = 0; k < D; ++k) acc[k] = fma(-a, __ldg(X + (int64_t)j * D + k), acc[k]);
  }
#pragma unroll
  for (int k = 0; k < D; ++k) {
    y[(int64_t)i * D + k] = (float)acc[k];
    rr += acc[k] * acc[k];
    const double bk = b[(int64_t)i * D + k];
    bb += bk * bk;
  }
}

template <int D>
__global__ void __launch_bounds__(kVertexBlock) k_residual(const int32_t* __restrict__ col, const double* __restrict__ val,
                                                            int width, int nF, const double* __restrict__ X,
                                                            const double* __restrict__ b, float* __restrict__ y,
                                                            double* __restrict__ partials) {
  const int i = blockIdx.x * kVertexBlock + threadIdx.x;
  double rr = 0.0, bb = 0.0;
  if (i < nF) residual_row<D>(col, val, width, nF, X, b, y, i, rr, bb);
  if (partials) {
    __shared__ double red[2][kVertexBlock / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      rr += __shfl_xor_sync(0xffffffffu, rr, o);
      bb += __shfl_xor_sync(0xffffffffu, bb, o);
    }
    if ((threadIdx.x & 31) == 0) {
      red[0][threadIdx.x >> 5] = rr;
      red[1][threadIdx.x >> 5] = bb;
    }
    __syncthreads();
    if (threadIdx.x < 2) {
      double s = 0.0;
      for (int w = 0; w < kVertexBlock / 32; ++w) s += red[threadIdx.x][w];
      partials[(int64_t)blockIdx.x * 2 + threadIdx.x] = s;
    }
  }
}

// nu = S^-1 (A_F X - b'), on one block: the c x d residual of the constraints
// in shared memory, then the small dense product
template <int D>
__global__ void __launch_bounds__(256) k_constraint_nu(ConstraintLaunch C) {
  __shared__ double t[kMaxConstraints * D];
  for (int q = threadIdx.x; q < C.c * D; q += blockDim.x) {
    const int r = q / D, k = q - r * D;
    double a = -C.bprime[q];
    for (int64_t e = C.ptr[r]; e < C.ptr[r + 1]; ++e) a = fma(C.val[e], C.X[(int64_t)C.col[e] * D + k], a);
    t[q] = a;
  }
  __syncthreads();
  for (int q = threadIdx.x; q < C.c * D; q += blockDim.x) {
    const int r = q / D, k = q - r * D;
    double a = 0.0;
    for (int j = 0; j < C.c; ++j) a = fma(C.Sinv[(int64_t)r * C.c + j], t[j * D + k], a);
    C.nu[q] = a;
  }
}

// X <- X - Z nu, one thread per free row
template <int D>
__global__ void __launch_bounds__(kVertexBlock) k_constraint_project(ConstraintLaunch C) {
  __shared__ double nu[kMaxConstraints * D];
  for (int q = threadIdx.x; q < C.c * D; q += blockDim.x) nu[q] = C.nu[q];
  __syncthreads();
  const int i = blockIdx.x * kVertexBlock + threadIdx.x;
  if (i >= C.nF) return;
  double acc[D];
#pragma unroll
  for (int k = 0; k < D; ++k) acc[k] = 0.0;
  for (int r = 0; r < C.c; ++r) {
    const double zr = C.Z[(int64_t)r * C.nF + i];
#pragma unroll
    for (int k = 0; k < D; ++k) acc[k] = fma(zr, nu[r * D + k], acc[k]);
  }
#pragma unroll
  for (int k = 0; k < D; ++k) C.X[(int64_t)i * D + k] -= acc[k];
}

__global__ void k_copy_columns(const double* __restrict__ src, int d, double* __restrict__ dst, int c, int c0,
                               int count, int nF) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= (int64_t)nF * count) return;
  const int64_t i = q / count;
  const int k = (int)(q - i * count);
  dst[(int64_t)(c0 + k) * nF + i] = src[i * d + k];
}

__global__ void k_axpy(int n, double* __restrict__ X, const float* __restrict__ x) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) X[i] += (double)x[i];
}

// ---------------------------------------------------------------------------
// supernodal solves.  B_s is column-major with a leading dimension ld that is a
// multiple of 4, so every lane reads 4 consecutive rows of a column as one
// float4.  Every task below runs on a whole block of kSolveThreads threads.
//
// Wide task (node, r0, c0) of the forward pass: rows [r0, r0+128) of B_s times
// the slice [c0, c0+W) of f = y[cols(s)] (W = 32 per warp); warp w takes columns
// c0+32w .. c0+32w+31, the per-warp partial sums are added in shared memory and the 128 row
// results go out as one set of atomics: rows < n_s into z, rows >= n_s
// subtracted from y at the structure rows.
// ---------------------------------------------------------------------------
// Factor data is read once per pass: no L1 allocation, and in L2 either
// evict-first or, for the blocks the next pass reads first, evict-last.
__device__ __forceinline__ uint64_t l2_policy(int keep) {
  uint64_t pol;
  if (keep) asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
  else asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}

__device__ __forceinline__ float4 ldg_stream(const float* p, uint64_t pol) {
  float4 v;
  asm("ld.global.nc.L1::no_allocate.L2::cache_hint.v4.f32 {%0, %1, %2, %3}, [%4], %5;"
      : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
      : "l"(p), "l"(pol));
  return v;
}

template <int D>
__device__ __forceinline__ void forward_wide(const Task& t, const NodeDev& nd, const int32_t* __restrict__ rows,
                                             const float* __restrict__ blocks, float* __restrict__ y,
                                             float* __restrict__ z, float* smem) {
  const uint64_t pol = l2_policy(nd.l2_keep);
  const int W = t.kind;      // columns of this task: a multiple of 8, at most kFwdCols
  const int cpw = W / kSolveWarps;    // columns per warp
  float (*fs)[D] = reinterpret_cast<float (*)[D]>(smem);                       // [W][D]
  float (*red)[kFwdRows][D] = reinterpret_cast<float (*)[kFwdRows][D]>(smem + kFwdCols * D);  // [warps][128][D]
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ntot = nd.ncol + nd.nrow;
  const int nc = min(W, nd.ncol - t.c0);
  const int r = t.r0 + 4 * lane;
  const int cw0 = cpw * warp;
  const int ncw = (r < nd.ld) ? max(0, min(cpw, nc - cw0)) : 0;
  const float* B = blocks + nd.blk_off + (int64_t)(t.c0 + cw0) * nd.ld + r;
  // the first kFwdBatch columns are in flight while f is staged
  const int n0 = min(kFwdBatch, ncw);
  float4 b[kFwdBatch];
#pragma unroll
  for (int u = 0; u < kFwdBatch; ++u)
    b[u] = (u < n0) ? ldg_stream(B + (int64_t)u * nd.ld, pol) : make_float4(0.f, 0.f, 0.f, 0.f);
  for (int q = threadIdx.x; q < nc * D; q += kSolveThreads) {
    const int c = q / D, k = q - c * D;
    fs[c][k] = __ldcg(y + (int64_t)(nd.col0 + t.c0 + c) * D + k);
  }
  __syncthreads();
  float acc[4][D];
#pragma unroll
  for (int q = 0; q < 4; ++q)
#pragma unroll
    for (int k = 0; k < D; ++k) acc[q][k] = 0.f;
  auto fma_col = [&](const float4& bv, int c) {
#pragma unroll
    for (int k = 0; k < D; ++k) {
      const float f = fs[cw0 + c][k];
      acc[0][k] = fmaf(bv.x, f, acc[0][k]);
      acc[1][k] = fmaf(bv.y, f, acc[1][k]);
      acc[2][k] = fmaf(bv.z, f, acc[2][k]);
      acc[3][k] = fmaf(bv.w, f, acc[3][k]);
    }
  };
#pragma unroll
  for (int u = 0; u < kFwdBatch; ++u)
    if (u < n0) fma_col(b[u], u);
  int c = n0;
  for (; c + kFwdBatch <= ncw; c += kFwdBatch) {
#pragma unroll
    for (int u = 0; u < kFwdBatch; ++u) b[u] = ldg_stream(B + (int64_t)(c + u) * nd.ld, pol);
#pragma unroll
    for (int u = 0; u < kFwdBatch; ++u) fma_col(b[u], c + u);
  }
  for (; c < ncw; ++c) fma_col(ldg_stream(B + (int64_t)c * nd.ld, pol), c);
#pragma unroll
  for (int q = 0; q < 4; ++q)
#pragma unroll
    for (int k = 0; k < D; ++k) red[warp][4 * lane + q][k] = acc[q][k];
  __syncthreads();
  if (threadIdx.x < kFwdRows) {
    const int row = t.r0 + threadIdx.x;
    if (row < ntot && !(row < nd.ncol && row < t.c0)) {
      float sum[D];
#pragma unroll
      for (int k = 0; k < D; ++k) {
        float a = 0.f;
#pragma unroll
        for (int w = 0; w < kSolveWarps; ++w) a += red[w][threadIdx.x][k];
        sum[k] = a;
      }
      if (row < nd.ncol) {
#pragma unroll
        for (int k = 0; k < D; ++k) atomicAdd(z + (int64_t)(nd.col0 + row) * D + k, sum[k]);
      } else {
        const int rr = __ldg(rows + nd.row_off + (row - nd.ncol));
#pragma unroll
        for (int k = 0; k < D; ++k) atomicAdd(y + (int64_t)rr * D + k, -sum[k]);
      }
    }
  }
}

// Node task of the forward pass: a whole small node (at most kNarrowCols columns,
// ld <= kNodeMaxLd, at most kNodeMaxBytes of B_s) on one block.  Thread (g, j) owns the 4-row group g of the
// ld/4 groups and the column slice j (columns j, j + S, j + 2S, ...) with
// S = floor(kSolveThreads / (ld/4)) slices, so a small node is streamed in one or two
// rounds of loads; the S partial sums of each row meet in shared memory.  z_s
// is stored directly (no other task touches it).
template <int D>
__device__ __forceinline__ void forward_node(const NodeDev& nd, const int32_t* __restrict__ rows,
                                             const float* __restrict__ blocks, float* __restrict__ y,
                                             float* __restrict__ z, float* smem) {
  const uint64_t pol = l2_policy(nd.l2_keep);
  float (*f)[D] = reinterpret_cast<float (*)[D]>(smem);    // [kNarrowCols][D]
  float* red = smem + kNarrowCols * D;                     // [D][S][ld]
  const int ntot = nd.ncol + nd.nrow;
  const int G = nd.ld >> 2;
  const int S = kSolveThreads / G;
  const int g = threadIdx.x % G, j = threadIdx.x / G;
  const bool active = j < S;
  const float* B = blocks + nd.blk_off + 4 * g;
  // columns j, j + S, ..., j + 7S are in flight while f is staged
  float4 b[8];
#pragma unroll
  for (int u = 0; u < 8; ++u)
    b[u] = (active && j + u * S < nd.ncol) ? ldg_stream(B + (int64_t)(j + u * S) * nd.ld, pol) : make_float4(0.f, 0.f, 0.f, 0.f);
  for (int q = threadIdx.x; q < nd.ncol * D; q += kSolveThreads) {
    const int c = q / D, k = q - c * D;
    f[c][k] = __ldcg(y + (int64_t)(nd.col0 + c) * D + k);
  }
  __syncthreads();
  if (active) {
    float acc[4][D];
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int k = 0; k < D; ++k) acc[q][k] = 0.f;
#pragma unroll
    for (int u = 0; u < 8; ++u)
      if (j + u * S < nd.ncol) {
#pragma unroll
        for (int k = 0; k < D; ++k) {
          const float fv = f[j + u * S][k];
          acc[0][k] = fmaf(b[u].x, fv, acc[0][k]);
          acc[1][k] = fmaf(b[u].y, fv, acc[1][k]);
          acc[2][k] = fmaf(b[u].z, fv, acc[2][k]);
          acc[3][k] = fmaf(b[u].w, fv, acc[3][k]);
        }
      }
    int c = j + 8 * S;
    for (; c + 7 * S < nd.ncol; c += 8 * S) {
#pragma unroll
      for (int u = 0; u < 8; ++u) b[u] = ldg_stream(B + (int64_t)(c + u * S) * nd.ld, pol);
#pragma unroll
      for (int u = 0; u < 8; ++u)
#pragma unroll
        for (int k = 0; k < D; ++k) {
          const float fv = f[c + u * S][k];
          acc[0][k] = fmaf(b[u].x, fv, acc[0][k]);
          acc[1][k] = fmaf(b[u].y, fv, acc[1][k]);
          acc[2][k] = fmaf(b[u].z, fv, acc[2][k]);
          acc[3][k] = fmaf(b[u].w, fv, acc[3][k]);
        }
    }
    for (; c < nd.ncol; c += S) {
      const float4 bv = ldg_stream(B + (int64_t)c * nd.ld, pol);
#pragma unroll
      for (int k = 0; k < D; ++k) {
        const float fv = f[c][k];
        acc[0][k] = fmaf(bv.x, fv, acc[0][k]);
        acc[1][k] = fmaf(bv.y, fv, acc[1][k]);
        acc[2][k] = fmaf(bv.z, fv, acc[2][k]);
        acc[3][k] = fmaf(bv.w, fv, acc[3][k]);
      }
    }
#pragma unroll
    for (int k = 0; k < D; ++k)
      *reinterpret_cast<float4*>(red + (k * S + j) * nd.ld + 4 * g) =
          make_float4(acc[0][k], acc[1][k], acc[2][k], acc[3][k]);
  }
  __syncthreads();
  for (int r = threadIdx.x; r < ntot; r += kSolveThreads) {
    float s[D];
#pragma unroll
    for (int k = 0; k < D; ++k) {
      float a = 0.f;
      for (int jj = 0; jj < S; ++jj) a += red[(k * S + jj) * nd.ld + r];
      s[k] = a;
    }
    if (r < nd.ncol) {
#pragma unroll
      for (int k = 0; k < D; ++k) z[(int64_t)(nd.col0 + r) * D + k] = s[k];
    } else {
      const int rr = __ldg(rows + nd.row_off + (r - nd.ncol));
#pragma unroll
      for (int k = 0; k < D; ++k) atomicAdd(y + (int64_t)rr * D + k, -s[k]);
    }
  }
}

// v = [z_s ; -x at the structure rows] for rows [r0, r0 + nr) of a node into
// dst[k * dst_ld + r]: every thread first issues the index loads of all its rows,
// then all their z / x loads, so staging costs two load latencies, not two per row.
template <int D>
__device__ __forceinline__ void stage_v(const NodeDev& nd, int r0, int nr, const int32_t* __restrict__ rows,
                                        const float* __restrict__ z, const float* __restrict__ x, float* dst,
                                        int dst_ld) {
  constexpr int kIt = (kBwdRows > kNodeMaxLd ? kBwdRows : kNodeMaxLd) / kSolveThreads;
  const int ntot = nd.ncol + nd.nrow;
  int src[kIt];
  bool from_z[kIt];
#pragma unroll
  for (int u = 0; u < kIt; ++u) {
    const int r = threadIdx.x + u * kSolveThreads;
    const int row = r0 + r;
    src[u] = -1;
    from_z[u] = false;
    if (r < nr) {
      if (row < nd.ncol) {
        src[u] = nd.col0 + row;
        from_z[u] = true;
      } else if (row < ntot) {
        src[u] = __ldg(rows + nd.row_off + (row - nd.ncol));
      }
    }
  }
  float v[kIt][D];
#pragma unroll
  for (int u = 0; u < kIt; ++u)
#pragma unroll
    for (int k = 0; k < D; ++k)
      v[u][k] = src[u] < 0 ? 0.f
                           : (from_z[u] ? __ldcg(z + (int64_t)src[u] * D + k) : -__ldcg(x + (int64_t)src[u] * D + k));
#pragma unroll
  for (int u = 0; u < kIt; ++u) {
    const int r = threadIdx.x + u * kSolveThreads;
    if (r < nr) {
#pragma unroll
      for (int k = 0; k < D; ++k) dst[k * dst_ld + r] = v[u][k];
    }
  }
}

// Backward wide task (node, r0, c0): output columns [c0, c0+32) of x_s against rows
// [r0, r0+1024) of B_s, v = [z_s ; -x at the structure rows] staged in shared
// memory.  Warp w owns columns c0+4w .. c0+4w+3; each lane reads 4 rows of each
// of them per step; the 4 column dot products are reduced across the warp.
template <int D>
__device__ __forceinline__ void backward_wide(const Task& t, const NodeDev& nd, const int32_t* __restrict__ rows,
                                              const float* __restrict__ blocks, const float* __restrict__ z,
                                              float* __restrict__ x, float* smem) {
  const uint64_t pol = l2_policy(nd.l2_keep);
  float (*vs)[kBwdRows] = reinterpret_cast<float (*)[kBwdRows]>(smem);   // [D][1024]
  const int nr = min(t.kind, nd.ld - t.r0);     // rows of this task: a multiple of 4
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int j0 = t.c0 + 4 * warp;
  const int ncw = max(0, min(4, nd.ncol - j0));
  const float* B = blocks + nd.blk_off + (int64_t)min(j0, nd.ncol - 1) * nd.ld + t.r0;
  // rows above the diagonal of inv(L_ss) are stored zeros: start at the first
  // 4-row group that can be nonzero for this warp's first column
  const int rs = max(0, (j0 - t.r0) & ~3);
  // the first row step is in flight while v is staged
  const int ra = rs + 4 * lane;
  float4 pa[4];
#pragma unroll
  for (int q = 0; q < 4; ++q)
    pa[q] = (q < ncw && ra < nr) ? ldg_stream(B + (int64_t)q * nd.ld + ra, pol) : make_float4(0.f, 0.f, 0.f, 0.f);
  stage_v<D>(nd, t.r0, nr, rows, z, x, &vs[0][0], kBwdRows);
  __syncthreads();
  if (ncw == 0) return;
  float acc[4][D];
#pragma unroll
  for (int q = 0; q < 4; ++q)
#pragma unroll
    for (int k = 0; k < D; ++k) acc[q][k] = 0.f;
  auto step = [&](const float4 (&bq)[4], int r) {
#pragma unroll
    for (int k = 0; k < D; ++k) {
      const float4 v = *reinterpret_cast<const float4*>(&vs[k][r]);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        acc[q][k] = fmaf(bq[q].x, v.x, acc[q][k]);
        acc[q][k] = fmaf(bq[q].y, v.y, acc[q][k]);
        acc[q][k] = fmaf(bq[q].z, v.z, acc[q][k]);
        acc[q][k] = fmaf(bq[q].w, v.w, acc[q][k]);
      }
    }
  };
  if (ra < nr) step(pa, ra);
#pragma unroll 2
  for (int r = ra + 128; r < nr; r += 128) {
    float4 bq[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) bq[q] = (q < ncw) ? ldg_stream(B + (int64_t)q * nd.ld + r, pol) : make_float4(0.f, 0.f, 0.f, 0.f);
    step(bq, r);
  }
#pragma unroll
  for (int q = 0; q < 4; ++q)
#pragma unroll
    for (int k = 0; k < D; ++k) {
      float a = acc[q][k];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
      acc[q][k] = a;
    }
  if (lane == 0) {
    for (int q = 0; q < ncw; ++q)
#pragma unroll
      for (int k = 0; k < D; ++k) atomicAdd(x + (int64_t)(nd.col0 + j0 + q) * D + k, acc[q][k]);
  }
}

// Node task of the backward pass: a whole small node on one block.  v is staged
// in shared memory; each warp takes 4 columns at a time with 8 lanes per column,
// so a warp-wide load reads 128 contiguous bytes of each of 4 columns, and the
// 8 partial dot products of a column meet by shuffles.  Rows above the diagonal
// of inv(L_ss) are stored zeros: a column j starts at row 32 floor(j / 32).
template <int D>
__device__ __forceinline__ void backward_node(const NodeDev& nd, const int32_t* __restrict__ rows,
                                              const float* __restrict__ blocks, const float* __restrict__ z,
                                              float* __restrict__ x, float* smem) {
  const uint64_t pol = l2_policy(nd.l2_keep);
  const int ld = nd.ld;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int cg = lane >> 3, rl = lane & 7;
  // the first 4 row steps of this lane's first column are in flight while v is staged
  float4 pre[4];
  {
    const int j = 4 * warp + cg;
    const float* B = blocks + nd.blk_off + (int64_t)min(j, nd.ncol - 1) * ld;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int r = 4 * rl + 32 * u;
      pre[u] = (j < nd.ncol && r < ld) ? ldg_stream(B + r, pol) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
  }
  stage_v<D>(nd, 0, ld, rows, z, x, smem, ld);
  __syncthreads();
  for (int j0 = 4 * warp; j0 < nd.ncol; j0 += 4 * kSolveWarps) {
    const int j = j0 + cg;
    float acc[D];
#pragma unroll
    for (int k = 0; k < D; ++k) acc[k] = 0.f;
    if (j < nd.ncol) {
      const float* B = blocks + nd.blk_off + (int64_t)j * ld;
      int r = (j0 & ~31) + 4 * rl;
      if (j0 < 32) {   // the prefetched rows 4 rl + 32 u, u < 4
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int rr = 4 * rl + 32 * u;
          if (rr < ld) {
#pragma unroll
            for (int k = 0; k < D; ++k) {
              const float4 v = *reinterpret_cast<const float4*>(smem + k * ld + rr);
              acc[k] = fmaf(pre[u].x, v.x, acc[k]);
              acc[k] = fmaf(pre[u].y, v.y, acc[k]);
              acc[k] = fmaf(pre[u].z, v.z, acc[k]);
              acc[k] = fmaf(pre[u].w, v.w, acc[k]);
            }
          }
        }
        r += 128;
      }
#pragma unroll 4
      for (; r < ld; r += 32) {
        const float4 b = ldg_stream(B + r, pol);
#pragma unroll
        for (int k = 0; k < D; ++k) {
          const float4 v = *reinterpret_cast<const float4*>(smem + k * ld + r);
          acc[k] = fmaf(b.x, v.x, acc[k]);
          acc[k] = fmaf(b.y, v.y, acc[k]);
          acc[k] = fmaf(b.z, v.z, acc[k]);
          acc[k] = fmaf(b.w, v.w, acc[k]);
        }
      }
    }
#pragma unroll
    for (int k = 0; k < D; ++k) {
      float a = acc[k];
      a += __shfl_xor_sync(0xffffffffu, a, 4);
      a += __shfl_xor_sync(0xffffffffu, a, 2);
      a += __shfl_xor_sync(0xffffffffu, a, 1);
      acc[k] = a;
    }
    if (rl == 0 && j < nd.ncol) {
#pragma unroll
      for (int k = 0; k < D; ++k) x[(int64_t)(nd.col0 + j) * D + k] = acc[k];
    }
  }
}

// shared memory of one solve block (floats): the larger of the wide and node tasks
template <int D>
struct SolveSmem {
  static constexpr int kFwd = (kFwdCols + kSolveWarps * kFwdRows) * D > (kNarrowCols + kNodeMaxLd) * D
                                  ? (kFwdCols + kSolveWarps * kFwdRows) * D : (kNarrowCols + kNodeMaxLd) * D;
  static constexpr int kBwd = D * (kBwdRows > kNodeMaxLd ? kBwdRows : kNodeMaxLd);
};

template <int D>
__device__ __forceinline__ void forward_task(const Task& t, const NodeDev& nd, const int32_t* __restrict__ rows,
                                             const float* __restrict__ blocks, float* __restrict__ y,
                                             float* __restrict__ z, float* smem) {
  if (t.kind != 1) forward_wide<D>(t, nd, rows, blocks, y, z, smem);
  else forward_node<D>(nd, rows, blocks, y, z, smem);
}

template <int D>
__device__ __forceinline__ void backward_task(const Task& t, const NodeDev& nd, const int32_t* __restrict__ rows,
                                              const float* __restrict__ blocks, const float* __restrict__ z,
                                              float* __restrict__ x, float* smem) {
  if (t.kind != 1) backward_wide<D>(t, nd, rows, blocks, z, x, smem);
  else backward_node<D>(nd, rows, blocks, z, x, smem);
}

// level-synchronous schedule: one launch per level, one task per block
template <int D>
__global__ void __launch_bounds__(kSolveThreads, kSolveMinBlocks) k_forward(const Task* __restrict__ tasks,
                                                 const int32_t* __restrict__ rows, const float* __restrict__ blocks,
                                                 float* __restrict__ y, float* __restrict__ z) {
  __shared__ __align__(16) float smem[SolveSmem<D>::kFwd];
  const Task& t = tasks[blockIdx.x];
  forward_task<D>(t, t.nd, rows, blocks, y, z, smem);
}

template <int D>
__global__ void __launch_bounds__(kSolveThreads, kSolveMinBlocks) k_backward(const Task* __restrict__ tasks,
                                                  const int32_t* __restrict__ rows, const float* __restrict__ blocks,
                                                  const float* __restrict__ z, float* __restrict__ x) {
  __shared__ __align__(16) float smem[SolveSmem<D>::kBwd];
  const Task& t = tasks[blockIdx.x];
  backward_task<D>(t, t.nd, rows, blocks, z, x, smem);
}

// ---------------------------------------------------------------------------
// Dynamic schedule: one launch per pass over a ready queue.  The queue starts
// with the tasks of the nodes that depend on nothing (forward: the nodes with no
// descendant that has tasks; backward: the roots).  Blocks claim queue slots in
// order and run the task found there.  Forward, every finished task decrements
// the pending count of the node waiting on its node (the count starts at the
// number of tasks it waits on); backward, the task that completes its node
// releases the nodes waiting on it, each of which waits on that node alone.  A
// released node's tasks are appended to the queue, so a block only ever waits
// for a slot to be filled, never for a particular node, and no block holds a
// task whose inputs are incomplete.  What a completion releases (the push
// record of the node) is fetched asynchronously when the task starts, so the
// completion itself costs a fence, one counter atomic and, when something is
// released, one queue reservation.  Every slot is filled exactly once (each
// node becomes ready once), so the waits end; each is still bounded and sets
// err_flag instead of spinning on.
// ---------------------------------------------------------------------------
struct DynView {
  DynPass P;
  const NodeDev* sub;   // merged subtrees' nodes
  const int32_t* rows;
  const float* blocks;
  float* y;
  float* z;
  float* x;
  int32_t* err_flag;
  long long spin_limit;   // polls of an empty slot before the wait gives up
};

__device__ __forceinline__ int ld_acquire(const int32_t* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_relaxed(int32_t* p, int v) {
  asm volatile("st.relaxed.gpu.global.s32 [%0], %1;" :: "l"(p), "r"(v) : "memory");
}

// 16-byte asynchronous global -> shared copy (completes by cp_async_wait_all)
__device__ __forceinline__ void cp_async16(void* dst_smem, const void* src) {
  const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(dst_smem));
  asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" :: "r"(d), "l"(src) : "memory");
}

__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;" ::: "memory");
}

template <int D, bool FWD>
__global__ void __launch_bounds__(kSolveThreads, kSolveMinBlocks) k_solve_dynamic(DynView V) {
  constexpr int kRec = FWD ? 1 : 1 + kPushKids;   // int4 entries of a push record
  __shared__ __align__(16) float smem[FWD ? SolveSmem<D>::kFwd : SolveSmem<D>::kBwd];
  __shared__ __align__(16) int4 rec_s[kRec];
  __shared__ __align__(16) Task task_s;   // the task to run next
  __shared__ __align__(16) NodeDev sub_s[kSubtreeMaxNodes];   // a merged subtree's nodes
  __shared__ int item_s, slot_s, next_s, base_s;
  const DynPass& P = V.P;
  if (threadIdx.x == 0) {
    slot_s = atomicAdd(P.ctr, 1);
    next_s = -1;
  }
  for (;;) {
    if (threadIdx.x == 0) {
      int t = -1;
      const int h = slot_s;
      if (h < P.n_tasks) {
        t = next_s;   // >= 0: the slot was already filled and task_s holds its task
        if (t < 0) {
          long long it = 0;
          while ((t = ld_acquire(P.queue + h)) < 0) {
            if (++it > V.spin_limit || ld_acquire(V.err_flag) != 0) {
              atomicExch(V.err_flag, 1);
              t = -1;
              break;
            }
            __nanosleep(64);
          }
          if (t >= 0) task_s = P.tasks[t];
        }
      }
      item_s = t;
    }
    __syncthreads();
    const int ti = item_s;
    if (ti < 0) break;
    const Task& t = task_s;   // read in place: task_s is rewritten only after the completion
    if (threadIdx.x == 0) {
#pragma unroll
      for (int e = 0; e < kRec; ++e) cp_async16(&rec_s[e], P.push + (int64_t)t.node * kRec + e);
    }
    const NodeDev& nd = task_s.nd;
    if (t.kind == 0) {
      // a merged bottom subtree: its nodes in order (forward children first,
      // backward parents first), each on the whole block; a barrier makes one
      // node's results visible to the next
      const int n_sub = t.c0;
      for (int i = threadIdx.x; i < n_sub * (int)(sizeof(NodeDev) / 4); i += kSolveThreads)
        reinterpret_cast<int32_t*>(sub_s)[i] = reinterpret_cast<const int32_t*>(V.sub + t.r0)[i];
      __syncthreads();
      for (int q = 0; q < n_sub; ++q) {
        if constexpr (FWD) forward_node<D>(sub_s[q], V.rows, V.blocks, V.y, V.z, smem);
        else backward_node<D>(sub_s[n_sub - 1 - q], V.rows, V.blocks, V.z, V.x, smem);
        __syncthreads();
      }
    } else {
      if constexpr (FWD) forward_task<D>(t, nd, V.rows, V.blocks, V.y, V.z, smem);
      else backward_task<D>(t, nd, V.rows, V.blocks, V.z, V.x, smem);
      __syncthreads();
    }
    // the next slot is claimed, and read once, while the completion below is
    // worked out
    if (threadIdx.x == 32) {
      const int h = atomicAdd(P.ctr, 1);
      slot_s = h;
      next_s = h < P.n_tasks ? ld_acquire(P.queue + h) : -1;
    }
    // completion: the block's writes are released by one fence after the barrier
    // (fences are cumulative); a release reserves queue room for everything it
    // releases, and the whole block then writes the released tasks' ids
    if (threadIdx.x == 0) {
      cp_async_wait_all();
      const int4 r = rec_s[0];
      int base = -1;
      __threadfence();
      if constexpr (FWD) {
        if (r.x >= 0 && atomicSub(P.pending + r.x, 1) == 1) base = atomicAdd(P.ctr + 1, r.z);
      } else if (r.z > 0 && (t.kind <= 1 || atomicAdd(P.done + t.node, 1) == r.w - 1)) {
        base = atomicAdd(P.ctr + 1, r.z);
      }
      if (base >= 0) __threadfence();   // acquire the other tasks' releases
      base_s = base;
    }
    __syncthreads();
    const int base = base_s;
    if (base >= 0) {
      __threadfence();
      const int4 r = rec_s[0];
      if constexpr (FWD) {
        for (int i = threadIdx.x; i < r.z; i += kSolveThreads) st_relaxed(P.queue + base + i, r.y + i);
      } else {
        for (int k = r.x; k < r.y; ++k) {   // block-uniform
          const int j = k - r.x;
          const int4 e = j < kPushKids ? rec_s[1 + j] : P.kids[k];
          for (int i = threadIdx.x; i < e.y; i += kSolveThreads) st_relaxed(P.queue + base + e.z + i, e.x + i);
        }
      }
    }
    // the next task, when its slot was already filled, is fetched before the
    // block goes round
    constexpr int kTaskVecs = (int)(sizeof(Task) / sizeof(int4));
    if (threadIdx.x >= 32 && threadIdx.x < 32 + kTaskVecs) {
      const int nt = next_s;
      if (nt >= 0) reinterpret_cast<int4*>(&task_s)[threadIdx.x - 32] = reinterpret_cast<const int4*>(P.tasks + nt)[threadIdx.x - 32];
    }
    __syncthreads();   // item_s, slot_s, next_s, task_s, base_s and rec_s are reused
  }
}

// ---------------------------------------------------------------------------
// Pipelined schedule (solve_schedule 2).  The same ready queue, task lists and
// release protocol as the dynamic schedule above, but each block is one producer
// warp and kPipeConsumers consumer warps.  The producer claims the next queue slot
// as soon as one of kPipeSlots task entries is free, copies the task record, its
// node's push record and a merged subtree's node list into shared memory, and
// streams the task's factor data with 1D bulk copies (cp.async.bulk, completion
// counted in transaction bytes on an mbarrier) into a ring of kPipeStages chunks
// of kPipeChunkFloats floats.  The consumers stage the right-hand side, compute
// from the ring, release each chunk, and do the reduction, scatter and completion
// of the dynamic schedule.  The bytes in flight are set by the ring (64 KB per
// block), not by registers, and the next task's factor streams while the current
// one reduces and completes.  A producer claims a task only after it has issued
// every chunk of the previous one, so the consumers never wait on a task that
// depends on the producer.  Every wait is bounded: a producer that gives up on a
// queue slot sets err_flag and ends the block's task stream; a consumer wait that
// runs out sets err_flag and the consumers skip the remaining waits; the producer
// waits (bounded) for its own copies before it exits.
//
// Chunks (computed identically on both sides):
//   forward wide   : 32 columns of the task's 128-row band, one copy per column,
//                    stored 128 floats apart; rows above the diagonal of
//                    inv(L_ss) (row < column, stored zeros) start the copy at the
//                    column's 4-row group instead of the band's first row;
//   backward wide  : one 128-row band of the task's 32 columns, laid out the same;
//                    bands wholly above the diagonal of the first column are skipped;
//   node (whole supernode, also inside a merged subtree): floor(kPipeChunkFloats /
//                    ld) whole columns, contiguous in B_s, one copy.
// ---------------------------------------------------------------------------
constexpr int kPipeConsumers = kSolveWarps;                 // consumer warps (the task mappings assume 8)
constexpr int kPipeThreads = 32 * (kPipeConsumers + 1);     // plus one producer warp
constexpr int kPipeStages = 4;
constexpr int kPipeChunkFloats = 4096;                      // 16 KB per chunk
constexpr int kPipeSlots = 2;                               // task entries in flight
constexpr int kPipeEnd = -1000;                             // task kind that ends the stream
static_assert(kPipeConsumers * 32 == kSolveThreads, "consumers take the roles of a solve block");

template <int D>
struct PipeSmem {
  float ring[kPipeStages][kPipeChunkFloats];
  float rhs[D * 1024];      // f ([cols][D]) forward, v ([D][rows]) backward
  float red[D * 1024];      // forward partial sums
  Task task[kPipeSlots];
  int4 rec[kPipeSlots][1 + kPushKids];
  NodeDev sub[kPipeSlots][kSubtreeMaxNodes];
  unsigned long long full[kPipeStages], empty[kPipeStages], tfull[kPipeSlots], tempty[kPipeSlots];
  int base_s, stop_s;
  volatile int err_s;   // a consumer wait ran out: later waits are skipped
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(unsigned long long* b, int count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_u32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(unsigned long long* b) {
  asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" :: "r"(smem_u32(b)) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* b, uint32_t bytes) {
  asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}"
               :: "r"(smem_u32(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_test(unsigned long long* b, uint32_t parity) {
  uint32_t ok;
  asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
               : "=r"(ok) : "r"(smem_u32(b)), "r"(parity) : "memory");
  return ok != 0;
}
// bounded wait for the phase of the given parity; false when `limit` polls ran out
// or *stop became nonzero
__device__ __forceinline__ bool mbar_wait(unsigned long long* b, uint32_t parity, long long limit,
                                          const volatile int* stop) {
  long long it = 0;
  while (!mbar_test(b, parity)) {
    if (++it > limit || *stop) return false;
    if (it > 64) __nanosleep(32);
  }
  return true;
}
__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, uint32_t bytes, unsigned long long* bar,
                                              uint64_t pol) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;"
               :: "r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(pol) : "memory");
}
__device__ __forceinline__ void consumer_sync() { asm volatile("bar.sync 1, %0;" :: "n"(kSolveThreads) : "memory"); }

// chunks of a whole node and of the wide tasks (see above)
__device__ __forceinline__ int node_cpc(const NodeDev& nd) { return max(1, kPipeChunkFloats / nd.ld); }
__device__ __forceinline__ int node_chunks(const NodeDev& nd) {
  const int c = node_cpc(nd);
  return (nd.ncol + c - 1) / c;
}
__device__ __forceinline__ int fwd_wide_cols(const Task& t) { return min(t.kind, t.nd.ncol - t.c0); }
__device__ __forceinline__ int bwd_wide_rows(const Task& t) { return min(t.kind, t.nd.ld - t.r0); }
__device__ __forceinline__ int bwd_first_band(const Task& t) { return max(0, (t.c0 & ~3) - t.r0) / 128; }

__device__ __forceinline__ const float* blocks_at(const DynView& V, const NodeDev& nd, int col, int row) {
  return V.blocks + nd.blk_off + (int64_t)col * nd.ld + row;
}

// the bytes of column `col` of B_s from row max(row0, col & ~3) to row0 + nrows
// (rows above the diagonal of inv(L_ss) are not copied); 0 if none
__device__ __forceinline__ uint32_t band_copy(const NodeDev& nd, int col, int row0, int nrows, int& start) {
  start = max(row0, col & ~3);
  return start < row0 + nrows ? (uint32_t)(row0 + nrows - start) * 4u : 0u;
}

template <int D, bool FWD>
__device__ void pipe_producer(PipeSmem<D>& S, const DynView& V) {
  const int lane = threadIdx.x & 31;
  const DynPass& P = V.P;
  constexpr int kRec = FWD ? 1 : 1 + kPushKids;
  const long long wait_limit = 4 * V.spin_limit + (1 << 16);
  long long last_k[kPipeStages];
#pragma unroll
  for (int s = 0; s < kPipeStages; ++s) last_k[s] = -1;
  long long k = 0;   // chunks issued so far
  bool ok = true;
  // one chunk into the next stage: `bytes` of this lane's copy from src to the
  // stage at float offset dst_off (0 bytes: no copy)
  auto acquire_stage = [&]() -> int {
    const int s = (int)(k % kPipeStages);
    if (k >= kPipeStages) {
      bool w = true;
      if (lane == 0) w = mbar_wait(&S.empty[s], (uint32_t)(((k / kPipeStages) - 1) & 1), wait_limit, &S.err_s);
      w = __shfl_sync(0xffffffffu, w, 0);
      if (!w) return -1;
    }
    return s;
  };
  auto commit = [&](int s, const float* src, int dst_off, uint32_t bytes, uint64_t pol) {
    uint32_t tot = bytes;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) tot += __shfl_xor_sync(0xffffffffu, tot, o);
    if (lane == 0) mbar_expect_tx(&S.full[s], tot);
    __syncwarp();
    if (bytes) bulk_copy_g2s(&S.ring[s][dst_off], src, bytes, &S.full[s], pol);
    last_k[s] = k;
    ++k;
  };
  auto node_stream = [&](const NodeDev& nd) -> bool {
    const uint64_t pol = l2_policy(nd.l2_keep);
    const int cpc = node_cpc(nd), nq = node_chunks(nd);
    for (int q = 0; q < nq; ++q) {
      const int s = acquire_stage();
      if (s < 0) return false;
      const int nc = min(cpc, nd.ncol - q * cpc);
      commit(s, blocks_at(V, nd, q * cpc, 0), 0, lane == 0 ? (uint32_t)nc * nd.ld * 4u : 0u, pol);
    }
    return true;
  };
  for (int n = 0; ok; ++n) {
    const int e = n % kPipeSlots;
    if (n >= kPipeSlots) {
      bool w = true;
      if (lane == 0) w = mbar_wait(&S.tempty[e], (uint32_t)(((n / kPipeSlots) - 1) & 1), wait_limit, &S.err_s);
      if (!__shfl_sync(0xffffffffu, w, 0)) {
        ok = false;
        break;
      }
    }
    int t = -1;
    if (lane == 0) {
      const int h = atomicAdd(P.ctr, 1);
      if (h < P.n_tasks) {
        long long it = 0;
        while ((t = ld_acquire(P.queue + h)) < 0) {
          if (++it > V.spin_limit || ld_acquire(V.err_flag) != 0) {
            atomicExch(V.err_flag, 1);
            t = -1;
            break;
          }
          __nanosleep(64);
        }
      }
    }
    t = __shfl_sync(0xffffffffu, t, 0);
    if (t < 0) {
      if (lane == 0) {
        S.task[e].kind = kPipeEnd;
        __threadfence_block();
        mbar_arrive(&S.tfull[e]);
      }
      break;
    }
    // the task, its node's push record and a merged subtree's nodes
    if (lane < 4) reinterpret_cast<int4*>(&S.task[e])[lane] = __ldg(reinterpret_cast<const int4*>(P.tasks + t) + lane);
    __syncwarp();
    const Task& tk = S.task[e];
    if (lane < kRec) S.rec[e][lane] = __ldg(P.push + (int64_t)tk.node * kRec + lane);
    if (tk.kind == 0) {
      constexpr int kw = (int)(sizeof(NodeDev) / 4);
      for (int i = lane; i < tk.c0 * kw; i += 32)
        reinterpret_cast<int32_t*>(S.sub[e])[i] = __ldg(reinterpret_cast<const int32_t*>(V.sub + tk.r0) + i);
    }
    __syncwarp();
    if (lane == 0) {
      __threadfence_block();
      mbar_arrive(&S.tfull[e]);
    }
    // the factor chunks, in the order the consumers take them
    if (tk.kind == 0) {
      for (int i = 0; i < tk.c0 && ok; ++i) ok = node_stream(S.sub[e][FWD ? i : tk.c0 - 1 - i]);
    } else if (tk.kind == 1) {
      ok = node_stream(tk.nd);
    } else if (FWD) {
      const NodeDev& nd = tk.nd;
      const uint64_t pol = l2_policy(nd.l2_keep);
      const int nc = fwd_wide_cols(tk), R = min(kFwdRows, nd.ld - tk.r0);
      for (int q = 0; q * 32 < nc && ok; ++q) {
        const int s = acquire_stage();
        if (s < 0) { ok = false; break; }
        const int col = tk.c0 + 32 * q + lane;
        int start = 0;
        const uint32_t bytes = (32 * q + lane < nc) ? band_copy(nd, col, tk.r0, R, start) : 0u;
        commit(s, bytes ? blocks_at(V, nd, col, start) : nullptr, lane * kFwdRows + (start - tk.r0), bytes, pol);
      }
    } else {
      const NodeDev& nd = tk.nd;
      const uint64_t pol = l2_policy(nd.l2_keep);
      const int nr = bwd_wide_rows(tk), ncw = min(32, nd.ncol - tk.c0);
      for (int b = bwd_first_band(tk); b * 128 < nr && ok; ++b) {
        const int s = acquire_stage();
        if (s < 0) { ok = false; break; }
        const int rb = tk.r0 + 128 * b, Rb = min(128, nr - 128 * b);
        const int col = tk.c0 + lane;
        int start = 0;
        const uint32_t bytes = lane < ncw ? band_copy(nd, col, rb, Rb, start) : 0u;
        commit(s, bytes ? blocks_at(V, nd, col, start) : nullptr, lane * 128 + (start - rb), bytes, pol);
      }
    }
  }
  if (!ok) atomicExch(V.err_flag, 1);
  // every copy this warp issued has landed before the block may exit
  if (lane == 0) {
    const long long drain_limit = 4 * V.spin_limit + (1 << 16);
    volatile int never = 0;
#pragma unroll
    for (int s = 0; s < kPipeStages; ++s)
      if (last_k[s] >= 0) mbar_wait(&S.full[s], (uint32_t)((last_k[s] / kPipeStages) & 1), drain_limit, &never);
  }
}

template <int D, bool FWD>
__device__ void pipe_consumer(PipeSmem<D>& S, const DynView& V) {
  const DynPass& P = V.P;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long wait_limit = 4 * V.spin_limit + (1 << 16);
  const long long task_limit = 64 * V.spin_limit + (1 << 20);
  long long k = 0;   // chunks consumed so far
  // chunk k is in stage k % kPipeStages; a wait that runs out marks the block
  // failed (the remaining waits are skipped, the results are invalid)
  auto take = [&]() -> int {
    const int s = (int)(k % kPipeStages);
    if (!S.err_s && !mbar_wait(&S.full[s], (uint32_t)((k / kPipeStages) & 1), wait_limit, &S.err_s)) {
      S.err_s = 1;
      atomicExch(V.err_flag, 1);
    }
    return s;
  };
  auto release = [&](int s) {
    __syncwarp();
    if (lane == 0) mbar_arrive(&S.empty[s]);
    ++k;
  };

  // forward, whole node: z_s = inv(L_ss) y_s, y_r -= (L_rs inv(L_ss)) y_s
  auto fwd_node = [&](const NodeDev& nd) {
    float (*f)[D] = reinterpret_cast<float (*)[D]>(S.rhs);
    const int ntot = nd.ncol + nd.nrow;
    const int G = nd.ld >> 2, Sl = kSolveThreads / G;
    const int g = threadIdx.x % G, j = threadIdx.x / G;
    const bool active = j < Sl;
    for (int q = threadIdx.x; q < nd.ncol * D; q += kSolveThreads) {
      const int c = q / D, kk = q - c * D;
      f[c][kk] = __ldcg(V.y + (int64_t)(nd.col0 + c) * D + kk);
    }
    consumer_sync();
    float acc[4][D];
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int kk = 0; kk < D; ++kk) acc[q][kk] = 0.f;
    const int cpc = node_cpc(nd), nq = node_chunks(nd);
    for (int q = 0; q < nq; ++q) {
      const int s = take();
      if (active) {
        const int cb = q * cpc, ce = min(nd.ncol, cb + cpc);
        for (int c = cb + j; c < ce; c += Sl) {
          const float4 bv = *reinterpret_cast<const float4*>(&S.ring[s][(c - cb) * nd.ld + 4 * g]);
#pragma unroll
          for (int kk = 0; kk < D; ++kk) {
            const float fv = f[c][kk];
            acc[0][kk] = fmaf(bv.x, fv, acc[0][kk]);
            acc[1][kk] = fmaf(bv.y, fv, acc[1][kk]);
            acc[2][kk] = fmaf(bv.z, fv, acc[2][kk]);
            acc[3][kk] = fmaf(bv.w, fv, acc[3][kk]);
          }
        }
      }
      release(s);
    }
    if (active) {
#pragma unroll
      for (int kk = 0; kk < D; ++kk)
        *reinterpret_cast<float4*>(S.red + (kk * Sl + j) * nd.ld + 4 * g) =
            make_float4(acc[0][kk], acc[1][kk], acc[2][kk], acc[3][kk]);
    }
    consumer_sync();
    for (int r = threadIdx.x; r < ntot; r += kSolveThreads) {
      float sm[D];
#pragma unroll
      for (int kk = 0; kk < D; ++kk) {
        float a = 0.f;
        for (int jj = 0; jj < Sl; ++jj) a += S.red[(kk * Sl + jj) * nd.ld + r];
        sm[kk] = a;
      }
      if (r < nd.ncol) {
#pragma unroll
        for (int kk = 0; kk < D; ++kk) V.z[(int64_t)(nd.col0 + r) * D + kk] = sm[kk];
      } else {
        const int rr = __ldg(V.rows + nd.row_off + (r - nd.ncol));
#pragma unroll
        for (int kk = 0; kk < D; ++kk) atomicAdd(V.y + (int64_t)rr * D + kk, -sm[kk]);
      }
    }
  };

  // backward, whole node: x_s = inv(L_ss)^T z_s - (L_rs inv(L_ss))^T x_r
  auto bwd_node = [&](const NodeDev& nd) {
    const int ld = nd.ld;
    stage_v<D>(nd, 0, ld, V.rows, V.z, V.x, S.rhs, ld);
    consumer_sync();
    const int cg = lane >> 3, rl = lane & 7;
    const int cpc = node_cpc(nd), nq = node_chunks(nd);
    for (int q = 0; q < nq; ++q) {
      const int s = take();
      const int cb = q * cpc, ce = min(nd.ncol, cb + cpc);
      for (int jj = cb + 4 * warp; jj < ce; jj += 4 * kPipeConsumers) {   // warp-uniform
        const int j = jj + cg;
        float acc[D];
#pragma unroll
        for (int kk = 0; kk < D; ++kk) acc[kk] = 0.f;
        if (j < ce) {
          const float* Bc = &S.ring[s][(j - cb) * ld];
          for (int r = (j & ~31) + 4 * rl; r < ld; r += 32) {
            const float4 b = *reinterpret_cast<const float4*>(Bc + r);
#pragma unroll
            for (int kk = 0; kk < D; ++kk) {
              const float4 v = *reinterpret_cast<const float4*>(S.rhs + kk * ld + r);
              acc[kk] = fmaf(b.x, v.x, acc[kk]);
              acc[kk] = fmaf(b.y, v.y, acc[kk]);
              acc[kk] = fmaf(b.z, v.z, acc[kk]);
              acc[kk] = fmaf(b.w, v.w, acc[kk]);
            }
          }
        }
#pragma unroll
        for (int kk = 0; kk < D; ++kk) {
          float a = acc[kk];
          a += __shfl_xor_sync(0xffffffffu, a, 4);
          a += __shfl_xor_sync(0xffffffffu, a, 2);
          a += __shfl_xor_sync(0xffffffffu, a, 1);
          acc[kk] = a;
        }
        if (rl == 0 && j < ce) {
#pragma unroll
          for (int kk = 0; kk < D; ++kk) V.x[(int64_t)(nd.col0 + j) * D + kk] = acc[kk];
        }
      }
      release(s);
    }
  };

  // forward wide task: rows [r0, r0 + 128) of B_s times columns [c0, c0 + nc) of f
  auto fwd_wide = [&](const Task& t) {
    const NodeDev& nd = t.nd;
    const int nc = fwd_wide_cols(t), R = min(kFwdRows, nd.ld - t.r0), ntot = nd.ncol + nd.nrow;
    float (*fs)[D] = reinterpret_cast<float (*)[D]>(S.rhs);
    for (int q = threadIdx.x; q < nc * D; q += kSolveThreads) {
      const int c = q / D, kk = q - c * D;
      fs[c][kk] = __ldcg(V.y + (int64_t)(nd.col0 + t.c0 + c) * D + kk);
    }
    consumer_sync();
    float acc[4][D];
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int kk = 0; kk < D; ++kk) acc[q][kk] = 0.f;
    const int r = 4 * lane;
    for (int q = 0; q * 32 < nc; ++q) {
      const int s = take();
      if (r < R) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int cl = 32 * q + 4 * warp + u;
          const int col = t.c0 + cl;
          if (cl < nc && t.r0 + r >= (col & ~3)) {
            const float4 bv = *reinterpret_cast<const float4*>(&S.ring[s][(4 * warp + u) * kFwdRows + r]);
#pragma unroll
            for (int kk = 0; kk < D; ++kk) {
              const float fv = fs[cl][kk];
              acc[0][kk] = fmaf(bv.x, fv, acc[0][kk]);
              acc[1][kk] = fmaf(bv.y, fv, acc[1][kk]);
              acc[2][kk] = fmaf(bv.z, fv, acc[2][kk]);
              acc[3][kk] = fmaf(bv.w, fv, acc[3][kk]);
            }
          }
        }
      }
      release(s);
    }
    float (*red)[kFwdRows][D] = reinterpret_cast<float (*)[kFwdRows][D]>(S.red);
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int kk = 0; kk < D; ++kk) red[warp][4 * lane + q][kk] = acc[q][kk];
    consumer_sync();
    if (threadIdx.x < kFwdRows) {
      const int row = t.r0 + threadIdx.x;
      if (row < ntot && !(row < nd.ncol && row < t.c0)) {
        float sm[D];
#pragma unroll
        for (int kk = 0; kk < D; ++kk) {
          float a = 0.f;
#pragma unroll
          for (int w = 0; w < kPipeConsumers; ++w) a += red[w][threadIdx.x][kk];
          sm[kk] = a;
        }
        if (row < nd.ncol) {
#pragma unroll
          for (int kk = 0; kk < D; ++kk) atomicAdd(V.z + (int64_t)(nd.col0 + row) * D + kk, sm[kk]);
        } else {
          const int rr = __ldg(V.rows + nd.row_off + (row - nd.ncol));
#pragma unroll
          for (int kk = 0; kk < D; ++kk) atomicAdd(V.y + (int64_t)rr * D + kk, -sm[kk]);
        }
      }
    }
  };

  // backward wide task: output columns [c0, c0 + 32) against rows [r0, r0 + nr)
  auto bwd_wide = [&](const Task& t) {
    const NodeDev& nd = t.nd;
    const int nr = bwd_wide_rows(t);
    float (*vs)[kBwdRows] = reinterpret_cast<float (*)[kBwdRows]>(S.rhs);
    stage_v<D>(nd, t.r0, nr, V.rows, V.z, V.x, &vs[0][0], kBwdRows);
    consumer_sync();
    const int j0 = t.c0 + 4 * warp;
    const int ncw = max(0, min(4, nd.ncol - j0));
    float acc[4][D];
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int kk = 0; kk < D; ++kk) acc[q][kk] = 0.f;
    const int r = 4 * lane;
    for (int b = bwd_first_band(t); b * 128 < nr; ++b) {
      const int s = take();
      const int rb = t.r0 + 128 * b, Rb = min(128, nr - 128 * b);
      if (r < Rb) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int col = j0 + u;
          if (u < ncw && rb + r >= (col & ~3)) {
            const float4 bv = *reinterpret_cast<const float4*>(&S.ring[s][(4 * warp + u) * 128 + r]);
#pragma unroll
            for (int kk = 0; kk < D; ++kk) {
              const float4 v = *reinterpret_cast<const float4*>(&vs[kk][rb - t.r0 + r]);
              acc[u][kk] = fmaf(bv.x, v.x, acc[u][kk]);
              acc[u][kk] = fmaf(bv.y, v.y, acc[u][kk]);
              acc[u][kk] = fmaf(bv.z, v.z, acc[u][kk]);
              acc[u][kk] = fmaf(bv.w, v.w, acc[u][kk]);
            }
          }
        }
      }
      release(s);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int kk = 0; kk < D; ++kk) {
        float a = acc[u][kk];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
        acc[u][kk] = a;
      }
    if (lane == 0) {
      for (int u = 0; u < ncw; ++u)
#pragma unroll
        for (int kk = 0; kk < D; ++kk) atomicAdd(V.x + (int64_t)(nd.col0 + j0 + u) * D + kk, acc[u][kk]);
    }
  };

  for (int n = 0;; ++n) {
    const int e = n % kPipeSlots;
    if (threadIdx.x == 0) {
      if (!S.err_s && !mbar_wait(&S.tfull[e], (uint32_t)((n / kPipeSlots) & 1), task_limit, &S.err_s)) {
        S.err_s = 1;
        atomicExch(V.err_flag, 1);
      }
      S.stop_s = (S.err_s || S.task[e].kind == kPipeEnd) ? 1 : 0;
    }
    consumer_sync();
    if (S.stop_s) break;
    const Task& t = S.task[e];
    if (t.kind == 0) {
      // a merged bottom subtree: its nodes in order (forward children first,
      // backward parents first), each on all consumers
      const int n_sub = t.c0;
      for (int i = 0; i < n_sub; ++i) {
        if constexpr (FWD) fwd_node(S.sub[e][i]);
        else bwd_node(S.sub[e][n_sub - 1 - i]);
        consumer_sync();
      }
    } else if (t.kind == 1) {
      if constexpr (FWD) fwd_node(t.nd);
      else bwd_node(t.nd);
    } else {
      if constexpr (FWD) fwd_wide(t);
      else bwd_wide(t);
    }
    // completion, as in the dynamic schedule: one fence, one counter atomic and,
    // when something is released, one queue reservation; then every consumer
    // writes released task ids
    consumer_sync();
    if (threadIdx.x == 0) {
      const int4 r = S.rec[e][0];
      int base = -1;
      __threadfence();
      if constexpr (FWD) {
        if (r.x >= 0 && atomicSub(P.pending + r.x, 1) == 1) base = atomicAdd(P.ctr + 1, r.z);
      } else if (r.z > 0 && (t.kind <= 1 || atomicAdd(P.done + t.node, 1) == r.w - 1)) {
        base = atomicAdd(P.ctr + 1, r.z);
      }
      if (base >= 0) __threadfence();
      S.base_s = base;
    }
    consumer_sync();
    const int base = S.base_s;
    if (base >= 0) {
      __threadfence();
      const int4 r = S.rec[e][0];
      if constexpr (FWD) {
        for (int i = threadIdx.x; i < r.z; i += kSolveThreads) st_relaxed(P.queue + base + i, r.y + i);
      } else {
        for (int kq = r.x; kq < r.y; ++kq) {   // block-uniform
          const int jq = kq - r.x;
          const int4 ev = jq < kPushKids ? S.rec[e][1 + jq] : P.kids[kq];
          for (int i = threadIdx.x; i < ev.y; i += kSolveThreads) st_relaxed(P.queue + base + ev.z + i, ev.x + i);
        }
      }
    }
    consumer_sync();   // the entry (task, push record) and rhs / red are free again
    if (threadIdx.x == 0) mbar_arrive(&S.tempty[e]);
  }
}

template <int D, bool FWD>
__global__ void __launch_bounds__(kPipeThreads, 2) k_solve_pipe(DynView V) {
  extern __shared__ __align__(128) unsigned char ffa_pipe_smem[];
  PipeSmem<D>& S = *reinterpret_cast<PipeSmem<D>*>(ffa_pipe_smem);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int s = 0; s < kPipeStages; ++s) {
      mbar_init(&S.full[s], 1);
      mbar_init(&S.empty[s], kPipeConsumers);
    }
#pragma unroll
    for (int e = 0; e < kPipeSlots; ++e) {
      mbar_init(&S.tfull[e], 1);
      mbar_init(&S.tempty[e], 1);
    }
    S.err_s = 0;
    S.stop_s = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x >= kSolveThreads) pipe_producer<D, FWD>(S, V);
  else pipe_consumer<D, FWD>(S, V);
}

// restores the ready queues, pending counts and completion counts of both passes
// and zeroes z and x (both are accumulated with atomics)
__device__ __forceinline__ void dyn_reset_body(const DynPass& F, const DynPass& B, int n_nodes, float* __restrict__ z,
                                               float* __restrict__ x, int64_t nzx, int64_t n_all) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_all; i += stride) {
    if (i < nzx) {
      z[i] = 0.f;
      x[i] = 0.f;
    }
    if (i < F.n_tasks) F.queue[i] = F.q_init[i];
    if (i < B.n_tasks) B.queue[i] = B.q_init[i];
    if (i < n_nodes) {
      F.pending[i] = F.pending_init[i];
      B.done[i] = 0;
    }
    if (i == 0) {
      F.ctr[0] = 0;
      F.ctr[1] = F.n_init;
      B.ctr[0] = 0;
      B.ctr[1] = B.n_init;
    }
  }
}

__global__ void k_dyn_reset(DynPass F, DynPass B, int n_nodes, float* __restrict__ z, float* __restrict__ x,
                            int64_t nzx, int64_t n_all) {
  dyn_reset_body(F, B, n_nodes, z, x, nzx, n_all);
}

// the residual of a refinement sweep and the reset of the two passes that follow
// it in one launch (the residual writes y only; the reset touches z, x and the
// schedules' counters, which the previous passes no longer use)
template <int D>
__global__ void __launch_bounds__(kVertexBlock) k_residual_reset(const int32_t* __restrict__ col,
                                                                 const double* __restrict__ val, int width, int nF,
                                                                 const double* __restrict__ X,
                                                                 const double* __restrict__ b, float* __restrict__ y,
                                                                 DynPass F, DynPass B, int n_nodes,
                                                                 float* __restrict__ z, float* __restrict__ x,
                                                                 int64_t nzx, int64_t n_all) {
  const int i = blockIdx.x * kVertexBlock + threadIdx.x;
  double rr = 0.0, bb = 0.0;
  if (i < nF) residual_row<D>(col, val, width, nF, X, b, y, i, rr, bb);
  dyn_reset_body(F, B, n_nodes, z, x, nzx, n_all);
}

template <int D>
__global__ void __launch_bounds__(kVertexBlock) k_pin_rhs(int nF, const int64_t* __restrict__ ptr,
                                                          const int32_t* __restrict__ pc, const double* __restrict__ val,
                                                          const double* __restrict__ pin_pos, double* __restrict__ cst) {
  const int i = blockIdx.x * kVertexBlock + threadIdx.x;
  if (i >= nF) return;
  double acc[D];
#pragma unroll
  for (int k = 0; k < D; ++k) acc[k] = 0.0;
  for (int64_t q = ptr[i]; q < ptr[i + 1]; ++q) {
    const double a = val[q];
    const int p = pc[q];
#pragma unroll
    for (int k = 0; k < D; ++k) acc[k] -= a * pin_pos[(int64_t)p * D + k];
  }
#pragma unroll
  for (int k = 0; k < D; ++k) cst[(int64_t)i * D + k] = acc[k];
}

// ---------------------------------------------------------------------------
// termination test (eqs. primaldualerror/primaldualthresholds): block q sums
// quantity q of the per-block partials; one thread then forms the statistics
// ---------------------------------------------------------------------------
__global__ void k_reduce_quantities(FinalLaunch F, double* __restrict__ sums) {
  const int q = blockIdx.x;
  double s = 0.0;
  if (q < NQ) {
    for (int64_t b = threadIdx.x; b < F.n_local_blocks; b += blockDim.x) s += F.local_partials[b * NQ + q];
  } else {
    for (int64_t b = threadIdx.x; b < F.n_vert_blocks; b += blockDim.x) s += F.vert_partials[b];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  __shared__ double wsum[32];
  if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += wsum[w];
    sums[q] = t;
  }
}

__global__ void k_stats(FinalLaunch F, const double* __restrict__ acc) {
  if (threadIdx.x != 0) return;
  ffa_stats st;
  st.iters = 0;
  st.checked_iter = F.iter;
  st.e_prim = sqrt(acc[Q_EPRIM]);
  st.e_dual = sqrt(acc[Q_EDUAL]);
  st.norm_GW = sqrt(acc[Q_GW]);
  st.norm_P = sqrt(acc[Q_P]);
  st.norm_GtLambda = sqrt(acc[NQ]);
  st.energy_P = acc[Q_ENERGY];
  st.n_flipped = (int32_t)(acc[Q_FLIPS] + 0.5);
  const double base = F.eps_abs * sqrt((double)F.d * (double)F.m);
  st.thr_prim = base + F.eps_rel * fmax(st.norm_GW, st.norm_P);
  st.thr_dual = base + F.eps_rel * st.norm_GtLambda;
  const bool finite_ok = acc[Q_NONFINITE] == 0.0 && isfinite(st.e_prim) && isfinite(st.e_dual);
  st.converged = (finite_ok && st.e_prim < st.thr_prim && st.e_dual < st.thr_dual &&
                  (!F.require_flip_free || st.n_flipped == 0)) ? 1 : 0;
  if (!finite_ok) st.converged = -1;
  *F.out = st;
}

__global__ void k_mesh_stats(MeshStatsLaunch M) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= M.n_mesh) return;
  const double* acc = M.mesh_acc + (int64_t)k * (NQ + 1);
  ffa_stats st;
  st.iters = 0;
  st.checked_iter = 0;
  st.e_prim = sqrt(acc[Q_EPRIM]);
  st.e_dual = sqrt(acc[Q_EDUAL]);
  st.norm_GW = sqrt(acc[Q_GW]);
  st.norm_P = sqrt(acc[Q_P]);
  st.norm_GtLambda = sqrt(acc[NQ]);
  st.energy_P = acc[Q_ENERGY];
  st.n_flipped = (int32_t)(acc[Q_FLIPS] + 0.5);
  const double base = M.mesh_eps[2 * k] * sqrt((double)M.mesh_d[k] * (double)M.mesh_m[k]);
  st.thr_prim = base + M.mesh_eps[2 * k + 1] * fmax(st.norm_GW, st.norm_P);
  st.thr_dual = base + M.mesh_eps[2 * k + 1] * st.norm_GtLambda;
  const bool finite_ok = acc[Q_NONFINITE] == 0.0 && isfinite(st.e_prim) && isfinite(st.e_dual);
  st.converged = (finite_ok && st.e_prim < st.thr_prim && st.e_dual < st.thr_dual &&
                  (!M.require_flip_free || st.n_flipped == 0)) ? 1 : 0;
  if (!finite_ok) st.converged = -1;
  if (st.converged == 1) atomicAdd(M.n_converged, 1);
  M.out[k] = st;
}

// one warp per mesh: the block sums of the mesh's first and last blocks in block
// order (lanes stride over the blocks, then a fixed shuffle tree)
__global__ void k_mesh_partials(MeshPartialsLaunch M) {
  const int k = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (k >= M.n_mesh) return;   // warp-uniform
  const int64_t e0 = M.seg_off[k], e1 = M.seg_off[k + 1];
  if (e1 <= e0) return;
  const int64_t b0 = e0 / M.items_per_block, b1 = (e1 - 1) / M.items_per_block;
  auto first_of = [&](int64_t b) { return M.seg_of[b * M.items_per_block]; };
  auto last_of = [&](int64_t b) { return M.seg_of[min(M.n_items, (b + 1) * M.items_per_block) - 1]; };
  if (b0 == b1 && first_of(b0) != k && last_of(b0) != k) return;   // written by its block
  for (int q = 0; q < M.nq; ++q) {
    double s = 0.0;
    for (int64_t b = b0 + lane; b <= b1; b += 32) {
      const int fo = first_of(b), la = last_of(b);
      if (fo == k) s += M.part[(b * 2 + 0) * M.nq + q];
      else if (la == k) s += M.part[(b * 2 + 1) * M.nq + q];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) M.acc[(int64_t)k * (NQ + 1) + M.q0 + q] = s;
  }
}

__global__ void k_sum_partials(const double* __restrict__ p, int64_t nb, int nq, double* __restrict__ out) {
  const int q = blockIdx.x;
  double s = 0.0;
  for (int64_t b = threadIdx.x; b < nb; b += blockDim.x) s += p[b * nq + q];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  __shared__ double wsum[32];
  if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += wsum[w];
    out[q] = t;
  }
}

inline int blocks_for(int64_t n, int b) { return (int)((n + b - 1) / b); }

}  // namespace

void launch_vertex_update(const VertexLaunch& V, cudaStream_t s) {
  const int g = blocks_for(V.n, kVertexBlock);
  if (V.d == 2) {
    if (V.fp64) k_vertex_update<2, true><<<g, kVertexBlock, 0, s>>>(V);
    else k_vertex_update<2, false><<<g, kVertexBlock, 0, s>>>(V);
  } else {
    if (V.fp64) k_vertex_update<3, true><<<g, kVertexBlock, 0, s>>>(V);
    else k_vertex_update<3, false><<<g, kVertexBlock, 0, s>>>(V);
  }
}

void launch_gather(const GatherLaunch& G, cudaStream_t s) {
  const int g = blocks_for((int64_t)G.rows * kGatherLanes, kVertexBlock);
  if (G.d == 2) {
    if (G.fp64) k_gather<2, true><<<g, kVertexBlock, 0, s>>>(G);
    else k_gather<2, false><<<g, kVertexBlock, 0, s>>>(G);
  } else {
    if (G.fp64) k_gather<3, true><<<g, kVertexBlock, 0, s>>>(G);
    else k_gather<3, false><<<g, kVertexBlock, 0, s>>>(G);
  }
}

void launch_residual(const SolveData& S, double* partials, int n_blocks, cudaStream_t s) {
  (void)n_blocks;
  const int g = blocks_for(S.nF, kVertexBlock);
  if (S.d == 2) k_residual<2><<<g, kVertexBlock, 0, s>>>(S.ell_col, S.ell_val, S.ell_width, S.nF, S.X, S.b, S.y, partials);
  else k_residual<3><<<g, kVertexBlock, 0, s>>>(S.ell_col, S.ell_val, S.ell_width, S.nF, S.X, S.b, S.y, partials);
}

void launch_constraint_projection(const ConstraintLaunch& C, cudaStream_t s) {
  if (C.c <= 0 || C.nF <= 0) return;
  const int g = blocks_for(C.nF, kVertexBlock);
  if (C.d == 2) {
    k_constraint_nu<2><<<1, 256, 0, s>>>(C);
    k_constraint_project<2><<<g, kVertexBlock, 0, s>>>(C);
  } else {
    k_constraint_nu<3><<<1, 256, 0, s>>>(C);
    k_constraint_project<3><<<g, kVertexBlock, 0, s>>>(C);
  }
}

void launch_copy_columns(const double* src, int d, double* dst, int c, int c0, int count, int nF, cudaStream_t s) {
  const int64_t n = (int64_t)nF * count;
  if (n <= 0) return;
  k_copy_columns<<<blocks_for(n, 256), 256, 0, s>>>(src, d, dst, c, c0, count, nF);
}

void launch_axpy_correction(const SolveData& S, cudaStream_t s) {
  const int64_t n = (int64_t)S.nF * S.d;
  k_axpy<<<blocks_for(n, 256), 256, 0, s>>>((int)n, S.X, S.x);
}

void launch_levels(const SolveData& S, int l0, int l1, bool forward, cudaStream_t s);

void launch_residual_reset(const SolveData& S, cudaStream_t s) {
  const int64_t nzx = (int64_t)S.nF * S.d;
  const int64_t n_all = std::max<int64_t>(std::max<int64_t>(nzx, S.n_nodes),
                                          std::max<int64_t>(S.fdyn.n_tasks, S.bdyn.n_tasks));
  const int g = blocks_for(S.nF, kVertexBlock);
  if (S.d == 2)
    k_residual_reset<2><<<g, kVertexBlock, 0, s>>>(S.ell_col, S.ell_val, S.ell_width, S.nF, S.X, S.b, S.y, S.fdyn,
                                                   S.bdyn, S.n_nodes, S.z, S.x, nzx, n_all);
  else
    k_residual_reset<3><<<g, kVertexBlock, 0, s>>>(S.ell_col, S.ell_val, S.ell_width, S.nF, S.X, S.b, S.y, S.fdyn,
                                                   S.bdyn, S.n_nodes, S.z, S.x, nzx, n_all);
}

// with the top levels as one operator: x_T = S^-1 t_T, t_T the forward pass's
// running right-hand side at the T columns
static void top_product(const SolveData& S, cudaStream_t s) {
  if (!S.top_on) return;
  launch_top_product(S.top, S.d, S.y, S.x, s);
  if (S.ev[3]) cudaEventRecord(S.ev[3], s);
}

void launch_supernodal_solve(const SolveData& S, cudaStream_t s, bool reset) {
  const int64_t nzx = (int64_t)S.nF * S.d;
  const int64_t n_all = std::max<int64_t>(std::max<int64_t>(nzx, S.n_nodes),
                                          std::max<int64_t>(S.fdyn.n_tasks, S.bdyn.n_tasks));
  const int reset_grid = (int)std::min<int64_t>((n_all + 255) / 256, 4096);
  if (reset) k_dyn_reset<<<reset_grid, 256, 0, s>>>(S.fdyn, S.bdyn, S.n_nodes, S.z, S.x, nzx, n_all);
  if (S.ev[0]) cudaEventRecord(S.ev[0], s);
  const int L = (int)S.fwd_off.size() - 1;
  if (S.schedule == 1 || S.schedule == 2) {
    const DynView vf{S.fdyn, S.sub_nodes, S.rows, S.blocks, S.y, S.z, S.x, S.err_flag, S.spin_limit};
    const DynView vb{S.bdyn, S.sub_nodes, S.rows, S.blocks, S.y, S.z, S.x, S.err_flag, S.spin_limit};
    const int nb = std::min(S.bottom_levels, L);
    launch_levels(S, 0, nb, true, s);
    if (S.schedule == 2) {
      if (S.d == 2) k_solve_pipe<2, true><<<S.pgrid_f, kPipeThreads, sizeof(PipeSmem<2>), s>>>(vf);
      else k_solve_pipe<3, true><<<S.pgrid_f, kPipeThreads, sizeof(PipeSmem<3>), s>>>(vf);
    } else {
      if (S.d == 2) k_solve_dynamic<2, true><<<S.grid_f, kSolveThreads, 0, s>>>(vf);
      else k_solve_dynamic<3, true><<<S.grid_f, kSolveThreads, 0, s>>>(vf);
    }
    if (S.ev[1]) cudaEventRecord(S.ev[1], s);
    top_product(S, s);
    if (S.schedule == 2) {
      if (S.d == 2) k_solve_pipe<2, false><<<S.pgrid_b, kPipeThreads, sizeof(PipeSmem<2>), s>>>(vb);
      else k_solve_pipe<3, false><<<S.pgrid_b, kPipeThreads, sizeof(PipeSmem<3>), s>>>(vb);
    } else {
      if (S.d == 2) k_solve_dynamic<2, false><<<S.grid_b, kSolveThreads, 0, s>>>(vb);
      else k_solve_dynamic<3, false><<<S.grid_b, kSolveThreads, 0, s>>>(vb);
    }
    launch_levels(S, 0, nb, false, s);
    if (S.ev[2]) cudaEventRecord(S.ev[2], s);
    return;
  }
  launch_levels(S, 0, L, true, s);
  if (S.ev[1]) cudaEventRecord(S.ev[1], s);
  top_product(S, s);
  launch_levels(S, 0, L, false, s);
  if (S.ev[2]) cudaEventRecord(S.ev[2], s);
}

// one launch per level: forward over levels [l0, l1) bottom up, backward top down
void launch_levels(const SolveData& S, int l0, int l1, bool forward, cudaStream_t s) {
  if (forward) {
    for (int l = l0; l < l1; ++l) {
      const int64_t nt = S.fwd_off[l + 1] - S.fwd_off[l];
      if (nt <= 0) continue;
      if (S.d == 2) k_forward<2><<<(unsigned)nt, kSolveThreads, 0, s>>>(S.fwd_tasks + S.fwd_off[l], S.rows, S.blocks, S.y, S.z);
      else k_forward<3><<<(unsigned)nt, kSolveThreads, 0, s>>>(S.fwd_tasks + S.fwd_off[l], S.rows, S.blocks, S.y, S.z);
    }
    return;
  }
  for (int l = l1 - 1; l >= l0; --l) {
    const int64_t nt = S.bwd_off[l + 1] - S.bwd_off[l];
    if (nt <= 0) continue;
    if (S.d == 2) k_backward<2><<<(unsigned)nt, kSolveThreads, 0, s>>>(S.bwd_tasks + S.bwd_off[l], S.rows, S.blocks, S.z, S.x);
    else k_backward<3><<<(unsigned)nt, kSolveThreads, 0, s>>>(S.bwd_tasks + S.bwd_off[l], S.rows, S.blocks, S.z, S.x);
  }
}

int persistent_grid(int d, bool forward) {
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaError_t e;
  if (forward) e = d == 2 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_solve_dynamic<2, true>, kSolveThreads, 0)
                          : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_solve_dynamic<3, true>, kSolveThreads, 0);
  else e = d == 2 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_solve_dynamic<2, false>, kSolveThreads, 0)
                  : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_solve_dynamic<3, false>, kSolveThreads, 0);
  if (e != cudaSuccess || per < 1) per = 1;
  return sms * per;
}

// resident blocks of the pipelined solve kernels (dynamic shared memory above the
// default 48 KB limit is enabled here, once, before any launch or capture)
template <int D, bool FWD>
int pipe_grid_for() {
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int bytes = (int)sizeof(PipeSmem<D>);
  if (cudaFuncSetAttribute(k_solve_pipe<D, FWD>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) != cudaSuccess)
    return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_solve_pipe<D, FWD>, kPipeThreads, bytes) != cudaSuccess)
    return 0;
  return sms * per;
}

int persistent_pipe_grid(int d, bool forward) {
  if (d == 2) return forward ? pipe_grid_for<2, true>() : pipe_grid_for<2, false>();
  return forward ? pipe_grid_for<3, true>() : pipe_grid_for<3, false>();
}

void launch_pin_rhs(int d, int nF, const int64_t* ptr, const int32_t* pin_col, const double* val,
                    const double* pin_pos, double* cst, cudaStream_t s) {
  const int g = blocks_for(nF, kVertexBlock);
  if (d == 2) k_pin_rhs<2><<<g, kVertexBlock, 0, s>>>(nF, ptr, pin_col, val, pin_pos, cst);
  else k_pin_rhs<3><<<g, kVertexBlock, 0, s>>>(nF, ptr, pin_col, val, pin_pos, cst);
}

void launch_final_reduce(const FinalLaunch& F, cudaStream_t s) {
  k_reduce_quantities<<<NQ + 1, 512, 0, s>>>(F, F.scratch);
  k_stats<<<1, 32, 0, s>>>(F, F.scratch);
}

void launch_mesh_stats(const MeshStatsLaunch& M, cudaStream_t s) {
  k_mesh_stats<<<(M.n_mesh + 127) / 128, 128, 0, s>>>(M);
}

void launch_mesh_partials(const MeshPartialsLaunch& M, cudaStream_t s) {
  if (M.n_mesh <= 0) return;
  k_mesh_partials<<<(M.n_mesh * 32 + 255) / 256, 256, 0, s>>>(M);
}

void launch_sum_partials(const double* partials, int64_t n_blocks, int nq, double* out, cudaStream_t s) {
  k_sum_partials<<<nq, 256, 0, s>>>(partials, n_blocks, nq, out);
}

}  // namespace ffa
