// Vertex-side kernels of the W step (eq. solvinginw): right-hand-side gather G^T r,
// the double-precision residual b - L_FF W_F, the float supernodal triangular
// solves that turn the residual into a correction (mixed-precision refinement),
// and the vertex update that publishes W for the next local step.  Also the
// reductions that evaluate the termination test of eqs. primaldualerror/primaldualthresholds.
#include <math.h>

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
// row's vertex (+ add_row); float terms are summed in double-float
// ---------------------------------------------------------------------------
template <int D, bool FP64>
__global__ void __launch_bounds__(kVertexBlock) k_gather(GatherLaunch G) {
  const int row = blockIdx.x * kVertexBlock + threadIdx.x;
  double outv[D];
  double sq = 0.0;
  if (row < G.rows) {
    const int v = G.row_vertex ? G.row_vertex[row] : row;
    const int64_t q0 = G.inc_ptr[v], q1 = G.inc_ptr[v + 1];
    if constexpr (FP64) {
      const double* c = reinterpret_cast<const double*>(G.contrib);
      double acc[D];
#pragma unroll
      for (int k = 0; k < D; ++k) acc[k] = 0.0;
      for (int64_t q = q0; q < q1; ++q) {
        const int64_t base = (int64_t)__ldg(G.inc + q) * D;
#pragma unroll
        for (int k = 0; k < D; ++k) acc[k] += __ldg(c + base + k);
      }
#pragma unroll
      for (int k = 0; k < D; ++k) outv[k] = acc[k];
    } else {
      const float* c = reinterpret_cast<const float*>(G.contrib);
      FF acc[2][D];
#pragma unroll
      for (int k = 0; k < D; ++k) acc[0][k] = acc[1][k] = FF{0.f, 0.f};
      int64_t q = q0;
      for (; q + 4 <= q1; q += 4) {
        int64_t base[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) base[u] = (int64_t)__ldg(G.inc + q + u) * D;
        float v[4][D];
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int k = 0; k < D; ++k) v[u][k] = __ldg(c + base[u] + k);
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int k = 0; k < D; ++k) acc[u & 1][k] = ff_addf(acc[u & 1][k], v[u][k]);
      }
      for (; q < q1; ++q) {
        const int64_t base = (int64_t)__ldg(G.inc + q) * D;
#pragma unroll
        for (int k = 0; k < D; ++k) acc[0][k] = ff_addf(acc[0][k], __ldg(c + base + k));
      }
#pragma unroll
      for (int k = 0; k < D; ++k) {
        const FF a = ff_add(acc[0][k], acc[1][k]);
        outv[k] = (double)a.hi + (double)a.lo;
      }
    }
#pragma unroll
    for (int k = 0; k < D; ++k) {
      if (G.add) outv[k] += G.add[(int64_t)row * D + k];
      if (G.out) G.out[(int64_t)row * D + k] = outv[k];
      sq += outv[k] * outv[k];
    }
  }
  if (G.mesh_of) {
    // batched meshes: per-mesh sum of squares, warp-aggregated when the warp is uniform
    const int mesh = (row < G.rows) ? G.mesh_of[G.row_vertex ? G.row_vertex[row] : row] : -1;
    const int m0 = __shfl_sync(0xffffffffu, mesh, 0);
    if (__all_sync(0xffffffffu, mesh == m0)) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
      if ((threadIdx.x & 31) == 0 && m0 >= 0) atomicAdd(G.mesh_acc + (int64_t)m0 * (NQ + 1) + NQ, sq);
    } else if (mesh >= 0) {
      atomicAdd(G.mesh_acc + (int64_t)mesh * (NQ + 1) + NQ, sq);
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
__global__ void __launch_bounds__(kVertexBlock) k_residual(const int32_t* __restrict__ col, const double* __restrict__ val,
                                                            int width, int nF, const double* __restrict__ X,
                                                            const double* __restrict__ b, float* __restrict__ y,
                                                            double* __restrict__ partials) {
  const int i = blockIdx.x * kVertexBlock + threadIdx.x;
  double rr = 0.0, bb = 0.0;
  if (i < nF) {
    double acc[D];
#pragma unroll
    for (int k = 0; k < D; ++k) acc[k] = b[(int64_t)i * D + k];
    for (int q = 0; q < width; ++q) {
      const int j = __ldg(col + (int64_t)q * nF + i);
      const double a = __ldg(val + (int64_t)q * nF + i);
#pragma unroll
      for (int k = 0; k < D; ++k) acc[k] = fma(-a, X[(int64_t)j * D + k], acc[k]);
    }
#pragma unroll
    for (int k = 0; k < D; ++k) {
      y[(int64_t)i * D + k] = (float)acc[k];
      rr += acc[k] * acc[k];
      const double bk = b[(int64_t)i * D + k];
      bb += bk * bk;
    }
  }
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

__global__ void k_axpy(int n, double* __restrict__ X, const float* __restrict__ x) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) X[i] += (double)x[i];
}

// ---------------------------------------------------------------------------
// supernodal solves.  B_s is column-major with a leading dimension ld that is a
// multiple of 4, so every lane reads 4 consecutive rows of a column as one
// float4 and a warp reads 512 contiguous bytes per column.
//
// Forward task (node, r0, c0): rows [r0, r0+128) of B_s times the slice
// [c0, c0+256) of f = y[cols(s)]; warp w takes columns c0+32w .. c0+32w+31, the
// eight partial sums are added in shared memory and the 128 row results go out
// as one set of atomics: rows < n_s into z, rows >= n_s subtracted from y at the
// structure rows.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float4 ldg_stream(const float* p) {
  return __ldg(reinterpret_cast<const float4*>(p));
}

// Narrow nodes (at most 64 columns, the leaves and small separators) would
// leave most of a wide task's warps idle, so one warp takes one 128-row slice of
// such a node over all its columns, eight independent warps per block.  The
// level's task list holds its wide tasks first, then the narrow warp tasks
// (padded with node = -1 to a multiple of 8).
constexpr int kNarrowCols = 64;

template <int D>
__device__ __forceinline__ void forward_wide(const Task& t, const NodeDev& nd, const int32_t* __restrict__ rows,
                                             const float* __restrict__ blocks, float* __restrict__ y,
                                             float* __restrict__ z, float* smem) {
  float (*fs)[D] = reinterpret_cast<float (*)[D]>(smem);                       // [256][D]
  float (*red)[kFwdRows][D] = reinterpret_cast<float (*)[kFwdRows][D]>(smem + kFwdCols * D);  // [8][128][D]
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ntot = nd.ncol + nd.nrow;
  const int nc = min(kFwdCols, nd.ncol - t.c0);
  for (int q = threadIdx.x; q < nc * D; q += 256) {
    const int c = q / D, k = q - c * D;
    fs[c][k] = __ldcg(y + (int64_t)(nd.col0 + t.c0 + c) * D + k);
  }
  __syncthreads();
  const int r = t.r0 + 4 * lane;
  const int cw0 = 32 * warp;
  const int ncw = max(0, min(32, nc - cw0));
  float acc[4][D];
#pragma unroll
  for (int q = 0; q < 4; ++q)
#pragma unroll
    for (int k = 0; k < D; ++k) acc[q][k] = 0.f;
  if (r < nd.ld && ncw > 0) {
    const float* B = blocks + nd.blk_off + (int64_t)(t.c0 + cw0) * nd.ld + r;
    int c = 0;
    for (; c + 16 <= ncw; c += 16) {
      float4 b[16];
#pragma unroll
      for (int u = 0; u < 16; ++u) b[u] = ldg_stream(B + (int64_t)(c + u) * nd.ld);
#pragma unroll
      for (int u = 0; u < 16; ++u)
#pragma unroll
        for (int k = 0; k < D; ++k) {
          const float f = fs[cw0 + c + u][k];
          acc[0][k] = fmaf(b[u].x, f, acc[0][k]);
          acc[1][k] = fmaf(b[u].y, f, acc[1][k]);
          acc[2][k] = fmaf(b[u].z, f, acc[2][k]);
          acc[3][k] = fmaf(b[u].w, f, acc[3][k]);
        }
    }
    for (; c < ncw; ++c) {
      const float4 bv = ldg_stream(B + (int64_t)c * nd.ld);
#pragma unroll
      for (int k = 0; k < D; ++k) {
        const float f = fs[cw0 + c][k];
        acc[0][k] = fmaf(bv.x, f, acc[0][k]);
        acc[1][k] = fmaf(bv.y, f, acc[1][k]);
        acc[2][k] = fmaf(bv.z, f, acc[2][k]);
        acc[3][k] = fmaf(bv.w, f, acc[3][k]);
      }
    }
  }
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
        for (int w = 0; w < 8; ++w) a += red[w][threadIdx.x][k];
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

// one warp: rows [r0, r0+128) of a narrow node times all of f = y[cols(s)].
// The node's z rows lie in its first slice and only this warp writes them.
template <int D>
__device__ __forceinline__ void forward_narrow(const Task& t, const NodeDev& nd, const int32_t* __restrict__ rows,
                                               const float* __restrict__ blocks, float* __restrict__ y,
                                               float* __restrict__ z, float (*fw)[D]) {
  const int lane = threadIdx.x & 31;
  const int ntot = nd.ncol + nd.nrow;
  for (int q = lane; q < nd.ncol * D; q += 32) {
    const int c = q / D, k = q - c * D;
    fw[c][k] = __ldcg(y + (int64_t)(nd.col0 + c) * D + k);
  }
  __syncwarp();
  const int r = t.r0 + 4 * lane;
  float acc[4][D];
#pragma unroll
  for (int q = 0; q < 4; ++q)
#pragma unroll
    for (int k = 0; k < D; ++k) acc[q][k] = 0.f;
  if (r < nd.ld) {
    const float* B = blocks + nd.blk_off + r;
    int c = 0;
    for (; c + 8 <= nd.ncol; c += 8) {
      float4 b[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) b[u] = ldg_stream(B + (int64_t)(c + u) * nd.ld);
#pragma unroll
      for (int u = 0; u < 8; ++u)
#pragma unroll
        for (int k = 0; k < D; ++k) {
          const float f = fw[c + u][k];
          acc[0][k] = fmaf(b[u].x, f, acc[0][k]);
          acc[1][k] = fmaf(b[u].y, f, acc[1][k]);
          acc[2][k] = fmaf(b[u].z, f, acc[2][k]);
          acc[3][k] = fmaf(b[u].w, f, acc[3][k]);
        }
    }
    for (; c < nd.ncol; ++c) {
      const float4 bv = ldg_stream(B + (int64_t)c * nd.ld);
#pragma unroll
      for (int k = 0; k < D; ++k) {
        const float f = fw[c][k];
        acc[0][k] = fmaf(bv.x, f, acc[0][k]);
        acc[1][k] = fmaf(bv.y, f, acc[1][k]);
        acc[2][k] = fmaf(bv.z, f, acc[2][k]);
        acc[3][k] = fmaf(bv.w, f, acc[3][k]);
      }
    }
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int row = r + q;
    if (row >= ntot) break;
    if (row < nd.ncol) {
#pragma unroll
      for (int k = 0; k < D; ++k) z[(int64_t)(nd.col0 + row) * D + k] = acc[q][k];
    } else {
      const int rr = __ldg(rows + nd.row_off + (row - nd.ncol));
#pragma unroll
      for (int k = 0; k < D; ++k) atomicAdd(y + (int64_t)rr * D + k, -acc[q][k]);
    }
  }
}

template <int D>
__global__ void __launch_bounds__(256) k_forward(const Task* __restrict__ tasks, int n_wide,
                                                 const NodeDev* __restrict__ nodes, const int32_t* __restrict__ rows,
                                                 const float* __restrict__ blocks, float* __restrict__ y,
                                                 float* __restrict__ z) {
  __shared__ __align__(16) float smem[kFwdCols * D + 8 * kFwdRows * D];
  if ((int)blockIdx.x < n_wide) {
    const Task t = tasks[blockIdx.x];
    const NodeDev nd = nodes[t.node];
    forward_wide<D>(t, nd, rows, blocks, y, z, smem);
    return;
  }
  const int warp = threadIdx.x >> 5;
  const Task t = tasks[n_wide + ((int)blockIdx.x - n_wide) * 8 + warp];
  if (t.node < 0) return;
  const NodeDev nd = nodes[t.node];
  float (*fw)[D] = reinterpret_cast<float (*)[D]>(smem + warp * kNarrowCols * D);
  forward_narrow<D>(t, nd, rows, blocks, y, z, fw);
}

// Backward task (node, r0, c0): output columns [c0, c0+32) of x_s against rows
// [r0, r0+1024) of B_s, v = [z_s ; -x at the structure rows] staged in shared
// memory.  Warp w owns columns c0+4w .. c0+4w+3; each lane reads 4 rows of each
// of them per step; the 4 column dot products are reduced across the warp.
template <int D>
__device__ __forceinline__ void backward_wide(const Task& t, const NodeDev& nd, const int32_t* __restrict__ rows,
                                              const float* __restrict__ blocks, const float* __restrict__ z,
                                              float* __restrict__ x, float* smem) {
  float (*vs)[kBwdRows] = reinterpret_cast<float (*)[kBwdRows]>(smem);   // [D][1024]
  const int ntot = nd.ncol + nd.nrow;
  const int nr = min(kBwdRows, nd.ld - t.r0);     // a multiple of 4
  for (int r = threadIdx.x; r < nr; r += 256) {
    const int row = t.r0 + r;
#pragma unroll
    for (int k = 0; k < D; ++k) {
      float v = 0.f;
      if (row < nd.ncol) v = __ldcg(z + (int64_t)(nd.col0 + row) * D + k);
      else if (row < ntot) v = -__ldcg(x + (int64_t)__ldg(rows + nd.row_off + (row - nd.ncol)) * D + k);
      vs[k][r] = v;
    }
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int j0 = t.c0 + 4 * warp;
  if (j0 >= nd.ncol) return;
  const int ncw = min(4, nd.ncol - j0);
  float acc[4][D];
#pragma unroll
  for (int q = 0; q < 4; ++q)
#pragma unroll
    for (int k = 0; k < D; ++k) acc[q][k] = 0.f;
  const float* B = blocks + nd.blk_off + (int64_t)j0 * nd.ld + t.r0;
  // rows above the diagonal of inv(L_ss) are stored zeros: start at the first
  // 4-row group that can be nonzero for this warp's first column
  const int rs = max(0, (j0 - t.r0) & ~3);
#pragma unroll 4
  for (int r = rs + 4 * lane; r < nr; r += 128) {
    float4 b[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) b[q] = (q < ncw) ? ldg_stream(B + (int64_t)q * nd.ld + r) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int k = 0; k < D; ++k) {
      const float4 v = *reinterpret_cast<const float4*>(&vs[k][r]);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        acc[q][k] = fmaf(b[q].x, v.x, acc[q][k]);
        acc[q][k] = fmaf(b[q].y, v.y, acc[q][k]);
        acc[q][k] = fmaf(b[q].z, v.z, acc[q][k]);
        acc[q][k] = fmaf(b[q].w, v.w, acc[q][k]);
      }
    }
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

// one warp: a whole narrow node (<= 64 columns, ld <= 256).  v is staged in the
// warp's shared slice; lane j owns output columns j and j+32 and streams its own
// column of B_s (rows below the diagonal only), so no cross-lane reduction is
// needed and x_s is written directly (no other task touches it).
template <int D>
__device__ __forceinline__ void backward_narrow(const NodeDev& nd, const int32_t* __restrict__ rows,
                                                const float* __restrict__ blocks, const float* __restrict__ z,
                                                float* __restrict__ x, float (*vw)[256]) {
  const int lane = threadIdx.x & 31;
  const int ntot = nd.ncol + nd.nrow;
  for (int r = lane; r < nd.ld; r += 32) {
#pragma unroll
    for (int k = 0; k < D; ++k) {
      float val = 0.f;
      if (r < nd.ncol) val = __ldcg(z + (int64_t)(nd.col0 + r) * D + k);
      else if (r < ntot) val = -__ldcg(x + (int64_t)__ldg(rows + nd.row_off + (r - nd.ncol)) * D + k);
      vw[k][r] = val;
    }
  }
  __syncwarp();
  for (int j = lane; j < nd.ncol; j += 32) {
    const float* B = blocks + nd.blk_off + (int64_t)j * nd.ld;
    float acc[D];
#pragma unroll
    for (int k = 0; k < D; ++k) acc[k] = 0.f;
    int r = j & ~3;
    for (; r + 16 <= nd.ld; r += 16) {
      float4 b[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) b[u] = ldg_stream(B + r + 4 * u);
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int k = 0; k < D; ++k) {
          const float4 v = *reinterpret_cast<const float4*>(&vw[k][r + 4 * u]);
          acc[k] = fmaf(b[u].x, v.x, acc[k]);
          acc[k] = fmaf(b[u].y, v.y, acc[k]);
          acc[k] = fmaf(b[u].z, v.z, acc[k]);
          acc[k] = fmaf(b[u].w, v.w, acc[k]);
        }
    }
    for (; r < nd.ld; r += 4) {
      const float4 bv = ldg_stream(B + r);
#pragma unroll
      for (int k = 0; k < D; ++k) {
        const float4 v = *reinterpret_cast<const float4*>(&vw[k][r]);
        acc[k] = fmaf(bv.x, v.x, acc[k]);
        acc[k] = fmaf(bv.y, v.y, acc[k]);
        acc[k] = fmaf(bv.z, v.z, acc[k]);
        acc[k] = fmaf(bv.w, v.w, acc[k]);
      }
    }
#pragma unroll
    for (int k = 0; k < D; ++k) x[(int64_t)(nd.col0 + j) * D + k] = acc[k];
  }
}

template <int D>
__global__ void __launch_bounds__(256) k_backward(const Task* __restrict__ tasks, int n_wide,
                                                  const NodeDev* __restrict__ nodes, const int32_t* __restrict__ rows,
                                                  const float* __restrict__ blocks, const float* __restrict__ z,
                                                  float* __restrict__ x) {
  constexpr int kSmem = (D * kBwdRows > 8 * D * 256) ? D * kBwdRows : 8 * D * 256;
  __shared__ __align__(16) float smem[kSmem];
  if ((int)blockIdx.x < n_wide) {
    const Task t = tasks[blockIdx.x];
    const NodeDev nd = nodes[t.node];
    backward_wide<D>(t, nd, rows, blocks, z, x, smem);
    return;
  }
  const int warp = threadIdx.x >> 5;
  const Task t = tasks[n_wide + ((int)blockIdx.x - n_wide) * 8 + warp];
  if (t.node < 0) return;
  backward_narrow<D>(nodes[t.node], rows, blocks, z, x, reinterpret_cast<float (*)[256]>(smem + warp * D * 256));
}

// ---------------------------------------------------------------------------
// Persistent schedule: one launch per pass.  Blocks claim work items in
// dependency order (forward: leaves first; backward: root first) from a global
// counter, wait until the tasks their node depends on are done (forward: its
// nearest descendants with tasks; backward: its nearest ancestor with tasks),
// run the same per-task code as the level-synchronous kernels, and count the
// task as done.  Every waited-on task was claimed earlier by a running block,
// so the waits end; each wait is still bounded and sets err_flag instead of
// spinning on.
// ---------------------------------------------------------------------------
constexpr long long kSpinLimit = 1LL << 22;   // polls of ~100 ns (~0.4 s) before giving up

// the plain-data part of SolveData that the persistent kernels need
struct PersistView {
  const Task* fwd_tasks;
  const Task* bwd_tasks;
  const NodeDev* nodes;
  const int32_t* rows;
  const float* blocks;
  float* y;
  float* z;
  float* x;
  const int2* items_f;
  const int2* items_b;
  int n_items_f, n_items_b;
  const int32_t* need_f;
  const int32_t* need_b;
  const int32_t* fchild_ptr;
  const int32_t* fchild;
  const int32_t* bpar;
  int32_t* sync;
  int n_nodes;
  int32_t* err_flag;
};

__device__ __forceinline__ int ld_acquire(const int32_t* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Once any wait has given up (err set), every later wait returns at once, so a
// failure costs one timeout, not one per task.
__device__ __forceinline__ void wait_count(const int32_t* p, int need, int32_t* err) {
  long long it = 0;
  while (ld_acquire(p) < need) {
    if (++it > kSpinLimit || ld_acquire(err) != 0) {
      atomicExch(err, 1);
      return;
    }
    __nanosleep(100);
  }
}

__device__ __forceinline__ void wait_children(const PersistView& S, int node) {
  for (int q = S.fchild_ptr[node]; q < S.fchild_ptr[node + 1]; ++q) {
    const int c = S.fchild[q];
    wait_count(S.sync + c, S.need_f[c], S.err_flag);
  }
}

template <int D>
__global__ void __launch_bounds__(256) k_forward_persistent(PersistView S) {
  __shared__ __align__(16) float smem[kFwdCols * D + 8 * kFwdRows * D];
  __shared__ int item_s;
  int32_t* counter = S.sync + 2 * S.n_nodes;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (;;) {
    if (threadIdx.x == 0) item_s = atomicAdd(counter, 1);
    __syncthreads();
    const int item = item_s;
    if (item >= S.n_items_f) break;
    const int2 it = S.items_f[item];
    if (it.y == 0) {
      const Task t = S.fwd_tasks[it.x];
      const NodeDev nd = S.nodes[t.node];
      if (threadIdx.x == 0) wait_children(S, t.node);
      __syncthreads();
      forward_wide<D>(t, nd, S.rows, S.blocks, S.y, S.z, smem);
      __threadfence();
      __syncthreads();
      if (threadIdx.x == 0) atomicAdd(S.sync + t.node, 1);
    } else {
      const Task t = S.fwd_tasks[it.x + warp];
      if (t.node >= 0) {
        if (lane == 0) wait_children(S, t.node);
        __syncwarp();
        const NodeDev nd = S.nodes[t.node];
        forward_narrow<D>(t, nd, S.rows, S.blocks, S.y, S.z,
                          reinterpret_cast<float (*)[D]>(smem + warp * kNarrowCols * D));
        __threadfence();
        __syncwarp();
        if (lane == 0) atomicAdd(S.sync + t.node, 1);
      }
    }
    __syncthreads();   // item_s and smem are reused by the next item
  }
}

template <int D>
__global__ void __launch_bounds__(256) k_backward_persistent(PersistView S) {
  constexpr int kSmem = (D * kBwdRows > 8 * D * 256) ? D * kBwdRows : 8 * D * 256;
  __shared__ __align__(16) float smem[kSmem];
  __shared__ int item_s;
  int32_t* counter = S.sync + 2 * S.n_nodes + 1;
  int32_t* done_b = S.sync + S.n_nodes;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (;;) {
    if (threadIdx.x == 0) item_s = atomicAdd(counter, 1);
    __syncthreads();
    const int item = item_s;
    if (item >= S.n_items_b) break;
    const int2 it = S.items_b[item];
    if (it.y == 0) {
      const Task t = S.bwd_tasks[it.x];
      const NodeDev nd = S.nodes[t.node];
      const int p = S.bpar[t.node];
      if (threadIdx.x == 0 && p >= 0) wait_count(done_b + p, S.need_b[p], S.err_flag);
      __syncthreads();
      backward_wide<D>(t, nd, S.rows, S.blocks, S.z, S.x, smem);
      __threadfence();
      __syncthreads();
      if (threadIdx.x == 0) atomicAdd(done_b + t.node, 1);
    } else {
      const Task t = S.bwd_tasks[it.x + warp];
      if (t.node >= 0) {
        const int p = S.bpar[t.node];
        if (lane == 0 && p >= 0) wait_count(done_b + p, S.need_b[p], S.err_flag);
        __syncwarp();
        backward_narrow<D>(S.nodes[t.node], S.rows, S.blocks, S.z, S.x,
                           reinterpret_cast<float (*)[256]>(smem + warp * D * 256));
        __threadfence();
        __syncwarp();
        if (lane == 0) atomicAdd(done_b + t.node, 1);
      }
    }
    __syncthreads();
  }
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
  const int g = blocks_for(G.rows, kVertexBlock);
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

void launch_axpy_correction(const SolveData& S, cudaStream_t s) {
  const int64_t n = (int64_t)S.nF * S.d;
  k_axpy<<<blocks_for(n, 256), 256, 0, s>>>((int)n, S.X, S.x);
}

void launch_supernodal_solve(const SolveData& S, cudaStream_t s) {
  const size_t bytes = (size_t)S.nF * S.d * sizeof(float);
  cudaMemsetAsync(S.z, 0, bytes, s);
  cudaMemsetAsync(S.x, 0, bytes, s);
  if (S.schedule == 1) {
    cudaMemsetAsync(S.sync, 0, (size_t)(2 * S.n_nodes + 2) * sizeof(int32_t), s);
    PersistView v{S.fwd_tasks, S.bwd_tasks, S.nodes, S.rows, S.blocks, S.y, S.z, S.x, S.items_f, S.items_b,
                  S.n_items_f, S.n_items_b, S.need_f, S.need_b, S.fchild_ptr, S.fchild, S.bpar, S.sync,
                  S.n_nodes, S.err_flag};
    if (S.d == 2) {
      k_forward_persistent<2><<<S.grid_f, 256, 0, s>>>(v);
      k_backward_persistent<2><<<S.grid_b, 256, 0, s>>>(v);
    } else {
      k_forward_persistent<3><<<S.grid_f, 256, 0, s>>>(v);
      k_backward_persistent<3><<<S.grid_b, 256, 0, s>>>(v);
    }
    return;
  }
  const int L = (int)S.fwd_off.size() - 1;
  for (int l = 0; l < L; ++l) {
    const int64_t nt = S.fwd_off[l + 1] - S.fwd_off[l];
    if (nt <= 0) continue;
    const int nw = (int)S.fwd_wide[l];
    const unsigned grid = (unsigned)(nw + (nt - nw) / 8);
    if (S.d == 2) k_forward<2><<<grid, 256, 0, s>>>(S.fwd_tasks + S.fwd_off[l], nw, S.nodes, S.rows, S.blocks, S.y, S.z);
    else k_forward<3><<<grid, 256, 0, s>>>(S.fwd_tasks + S.fwd_off[l], nw, S.nodes, S.rows, S.blocks, S.y, S.z);
  }
  for (int l = L - 1; l >= 0; --l) {
    const int64_t nt = S.bwd_off[l + 1] - S.bwd_off[l];
    if (nt <= 0) continue;
    const int nw = (int)S.bwd_wide[l];
    const unsigned grid = (unsigned)(nw + (nt - nw) / 8);
    if (S.d == 2) k_backward<2><<<grid, 256, 0, s>>>(S.bwd_tasks + S.bwd_off[l], nw, S.nodes, S.rows, S.blocks, S.z, S.x);
    else k_backward<3><<<grid, 256, 0, s>>>(S.bwd_tasks + S.bwd_off[l], nw, S.nodes, S.rows, S.blocks, S.z, S.x);
  }
}

int persistent_grid(int d, bool forward) {
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaError_t e;
  if (forward) e = d == 2 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_forward_persistent<2>, 256, 0)
                          : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_forward_persistent<3>, 256, 0);
  else e = d == 2 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_backward_persistent<2>, 256, 0)
                  : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_backward_persistent<3>, 256, 0);
  if (e != cudaSuccess || per < 1) per = 1;
  return sms * per;
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

void launch_sum_partials(const double* partials, int64_t n_blocks, int nq, double* out, cudaStream_t s) {
  k_sum_partials<<<nq, 256, 0, s>>>(partials, n_blocks, nq, out);
}

}  // namespace ffa
