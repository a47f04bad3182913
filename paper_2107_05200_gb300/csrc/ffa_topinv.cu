// The top-of-tree inverse (ffa_topinv.h): its setup after each decomposition and
// the product x_T = S^-1 t_T of every solve.
//
// Setup tile products run on one block of 256 threads per 64 x 64 output tile,
// each thread 4 x 4 outputs (rows 4 tx + i, columns 4 ty + j), operands staged in
// shared memory 32 steps of the sum at a time; rows and columns past an operand's
// end are read as zero.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "ffa_topinv_launch.h"

namespace ffa {
namespace {

constexpr int kT = kTiTile;
constexpr int kKc = 32;
constexpr int kThreads = 256;
constexpr int kLd = kT + 4;   // shared rows padded so that every group of four starts on 16 bytes

struct __align__(16) TiSmem {
  float a[kKc][kLd];
  float b[kKc][kLd];
};

// acc[i][j] += sum_{k < K} A(4 tx + i, k) B(4 ty + j, k) with B(c, k) = B[c ldb + k]
// (c < cb) and A(r, k) = A[k lda + r] (!AK) or A[r lda + k] (AK), r < ra
template <bool AK>
__device__ __forceinline__ void tile_products(float (&acc)[4][4], const float* A, int64_t lda, int ra,
                                              const float* B, int64_t ldb, int cb, int K, TiSmem& sm) {
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  for (int k0 = 0; k0 < K; k0 += kKc) {
    const int kc = min(kKc, K - k0);
    for (int e = tid; e < kKc * kT; e += kThreads) {
      if (AK) {
        const int r = e >> 5, k = e & 31;
        sm.a[k][r] = (k < kc && r < ra) ? A[(int64_t)r * lda + k0 + k] : 0.f;
      } else {
        const int k = e >> 6, r = e & 63;
        sm.a[k][r] = (k < kc && r < ra) ? A[(int64_t)(k0 + k) * lda + r] : 0.f;
      }
      const int c = e >> 5, k = e & 31;
      sm.b[k][c] = (k < kc && c < cb) ? B[(int64_t)c * ldb + k0 + k] : 0.f;
    }
    __syncthreads();
#pragma unroll 4
    for (int k = 0; k < kc; ++k) {
      const float4 a = *reinterpret_cast<const float4*>(&sm.a[k][4 * tx]);
      const float4 b = *reinterpret_cast<const float4*>(&sm.b[k][4 * ty]);
      const float av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
    }
    __syncthreads();
  }
}

__global__ void k_ti_eye(float* G, int64_t ldG, int nT) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < nT) G[(int64_t)p * ldG + p] = 1.f;
}

// One step of the forward pass over T applied to G (columns lo .. lo + C of
// supernode s): out rows of F_s = inv(L_ss) G_s (rmap null), or the structure rows
// of G minus (L_rs inv(L_ss)) G_s (rmap: their T positions).
struct TiApply {
  const float* A;      // inv(L_ss) or L_rs inv(L_ss): A(r, k) = A[k lda + r]
  int64_t lda;
  int R, K;            // rows of A, n_s
  int tri;             // A lower triangular: the sum of a row tile stops at its last row
  const float* B;      // G_s: B(c, k) = B[c ldb + k]
  int64_t ldb;
  int C;               // columns
  float* out;          // column c of the output at out + c ldo
  int64_t ldo;
  int row0;            // F: first output row
  const int32_t* rmap; // G: output row of each row of A
};

__global__ void __launch_bounds__(kThreads) k_ti_apply(TiApply P) {
  __shared__ TiSmem sm;
  const int r0 = blockIdx.x * kT, c0 = blockIdx.y * kT;
  const int ra = min(kT, P.R - r0), cb = min(kT, P.C - c0);
  const int K = P.tri ? min(P.K, r0 + kT) : P.K;
  float acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
  tile_products<false>(acc, P.A + r0, P.lda, ra, P.B + (int64_t)c0 * P.ldb, P.ldb, cb, K, sm);
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int r = 4 * tx + i, c = 4 * ty + j;
      if (r >= ra || c >= cb) continue;
      float* col = P.out + (int64_t)(c0 + c) * P.ldo;
      if (P.rmap) col[P.rmap[r0 + r]] -= acc[i][j];
      else col[P.row0 + r0 + r] = acc[i][j];
    }
}

// packed tile p = I (I + 1) / 2 + J of F^T F: sum over k >= 64 I (F is lower
// triangular) of F(k, 64 I + r) F(k, 64 J + c); the whole tile is written
__global__ void __launch_bounds__(kThreads) k_ti_gram(const float* __restrict__ F, int64_t ldG, int nT,
                                                      float* __restrict__ S) {
  __shared__ TiSmem sm;
  const int64_t p = blockIdx.x;
  int I = (int)((sqrt(8.0 * (double)p + 1.0) - 1.0) * 0.5);
  while ((int64_t)(I + 1) * (I + 2) / 2 <= p) ++I;
  while ((int64_t)I * (I + 1) / 2 > p) --I;
  const int J = (int)(p - (int64_t)I * (I + 1) / 2);
  const int k0 = I * kT;
  float acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
  tile_products<true>(acc, F + (int64_t)I * kT * ldG + k0, ldG, min(kT, nT - I * kT), F + (int64_t)J * kT * ldG + k0,
                      ldG, min(kT, nT - J * kT), nT - k0, sm);
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  float* T = S + p * kT * kT;
#pragma unroll
  for (int j = 0; j < 4; ++j)
    *reinterpret_cast<float4*>(T + (4 * ty + j) * kT + 4 * tx) = make_float4(acc[0][j], acc[1][j], acc[2][j], acc[3][j]);
}

// ---------------------------------------------------------------------------
// The product x_T = S^-1 t_T.  Work unit (a, c): the tiles (I, J) of S^-1 with
// I = 2a + i (i < 2) and J = 4c + j (j < 4), J <= I; each contributes S_IJ t_J to
// rows I and, below the diagonal, S_IJ^T t_I to rows J.  One thread streams the
// unit's tiles (16 KB each, contiguous in the packed layout) with bulk copies
// into a ring of kTiSlots shared-memory slots, one mbarrier each, and refills a
// slot as soon as the block has read it, so that the later tiles are in flight
// while the earlier ones are used; the block meanwhile stages t at its rows and
// columns.  Thread (rq, cs) = (t mod 16, t / 16) reads rows 4 rq .. 4 rq + 3 of
// each tile's columns cs + 16 m (m < 4): its row sums stay in registers across
// the unit's tiles, its column sums are reduced across the 16 threads of a half
// warp after each column of tiles, and the unit's sums go to x by atomic adds (x
// is zero at T before the product).  Every wait is bounded: on expiry the block
// sets the error flag, waits (bounded) for the copies it still has in flight and
// returns.
// ---------------------------------------------------------------------------
constexpr int kTiSlots = 4;
constexpr int kTiRowTiles = kTiUnitRows;   // i
constexpr int kTiColTiles = kTiUnitCols;   // j

__device__ __forceinline__ int top_column(const TopInvDev& T, int p) {
  int q = 0;
  while (q + 1 < T.n_nodes && p >= T.pos[q + 1]) ++q;
  return T.col0[q] + (p - T.pos[q]);
}

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ bool ti_mbar_test(unsigned long long* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
               : "=r"(ok) : "r"(smem_addr(bar)), "r"(parity) : "memory");
  return ok != 0;
}

__device__ __forceinline__ bool ti_mbar_wait(unsigned long long* bar, uint32_t parity, long long limit) {
  long long it = 0;
  while (!ti_mbar_test(bar, parity)) {
    if (++it > limit) return false;
    if (it > 64) __nanosleep(32);
  }
  return true;
}

template <int D>
struct TiProductSmem {
  float ring[kTiSlots][kT * kT];   // tiles in flight; afterwards the per-warp row sums
  float zr[kTiRowTiles][D][kT];    // t at the unit's rows
  float zc[kTiColTiles][D][kT];    // t at the unit's columns
  float colp[kTiColTiles][D][kT];  // column sums
  unsigned long long bar[kTiSlots];
  int ok;
};

// the unit's q-th tile (columns of tiles outer), packed index; nt = its tile count
__device__ __forceinline__ int64_t unit_tile(const TopInvDev& T, int a, int c, int q) {
  for (int j = 0; j < kTiColTiles; ++j)
    for (int i = 0; i < kTiRowTiles; ++i) {
      const int I = kTiRowTiles * a + i, J = kTiColTiles * c + j;
      if (I >= T.tiles_n || J > I) continue;
      if (q-- == 0) return (int64_t)I * (I + 1) / 2 + J;
    }
  return -1;
}

template <int D>
__global__ void __launch_bounds__(kThreads, 3) k_ti_product(TopInvDev T, const float* __restrict__ y,
                                                           float* __restrict__ x) {
  extern __shared__ __align__(128) unsigned char ti_smem_raw[];
  TiProductSmem<D>& S = *reinterpret_cast<TiProductSmem<D>*>(ti_smem_raw);
  float (*red)[kTiRowTiles][D][kT] = reinterpret_cast<float (*)[kTiRowTiles][D][kT]>(&S.ring[0][0]);   // [8 warps]
  const int2 u = T.units[blockIdx.x];
  const int a = u.x, c = u.y;
  const int t = threadIdx.x, rq = t & 15, cs = t >> 4, lane = t & 31, warp = t >> 5;
  int nt = 0;
  for (int j = 0; j < kTiColTiles; ++j)
    for (int i = 0; i < kTiRowTiles; ++i) {
      const int I = kTiRowTiles * a + i, J = kTiColTiles * c + j;
      nt += (I < T.tiles_n && J <= I) ? 1 : 0;
    }
  uint64_t pol = 0;
  auto issue = [&](int q) {   // thread 0: tile q into slot q mod kTiSlots
    unsigned long long* bar = &S.bar[q % kTiSlots];
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}"
                 :: "r"(smem_addr(bar)), "r"((uint32_t)(kT * kT * 4)) : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;"
        :: "r"(smem_addr(&S.ring[q % kTiSlots][0])), "l"(T.tiles + unit_tile(T, a, c, q) * kT * kT),
           "r"((uint32_t)(kT * kT * 4)), "r"(smem_addr(bar)), "l"(pol)
        : "memory");
  };
  if (t == 0) {
    for (int s = 0; s < kTiSlots; ++s)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_addr(&S.bar[s])) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    for (int q = 0; q < nt && q < kTiSlots; ++q) issue(q);
    S.ok = 1;
  }
  for (int e = t; e < (kTiRowTiles + kTiColTiles) * D * kT; e += kThreads) {
    const bool row = e < kTiRowTiles * D * kT;
    const int rem = row ? e : e - kTiRowTiles * D * kT;
    const int i = rem / (D * kT), k = (rem / kT) % D, r = rem % kT;
    const int p = (row ? kTiRowTiles * a : kTiColTiles * c) * kT + i * kT + r;
    const float val = p < T.nT ? __ldcg(y + (int64_t)top_column(T, p) * D + k) : 0.f;
    if (row) S.zr[i][k][r] = val;
    else S.zc[i][k][r] = val;
  }
  for (int e = t; e < kTiColTiles * D * kT; e += kThreads) (&S.colp[0][0][0])[e] = 0.f;
  __syncthreads();
  float racc[kTiRowTiles][4][D];
#pragma unroll
  for (int i = 0; i < kTiRowTiles; ++i)
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int k = 0; k < D; ++k) racc[i][r][k] = 0.f;
  // tiles in the order they were issued, with compile-time (i, j) so that the
  // row sums stay in registers
  int q = 0;
  bool ok = true;
#pragma unroll
  for (int j = 0; j < kTiColTiles; ++j) {
    float zcv[4][D];   // t at this thread's columns of the column of tiles j
#pragma unroll
    for (int m = 0; m < 4; ++m)
#pragma unroll
      for (int k = 0; k < D; ++k) zcv[m][k] = S.zc[j][k][cs + 16 * m];
    float cacc[4][D];
#pragma unroll
    for (int m = 0; m < 4; ++m)
#pragma unroll
      for (int k = 0; k < D; ++k) cacc[m][k] = 0.f;
    bool any_off = false;
#pragma unroll
    for (int i = 0; i < kTiRowTiles; ++i) {
      const int I = kTiRowTiles * a + i, J = kTiColTiles * c + j;
      if (!ok || I >= T.tiles_n || J > I) continue;
      if (t == 0 && !ti_mbar_wait(&S.bar[q % kTiSlots], (uint32_t)((q / kTiSlots) & 1), T.wait_limit)) S.ok = 0;
      __syncthreads();
      if (!S.ok) {
        ok = false;
        continue;
      }
      const bool diag = I == J;
      any_off |= !diag;
      const float* tl = &S.ring[q % kTiSlots][4 * rq];
      float4 zrv[D];   // t at this thread's rows of the row of tiles i
      if (!diag) {
#pragma unroll
        for (int k = 0; k < D; ++k) zrv[k] = *reinterpret_cast<const float4*>(&S.zr[i][k][4 * rq]);
      }
      float4 w[4];
#pragma unroll
      for (int m = 0; m < 4; ++m) w[m] = *reinterpret_cast<const float4*>(tl + (cs + 16 * m) * kT);
      __syncthreads();   // the slot is read: refill it
      if (t == 0 && q + kTiSlots < nt) issue(q + kTiSlots);
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        const float wm[4] = {w[m].x, w[m].y, w[m].z, w[m].w};
#pragma unroll
        for (int k = 0; k < D; ++k) {
#pragma unroll
          for (int r = 0; r < 4; ++r) racc[i][r][k] = fmaf(wm[r], zcv[m][k], racc[i][r][k]);
          if (!diag)
            cacc[m][k] = fmaf(wm[0], zrv[k].x, fmaf(wm[1], zrv[k].y, fmaf(wm[2], zrv[k].z, fmaf(wm[3], zrv[k].w, cacc[m][k]))));
        }
      }
      ++q;
    }
    if (any_off) {
#pragma unroll
      for (int m = 0; m < 4; ++m)
#pragma unroll
        for (int k = 0; k < D; ++k) {
          float s = cacc[m][k];
          s += __shfl_xor_sync(0xffffffffu, s, 1);
          s += __shfl_xor_sync(0xffffffffu, s, 2);
          s += __shfl_xor_sync(0xffffffffu, s, 4);
          s += __shfl_xor_sync(0xffffffffu, s, 8);
          if (rq == 0) S.colp[j][k][cs + 16 * m] = s;
        }
    }
  }
  if (!ok) {
    if (t == 0) {
      atomicExch(T.err, 1);
      // the copies issued and not yet waited for still land in this block's memory
      for (int r = q; r < nt && r < q + kTiSlots; ++r)
        ti_mbar_wait(&S.bar[r % kTiSlots], (uint32_t)((r / kTiSlots) & 1), T.wait_limit);
    }
    return;
  }
  __syncthreads();   // every tile is read: the ring takes the row sums
  // row sums: the two half warps of a warp, then the eight warps
#pragma unroll
  for (int i = 0; i < kTiRowTiles; ++i)
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int k = 0; k < D; ++k) {
        const float s = racc[i][r][k] + __shfl_xor_sync(0xffffffffu, racc[i][r][k], 16);
        if (lane < 16) red[warp][i][k][4 * rq + r] = s;
      }
  __syncthreads();
  for (int e = t; e < kTiRowTiles * D * kT; e += kThreads) {
    const int i = e / (D * kT), k = (e / kT) % D, r = e % kT;
    float s = 0.f;
#pragma unroll
    for (int w = 0; w < 8; ++w) s += red[w][i][k][r];
    const int pr = (kTiRowTiles * a + i) * kT + r;
    if (pr < T.nT) atomicAdd(x + (int64_t)top_column(T, pr) * D + k, s);
  }
  for (int e = t; e < kTiColTiles * D * kT; e += kThreads) {
    const int j = e / (D * kT), k = (e / kT) % D, r = e % kT;
    const int pc = (kTiColTiles * c + j) * kT + r;
    const float s = S.colp[j][k][r];
    if (pc < T.nT && s != 0.f) atomicAdd(x + (int64_t)top_column(T, pc) * D + k, s);
  }
}

}  // namespace

cudaError_t compute_top_inverse(const TopInvSetup& U, const float* blocks, float* tiles, cudaStream_t s) {
  const size_t work = (size_t)U.ldG * U.nT * sizeof(float);
  float *G = nullptr, *F = nullptr;
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(&G), work);
  if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&F), work);
  if (e == cudaSuccess) e = cudaMemsetAsync(G, 0, work, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(F, 0, work, s);
  if (e == cudaSuccess) {
    k_ti_eye<<<(U.nT + 255) / 256, 256, 0, s>>>(G, U.ldG, U.nT);
    for (size_t q = 0; q < U.pos.size(); ++q) {
      const int ns = U.ncol[q], pos = U.pos[q], lo = U.lo[q];
      const int C = pos + ns - lo;
      TiApply P{};
      P.lda = U.ld[q];
      P.K = ns;
      P.B = G + (int64_t)lo * U.ldG + pos;
      P.ldb = U.ldG;
      P.C = C;
      P.ldo = U.ldG;
      // F_s = inv(L_ss) G_s
      P.A = blocks + U.blk_off[q];
      P.R = ns;
      P.tri = 1;
      P.out = F + (int64_t)lo * U.ldG;
      P.row0 = pos;
      P.rmap = nullptr;
      k_ti_apply<<<dim3((ns + kT - 1) / kT, (C + kT - 1) / kT), kThreads, 0, s>>>(P);
      // G_r -= (L_rs inv(L_ss)) G_s at the structure rows
      if (U.nrow[q] > 0) {
        P.A = blocks + U.blk_off[q] + ns;
        P.R = U.nrow[q];
        P.tri = 0;
        P.out = G + (int64_t)lo * U.ldG;
        P.row0 = 0;
        P.rmap = U.rmap + U.rmap_off[q];
        k_ti_apply<<<dim3((U.nrow[q] + kT - 1) / kT, (C + kT - 1) / kT), kThreads, 0, s>>>(P);
      }
    }
    const int64_t n_tiles = (int64_t)U.tiles * (U.tiles + 1) / 2;
    k_ti_gram<<<(unsigned)n_tiles, kThreads, 0, s>>>(F, U.ldG, U.nT, tiles);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  }
  if (G) cudaFree(G);
  if (F) cudaFree(F);
  return e;
}

}  // namespace ffa

namespace ffa {

void launch_top_product(const TopInvDev& T, int d, const float* y, float* x, cudaStream_t s) {
  const unsigned grid = (unsigned)T.n_units;
  if (d == 2) k_ti_product<2><<<grid, kThreads, sizeof(TiProductSmem<2>), s>>>(T, y, x);
  else k_ti_product<3><<<grid, kThreads, sizeof(TiProductSmem<3>), s>>>(T, y, x);
}

// three blocks per SM (3 x 70 KB of shared memory) need the largest carveout
cudaError_t prepare_top_product() {
  cudaError_t e = cudaFuncSetAttribute(k_ti_product<2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)sizeof(TiProductSmem<2>));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_ti_product<3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sizeof(TiProductSmem<3>));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_ti_product<2>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxShared);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_ti_product<3>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxShared);
  return e;
}

}  // namespace ffa
