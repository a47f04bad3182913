// Device side of the top-of-tree inverse (ffa_topinv.h): the buffers the solve
// reads, the setup after a decomposition, and the product x_T = S^-1 t_T.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "ffa_topinv.h"

namespace ffa {

// what the product needs (plain values: the struct is a kernel argument)
struct TopInvDev {
  const float* tiles = nullptr;   // packed lower tiles of S^-1 (tile_bytes)
  int32_t* err = nullptr;         // set to 1 if a wait for the tiles' copies ran out
  long long wait_limit = 0;       // polls of that wait
  const int2* units = nullptr;    // the product's work units (a, c): rows of 2 tiles x columns of 4 tiles
  int32_t n_units = 0;
  int32_t nT = 0, tiles_n = 0, nblk = 0;
  int32_t n_nodes = 0;            // T supernodes: T positions [pos, pos + n) are columns [col0, col0 + n)
  int32_t pos[kTiMaxNodes], col0[kTiMaxNodes], n[kTiMaxNodes];
};

// what the setup needs, besides the factor blocks (device: rmap; host: the rest)
struct TopInvSetup {
  int32_t nT = 0, ldG = 0, tiles = 0;
  std::vector<int32_t> ncol, ld, pos, lo, nrow;
  std::vector<int64_t> blk_off, rmap_off;
  const int32_t* rmap = nullptr;   // device copy of TopInvPlan::rmap
};

// S^-1 of the current blocks into T.tiles (which the caller owns); allocates and
// frees two nT x nT float work arrays on the stream's device; synchronous
cudaError_t compute_top_inverse(const TopInvSetup& U, const float* blocks, float* tiles, cudaStream_t s);

// x at the T columns += S^-1 (y at the T columns); y and x are n x d, d = 2 or 3
void launch_top_product(const TopInvDev& T, int d, const float* y, float* x, cudaStream_t s);
// enables the product kernels' shared memory (above the default limit); once,
// before any launch or graph capture
cudaError_t prepare_top_product();

}  // namespace ffa
