// Host-side preparation of the fixed W-step operator (paper Sec. 4, "Efficient
// evaluation": L does not change while the penalties do not, so it is decomposed
// once and only back-substitution runs per iteration; Algorithm 2, decompose(L)).
//
// The free-vertex block L_FF of L = sum_i mu_i G_i^T G_i (eq. solvinginw) is ordered by
// geometric nested dissection and factored by a multifrontal Cholesky in double.
// Every supernode s (a separator or a leaf block) stores one dense block
//     B_s = [ inv(L_ss) ; L_rs inv(L_ss) ]     ((n_s + m_s) x n_s, column-major,
//                                               zero-padded to ld rows)
// so that the forward solve is  z_s = inv(L_ss) y_s,  y_r -= (L_rs inv(L_ss)) y_s
// and the backward solve is     x_s = inv(L_ss)^T z_s - (L_rs inv(L_ss))^T x_r:
// both passes become dense matrix-vector products that the GPU runs in parallel.
#pragma once

#include <cstdint>
#include <functional>
#include <string>
#include <vector>

namespace ffa {

// Runs worker(0) on the calling thread and worker(1 .. count-1) on new threads,
// then joins every thread that was started, also when starting one fails.  An
// exception thrown by any worker (or by starting a thread) is rethrown on the
// calling thread after the joins, so no joinable thread is ever destroyed and no
// exception escapes a thread.
void run_threads(int count, const std::function<void(int)>& worker);

struct Supernode {
  int32_t col0 = 0;     // first column in the eliminated order
  int32_t ncol = 0;     // n_s
  int32_t nrow = 0;     // m_s: rows below the diagonal block (the structure)
  int32_t parent = -1;
  int32_t level = 0;    // 0 = leaf; 1 + max(children) otherwise
  int32_t ld = 0;       // leading dimension of B_s: n_s + m_s rounded up to 4 (16-byte columns)
  int64_t row_off = 0;  // offset of the structure in Factor::rows
  int64_t blk_off = 0;  // offset of B_s in Factor::blocks (a multiple of 4 floats)
};

struct Factor {
  int32_t nF = 0;
  std::vector<int32_t> perm;   // eliminated position -> free index
  std::vector<int32_t> iperm;  // free index -> eliminated position
  std::vector<Supernode> nodes;  // postorder: children before parents
  std::vector<int32_t> rows;     // concatenated structures (eliminated numbering)
  std::vector<float> blocks;     // B_s in float, column-major, leading dimension ld
  std::vector<double> blocks64;  // B_s in double (kept only on request), same layout
  int32_t n_levels = 0;
  int64_t flops = 0;
  double t_analyze = 0.0, t_factor = 0.0;
};

struct FactorInput {
  int32_t nF = 0;
  const int64_t* Ap = nullptr;   // CSR of L_FF (full symmetric pattern), free numbering
  const int32_t* Ai = nullptr;
  const double* Ax = nullptr;
  const double* coords = nullptr;  // nF x 3 source positions (d_in = 2 padded with 0)
  int32_t leaf_size = 64;
  int32_t threads = 0;             // 0 = hardware concurrency
  bool keep_double = false;
  bool numeric = true;             // false: analysis only (the blocks are computed on the device)
};

// Returns 0 on success, 3 if L_FF is not positive definite, 1 on bad input.
int build_factor(const FactorInput& in, Factor& f, std::string& err);

// New values on the same pattern (the penalties changed, the mesh did not): the
// ordering and the supernode structure of f are kept and only the blocks are
// recomputed.  Same return codes.
int refactor(const FactorInput& in, Factor& f, std::string& err);

// Double-precision host application of the factor (setup diagnostics only):
// x = L_FF^{-1} b for nrhs interleaved right-hand sides, eliminated numbering
// handled internally (b and x in free numbering).  Needs keep_double.
void host_solve(const Factor& f, const double* b, double* x, int nrhs);

}  // namespace ffa
