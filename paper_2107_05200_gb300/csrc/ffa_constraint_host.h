// Host-only parts of the general constraints A W = b (Sec. 4, W update): the
// split of A into its free and pinned parts and the inverse of the Schur
// complement S = A_F L_FF^-1 A_F^T.
#pragma once

#include <cstdint>
#include <vector>

namespace ffa {

struct ConstraintSplit {
  std::vector<int64_t> fptr;  // c + 1: rows of A_F
  std::vector<int32_t> fcol;  // eliminated index of the free vertex, ascending per row
  std::vector<double> fval;   // entries; repeated columns of a row summed
  struct PinEntry { int32_t row, slot; double val; };
  std::vector<PinEntry> pin;  // entries on pinned vertices (slot = index into the pins)
};

// A (c x n CSR over vertices, indices already checked to lie in [0, n)) split by
// v2e (vertex -> eliminated index, -1 for a pinned vertex) and slot_of (vertex ->
// pin slot).
void split_constraints(int c, const int64_t* ptr, const int32_t* col, const double* val,
                       const std::vector<int32_t>& v2e, const std::vector<int32_t>& slot_of, ConstraintSplit& out);

// Sinv = S^-1 for the symmetric c x c S (row-major; its two triangles averaged) by
// Cholesky.  Returns -1, or the first row whose pivot fell to 1e-10 of its
// diagonal (or whose diagonal is not positive): that row is, to that tolerance,
// a combination of the rows before it once the pins are eliminated.
int schur_inverse(int c, const std::vector<double>& S, std::vector<double>& Sinv);

}  // namespace ffa
