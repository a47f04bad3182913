// Host-side assembly of the W-step operator: element geometry (the hat-function
// gradients and measures of each element) and L = sum_i mu_i G_i^T G_i restricted
// to the free vertices, with its device forms.
#pragma once

#include <cstdint>
#include <vector>

#include "ffa_factor.h"

namespace ffa {

// What the host keeps to assemble L = sum mu_i G_i^T G_i again for new penalties
// (the paper's penalty schedule).
struct OperatorHost {
  int n = 0, m = 0, d = 0, nF = 0, n_pin = 0;
  std::vector<double> g;            // m x d x d hat gradients of local vertices 1..d
  std::vector<int32_t> T;           // m x (d+1)
  std::vector<int64_t> inc_ptr;     // incidences per vertex (CSR over all vertices)
  std::vector<int32_t> inc;         // element * (d+1) + slot
  std::vector<int32_t> free_of, free_vertex, v2pin;
  std::vector<double> coords;       // nF x 3 source positions of the free vertices
  Factor fac;                       // ordering and supernode structure (blocks released after upload)
  std::vector<double> mu;           // the current penalties
};

// Element frames and P1 hat-function gradients (Supplemental, "Computing the
// Jacobian map"): E has rows v_j - v_0 in the element frame (the intrinsic frame
// e1 = (v1-v0)/|v1-v0|, e2 = n x e1 for a triangle in R^3); the gradient of the
// hat function of vertex j is column j of E^{-1}; w = |det E| / d!.
bool element_geometry(int d, int d_in, const double* V, const int32_t* t, double g[3][3], double& w);

// Rows of L = sum_i mu_i G_i^T G_i (eq. solvinginw) for the free vertices: the
// free-free block in free numbering with sorted columns (Ap, Ai, Ax) and the
// free-pinned block by pin slot (Cp, Ci, Cx).  The pattern depends on the mesh
// only, so new penalties give new values in the same positions.
void assemble_operator(const OperatorHost& H, const double* mu, std::vector<int64_t>& Ap, std::vector<int32_t>& Ai,
                       std::vector<double>& Ax, std::vector<int64_t>& Cp, std::vector<int32_t>& Ci,
                       std::vector<double>& Cx);

// The device forms of the operator in elimination order: L_FF as column-major ELL
// (the double residual), L_FC as CSR by free row (the pin right-hand side) and
// L_CF as CSR by pin (the adjoint's pin term).
struct OperatorArrays {
  int width = 1;
  std::vector<int32_t> ell_col;
  std::vector<double> ell_val;
  std::vector<int64_t> fc_ptr;
  std::vector<int32_t> fc_col;
  std::vector<double> fc_val;
  std::vector<int64_t> cf_ptr;
  std::vector<int32_t> cf_row;
  std::vector<double> cf_val;
};

void operator_arrays(const Factor& fac, int nF, int n_pin, const std::vector<int64_t>& Ap,
                     const std::vector<int32_t>& Ai, const std::vector<double>& Ax, const std::vector<int64_t>& Cp,
                     const std::vector<int32_t>& Ci, const std::vector<double>& Cx, OperatorArrays& A);

}  // namespace ffa
