// Device side of the W-step decomposition and of the device assembly of L
// (ffa_devfactor.h): the device copies of a plan and the two launchers.
#pragma once

#include <cuda_runtime.h>

#include <vector>

#include "ffa_devfactor.h"

namespace ffa {

struct DevFactorDev {
  const DfNode* nodes = nullptr;
  const int64_t* rel_off = nullptr;
  const int32_t* rel = nullptr;
  const DfItem* items = nullptr;
  const int64_t* orig_dst = nullptr;  // per ELL slot of L_FF
  void* F = nullptr;                  // fronts (float or double)
  void* Lv = nullptr;                 // inv(L_ss) of every supernode (float or double)
  int32_t* err = nullptr;             // set to 1 when a pivot is not positive and finite
  int fp64 = 0;
  int64_t front_elems = 0, linv_elems = 0, n_slots = 0;
};

// The whole decomposition on stream s: fronts and inverses cleared, L_FF
// (ell_val, the double ELL of the residual) scattered, then every launch of prog;
// the float blocks of every supernode are overwritten (padding rows untouched).
cudaError_t launch_devfactor(const DevFactorDev& D, const std::vector<DfLaunch>& prog, const double* ell_val,
                             float* blocks, cudaStream_t s);

struct DevAssemblyDev {
  const int64_t* ell_ptr = nullptr;
  const int32_t* ell_src = nullptr;
  int64_t n_ell = 0;                 // width * nF
  const int64_t* fc_ptr = nullptr;
  const int32_t* fc_src = nullptr;
  const int32_t* cf_src = nullptr;
  int64_t n_fc = 0;
  const double* g = nullptr;         // m x d x d hat gradients in double
};

// L_FF (ELL values), L_FC and L_CF from the penalties mu (double, device)
cudaError_t launch_device_assembly(const DevAssemblyDev& A, int d, const double* mu, double* ell_val, double* fc_val,
                                   double* cf_val, cudaStream_t s);

}  // namespace ffa
