// Context-free energy evaluation that allocates no memory.
//
// Some callers cannot call cudaMalloc: code running under a custom or frozen
// allocator, inside a memory pool that must not grow, or in a host process that
// only receives device buffers from elsewhere.  ffa_energy_noalloc serves them:
// it needs no context (no setup, no factorization) and writes the energy of
// a map into a caller-provided location.  Its per-block partial sums live in a
// file-scope static device array of fixed size instead of allocated scratch.
//
// The array is shared by every call on a device and keeps the last call's
// contents; each call overwrites exactly the slots it then reads, so nothing
// needs clearing, but calls that overlap on the GPU (different streams, or
// host threads calling concurrently) race on it.
//
// Invalid meshes are reported through the result, because the call only
// enqueues work and never waits for it: an element with a vertex index outside
// [0, n) is skipped before any load through that index, and a source element of
// zero (or non-finite) measure is not evaluated; either makes *E a NaN, where a
// valid mesh with a flipped element gives +infinity.
#include <cuda_runtime.h>

#include <cmath>
#include <string>

#include "ffa_internal.h"

namespace {

constexpr int kNaBlock = 256;
constexpr int kNaMaxBlocks = 1 << 16;  // 65,536 blocks -> up to 16,777,216 elements

constexpr int kNaSlots = 3;
// three doubles per block: sum of w_i f(J_i) over unflipped elements, flip count,
// invalid elements (an index outside [0, n) or a source element of zero measure)
static __device__ __align__(256) double g_na_partials[kNaSlots * kNaMaxBlocks];

// Per element: source edge matrix in the element frame (intrinsic for a triangle
// in R^3), hat gradients as the columns of its inverse, J = G W with column k
// the gradient of target coordinate k, then w f(J) (Supplemental "Computing the
// Jacobian Map"; eq. genericdeformationenergy with eq. symmetricdirichletdefiningfunction
// or eq. symmetricgradientdefiningfunction).
enum NaResult { kNaValue = 0, kNaFlipped = 1, kNaInvalid = 2 };

template <int D>
__device__ NaResult na_element(int n, int d_in, const double* __restrict__ V, const int32_t* __restrict__ T,
                               const double* __restrict__ W, int i, int energy, double& wf) {
  const int32_t* t = T + (int64_t)i * (D + 1);
  // every index is checked before anything is loaded through it
  for (int j = 0; j <= D; ++j)
    if (t[j] < 0 || t[j] >= n) return kNaInvalid;
  double E[D][D];
  const double* v0 = V + (int64_t)t[0] * d_in;
  if (d_in == D) {
    for (int j = 0; j < D; ++j)
      for (int a = 0; a < D; ++a) E[j][a] = V[(int64_t)t[j + 1] * d_in + a] - v0[a];
  } else {
    // D == 2, d_in == 3
    const double* v1 = V + (int64_t)t[1] * 3;
    const double* v2 = V + (int64_t)t[2] * 3;
    const double a0 = v1[0] - v0[0], a1 = v1[1] - v0[1], a2 = v1[2] - v0[2];
    const double b0 = v2[0] - v0[0], b1 = v2[1] - v0[1], b2 = v2[2] - v0[2];
    const double la = sqrt(a0 * a0 + a1 * a1 + a2 * a2);
    double n0 = a1 * b2 - a2 * b1, n1 = a2 * b0 - a0 * b2, n2 = a0 * b1 - a1 * b0;
    const double ln = sqrt(n0 * n0 + n1 * n1 + n2 * n2);
    n0 /= ln; n1 /= ln; n2 /= ln;
    const double e10 = a0 / la, e11 = a1 / la, e12 = a2 / la;
    const double e20 = n1 * e12 - n2 * e11, e21 = n2 * e10 - n0 * e12, e22 = n0 * e11 - n1 * e10;
    E[0][0] = la;
    E[0][1] = 0.0;
    E[1][0] = b0 * e10 + b1 * e11 + b2 * e12;
    E[1][1] = b0 * e20 + b1 * e21 + b2 * e22;
  }
  double Ei[D][D], detE;
  if (D == 2) {
    detE = E[0][0] * E[1][1] - E[0][1] * E[1][0];
    Ei[0][0] = E[1][1] / detE; Ei[0][1] = -E[0][1] / detE; Ei[1][0] = -E[1][0] / detE; Ei[1][1] = E[0][0] / detE;
  } else {
    const double c00 = E[1][1] * E[2][2] - E[1][2] * E[2][1];
    const double c01 = E[1][2] * E[2][0] - E[1][0] * E[2][2];
    const double c02 = E[1][0] * E[2][1] - E[1][1] * E[2][0];
    detE = E[0][0] * c00 + E[0][1] * c01 + E[0][2] * c02;
    Ei[0][0] = c00 / detE; Ei[1][0] = c01 / detE; Ei[2][0] = c02 / detE;
    Ei[0][1] = (E[0][2] * E[2][1] - E[0][1] * E[2][2]) / detE;
    Ei[1][1] = (E[0][0] * E[2][2] - E[0][2] * E[2][0]) / detE;
    Ei[2][1] = (E[0][1] * E[2][0] - E[0][0] * E[2][1]) / detE;
    Ei[0][2] = (E[0][1] * E[1][2] - E[0][2] * E[1][1]) / detE;
    Ei[1][2] = (E[0][2] * E[1][0] - E[0][0] * E[1][2]) / detE;
    Ei[2][2] = (E[0][0] * E[1][1] - E[0][1] * E[1][0]) / detE;
  }
  const double w = fabs(detE) / (D == 2 ? 2.0 : 6.0);
  if (!(w > 0.0) || !isfinite(w)) return kNaInvalid;   // zero-measure source element (or NaN frame)
  // J[a][k] = sum_j g_j[a] (W_j - W_0)[k], g_j[a] = Ei[a][j-1]
  double J[D][D];
  const double* w0 = W + (int64_t)t[0] * D;
  for (int a = 0; a < D; ++a)
    for (int k = 0; k < D; ++k) J[a][k] = 0.0;
  for (int j = 0; j < D; ++j) {
    const double* wj = W + (int64_t)t[j + 1] * D;
    for (int k = 0; k < D; ++k) {
      const double del = wj[k] - w0[k];
      for (int a = 0; a < D; ++a) J[a][k] += Ei[a][j] * del;
    }
  }
  double det, fro = 0.0, fri = 0.0;
  if (D == 2) {
    det = J[0][0] * J[1][1] - J[0][1] * J[1][0];
    fri = (J[0][0] * J[0][0] + J[0][1] * J[0][1] + J[1][0] * J[1][0] + J[1][1] * J[1][1]) / (det * det);
  } else {
    const double c00 = J[1][1] * J[2][2] - J[1][2] * J[2][1];
    const double c01 = J[1][2] * J[2][0] - J[1][0] * J[2][2];
    const double c02 = J[1][0] * J[2][1] - J[1][1] * J[2][0];
    const double c10 = J[0][2] * J[2][1] - J[0][1] * J[2][2];
    const double c11 = J[0][0] * J[2][2] - J[0][2] * J[2][0];
    const double c12 = J[0][1] * J[2][0] - J[0][0] * J[2][1];
    const double c20 = J[0][1] * J[1][2] - J[0][2] * J[1][1];
    const double c21 = J[0][2] * J[1][0] - J[0][0] * J[1][2];
    const double c22 = J[0][0] * J[1][1] - J[0][1] * J[1][0];
    det = J[0][0] * c00 + J[0][1] * c01 + J[0][2] * c02;
    fri = (c00 * c00 + c01 * c01 + c02 * c02 + c10 * c10 + c11 * c11 + c12 * c12 + c20 * c20 + c21 * c21 +
           c22 * c22) / (det * det);
  }
  for (int a = 0; a < D; ++a)
    for (int k = 0; k < D; ++k) fro += J[a][k] * J[a][k];
  if (!(det > 0.0)) return kNaFlipped;
  wf = w * (energy == FFA_SYM_DIRICHLET ? 0.5 * (fro + fri) : 0.5 * fro - log(det));
  return kNaValue;
}

template <int D>
__global__ void __launch_bounds__(kNaBlock) k_na_energy(int n, int m, int d_in, const double* __restrict__ V,
                                                        const int32_t* __restrict__ T, const double* __restrict__ W,
                                                        int energy, double* __restrict__ partials) {
  const int i = blockIdx.x * kNaBlock + threadIdx.x;
  double q[kNaSlots] = {0.0, 0.0, 0.0};   // energy, flips, invalid elements
  if (i < m) {
    double wf = 0.0;
    const NaResult r = na_element<D>(n, d_in, V, T, W, i, energy, wf);
    if (r == kNaValue) q[0] = wf;
    else if (r == kNaFlipped) q[1] = 1.0;
    else q[2] = 1.0;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
#pragma unroll
    for (int k = 0; k < kNaSlots; ++k) q[k] += __shfl_xor_sync(0xffffffffu, q[k], o);
  __shared__ double red[kNaSlots][kNaBlock / 32];
  if ((threadIdx.x & 31) == 0)
#pragma unroll
    for (int k = 0; k < kNaSlots; ++k) red[k][threadIdx.x >> 5] = q[k];
  __syncthreads();
  if (threadIdx.x < kNaSlots) {
    double s = 0.0;
    for (int w = 0; w < kNaBlock / 32; ++w) s += red[threadIdx.x][w];
    partials[kNaSlots * (int64_t)blockIdx.x + threadIdx.x] = s;
  }
}

__global__ void k_na_finish(const double* __restrict__ partials, int nblocks, double* __restrict__ E) {
  double q[kNaSlots] = {0.0, 0.0, 0.0};
  for (int b = threadIdx.x; b < nblocks; b += blockDim.x)
#pragma unroll
    for (int k = 0; k < kNaSlots; ++k) q[k] += partials[kNaSlots * (int64_t)b + k];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
#pragma unroll
    for (int k = 0; k < kNaSlots; ++k) q[k] += __shfl_xor_sync(0xffffffffu, q[k], o);
  __shared__ double red[kNaSlots][32];
  if ((threadIdx.x & 31) == 0)
#pragma unroll
    for (int k = 0; k < kNaSlots; ++k) red[k][threadIdx.x >> 5] = q[k];
  __syncthreads();
  if (threadIdx.x == 0) {
    double t[kNaSlots] = {0.0, 0.0, 0.0};
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w)
#pragma unroll
      for (int k = 0; k < kNaSlots; ++k) t[k] += red[k][w];
    *E = t[2] > 0.5 ? NAN : (t[1] > 0.5 ? INFINITY : t[0]);
  }
}

ffa_status na_fail(const char* msg, ffa_status st) {
  ffa::set_thread_error(msg);
  return st;
}

}  // namespace

extern "C" {

ffa_status ffa_energy_noalloc(int32_t n, int32_t m, int32_t d, int32_t d_in, const double* V, const int32_t* T,
                              const double* W, ffa_energy_kind energy, double* E, void* stream) {
  if (d != 2 && d != 3) return na_fail("d must be 2 or 3", FFA_ERR_INVALID_ARG);
  if (d_in < d || d_in > 3) return na_fail("d_in must be in [d, 3]", FFA_ERR_INVALID_ARG);
  if (n < d + 1 || m < 1) return na_fail("need n >= d+1 and m >= 1", FFA_ERR_INVALID_ARG);
  if (m > kNaMaxBlocks * kNaBlock)
    return na_fail("m exceeds the 16,777,216 elements that the static scratch of ffa_energy_noalloc covers",
                   FFA_ERR_INVALID_ARG);
  if (!V || !T || !W || !E) return na_fail("a pointer argument is NULL", FFA_ERR_INVALID_ARG);
  if (energy != FFA_SYM_DIRICHLET && energy != FFA_SYM_GRADIENT) return na_fail("unknown energy", FFA_ERR_INVALID_ARG);
  // an error left pending by earlier work on this thread is reported as its own
  // and left in place for its owner
  const cudaError_t pending = cudaPeekAtLastError();
  if (pending != cudaSuccess)
    return na_fail((std::string("a CUDA error was pending before the call: ") + cudaGetErrorString(pending)).c_str(),
                   FFA_ERR_CUDA);
  // the device address of the static array on the current device (its host-side
  // name is only a stand-in); looked up on every call, so it follows the current
  // device and survives a device reset.  The first call on a device loads the
  // library's device code there, so make it before any stream capture.
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, g_na_partials) != cudaSuccess || !p) {
    cudaGetLastError();
    return na_fail("cudaGetSymbolAddress of the static scratch failed", FFA_ERR_CUDA);
  }
  double* scratch = static_cast<double*>(p);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int nb = (m + kNaBlock - 1) / kNaBlock;
  if (d == 2) k_na_energy<2><<<nb, kNaBlock, 0, s>>>(n, m, d_in, V, T, W, (int)energy, scratch);
  else k_na_energy<3><<<nb, kNaBlock, 0, s>>>(n, m, d_in, V, T, W, (int)energy, scratch);
  k_na_finish<<<1, 1024, 0, s>>>(scratch, nb, E);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess)
    return na_fail((std::string("kernel launch failed: ") + cudaGetErrorString(e)).c_str(), FFA_ERR_CUDA);
  return FFA_OK;
}

}  // extern "C"
