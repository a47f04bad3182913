// Internal interfaces between the C ABI (ffa_api.cu) and the CUDA kernels.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/ffadmm.h"
#include "ffa_factor.h"
#include "ffa_schedule.h"
#include "ffa_topinv_launch.h"

namespace ffa {

// Quantities reduced by the local step on check iterations (FP64 partials per block).
enum { Q_EPRIM = 0, Q_EDUAL, Q_GW, Q_P, Q_ENERGY, Q_FLIPS, Q_NONFINITE, NQ };
// Quantities reduced by the vertex gathers.
enum { QV_GTL = 0, QV_NUM, QV_DEN, NQV };

// defining functions (the values of ffa_energy_kind) and, for batches, the
// per-element choice
constexpr int kEnSD = 0;      // symmetric Dirichlet
constexpr int kEnSG = 1;      // symmetric gradient
constexpr int kEnSA = 2;      // symmetric ARAP
constexpr int kEnMixed = 3;   // per element, from energy_of[i]

constexpr int kLocalBlock = 128;
constexpr int kVertexBlock = 256;
constexpr int kGatherLanes = 4;   // lanes sharing one row of the vertex gathers
// (the supernodal-solve task shapes, Task, NodeDev and the schedule records
// are in ffa_schedule.h)

// A dynamic pass as the device sees it: the PassSchedule arrays of
// ffa_schedule.h (push and kids as 16-byte vectors) plus its working state.
struct DynPass {
  const Task* tasks = nullptr;
  int n_tasks = 0, n_init = 0;
  const int4* push = nullptr;
  const int4* kids = nullptr;   // backward only
  const int32_t* q_init = nullptr;
  const int32_t* pending_init = nullptr;   // forward only
  int32_t* queue = nullptr;     // n_tasks slots
  int32_t* pending = nullptr;   // forward: per node
  int32_t* done = nullptr;      // backward: per node, tasks finished
  int32_t* ctr = nullptr;       // [0] next slot to claim, [1] next slot to fill
};


// Element state.  Real-typed arrays are float or double depending on the
// precision of the local step; all are structure-of-arrays with stride m,
// except contrib (m x (d+1) x d, element-major).
struct ElemBufs {
  int32_t* idx = nullptr;  // (d+1) x m
  void* g = nullptr;       // d*d x m  (hat gradients of vertices 1..d)
  void* w = nullptr;       // m
  void* mu = nullptr;      // m
  void* P = nullptr;       // d(d+1)/2 x m  (00,01,11 | 00,01,02,11,12,22)
  void* Lam = nullptr;     // d*d x m  (row-major entries)
  void* U = nullptr;       // 2 x m (cos, sin) for d = 2, 4 x m quaternion for d = 3
  void* contrib = nullptr;   // m x (d+1) x d : g_j . r_i  (W-step right-hand side terms)
  void* contrib2 = nullptr;  // m x (d+1) x d : g_j . Lambda_i (check iterations) / energy gradient
  // batched meshes (null for a single mesh)
  const int8_t* energy_of = nullptr;   // m: 0 = SD, 1 = SG (kernels instantiated with EN = 2)
  const int32_t* mesh_of = nullptr;    // m: mesh of each element
  double* mesh_acc = nullptr;          // n_mesh x (NQ + 1) per-mesh sums of the check quantities
  double* mesh_part = nullptr;         // blocks x 2 x NQ: sums of each block's first and last mesh
  int32_t joint = 0;                   // 1: the joint (U, P) prox variant of the local step
  void* hmu = nullptr;                 // m: h_i / mu_i of the proximal U term (null: h = 0)
};

struct LocalLaunch {
  int d, energy, fp64, check;
  int m;
  int block;          // threads per block of the local step (64, 128 or 256; 0 = 128)
  ElemBufs e;
  const void* vrec;   // vertex records
  double* partials;   // [blocks][NQ]
  int64_t n_blocks;
};

void launch_local_step(const LocalLaunch& L, cudaStream_t s);
void launch_init_polar(const LocalLaunch& L, cudaStream_t s);
// h_i / mu_i of the proximal U term at the bound of Prop. 1 from the current P:
// 4 w_i^2 B_i^2 / mu_i^2, B_i^2 = 5 (1 + |grad f(P_i)|^2) (single-energy contexts)
void launch_prox_weight(const LocalLaunch& L, cudaStream_t s);
// W-step right-hand-side terms from the stored U, P, Lambda (after a state restore)
void launch_rhs_terms(const LocalLaunch& L, cudaStream_t s);
// the paper's penalty schedule: mode 0 mu = max(mu_min(P), w) after the polar
// initialization, mode 1 the rescaling after an iteration (mu and Lambda updated,
// mu64 = the penalties in double); single-energy contexts only
void launch_penalty(const LocalLaunch& L, int mode, double* mu64, double rho, cudaStream_t s);
// energy (mode 0: sum w f(J) + flips into partials) or gradient terms (mode 1: contrib2)
void launch_energy_terms(const LocalLaunch& L, int mode, cudaStream_t s);

// vertex records from W (double, n x d) and the previous W; also writes W_out.
struct VertexLaunch {
  int d, fp64;
  int n;
  const double* Wnew_free;   // eliminated-order values of the free vertices (nF x d) or null
  const float* corr;         // eliminated-order correction added to Wnew_free (or null)
  const int32_t* v2e;        // vertex -> eliminated index (-1 if pinned)
  const int32_t* v2pin;      // vertex -> pin slot (-1 if free)
  const double* pin_pos;     // n_pin x d
  const double* W_in;        // full W (n x d) used instead of the free/pinned sources if non-null
  double* W;                 // n x d: current W, overwritten with the new W
  double* X;                 // eliminated-order free W (nF x d) to keep in sync, or null
  void* vrec;                // records written
  int write_dw;              // 1: dW = new - old; 0: dW = 0
};
void launch_vertex_update(const VertexLaunch& V, cudaStream_t s);

// General linear constraints on the free vertices after the pinned ones are
// eliminated: A_F W_F = b' (c rows, CSR over eliminated indices).  With
// Z = L_FF^-1 A_F^T (nF x c, row-major) and S^-1 = (A_F Z)^-1 (c x c), the W step's
// unconstrained solution X is projected onto the constraints:
// X <- X - Z S^-1 (A_F X - b'), the exact constrained minimizer.
constexpr int kMaxConstraints = 256;
struct ConstraintLaunch {
  int d = 0, c = 0, nF = 0;
  const int64_t* ptr = nullptr;
  const int32_t* col = nullptr;
  const double* val = nullptr;
  const double* bprime = nullptr;   // c x d
  const double* Sinv = nullptr;     // c x c
  const double* Z = nullptr;        // c x nF (column r of L_FF^-1 A_F^T contiguous)
  double* nu = nullptr;             // c x d: S^-1 (A_F X - b')
  double* X = nullptr;              // nF x d, projected in place
};
void launch_constraint_projection(const ConstraintLaunch& C, cudaStream_t s);
// column c0 + k of dst (c x nF, column-major) = column k of src (nF x d) for k < count
void launch_copy_columns(const double* src, int d, double* dst, int c, int c0, int count, int nF, cudaStream_t s);

struct GatherLaunch {
  int d, fp64;
  int rows;                  // vertices gathered
  const int32_t* row_vertex; // row -> original vertex (null = identity)
  const int64_t* inc_ptr;    // incidence CSR over original vertices
  const int32_t* inc;        // element * (d+1) + slot
  const void* contrib;       // element terms
  const double* add;         // optional row-aligned addend (rows x d)
  double* out;               // rows x d
  double* partials;          // optional: sum of squares of out per block (QV_GTL)
  const int32_t* mesh_of;    // optional (batched meshes): mesh of each row's vertex (rows sorted by mesh)
  double* mesh_acc;          // with mesh_of: sums of squares go to mesh_acc[mesh * (NQ + 1) + NQ]
  double* mesh_part;         // with mesh_of: blocks x 2 sums of each block's first and last mesh
};
void launch_gather(const GatherLaunch& G, cudaStream_t s);

// polls (of ~100 ns each) a dynamic-schedule block makes on an empty queue slot
// before it gives up, sets err_flag and exits (about 0.4 s)
constexpr long long kDefaultSpinLimit = 1LL << 22;

struct SolveData {
  int d;
  int nF;
  int ell_width;
  const int32_t* ell_col;    // width x nF (eliminated numbering)
  const double* ell_val;     // width x nF
  const int32_t* rows;
  const float* blocks;
  const Task* fwd_tasks;
  const Task* bwd_tasks;
  const NodeDev* sub_nodes;  // merged subtrees of the dynamic passes
  std::vector<int64_t> fwd_off, bwd_off;  // per level task ranges (host)
  int schedule = 0;          // 0: one launch per level, 1: one dynamic launch per pass,
                             // 2: one pipelined launch per pass (bulk-copy ring)
  DynPass fdyn, bdyn;            // dynamic passes over the levels >= bottom_levels
  int bottom_levels = 0;         // levels below run as one launch per level (schedule 1)
  int n_nodes = 0;
  int32_t* err_flag = nullptr;      // set to 1 if a wait ran out of polls
  long long spin_limit = kDefaultSpinLimit;  // polls per wait before giving up
  int grid_f = 0, grid_b = 0;     // resident blocks of the dynamic passes (schedule 1)
  int pgrid_f = 0, pgrid_b = 0;   // resident blocks of the pipelined passes (schedule 2)
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};  // optional: before forward, after forward,
                                                               // after backward, after the top product
  bool top_on = false;       // the top levels run as x_T = S^-1 t_T between the passes
  TopInvDev top;
  float* y;                  // nF x d residual / forward work vector
  float* z;                  // nF x d forward result
  float* x;                  // nF x d correction
  double* X;                 // nF x d current free W (eliminated order)
  const double* b;           // nF x d right-hand side
};
// y = float(b - L_FF X); partials (optional) gets |b - L X|^2 and |b|^2
void launch_residual(const SolveData& S, double* partials, int n_blocks, cudaStream_t s);
void launch_axpy_correction(const SolveData& S, cudaStream_t s);   // X += x
// x = L_FF^{-1} y (FP32); reset = false when launch_residual_reset already reset the passes
void launch_supernodal_solve(const SolveData& S, cudaStream_t s, bool reset = true);
// the residual y = b - L_FF X of a sweep together with the reset of its passes (one launch)
void launch_residual_reset(const SolveData& S, cudaStream_t s);
int persistent_grid(int d, bool forward);  // resident blocks of the dynamic solve kernels
int persistent_pipe_grid(int d, bool forward);  // resident blocks of the pipelined ones (0: unavailable)

// constant part of the right-hand side: cst = -L_FC b (eliminated order)
void launch_pin_rhs(int d, int nF, const int64_t* ptr, const int32_t* pin_col, const double* val,
                    const double* pin_pos, double* cst, cudaStream_t s);

struct FinalLaunch {
  const double* local_partials;
  int64_t n_local_blocks;
  const double* vert_partials;
  int64_t n_vert_blocks;
  double eps_abs, eps_rel;
  int d, m, require_flip_free;
  int32_t iter;
  ffa_stats* out;
  double* scratch;   // NQ + 1 doubles
};
void launch_final_reduce(const FinalLaunch& F, cudaStream_t s);
// per-mesh statistics of batched meshes from mesh_acc (one thread per mesh)
struct MeshStatsLaunch {
  int n_mesh;
  const double* mesh_acc;     // n_mesh x (NQ + 1)
  const int32_t* mesh_d;      // element dimension of each mesh
  const int32_t* mesh_m;      // elements of each mesh
  const double* mesh_eps;     // n_mesh x 2 (eps_abs, eps_rel)
  int require_flip_free;
  ffa_stats* out;             // n_mesh
  int32_t* n_converged;       // incremented per converged mesh (zeroed by the caller)
};
void launch_mesh_stats(const MeshStatsLaunch& M, cudaStream_t s);
// Deterministic per-mesh sums of batched meshes, second pass: items (elements or
// vertex rows) are sorted by mesh; each block of items_per_block items has
// written the sums of a mesh that lies wholly inside it to acc directly and the
// sums of its first and last mesh to part[block][0 / 1][nq]; here one warp per
// mesh adds those block sums in block order into acc[mesh * (NQ + 1) + q0 + q].
struct MeshPartialsLaunch {
  int n_mesh = 0, nq = 0, q0 = 0;
  const int64_t* seg_off = nullptr;  // n_mesh + 1 item offsets
  const int32_t* seg_of = nullptr;   // mesh of each item
  int64_t n_items = 0;
  int items_per_block = 0;
  const double* part = nullptr;
  double* acc = nullptr;
};
void launch_mesh_partials(const MeshPartialsLaunch& M, cudaStream_t s);
void launch_sum_partials(const double* partials, int64_t n_blocks, int nq, double* out, cudaStream_t s);

// adjoint of one unrolled iteration, per element (ffa_adjoint.cu)
struct AdjointLaunch {
  int d, energy, fp64, m;
  ElemBufs e;            // idx, g, w, mu
  const void* P_prev;    // state_{k-1}: P (d(d+1)/2 x m), Lambda (d*d x m), U (2 or 4 x m)
  const void* Lam_prev;
  const void* U_prev;
  const void* vrec;      // vertex records of W^k
  const void* xi;        // xi^{k+1} per vertex (n x d, Real; zero at pins) or null
  void* Pbar;            // d*d x m, in: adjoint of P^k, out: adjoint of P^{k-1}
  void* Lbar;            // d*d x m, same for Lambda
  void* contribJ;        // m x (d+1) x d: g_j . J_bar
};
void launch_adjoint_local(const AdjointLaunch& a, cudaStream_t s);
void launch_xi_to_vertices(int n, int d, int fp64, const int32_t* v2e, const double* xi_e, void* xi_v,
                           cudaStream_t s);
void launch_adj_rhs(int nF, int n_pin, int d, const int32_t* row_vertex, const int32_t* pins, const double* Wbar,
                    double* b_adj, double* bbar, cudaStream_t s);
void launch_adj_pins(int n_pin, int d, const int64_t* ptr, const int32_t* row, const double* val, const double* xi,
                     double* bbar, cudaStream_t s);

// message returned by ffa_last_error(NULL) on the calling thread
void set_thread_error(const std::string& msg);

}  // namespace ffa
