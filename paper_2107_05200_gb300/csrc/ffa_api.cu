// C ABI of libffadmm (include/ffadmm.h): setup of the mesh operators and the
// factorized W-step operator, device state, and the CUDA-graph driver of the
// iteration (paper Algorithm 1; Algorithm 2 without the rescaling branch).
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <new>
#include <stdexcept>
#include <string>
#include <thread>
#include <vector>

#include "ffa_internal.h"
#include "ffa_constraint_host.h"
#include "ffa_devfactor_launch.h"
#include "ffa_topinv.h"
#include "ffa_operator_host.h"
#include "ffa_state.h"

using namespace ffa;

// Per-element and per-mesh data of a group of batched meshes concatenated into
// one context (disjoint vertex sets, so L_FF is block diagonal).
struct BatchSpec {
  std::vector<int8_t> energy_of;       // per element: 0 SD, 1 SG, 2 SA
  std::vector<double> rho_of;          // per element penalty scale
  std::vector<int32_t> mesh_of_elem;   // per element
  std::vector<int32_t> mesh_of_vertex; // per vertex
  std::vector<int32_t> mesh_d, mesh_m; // per mesh
  std::vector<double> mesh_eps;        // per mesh: eps_abs, eps_rel
};

struct ffa_ctx {
  int n = 0, m = 0, d = 0, d_in = 0, n_pin = 0, nF = 0;
  ffa_params prm{};
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::string err;
  int fp64 = 0;
  size_t rsz = 4;

  std::vector<void*> allocs;
  ElemBufs e;
  double *W = nullptr, *X = nullptr, *b = nullptr, *cst = nullptr, *pin_pos = nullptr;
  double *Wtmp = nullptr, *Wtmp2 = nullptr, *vout = nullptr;
  float *y = nullptr, *z = nullptr, *x = nullptr;
  void *vrec = nullptr, *vrec_scratch = nullptr;
  int32_t *v2e = nullptr, *v2pin = nullptr, *row_vertex = nullptr;
  int64_t* inc_ptr = nullptr;
  int32_t* inc = nullptr;
  int32_t* ell_col = nullptr;
  double* ell_val = nullptr;
  int ell_width = 0;
  int64_t* fc_ptr = nullptr;
  int32_t* fc_col = nullptr;
  double* fc_val = nullptr;
  int32_t* rows = nullptr;
  float* blocks = nullptr;
  Task *fwd_t = nullptr, *bwd_t = nullptr;
  Task *fdyn_t = nullptr, *bdyn_t = nullptr;   // task lists of the dynamic passes
  NodeDev* sub_nodes = nullptr;                 // their merged subtrees' nodes
  std::vector<int64_t> fwd_off, bwd_off;
  double* local_partials = nullptr;
  int64_t n_local_blocks = 0;
  double* vert_partials = nullptr;
  int64_t n_vert_blocks = 0;
  double* res_partials = nullptr;
  int64_t n_res_blocks = 0;
  ffa_stats* stats_d = nullptr;
  ffa_stats* stats_h = nullptr;
  double* sums_d = nullptr;
  double* sums_h = nullptr;

  cudaGraphExec_t g_batch = nullptr, g_one = nullptr, g_one_check = nullptr;
  bool initialized = false;
  int64_t iter_total = 0;
  ffa_stats last{};
  ffa_info info{};
  std::vector<int32_t> pins_h;
  std::vector<int32_t> v2e_h;   // vertex -> eliminated index (-1 pinned), host copy
  bool pins_user = true;        // false: made without pins, vertex 0 held at the origin
  // general constraints A W = b (ffa_set_constraints): the device arrays of the
  // projection, and on the host the entries on pinned vertices and b, from which
  // b' = b - (entries on pins) pin_pos is rebuilt when the pins move
  int n_con = 0;
  ConstraintLaunch con;
  std::vector<ConstraintSplit::PinEntry> con_pin;
  std::vector<double> con_b;
  double* con_bprime = nullptr;

  // differentiation through unrolled iterations (ffa_forward_unrolled / ffa_backward_unrolled)
  struct Slot {
    void* P = nullptr;
    void* Lam = nullptr;
    void* U = nullptr;
    double* W = nullptr;
    double* X = nullptr;
  };
  int32_t adj_K = 0, adj_C = 0;
  std::vector<Slot> ckpt, seg;
  Slot final_state;
  void *Pbar = nullptr, *Lbar = nullptr, *xi_v = nullptr;
  double *Wbar = nullptr, *Wloss = nullptr, *Xadj = nullptr, *b_adj = nullptr, *bbar = nullptr;
  int64_t* cf_ptr = nullptr;
  int32_t* cf_row = nullptr;
  double* cf_val = nullptr;
  int32_t* pins_d = nullptr;

  // launch shapes chosen by ffa_autotune
  int local_block = 128;
  int narrow_cols = 64;
  int schedule = 0;             // supernodal solves: 0 one launch per level, 1 dynamic
  DynPass fdyn, bdyn;           // dynamic schedule of the forward and backward passes
  // the paper's penalty schedule (penalty_schedule = 1)
  OperatorHost op;
  double* mu64 = nullptr;       // device: the penalties in double
  int32_t n_rescales = 0;
  int64_t last_event_iter = 0;
  double seconds_refactor = 0.0;
  int bottom_levels = 0;        // dynamic schedule: lowest tree levels run as one launch each
  int bottom_used = 0;          // min(bottom_levels, levels) of the current task lists
  int subtree_height_f = 2;     // dynamic schedule: bottom subtrees up to this height run as one task
  int subtree_height_b = 1;     // (forward / backward pass; measured best on the benchmark cube)
  cudaEvent_t solve_ev[4] = {nullptr, nullptr, nullptr, nullptr};  // set only while ffa_profile_phases runs
  int32_t* err_flag = nullptr;
  long long spin_limit = kDefaultSpinLimit;  // ffa_set_wait_limit
  int grid_f = 0, grid_b = 0;
  int pgrid_f = 0, pgrid_b = 0;
  std::vector<Supernode> nodes_h;  // host copy of the supernode table (task lists are rebuilt from it)
  int n_levels = 0;
  Slot tune_slot;
  // numeric decomposition on the device (factor_device 1 or 2): the plan's device
  // arrays and launch program, and the device assembly of L for rescaling events
  DevFactorDev df;
  std::vector<DfLaunch> df_prog;
  DevAssemblyDev da;
  // the top levels of the tree as one operator, x_T = S^-1 t_T (top_inverse_levels)
  TopInvPlan ti_plan;
  TopInvSetup ti_setup;
  TopInvDev ti;
  float* ti_tiles = nullptr;

  // batched meshes (set for contexts made by ffa_batch_create)
  int n_mesh = 0;
  int8_t* energy_of = nullptr;
  int32_t *mesh_of_elem = nullptr, *mesh_of_vertex = nullptr, *mesh_d = nullptr, *mesh_m = nullptr;
  double *mesh_eps = nullptr, *mesh_acc = nullptr;
  int64_t *mesh_eoff = nullptr, *mesh_voff = nullptr;   // per-mesh element / vertex offsets (n_mesh + 1)
  double *mesh_part_local = nullptr, *mesh_part_vert = nullptr;   // block sums of boundary meshes
  ffa_stats* mesh_stats = nullptr;
  int32_t* n_converged = nullptr;
};

struct ffa_batch {
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::string err;
  int n_mesh = 0;
  int check_every = 10;
  std::vector<ffa_ctx*> groups;            // one context per (d, d_in)
  std::vector<int> mesh_group, mesh_local;  // group of each mesh and its index there
  std::vector<int64_t> mesh_voff;           // first vertex of each mesh in its group
  std::vector<int32_t> mesh_n, mesh_dim;
  cudaGraphExec_t g_batch = nullptr, g_one = nullptr, g_one_check = nullptr;
  bool initialized = false;
  std::vector<ffa_stats> host_stats;
};

namespace {

thread_local std::string g_create_error = "no error";

#define FFA_CUDA(call)                                                                  \
  do {                                                                                  \
    cudaError_t _e = (call);                                                            \
    if (_e != cudaSuccess) {                                                            \
      ctx->err = std::string(#call) + ": " + cudaGetErrorString(_e);                   \
      return FFA_ERR_CUDA;                                                              \
    }                                                                                   \
  } while (0)

ffa_status fail(ffa_ctx* ctx, ffa_status st, const std::string& msg) {
  if (ctx) ctx->err = msg;
  return st;
}

template <typename T>
ffa_status dalloc(ffa_ctx* ctx, T** p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(p), count * sizeof(T));
  if (e != cudaSuccess) {
    ctx->err = std::string("cudaMalloc: ") + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? FFA_ERR_OOM : FFA_ERR_CUDA;
  }
  ctx->allocs.push_back(*p);
  ctx->info.device_bytes += (int64_t)(count * sizeof(T));
  return FFA_OK;
}

ffa_status dalloc_bytes(ffa_ctx* ctx, void** p, size_t bytes) {
  return dalloc<unsigned char>(ctx, reinterpret_cast<unsigned char**>(p), bytes);
}

template <typename T>
ffa_status upload(ffa_ctx* ctx, T** p, const std::vector<T>& h) {
  ffa_status st = dalloc(ctx, p, h.size());
  if (st != FFA_OK) return st;
  if (!h.empty()) FFA_CUDA(cudaMemcpyAsync(*p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, ctx->stream));
  return FFA_OK;
}

template <typename T>
ffa_status copy_in(ffa_ctx* ctx, std::vector<T>& dst, const T* src, size_t count) {
  dst.resize(count);
  if (count == 0) return FFA_OK;
  FFA_CUDA(cudaMemcpy(dst.data(), src, count * sizeof(T), cudaMemcpyDefault));
  return FFA_OK;
}

// host data out to a caller's buffer (host or device): on the context stream and
// complete on return, whichever stream the caller then reads it from (a plain
// synchronous copy from pageable memory may return before its last transfer lands)
ffa_status copy_out(ffa_ctx* ctx, void* dst, const void* src, size_t bytes) {
  if (bytes == 0) return FFA_OK;
  FFA_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, ctx->stream));
  FFA_CUDA(cudaStreamSynchronize(ctx->stream));
  return FFA_OK;
}

// upload a double array as the local-step scalar type
ffa_status upload_real(ffa_ctx* ctx, void** p, const std::vector<double>& h) {
  ffa_status st = dalloc_bytes(ctx, p, h.size() * ctx->rsz);
  if (st != FFA_OK) return st;
  if (ctx->fp64) {
    FFA_CUDA(cudaMemcpyAsync(*p, h.data(), h.size() * 8, cudaMemcpyHostToDevice, ctx->stream));
  } else {
    std::vector<float> f(h.begin(), h.end());
    FFA_CUDA(cudaMemcpyAsync(*p, f.data(), f.size() * 4, cudaMemcpyHostToDevice, ctx->stream));
    FFA_CUDA(cudaStreamSynchronize(ctx->stream));
  }
  return FFA_OK;
}

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// frees one of the context's device allocations before the context ends
void dfree(ffa_ctx* ctx, void* p, size_t bytes) {
  auto it = std::find(ctx->allocs.begin(), ctx->allocs.end(), p);
  if (it == ctx->allocs.end()) return;
  cudaFree(p);
  ctx->allocs.erase(it);
  ctx->info.device_bytes -= (int64_t)bytes;
}

// factor_device 1 or 2: the plan of the device decomposition (fronts, extend-add
// maps, launch program) and its work arrays; with H (the penalty schedule) also
// the term lists of the device assembly of L and the gradients in double
ffa_status devfactor_setup(ffa_ctx* ctx, const Factor& fac, const OperatorArrays& OA, const std::vector<int64_t>& Ap,
                           const OperatorHost* H) {
  std::vector<int32_t> cnt(fac.nF);
  for (int c = 0; c < fac.nF; ++c) cnt[c] = (int32_t)(Ap[fac.perm[c] + 1] - Ap[fac.perm[c]]);
  DevFactorPlan P;
  std::string msg;
  if (!build_devfactor_plan(fac, OA.width, OA.ell_col, cnt, P, msg)) return fail(ctx, FFA_ERR_INVALID_ARG, msg);
  DevFactorDev& D = ctx->df;
  D.fp64 = ctx->prm.factor_device == 2 ? 1 : 0;
  const size_t tsz = D.fp64 ? 8 : 4;
  ffa_status st;
  DfNode* nodes = nullptr;
  int64_t *rel_off = nullptr, *orig_dst = nullptr;
  int32_t* rel = nullptr;
  DfItem* items = nullptr;
  if ((st = upload(ctx, &nodes, P.nodes)) != FFA_OK) return st;
  if ((st = upload(ctx, &rel_off, P.rel_off)) != FFA_OK) return st;
  if ((st = upload(ctx, &rel, P.rel)) != FFA_OK) return st;
  if ((st = upload(ctx, &items, P.items)) != FFA_OK) return st;
  if ((st = upload(ctx, &orig_dst, P.orig_dst)) != FFA_OK) return st;
  D.nodes = nodes;
  D.rel_off = rel_off;
  D.rel = rel;
  D.items = items;
  D.orig_dst = orig_dst;
  D.front_elems = P.front_elems;
  D.linv_elems = P.linv_elems;
  D.n_slots = (int64_t)P.orig_dst.size();
  if ((st = dalloc_bytes(ctx, &D.F, (size_t)P.front_elems * tsz)) != FFA_OK) return st;
  if ((st = dalloc_bytes(ctx, &D.Lv, (size_t)P.linv_elems * tsz)) != FFA_OK) return st;
  if ((st = dalloc(ctx, &D.err, 1)) != FFA_OK) return st;
  FFA_CUDA(cudaMemsetAsync(D.err, 0, sizeof(int32_t), ctx->stream));
  ctx->df_prog = P.prog;
  if (H) {
    DevAssemblyPlan Q;
    if (!build_assembly_plan(*H, fac, OA, Ap, Q, msg)) return fail(ctx, FFA_ERR_INVALID_ARG, msg);
    DevAssemblyDev& A = ctx->da;
    int64_t *ell_ptr = nullptr, *fc_ptr = nullptr;
    int32_t *ell_src = nullptr, *fc_src = nullptr, *cf_src = nullptr;
    double* g = nullptr;
    if ((st = upload(ctx, &ell_ptr, Q.ell_ptr)) != FFA_OK) return st;
    if ((st = upload(ctx, &ell_src, Q.ell_src)) != FFA_OK) return st;
    if ((st = upload(ctx, &fc_ptr, Q.fc_ptr)) != FFA_OK) return st;
    if ((st = upload(ctx, &fc_src, Q.fc_src)) != FFA_OK) return st;
    if ((st = upload(ctx, &cf_src, Q.cf_src)) != FFA_OK) return st;
    if ((st = upload(ctx, &g, H->g)) != FFA_OK) return st;
    A.ell_ptr = ell_ptr;
    A.ell_src = ell_src;
    A.n_ell = (int64_t)Q.ell_ptr.size() - 1;
    A.fc_ptr = fc_ptr;
    A.fc_src = fc_src;
    A.cf_src = cf_src;
    A.n_fc = (int64_t)Q.fc_ptr.size() - 1;
    A.g = g;
    FFA_CUDA(cudaStreamSynchronize(ctx->stream));   // the host vectors above end here
  }
  FFA_CUDA(cudaStreamSynchronize(ctx->stream));
  return FFA_OK;
}

// the decomposition on the device from the current ELL of L_FF into ctx->blocks;
// a pivot that is not positive gives FFA_ERR_SINGULAR_SYSTEM
ffa_status devfactor_run(ffa_ctx* ctx) {
  FFA_CUDA(launch_devfactor(ctx->df, ctx->df_prog, ctx->ell_val, ctx->blocks, ctx->stream));
  int32_t flag = 0;
  FFA_CUDA(cudaMemcpyAsync(&flag, ctx->df.err, sizeof(int32_t), cudaMemcpyDeviceToHost, ctx->stream));
  FFA_CUDA(cudaStreamSynchronize(ctx->stream));
  if (flag) {
    FFA_CUDA(cudaMemsetAsync(ctx->df.err, 0, sizeof(int32_t), ctx->stream));
    FFA_CUDA(cudaStreamSynchronize(ctx->stream));
    return fail(ctx, FFA_ERR_SINGULAR_SYSTEM,
                "the W-step matrix is not positive definite (a pivot of the device decomposition)");
  }
  return FFA_OK;
}

// The top levels of the elimination tree as one operator (top_inverse_levels):
// which levels, their column numbering, and the device buffers of S^-1 and of
// its product.  Batched contexts (block-diagonal operators) do not use it.
ffa_status topinv_setup(ffa_ctx* ctx, const Factor& fac, bool batch) {
  std::string msg;
  if (!plan_top_inverse(fac, batch ? 0 : ctx->prm.top_inverse_levels, ctx->ti_plan, msg))
    return fail(ctx, FFA_ERR_INVALID_ARG, msg);
  const TopInvPlan& P = ctx->ti_plan;
  if (P.levels == 0) return FFA_OK;
  ffa_status st;
  TopInvSetup& U = ctx->ti_setup;
  U = TopInvSetup{};
  U.nT = P.nT;
  U.ldG = P.ldG;
  U.tiles = P.tiles;
  U.pos = P.pos;
  U.lo = P.lo;
  U.rmap_off = P.rmap_off;
  TopInvDev& T = ctx->ti;
  T = TopInvDev{};
  T.nT = P.nT;
  T.tiles_n = P.tiles;
  T.nblk = P.nblk;
  T.n_nodes = (int32_t)P.nodes.size();
  for (size_t q = 0; q < P.nodes.size(); ++q) {
    const Supernode& sn = fac.nodes[P.nodes[q]];
    U.ncol.push_back(sn.ncol);
    U.ld.push_back(sn.ld);
    U.nrow.push_back(sn.nrow);
    U.blk_off.push_back(sn.blk_off);
    T.pos[q] = P.pos[q];
    T.col0[q] = sn.col0;
    T.n[q] = sn.ncol;
  }
  int32_t* rmap = nullptr;
  if ((st = upload(ctx, &rmap, P.rmap)) != FFA_OK) return st;
  U.rmap = rmap;
  if ((st = dalloc(ctx, &ctx->ti_tiles, (size_t)(P.tile_bytes / 4))) != FFA_OK) return st;
  T.tiles = ctx->ti_tiles;
  {
    const std::vector<int32_t> units = top_product_units(P.tiles);
    int32_t* ud = nullptr;
    if ((st = upload(ctx, &ud, units)) != FFA_OK) return st;
    T.units = reinterpret_cast<const int2*>(ud);
    T.n_units = (int32_t)(units.size() / 2);
  }
  FFA_CUDA(prepare_top_product());
  FFA_CUDA(cudaStreamSynchronize(ctx->stream));
  return FFA_OK;
}

// S^-1 from the current factor blocks (after every decomposition of L)
ffa_status topinv_compute(ffa_ctx* ctx) {
  if (ctx->ti_plan.levels == 0) return FFA_OK;
  const double t0 = now_s();
  FFA_CUDA(compute_top_inverse(ctx->ti_setup, ctx->blocks, ctx->ti_tiles, ctx->stream));
  ctx->info.setup_seconds_top_inverse = now_s() - t0;
  return FFA_OK;
}

LocalLaunch local_launch(ffa_ctx* ctx, bool check, const void* vrec) {
  LocalLaunch L;
  L.d = ctx->d;
  L.energy = (int)ctx->prm.energy;
  L.fp64 = ctx->fp64;
  L.check = check ? 1 : 0;
  L.m = ctx->m;
  L.e = ctx->e;
  L.vrec = vrec;
  L.partials = ctx->local_partials;
  L.n_blocks = ctx->n_local_blocks;
  L.block = ctx->local_block;
  return L;
}

SolveData solve_data(ffa_ctx* ctx) {
  SolveData S;
  S.d = ctx->d;
  S.nF = ctx->nF;
  S.ell_width = ctx->ell_width;
  S.ell_col = ctx->ell_col;
  S.ell_val = ctx->ell_val;
  S.rows = ctx->rows;
  S.blocks = ctx->blocks;
  S.fwd_tasks = ctx->fwd_t;
  S.bwd_tasks = ctx->bwd_t;
  S.sub_nodes = ctx->sub_nodes;
  S.fwd_off = ctx->fwd_off;
  S.bwd_off = ctx->bwd_off;
  S.schedule = ctx->schedule;
  S.fdyn = ctx->fdyn;
  S.bdyn = ctx->bdyn;
  S.bottom_levels = ctx->bottom_used;
  for (int i = 0; i < 4; ++i) S.ev[i] = ctx->solve_ev[i];
  S.top_on = ctx->ti_plan.levels > 0;
  S.top = ctx->ti;
  S.top.err = ctx->err_flag;
  S.top.wait_limit = ctx->spin_limit;
  S.n_nodes = (int)ctx->nodes_h.size();
  S.err_flag = ctx->err_flag;
  S.spin_limit = ctx->spin_limit;
  S.grid_f = ctx->grid_f;
  S.grid_b = ctx->grid_b;
  S.pgrid_f = ctx->pgrid_f;
  S.pgrid_b = ctx->pgrid_b;
  S.y = ctx->y;
  S.z = ctx->z;
  S.x = ctx->x;
  S.X = ctx->X;
  S.b = ctx->b;
  return S;
}

enum Phase { PH_GATHER = 0, PH_WSTEP, PH_VERTEX, PH_LOCAL, PH_CHECK, PH_N };

// One iteration of Algorithm 1 on the context stream; ev (optional) gets an
// event recorded after each phase.
void enqueue_iteration(ffa_ctx* ctx, bool check, cudaEvent_t* ev = nullptr) {
  cudaStream_t s = ctx->stream;
  // W step: b = G^T r (free rows, eliminated order) - L_FC b_pins
  GatherLaunch G{};
  G.d = ctx->d;
  G.fp64 = ctx->fp64;
  G.rows = ctx->nF;
  G.row_vertex = ctx->row_vertex;
  G.inc_ptr = ctx->inc_ptr;
  G.inc = ctx->inc;
  G.contrib = ctx->e.contrib;
  G.add = ctx->cst;
  G.out = ctx->b;
  G.partials = nullptr;
  launch_gather(G, s);
  if (ev) cudaEventRecord(ev[PH_GATHER], s);
  SolveData S = solve_data(ctx);
  for (int sw = 0; sw < ctx->prm.refine_sweeps; ++sw) {
    if (sw > 0) launch_axpy_correction(S, s);
    launch_residual_reset(S, s);
    launch_supernodal_solve(S, s, false);
  }
  if (ctx->n_con > 0) {
    // general constraints: the last correction joins X, which is then projected
    launch_axpy_correction(S, s);
    launch_constraint_projection(ctx->con, s);
  }
  if (ev) cudaEventRecord(ev[PH_WSTEP], s);
  VertexLaunch V{};
  V.d = ctx->d;
  V.fp64 = ctx->fp64;
  V.n = ctx->n;
  V.Wnew_free = ctx->X;
  V.corr = ctx->n_con > 0 ? nullptr : ctx->x;
  V.v2e = ctx->v2e;
  V.v2pin = ctx->v2pin;
  V.pin_pos = ctx->pin_pos;
  V.W_in = nullptr;
  V.W = ctx->W;
  V.X = ctx->X;
  V.vrec = ctx->vrec;
  V.write_dw = 1;
  launch_vertex_update(V, s);
  if (ev) cudaEventRecord(ev[PH_VERTEX], s);
  // U, P, Lambda steps
  if (check && ctx->n_mesh > 0) {
    cudaMemsetAsync(ctx->mesh_acc, 0, (size_t)ctx->n_mesh * (NQ + 1) * sizeof(double), s);
    cudaMemsetAsync(ctx->n_converged, 0, sizeof(int32_t), s);
  }
  launch_local_step(local_launch(ctx, check, ctx->vrec), s);
  if (ev) cudaEventRecord(ev[PH_LOCAL], s);
  if (check && ctx->n_mesh > 0) {
    MeshPartialsLaunch PL;
    PL.n_mesh = ctx->n_mesh;
    PL.nq = NQ;
    PL.q0 = 0;
    PL.seg_off = ctx->mesh_eoff;
    PL.seg_of = ctx->mesh_of_elem;
    PL.n_items = ctx->m;
    PL.items_per_block = ctx->local_block;
    PL.part = ctx->mesh_part_local;
    PL.acc = ctx->mesh_acc;
    launch_mesh_partials(PL, s);
    GatherLaunch H{};
    H.d = ctx->d;
    H.fp64 = ctx->fp64;
    H.rows = ctx->n;
    H.row_vertex = nullptr;
    H.inc_ptr = ctx->inc_ptr;
    H.inc = ctx->inc;
    H.contrib = ctx->e.contrib2;
    H.add = nullptr;
    H.out = nullptr;
    H.partials = nullptr;
    H.mesh_of = ctx->mesh_of_vertex;
    H.mesh_acc = ctx->mesh_acc;
    H.mesh_part = ctx->mesh_part_vert;
    launch_gather(H, s);
    MeshPartialsLaunch PV;
    PV.n_mesh = ctx->n_mesh;
    PV.nq = 1;
    PV.q0 = NQ;
    PV.seg_off = ctx->mesh_voff;
    PV.seg_of = ctx->mesh_of_vertex;
    PV.n_items = ctx->n;
    PV.items_per_block = kVertexBlock / kGatherLanes;
    PV.part = ctx->mesh_part_vert;
    PV.acc = ctx->mesh_acc;
    launch_mesh_partials(PV, s);
    MeshStatsLaunch M{};
    M.n_mesh = ctx->n_mesh;
    M.mesh_acc = ctx->mesh_acc;
    M.mesh_d = ctx->mesh_d;
    M.mesh_m = ctx->mesh_m;
    M.mesh_eps = ctx->mesh_eps;
    M.require_flip_free = ctx->prm.require_flip_free;
    M.out = ctx->mesh_stats;
    M.n_converged = ctx->n_converged;
    launch_mesh_stats(M, s);
  } else if (check) {
    GatherLaunch H{};
    H.d = ctx->d;
    H.fp64 = ctx->fp64;
    H.rows = ctx->n;
    H.row_vertex = nullptr;
    H.inc_ptr = ctx->inc_ptr;
    H.inc = ctx->inc;
    H.contrib = ctx->e.contrib2;
    H.add = nullptr;
    H.out = nullptr;
    H.partials = ctx->vert_partials;
    launch_gather(H, s);
    FinalLaunch F{};
    F.local_partials = ctx->local_partials;
    F.n_local_blocks = ctx->n_local_blocks;
    F.vert_partials = ctx->vert_partials;
    F.n_vert_blocks = ctx->n_vert_blocks;
    F.eps_abs = ctx->prm.eps_abs;
    F.eps_rel = ctx->prm.eps_rel;
    F.d = ctx->d;
    F.m = ctx->m;
    F.require_flip_free = ctx->prm.require_flip_free;
    F.iter = 0;
    F.out = ctx->stats_d;
    F.scratch = ctx->sums_d + 8;
    launch_final_reduce(F, s);
  }
  if (ev) cudaEventRecord(ev[PH_CHECK], s);
}

ffa_status capture(ffa_ctx* ctx, int n_iter, bool check_last, cudaGraphExec_t* out) {
  cudaGraph_t graph = nullptr;
  FFA_CUDA(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
  for (int k = 0; k < n_iter; ++k) enqueue_iteration(ctx, check_last && k == n_iter - 1);
  cudaError_t e = cudaStreamEndCapture(ctx->stream, &graph);
  if (e != cudaSuccess) return fail(ctx, FFA_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
  e = cudaGraphInstantiate(out, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return fail(ctx, FFA_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
  return FFA_OK;
}

ffa_status ensure_graphs(ffa_ctx* ctx) {
  ffa_status st;
  if (!ctx->g_batch && (st = capture(ctx, ctx->prm.check_every, true, &ctx->g_batch)) != FFA_OK) return st;
  if (!ctx->g_one && (st = capture(ctx, 1, false, &ctx->g_one)) != FFA_OK) return st;
  if (!ctx->g_one_check && (st = capture(ctx, 1, true, &ctx->g_one_check)) != FFA_OK) return st;
  return FFA_OK;
}

ffa_status validate_params(const ffa_params& p, std::string& msg) {
  if (p.energy != FFA_SYM_DIRICHLET && p.energy != FFA_SYM_GRADIENT && p.energy != FFA_SYM_ARAP) msg = "unknown energy";
  else if (!(p.rho > 0) || !std::isfinite(p.rho)) msg = "rho must be positive";
  else if (!(p.eps_abs >= 0) || !(p.eps_rel >= 0)) msg = "eps_abs/eps_rel must be >= 0";
  else if (p.check_every < 1 || p.check_every > 100000) msg = "check_every must be in [1, 100000]";
  else if (p.local_precision != FFA_LOCAL_FP32 && p.local_precision != FFA_LOCAL_FP64) msg = "unknown precision";
  else if (p.refine_sweeps < 1 || p.refine_sweeps > 16) msg = "refine_sweeps must be in [1, 16]";
  else if (p.nd_leaf_size < 8 || p.nd_leaf_size > 512) msg = "nd_leaf_size must be in [8, 512]";
  else if (p.host_threads < 0) msg = "host_threads must be >= 0";
  else if (p.solve_schedule < 0 || p.solve_schedule > 2) msg = "solve_schedule must be 0, 1 or 2";
  else if (p.penalty_schedule != 0 && p.penalty_schedule != 1) msg = "penalty_schedule must be 0 or 1";
  else if (p.local_variant != 0 && p.local_variant != 1) msg = "local_variant must be 0 or 1";
  else if (p.penalty_schedule == 1 && !(p.rescale_rho > 2.0 && std::isfinite(p.rescale_rho)))
    msg = "rescale_rho must be finite and > 2";
  else if (p.penalty_schedule == 1 && p.energy == FFA_SYM_ARAP)
    msg = "penalty_schedule 1 needs the penalty bound of Lemma 1, derived for SD and SG only";
  else if (p.solve_subtree_height[0] < -1 || p.solve_subtree_height[0] > 8 || p.solve_subtree_height[1] < -1 ||
           p.solve_subtree_height[1] > 8)
    msg = "solve_subtree_height must be in [-1, 8]";
  else if (p.prox_h != 0 && p.prox_h != 1) msg = "prox_h must be 0 or 1";
  else if (p.prox_h == 1 && p.penalty_schedule == 1)
    msg = "prox_h 1 is implemented with fixed penalties (its bound depends on mu_i)";
  else if (p.prox_h == 1 && p.local_variant == 1) msg = "the joint (U, P) variant has no proximal U term";
  else if (p.factor_device < 0 || p.factor_device > 2) msg = "factor_device must be 0, 1 or 2";
  else if (p.top_inverse_levels < -1 || p.top_inverse_levels > 32) msg = "top_inverse_levels must be in [-1, 32]";
  else return FFA_OK;
  return FFA_ERR_INVALID_ARG;
}

// kernels one iteration launches: the gather, per refinement sweep the residual
// (which also resets the schedules) and the solve launches (2 dynamic plus one per non-empty
// bottom level and pass, or one per non-empty level and pass), the sweeps - 1
// corrections, the vertex update and the local step
int kernels_per_iteration(const ffa_ctx* ctx) {
  int solve = 2;
  for (int l = 0; l < ctx->bottom_used && ctx->schedule >= 1; ++l)
    solve += (ctx->fwd_off[l + 1] > ctx->fwd_off[l]) + (ctx->bwd_off[l + 1] > ctx->bwd_off[l]);
  if (ctx->schedule == 0) {
    solve = 0;
    for (size_t l = 0; l + 1 < ctx->fwd_off.size(); ++l)
      solve += (ctx->fwd_off[l + 1] > ctx->fwd_off[l]) + (ctx->bwd_off[l + 1] > ctx->bwd_off[l]);
  }
  if (ctx->ti_plan.levels > 0) solve += 1;   // the top product between the passes
  const int sweeps = ctx->prm.refine_sweeps;
  return 1 + sweeps * (1 + solve) + (sweeps - 1) + 1 + 1 + (ctx->n_con > 0 ? 3 : 0);
}

// Supernode table and task lists of the supernodal solves.  A node with at most
// narrow_cols columns and ld <= kNodeMaxLd is one node task (a whole block on the
// whole node); larger nodes are cut into wide tasks.  The level-synchronous
// schedule launches the tasks of one level at a time (fwd_off / bwd_off); the
// dynamic schedule uses the same task arrays with the per-node dependencies.
ffa_status upload_dyn(ffa_ctx* ctx, DynPass& P, const Task* tasks, const PassSchedule& sch, bool forward) {
  ffa_status st;
  PushRec *pu = nullptr, *kd = nullptr;
  int32_t *qi, *pi = nullptr, *q, *pe = nullptr, *dn = nullptr, *ct;
  const int nn = (int)(forward ? sch.push.size() : sch.push.size() / (1 + kPushKids));
  if ((st = upload(ctx, &pu, sch.push)) != FFA_OK) return st;
  if (!sch.kids.empty() && (st = upload(ctx, &kd, sch.kids)) != FFA_OK) return st;
  if ((st = upload(ctx, &qi, sch.queue)) != FFA_OK) return st;
  if ((st = dalloc(ctx, &q, sch.queue.size())) != FFA_OK) return st;
  if (forward) {
    if ((st = upload(ctx, &pi, sch.pending)) != FFA_OK) return st;
    if ((st = dalloc(ctx, &pe, nn)) != FFA_OK) return st;
  } else if ((st = dalloc(ctx, &dn, nn)) != FFA_OK) {
    return st;
  }
  if ((st = dalloc(ctx, &ct, 2)) != FFA_OK) return st;
  P.tasks = tasks;
  P.n_tasks = (int)sch.tasks.size();
  P.n_init = sch.n_init;
  P.push = reinterpret_cast<const int4*>(pu);
  P.kids = reinterpret_cast<const int4*>(kd);
  P.q_init = qi;
  P.pending_init = pi;
  P.queue = q;
  P.pending = pe;
  P.done = dn;
  P.ctr = ct;
  return FFA_OK;
}

ffa_status build_tasks(ffa_ctx* ctx) {
  ScheduleOptions opt;
  opt.narrow_cols = ctx->narrow_cols;
  opt.bottom_levels = ctx->bottom_levels;
  opt.subtree_height_f = ctx->subtree_height_f;
  opt.subtree_height_b = ctx->subtree_height_b;
  opt.top_levels = ctx->ti_plan.levels;
  Schedule sch;
  build_schedule(ctx->nodes_h, ctx->n_levels, opt, sch);
  ctx->grid_f = persistent_grid(ctx->d, true);
  ctx->grid_b = persistent_grid(ctx->d, false);
  ctx->pgrid_f = persistent_pipe_grid(ctx->d, true);
  ctx->pgrid_b = persistent_pipe_grid(ctx->d, false);
  if (ctx->schedule == 2 && (ctx->pgrid_f < 1 || ctx->pgrid_b < 1))
    return fail(ctx, FFA_ERR_CUDA, "the pipelined solve kernels cannot be made resident on this device");
  // the task shapes the solve kernels' shared-memory buffers assume
  for (int pass = 0; pass < 2; ++pass) {
    const PassSchedule& P = pass ? sch.bwd : sch.fwd;
    for (const Task& t : P.tasks) {
      const bool node_ok = t.nd.ld > 0 && t.nd.ld % 4 == 0;
      const bool shape_ok = t.kind == 0 ? (t.c0 >= 1 && t.c0 <= kSubtreeMaxNodes)
                          : t.kind == 1 ? t.nd.ld <= kNodeMaxLd
                          : (pass == 0 ? t.kind <= kFwdCols && t.r0 % kFwdRows == 0 : t.kind <= kBwdRows && t.r0 % 4 == 0);
      if (!node_ok || !shape_ok) return fail(ctx, FFA_ERR_INVALID_ARG, "internal: a solve task exceeds the kernels' tile limits");
    }
  }
  for (const NodeDev& nd : sch.sub_nodes)
    if (nd.ld > kNodeMaxLd || nd.ld % 4 != 0)
      return fail(ctx, FFA_ERR_INVALID_ARG, "internal: a merged subtree node exceeds the kernels' tile limits");
  ctx->fwd_off = sch.fwd_off;
  ctx->bwd_off = sch.bwd_off;
  ffa_status st;
  if ((st = upload(ctx, &ctx->fwd_t, sch.fwd_levels)) != FFA_OK) return st;
  if ((st = upload(ctx, &ctx->bwd_t, sch.bwd_levels)) != FFA_OK) return st;
  if ((st = upload(ctx, &ctx->fdyn_t, sch.fwd.tasks)) != FFA_OK) return st;
  if ((st = upload(ctx, &ctx->bdyn_t, sch.bwd.tasks)) != FFA_OK) return st;
  if ((st = upload(ctx, &ctx->sub_nodes, sch.sub_nodes)) != FFA_OK) return st;
  if ((st = upload_dyn(ctx, ctx->fdyn, ctx->fdyn_t, sch.fwd, true)) != FFA_OK) return st;
  if ((st = upload_dyn(ctx, ctx->bdyn, ctx->bdyn_t, sch.bwd, false)) != FFA_OK) return st;
  ctx->bottom_used = sch.bottom_used;
  if (!ctx->err_flag) {
    if ((st = dalloc(ctx, &ctx->err_flag, 1)) != FFA_OK) return st;
    FFA_CUDA(cudaMemsetAsync(ctx->err_flag, 0, sizeof(int32_t), ctx->stream));
  }
  const int n_top_f = (int)sch.fwd.tasks.size(), n_top_b = (int)sch.bwd.tasks.size();
  ctx->grid_f = std::max(1, std::min(ctx->grid_f, n_top_f));
  ctx->grid_b = std::max(1, std::min(ctx->grid_b, n_top_b));
  ctx->pgrid_f = std::max(1, std::min(ctx->pgrid_f, n_top_f));
  ctx->pgrid_b = std::max(1, std::min(ctx->pgrid_b, n_top_b));
  FFA_CUDA(cudaStreamSynchronize(ctx->stream));
  return FFA_OK;
}

ffa_status create_impl(ffa_ctx* ctx, const ffa_mesh* mesh, const int32_t* pin_idx, int32_t n_pin,
                       const double* pin_pos_in, const ffa_params* params, void* stream,
                       const BatchSpec* batch = nullptr) {
  if (!mesh) return fail(ctx, FFA_ERR_INVALID_ARG, "mesh is NULL");
  ffa_default_params(&ctx->prm);
  if (params) ctx->prm = *params;
  {
    std::string msg;
    if (validate_params(ctx->prm, msg) != FFA_OK) return fail(ctx, FFA_ERR_INVALID_ARG, msg);
  }
  const int n = mesh->n, m = mesh->m, d = mesh->d, d_in = mesh->d_in;
  if (batch && ctx->prm.penalty_schedule != 0)
    return fail(ctx, FFA_ERR_INVALID_ARG, "the penalty schedule is for single-mesh contexts");
  if (d != 2 && d != 3) return fail(ctx, FFA_ERR_INVALID_ARG, "d must be 2 or 3");
  if (d_in < d || d_in > 3) return fail(ctx, FFA_ERR_INVALID_ARG, "d_in must be in [d, 3]");
  if (n < d + 1 || m < 1) return fail(ctx, FFA_ERR_INVALID_ARG, "need n >= d+1 and m >= 1");
  if ((int64_t)m * (d + 1) >= (int64_t)1 << 31) return fail(ctx, FFA_ERR_INVALID_ARG, "mesh too large for int32 incidences");
  if (!mesh->V || !mesh->T) return fail(ctx, FFA_ERR_INVALID_ARG, "V or T is NULL");
  if (n_pin < 0 || n_pin >= n) return fail(ctx, FFA_ERR_INVALID_ARG, "n_pin must be in [0, n)");
  if (n_pin > 0 && (!pin_idx || !pin_pos_in)) return fail(ctx, FFA_ERR_INVALID_ARG, "pin arrays are NULL");
  ctx->n = n;
  ctx->m = m;
  ctx->d = d;
  ctx->d_in = d_in;
  ctx->fp64 = ctx->prm.local_precision == FFA_LOCAL_FP64;
  ctx->rsz = ctx->fp64 ? 8 : 4;
  ctx->schedule = ctx->prm.solve_schedule;
  if (ctx->prm.solve_subtree_height[0] >= 0) ctx->subtree_height_f = ctx->prm.solve_subtree_height[0];
  if (ctx->prm.solve_subtree_height[1] >= 0) ctx->subtree_height_b = ctx->prm.solve_subtree_height[1];
  if (stream) {
    ctx->stream = reinterpret_cast<cudaStream_t>(stream);
  } else {
    FFA_CUDA(cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking));
    ctx->own_stream = true;
  }
  const double t_setup0 = now_s();
  std::vector<double> V;
  std::vector<int32_t> T, pins;
  std::vector<double> pin_pos;
  ffa_status st;
  if ((st = copy_in(ctx, V, mesh->V, (size_t)n * d_in)) != FFA_OK) return st;
  if ((st = copy_in(ctx, T, mesh->T, (size_t)m * (d + 1))) != FFA_OK) return st;
  if (n_pin > 0) {
    if ((st = copy_in(ctx, pins, pin_idx, (size_t)n_pin)) != FFA_OK) return st;
    if ((st = copy_in(ctx, pin_pos, pin_pos_in, (size_t)n_pin * d)) != FFA_OK) return st;
  } else {
    pins = {0};
    pin_pos.assign(d, 0.0);
    n_pin = 1;
    ctx->pins_user = false;
  }
  ctx->n_pin = n_pin;
  for (int32_t v : T)
    if (v < 0 || v >= n) return fail(ctx, FFA_ERR_INVALID_ARG, "element index out of range");
  std::vector<int32_t> v2pin(n, -1);
  for (int p = 0; p < n_pin; ++p) {
    if (pins[p] < 0 || pins[p] >= n) return fail(ctx, FFA_ERR_INVALID_ARG, "pin index out of range");
    if (v2pin[pins[p]] >= 0) return fail(ctx, FFA_ERR_INVALID_ARG, "repeated pin index");
    v2pin[pins[p]] = p;
  }
  for (double c : pin_pos)
    if (!std::isfinite(c)) return fail(ctx, FFA_ERR_INVALID_ARG, "non-finite pin position");
  ctx->pins_h = pins;

  // ---- element geometry (double, host; setup only)
  std::vector<double> g((size_t)m * d * d), w(m);
  for (int i = 0; i < m; ++i) {
    double gi[3][3], wi;
    if (!element_geometry(d, d_in, V.data(), T.data() + (int64_t)i * (d + 1), gi, wi) || !(wi > 0))
      return fail(ctx, FFA_ERR_DEGENERATE_ELEMENT, "degenerate source element " + std::to_string(i));
    for (int j = 0; j < d; ++j)
      for (int a = 0; a < d; ++a) g[(int64_t)i * d * d + j * d + a] = gi[j][a];
    w[i] = wi;
  }
  const double rho = ctx->prm.rho;

  // ---- free vertices and the operator L = sum mu_i G_i^T G_i
  OperatorHost H;
  H.n = n;
  H.m = m;
  H.d = d;
  H.n_pin = n_pin;
  H.v2pin = v2pin;
  H.free_of.assign(n, -1);
  for (int v = 0; v < n; ++v)
    if (v2pin[v] < 0) {
      H.free_of[v] = (int32_t)H.free_vertex.size();
      H.free_vertex.push_back(v);
    }
  const int nF = (int)H.free_vertex.size();
  H.nF = nF;
  ctx->nF = nF;
  // incidence CSR over all vertices
  H.inc_ptr.assign(n + 1, 0);
  for (int64_t q = 0; q < (int64_t)m * (d + 1); ++q) H.inc_ptr[T[q] + 1]++;
  for (int v = 0; v < n; ++v) H.inc_ptr[v + 1] += H.inc_ptr[v];
  H.inc.resize(H.inc_ptr[n]);
  {
    std::vector<int64_t> fill(H.inc_ptr.begin(), H.inc_ptr.end() - 1);
    for (int i = 0; i < m; ++i)
      for (int j = 0; j <= d; ++j) H.inc[fill[T[(int64_t)i * (d + 1) + j]]++] = i * (d + 1) + j;
  }
  H.g = g;
  H.T = T;
  H.mu.resize(m);
  for (int i = 0; i < m; ++i) H.mu[i] = (batch ? batch->rho_of[i] : rho) * w[i];
  std::vector<int64_t> Ap, Cp;
  std::vector<int32_t> Ai, Ci;
  std::vector<double> Ax, Cx;
  assemble_operator(H, H.mu.data(), Ap, Ai, Ax, Cp, Ci, Cx);
  const std::vector<int32_t>& free_vertex = H.free_vertex;
  const std::vector<int64_t>& inc_ptr = H.inc_ptr;
  const std::vector<int32_t>& inc = H.inc;
  H.coords.assign((size_t)nF * 3, 0.0);
  for (int f = 0; f < nF; ++f)
    for (int a = 0; a < d_in; ++a) H.coords[(size_t)f * 3 + a] = V[(int64_t)free_vertex[f] * d_in + a];
  const std::vector<double>& coords = H.coords;

  // ---- factorization (once per mesh and rho)
  Factor fac;
  {
    FactorInput in;
    in.nF = nF;
    in.Ap = Ap.data();
    in.Ai = Ai.data();
    in.Ax = Ax.data();
    in.coords = coords.data();
    in.leaf_size = ctx->prm.nd_leaf_size;
    in.threads = ctx->prm.host_threads;
    in.numeric = ctx->prm.factor_device == 0;
    std::string msg;
    int rc = build_factor(in, fac, msg);
    if (rc == 3) return fail(ctx, FFA_ERR_SINGULAR_SYSTEM, msg);
    if (rc != 0) return fail(ctx, FFA_ERR_INVALID_ARG, msg);
  }
  ctx->info.setup_seconds_analyze = fac.t_analyze;
  ctx->info.setup_seconds_factor = fac.t_factor;
  int64_t block_floats = 0;
  for (const Supernode& sn : fac.nodes) block_floats = std::max<int64_t>(block_floats, sn.blk_off + (int64_t)sn.ld * sn.ncol);
  ctx->info.factor_entries = block_floats;
  ctx->info.factor_flops = fac.flops;
  ctx->info.n_supernodes = (int32_t)fac.nodes.size();
  ctx->info.n_levels = fac.n_levels;

  // ---- eliminated-order vertex maps, ELL of L_FF, CSR of L_FC
  std::vector<int32_t> row_vertex(nF), v2e(n, -1);
  for (int c = 0; c < nF; ++c) {
    row_vertex[c] = free_vertex[fac.perm[c]];
    v2e[row_vertex[c]] = c;
  }
  OperatorArrays OA;
  operator_arrays(fac, nF, n_pin, Ap, Ai, Ax, Cp, Ci, Cx, OA);
  const int width = OA.width;
  ctx->ell_width = width;
  const std::vector<int32_t>& ell_col = OA.ell_col;
  const std::vector<double>& ell_val = OA.ell_val;
  const std::vector<int64_t>& fc_ptr = OA.fc_ptr;
  const std::vector<int32_t>& fc_col = OA.fc_col;
  const std::vector<double>& fc_val = OA.fc_val;
  const std::vector<int64_t>& cf_ptr = OA.cf_ptr;
  const std::vector<int32_t>& cf_row = OA.cf_row;
  const std::vector<double>& cf_val = OA.cf_val;

  ctx->nodes_h = fac.nodes;
  ctx->n_levels = fac.n_levels;
  if ((st = topinv_setup(ctx, fac, batch != nullptr)) != FFA_OK) return st;
  // ---- device uploads
  if ((st = upload(ctx, &ctx->rows, fac.rows)) != FFA_OK) return st;
  if (ctx->prm.factor_device == 0) {
    if ((st = upload(ctx, &ctx->blocks, fac.blocks)) != FFA_OK) return st;
  } else {
    // written by the device decomposition below; the padding rows stay zero
    if ((st = dalloc(ctx, &ctx->blocks, (size_t)block_floats)) != FFA_OK) return st;
    FFA_CUDA(cudaMemsetAsync(ctx->blocks, 0, (size_t)block_floats * sizeof(float), ctx->stream));
  }
  if ((st = build_tasks(ctx)) != FFA_OK) return st;
  if ((st = upload(ctx, &ctx->ell_col, ell_col)) != FFA_OK) return st;
  if ((st = upload(ctx, &ctx->ell_val, ell_val)) != FFA_OK) return st;
  if ((st = upload(ctx, &ctx->fc_ptr, fc_ptr)) != FFA_OK) return st;
  if ((st = upload(ctx, &ctx->fc_col, fc_col)) != FFA_OK) return st;
  if ((st = upload(ctx, &ctx->fc_val, fc_val)) != FFA_OK) return st;
  if ((st = upload(ctx, &ctx->inc_ptr, inc_ptr)) != FFA_OK) return st;
  if ((st = upload(ctx, &ctx->inc, inc)) != FFA_OK) return st;
  if ((st = upload(ctx, &ctx->row_vertex, row_vertex)) != FFA_OK) return st;
  if ((st = upload(ctx, &ctx->v2e, v2e)) != FFA_OK) return st;
  ctx->v2e_h = v2e;
  if ((st = upload(ctx, &ctx->v2pin, v2pin)) != FFA_OK) return st;
  if ((st = upload(ctx, &ctx->pin_pos, pin_pos)) != FFA_OK) return st;
  if ((st = upload(ctx, &ctx->pins_d, pins)) != FFA_OK) return st;
  if ((st = upload(ctx, &ctx->cf_ptr, cf_ptr)) != FFA_OK) return st;
  if ((st = upload(ctx, &ctx->cf_row, cf_row)) != FFA_OK) return st;
  if ((st = upload(ctx, &ctx->cf_val, cf_val)) != FFA_OK) return st;
  if (ctx->prm.factor_device != 0) {
    const bool keep = ctx->prm.penalty_schedule == 1;
    if ((st = devfactor_setup(ctx, fac, OA, Ap, keep ? &H : nullptr)) != FFA_OK) return st;
    const double t0 = now_s();
    if ((st = devfactor_run(ctx)) != FFA_OK) return st;
    ctx->info.setup_seconds_factor = now_s() - t0;
    if (!keep) {
      // fixed penalties: the fronts and inverses are not needed again
      const size_t tsz = ctx->df.fp64 ? 8 : 4;
      dfree(ctx, ctx->df.F, (size_t)ctx->df.front_elems * tsz);
      dfree(ctx, ctx->df.Lv, (size_t)ctx->df.linv_elems * tsz);
      ctx->df.F = ctx->df.Lv = nullptr;
    }
  }
  if ((st = topinv_compute(ctx)) != FFA_OK) return st;
  // element arrays: indices (d+1) x m, gradients d*d x m, w, mu
  {
    std::vector<int32_t> idx((size_t)(d + 1) * m);
    for (int i = 0; i < m; ++i)
      for (int j = 0; j <= d; ++j) idx[(size_t)j * m + i] = T[(int64_t)i * (d + 1) + j];
    if ((st = upload(ctx, &ctx->e.idx, idx)) != FFA_OK) return st;
    std::vector<double> gs((size_t)d * d * m), mu(m);
    for (int i = 0; i < m; ++i) {
      for (int q = 0; q < d * d; ++q) gs[(size_t)q * m + i] = g[(int64_t)i * d * d + q];
      mu[i] = (batch ? batch->rho_of[i] : rho) * w[i];
    }
    if ((st = upload_real(ctx, &ctx->e.g, gs)) != FFA_OK) return st;
    if ((st = upload_real(ctx, &ctx->e.w, w)) != FFA_OK) return st;
    if ((st = upload_real(ctx, &ctx->e.mu, mu)) != FFA_OK) return st;
  }
  if (batch) {
    ctx->n_mesh = (int)batch->mesh_m.size();
    bool mixed = false;
    for (int8_t en : batch->energy_of) mixed |= (en != batch->energy_of[0]);
    ctx->prm.energy = mixed ? (ffa_energy_kind)kEnMixed : (ffa_energy_kind)batch->energy_of[0];
    if ((st = upload(ctx, &ctx->energy_of, batch->energy_of)) != FFA_OK) return st;
    if ((st = upload(ctx, &ctx->mesh_of_elem, batch->mesh_of_elem)) != FFA_OK) return st;
    if ((st = upload(ctx, &ctx->mesh_of_vertex, batch->mesh_of_vertex)) != FFA_OK) return st;
    if ((st = upload(ctx, &ctx->mesh_d, batch->mesh_d)) != FFA_OK) return st;
    if ((st = upload(ctx, &ctx->mesh_m, batch->mesh_m)) != FFA_OK) return st;
    if ((st = upload(ctx, &ctx->mesh_eps, batch->mesh_eps)) != FFA_OK) return st;
    if ((st = dalloc(ctx, &ctx->mesh_acc, (size_t)ctx->n_mesh * (NQ + 1))) != FFA_OK) return st;
    if ((st = dalloc(ctx, &ctx->mesh_stats, (size_t)ctx->n_mesh)) != FFA_OK) return st;
    if ((st = dalloc(ctx, &ctx->n_converged, 1)) != FFA_OK) return st;
    {
      // per-mesh element and vertex offsets (meshes are concatenated in order)
      std::vector<int64_t> eoff(ctx->n_mesh + 1, 0), voff(ctx->n_mesh + 1, 0);
      for (int i = 0; i < m; ++i) eoff[batch->mesh_of_elem[i] + 1]++;
      for (int v = 0; v < n; ++v) voff[batch->mesh_of_vertex[v] + 1]++;
      for (int k = 0; k < ctx->n_mesh; ++k) {
        eoff[k + 1] += eoff[k];
        voff[k + 1] += voff[k];
      }
      for (int i = 1; i < m; ++i)
        if (batch->mesh_of_elem[i] < batch->mesh_of_elem[i - 1])
          return fail(ctx, FFA_ERR_INVALID_ARG, "internal: batched elements are not sorted by mesh");
      for (int v = 1; v < n; ++v)
        if (batch->mesh_of_vertex[v] < batch->mesh_of_vertex[v - 1])
          return fail(ctx, FFA_ERR_INVALID_ARG, "internal: batched vertices are not sorted by mesh");
      if ((st = upload(ctx, &ctx->mesh_eoff, eoff)) != FFA_OK) return st;
      if ((st = upload(ctx, &ctx->mesh_voff, voff)) != FFA_OK) return st;
      // block sums, sized for the smallest local-step block the autotuner may pick (64)
      if ((st = dalloc(ctx, &ctx->mesh_part_local, (size_t)((m + 63) / 64) * 2 * NQ)) != FFA_OK) return st;
      const int64_t vblocks = ((int64_t)n * kGatherLanes + kVertexBlock - 1) / kVertexBlock;
      if ((st = dalloc(ctx, &ctx->mesh_part_vert, (size_t)vblocks * 2)) != FFA_OK) return st;
    }
    ctx->e.energy_of = ctx->energy_of;
    ctx->e.mesh_of = ctx->mesh_of_elem;
    ctx->e.mesh_acc = ctx->mesh_acc;
    ctx->e.mesh_part = ctx->mesh_part_local;
  }
  ctx->e.joint = ctx->prm.local_variant == 1 ? 1 : 0;
  const size_t R = ctx->rsz;
  if (ctx->prm.prox_h == 1) {
    if (batch) return fail(ctx, FFA_ERR_INVALID_ARG, "prox_h 1 is implemented for single meshes");
    if ((st = dalloc_bytes(ctx, &ctx->e.hmu, (size_t)m * R)) != FFA_OK) return st;
  }
  if ((st = dalloc_bytes(ctx, &ctx->e.P, (size_t)m * (d == 2 ? 3 : 6) * R)) != FFA_OK) return st;
  if ((st = dalloc_bytes(ctx, &ctx->e.Lam, (size_t)m * d * d * R)) != FFA_OK) return st;
  if ((st = dalloc_bytes(ctx, &ctx->e.U, (size_t)m * (d == 2 ? 2 : 4) * R)) != FFA_OK) return st;
  if ((st = dalloc_bytes(ctx, &ctx->e.contrib, (size_t)m * (d + 1) * d * R)) != FFA_OK) return st;
  if ((st = dalloc_bytes(ctx, &ctx->e.contrib2, (size_t)m * (d + 1) * d * R)) != FFA_OK) return st;
  if ((st = dalloc(ctx, &ctx->W, (size_t)n * d)) != FFA_OK) return st;
  if ((st = dalloc(ctx, &ctx->Wtmp, (size_t)n * d)) != FFA_OK) return st;
  if ((st = dalloc(ctx, &ctx->Wtmp2, (size_t)n * d)) != FFA_OK) return st;
  if ((st = dalloc(ctx, &ctx->vout, (size_t)n * d)) != FFA_OK) return st;
  if ((st = dalloc(ctx, &ctx->X, (size_t)nF * d)) != FFA_OK) return st;
  if ((st = dalloc(ctx, &ctx->b, (size_t)nF * d)) != FFA_OK) return st;
  if ((st = dalloc(ctx, &ctx->cst, (size_t)nF * d)) != FFA_OK) return st;
  if ((st = dalloc(ctx, &ctx->y, (size_t)nF * d)) != FFA_OK) return st;
  if ((st = dalloc(ctx, &ctx->z, (size_t)nF * d)) != FFA_OK) return st;
  if ((st = dalloc(ctx, &ctx->x, (size_t)nF * d)) != FFA_OK) return st;
  const size_t rec_bytes = (size_t)n * d * (ctx->fp64 ? 16 : 16);
  if ((st = dalloc_bytes(ctx, &ctx->vrec, rec_bytes)) != FFA_OK) return st;
  if ((st = dalloc_bytes(ctx, &ctx->vrec_scratch, rec_bytes)) != FFA_OK) return st;
  ctx->n_local_blocks = (m + ctx->local_block - 1) / ctx->local_block;
  ctx->n_vert_blocks = ((int64_t)n * kGatherLanes + kVertexBlock - 1) / kVertexBlock;
  ctx->n_res_blocks = (nF + kVertexBlock - 1) / kVertexBlock;
  // sized for the smallest local-step block (64 threads) the autotuner may pick
  if ((st = dalloc(ctx, &ctx->local_partials, (size_t)((m + 63) / 64) * NQ)) != FFA_OK) return st;
  if ((st = dalloc(ctx, &ctx->vert_partials, (size_t)ctx->n_vert_blocks)) != FFA_OK) return st;
  if ((st = dalloc(ctx, &ctx->res_partials, (size_t)ctx->n_res_blocks * 2)) != FFA_OK) return st;
  if ((st = dalloc(ctx, &ctx->stats_d, 1)) != FFA_OK) return st;
  if ((st = dalloc(ctx, &ctx->sums_d, 16)) != FFA_OK) return st;
  FFA_CUDA(cudaMallocHost(reinterpret_cast<void**>(&ctx->stats_h), sizeof(ffa_stats)));
  FFA_CUDA(cudaMallocHost(reinterpret_cast<void**>(&ctx->sums_h), 16 * sizeof(double)));
  FFA_CUDA(cudaMemsetAsync(ctx->W, 0, (size_t)n * d * 8, ctx->stream));
  FFA_CUDA(cudaMemsetAsync(ctx->e.U, 0, (size_t)m * (d == 2 ? 2 : 4) * R, ctx->stream));
  launch_pin_rhs(d, nF, ctx->fc_ptr, ctx->fc_col, ctx->fc_val, ctx->pin_pos, ctx->cst, ctx->stream);
  FFA_CUDA(cudaGetLastError());
  FFA_CUDA(cudaStreamSynchronize(ctx->stream));

  // algorithmic bytes (see the design notes): element state read+written once per
  // local step, vertex records, and the factor blocks read twice per sweep
  const int64_t ps = d == 2 ? 3 : 6, us = d == 2 ? 2 : 4;
  ctx->info.bytes_local_step =
      (int64_t)m * ((d + 1) * 4 + (int64_t)(d * d + 2) * R + (ps + d * d) * R * 2 + us * R + (int64_t)(d + 1) * d * R) +
      (int64_t)n * d * 16 + (ctx->e.hmu ? (int64_t)m * (us + 1) * R : 0);   // prox_h: U^{k-1} and h/mu read
  // the passes read every nonzero of every B_s below the top levels once (and
  // its structure indices); the top product reads the tiles of S^-1 once
  const int top_min = ctx->ti_plan.levels > 0 ? fac.n_levels - ctx->ti_plan.levels : INT32_MAX;
  int64_t nz = 0, nstruct = 0;
  for (const Supernode& sn : fac.nodes) {
    if (sn.level >= top_min) continue;
    nz += (int64_t)sn.ncol * sn.nrow + (int64_t)sn.ncol * (sn.ncol + 1) / 2;
    nstruct += sn.nrow;
  }
  const int64_t top_bytes = ctx->ti_plan.levels > 0 ? ctx->ti_plan.tile_bytes + (int64_t)2 * ctx->ti_plan.nT * d * 4 : 0;
  ctx->info.bytes_global_sweep = 2 * nz * 4 + top_bytes + (int64_t)width * nF * 12 + (int64_t)nF * d * (8 * 3 + 4 * 6);
  ctx->info.bytes_solve_pass = nz * 4 + nstruct * 4 + (int64_t)2 * nF * d * 4;
  ctx->info.top_inverse_levels = ctx->ti_plan.levels;
  ctx->info.top_inverse_cols = ctx->ti_plan.nT;
  ctx->info.bytes_top_product = top_bytes;
  ctx->info.n = n;
  ctx->info.m = m;
  ctx->info.d = d;
  ctx->info.d_in = d_in;
  ctx->info.n_pin = n_pin;
  ctx->info.n_free = nF;
  ctx->info.kernels_per_iteration = kernels_per_iteration(ctx);
  ctx->info.kernels_per_check = ctx->n_mesh > 0 ? 4 : 3;
  if (ctx->prm.penalty_schedule == 1) {
    if ((st = upload(ctx, &ctx->mu64, H.mu)) != FFA_OK) return st;
    FFA_CUDA(cudaStreamSynchronize(ctx->stream));
    std::vector<float>().swap(fac.blocks);
    std::vector<double>().swap(fac.blocks64);
    ctx->op = std::move(H);
    ctx->op.fac = std::move(fac);
  }
  (void)t_setup0;
  return FFA_OK;
}

// New penalties from ctx->mu64 (the paper's schedule): assemble L again on the
// host, decompose it on the same ordering and supernodes (Algorithm 2,
// decompose(L)), and refresh every device form of L and the W-step
// right-hand-side terms of the current state.
ffa_status apply_penalties(ffa_ctx* ctx) {
  OperatorHost& H = ctx->op;
  cudaStream_t s = ctx->stream;
  if (ctx->prm.factor_device != 0) {
    // all on the device: L from the new penalties, its decomposition, and the
    // terms that depend on it
    FFA_CUDA(cudaStreamSynchronize(s));
    const double t0 = now_s();
    FFA_CUDA(launch_device_assembly(ctx->da, ctx->d, ctx->mu64, ctx->ell_val, ctx->fc_val, ctx->cf_val, s));
    launch_pin_rhs(ctx->d, ctx->nF, ctx->fc_ptr, ctx->fc_col, ctx->fc_val, ctx->pin_pos, ctx->cst, s);
    FFA_CUDA(cudaGetLastError());
    ffa_status st = devfactor_run(ctx);
    if (st != FFA_OK) return st;
    if ((st = topinv_compute(ctx)) != FFA_OK) return st;
    launch_rhs_terms(local_launch(ctx, false, ctx->vrec), s);
    FFA_CUDA(cudaGetLastError());
    FFA_CUDA(cudaStreamSynchronize(s));
    ctx->seconds_refactor += now_s() - t0;
    return FFA_OK;
  }
  FFA_CUDA(cudaMemcpyAsync(H.mu.data(), ctx->mu64, (size_t)H.m * sizeof(double), cudaMemcpyDeviceToHost, s));
  FFA_CUDA(cudaStreamSynchronize(s));
  const double t0 = now_s();
  std::vector<int64_t> Ap, Cp;
  std::vector<int32_t> Ai, Ci;
  std::vector<double> Ax, Cx;
  assemble_operator(H, H.mu.data(), Ap, Ai, Ax, Cp, Ci, Cx);
  FactorInput in;
  in.nF = H.nF;
  in.Ap = Ap.data();
  in.Ai = Ai.data();
  in.Ax = Ax.data();
  in.coords = H.coords.data();
  in.leaf_size = ctx->prm.nd_leaf_size;
  in.threads = ctx->prm.host_threads;
  std::string msg;
  const int rc = refactor(in, H.fac, msg);
  if (rc == 3) return fail(ctx, FFA_ERR_SINGULAR_SYSTEM, msg);
  if (rc != 0) return fail(ctx, FFA_ERR_INVALID_ARG, msg);
  // uploads on the context stream, so that the kernels below and the next
  // iteration are ordered after them (a synchronous copy from pageable memory may
  // return before its last transfer lands); each host buffer outlives its copy
  FFA_CUDA(cudaMemcpyAsync(ctx->blocks, H.fac.blocks.data(), H.fac.blocks.size() * sizeof(float),
                           cudaMemcpyHostToDevice, s));
  FFA_CUDA(cudaStreamSynchronize(s));
  std::vector<float>().swap(H.fac.blocks);
  {
    const ffa_status st = topinv_compute(ctx);
    if (st != FFA_OK) return st;
  }
  OperatorArrays OA;
  operator_arrays(H.fac, H.nF, H.n_pin, Ap, Ai, Ax, Cp, Ci, Cx, OA);
  FFA_CUDA(cudaMemcpyAsync(ctx->ell_val, OA.ell_val.data(), OA.ell_val.size() * sizeof(double), cudaMemcpyHostToDevice,
                           s));
  if (!OA.fc_val.empty()) {
    FFA_CUDA(cudaMemcpyAsync(ctx->fc_val, OA.fc_val.data(), OA.fc_val.size() * sizeof(double), cudaMemcpyHostToDevice,
                             s));
    FFA_CUDA(cudaMemcpyAsync(ctx->cf_val, OA.cf_val.data(), OA.cf_val.size() * sizeof(double), cudaMemcpyHostToDevice,
                             s));
  }
  launch_pin_rhs(ctx->d, ctx->nF, ctx->fc_ptr, ctx->fc_col, ctx->fc_val, ctx->pin_pos, ctx->cst, s);
  launch_rhs_terms(local_launch(ctx, false, ctx->vrec), s);
  FFA_CUDA(cudaGetLastError());
  FFA_CUDA(cudaStreamSynchronize(s));
  ctx->seconds_refactor += now_s() - t0;
  return FFA_OK;
}

// iteration (counted from ffa_init) after which the next rescaling happens:
// 1..5, then every floor(5 (3/2)^p) iterations, p = events so far (Sec. 6)
int64_t next_rescale_iter(const ffa_ctx* ctx) {
  const int p = ctx->n_rescales;
  if (p < 5) return p + 1;
  return ctx->last_event_iter + (int64_t)std::floor(5.0 * std::pow(1.5, (double)p));
}

ffa_status device_wait_status(ffa_ctx* ctx, const char* what);

// The Tutte initializer (App. A, "Tutte's Energy"): the minimizer of
// E_T(W) = sum over edges (i, j) of |W_i - W_j|^2 / |V_i - V_j| with the boundary
// held.  Its interior rows are the weighted graph Laplacian L_II W_I = -L_IB W_B,
// solved once with the W step's machinery: host ordering and factorization,
// FP32 supernodal passes with FP64 residual correction on the GPU.
ffa_status tutte_impl(ffa_ctx* ctx, const ffa_mesh* mesh, const int32_t* bnd_in, int32_t nb, const double* bpos_in,
                      const ffa_params* params, void* stream, double* W_out, double* rel_out) {
  if (!mesh || !W_out) return fail(ctx, FFA_ERR_INVALID_ARG, "mesh or W_out is NULL");
  ffa_default_params(&ctx->prm);
  if (params) ctx->prm = *params;
  ctx->prm.penalty_schedule = 0;
  {
    std::string msg;
    if (validate_params(ctx->prm, msg) != FFA_OK) return fail(ctx, FFA_ERR_INVALID_ARG, msg);
  }
  const int n = mesh->n, m = mesh->m, d = mesh->d, d_in = mesh->d_in;
  if (d != 2 && d != 3) return fail(ctx, FFA_ERR_INVALID_ARG, "d must be 2 or 3");
  if (d_in < d || d_in > 3) return fail(ctx, FFA_ERR_INVALID_ARG, "d_in must be in [d, 3]");
  if (n < 1 || m < 1) return fail(ctx, FFA_ERR_INVALID_ARG, "need n >= 1 and m >= 1");
  if ((int64_t)m * (d + 1) >= (int64_t)1 << 31) return fail(ctx, FFA_ERR_INVALID_ARG, "mesh too large");
  if (!mesh->V || !mesh->T) return fail(ctx, FFA_ERR_INVALID_ARG, "V or T is NULL");
  if (nb < 1 || nb > n || !bnd_in || !bpos_in) return fail(ctx, FFA_ERR_INVALID_ARG, "need 1 <= n_boundary <= n and boundary arrays");
  if (stream) {
    ctx->stream = reinterpret_cast<cudaStream_t>(stream);
  } else {
    FFA_CUDA(cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking));
    ctx->own_stream = true;
  }
  ffa_status st;
  std::vector<double> V, bpos;
  std::vector<int32_t> T, bnd;
  if ((st = copy_in(ctx, V, mesh->V, (size_t)n * d_in)) != FFA_OK) return st;
  if ((st = copy_in(ctx, T, mesh->T, (size_t)m * (d + 1))) != FFA_OK) return st;
  if ((st = copy_in(ctx, bnd, bnd_in, (size_t)nb)) != FFA_OK) return st;
  if ((st = copy_in(ctx, bpos, bpos_in, (size_t)nb * d)) != FFA_OK) return st;
  for (int32_t v : T)
    if (v < 0 || v >= n) return fail(ctx, FFA_ERR_INVALID_ARG, "element index out of range");
  std::vector<int32_t> v2pin(n, -1);
  for (int p = 0; p < nb; ++p) {
    if (bnd[p] < 0 || bnd[p] >= n) return fail(ctx, FFA_ERR_INVALID_ARG, "boundary index out of range");
    if (v2pin[bnd[p]] >= 0) return fail(ctx, FFA_ERR_INVALID_ARG, "repeated boundary index");
    v2pin[bnd[p]] = p;
  }
  for (double c : bpos)
    if (!std::isfinite(c)) return fail(ctx, FFA_ERR_INVALID_ARG, "non-finite boundary position");
  // neighbours of every vertex (each edge once per endpoint)
  std::vector<int64_t> nptr(n + 1, 0);
  for (int i = 0; i < m; ++i)
    for (int a = 0; a <= d; ++a) nptr[T[(int64_t)i * (d + 1) + a] + 1] += d;
  for (int v = 0; v < n; ++v) nptr[v + 1] += nptr[v];
  std::vector<int32_t> nbr(nptr[n]);
  {
    std::vector<int64_t> fill(nptr.begin(), nptr.end() - 1);
    for (int i = 0; i < m; ++i)
      for (int a = 0; a <= d; ++a)
        for (int b = 0; b <= d; ++b)
          if (a != b) {
            const int u = T[(int64_t)i * (d + 1) + a];
            nbr[fill[u]++] = T[(int64_t)i * (d + 1) + b];
          }
  }
  std::vector<int32_t> free_of(n, -1), free_vertex;
  for (int v = 0; v < n; ++v)
    if (v2pin[v] < 0) {
      free_of[v] = (int32_t)free_vertex.size();
      free_vertex.push_back(v);
    }
  const int nF = (int)free_vertex.size();
  std::vector<double> Wh((size_t)n * d, 0.0);
  for (int p = 0; p < nb; ++p)
    for (int k = 0; k < d; ++k) Wh[(size_t)bnd[p] * d + k] = bpos[(size_t)p * d + k];
  if (nF == 0) {
    if ((st = copy_out(ctx, W_out, Wh.data(), Wh.size() * 8)) != FFA_OK) return st;
    if (rel_out) *rel_out = 0.0;
    return FFA_OK;
  }
  // rows of the interior vertices: L_II (free numbering) and L_IB (boundary slots)
  std::vector<int64_t> Ap(nF + 1, 0), Cp(nF + 1, 0);
  std::vector<int32_t> Ai, Ci;
  std::vector<double> Ax, Cx;
  for (int f = 0; f < nF; ++f) {
    const int v = free_vertex[f];
    std::vector<int32_t> js(nbr.begin() + nptr[v], nbr.begin() + nptr[v + 1]);
    std::sort(js.begin(), js.end());
    js.erase(std::unique(js.begin(), js.end()), js.end());
    double diag = 0.0;
    std::vector<std::pair<int32_t, double>> fr, cr;
    for (int j : js) {
      double l2 = 0.0;
      for (int a = 0; a < d_in; ++a) {
        const double t = V[(size_t)v * d_in + a] - V[(size_t)j * d_in + a];
        l2 += t * t;
      }
      if (!(l2 > 0.0)) return fail(ctx, FFA_ERR_INVALID_ARG, "zero-length edge at vertex " + std::to_string(v));
      const double c = 1.0 / std::sqrt(l2);
      diag += c;
      if (free_of[j] >= 0) fr.push_back({free_of[j], -c});
      else cr.push_back({v2pin[j], -c});
    }
    fr.push_back({f, diag});
    std::sort(fr.begin(), fr.end());
    std::sort(cr.begin(), cr.end());
    for (auto& pr : fr) { Ai.push_back(pr.first); Ax.push_back(pr.second); }
    for (auto& pr : cr) { Ci.push_back(pr.first); Cx.push_back(pr.second); }
    Ap[f + 1] = (int64_t)Ai.size();
    Cp[f + 1] = (int64_t)Ci.size();
  }
  std::vector<double> coords((size_t)nF * 3, 0.0);
  for (int f = 0; f < nF; ++f)
    for (int a = 0; a < d_in; ++a) coords[(size_t)f * 3 + a] = V[(size_t)free_vertex[f] * d_in + a];
  Factor fac;
  {
    FactorInput in;
    in.nF = nF;
    in.Ap = Ap.data();
    in.Ai = Ai.data();
    in.Ax = Ax.data();
    in.coords = coords.data();
    in.leaf_size = ctx->prm.nd_leaf_size;
    in.threads = ctx->prm.host_threads;
    in.numeric = ctx->prm.factor_device == 0;
    std::string msg;
    const int rc = build_factor(in, fac, msg);
    if (rc == 3) return fail(ctx, FFA_ERR_SINGULAR_SYSTEM, "Tutte system: " + msg + " (an interior part without a boundary vertex?)");
    if (rc != 0) return fail(ctx, FFA_ERR_INVALID_ARG, msg);
  }
  OperatorArrays OA;
  operator_arrays(fac, nF, nb, Ap, Ai, Ax, Cp, Ci, Cx, OA);
  ctx->n = n;
  ctx->m = m;
  ctx->d = d;
  ctx->d_in = d_in;
  ctx->nF = nF;
  ctx->n_pin = nb;
  ctx->fp64 = 1;
  ctx->rsz = 8;
  ctx->schedule = ctx->prm.solve_schedule;
  if (ctx->prm.solve_subtree_height[0] >= 0) ctx->subtree_height_f = ctx->prm.solve_subtree_height[0];
  if (ctx->prm.solve_subtree_height[1] >= 0) ctx->subtree_height_b = ctx->prm.solve_subtree_height[1];
  ctx->ell_width = OA.width;
  ctx->nodes_h = fac.nodes;
  ctx->n_levels = fac.n_levels;
  std::vector<int32_t> v2e(n, -1);
  for (int c = 0; c < nF; ++c) v2e[free_vertex[fac.perm[c]]] = c;
  if ((st = upload(ctx, &ctx->rows, fac.rows)) != FFA_OK) return st;
  int64_t block_floats = 0;
  for (const Supernode& sn : fac.nodes) block_floats = std::max<int64_t>(block_floats, sn.blk_off + (int64_t)sn.ld * sn.ncol);
  if (ctx->prm.factor_device == 0) {
    if ((st = upload(ctx, &ctx->blocks, fac.blocks)) != FFA_OK) return st;
  } else {
    if ((st = dalloc(ctx, &ctx->blocks, (size_t)block_floats)) != FFA_OK) return st;
    FFA_CUDA(cudaMemsetAsync(ctx->blocks, 0, (size_t)block_floats * sizeof(float), ctx->stream));
  }
  if ((st = build_tasks(ctx)) != FFA_OK) return st;
  if ((st = upload(ctx, &ctx->ell_col, OA.ell_col)) != FFA_OK) return st;
  if ((st = upload(ctx, &ctx->ell_val, OA.ell_val)) != FFA_OK) return st;
  if ((st = upload(ctx, &ctx->fc_ptr, OA.fc_ptr)) != FFA_OK) return st;
  if ((st = upload(ctx, &ctx->fc_col, OA.fc_col)) != FFA_OK) return st;
  if ((st = upload(ctx, &ctx->fc_val, OA.fc_val)) != FFA_OK) return st;
  if (ctx->prm.factor_device != 0) {
    if ((st = devfactor_setup(ctx, fac, OA, Ap, nullptr)) != FFA_OK) return st;
    if ((st = devfactor_run(ctx)) != FFA_OK) {
      if (st == FFA_ERR_SINGULAR_SYSTEM)
        return fail(ctx, st, "Tutte system: " + ctx->err + " (an interior part without a boundary vertex?)");
      return st;
    }
  }
  if ((st = upload(ctx, &ctx->pin_pos, bpos)) != FFA_OK) return st;
  if ((st = upload(ctx, &ctx->v2e, v2e)) != FFA_OK) return st;
  if ((st = upload(ctx, &ctx->v2pin, v2pin)) != FFA_OK) return st;
  if ((st = dalloc(ctx, &ctx->W, (size_t)n * d)) != FFA_OK) return st;
  if ((st = dalloc(ctx, &ctx->X, (size_t)nF * d)) != FFA_OK) return st;
  if ((st = dalloc(ctx, &ctx->b, (size_t)nF * d)) != FFA_OK) return st;
  if ((st = dalloc(ctx, &ctx->y, (size_t)nF * d)) != FFA_OK) return st;
  if ((st = dalloc(ctx, &ctx->z, (size_t)nF * d)) != FFA_OK) return st;
  if ((st = dalloc(ctx, &ctx->x, (size_t)nF * d)) != FFA_OK) return st;
  if ((st = dalloc_bytes(ctx, &ctx->vrec, (size_t)n * d * 16)) != FFA_OK) return st;
  ctx->n_res_blocks = (nF + kVertexBlock - 1) / kVertexBlock;
  if ((st = dalloc(ctx, &ctx->res_partials, (size_t)ctx->n_res_blocks * 2)) != FFA_OK) return st;
  cudaStream_t s = ctx->stream;
  // b = -L_IB W_B, X = 0
  launch_pin_rhs(d, nF, ctx->fc_ptr, ctx->fc_col, ctx->fc_val, ctx->pin_pos, ctx->b, s);
  FFA_CUDA(cudaMemsetAsync(ctx->X, 0, (size_t)nF * d * 8, s));
  FFA_CUDA(cudaMemsetAsync(ctx->W, 0, (size_t)n * d * 8, s));
  // residual-correction sweeps until the relative residual stops improving or is
  // at double rounding level
  SolveData S = solve_data(ctx);
  std::vector<double> part((size_t)ctx->n_res_blocks * 2);
  double rel = 1.0, prev = 2.0;
  for (int sw = 0; sw < 10; ++sw) {
    launch_residual(S, ctx->res_partials, (int)ctx->n_res_blocks, s);
    FFA_CUDA(cudaMemcpyAsync(part.data(), ctx->res_partials, part.size() * 8, cudaMemcpyDeviceToHost, s));
    FFA_CUDA(cudaStreamSynchronize(s));
    double rr = 0.0, bb = 0.0;
    for (int64_t q = 0; q < ctx->n_res_blocks; ++q) {
      rr += part[2 * q];
      bb += part[2 * q + 1];
    }
    rel = bb > 0.0 ? std::sqrt(rr / bb) : std::sqrt(rr);
    if (rel < 1e-13 || rel > 0.5 * prev || sw == 9) break;
    prev = rel;
    launch_supernodal_solve(S, s);
    launch_axpy_correction(S, s);
  }
  if ((st = device_wait_status(ctx, "supernodal solve")) != FFA_OK) return st;
  VertexLaunch Vl{};
  Vl.d = d;
  Vl.fp64 = 1;
  Vl.n = n;
  Vl.Wnew_free = ctx->X;
  Vl.corr = nullptr;
  Vl.v2e = ctx->v2e;
  Vl.v2pin = ctx->v2pin;
  Vl.pin_pos = ctx->pin_pos;
  Vl.W_in = nullptr;
  Vl.W = ctx->W;
  Vl.X = nullptr;
  Vl.vrec = ctx->vrec;
  Vl.write_dw = 0;
  launch_vertex_update(Vl, s);
  FFA_CUDA(cudaGetLastError());
  FFA_CUDA(cudaMemcpyAsync(W_out, ctx->W, (size_t)n * d * 8, cudaMemcpyDefault, s));
  FFA_CUDA(cudaStreamSynchronize(s));
  if (rel_out) *rel_out = rel;
  return FFA_OK;
}

void destroy_impl(ffa_ctx* ctx) {
  if (ctx->g_batch) cudaGraphExecDestroy(ctx->g_batch);
  if (ctx->g_one) cudaGraphExecDestroy(ctx->g_one);
  if (ctx->g_one_check) cudaGraphExecDestroy(ctx->g_one_check);
  for (void* p : ctx->allocs) cudaFree(p);
  if (ctx->stats_h) cudaFreeHost(ctx->stats_h);
  if (ctx->sums_h) cudaFreeHost(ctx->sums_h);
  if (ctx->own_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
}

ffa_status load_W_records(ffa_ctx* ctx, const double* W, bool write_X, double* W_target, void* vrec) {
  FFA_CUDA(cudaMemcpyAsync(ctx->Wtmp, W, (size_t)ctx->n * ctx->d * 8, cudaMemcpyDefault, ctx->stream));
  VertexLaunch V{};
  V.d = ctx->d;
  V.fp64 = ctx->fp64;
  V.n = ctx->n;
  V.v2e = ctx->v2e;
  V.v2pin = nullptr;  // every row comes from the input as given
  V.pin_pos = ctx->pin_pos;
  V.W_in = ctx->Wtmp;
  V.W = W_target;
  V.X = write_X ? ctx->X : nullptr;
  V.vrec = vrec;
  V.write_dw = 0;
  launch_vertex_update(V, ctx->stream);
  FFA_CUDA(cudaGetLastError());
  return FFA_OK;
}

// ---- state slots for checkpointed differentiation ---------------------------
size_t state_bytes_P(const ffa_ctx* c) { return (size_t)c->m * (c->d == 2 ? 3 : 6) * c->rsz; }
size_t state_bytes_L(const ffa_ctx* c) { return (size_t)c->m * c->d * c->d * c->rsz; }
size_t state_bytes_U(const ffa_ctx* c) { return (size_t)c->m * (c->d == 2 ? 2 : 4) * c->rsz; }

ffa_status alloc_slot(ffa_ctx* ctx, ffa_ctx::Slot& sl) {
  ffa_status st;
  if ((st = dalloc_bytes(ctx, &sl.P, state_bytes_P(ctx))) != FFA_OK) return st;
  if ((st = dalloc_bytes(ctx, &sl.Lam, state_bytes_L(ctx))) != FFA_OK) return st;
  if ((st = dalloc_bytes(ctx, &sl.U, state_bytes_U(ctx))) != FFA_OK) return st;
  if ((st = dalloc(ctx, &sl.W, (size_t)ctx->n * ctx->d)) != FFA_OK) return st;
  if ((st = dalloc(ctx, &sl.X, (size_t)ctx->nF * ctx->d)) != FFA_OK) return st;
  return FFA_OK;
}

ffa_status save_slot(ffa_ctx* ctx, ffa_ctx::Slot& sl) {
  cudaStream_t s = ctx->stream;
  FFA_CUDA(cudaMemcpyAsync(sl.P, ctx->e.P, state_bytes_P(ctx), cudaMemcpyDeviceToDevice, s));
  FFA_CUDA(cudaMemcpyAsync(sl.Lam, ctx->e.Lam, state_bytes_L(ctx), cudaMemcpyDeviceToDevice, s));
  FFA_CUDA(cudaMemcpyAsync(sl.U, ctx->e.U, state_bytes_U(ctx), cudaMemcpyDeviceToDevice, s));
  FFA_CUDA(cudaMemcpyAsync(sl.W, ctx->W, (size_t)ctx->n * ctx->d * 8, cudaMemcpyDeviceToDevice, s));
  FFA_CUDA(cudaMemcpyAsync(sl.X, ctx->X, (size_t)ctx->nF * ctx->d * 8, cudaMemcpyDeviceToDevice, s));
  return FFA_OK;
}

// make a slot the live state (element state, W, X, and the vertex records of W)
ffa_status load_slot(ffa_ctx* ctx, const ffa_ctx::Slot& sl) {
  cudaStream_t s = ctx->stream;
  FFA_CUDA(cudaMemcpyAsync(ctx->e.P, sl.P, state_bytes_P(ctx), cudaMemcpyDeviceToDevice, s));
  FFA_CUDA(cudaMemcpyAsync(ctx->e.Lam, sl.Lam, state_bytes_L(ctx), cudaMemcpyDeviceToDevice, s));
  FFA_CUDA(cudaMemcpyAsync(ctx->e.U, sl.U, state_bytes_U(ctx), cudaMemcpyDeviceToDevice, s));
  FFA_CUDA(cudaMemcpyAsync(ctx->X, sl.X, (size_t)ctx->nF * ctx->d * 8, cudaMemcpyDeviceToDevice, s));
  FFA_CUDA(cudaMemcpyAsync(ctx->Wtmp, sl.W, (size_t)ctx->n * ctx->d * 8, cudaMemcpyDeviceToDevice, s));
  VertexLaunch V{};
  V.d = ctx->d;
  V.fp64 = ctx->fp64;
  V.n = ctx->n;
  V.v2e = ctx->v2e;
  V.v2pin = nullptr;
  V.pin_pos = ctx->pin_pos;
  V.W_in = ctx->Wtmp;
  V.W = ctx->W;
  V.X = nullptr;
  V.vrec = ctx->vrec;
  V.write_dw = 0;
  launch_vertex_update(V, s);
  // the next W step reads the right-hand-side terms of the restored state
  launch_rhs_terms(local_launch(ctx, false, ctx->vrec), s);
  FFA_CUDA(cudaGetLastError());
  return FFA_OK;
}

// vertex records of a stored W into vrec_scratch
ffa_status records_of(ffa_ctx* ctx, const double* W) {
  VertexLaunch V{};
  V.d = ctx->d;
  V.fp64 = ctx->fp64;
  V.n = ctx->n;
  V.v2e = ctx->v2e;
  V.v2pin = nullptr;
  V.pin_pos = ctx->pin_pos;
  V.W_in = W;
  V.W = ctx->Wtmp2;
  V.X = nullptr;
  V.vrec = ctx->vrec_scratch;
  V.write_dw = 0;
  launch_vertex_update(V, ctx->stream);
  FFA_CUDA(cudaGetLastError());
  return FFA_OK;
}

// reads (and clears) the flag the persistent solve kernels set when a bounded
// wait ran out (FFA_ERR_TIMEOUT); a read that fails reports the CUDA error
ffa_status device_wait_status(ffa_ctx* ctx, const char* what) {
  if (!ctx->err_flag) return FFA_OK;
  int32_t f = 0;
  const cudaError_t e = cudaMemcpy(&f, ctx->err_flag, sizeof(f), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return fail(ctx, FFA_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
  if (!f) return FFA_OK;
  cudaMemset(ctx->err_flag, 0, sizeof(f));
  return fail(ctx, FFA_ERR_TIMEOUT, std::string("a device-side wait gave up: ") + what);
}

// b' = b - A_C b_pins (c x d): the constraint entries on pinned vertices times
// the current pinned positions move to the right-hand side
ffa_status constraint_rhs(ffa_ctx* ctx) {
  const int d = ctx->d;
  // on the context stream: ordered after the pin upload and before the next W step
  std::vector<double> pp((size_t)ctx->n_pin * d);
  FFA_CUDA(cudaMemcpyAsync(pp.data(), ctx->pin_pos, pp.size() * 8, cudaMemcpyDeviceToHost, ctx->stream));
  FFA_CUDA(cudaStreamSynchronize(ctx->stream));
  std::vector<double> bp = ctx->con_b;
  for (const auto& e : ctx->con_pin)
    for (int k = 0; k < d; ++k) bp[(size_t)e.row * d + k] -= e.val * pp[(size_t)e.slot * d + k];
  FFA_CUDA(cudaMemcpyAsync(ctx->con_bprime, bp.data(), bp.size() * 8, cudaMemcpyHostToDevice, ctx->stream));
  FFA_CUDA(cudaStreamSynchronize(ctx->stream));
  return FFA_OK;
}

// Columns c0 .. c0+count-1 of Z = L_FF^-1 A_F^T: each coordinate column of the
// solve carries one constraint row (b = that row of A_F, X = 0), refined in FP64
// until the relative residual reaches double rounding level.
ffa_status constraint_columns(ffa_ctx* ctx, const std::vector<int64_t>& fptr, const std::vector<int32_t>& fcol,
                              const std::vector<double>& fval, double* Z, int c, int c0, int count,
                              std::vector<double>& Xh) {
  const int d = ctx->d, nF = ctx->nF;
  cudaStream_t s = ctx->stream;
  std::vector<double> Bh((size_t)nF * d, 0.0);
  for (int j = 0; j < count; ++j)
    for (int64_t q = fptr[c0 + j]; q < fptr[c0 + j + 1]; ++q) Bh[(size_t)fcol[q] * d + j] = fval[q];
  FFA_CUDA(cudaMemcpyAsync(ctx->b, Bh.data(), Bh.size() * 8, cudaMemcpyHostToDevice, s));
  FFA_CUDA(cudaMemsetAsync(ctx->X, 0, (size_t)nF * d * 8, s));
  SolveData S = solve_data(ctx);
  std::vector<double> part((size_t)ctx->n_res_blocks * 2);
  double rel = 1.0, prev = 2.0;
  for (int sw = 0; sw < 12; ++sw) {
    launch_residual(S, ctx->res_partials, (int)ctx->n_res_blocks, s);
    FFA_CUDA(cudaMemcpyAsync(part.data(), ctx->res_partials, part.size() * 8, cudaMemcpyDeviceToHost, s));
    FFA_CUDA(cudaStreamSynchronize(s));
    double rr = 0.0, bb = 0.0;
    for (int64_t q = 0; q < ctx->n_res_blocks; ++q) {
      rr += part[2 * q];
      bb += part[2 * q + 1];
    }
    rel = bb > 0.0 ? std::sqrt(rr / bb) : std::sqrt(rr);
    if (rel < 1e-13 || rel > 0.5 * prev) break;
    prev = rel;
    launch_supernodal_solve(S, s);
    launch_axpy_correction(S, s);
  }
  ffa_status st = device_wait_status(ctx, "constraint solves");
  if (st != FFA_OK) return st;
  if (!(rel < 1e-10))
    return fail(ctx, FFA_ERR_SINGULAR_SYSTEM, "the solves for the constraint columns did not converge (relative residual " +
                                                  std::to_string(rel) + ")");
  launch_copy_columns(ctx->X, d, Z, c, c0, count, nF, s);
  FFA_CUDA(cudaGetLastError());
  Xh.resize((size_t)nF * d);
  FFA_CUDA(cudaMemcpyAsync(Xh.data(), ctx->X, Xh.size() * 8, cudaMemcpyDeviceToHost, s));
  FFA_CUDA(cudaStreamSynchronize(s));
  return FFA_OK;
}

}  // namespace

void ffa::set_thread_error(const std::string& msg) { g_create_error = msg; }

// ===========================================================================
extern "C" {

ffa_status ffa_default_params(ffa_params* p) {
  if (!p) return FFA_ERR_INVALID_ARG;
  std::memset(p, 0, sizeof(*p));
  p->energy = FFA_SYM_DIRICHLET;
  p->rho = 1.0;
  p->eps_abs = 1e-6;
  p->eps_rel = 1e-5;
  p->check_every = 10;
  p->require_flip_free = 1;
  p->local_precision = FFA_LOCAL_FP32;
  p->refine_sweeps = 2;
  p->nd_leaf_size = 64;
  p->host_threads = 0;
  p->solve_schedule = 1;
  p->penalty_schedule = 0;
  p->rescale_rho = 5.0;
  p->local_variant = 0;
  p->solve_subtree_height[0] = p->solve_subtree_height[1] = -1;
  p->prox_h = 0;
  p->factor_device = 0;
  p->top_inverse_levels = 0;
  return FFA_OK;
}

ffa_status ffa_tutte(const ffa_mesh* mesh, const int32_t* boundary, int32_t n_boundary, const double* boundary_pos,
                     const ffa_params* params, void* stream, double* W_out, double* rel_residual) {
  ffa_ctx* ctx = nullptr;
  try {
    ctx = new ffa_ctx();
  } catch (...) {
    return FFA_ERR_OOM;
  }
  ffa_status st;
  try {
    st = tutte_impl(ctx, mesh, boundary, n_boundary, boundary_pos, params, stream, W_out, rel_residual);
  } catch (const std::bad_alloc&) {
    st = FFA_ERR_OOM;
  } catch (...) {
    st = FFA_ERR_INVALID_ARG;
  }
  if (st != FFA_OK) g_create_error = ctx->err.empty() ? "ffa_tutte failed" : ctx->err;
  destroy_impl(ctx);
  delete ctx;
  return st;
}

ffa_status ffa_create(const ffa_mesh* mesh, const int32_t* pin_idx, int32_t n_pin, const double* pin_pos,
                      const ffa_params* params, void* stream, ffa_ctx** out) {
  if (!out) return FFA_ERR_INVALID_ARG;
  *out = nullptr;
  ffa_ctx* ctx = nullptr;
  try {
    ctx = new ffa_ctx();
  } catch (...) {
    return FFA_ERR_OOM;
  }
  ffa_status st;
  try {
    st = create_impl(ctx, mesh, pin_idx, n_pin, pin_pos, params, stream);
  } catch (const std::bad_alloc&) {
    st = FFA_ERR_OOM;
  } catch (...) {
    st = FFA_ERR_INVALID_ARG;
  }
  if (st != FFA_OK) {
    // no context is returned: keep the message for ffa_last_error(NULL)
    g_create_error = ctx->err.empty() ? "ffa_create failed" : ctx->err;
    destroy_impl(ctx);
    delete ctx;
    return st;
  }
  *out = ctx;
  return FFA_OK;
}

void ffa_destroy(ffa_ctx* ctx) {
  if (!ctx) return;
  destroy_impl(ctx);
  delete ctx;
}

const char* ffa_last_error(const ffa_ctx* ctx) { return ctx ? ctx->err.c_str() : g_create_error.c_str(); }

ffa_status ffa_set_handles(ffa_ctx* ctx, const double* pin_pos) {
  if (!ctx) return FFA_ERR_INVALID_ARG;
  if (!pin_pos) return fail(ctx, FFA_ERR_INVALID_ARG, "pin_pos is NULL");
  ctx->err.clear();
  FFA_CUDA(cudaMemcpyAsync(ctx->pin_pos, pin_pos, (size_t)ctx->n_pin * ctx->d * 8, cudaMemcpyDefault, ctx->stream));
  launch_pin_rhs(ctx->d, ctx->nF, ctx->fc_ptr, ctx->fc_col, ctx->fc_val, ctx->pin_pos, ctx->cst, ctx->stream);
  FFA_CUDA(cudaGetLastError());
  FFA_CUDA(cudaStreamSynchronize(ctx->stream));
  if (ctx->n_con > 0) return constraint_rhs(ctx);
  return FFA_OK;
}

ffa_status ffa_set_constraints(ffa_ctx* ctx, int32_t c, const int64_t* row_ptr, const int32_t* col,
                               const double* val, const double* b) {
  if (!ctx) return FFA_ERR_INVALID_ARG;
  ctx->err.clear();
  if (ctx->initialized) return fail(ctx, FFA_ERR_INVALID_ARG, "constraints are set before ffa_init");
  if (ctx->n_con > 0) return fail(ctx, FFA_ERR_INVALID_ARG, "constraints are already set");
  if (c < 1 || c > kMaxConstraints) return fail(ctx, FFA_ERR_INVALID_ARG, "need 1 <= c <= 256 constraint rows");
  if (!row_ptr || !col || !val || !b) return fail(ctx, FFA_ERR_INVALID_ARG, "constraint arrays are NULL");
  if (ctx->prm.penalty_schedule != 0)
    return fail(ctx, FFA_ERR_INVALID_ARG, "constraints do not combine with the penalty schedule (it refactors L)");
  if (!ctx->pins_user)
    return fail(ctx, FFA_ERR_INVALID_ARG, "constraints need at least one pinned vertex (L_FF must be definite)");
  const int d = ctx->d, n = ctx->n, nF = ctx->nF;
  ffa_status st;
  try {
    std::vector<int64_t> ptr;
    if ((st = copy_in(ctx, ptr, row_ptr, (size_t)c + 1)) != FFA_OK) return st;
    if (ptr[0] != 0) return fail(ctx, FFA_ERR_INVALID_ARG, "row_ptr[0] must be 0");
    for (int r = 0; r < c; ++r)
      if (ptr[r + 1] < ptr[r]) return fail(ctx, FFA_ERR_INVALID_ARG, "row_ptr is not non-decreasing");
    const int64_t nnz = ptr[c];
    if (nnz > (int64_t)c * n) return fail(ctx, FFA_ERR_INVALID_ARG, "more constraint entries than c x n");
    std::vector<int32_t> ci;
    std::vector<double> cv, bh;
    if ((st = copy_in(ctx, ci, col, (size_t)nnz)) != FFA_OK) return st;
    if ((st = copy_in(ctx, cv, val, (size_t)nnz)) != FFA_OK) return st;
    if ((st = copy_in(ctx, bh, b, (size_t)c * d)) != FFA_OK) return st;
    for (int64_t q = 0; q < nnz; ++q) {
      if (ci[q] < 0 || ci[q] >= n) return fail(ctx, FFA_ERR_INVALID_ARG, "constraint column out of range");
      if (!std::isfinite(cv[q])) return fail(ctx, FFA_ERR_INVALID_ARG, "non-finite constraint entry");
    }
    for (double x : bh)
      if (!std::isfinite(x)) return fail(ctx, FFA_ERR_INVALID_ARG, "non-finite constraint right-hand side");
    // split A = [A_F A_C]: entries on free vertices by eliminated index (repeated
    // columns of a row summed), entries on pinned vertices by pin slot
    std::vector<int32_t> slot_of(n, -1);
    for (size_t p = 0; p < ctx->pins_h.size(); ++p) slot_of[ctx->pins_h[p]] = (int32_t)p;
    ConstraintSplit sp;
    split_constraints(c, ptr.data(), ci.data(), cv.data(), ctx->v2e_h, slot_of, sp);
    const std::vector<int64_t>& fptr = sp.fptr;
    const std::vector<int32_t>& fcol = sp.fcol;
    const std::vector<double>& fval = sp.fval;
    ctx->con_pin = sp.pin;
    // Z = L_FF^-1 A_F^T, d rows of A_F per refined solve, and S = A_F Z (host)
    double* Z = nullptr;
    if ((st = dalloc(ctx, &Z, (size_t)c * nF)) != FFA_OK) return st;
    std::vector<double> Sm((size_t)c * c, 0.0), Xh;
    for (int c0 = 0; c0 < c; c0 += d) {
      const int cnt = std::min(d, c - c0);
      if ((st = constraint_columns(ctx, fptr, fcol, fval, Z, c, c0, cnt, Xh)) != FFA_OK) return st;
      for (int r = 0; r < c; ++r)
        for (int64_t q = fptr[r]; q < fptr[r + 1]; ++q)
          for (int j = 0; j < cnt; ++j) Sm[(size_t)r * c + c0 + j] += fval[q] * Xh[(size_t)fcol[q] * d + j];
    }
    std::vector<double> Sinv;
    const int dep = schur_inverse(c, Sm, Sinv);
    if (dep >= 0)
      return fail(ctx, FFA_ERR_INVALID_ARG, "constraint row " + std::to_string(dep) +
                                                " depends on the pins or on the rows before it");
    int64_t* dptr = nullptr;
    int32_t* dcol = nullptr;
    double *dval = nullptr, *dSinv = nullptr, *dnu = nullptr;
    if ((st = upload(ctx, &dptr, fptr)) != FFA_OK) return st;
    if ((st = upload(ctx, &dcol, fcol)) != FFA_OK) return st;
    if ((st = upload(ctx, &dval, fval)) != FFA_OK) return st;
    if ((st = upload(ctx, &dSinv, Sinv)) != FFA_OK) return st;
    if ((st = dalloc(ctx, &dnu, (size_t)c * d)) != FFA_OK) return st;
    if ((st = dalloc(ctx, &ctx->con_bprime, (size_t)c * d)) != FFA_OK) return st;
    FFA_CUDA(cudaStreamSynchronize(ctx->stream));
    ctx->con_b = bh;
    ctx->con.d = d;
    ctx->con.c = c;
    ctx->con.nF = nF;
    ctx->con.ptr = dptr;
    ctx->con.col = dcol;
    ctx->con.val = dval;
    ctx->con.bprime = ctx->con_bprime;
    ctx->con.Sinv = dSinv;
    ctx->con.Z = Z;
    ctx->con.nu = dnu;
    ctx->con.X = ctx->X;
    ctx->n_con = c;
  } catch (const std::bad_alloc&) {
    return fail(ctx, FFA_ERR_OOM, "host allocation failed");
  }
  // graphs captured before (none before ffa_init, kept for safety) lack the projection
  if (ctx->g_batch) { cudaGraphExecDestroy(ctx->g_batch); ctx->g_batch = nullptr; }
  if (ctx->g_one) { cudaGraphExecDestroy(ctx->g_one); ctx->g_one = nullptr; }
  if (ctx->g_one_check) { cudaGraphExecDestroy(ctx->g_one_check); ctx->g_one_check = nullptr; }
  return constraint_rhs(ctx);
}

static ffa_status init_body(ffa_ctx* ctx, const double* W0) {
  if (!ctx) return FFA_ERR_INVALID_ARG;
  if (!W0) return fail(ctx, FFA_ERR_INVALID_ARG, "W0 is NULL");
  ctx->err.clear();
  ffa_status st = load_W_records(ctx, W0, true, ctx->W, ctx->vrec);
  if (st != FFA_OK) return st;
  launch_init_polar(local_launch(ctx, false, ctx->vrec), ctx->stream);
  FFA_CUDA(cudaGetLastError());
  if (ctx->e.hmu) {
    launch_prox_weight(local_launch(ctx, false, ctx->vrec), ctx->stream);
    FFA_CUDA(cudaGetLastError());
  }
  if (ctx->prm.penalty_schedule == 1) {
    // Algorithm 2: mu_i = max(mu_min,i, w_i) from P^0, then decompose(L)
    launch_penalty(local_launch(ctx, false, ctx->vrec), 0, ctx->mu64, ctx->prm.rescale_rho, ctx->stream);
    FFA_CUDA(cudaGetLastError());
    if ((st = apply_penalties(ctx)) != FFA_OK) return st;
    ctx->n_rescales = 0;
    ctx->last_event_iter = 0;
  }
  FFA_CUDA(cudaStreamSynchronize(ctx->stream));
  ctx->initialized = true;
  ctx->iter_total = 0;
  return FFA_OK;
}

static ffa_status iterate_body(ffa_ctx* ctx, int32_t max_iter, int32_t stop_at_tol, ffa_stats* stats) {
  if (!ctx) return FFA_ERR_INVALID_ARG;
  ctx->err.clear();
  if (!ctx->initialized) return fail(ctx, FFA_ERR_NOT_INITIALIZED, "ffa_init has not been called");
  if (max_iter < 0) return fail(ctx, FFA_ERR_INVALID_ARG, "max_iter < 0");
  ffa_status st = ensure_graphs(ctx);
  if (st != FFA_OK) return st;
  const int ce = ctx->prm.check_every;
  const bool sched = ctx->prm.penalty_schedule == 1;
  int done = 0;
  bool have = false;
  while (done < max_iter) {
    int step = std::min(max_iter - done, ce);
    bool at_event = false;
    if (sched) {
      const int64_t ev = next_rescale_iter(ctx) - (ctx->iter_total + done);
      if (ev <= step) {
        step = (int)std::max<int64_t>(ev, 1);
        at_event = true;
      }
    }
    if (step == ce) {
      FFA_CUDA(cudaGraphLaunch(ctx->g_batch, ctx->stream));
    } else {
      for (int k = 0; k < step - 1; ++k) FFA_CUDA(cudaGraphLaunch(ctx->g_one, ctx->stream));
      FFA_CUDA(cudaGraphLaunch(ctx->g_one_check, ctx->stream));
    }
    done += step;
    if (stop_at_tol || done == max_iter || at_event) {
      FFA_CUDA(cudaMemcpyAsync(ctx->stats_h, ctx->stats_d, sizeof(ffa_stats), cudaMemcpyDeviceToHost, ctx->stream));
      FFA_CUDA(cudaStreamSynchronize(ctx->stream));
      if (const ffa_status ws = device_wait_status(ctx, "supernodal solve")) {
        ctx->iter_total += done;
        return ws;
      }
      have = true;
      ctx->last = *ctx->stats_h;
      ctx->last.checked_iter = (int32_t)(ctx->iter_total + done);
      if (ctx->last.converged < 0) {
        ctx->iter_total += done;
        ctx->last.converged = 0;
        ctx->last.iters = done;
        if (stats) *stats = ctx->last;
        return fail(ctx, FFA_ERR_NAN, "non-finite values in the iterate");
      }
      if (stop_at_tol && ctx->last.converged) break;
    }
    if (at_event) {
      // the test of an event iteration is taken before its rescaling
      launch_penalty(local_launch(ctx, false, ctx->vrec), 1, ctx->mu64, ctx->prm.rescale_rho, ctx->stream);
      FFA_CUDA(cudaGetLastError());
      if ((st = apply_penalties(ctx)) != FFA_OK) {
        ctx->iter_total += done;
        return st;
      }
      ctx->n_rescales++;
      ctx->last_event_iter = ctx->iter_total + done;
    }
  }
  ctx->iter_total += done;
  if (!have) {
    ctx->last = ffa_stats{};
  }
  ctx->last.iters = done;
  ctx->last.rescales = ctx->n_rescales;
  if (stats) *stats = ctx->last;
  return FFA_OK;
}

// The penalty schedule's host work (operator assembly, factorization on several
// threads) can throw; nothing may leave the C ABI as an exception.
ffa_status ffa_init(ffa_ctx* ctx, const double* W0) {
  if (!ctx) return FFA_ERR_INVALID_ARG;
  try {
    return init_body(ctx, W0);
  } catch (const std::bad_alloc&) {
    return fail(ctx, FFA_ERR_OOM, "host allocation failed in ffa_init");
  } catch (const std::exception& e) {
    return fail(ctx, FFA_ERR_INVALID_ARG, std::string("ffa_init: ") + e.what());
  } catch (...) {
    return fail(ctx, FFA_ERR_INVALID_ARG, "ffa_init: unexpected host error");
  }
}

ffa_status ffa_iterate(ffa_ctx* ctx, int32_t max_iter, int32_t stop_at_tol, ffa_stats* stats) {
  if (!ctx) return FFA_ERR_INVALID_ARG;
  try {
    return iterate_body(ctx, max_iter, stop_at_tol, stats);
  } catch (const std::bad_alloc&) {
    return fail(ctx, FFA_ERR_OOM, "host allocation failed in ffa_iterate");
  } catch (const std::exception& e) {
    return fail(ctx, FFA_ERR_INVALID_ARG, std::string("ffa_iterate: ") + e.what());
  } catch (...) {
    return fail(ctx, FFA_ERR_INVALID_ARG, "ffa_iterate: unexpected host error");
  }
}

ffa_status ffa_get_W(ffa_ctx* ctx, double* W_out) {
  if (!ctx) return FFA_ERR_INVALID_ARG;
  if (const ffa_status ws = device_wait_status(ctx, "supernodal solve")) return ws;
  if (!W_out) return fail(ctx, FFA_ERR_INVALID_ARG, "W_out is NULL");
  ctx->err.clear();
  FFA_CUDA(cudaMemcpyAsync(W_out, ctx->W, (size_t)ctx->n * ctx->d * 8, cudaMemcpyDefault, ctx->stream));
  FFA_CUDA(cudaStreamSynchronize(ctx->stream));
  return FFA_OK;
}

ffa_status ffa_get_penalties(ffa_ctx* ctx, double* mu) {
  if (!ctx || !mu) return FFA_ERR_INVALID_ARG;
  ctx->err.clear();
  const int m = ctx->m;
  std::vector<double> h(m);
  if (ctx->mu64) {
    FFA_CUDA(cudaMemcpyAsync(h.data(), ctx->mu64, (size_t)m * 8, cudaMemcpyDeviceToHost, ctx->stream));
    FFA_CUDA(cudaStreamSynchronize(ctx->stream));
  } else if (ctx->fp64) {
    FFA_CUDA(cudaMemcpyAsync(h.data(), ctx->e.mu, (size_t)m * 8, cudaMemcpyDeviceToHost, ctx->stream));
    FFA_CUDA(cudaStreamSynchronize(ctx->stream));
  } else {
    std::vector<float> f(m);
    FFA_CUDA(cudaMemcpyAsync(f.data(), ctx->e.mu, (size_t)m * 4, cudaMemcpyDeviceToHost, ctx->stream));
    FFA_CUDA(cudaStreamSynchronize(ctx->stream));
    for (int i = 0; i < m; ++i) h[i] = f[i];
  }
  return copy_out(ctx, mu, h.data(), (size_t)m * 8);
}

ffa_status ffa_get_state(ffa_ctx* ctx, double* U, double* P, double* Lam) {
  if (!ctx) return FFA_ERR_INVALID_ARG;
  ctx->err.clear();
  const int m = ctx->m, d = ctx->d;
  const size_t R = ctx->rsz;
  const int ps = state_p_size(d), us = state_u_size(d);
  std::vector<unsigned char> hu((size_t)m * us * R), hp((size_t)m * ps * R), hl((size_t)m * d * d * R);
  FFA_CUDA(cudaMemcpyAsync(hu.data(), ctx->e.U, hu.size(), cudaMemcpyDeviceToHost, ctx->stream));
  FFA_CUDA(cudaMemcpyAsync(hp.data(), ctx->e.P, hp.size(), cudaMemcpyDeviceToHost, ctx->stream));
  FFA_CUDA(cudaMemcpyAsync(hl.data(), ctx->e.Lam, hl.size(), cudaMemcpyDeviceToHost, ctx->stream));
  FFA_CUDA(cudaStreamSynchronize(ctx->stream));
  auto as_double = [&](const std::vector<unsigned char>& h) {
    std::vector<double> v(h.size() / R);
    for (size_t k = 0; k < v.size(); ++k)
      v[k] = ctx->fp64 ? reinterpret_cast<const double*>(h.data())[k] : (double)reinterpret_cast<const float*>(h.data())[k];
    return v;
  };
  const std::vector<double> u = as_double(hu), p = as_double(hp), l = as_double(hl);
  std::vector<double> oU((size_t)m * d * d), oP((size_t)m * d * d), oL((size_t)m * d * d);
  unpack_state(d, m, u.data(), p.data(), l.data(), oU.data(), oP.data(), oL.data());
  const size_t bytes = (size_t)m * d * d * 8;
  ffa_status st;
  if (U && (st = copy_out(ctx, U, oU.data(), bytes)) != FFA_OK) return st;
  if (P && (st = copy_out(ctx, P, oP.data(), bytes)) != FFA_OK) return st;
  if (Lam && (st = copy_out(ctx, Lam, oL.data(), bytes)) != FFA_OK) return st;
  return FFA_OK;
}

ffa_status ffa_set_state(ffa_ctx* ctx, const double* W, const double* U, const double* P, const double* Lam) {
  if (!ctx) return FFA_ERR_INVALID_ARG;
  ctx->err.clear();
  if (!W || !U || !P || !Lam) return fail(ctx, FFA_ERR_INVALID_ARG, "W, U, P and Lambda are all required");
  if (ctx->prm.penalty_schedule != 0)
    return fail(ctx, FFA_ERR_INVALID_ARG, "with the penalty schedule the state also holds mu and its event counters");
  const int m = ctx->m, d = ctx->d;
  const size_t mdd = (size_t)m * d * d;
  ffa_status st;
  try {
    std::vector<double> hU, hP, hL, hW;
    if ((st = copy_in(ctx, hU, U, mdd)) != FFA_OK) return st;
    if ((st = copy_in(ctx, hP, P, mdd)) != FFA_OK) return st;
    if ((st = copy_in(ctx, hL, Lam, mdd)) != FFA_OK) return st;
    if ((st = copy_in(ctx, hW, W, (size_t)ctx->n * d)) != FFA_OK) return st;
    for (double x : hW)
      if (!std::isfinite(x)) return fail(ctx, FFA_ERR_INVALID_ARG, "non-finite entry in W");
    std::vector<double> u((size_t)m * state_u_size(d)), p((size_t)m * state_p_size(d)), l(mdd);
    std::string msg;
    if (!pack_state(d, m, hU.data(), hP.data(), hL.data(), u.data(), p.data(), l.data(), msg))
      return fail(ctx, FFA_ERR_INVALID_ARG, msg);
    // copies on the context stream, complete before their host buffers go away,
    // and ordered before the kernels below
    auto put = [&](void* dst, const std::vector<double>& h) -> ffa_status {
      if (ctx->fp64) {
        FFA_CUDA(cudaMemcpyAsync(dst, h.data(), h.size() * 8, cudaMemcpyHostToDevice, ctx->stream));
        FFA_CUDA(cudaStreamSynchronize(ctx->stream));
      } else {
        std::vector<float> f(h.begin(), h.end());
        FFA_CUDA(cudaMemcpyAsync(dst, f.data(), f.size() * 4, cudaMemcpyHostToDevice, ctx->stream));
        FFA_CUDA(cudaStreamSynchronize(ctx->stream));
      }
      return FFA_OK;
    };
    // nothing may still read the old state
    FFA_CUDA(cudaStreamSynchronize(ctx->stream));
    if ((st = put(ctx->e.U, u)) != FFA_OK) return st;
    if ((st = put(ctx->e.P, p)) != FFA_OK) return st;
    if ((st = put(ctx->e.Lam, l)) != FFA_OK) return st;
    // W, its free rows as the W step's starting point, the vertex records, and the
    // right-hand-side terms r_i = mu_i (U_i P_i - Lambda_i) the next W step gathers
    if ((st = load_W_records(ctx, hW.data(), true, ctx->W, ctx->vrec)) != FFA_OK) return st;
    launch_rhs_terms(local_launch(ctx, false, ctx->vrec), ctx->stream);
    FFA_CUDA(cudaGetLastError());
    if (ctx->e.hmu) {   // the proximal weight from the P given here
      launch_prox_weight(local_launch(ctx, false, ctx->vrec), ctx->stream);
      FFA_CUDA(cudaGetLastError());
    }
    FFA_CUDA(cudaStreamSynchronize(ctx->stream));
  } catch (const std::bad_alloc&) {
    return fail(ctx, FFA_ERR_OOM, "host allocation failed");
  }
  ctx->initialized = true;
  ctx->iter_total = 0;
  ctx->adj_K = 0;
  return FFA_OK;
}

ffa_status ffa_energy(ffa_ctx* ctx, const double* W, double* E) {
  if (!ctx) return FFA_ERR_INVALID_ARG;
  if (!E) return fail(ctx, FFA_ERR_INVALID_ARG, "E is NULL");
  ctx->err.clear();
  ffa_status st = load_W_records(ctx, W ? W : ctx->W, false, ctx->Wtmp2, ctx->vrec_scratch);
  if (st != FFA_OK) return st;
  LocalLaunch L = local_launch(ctx, false, ctx->vrec_scratch);
  launch_energy_terms(L, 0, ctx->stream);
  launch_sum_partials(ctx->local_partials, (ctx->m + kLocalBlock - 1) / kLocalBlock, NQ, ctx->sums_d, ctx->stream);
  FFA_CUDA(cudaGetLastError());
  FFA_CUDA(cudaMemcpyAsync(ctx->sums_h, ctx->sums_d, NQ * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  FFA_CUDA(cudaStreamSynchronize(ctx->stream));
  *E = ctx->sums_h[Q_FLIPS] > 0.5 ? INFINITY : ctx->sums_h[Q_ENERGY];
  return FFA_OK;
}

ffa_status ffa_gradient(ffa_ctx* ctx, const double* W, double* dEdW) {
  if (!ctx) return FFA_ERR_INVALID_ARG;
  if (!dEdW) return fail(ctx, FFA_ERR_INVALID_ARG, "dEdW is NULL");
  ctx->err.clear();
  ffa_status st = load_W_records(ctx, W ? W : ctx->W, false, ctx->Wtmp2, ctx->vrec_scratch);
  if (st != FFA_OK) return st;
  LocalLaunch L = local_launch(ctx, false, ctx->vrec_scratch);
  launch_energy_terms(L, 1, ctx->stream);
  launch_sum_partials(ctx->local_partials, (ctx->m + kLocalBlock - 1) / kLocalBlock, NQ, ctx->sums_d, ctx->stream);
  GatherLaunch G{};
  G.d = ctx->d;
  G.fp64 = ctx->fp64;
  G.rows = ctx->n;
  G.row_vertex = nullptr;
  G.inc_ptr = ctx->inc_ptr;
  G.inc = ctx->inc;
  G.contrib = ctx->e.contrib2;
  G.add = nullptr;
  G.out = ctx->vout;
  G.partials = nullptr;
  launch_gather(G, ctx->stream);
  FFA_CUDA(cudaGetLastError());
  FFA_CUDA(cudaMemcpyAsync(ctx->sums_h, ctx->sums_d, NQ * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  FFA_CUDA(cudaStreamSynchronize(ctx->stream));
  if (ctx->sums_h[Q_FLIPS] > 0.5) return fail(ctx, FFA_ERR_FLIPPED, "gradient requested at a flipped map");
  FFA_CUDA(cudaMemcpyAsync(dEdW, ctx->vout, (size_t)ctx->n * ctx->d * 8, cudaMemcpyDefault, ctx->stream));
  FFA_CUDA(cudaStreamSynchronize(ctx->stream));
  return FFA_OK;
}

ffa_status ffa_get_info(ffa_ctx* ctx, ffa_info* info) {
  if (!ctx || !info) return FFA_ERR_INVALID_ARG;
  ctx->info.kernels_per_iteration = kernels_per_iteration(ctx);   // the schedule may have been retuned
  ctx->info.seconds_refactor = ctx->seconds_refactor;
  *info = ctx->info;
  return FFA_OK;
}

ffa_status ffa_copy_factor(ffa_ctx* ctx, float* out, int64_t count) {
  if (!ctx) return FFA_ERR_INVALID_ARG;
  ctx->err.clear();
  if (!out) return fail(ctx, FFA_ERR_INVALID_ARG, "out is NULL");
  if (count != ctx->info.factor_entries)
    return fail(ctx, FFA_ERR_INVALID_ARG, "count must equal factor_entries (" + std::to_string(ctx->info.factor_entries) + ")");
  return copy_out(ctx, out, ctx->blocks, (size_t)count * sizeof(float));
}

ffa_status ffa_profile_phases(ffa_ctx* ctx, int32_t reps, ffa_phase_times* out) {
  if (!ctx || !out) return FFA_ERR_INVALID_ARG;
  ctx->err.clear();
  if (!ctx->initialized) return fail(ctx, FFA_ERR_NOT_INITIALIZED, "ffa_init has not been called");
  if (reps < 1) return fail(ctx, FFA_ERR_INVALID_ARG, "reps < 1");
  cudaEvent_t ev[PH_N + 1];
  for (auto& e : ev) FFA_CUDA(cudaEventCreate(&e));
  for (auto& e : ctx->solve_ev) FFA_CUDA(cudaEventCreate(&e));
  double acc[PH_N + 1] = {0};
  double acc_f = 0.0, acc_b = 0.0, acc_t = 0.0;
  const bool top = ctx->ti_plan.levels > 0;
  for (int r = 0; r < reps; ++r) {
    FFA_CUDA(cudaEventRecord(ev[PH_N], ctx->stream));
    enqueue_iteration(ctx, r == reps - 1, ev);
    FFA_CUDA(cudaGetLastError());
    FFA_CUDA(cudaEventSynchronize(ev[PH_CHECK]));
    float tf, tb, tt = 0.f;
    FFA_CUDA(cudaEventElapsedTime(&tf, ctx->solve_ev[0], ctx->solve_ev[1]));
    if (top) {
      FFA_CUDA(cudaEventElapsedTime(&tt, ctx->solve_ev[1], ctx->solve_ev[3]));
      FFA_CUDA(cudaEventElapsedTime(&tb, ctx->solve_ev[3], ctx->solve_ev[2]));
    } else {
      FFA_CUDA(cudaEventElapsedTime(&tb, ctx->solve_ev[1], ctx->solve_ev[2]));
    }
    acc_f += tf;
    acc_b += tb;
    acc_t += tt;
    float t[PH_N];
    FFA_CUDA(cudaEventElapsedTime(&t[PH_GATHER], ev[PH_N], ev[PH_GATHER]));
    for (int p = 1; p < PH_N; ++p) FFA_CUDA(cudaEventElapsedTime(&t[p], ev[p - 1], ev[p]));
    for (int p = 0; p < PH_N; ++p) acc[p] += (p == PH_CHECK) ? 0.0 : t[p];
    if (r == reps - 1) acc[PH_CHECK] = t[PH_CHECK];
    float whole;
    FFA_CUDA(cudaEventElapsedTime(&whole, ev[PH_N], ev[PH_LOCAL]));
    acc[PH_N] += whole;
  }
  for (auto& e : ev) cudaEventDestroy(e);
  for (auto& e : ctx->solve_ev) {
    cudaEventDestroy(e);
    e = nullptr;
  }
  ctx->iter_total += reps;
  out->reps = reps;
  out->ms_solve_forward = acc_f / reps;
  out->ms_solve_backward = acc_b / reps;
  out->ms_top_product = acc_t / reps;
  out->ms_gather = acc[PH_GATHER] / reps;
  out->ms_wstep = acc[PH_WSTEP] / reps;
  out->ms_vertex = acc[PH_VERTEX] / reps;
  out->ms_local = acc[PH_LOCAL] / reps;
  out->ms_check = acc[PH_CHECK];
  out->ms_iteration = acc[PH_N] / reps;
  return FFA_OK;
}

ffa_status ffa_forward_unrolled(ffa_ctx* ctx, int32_t K, int32_t ckpt_every) {
  if (!ctx) return FFA_ERR_INVALID_ARG;
  ctx->err.clear();
  if (!ctx->initialized) return fail(ctx, FFA_ERR_NOT_INITIALIZED, "ffa_init has not been called");
  if (K < 1 || ckpt_every < 1) return fail(ctx, FFA_ERR_INVALID_ARG, "K and ckpt_every must be >= 1");
  if (ctx->prm.penalty_schedule != 0)
    return fail(ctx, FFA_ERR_INVALID_ARG, "differentiation needs fixed penalties (penalty_schedule 0)");
  if (ctx->prm.local_variant != 0)
    return fail(ctx, FFA_ERR_INVALID_ARG, "differentiation is implemented for the paper's local step (local_variant 0)");
  if (ctx->e.hmu)
    return fail(ctx, FFA_ERR_INVALID_ARG, "differentiation is implemented for the U step without the proximal term (prox_h 0)");
  if (ctx->n_con > 0)
    return fail(ctx, FFA_ERR_INVALID_ARG, "differentiation is implemented for pinned constraints only");
  ffa_status st = ensure_graphs(ctx);
  if (st != FFA_OK) return st;
  const int C = std::min(ckpt_every, K);
  const int nseg = (K + C - 1) / C;
  while ((int)ctx->ckpt.size() < nseg) {
    ctx->ckpt.emplace_back();
    if ((st = alloc_slot(ctx, ctx->ckpt.back())) != FFA_OK) return st;
  }
  while ((int)ctx->seg.size() < C + 1) {
    ctx->seg.emplace_back();
    if ((st = alloc_slot(ctx, ctx->seg.back())) != FFA_OK) return st;
  }
  if (!ctx->final_state.P && (st = alloc_slot(ctx, ctx->final_state)) != FFA_OK) return st;
  const size_t md = (size_t)ctx->m * ctx->d * ctx->d * ctx->rsz;
  if (!ctx->Pbar) {
    if ((st = dalloc_bytes(ctx, &ctx->Pbar, md)) != FFA_OK) return st;
    if ((st = dalloc_bytes(ctx, &ctx->Lbar, md)) != FFA_OK) return st;
    if ((st = dalloc_bytes(ctx, &ctx->xi_v, (size_t)ctx->n * ctx->d * ctx->rsz)) != FFA_OK) return st;
    if ((st = dalloc(ctx, &ctx->Wbar, (size_t)ctx->n * ctx->d)) != FFA_OK) return st;
    if ((st = dalloc(ctx, &ctx->Wloss, (size_t)ctx->n * ctx->d)) != FFA_OK) return st;
    if ((st = dalloc(ctx, &ctx->Xadj, (size_t)ctx->nF * ctx->d)) != FFA_OK) return st;
    if ((st = dalloc(ctx, &ctx->b_adj, (size_t)ctx->nF * ctx->d)) != FFA_OK) return st;
    if ((st = dalloc(ctx, &ctx->bbar, (size_t)ctx->n_pin * ctx->d)) != FFA_OK) return st;
  }
  for (int sgi = 0; sgi < nseg; ++sgi) {
    if ((st = save_slot(ctx, ctx->ckpt[sgi])) != FFA_OK) return st;
    const int steps = std::min(C, K - sgi * C);
    for (int j = 0; j < steps; ++j) FFA_CUDA(cudaGraphLaunch(ctx->g_one, ctx->stream));
  }
  if ((st = save_slot(ctx, ctx->final_state)) != FFA_OK) return st;
  FFA_CUDA(cudaStreamSynchronize(ctx->stream));
  ctx->iter_total += K;
  ctx->adj_K = K;
  ctx->adj_C = C;
  return FFA_OK;
}

ffa_status ffa_backward_unrolled(ffa_ctx* ctx, const double* dL_dW, double* dL_db) {
  if (!ctx) return FFA_ERR_INVALID_ARG;
  ctx->err.clear();
  if (ctx->adj_K < 1) return fail(ctx, FFA_ERR_NOT_INITIALIZED, "ffa_forward_unrolled has not been called");
  if (!dL_dW || !dL_db) return fail(ctx, FFA_ERR_INVALID_ARG, "dL_dW or dL_db is NULL");
  cudaStream_t s = ctx->stream;
  const int K = ctx->adj_K, C = ctx->adj_C, d = ctx->d;
  const size_t md = (size_t)ctx->m * d * d * ctx->rsz;
  FFA_CUDA(cudaMemcpyAsync(ctx->Wloss, dL_dW, (size_t)ctx->n * d * 8, cudaMemcpyDefault, s));
  FFA_CUDA(cudaMemsetAsync(ctx->Pbar, 0, md, s));
  FFA_CUDA(cudaMemsetAsync(ctx->Lbar, 0, md, s));
  FFA_CUDA(cudaMemsetAsync(ctx->bbar, 0, (size_t)ctx->n_pin * d * 8, s));
  ffa_status st;
  bool have_xi = false;
  const int nseg = (K + C - 1) / C;
  for (int sgi = nseg - 1; sgi >= 0; --sgi) {
    const int k0 = sgi * C, k1 = std::min(K, k0 + C);
    // recompute the segment's states from its checkpoint
    if ((st = load_slot(ctx, ctx->ckpt[sgi])) != FFA_OK) return st;
    if ((st = save_slot(ctx, ctx->seg[0])) != FFA_OK) return st;
    for (int j = 1; j <= k1 - k0; ++j) {
      FFA_CUDA(cudaGraphLaunch(ctx->g_one, s));
      if ((st = save_slot(ctx, ctx->seg[j])) != FFA_OK) return st;
    }
    for (int k = k1; k > k0; --k) {
      const int j = k - k0;
      if ((st = records_of(ctx, ctx->seg[j].W)) != FFA_OK) return st;
      if (have_xi) launch_xi_to_vertices(ctx->n, d, ctx->fp64, ctx->v2e, ctx->Xadj, ctx->xi_v, s);
      AdjointLaunch a{};
      a.d = d;
      a.energy = (int)ctx->prm.energy;
      a.fp64 = ctx->fp64;
      a.m = ctx->m;
      a.e = ctx->e;
      a.P_prev = ctx->seg[j - 1].P;
      a.Lam_prev = ctx->seg[j - 1].Lam;
      a.U_prev = ctx->seg[j - 1].U;
      a.vrec = ctx->vrec_scratch;
      a.xi = have_xi ? ctx->xi_v : nullptr;
      a.Pbar = ctx->Pbar;
      a.Lbar = ctx->Lbar;
      a.contribJ = ctx->e.contrib2;
      launch_adjoint_local(a, s);
      // W_bar = G^T J_bar (+ the loss gradient at the last iteration)
      GatherLaunch G{};
      G.d = d;
      G.fp64 = ctx->fp64;
      G.rows = ctx->n;
      G.row_vertex = nullptr;
      G.inc_ptr = ctx->inc_ptr;
      G.inc = ctx->inc;
      G.contrib = ctx->e.contrib2;
      G.add = (k == K) ? ctx->Wloss : nullptr;
      G.out = ctx->Wbar;
      G.partials = nullptr;
      launch_gather(G, s);
      launch_adj_rhs(ctx->nF, ctx->n_pin, d, ctx->row_vertex, ctx->pins_d, ctx->Wbar, ctx->b_adj, ctx->bbar, s);
      // xi = L_FF^{-1} W_bar_F with the same factor (L is symmetric) and refinement
      FFA_CUDA(cudaMemsetAsync(ctx->Xadj, 0, (size_t)ctx->nF * d * 8, s));
      SolveData S = solve_data(ctx);
      S.X = ctx->Xadj;
      S.b = ctx->b_adj;
      for (int sw = 0; sw < ctx->prm.refine_sweeps; ++sw) {
        if (sw > 0) launch_axpy_correction(S, s);
        launch_residual(S, nullptr, 0, s);
        launch_supernodal_solve(S, s);
      }
      launch_axpy_correction(S, s);
      launch_adj_pins(ctx->n_pin, d, ctx->cf_ptr, ctx->cf_row, ctx->cf_val, ctx->Xadj, ctx->bbar, s);
      FFA_CUDA(cudaGetLastError());
      have_xi = true;
    }
  }
  // leave the live state at the end of the forward pass
  if ((st = load_slot(ctx, ctx->final_state)) != FFA_OK) return st;
  FFA_CUDA(cudaMemcpyAsync(dL_db, ctx->bbar, (size_t)ctx->n_pin * d * 8, cudaMemcpyDefault, s));
  FFA_CUDA(cudaStreamSynchronize(s));
  return FFA_OK;
}

ffa_status ffa_autotune(ffa_ctx* ctx, int32_t reps, ffa_tuning* out) {
  if (!ctx) return FFA_ERR_INVALID_ARG;
  ctx->err.clear();
  if (!ctx->initialized) return fail(ctx, FFA_ERR_NOT_INITIALIZED, "ffa_init has not been called");
  if (reps < 1) return fail(ctx, FFA_ERR_INVALID_ARG, "reps < 1");
  ffa_status st;
  if (!ctx->tune_slot.P && (st = alloc_slot(ctx, ctx->tune_slot)) != FFA_OK) return st;
  if ((st = save_slot(ctx, ctx->tune_slot)) != FFA_OK) return st;
  cudaStream_t s = ctx->stream;
  cudaEvent_t e0, e1;
  FFA_CUDA(cudaEventCreate(&e0));
  FFA_CUDA(cudaEventCreate(&e1));
  ffa_tuning t{};
  // 1) local step: threads per block
  const int blocks[3] = {64, 128, 256};
  double best = 1e300;
  int best_block = ctx->local_block;
  for (int c = 0; c < 3; ++c) {
    ctx->local_block = blocks[c];
    ctx->n_local_blocks = (ctx->m + blocks[c] - 1) / blocks[c];
    launch_local_step(local_launch(ctx, false, ctx->vrec), s);  // warm-up
    FFA_CUDA(cudaEventRecord(e0, s));
    for (int r = 0; r < reps; ++r) launch_local_step(local_launch(ctx, false, ctx->vrec), s);
    FFA_CUDA(cudaEventRecord(e1, s));
    FFA_CUDA(cudaEventSynchronize(e1));
    float ms;
    FFA_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    t.ms_local[c] = ms / reps;
    if (t.ms_local[c] < best) {
      best = t.ms_local[c];
      best_block = blocks[c];
    }
  }
  ctx->local_block = best_block;
  ctx->n_local_blocks = (ctx->m + best_block - 1) / best_block;
  // 2) supernodal solves: which small nodes run as one node task
  const int narrows[2] = {32, 64};
  best = 1e300;
  int best_narrow = ctx->narrow_cols;
  for (int c = 0; c < 2; ++c) {
    ctx->narrow_cols = narrows[c];
    if ((st = build_tasks(ctx)) != FFA_OK) return st;
    SolveData S = solve_data(ctx);
    launch_supernodal_solve(S, s);
    FFA_CUDA(cudaEventRecord(e0, s));
    for (int r = 0; r < reps; ++r) launch_supernodal_solve(S, s);
    FFA_CUDA(cudaEventRecord(e1, s));
    FFA_CUDA(cudaEventSynchronize(e1));
    float ms;
    FFA_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    t.ms_solve[c] = ms / reps;
    if (t.ms_solve[c] < best) {
      best = t.ms_solve[c];
      best_narrow = narrows[c];
    }
  }
  ctx->narrow_cols = best_narrow;
  if ((st = build_tasks(ctx)) != FFA_OK) return st;
  // 3) supernodal solves: per-level launches or one persistent launch per pass
  best = 1e300;
  int best_sched = ctx->schedule;
  for (int c = 0; c < 3; ++c) {
    ctx->schedule = c;
    if (c == 2 && (ctx->pgrid_f < 1 || ctx->pgrid_b < 1)) {
      t.ms_schedule[c] = 0.0;
      continue;
    }
    SolveData S = solve_data(ctx);
    launch_supernodal_solve(S, s);
    FFA_CUDA(cudaEventRecord(e0, s));
    for (int r = 0; r < reps; ++r) launch_supernodal_solve(S, s);
    FFA_CUDA(cudaEventRecord(e1, s));
    FFA_CUDA(cudaEventSynchronize(e1));
    float ms;
    FFA_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    t.ms_schedule[c] = ms / reps;
    if (t.ms_schedule[c] < best) {
      best = t.ms_schedule[c];
      best_sched = c;
    }
  }
  ctx->schedule = best_sched;
  // 4) dynamic schedules: how many of the lowest tree levels run as one launch per level
  if (ctx->schedule >= 1) {
    const int bottoms[4] = {0, 2, 3, 4};
    best = 1e300;
    int best_bottom = ctx->bottom_levels;
    for (int c = 0; c < 4; ++c) {
      ctx->bottom_levels = bottoms[c];
      if ((st = build_tasks(ctx)) != FFA_OK) return st;
      SolveData S = solve_data(ctx);
      launch_supernodal_solve(S, s);
      FFA_CUDA(cudaEventRecord(e0, s));
      for (int r = 0; r < reps; ++r) launch_supernodal_solve(S, s);
      FFA_CUDA(cudaEventRecord(e1, s));
      FFA_CUDA(cudaEventSynchronize(e1));
      float ms;
      FFA_CUDA(cudaEventElapsedTime(&ms, e0, e1));
      t.ms_bottom[c] = ms / reps;
      if (t.ms_bottom[c] < best) {
        best = t.ms_bottom[c];
        best_bottom = bottoms[c];
      }
    }
    ctx->bottom_levels = best_bottom;
    if ((st = build_tasks(ctx)) != FFA_OK) return st;
  }
  // 5) dynamic schedule without bottom launches: the height of the merged bottom
  // subtrees, per pass (each pass timed on its own)
  t.subtree_height[0] = ctx->subtree_height_f;
  t.subtree_height[1] = ctx->subtree_height_b;
  for (int c = 0; c < 4; ++c) t.ms_subtree[0][c] = t.ms_subtree[1][c] = 0.0;
  if (ctx->schedule >= 1 && ctx->bottom_levels == 0) {
    for (auto& e : ctx->solve_ev) FFA_CUDA(cudaEventCreate(&e));
    double best_f = 1e300, best_b = 1e300;
    int hf = ctx->subtree_height_f, hb = ctx->subtree_height_b;
    for (int c = 0; c < 4; ++c) {
      ctx->subtree_height_f = ctx->subtree_height_b = c;
      if ((st = build_tasks(ctx)) != FFA_OK) return st;
      SolveData S = solve_data(ctx);
      double af = 0.0, ab = 0.0;
      for (int r = 0; r <= reps; ++r) {   // the first launch warms up
        launch_supernodal_solve(S, s);
        FFA_CUDA(cudaEventSynchronize(ctx->solve_ev[2]));
        float tf, tb;
        FFA_CUDA(cudaEventElapsedTime(&tf, ctx->solve_ev[0], ctx->solve_ev[1]));
        FFA_CUDA(cudaEventElapsedTime(&tb, ctx->solve_ev[1], ctx->solve_ev[2]));
        if (r > 0) {
          af += tf;
          ab += tb;
        }
      }
      t.ms_subtree[0][c] = af / reps;
      t.ms_subtree[1][c] = ab / reps;
      if (t.ms_subtree[0][c] < best_f) {
        best_f = t.ms_subtree[0][c];
        hf = c;
      }
      if (t.ms_subtree[1][c] < best_b) {
        best_b = t.ms_subtree[1][c];
        hb = c;
      }
    }
    for (auto& e : ctx->solve_ev) {
      cudaEventDestroy(e);
      e = nullptr;
    }
    ctx->subtree_height_f = hf;
    ctx->subtree_height_b = hb;
    t.subtree_height[0] = hf;
    t.subtree_height[1] = hb;
    if ((st = build_tasks(ctx)) != FFA_OK) return st;
  }
  if ((st = device_wait_status(ctx, "tuning")) != FFA_OK) return st;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  // the graphs captured the old launch shapes
  if (ctx->g_batch) { cudaGraphExecDestroy(ctx->g_batch); ctx->g_batch = nullptr; }
  if (ctx->g_one) { cudaGraphExecDestroy(ctx->g_one); ctx->g_one = nullptr; }
  if (ctx->g_one_check) { cudaGraphExecDestroy(ctx->g_one_check); ctx->g_one_check = nullptr; }
  if ((st = load_slot(ctx, ctx->tune_slot)) != FFA_OK) return st;
  FFA_CUDA(cudaStreamSynchronize(s));
  t.local_block = ctx->local_block;
  t.narrow_cols = ctx->narrow_cols;
  t.schedule = ctx->schedule;
  t.bottom_levels = ctx->bottom_levels;
  if (out) *out = t;
  return FFA_OK;
}

ffa_status ffa_last_wstep_residual(ffa_ctx* ctx, double* rel) {
  if (!ctx || !rel) return FFA_ERR_INVALID_ARG;
  ctx->err.clear();
  if (ctx->n_con > 0)
    return fail(ctx, FFA_ERR_INVALID_ARG, "with general constraints L_FF W_F - b_F holds the multiplier term A_F^T nu");
  SolveData S = solve_data(ctx);
  launch_residual(S, ctx->res_partials, (int)ctx->n_res_blocks, ctx->stream);
  launch_sum_partials(ctx->res_partials, ctx->n_res_blocks, 2, ctx->sums_d, ctx->stream);
  FFA_CUDA(cudaGetLastError());
  FFA_CUDA(cudaMemcpyAsync(ctx->sums_h, ctx->sums_d, 2 * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  FFA_CUDA(cudaStreamSynchronize(ctx->stream));
  *rel = ctx->sums_h[1] > 0 ? std::sqrt(ctx->sums_h[0] / ctx->sums_h[1]) : std::sqrt(ctx->sums_h[0]);
  return FFA_OK;
}

ffa_status ffa_set_wait_limit(ffa_ctx* ctx, int64_t polls) {
  if (!ctx) return FFA_ERR_INVALID_ARG;
  ctx->err.clear();
  if (polls < 0) return fail(ctx, FFA_ERR_INVALID_ARG, "polls must be >= 0");
  ctx->spin_limit = (long long)polls;
  // the graphs hold the launch parameters they were captured with
  if (ctx->g_batch) { cudaGraphExecDestroy(ctx->g_batch); ctx->g_batch = nullptr; }
  if (ctx->g_one) { cudaGraphExecDestroy(ctx->g_one); ctx->g_one = nullptr; }
  if (ctx->g_one_check) { cudaGraphExecDestroy(ctx->g_one_check); ctx->g_one_check = nullptr; }
  return FFA_OK;
}

}  // extern "C"

// ===========================================================================
// batched meshes
// ===========================================================================
namespace {

#define FFA_BCUDA(call)                                                                 \
  do {                                                                                  \
    cudaError_t _e = (call);                                                            \
    if (_e != cudaSuccess) {                                                            \
      b->err = std::string(#call) + ": " + cudaGetErrorString(_e);                     \
      return FFA_ERR_CUDA;                                                              \
    }                                                                                   \
  } while (0)

ffa_status batch_capture(ffa_batch* b, int n_iter, bool check_last, cudaGraphExec_t* out) {
  cudaGraph_t graph = nullptr;
  FFA_BCUDA(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
  for (int k = 0; k < n_iter; ++k)
    for (ffa_ctx* c : b->groups) enqueue_iteration(c, check_last && k == n_iter - 1);
  cudaError_t e = cudaStreamEndCapture(b->stream, &graph);
  if (e != cudaSuccess) {
    b->err = std::string("graph capture: ") + cudaGetErrorString(e);
    return FFA_ERR_CUDA;
  }
  e = cudaGraphInstantiate(out, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    b->err = std::string("graph instantiate: ") + cudaGetErrorString(e);
    return FFA_ERR_CUDA;
  }
  return FFA_OK;
}

void batch_destroy_impl(ffa_batch* b) {
  if (b->g_batch) cudaGraphExecDestroy(b->g_batch);
  if (b->g_one) cudaGraphExecDestroy(b->g_one);
  if (b->g_one_check) cudaGraphExecDestroy(b->g_one_check);
  for (ffa_ctx* c : b->groups) {
    destroy_impl(c);
    delete c;
  }
  if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
}

ffa_status batch_create_impl(ffa_batch* b, int32_t n_meshes, const ffa_mesh* meshes, const int32_t* const* pin_idx,
                             const int32_t* n_pin, const double* const* pin_pos, const ffa_energy_kind* energies,
                             const double* rho, const ffa_params* params, void* stream) {
  if (n_meshes < 1 || !meshes) {
    b->err = "need at least one mesh";
    return FFA_ERR_INVALID_ARG;
  }
  ffa_params prm;
  ffa_default_params(&prm);
  if (params) prm = *params;
  b->check_every = prm.check_every;
  b->n_mesh = n_meshes;
  if (stream) {
    b->stream = reinterpret_cast<cudaStream_t>(stream);
  } else {
    FFA_BCUDA(cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking));
    b->own_stream = true;
  }
  // group the meshes by (d, d_in)
  std::vector<std::pair<int, int>> keys;
  b->mesh_group.assign(n_meshes, -1);
  b->mesh_local.assign(n_meshes, -1);
  b->mesh_voff.assign(n_meshes, 0);
  b->mesh_n.assign(n_meshes, 0);
  b->mesh_dim.assign(n_meshes, 0);
  for (int k = 0; k < n_meshes; ++k) {
    const ffa_mesh& mk = meshes[k];
    if ((mk.d != 2 && mk.d != 3) || mk.d_in < mk.d || mk.d_in > 3 || mk.n < mk.d + 1 || mk.m < 1 || !mk.V || !mk.T) {
      b->err = "mesh " + std::to_string(k) + ": invalid sizes or pointers";
      return FFA_ERR_INVALID_ARG;
    }
    const std::pair<int, int> key{mk.d, mk.d_in};
    auto it = std::find(keys.begin(), keys.end(), key);
    if (it == keys.end()) {
      keys.push_back(key);
      it = keys.end() - 1;
    }
    b->mesh_group[k] = (int)(it - keys.begin());
    b->mesh_n[k] = mk.n;
    b->mesh_dim[k] = mk.d;
  }
  for (size_t gi = 0; gi < keys.size(); ++gi) {
    const int d = keys[gi].first, d_in = keys[gi].second;
    std::vector<double> V;
    std::vector<int32_t> T, pins;
    std::vector<double> pos;
    BatchSpec spec;
    int64_t n_tot = 0, m_tot = 0;
    double xoff = 0.0;
    int local = 0;
    for (int k = 0; k < n_meshes; ++k) {
      if (b->mesh_group[k] != (int)gi) continue;
      const ffa_mesh& mk = meshes[k];
      std::vector<double> Vk((size_t)mk.n * d_in);
      std::vector<int32_t> Tk((size_t)mk.m * (d + 1));
      FFA_BCUDA(cudaMemcpy(Vk.data(), mk.V, Vk.size() * 8, cudaMemcpyDefault));
      FFA_BCUDA(cudaMemcpy(Tk.data(), mk.T, Tk.size() * 4, cudaMemcpyDefault));
      // shift the source along x so that the meshes do not overlap (the nested
      // dissection then separates them first); gradients and areas do not change
      double lo = 1e300, hi = -1e300;
      for (int v = 0; v < mk.n; ++v) {
        lo = std::min(lo, Vk[(size_t)v * d_in]);
        hi = std::max(hi, Vk[(size_t)v * d_in]);
      }
      const double shift = xoff - lo;
      for (int v = 0; v < mk.n; ++v) Vk[(size_t)v * d_in] += shift;
      xoff += (hi - lo) * 1.5 + 1.0;
      for (int32_t t : Tk) {
        if (t < 0 || t >= mk.n) {
          b->err = "mesh " + std::to_string(k) + ": element index out of range";
          return FFA_ERR_INVALID_ARG;
        }
      }
      for (auto& t : Tk) t += (int32_t)n_tot;
      V.insert(V.end(), Vk.begin(), Vk.end());
      T.insert(T.end(), Tk.begin(), Tk.end());
      const int np = n_pin ? n_pin[k] : 0;
      if (np > 0) {
        std::vector<int32_t> pk(np);
        std::vector<double> bk((size_t)np * d);
        FFA_BCUDA(cudaMemcpy(pk.data(), pin_idx[k], pk.size() * 4, cudaMemcpyDefault));
        FFA_BCUDA(cudaMemcpy(bk.data(), pin_pos[k], bk.size() * 8, cudaMemcpyDefault));
        for (int32_t p : pk) {
          if (p < 0 || p >= mk.n) {
            b->err = "mesh " + std::to_string(k) + ": pin index out of range";
            return FFA_ERR_INVALID_ARG;
          }
          pins.push_back(p + (int32_t)n_tot);
        }
        pos.insert(pos.end(), bk.begin(), bk.end());
      } else {
        pins.push_back((int32_t)n_tot);       // vertex 0 of this mesh at the origin
        for (int c = 0; c < d; ++c) pos.push_back(0.0);
      }
      const int en_k = energies ? (int)energies[k] : (int)prm.energy;
      if (en_k != FFA_SYM_DIRICHLET && en_k != FFA_SYM_GRADIENT && en_k != FFA_SYM_ARAP) {
        b->err = "mesh " + std::to_string(k) + ": unknown energy";
        return FFA_ERR_INVALID_ARG;
      }
      const int8_t en = (int8_t)en_k;
      const double rk = rho ? rho[k] : prm.rho;
      for (int i = 0; i < mk.m; ++i) {
        spec.energy_of.push_back(en);
        spec.rho_of.push_back(rk);
        spec.mesh_of_elem.push_back(local);
      }
      for (int v = 0; v < mk.n; ++v) spec.mesh_of_vertex.push_back(local);
      spec.mesh_d.push_back(d);
      spec.mesh_m.push_back(mk.m);
      spec.mesh_eps.push_back(prm.eps_abs);
      spec.mesh_eps.push_back(prm.eps_rel);
      b->mesh_local[k] = local++;
      b->mesh_voff[k] = n_tot;
      n_tot += mk.n;
      m_tot += mk.m;
    }
    if (n_tot >= INT32_MAX || m_tot * (d + 1) >= INT32_MAX) {
      b->err = "batch group too large for int32 indices";
      return FFA_ERR_INVALID_ARG;
    }
    ffa_mesh gm{(int32_t)n_tot, (int32_t)m_tot, d, d_in, V.data(), T.data()};
    ffa_ctx* c = new ffa_ctx();
    b->groups.push_back(c);
    ffa_params gp = prm;
    ffa_status st = create_impl(c, &gm, pins.data(), (int32_t)pins.size(), pos.data(), &gp, b->stream, &spec);
    if (st != FFA_OK) {
      b->err = c->err;
      return st;
    }
  }
  b->host_stats.assign(n_meshes, ffa_stats{});
  return FFA_OK;
}

}  // namespace

extern "C" {

ffa_status ffa_batch_create(int32_t n_meshes, const ffa_mesh* meshes, const int32_t* const* pin_idx,
                            const int32_t* n_pin, const double* const* pin_pos, const ffa_energy_kind* energies,
                            const double* rho, const ffa_params* params, void* stream, ffa_batch** out) {
  if (!out) return FFA_ERR_INVALID_ARG;
  *out = nullptr;
  ffa_batch* b = new (std::nothrow) ffa_batch();
  if (!b) return FFA_ERR_OOM;
  ffa_status st;
  try {
    st = batch_create_impl(b, n_meshes, meshes, pin_idx, n_pin, pin_pos, energies, rho, params, stream);
  } catch (const std::bad_alloc&) {
    st = FFA_ERR_OOM;
  } catch (...) {
    st = FFA_ERR_INVALID_ARG;
  }
  if (st != FFA_OK) {
    g_create_error = b->err.empty() ? "ffa_batch_create failed" : b->err;
    batch_destroy_impl(b);
    delete b;
    return st;
  }
  *out = b;
  return FFA_OK;
}

void ffa_batch_destroy(ffa_batch* b) {
  if (!b) return;
  batch_destroy_impl(b);
  delete b;
}

const char* ffa_batch_last_error(const ffa_batch* b) { return b ? b->err.c_str() : g_create_error.c_str(); }

ffa_status ffa_batch_init(ffa_batch* b, const double* const* W0) {
  if (!b || !W0) return FFA_ERR_INVALID_ARG;
  b->err.clear();
  for (int k = 0; k < b->n_mesh; ++k) {
    ffa_ctx* c = b->groups[b->mesh_group[k]];
    FFA_BCUDA(cudaMemcpyAsync(c->Wtmp2 + b->mesh_voff[k] * c->d, W0[k], (size_t)b->mesh_n[k] * c->d * 8,
                              cudaMemcpyDefault, b->stream));
  }
  for (ffa_ctx* c : b->groups) {
    ffa_status st = load_W_records(c, c->Wtmp2, true, c->W, c->vrec);
    if (st != FFA_OK) {
      b->err = c->err;
      return st;
    }
    launch_init_polar(local_launch(c, false, c->vrec), b->stream);
    c->initialized = true;
    c->iter_total = 0;
  }
  FFA_BCUDA(cudaGetLastError());
  FFA_BCUDA(cudaStreamSynchronize(b->stream));
  b->initialized = true;
  return FFA_OK;
}

ffa_status ffa_batch_iterate(ffa_batch* b, int32_t max_iter, int32_t stop_at_tol, ffa_stats* stats,
                             int32_t* n_converged) {
  if (!b) return FFA_ERR_INVALID_ARG;
  b->err.clear();
  if (!b->initialized) {
    b->err = "ffa_batch_init has not been called";
    return FFA_ERR_NOT_INITIALIZED;
  }
  if (max_iter < 0) {
    b->err = "max_iter < 0";
    return FFA_ERR_INVALID_ARG;
  }
  ffa_status st;
  if (!b->g_batch && (st = batch_capture(b, b->check_every, true, &b->g_batch)) != FFA_OK) return st;
  if (!b->g_one && (st = batch_capture(b, 1, false, &b->g_one)) != FFA_OK) return st;
  if (!b->g_one_check && (st = batch_capture(b, 1, true, &b->g_one_check)) != FFA_OK) return st;
  const int ce = b->check_every;
  int done = 0, conv = 0;
  std::vector<int32_t> nconv(b->groups.size(), 0);
  while (done < max_iter) {
    const int left = max_iter - done;
    if (left >= ce) {
      FFA_BCUDA(cudaGraphLaunch(b->g_batch, b->stream));
      done += ce;
    } else {
      for (int k = 0; k < left - 1; ++k) FFA_BCUDA(cudaGraphLaunch(b->g_one, b->stream));
      FFA_BCUDA(cudaGraphLaunch(b->g_one_check, b->stream));
      done += left;
    }
    if (stop_at_tol || done == max_iter) {
      for (size_t gi = 0; gi < b->groups.size(); ++gi)
        FFA_BCUDA(cudaMemcpyAsync(&nconv[gi], b->groups[gi]->n_converged, sizeof(int32_t), cudaMemcpyDeviceToHost,
                                  b->stream));
      FFA_BCUDA(cudaStreamSynchronize(b->stream));
      conv = 0;
      for (int32_t x : nconv) conv += x;
      if (stop_at_tol && conv == b->n_mesh) break;
    }
  }
  for (ffa_ctx* c : b->groups) c->iter_total += done;
  if (stats) {
    for (int k = 0; k < b->n_mesh; ++k) {
      ffa_ctx* c = b->groups[b->mesh_group[k]];
      FFA_BCUDA(cudaMemcpy(&b->host_stats[k], c->mesh_stats + b->mesh_local[k], sizeof(ffa_stats),
                           cudaMemcpyDeviceToHost));
      b->host_stats[k].iters = done;
      b->host_stats[k].checked_iter = (int32_t)c->iter_total;
      stats[k] = b->host_stats[k];
    }
  }
  if (n_converged) *n_converged = conv;
  return FFA_OK;
}

ffa_status ffa_batch_autotune(ffa_batch* b, int32_t reps, ffa_tuning* out) {
  if (!b) return FFA_ERR_INVALID_ARG;
  b->err.clear();
  for (size_t gi = 0; gi < b->groups.size(); ++gi) {
    ffa_tuning t{};
    ffa_status st = ffa_autotune(b->groups[gi], reps, &t);
    if (st != FFA_OK) {
      b->err = b->groups[gi]->err;
      return st;
    }
    if (out) out[gi] = t;
  }
  if (b->g_batch) { cudaGraphExecDestroy(b->g_batch); b->g_batch = nullptr; }
  if (b->g_one) { cudaGraphExecDestroy(b->g_one); b->g_one = nullptr; }
  if (b->g_one_check) { cudaGraphExecDestroy(b->g_one_check); b->g_one_check = nullptr; }
  return FFA_OK;
}

int32_t ffa_batch_groups(const ffa_batch* b) { return b ? (int32_t)b->groups.size() : 0; }

ffa_status ffa_batch_get_W(ffa_batch* b, int32_t mesh, double* W_out) {
  if (!b || !W_out || mesh < 0 || mesh >= b->n_mesh) return FFA_ERR_INVALID_ARG;
  ffa_ctx* c = b->groups[b->mesh_group[mesh]];
  FFA_BCUDA(cudaMemcpyAsync(W_out, c->W + b->mesh_voff[mesh] * c->d, (size_t)b->mesh_n[mesh] * c->d * 8,
                            cudaMemcpyDefault, b->stream));
  FFA_BCUDA(cudaStreamSynchronize(b->stream));
  return FFA_OK;
}

}  // extern "C"
