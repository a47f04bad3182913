// C ABI of libffadmm (include/ffadmm.h): setup of the mesh operators and the
// factorized W-step operator, device state, and the CUDA-graph driver of the
// iteration (paper Algorithm 1; Algorithm 2 without the rescaling branch).
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "ffa_internal.h"

using namespace ffa;

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
  NodeDev* nodes = nullptr;
  int32_t* rows = nullptr;
  float* blocks = nullptr;
  Task *fwd_t = nullptr, *bwd_t = nullptr;
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

// Element frames and P1 hat-function gradients (Supplemental, "Computing the
// Jacobian map"): E has rows v_j - v_0 in the element frame (the intrinsic frame
// e1 = (v1-v0)/|v1-v0|, e2 = n x e1 for a triangle in R^3); the gradient of the
// hat function of vertex j is column j of E^{-1}; w = |det E| / d!.
bool element_geometry(int d, int d_in, const double* V, const int32_t* t, double g[3][3], double& w) {
  double E[3][3] = {{0}};
  const double* v0 = V + (int64_t)t[0] * d_in;
  if (d_in == d) {
    for (int j = 0; j < d; ++j) {
      const double* vj = V + (int64_t)t[j + 1] * d_in;
      for (int a = 0; a < d; ++a) E[j][a] = vj[a] - v0[a];
    }
  } else {
    const double* v1 = V + (int64_t)t[1] * 3;
    const double* v2 = V + (int64_t)t[2] * 3;
    double a[3] = {v1[0] - v0[0], v1[1] - v0[1], v1[2] - v0[2]};
    double b[3] = {v2[0] - v0[0], v2[1] - v0[1], v2[2] - v0[2]};
    const double la = std::sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
    double nrm[3] = {a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]};
    const double ln = std::sqrt(nrm[0] * nrm[0] + nrm[1] * nrm[1] + nrm[2] * nrm[2]);
    if (!(la > 0) || !(ln > 0)) return false;
    double e1[3] = {a[0] / la, a[1] / la, a[2] / la};
    for (double& c : nrm) c /= ln;
    double e2[3] = {nrm[1] * e1[2] - nrm[2] * e1[1], nrm[2] * e1[0] - nrm[0] * e1[2], nrm[0] * e1[1] - nrm[1] * e1[0]};
    E[0][0] = la;
    E[0][1] = 0.0;
    E[1][0] = b[0] * e1[0] + b[1] * e1[1] + b[2] * e1[2];
    E[1][1] = b[0] * e2[0] + b[1] * e2[1] + b[2] * e2[2];
  }
  double inv[3][3];
  double det;
  if (d == 2) {
    det = E[0][0] * E[1][1] - E[0][1] * E[1][0];
    if (!(std::fabs(det) > 0) || !std::isfinite(det)) return false;
    inv[0][0] = E[1][1] / det;
    inv[0][1] = -E[0][1] / det;
    inv[1][0] = -E[1][0] / det;
    inv[1][1] = E[0][0] / det;
    w = std::fabs(det) / 2.0;
  } else {
    const double c00 = E[1][1] * E[2][2] - E[1][2] * E[2][1];
    const double c01 = E[1][2] * E[2][0] - E[1][0] * E[2][2];
    const double c02 = E[1][0] * E[2][1] - E[1][1] * E[2][0];
    det = E[0][0] * c00 + E[0][1] * c01 + E[0][2] * c02;
    if (!(std::fabs(det) > 0) || !std::isfinite(det)) return false;
    inv[0][0] = c00 / det;
    inv[1][0] = c01 / det;
    inv[2][0] = c02 / det;
    inv[0][1] = (E[0][2] * E[2][1] - E[0][1] * E[2][2]) / det;
    inv[1][1] = (E[0][0] * E[2][2] - E[0][2] * E[2][0]) / det;
    inv[2][1] = (E[0][1] * E[2][0] - E[0][0] * E[2][1]) / det;
    inv[0][2] = (E[0][1] * E[1][2] - E[0][2] * E[1][1]) / det;
    inv[1][2] = (E[0][2] * E[1][0] - E[0][0] * E[1][2]) / det;
    inv[2][2] = (E[0][0] * E[1][1] - E[0][1] * E[1][0]) / det;
    w = std::fabs(det) / 6.0;
  }
  for (int j = 0; j < d; ++j)
    for (int a = 0; a < d; ++a) g[j][a] = inv[a][j];  // g_{j+1}[a] = (E^{-1})[a][j]
  return true;
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
  return L;
}

SolveData solve_data(ffa_ctx* ctx) {
  SolveData S;
  S.d = ctx->d;
  S.nF = ctx->nF;
  S.ell_width = ctx->ell_width;
  S.ell_col = ctx->ell_col;
  S.ell_val = ctx->ell_val;
  S.nodes = ctx->nodes;
  S.rows = ctx->rows;
  S.blocks = ctx->blocks;
  S.fwd_tasks = ctx->fwd_t;
  S.bwd_tasks = ctx->bwd_t;
  S.fwd_off = ctx->fwd_off;
  S.bwd_off = ctx->bwd_off;
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
    launch_residual(S, nullptr, 0, s);
    launch_supernodal_solve(S, s);
  }
  if (ev) cudaEventRecord(ev[PH_WSTEP], s);
  VertexLaunch V{};
  V.d = ctx->d;
  V.fp64 = ctx->fp64;
  V.n = ctx->n;
  V.Wnew_free = ctx->X;
  V.corr = ctx->x;
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
  launch_local_step(local_launch(ctx, check, ctx->vrec), s);
  if (ev) cudaEventRecord(ev[PH_LOCAL], s);
  if (check) {
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
  if (p.energy != FFA_SYM_DIRICHLET && p.energy != FFA_SYM_GRADIENT) msg = "unknown energy";
  else if (!(p.rho > 0) || !std::isfinite(p.rho)) msg = "rho must be positive";
  else if (!(p.eps_abs >= 0) || !(p.eps_rel >= 0)) msg = "eps_abs/eps_rel must be >= 0";
  else if (p.check_every < 1 || p.check_every > 100000) msg = "check_every must be in [1, 100000]";
  else if (p.local_precision != FFA_LOCAL_FP32 && p.local_precision != FFA_LOCAL_FP64) msg = "unknown precision";
  else if (p.refine_sweeps < 1 || p.refine_sweeps > 16) msg = "refine_sweeps must be in [1, 16]";
  else if (p.nd_leaf_size < 8 || p.nd_leaf_size > 512) msg = "nd_leaf_size must be in [8, 512]";
  else if (p.host_threads < 0) msg = "host_threads must be >= 0";
  else return FFA_OK;
  return FFA_ERR_INVALID_ARG;
}

ffa_status create_impl(ffa_ctx* ctx, const ffa_mesh* mesh, const int32_t* pin_idx, int32_t n_pin,
                       const double* pin_pos_in, const ffa_params* params, void* stream) {
  if (!mesh) return fail(ctx, FFA_ERR_INVALID_ARG, "mesh is NULL");
  ffa_default_params(&ctx->prm);
  if (params) ctx->prm = *params;
  {
    std::string msg;
    if (validate_params(ctx->prm, msg) != FFA_OK) return fail(ctx, FFA_ERR_INVALID_ARG, msg);
  }
  const int n = mesh->n, m = mesh->m, d = mesh->d, d_in = mesh->d_in;
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
  std::vector<int32_t> free_of(n, -1), free_vertex;
  for (int v = 0; v < n; ++v)
    if (v2pin[v] < 0) {
      free_of[v] = (int32_t)free_vertex.size();
      free_vertex.push_back(v);
    }
  const int nF = (int)free_vertex.size();
  ctx->nF = nF;
  // incidence CSR over all vertices
  std::vector<int64_t> inc_ptr(n + 1, 0);
  for (int64_t q = 0; q < (int64_t)m * (d + 1); ++q) inc_ptr[T[q] + 1]++;
  for (int v = 0; v < n; ++v) inc_ptr[v + 1] += inc_ptr[v];
  std::vector<int32_t> inc(inc_ptr[n]);
  {
    std::vector<int64_t> fill(inc_ptr.begin(), inc_ptr.end() - 1);
    for (int i = 0; i < m; ++i)
      for (int j = 0; j <= d; ++j) inc[fill[T[(int64_t)i * (d + 1) + j]]++] = i * (d + 1) + j;
  }
  auto grad_of = [&](int i, int j, double out[3]) {  // hat gradient of local vertex j
    for (int a = 0; a < d; ++a) {
      if (j > 0) out[a] = g[(int64_t)i * d * d + (j - 1) * d + a];
      else {
        double s = 0;
        for (int jj = 0; jj < d; ++jj) s += g[(int64_t)i * d * d + jj * d + a];
        out[a] = -s;
      }
    }
  };
  // rows of L for free vertices: free-free (free numbering) and free-pinned parts
  std::vector<int64_t> Ap(nF + 1, 0), Cp(nF + 1, 0);
  std::vector<int32_t> Ai, Ci;
  std::vector<double> Ax, Cx;
  {
    std::vector<int32_t> pos(n, -1), touched;
    std::vector<double> acc;
    for (int f = 0; f < nF; ++f) {
      const int v = free_vertex[f];
      touched.clear();
      acc.clear();
      for (int64_t q = inc_ptr[v]; q < inc_ptr[v + 1]; ++q) {
        const int i = inc[q] / (d + 1), j = inc[q] % (d + 1);
        double gj[3], gl[3];
        grad_of(i, j, gj);
        const double mu = rho * w[i];
        for (int l = 0; l <= d; ++l) {
          grad_of(i, l, gl);
          double dotv = 0;
          for (int a = 0; a < d; ++a) dotv += gj[a] * gl[a];
          const int u = T[(int64_t)i * (d + 1) + l];
          if (pos[u] < 0) {
            pos[u] = (int32_t)touched.size();
            touched.push_back(u);
            acc.push_back(0.0);
          }
          acc[pos[u]] += mu * dotv;
        }
      }
      std::vector<std::pair<int32_t, double>> fr, cr;
      for (size_t k = 0; k < touched.size(); ++k) {
        const int u = touched[k];
        if (free_of[u] >= 0) fr.push_back({free_of[u], acc[k]});
        else cr.push_back({v2pin[u], acc[k]});
        pos[u] = -1;
      }
      std::sort(fr.begin(), fr.end());
      std::sort(cr.begin(), cr.end());
      for (auto& pr : fr) { Ai.push_back(pr.first); Ax.push_back(pr.second); }
      for (auto& pr : cr) { Ci.push_back(pr.first); Cx.push_back(pr.second); }
      Ap[f + 1] = (int64_t)Ai.size();
      Cp[f + 1] = (int64_t)Ci.size();
    }
  }
  std::vector<double> coords((size_t)nF * 3, 0.0);
  for (int f = 0; f < nF; ++f)
    for (int a = 0; a < d_in; ++a) coords[(size_t)f * 3 + a] = V[(int64_t)free_vertex[f] * d_in + a];

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
    std::string msg;
    int rc = build_factor(in, fac, msg);
    if (rc == 3) return fail(ctx, FFA_ERR_SINGULAR_SYSTEM, msg);
    if (rc != 0) return fail(ctx, FFA_ERR_INVALID_ARG, msg);
  }
  ctx->info.setup_seconds_analyze = fac.t_analyze;
  ctx->info.setup_seconds_factor = fac.t_factor;
  ctx->info.factor_entries = (int64_t)fac.blocks.size();
  ctx->info.factor_flops = fac.flops;
  ctx->info.n_supernodes = (int32_t)fac.nodes.size();
  ctx->info.n_levels = fac.n_levels;

  // ---- eliminated-order vertex maps, ELL of L_FF, CSR of L_FC
  std::vector<int32_t> row_vertex(nF), v2e(n, -1);
  for (int c = 0; c < nF; ++c) {
    row_vertex[c] = free_vertex[fac.perm[c]];
    v2e[row_vertex[c]] = c;
  }
  int width = 1;
  for (int f = 0; f < nF; ++f) width = std::max<int>(width, (int)(Ap[f + 1] - Ap[f]));
  std::vector<int32_t> ell_col((size_t)width * nF);
  std::vector<double> ell_val((size_t)width * nF, 0.0);
  std::vector<int64_t> fc_ptr(nF + 1, 0);
  std::vector<int32_t> fc_col;
  std::vector<double> fc_val;
  for (int c = 0; c < nF; ++c) {
    const int f = fac.perm[c];
    int q = 0;
    for (int64_t k = Ap[f]; k < Ap[f + 1]; ++k, ++q) {
      ell_col[(size_t)q * nF + c] = fac.iperm[Ai[k]];
      ell_val[(size_t)q * nF + c] = Ax[k];
    }
    for (; q < width; ++q) ell_col[(size_t)q * nF + c] = c;
    for (int64_t k = Cp[f]; k < Cp[f + 1]; ++k) {
      fc_col.push_back(Ci[k]);
      fc_val.push_back(Cx[k]);
    }
    fc_ptr[c + 1] = (int64_t)fc_col.size();
  }
  ctx->ell_width = width;

  // ---- supernode tables and per-level task lists
  std::vector<NodeDev> nodes(fac.nodes.size());
  std::vector<std::vector<Task>> fl(fac.n_levels), bl(fac.n_levels);
  for (size_t s = 0; s < fac.nodes.size(); ++s) {
    const Supernode& sn = fac.nodes[s];
    nodes[s] = NodeDev{sn.col0, sn.ncol, sn.nrow, sn.ld, sn.row_off, sn.blk_off};
    const int ntot = sn.ncol + sn.nrow;
    if (sn.ncol == 0) continue;
    for (int r0 = 0; r0 < ntot; r0 += kFwdRows)
      for (int c0 = 0; c0 < sn.ncol; c0 += kFwdCols) {
        const int rmax = std::min(r0 + kFwdRows, ntot) - 1;
        if (rmax < c0) continue;  // entirely above the diagonal of inv(L_ss)
        fl[sn.level].push_back(Task{(int32_t)s, r0, c0, 0});
      }
    for (int c0 = 0; c0 < sn.ncol; c0 += kBwdCols)
      for (int r0 = 0; r0 < ntot; r0 += kBwdRows) {
        const int rmax = std::min(r0 + kBwdRows, ntot) - 1;
        if (rmax < c0) continue;
        bl[sn.level].push_back(Task{(int32_t)s, r0, c0, 0});
      }
  }
  std::vector<Task> fwd_all, bwd_all;
  ctx->fwd_off.assign(1, 0);
  ctx->bwd_off.assign(1, 0);
  for (int l = 0; l < fac.n_levels; ++l) {
    fwd_all.insert(fwd_all.end(), fl[l].begin(), fl[l].end());
    bwd_all.insert(bwd_all.end(), bl[l].begin(), bl[l].end());
    ctx->fwd_off.push_back((int64_t)fwd_all.size());
    ctx->bwd_off.push_back((int64_t)bwd_all.size());
  }

  // ---- device uploads
  if ((st = upload(ctx, &ctx->nodes, nodes)) != FFA_OK) return st;
  if ((st = upload(ctx, &ctx->rows, fac.rows)) != FFA_OK) return st;
  if ((st = upload(ctx, &ctx->blocks, fac.blocks)) != FFA_OK) return st;
  if ((st = upload(ctx, &ctx->fwd_t, fwd_all)) != FFA_OK) return st;
  if ((st = upload(ctx, &ctx->bwd_t, bwd_all)) != FFA_OK) return st;
  if ((st = upload(ctx, &ctx->ell_col, ell_col)) != FFA_OK) return st;
  if ((st = upload(ctx, &ctx->ell_val, ell_val)) != FFA_OK) return st;
  if ((st = upload(ctx, &ctx->fc_ptr, fc_ptr)) != FFA_OK) return st;
  if ((st = upload(ctx, &ctx->fc_col, fc_col)) != FFA_OK) return st;
  if ((st = upload(ctx, &ctx->fc_val, fc_val)) != FFA_OK) return st;
  if ((st = upload(ctx, &ctx->inc_ptr, inc_ptr)) != FFA_OK) return st;
  if ((st = upload(ctx, &ctx->inc, inc)) != FFA_OK) return st;
  if ((st = upload(ctx, &ctx->row_vertex, row_vertex)) != FFA_OK) return st;
  if ((st = upload(ctx, &ctx->v2e, v2e)) != FFA_OK) return st;
  if ((st = upload(ctx, &ctx->v2pin, v2pin)) != FFA_OK) return st;
  if ((st = upload(ctx, &ctx->pin_pos, pin_pos)) != FFA_OK) return st;
  // element arrays: indices (d+1) x m, gradients d*d x m, w, mu
  {
    std::vector<int32_t> idx((size_t)(d + 1) * m);
    for (int i = 0; i < m; ++i)
      for (int j = 0; j <= d; ++j) idx[(size_t)j * m + i] = T[(int64_t)i * (d + 1) + j];
    if ((st = upload(ctx, &ctx->e.idx, idx)) != FFA_OK) return st;
    std::vector<double> gs((size_t)d * d * m), mu(m);
    for (int i = 0; i < m; ++i) {
      for (int q = 0; q < d * d; ++q) gs[(size_t)q * m + i] = g[(int64_t)i * d * d + q];
      mu[i] = rho * w[i];
    }
    if ((st = upload_real(ctx, &ctx->e.g, gs)) != FFA_OK) return st;
    if ((st = upload_real(ctx, &ctx->e.w, w)) != FFA_OK) return st;
    if ((st = upload_real(ctx, &ctx->e.mu, mu)) != FFA_OK) return st;
  }
  const size_t R = ctx->rsz;
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
  ctx->n_local_blocks = (m + kLocalBlock - 1) / kLocalBlock;
  ctx->n_vert_blocks = (n + kVertexBlock - 1) / kVertexBlock;
  ctx->n_res_blocks = (nF + kVertexBlock - 1) / kVertexBlock;
  if ((st = dalloc(ctx, &ctx->local_partials, (size_t)ctx->n_local_blocks * NQ)) != FFA_OK) return st;
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
      (int64_t)n * d * 16;
  int64_t nz = 0;
  for (const Supernode& sn : fac.nodes) nz += (int64_t)sn.ncol * sn.nrow + (int64_t)sn.ncol * (sn.ncol + 1) / 2;
  // (forward and backward each read every nonzero of every B_s once)
  ctx->info.bytes_global_sweep = 2 * nz * 4 + (int64_t)width * nF * 12 + (int64_t)nF * d * (8 * 3 + 4 * 6);
  ctx->info.n = n;
  ctx->info.m = m;
  ctx->info.d = d;
  ctx->info.d_in = d_in;
  ctx->info.n_pin = n_pin;
  ctx->info.n_free = nF;
  int lev_launch = 0;
  for (int l = 0; l < fac.n_levels; ++l)
    lev_launch += (ctx->fwd_off[l + 1] > ctx->fwd_off[l]) + (ctx->bwd_off[l + 1] > ctx->bwd_off[l]);
  const int sweeps = ctx->prm.refine_sweeps;
  ctx->info.kernels_per_iteration = 1 + sweeps * (1 + lev_launch) + (sweeps - 1) + 1 + 1;
  ctx->info.kernels_per_check = 3;
  (void)t_setup0;
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
  return FFA_OK;
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
  return FFA_OK;
}

ffa_status ffa_init(ffa_ctx* ctx, const double* W0) {
  if (!ctx) return FFA_ERR_INVALID_ARG;
  if (!W0) return fail(ctx, FFA_ERR_INVALID_ARG, "W0 is NULL");
  ctx->err.clear();
  ffa_status st = load_W_records(ctx, W0, true, ctx->W, ctx->vrec);
  if (st != FFA_OK) return st;
  launch_init_polar(local_launch(ctx, false, ctx->vrec), ctx->stream);
  FFA_CUDA(cudaGetLastError());
  FFA_CUDA(cudaStreamSynchronize(ctx->stream));
  ctx->initialized = true;
  ctx->iter_total = 0;
  return FFA_OK;
}

ffa_status ffa_iterate(ffa_ctx* ctx, int32_t max_iter, int32_t stop_at_tol, ffa_stats* stats) {
  if (!ctx) return FFA_ERR_INVALID_ARG;
  ctx->err.clear();
  if (!ctx->initialized) return fail(ctx, FFA_ERR_NOT_INITIALIZED, "ffa_init has not been called");
  if (max_iter < 0) return fail(ctx, FFA_ERR_INVALID_ARG, "max_iter < 0");
  ffa_status st = ensure_graphs(ctx);
  if (st != FFA_OK) return st;
  const int ce = ctx->prm.check_every;
  int done = 0;
  bool have = false;
  while (done < max_iter) {
    const int left = max_iter - done;
    if (left >= ce) {
      FFA_CUDA(cudaGraphLaunch(ctx->g_batch, ctx->stream));
      done += ce;
    } else {
      for (int k = 0; k < left - 1; ++k) FFA_CUDA(cudaGraphLaunch(ctx->g_one, ctx->stream));
      FFA_CUDA(cudaGraphLaunch(ctx->g_one_check, ctx->stream));
      done += left;
    }
    if (stop_at_tol || done == max_iter) {
      FFA_CUDA(cudaMemcpyAsync(ctx->stats_h, ctx->stats_d, sizeof(ffa_stats), cudaMemcpyDeviceToHost, ctx->stream));
      FFA_CUDA(cudaStreamSynchronize(ctx->stream));
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
  }
  ctx->iter_total += done;
  if (!have) {
    ctx->last = ffa_stats{};
  }
  ctx->last.iters = done;
  if (stats) *stats = ctx->last;
  return FFA_OK;
}

ffa_status ffa_get_W(ffa_ctx* ctx, double* W_out) {
  if (!ctx) return FFA_ERR_INVALID_ARG;
  if (!W_out) return fail(ctx, FFA_ERR_INVALID_ARG, "W_out is NULL");
  ctx->err.clear();
  FFA_CUDA(cudaMemcpyAsync(W_out, ctx->W, (size_t)ctx->n * ctx->d * 8, cudaMemcpyDefault, ctx->stream));
  FFA_CUDA(cudaStreamSynchronize(ctx->stream));
  return FFA_OK;
}

ffa_status ffa_get_state(ffa_ctx* ctx, double* U, double* P, double* Lam) {
  if (!ctx) return FFA_ERR_INVALID_ARG;
  ctx->err.clear();
  const int m = ctx->m, d = ctx->d;
  const size_t R = ctx->rsz;
  const int ps = d == 2 ? 3 : 6, us = d == 2 ? 2 : 4;
  std::vector<unsigned char> hu((size_t)m * us * R), hp((size_t)m * ps * R), hl((size_t)m * d * d * R);
  FFA_CUDA(cudaMemcpyAsync(hu.data(), ctx->e.U, hu.size(), cudaMemcpyDeviceToHost, ctx->stream));
  FFA_CUDA(cudaMemcpyAsync(hp.data(), ctx->e.P, hp.size(), cudaMemcpyDeviceToHost, ctx->stream));
  FFA_CUDA(cudaMemcpyAsync(hl.data(), ctx->e.Lam, hl.size(), cudaMemcpyDeviceToHost, ctx->stream));
  FFA_CUDA(cudaStreamSynchronize(ctx->stream));
  auto get = [&](const std::vector<unsigned char>& h, size_t k) -> double {
    return ctx->fp64 ? reinterpret_cast<const double*>(h.data())[k] : (double)reinterpret_cast<const float*>(h.data())[k];
  };
  std::vector<double> oU((size_t)m * d * d), oP((size_t)m * d * d), oL((size_t)m * d * d);
  for (int i = 0; i < m; ++i) {
    double* u = oU.data() + (size_t)i * d * d;
    double* p = oP.data() + (size_t)i * d * d;
    double* l = oL.data() + (size_t)i * d * d;
    if (d == 2) {
      const double c = get(hu, i), s = get(hu, (size_t)m + i);
      u[0] = c; u[1] = -s; u[2] = s; u[3] = c;
      p[0] = get(hp, i); p[1] = p[2] = get(hp, (size_t)m + i); p[3] = get(hp, 2 * (size_t)m + i);
    } else {
      const double w = get(hu, i), x = get(hu, (size_t)m + i), y = get(hu, 2 * (size_t)m + i), z = get(hu, 3 * (size_t)m + i);
      u[0] = 1 - 2 * (y * y + z * z); u[1] = 2 * (x * y - z * w); u[2] = 2 * (x * z + y * w);
      u[3] = 2 * (x * y + z * w); u[4] = 1 - 2 * (x * x + z * z); u[5] = 2 * (y * z - x * w);
      u[6] = 2 * (x * z - y * w); u[7] = 2 * (y * z + x * w); u[8] = 1 - 2 * (x * x + y * y);
      p[0] = get(hp, i); p[1] = p[3] = get(hp, (size_t)m + i); p[2] = p[6] = get(hp, 2 * (size_t)m + i);
      p[4] = get(hp, 3 * (size_t)m + i); p[5] = p[7] = get(hp, 4 * (size_t)m + i); p[8] = get(hp, 5 * (size_t)m + i);
    }
    for (int q = 0; q < d * d; ++q) l[q] = get(hl, (size_t)q * m + i);
  }
  const size_t bytes = (size_t)m * d * d * 8;
  if (U) FFA_CUDA(cudaMemcpy(U, oU.data(), bytes, cudaMemcpyDefault));
  if (P) FFA_CUDA(cudaMemcpy(P, oP.data(), bytes, cudaMemcpyDefault));
  if (Lam) FFA_CUDA(cudaMemcpy(Lam, oL.data(), bytes, cudaMemcpyDefault));
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
  launch_sum_partials(ctx->local_partials, ctx->n_local_blocks, NQ, ctx->sums_d, ctx->stream);
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
  launch_sum_partials(ctx->local_partials, ctx->n_local_blocks, NQ, ctx->sums_d, ctx->stream);
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
  *info = ctx->info;
  return FFA_OK;
}

ffa_status ffa_profile_phases(ffa_ctx* ctx, int32_t reps, ffa_phase_times* out) {
  if (!ctx || !out) return FFA_ERR_INVALID_ARG;
  ctx->err.clear();
  if (!ctx->initialized) return fail(ctx, FFA_ERR_NOT_INITIALIZED, "ffa_init has not been called");
  if (reps < 1) return fail(ctx, FFA_ERR_INVALID_ARG, "reps < 1");
  cudaEvent_t ev[PH_N + 1];
  for (auto& e : ev) FFA_CUDA(cudaEventCreate(&e));
  double acc[PH_N + 1] = {0};
  for (int r = 0; r < reps; ++r) {
    FFA_CUDA(cudaEventRecord(ev[PH_N], ctx->stream));
    enqueue_iteration(ctx, r == reps - 1, ev);
    FFA_CUDA(cudaGetLastError());
    FFA_CUDA(cudaEventSynchronize(ev[PH_CHECK]));
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
  ctx->iter_total += reps;
  out->reps = reps;
  out->ms_gather = acc[PH_GATHER] / reps;
  out->ms_wstep = acc[PH_WSTEP] / reps;
  out->ms_vertex = acc[PH_VERTEX] / reps;
  out->ms_local = acc[PH_LOCAL] / reps;
  out->ms_check = acc[PH_CHECK];
  out->ms_iteration = acc[PH_N] / reps;
  return FFA_OK;
}

ffa_status ffa_last_wstep_residual(ffa_ctx* ctx, double* rel) {
  if (!ctx || !rel) return FFA_ERR_INVALID_ARG;
  ctx->err.clear();
  SolveData S = solve_data(ctx);
  launch_residual(S, ctx->res_partials, (int)ctx->n_res_blocks, ctx->stream);
  launch_sum_partials(ctx->res_partials, ctx->n_res_blocks, 2, ctx->sums_d, ctx->stream);
  FFA_CUDA(cudaGetLastError());
  FFA_CUDA(cudaMemcpyAsync(ctx->sums_h, ctx->sums_d, 2 * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  FFA_CUDA(cudaStreamSynchronize(ctx->stream));
  *rel = ctx->sums_h[1] > 0 ? std::sqrt(ctx->sums_h[0] / ctx->sums_h[1]) : std::sqrt(ctx->sums_h[0]);
  return FFA_OK;
}

}  // extern "C"
