/*
 * ffadmm.h - C ABI of the GB300 flip-free ADMM library (libffadmm.so).
 *
 * The library minimizes a flip-free distortion energy
 *     E(W) = sum_i w_i f((G W)_i) + chi_+(det (G W)_i)              (paper eq. genericdeformationenergy)
 * over target vertex positions W with the three-block splitting scheme of
 * Stein, Li & Solomon, "A Splitting Scheme for Flip-Free Distortion Energies"
 * (Algorithm 1; Algorithm 2 without penalty rescaling): a global W step with a
 * fixed operator L = sum_i mu_i G_i^T G_i (eq. solvinginw), closed-form per-element U
 * (Procrustes, eqs. rawoptimizationinudecoupled/optimizationinudecoupled) and P (prox,
 * eqs. optimizinginp/rootfindinginp) steps, and the scaled multiplier update
 * (eq. lambdaupdate), with the primal/dual errors of eqs. primaldualerror/primaldualthresholds.
 *
 * Conventions shared by every call:
 *   - Sizes: n vertices, m elements, element dimension d (2 = triangles,
 *     3 = tetrahedra), source dimension d_in (2 or 3; d_in = 3 with d = 2 means a
 *     surface mesh with intrinsic 2x2 Jacobians, paper Supplemental).  The target
 *     dimension is d.
 *   - Arrays are dense and row-major: V is n x d_in, T is m x (d+1), W is n x d,
 *     per-element matrices are m x d x d.  Doubles unless stated otherwise.
 *   - J_i = (G W)_i has column k equal to the gradient of target coordinate k on
 *     element i (paper Supplemental, "Computing the Jacobian map").
 *   - Pointer arguments marked "host or device" may point to host memory or to
 *     device memory of the context's GPU; the library copies through unified
 *     addressing.  Input memory is owned by the caller and only read during the
 *     call; output memory is owned by the caller and written by the call.  The
 *     library never frees caller memory.
 *   - Every call returns an ffa_status; no exception crosses the ABI.  On error,
 *     ffa_last_error(ctx) returns a message owned by the context (valid until the
 *     next call on it).  A context is used by one host thread at a time.
 *   - All GPU work of a context runs on its stream, in order.  Calls that return
 *     values to the host synchronize that stream.
 *   - A context made without a stream works on a private non-blocking stream,
 *     which does not wait for work on any other stream (the legacy default
 *     stream included).  Device memory passed to a call must therefore already
 *     hold its contents (the work that writes it finished, or ordered before the
 *     call on the context's stream), and device memory the call writes must not
 *     be in use by pending work elsewhere.  The Python binding synchronizes
 *     the tensor's device before it passes a CUDA tensor.
 */
#ifndef FFADMM_H
#define FFADMM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ffa_ctx ffa_ctx;
typedef struct ffa_batch ffa_batch;

typedef enum {
  FFA_OK = 0,
  FFA_ERR_INVALID_ARG = 1,        /* bad size, index, pointer or parameter */
  FFA_ERR_DEGENERATE_ELEMENT = 2, /* a source element has w_i <= 0 */
  FFA_ERR_SINGULAR_SYSTEM = 3,    /* L restricted to free vertices is not SPD */
  FFA_ERR_CUDA = 4,               /* a CUDA runtime call failed */
  FFA_ERR_OOM = 5,                /* host or device allocation failed */
  FFA_ERR_NAN = 6,                /* a non-finite value appeared in the iterate */
  FFA_ERR_NOT_INITIALIZED = 7,    /* ffa_iterate before ffa_init */
  FFA_ERR_FLIPPED = 8,            /* gradient requested at a map with det J_i <= 0 */
  FFA_ERR_TIMEOUT = 9             /* a bounded device-side wait gave up; results are invalid */
} ffa_status;

typedef enum {
  FFA_SYM_DIRICHLET = 0, /* f(X) = (|X|^2 + |X^-1|^2) / 2          (eq. symmetricdirichletdefiningfunction) */
  FFA_SYM_GRADIENT = 1,  /* f(X) = |X|^2 / 2 - log det X            (eq. symmetricgradientdefiningfunction) */
  FFA_SYM_ARAP = 2       /* f(X) = (|X - R|^2 + |X^-1 - R^-1|^2) / 2, R the rotation of X: the
                            symmetric ARAP energy, one more rotation-invariant defining function
                            plugged into the same scheme (Sec. 3 leaves the choice of f open);
                            its P step solves (w+mu) p^4 - (w + mu q) p^3 + w p - w = 0 per
                            eigenvalue.  Not with penalty_schedule 1 (Lemma 1 bounds SD and SG
                            only) nor with ffa_energy_noalloc. */
} ffa_energy_kind;

typedef enum {
  FFA_LOCAL_FP32 = 0, /* local step in float; reductions and the W step in double */
  FFA_LOCAL_FP64 = 1  /* local step in double as well */
} ffa_precision;

typedef struct {
  int32_t n;         /* vertices, >= d+1 */
  int32_t m;         /* elements, >= 1 */
  int32_t d;         /* 2 or 3 */
  int32_t d_in;      /* 2 or 3, >= d */
  const double* V;   /* n x d_in source positions, host or device */
  const int32_t* T;  /* m x (d+1) vertex indices, host or device; positively oriented */
} ffa_mesh;

typedef struct {
  ffa_energy_kind energy;
  double rho;              /* penalties mu_i = rho * w_i (rho = 1: the paper's initial mu_i = w_i) */
  double eps_abs;          /* thresholds of eq. primaldualthresholds */
  double eps_rel;
  int32_t check_every;     /* evaluate the termination test every this many iterations (>= 1) */
  int32_t require_flip_free; /* 1: convergence also needs det J_i > 0 for all i (Sec. 6) */
  ffa_precision local_precision;
  int32_t refine_sweeps;   /* W step: residual-correction sweeps per iteration (>= 1) */
  int32_t nd_leaf_size;    /* W step setup: nested-dissection leaf size (8..512) */
  int32_t host_threads;    /* W step setup: host threads for the factorization (0 = all) */
  int32_t solve_schedule;  /* W step: 0 one launch per elimination-tree level, 1 one launch per
                              triangular solve whose blocks take ready tasks from a queue that
                              finished supernodes refill (default), 2 the same queue with each
                              block split into a producer warp that streams the factor with bulk
                              copies into a shared-memory ring and eight consumer warps */
  int32_t penalty_schedule;/* 0: mu_i = rho * w_i, fixed (default; L is decomposed once).
                              1: the paper's Algorithm 2 (Sec. 6, "Rescaling mu_i and Lambda"):
                              mu_i = max(mu_min,i, w_i) at ffa_init (mu_min of Prop. 1 with the
                              gradient bound B_i = sqrt(5 (1 + |grad f(P_i)|^2)) of Sec. 6), then
                              after iterations 1..5 and every floor(5 (3/2)^p) iterations (p =
                              events so far) each mu_i is multiplied (divided) by rescale_rho/2
                              when e_prim_i > rescale_rho e_dual_i (e_dual_i > rescale_rho
                              e_prim_i), never below mu_min,i/2, Lambda_i keeps mu_i Lambda_i, and L
                              is decomposed again (where factor_device says).  rho is ignored.  Single meshes of
                              one energy, SD or SG, only; not with ffa_forward_unrolled. */
  double rescale_rho;      /* the paper's rho of the rescaling rule (default 5) */
  int32_t local_variant;   /* 0: the paper's local step (Algorithm 1: U from (J + Lambda) P^{k-1}, then P;
                              default).  1: a joint (U, P) prox (not the paper's scheme): U is the
                              rotation nearest to J + Lambda and P the prox of symm(U^T (J + Lambda)),
                              the joint minimizer of w f(P) + mu/2 |U P - J - Lambda|^2 for the
                              rotation-invariant energies.  Not with ffa_forward_unrolled. */
  int32_t solve_subtree_height[2]; /* solve_schedule 1: bottom subtrees of the elimination tree of
                              at most this height whose supernodes are all small run as one task
                              of the forward / backward pass (one block, supernodes in order);
                              0 off, -1 the library's choice (default), at most 8 */
  int32_t prox_h;          /* proximal U term of eq. proximalfunctionu: 0 h_i = 0 (default; Sec. 6
                              switches it off when many elements start flipped), 1 h_i at the bound
                              of Prop. 1, h_i = 4 w_i^2 B_i^2 / mu_i with B_i = sqrt(5 (1 + |grad
                              f(P_i)|^2)) (gamma = 1, eps = 0 as Sec. 6 sets them), B_i from the P
                              given by ffa_init (P^0) or ffa_set_state.  The U step then takes
                              Q_i = (J_i + Lambda_i) P_i + (h_i / mu_i) U_i^{k-1}.  Fixed penalties,
                              the paper's local step and single meshes only (not with
                              penalty_schedule 1, local_variant 1, batches or ffa_forward_unrolled). */
  int32_t factor_device;   /* numeric decomposition of L_FF (Algorithm 2, decompose(L)), at setup and at
                              every rescaling of penalty_schedule 1: 0 on the host in double (default), 1 on
                              the device in float, 2 on the device in double.  The ordering and the
                              supernodes stay a host analysis; the device runs the multifrontal method over
                              the same tree and writes the same float blocks (1: each within float rounding
                              times the growth of the elimination; the W step's double residual sweeps
                              restore double accuracy).  With penalty_schedule 1 it also assembles the new
                              L on the device, so a rescaling event has no host work.  Device memory: every
                              front and every inv(L_ss) at once (sum over supernodes of (n_s + m_s)^2 +
                              n_s^2 elements), kept for the context's life with penalty_schedule 1 and
                              released after setup otherwise. */
  int32_t top_inverse_levels; /* the top levels of the elimination tree in the W step's solve (Sec. 4,
                              "Efficient Evaluation"): with T the columns of the supernodes on the top k
                              levels and S = L_TT L_TT^T the Schur complement of the rest, a solve runs the
                              forward pass below T, x_T = S^-1 t_T (t_T: the forward pass's right-hand
                              side at T) as one symmetric matrix-vector product, and the backward pass below
                              T.  S^-1 (float, lower 64 x 64 tiles) is computed on the device from the
                              factor blocks after every decomposition.  0 (default): off; -1: the
                              largest k whose S^-1 takes no more bytes than the factor blocks of those
                              levels (at most 16 supernodes and 16384 columns); k > 0: exactly the top k
                              levels (FFA_ERR_INVALID_ARG if that leaves no level below or exceeds those
                              limits).  Single-mesh contexts only (batched contexts use 0). */
} ffa_params;

typedef struct {
  int32_t iters;           /* iterations performed by the call */
  int32_t converged;       /* 1 if the termination test of eq. primaldualthresholds passed */
  int32_t n_flipped;       /* elements with det (G W)_i <= 0 at the last check */
  int32_t checked_iter;    /* total iteration count at which the stats were taken */
  double e_prim, e_dual;   /* eq. primaldualerror */
  double thr_prim, thr_dual; /* eq. primaldualthresholds */
  double energy_P;         /* sum_i w_i f(P_i) */
  double norm_GW, norm_P, norm_GtLambda;
  int32_t rescales;        /* penalty rescaling events since ffa_init (penalty_schedule 1) */
} ffa_stats;

typedef struct {
  int32_t n, m, d, d_in, n_pin, n_free;
  int64_t factor_entries;  /* stored entries of the supernodal factor blocks */
  int64_t factor_flops;    /* floating-point operations of the numeric factorization */
  int32_t n_supernodes, n_levels;
  double setup_seconds_analyze;   /* ordering + symbolic analysis (host) */
  double setup_seconds_factor;    /* numeric factorization (host) */
  int64_t device_bytes;    /* device memory held by the context */
  int64_t bytes_local_step;   /* algorithmic bytes of one local-step launch */
  int64_t bytes_global_sweep; /* algorithmic bytes of one W-step refinement sweep */
  int64_t bytes_solve_pass;   /* algorithmic bytes of one triangular pass (forward or backward):
                                 the stored nonzeros of every B_s, its structure indices, and
                                 the pass's input and output vectors */
  int32_t kernels_per_iteration; /* kernel launches of one iteration without the test */
  int32_t kernels_per_check;     /* extra launches of an iteration that runs the test */
  double seconds_refactor;       /* wall time spent assembling and decomposing L again at the rescaling
                                    events of penalty_schedule 1 (on the host or, with factor_device, on
                                    the device) */
  int32_t top_inverse_levels;    /* levels solved by S^-1 (top_inverse_levels), 0 if none */
  int32_t top_inverse_cols;      /* columns of those levels (the order of S) */
  int64_t bytes_top_product;     /* algorithmic bytes of one x_T = S^-1 t_T: the tiles of S^-1 and
                                    the two vectors */
  double setup_seconds_top_inverse; /* time of the last computation of S^-1 (device) */
} ffa_info;

typedef struct {
  int32_t reps;        /* iterations timed */
  double ms_gather;    /* W step: right-hand side G^T r */
  double ms_wstep;     /* W step: all refinement sweeps (residual + triangular solves) */
  double ms_vertex;    /* vertex update */
  double ms_local;     /* fused local step (U, P, Lambda) */
  double ms_check;     /* termination test of one check iteration */
  double ms_iteration; /* whole iteration, launched one kernel at a time */
  double ms_solve_forward;   /* one forward triangular pass of the W step (last sweep) */
  double ms_solve_backward;  /* one backward triangular pass of the W step (last sweep) */
  double ms_top_product;     /* x_T = S^-1 t_T between the passes (last sweep; 0 without it) */
} ffa_phase_times;

/* Initial map (the paper has no GPU counterpart; App. A, "Tutte's Energy"): the
 * minimizer of E_T(W) = sum over the mesh edges (i, j) of |W_i - W_j|^2 / |V_i - V_j|
 * with the boundary vertices held at boundary_pos.  Flip-free in 2D when the
 * boundary is convex (Tutte's theorem); the paper initializes with it.  One
 * sparse SPD solve: ordering and factorization on the host as for the W step,
 * FP32 supernodal passes with FP64 residual correction on the GPU until the
 * relative residual reaches 1e-13 or stops falling (at most 10 sweeps).
 *   mesh         : source mesh (V n x d_in, T); d = the target dimension (2 or 3)
 *   boundary     : n_boundary distinct vertex indices (host or device), >= 1
 *   boundary_pos : n_boundary x d positions (host or device)
 *   params       : nd_leaf_size, host_threads, solve_schedule are used (NULL = defaults)
 *   stream       : cudaStream_t or NULL (a private stream)
 *   W_out        : n x d result (host or device)
 *   rel_residual : optional: |b - L_II W_I| / |b| at the end
 * Errors: FFA_ERR_INVALID_ARG (sizes, indices, repeated boundary index, a zero-length
 * edge), FFA_ERR_SINGULAR_SYSTEM (an interior part with no boundary vertex), CUDA
 * errors; the message is in ffa_last_error(NULL).  Allocates and frees its own
 * device memory. */
ffa_status ffa_tutte(const ffa_mesh* mesh, const int32_t* boundary, int32_t n_boundary,
                     const double* boundary_pos, const ffa_params* params, void* stream,
                     double* W_out, double* rel_residual);

/* Fill *p with the defaults: symmetric Dirichlet, rho 1, eps_abs 1e-6, eps_rel 1e-5,
 * check_every 10, require_flip_free 1, FP32 local step, 2 refine sweeps,
 * leaf size 64, all host threads, solve schedule 1, fixed penalties (penalty
 * schedule 0), rescale_rho 5, the paper's local step, prox_h 0, factor_device 0,
 * top_inverse_levels 0. */
ffa_status ffa_default_params(ffa_params* p);

/* Prepare a solver for one mesh: element gradients and measures w_i (Supplemental,
 * "Computing the Jacobian map"; w_i of Sec. 3.1), the fixed operator
 * L = sum_i mu_i G_i^T G_i of eq. solvinginw restricted to the free vertices, and its
 * factorization, done once per mesh and rho (Sec. 4, "Efficient evaluation";
 * Algorithm 2, decompose(L)).
 *   mesh      : sizes and source geometry (host or device).
 *   pin_idx   : n_pin distinct vertex indices fixed by the constraint A W = b
 *               (eq. solvinginw / Algorithm 1); n_pin = 0 pins vertex 0 at the origin
 *               (Sec. 4, "Updating W").  Host or device; may be NULL if n_pin = 0.
 *   pin_pos   : n_pin x d positions b of the pinned vertices, host or device.
 *   params    : solver parameters (NULL = defaults).
 *   stream    : cudaStream_t to run on (NULL = a stream owned by the context).
 *   out       : receives the context; NULL on failure.
 * Errors: FFA_ERR_INVALID_ARG (sizes, indices out of range, repeated pins),
 * FFA_ERR_DEGENERATE_ELEMENT, FFA_ERR_SINGULAR_SYSTEM, FFA_ERR_OOM, FFA_ERR_CUDA. */
ffa_status ffa_create(const ffa_mesh* mesh, const int32_t* pin_idx, int32_t n_pin,
                      const double* pin_pos, const ffa_params* params, void* stream,
                      ffa_ctx** out);

/* Release every resource of the context (NULL is ignored). */
void ffa_destroy(ffa_ctx* ctx);

/* Message of the last failed call on ctx ("" if none).  With ctx NULL: the message
 * of the last failed ffa_create or ffa_energy_noalloc on the calling thread. */
const char* ffa_last_error(const ffa_ctx* ctx);

/* Replace the pinned positions b (n_pin x d, host or device).  The operator is
 * unchanged, so no refactorization happens; the next W step uses the new b. */
ffa_status ffa_set_handles(ffa_ctx* ctx, const double* pin_pos);

/* General linear constraints A W = b on the vertex positions, on top of the
 * pinned vertices (Sec. 4, W update: any feasible A W = b).  A is c x n in CSR
 * (row_ptr: c + 1 int64, col: int32 vertex indices, val: double), acting on every
 * coordinate column alike; b is c x d (row-major).  All arrays host or device,
 * copied.  Entries on pinned vertices move to the right-hand side (and follow
 * ffa_set_handles).  The W step stays the pinned one, L_FF W_F = G^T r - L_FC b_pins,
 * corrected by a Schur complement on the c rows: with Z = L_FF^-1 A_F^T (c
 * refined solves at this call) and S = A_F Z (c x c, Cholesky on the host), each
 * iteration projects W_F <- W_F - Z S^-1 (A_F W_F - b'), the exact constrained
 * minimizer.  Z is stored c x nF in double (8 c nF bytes on the device).  Call
 * after ffa_create (with at least one pinned vertex) and before ffa_init, once;
 * 1 <= c <= 256.  Not with penalty_schedule 1 nor with ffa_forward_unrolled.
 * Errors: FFA_ERR_INVALID_ARG (sizes, indices, non-finite values, c out of
 * range, after ffa_init or a second call, no pins, rows that are dependent once
 * the pinned vertices are eliminated: a Cholesky pivot of S below 1e-10 of its
 * diagonal), FFA_ERR_SINGULAR_SYSTEM (a column solve that does not converge),
 * FFA_ERR_TIMEOUT, FFA_ERR_CUDA, FFA_ERR_OOM.  A call that fails after the
 * column solves keeps their device scratch (8 c nF bytes) until ffa_destroy. */
ffa_status ffa_set_constraints(ffa_ctx* ctx, int32_t c, const int64_t* row_ptr, const int32_t* col,
                               const double* val, const double* b);

/* Start a solve from W0 (n x d, host or device): U0, P0 from the polar
 * decomposition of G W0 with singular values clamped to eps and the flipped case
 * of eq. polardecompositionapplied (eps = eps_m^(1/4) for SG, eps_m^(1/8) for SD, eps_m = 2^-52);
 * Lambda0 = 0 (Algorithm 2).  W0 is used as given, pinned rows included; the
 * pinned positions take effect from the first W step on. */
ffa_status ffa_init(ffa_ctx* ctx, const double* W0);

/* Run up to max_iter iterations of Algorithm 1 (W, U, P, Lambda steps; h_i per prox_h).
 * With stop_at_tol = 1 the termination test of eq. primaldualthresholds (plus flip-freeness when
 * require_flip_free) is evaluated every check_every iterations and the call
 * returns as soon as it passes; with stop_at_tol = 0 exactly max_iter iterations
 * run and the test is still evaluated at the last one.  *stats (may be NULL)
 * receives the last evaluated statistics.  Returns FFA_ERR_NAN if an evaluated
 * statistic is not finite; the state is then left as computed. */
ffa_status ffa_iterate(ffa_ctx* ctx, int32_t max_iter, int32_t stop_at_tol, ffa_stats* stats);

/* Copy the current W (n x d doubles) to W_out (host or device). */
ffa_status ffa_get_W(ffa_ctx* ctx, double* W_out);

/* Copy the per-element state out as doubles (m x d x d each, host or device;
 * any pointer may be NULL to skip it). */
ffa_status ffa_get_state(ffa_ctx* ctx, double* U, double* P, double* Lambda);

/* Make (W, U, P, Lambda) the current state, in place of ffa_init: the state of
 * Algorithm 1 between two iterations (W n x d, U, P, Lambda m x d x d each,
 * row-major, host or device, copied), e.g. from ffa_get_W and ffa_get_state of
 * an earlier run, to resume it or to restart from a checkpoint.  U must be a
 * rotation (U^T U = I and det U = 1 to 1e-5 per entry), P is symmetrized; the
 * free rows of W start the next W step, and r_i = mu_i (U_i P_i - Lambda_i) is
 * formed for it as the last local step would have.  The iteration counter
 * restarts at 0 and checkpoints of ffa_forward_unrolled are dropped.  On the
 * FP32 local step the state is rounded to float.  Not with penalty_schedule 1
 * (mu and the event counters are part of that state).
 * Errors: FFA_ERR_INVALID_ARG (NULL pointer, non-finite entry, U not a rotation,
 * penalty schedule), FFA_ERR_CUDA, FFA_ERR_OOM. */
ffa_status ffa_set_state(ffa_ctx* ctx, const double* W, const double* U, const double* P, const double* Lambda);

/* The current penalties mu_i (m values, host or device buffer): rho * w_i with
 * fixed penalties, the schedule's values with penalty_schedule 1 (eq.
 * augmentedlagrangian; Sec. 6, "Rescaling mu_i and Lambda").  With fixed
 * penalties and the FP32 local step they are read back from float. */
ffa_status ffa_get_penalties(ffa_ctx* ctx, double* mu);

/* Energy of eq. genericdeformationenergy at W (n x d, host or device; NULL = the current iterate):
 * sum_i w_i f((G W)_i), or +infinity (with FFA_OK) if some det (G W)_i <= 0. */
ffa_status ffa_energy(ffa_ctx* ctx, const double* W, double* E);

/* Gradient of the energy at W: dE/dW = G^T (w_i grad f((G W)_i)) with
 * grad f from eq. symmetricgradientdefininggrad / eq. symmetricdirichletdefininggrad, written to dEdW (n x d, host or device).
 * FFA_ERR_FLIPPED if some det (G W)_i <= 0 (the energy is infinite there). */
ffa_status ffa_gradient(ffa_ctx* ctx, const double* W, double* dEdW);

/* Sizes, setup timings and the algorithmic byte counts used for roofline reports. */
ffa_status ffa_get_info(ffa_ctx* ctx, ffa_info* info);

/* The current decomposition of L_FF (Algorithm 2, decompose(L)) as the W-step passes read it: for
 * every supernode s the float block B_s = [inv(L_ss); L_rs inv(L_ss)], column-major, zero above the
 * diagonal of inv(L_ss), concatenated with zero padding, factor_entries floats in all (ffa_info).
 * out (host or device, caller-owned) takes exactly count = factor_entries floats; another count is
 * FFA_ERR_INVALID_ARG.  A diagnostic for comparing where the decomposition ran (factor_device). */
ffa_status ffa_copy_factor(ffa_ctx* ctx, float* out, int64_t count);

/* Average device time of each phase of an iteration, measured with CUDA events
 * on the context stream over reps iterations launched eagerly (not as a graph).
 * The iterations are real: the state advances by reps iterations. */
ffa_status ffa_profile_phases(ffa_ctx* ctx, int32_t reps, ffa_phase_times* out);

/* Launch shapes picked by ffa_autotune (the paper has no counterpart). */
typedef struct {
  int32_t local_block;  /* threads per block of the local step: 64, 128 or 256 */
  int32_t narrow_cols;  /* supernodes with at most this many columns (and at most 1024 rows and
                           64 KB of factor) run as one task on one block: 32 or 64 */
  int32_t schedule;     /* supernodal solves: 0 per-level launches, 1 dynamic ready queue,
                           2 dynamic ready queue with the bulk-copy ring */
  int32_t bottom_levels;/* schedules 1, 2: lowest tree levels run as one launch per level: 0, 2, 3 or 4 */
  double ms_local[3];   /* measured local step for 64, 128, 256 threads */
  double ms_solve[2];   /* measured supernodal solve (forward + backward) for 32, 64 */
  double ms_schedule[3];/* measured supernodal solve for schedules 0, 1 and 2 */
  double ms_bottom[4];  /* measured supernodal solve (schedules 1, 2) for bottom_levels 0, 2, 3, 4 */
  int32_t subtree_height[2]; /* schedule 1 with bottom_levels 0: bottom subtrees of at most this
                           height run as one task, forward and backward pass: 0 (off) .. 3 */
  double ms_subtree[2][4];   /* measured forward / backward pass for heights 0 .. 3 */
} ffa_tuning;

/* Time the candidate launch shapes of the local step, of the supernodal solves and
 * their schedule
 * with CUDA events over reps launches each, keep the fastest, and restore the
 * iterate (needs ffa_init first; the state is saved and put back). */
ffa_status ffa_autotune(ffa_ctx* ctx, int32_t reps, ffa_tuning* out);

/* Differentiation through K unrolled iterations (the paper has no counterpart;
 * it is the adjoint of Algorithm 1's W, U, P and Lambda steps with h = 0).
 * ffa_forward_unrolled runs K iterations from the state set by ffa_init (no
 * termination test), storing the element state and W every ckpt_every
 * iterations.  ffa_backward_unrolled then takes dL/dW^K (n x d, host or device)
 * and writes dL/db (n_pin x d, host or device) for the pinned positions b: it
 * walks the checkpoint segments backwards, recomputes each segment's iterations,
 * applies the per-element vector-Jacobian products of the Lambda, P (matrix
 * function of S, divided differences of the scalar prox root) and U (polar
 * rotation) steps, and solves the W step's adjoint with the same factorized
 * L_FF (symmetric).  W^0 is taken as independent of b.  After the call the live
 * state is again the state after iteration K. */
ffa_status ffa_forward_unrolled(ffa_ctx* ctx, int32_t K, int32_t ckpt_every);
ffa_status ffa_backward_unrolled(ffa_ctx* ctx, const double* dL_dW, double* dL_db);

/* Relative residual |L_FF W_F - b_F| / |b_F| of the last W step, measured in
 * double on the device (a diagnostic of the refinement sweeps; eq. solvinginw).
 * FFA_ERR_INVALID_ARG on a context with general constraints, whose W step
 * leaves the multiplier term A_F^T nu in that residual. */
ffa_status ffa_last_wstep_residual(ffa_ctx* ctx, double* rel_residual);

/* Failure detection of the W step's device-side waits (the paper has no
 * counterpart: its back-substitution runs on one CPU thread).  With solve_schedule
 * 1 each block of a triangular pass polls its queue slot until a finished
 * supernode fills it; a wait that sees an empty slot for more than `polls` polls
 * (each about 100 ns; the default is 2^22, about 0.4 s) gives up, sets a device
 * flag that makes every other wait give up too, and the block exits.  The call
 * then returns FFA_ERR_TIMEOUT and the iterate is invalid; the context stays
 * usable (the next W step resets the queues), so a caller may restore the limit
 * and call ffa_init or ffa_set_state again.  polls = 0 gives up at the first
 * empty poll.  Takes effect from the next ffa_iterate (captured graphs are
 * dropped).  Errors: FFA_ERR_INVALID_ARG (NULL context, polls < 0). */
ffa_status ffa_set_wait_limit(ffa_ctx* ctx, int64_t polls);

/* Many independent meshes solved together (the paper solves one mesh at a time;
 * this batches its Algorithm 1 over independent problems).  Meshes of equal
 * (d, d_in) are concatenated into one block-diagonal problem: one factorization
 * per group, one set of launches per iteration for all meshes of the group,
 * element energy and penalty per mesh, and the termination test of
 * eq. primaldualthresholds evaluated per mesh.  All groups of a batch share one
 * stream and one CUDA graph per launch.
 *   meshes[k], pin_idx[k] / n_pin[k] / pin_pos[k] : as in ffa_create for mesh k
 *                   (n_pin[k] = 0 pins its vertex 0 at the origin); host or device.
 *   energies, rho : per mesh (NULL = params->energy / params->rho for all).
 *   params        : eps_abs, eps_rel, check_every, precision, sweeps, leaf size.
 * ffa_batch_iterate runs until every mesh passed its test (stop_at_tol = 1) or
 * max_iter iterations; stats[k] (may be NULL) receives mesh k's last statistics
 * and *n_converged (may be NULL) the number of meshes that passed.
 * ffa_batch_last_error(NULL) reports a failed ffa_batch_create. */
ffa_status ffa_batch_create(int32_t n_meshes, const ffa_mesh* meshes, const int32_t* const* pin_idx,
                            const int32_t* n_pin, const double* const* pin_pos, const ffa_energy_kind* energies,
                            const double* rho, const ffa_params* params, void* stream, ffa_batch** out);
void ffa_batch_destroy(ffa_batch* b);
const char* ffa_batch_last_error(const ffa_batch* b);
/* W0[k]: n_k x d initial map of mesh k (host or device), used as given. */
ffa_status ffa_batch_init(ffa_batch* b, const double* const* W0);
ffa_status ffa_batch_iterate(ffa_batch* b, int32_t max_iter, int32_t stop_at_tol, ffa_stats* stats,
                             int32_t* n_converged);
/* ffa_autotune for every group of the batch (one context per (d, d_in));
 * out (may be NULL) has ffa_batch_groups(b) entries. */
ffa_status ffa_batch_autotune(ffa_batch* b, int32_t reps, ffa_tuning* out);
int32_t ffa_batch_groups(const ffa_batch* b);
/* Copy mesh k's current W (n_k x d) to W_out (host or device). */
ffa_status ffa_batch_get_W(ffa_batch* b, int32_t mesh, double* W_out);

/* Energy of a map without a context and without allocating memory.
 *
 * The paper has no counterpart: this entry point exists for callers that cannot
 * call cudaMalloc -- code that runs under a custom or frozen device allocator,
 * inside a memory pool that must not grow, or in a process that only receives
 * device buffers from elsewhere -- and therefore cannot create a context.
 * It evaluates sum_i w_i f((G W)_i) (+infinity if some det (G W)_i <= 0) for the
 * mesh (V, T) and the map W directly, computing every element's frame, hat
 * gradients and Jacobian on the fly in double precision.
 *   n, m, d, d_in : sizes as in ffa_mesh; m may be at most 16,777,216
 *                   (larger m is rejected with FFA_ERR_INVALID_ARG).
 *   V, T, W       : device pointers (n x d_in doubles, m x (d+1) int32,
 *                   n x d doubles), read only.
 *   energy        : which defining function f (FFA_SYM_DIRICHLET or FFA_SYM_GRADIENT).
 *   E             : device pointer to one double, written by the call.
 *   stream        : cudaStream_t to run on (NULL = the legacy default stream).
 * The call only enqueues two kernels on the stream and returns; E is valid once
 * the stream has reached that point.  Because it never waits for its kernels, an
 * invalid mesh is reported in *E: an element with a vertex index outside [0, n)
 * (skipped before any load through that index) or a source element of zero
 * measure makes *E a NaN, whereas a valid mesh with some det (G W)_i <= 0 gives
 * +infinity (ffa_create refuses the same meshes with FFA_ERR_INVALID_ARG and
 * FFA_ERR_DEGENERATE_ELEMENT).  The per-block partial sums live in one fixed
 * static device array (1.5 MiB, held by every GPU that loads the library until the
 * process exits).  Every call looks up that array's device address on the current
 * device (cudaGetSymbolAddress); the first call on a device also loads the
 * library's device code there, so make the first call on a device before any
 * stream capture.  All calls share the array: each call overwrites the slots it
 * reads, so nothing has to be cleared, but calls that overlap on the GPU (other
 * streams, other host threads) race on it.
 * Errors: FFA_ERR_INVALID_ARG (sizes, NULL pointers, unknown energy),
 * FFA_ERR_CUDA (also when a CUDA error from earlier work is pending on the calling
 * thread; it is reported and left pending); the message is returned by
 * ffa_last_error(NULL). */
ffa_status ffa_energy_noalloc(int32_t n, int32_t m, int32_t d, int32_t d_in, const double* V,
                              const int32_t* T, const double* W, ffa_energy_kind energy, double* E,
                              void* stream);

#ifdef __cplusplus
}
#endif

#endif /* FFADMM_H */
