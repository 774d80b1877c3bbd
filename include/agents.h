/*
 * agents.h -- C ABI of the GB300 (sm_103a) agent-based optimal-control image solver.
 *
 * Method: O. Oliviero, S. Cacace, G. Visconti, "Agent-Based Optimal Control for Image
 * Processing" (arXiv 2510.16154).  Each pixel is an agent with a fixed position and an
 * evolving colour (Section 2, Eq. MAsystem, Eq. ellipsoid, Eq. kernel).  A spatially
 * uniform, time-dependent control eps(t) = (eps_x, eps_c) in a box E (Definition
 * control_space) steers the colours so that the final field minimises the regularised
 * total-variation cost L~ of Eq. complete_square; the control is optimised by ADMM
 * (Algorithm 2) whose eps-step is the direct-adjoint loop of Algorithm 1.
 *
 * Conventions shared by every call
 * --------------------------------
 *  - Colour fields are float32, row-major, channel-interleaved: [H][W][C].  Memory row
 *    k is the paper's k-th row counted from the bottom (Section 2), so the y component of
 *    the discrete gradient is (c[k+1] - c[k-1]) / (2 dy) with dy = 1/H, dx = 1/W
 *    (Definition discrete_gradient).  Pixel positions are (col dx, row dy) in [0,1]^2.
 *  - TV fields v (split variable) and mu (multiplier) are float32 [H][W][2][C]:
 *    component 0 along x (columns), component 1 along y (rows).
 *  - The control is float64 [T][2] = (eps_x^n, eps_c^n), piecewise constant on each of
 *    the T explicit Euler steps.
 *  - Field pointers ("_dev") are caller-owned DEVICE memory, 16-byte aligned, valid for
 *    the duration of the call; they are never retained.  Pointers documented as
 *    "host or device" may point to either; the library detects which.
 *  - All device work is issued on the stream given to agents_init.  A call whose outputs
 *    include host memory returns after those outputs are written (it synchronises the
 *    stream); a call whose outputs are all device memory may return before the work
 *    completes (stream-ordered).
 *  - Every call returns an int status: AGENTS_OK (0) or a negative error code.  On error
 *    the outputs are unspecified and agents_last_error(ctx) describes the failure.  A
 *    context is not thread-safe: one host thread at a time per context.
 */
#ifndef AGENTS_H_
#define AGENTS_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  AGENTS_OK = 0,
  AGENTS_EINVAL = -1,     /* bad argument, shape, alignment or null pointer          */
  AGENTS_ECUDA = -2,      /* a CUDA runtime call or kernel launch failed               */
  AGENTS_ENOMEM = -3,     /* device allocation failed                                  */
  AGENTS_ETIMEOUT = -4,   /* a bounded device-side wait gave up                        */
  AGENTS_EDIVERGED = -5,  /* NaN/Inf in the objective or residuals                     */
  AGENTS_ESTATE = -6      /* call order violated (e.g. adjoint without a stored forward) */
};

/* Problem constants.  agents_default_params fills the paper's values: dt = 0.25
 * (Section 3.2), E = [2, 1100]^2 (Section 3.2), rho = gamma = 1e-2 (Section 4.2),
 * alpha = 3000 (the fidelity weight of the ADMM comparison runs, Section 4.2). */
typedef struct {
  int32_t height, width, channels; /* H = N_R, W = N_C, C >= 1                              */
  int32_t radius;                  /* R >= 1: agent i interacts with in-image agents j != i
                                      with |row_j - row_i| <= R and |col_j - col_i| <= R     */
  int32_t nsteps;                  /* T >= 1 explicit Euler steps                           */
  double dt;                       /* Euler step, > 0                                       */
  double alpha, rho, gamma;        /* fidelity weight, penalty, dual step; all > 0           */
  double eps_lo[2], eps_hi[2];     /* the box E: eps_lo[k] <= eps_hi[k], eps_lo[k] >= 0      */
  int32_t norm_mode;               /* 0: weight 1/M, M = (2R+1)^2;  1: weight 1/N (Eq. MAsystem) */
  int32_t tv_mode;                 /* 0: |v_i| = Frobenius norm of the 2xC block (coupled);
                                      1: sum over channels of the 2-vector norms             */
  int32_t traj_mode;               /* 0: store all T+1 states for the adjoint; k > 0: store
                                      every k-th state and recompute the rest (checkpoints) */
} agents_params;

/* Fill *p with the defaults above for an H x W x C image, window radius R, T steps. */
void agents_default_params(agents_params* p, int32_t height, int32_t width, int32_t channels,
                           int32_t radius, int32_t nsteps);

typedef struct agents_ctx agents_ctx; /* opaque; owns its device workspaces and trajectory */

/* Create a context for one image.  c0 (host or device, [H][W][C]) is the input image
 * c^0 of Eq. MAsystem; it is copied into context-owned device memory.  cuda_stream is a
 * cudaStream_t (NULL = the legacy default stream).  Validates p (see agents_params);
 * returns AGENTS_EINVAL on a bad value, AGENTS_ENOMEM if the workspaces do not fit. */
int agents_init(const agents_params* p, const float* c0, void* cuda_stream, agents_ctx** out);

/* Replace the context's input image c^0 (host or device, [H][W][C]); same shape. */
int agents_set_image(agents_ctx* ctx, const float* c0);

/* Release every device buffer of the context.  NULL is accepted. */
int agents_destroy(agents_ctx* ctx);

/* Process-wide cap, in bytes, on the device memory that this library's contexts hold
 * (their workspaces, trajectories and solve buffers, across every context and device of
 * the process); 0 removes the cap, which is the default.  The paper has no counterpart:
 * this lets a service bound what the solver may take from a shared GPU.  An allocation
 * that would take the total above the cap fails as a failed cudaMalloc does:
 * agents_init (or the first solve, dal_solve or agents_solve_batch on a context, which
 * allocate the solve buffers) returns AGENTS_ENOMEM and agents_last_error names the
 * limit; the optional trajectory-reuse buffers of solve() are skipped instead (solve
 * then recomputes, with bitwise the same results).  Memory already held is not released
 * by lowering the cap.  Always returns AGENTS_OK. */
int agents_set_memory_limit(uint64_t bytes);

/* Device memory, in bytes, currently held by all contexts of the process. */
uint64_t agents_memory_held(void);

/* Test hook (no counterpart in the paper): bound every loop of the label union-find of
 * agents_labels and solve() at `cap` iterations instead of the pixel count (0 restores
 * the default; cap < 0 returns AGENTS_EINVAL).  With a bound below the tree depth the
 * loops give up -- they exit, nothing hangs or reads out of bounds -- and the call
 * returns AGENTS_ETIMEOUT, the status of a device-side wait that gave up.  Process-wide;
 * not for production use. */
int agents_debug_set_label_loop_cap(int32_t cap);

/* Test hook (no counterpart in the paper) for the whole-sweep launches.  For the tiled
 * (R, C) a sweep of agents_forward, agents_adjoint*, agents_flow_backward, dal_solve or
 * solve can run all its Euler (or adjoint) steps in one persistent launch: blocks take
 * (step, tile) jobs in order and wait, each wait bounded by a time limit, until the
 * 3 x 3 tiles around theirs have finished the previous step.  Results are bitwise those
 * of one launch per step.
 *   enable     0: one launch per step; 1 (the default): whole-sweep launches where they
 *              measured faster (adjoint sweeps of images with at most 4 tiles per
 *              resident block); 2: whole-sweep launches for every tiled sweep; other
 *              values return AGENTS_EINVAL.
 *   wait_ns    time limit of one wait in nanoseconds; 0 restores the default (2 s);
 *              < 0 returns AGENTS_EINVAL.
 *   skew_once  nonzero: the next whole-sweep launch waits for flag values that no tile
 *              ever writes, so its first wait runs out of time; the launch then winds
 *              down (no fault, no hang), and the API call that reads its status returns
 *              AGENTS_ETIMEOUT and re-arms the context's flags for the calls after it.
 * The status is read whenever a call copies a result to the host; a call whose outputs
 * are all device memory (agents_flow_backward without grad_eps_out) leaves it to the next
 * call on the context that does.  Process-wide; not for production use. */
int agents_debug_set_fused(int32_t enable, int64_t wait_ns, uint32_t skew_once);

/* Message of the last failure on ctx (or of the last failed agents_init when ctx is
 * NULL).  The string is owned by the library and valid until the next call. */
const char* agents_last_error(const agents_ctx* ctx);

/* Forward sweep (Eq. opt_system-a, explicit Euler, Section 3.2):
 *   c^{n+1}_i = c^n_i + dt/M sum_{j in W(i)} phi(r_ij)(c^n_j - c^n_i),
 *   r_ij = eps_x^n/2 |x_j - x_i|^2 + eps_c^n/2 |c^n_j - c^n_i|^2,
 *   phi(r) = (1 - r)^4 (4r + 1) on [0,1], 0 beyond (the C2 Wendland kernel of Eq. kernel).
 * eps: host or device [T][2] float64, entries finite and >= 0 (the semi-axes of the
 * ellipsoid; AGENTS_EINVAL otherwise).  cT_dev: device [H][W][C] output c^T (may be NULL).
 * store != 0 keeps the trajectory (or its checkpoints) for a following agents_adjoint. */
int agents_forward(agents_ctx* ctx, const double* eps, float* cT_dev, int store);

/* Reverse sweep: the exact discrete adjoint of the forward sweep (Eq. opt_system-b,
 * Section 3.1) for the terminal cost L~(c^T, v, mu) of Eq. complete_square.
 *   lambda^T = -dL~/dc(c^T) = -dx dy [G^T(rho G c^T - rho v - mu) + alpha (c^T - c^0)]
 *     (Eq. admm_terminal with the exact transpose G^T of the discrete gradient G),
 *   lambda^n = lambda^{n+1} + dt (dF/dc(c^n, eps^n))^T lambda^{n+1},
 *   D^n = sum_i lambda^{n+1}_i . dF_i/deps(c^n, eps^n)   (Algorithm 1, so that
 *     dL~/deps^n = -dt D^n).
 * Requires a preceding agents_forward(store != 0) with the same eps (else AGENTS_ESTATE).
 * eps: host or device [T][2]; v_dev, mu_dev: device [H][W][2][C]; D_out: host or device
 * [T][2] float64; obj_out: host or device, one float64 = L~(c^T, v, mu) (may be NULL);
 * lambda0_dev: device [H][W][C] output lambda^0 (may be NULL). */
int agents_adjoint(agents_ctx* ctx, const double* eps, const float* v_dev, const float* mu_dev,
                   double* D_out, double* obj_out, float* lambda0_dev);

/* Reverse sweep from a caller-given terminal adjoint, for any terminal cost L(c^T):
 * with lambdaT_dev = -dL/dc^T (device [H][W][C]) it returns D^n with
 * dL/deps^n = -dt D^n (D_out, host or device [T][2] float64) and lambda^0 = -dL/dc^0
 * (lambda0_dev, device [H][W][C], may be NULL) -- the exact discrete adjoint of the
 * forward sweep (Eq. opt_system-b, Section 3.1).  Requires a preceding
 * agents_forward(store != 0) with the same eps (else AGENTS_ESTATE); works with full
 * storage or checkpoints (traj_mode).  This is the backward pass of a differentiable
 * forward sweep. */
int agents_adjoint_from(agents_ctx* ctx, const double* eps, const float* lambdaT_dev,
                        double* D_out, float* lambda0_dev);

/* Backward pass of the differentiable forward sweep c^T = c(T; eps, c^0) for any
 * terminal cost L(c^T): given the upstream gradient grad_cT_dev = dL/dc^T (device
 * [H][W][C]) it runs the exact discrete adjoint (Eq. opt_system-b, Section 3.1) from
 * lambda^T = -dL/dc^T and writes grad_eps_out = dL/deps^n = -dt D^n (host or device
 * [T][2] float64, may be NULL) and grad_c0_dev = dL/dc^0 = -lambda^0 (device [H][W][C],
 * may be NULL).  The sign changes and the dt scaling run on the device.  Requires a
 * preceding agents_forward(store != 0) with the same eps (else AGENTS_ESTATE); full
 * storage or checkpoints (traj_mode). */
int agents_flow_backward(agents_ctx* ctx, const double* eps, const float* grad_cT_dev,
                         double* grad_eps_out, float* grad_c0_dev);

/* Terminal cost and adjoint only: obj_out (host or device) = L~(c, v, mu) of
 * Eq. complete_square; lambda_dev (device, may be NULL) = -dL~/dc (Eq. admm_terminal,
 * exact-transpose form).  c_dev: device [H][W][C]. */
int agents_objective(agents_ctx* ctx, const float* c_dev, const float* v_dev,
                     const float* mu_dev, double* obj_out, float* lambda_dev);

/* Primal TV step, the v-minimisation of Algorithm 2 (Eq. soft_threshold):
 *   a_i = (G c)_i - mu_i / rho,  v_i = max(|a_i| - 1/rho, 0) a_i / |a_i|   (v_i = 0 if a_i = 0),
 * with G the central-difference gradient with reflective boundaries (Definition
 * discrete_gradient, Eq. reflective_boundary) and |.| as selected by tv_mode; this is
 * a_i minus its projection onto the dual ball of radius 1/rho.
 * c_dev: device [H][W][C]; mu_dev, v_dev: device [H][W][2][C]. */
int pd_tv_step(agents_ctx* ctx, const float* c_dev, const float* mu_dev, float* v_dev);

/* Multiplier update, the mu-maximisation of Algorithm 2 (Eq. dual_ascent), in float64
 * arithmetic:  mu_i <- mu_i + gamma (v_i - (G c)_i).
 * stats (host or device, 5 float64, may be NULL), reductions in float64:
 *   [0] r   = |v - G c|_2                       (primal residual)
 *   [1] s   = rho |G^T (v - v_prev)|_2          (dual residual; 0 if v_prev is NULL)
 *   [2] gap = gamma dx dy |v - G c|^2           (increase of L across this mu-step, exact
 *                                                because L is linear in mu, Section 4.1)
 *   [3] rel = |c - c_prev|_2 / |c|_2            (0 if c_prev is NULL)
 *   [4] K(c) of Eq. cost_TV.
 * c_dev, c_prev_dev: device [H][W][C]; v_dev, v_prev_dev, mu_dev: device [H][W][2][C]. */
int alm_update(agents_ctx* ctx, const float* c_dev, const float* c_prev_dev, const float* v_dev,
               const float* v_prev_dev, float* mu_dev, double* stats);

/* Cluster labels of a colour field: connected components of the 4-neighbour graph in
 * which neighbours are joined when every channel differs by at most `threshold` (the
 * paper segments with threshold 0.02, Section 5), decided in float32.  Each label is the
 * smallest row-major index in its component.  labels_out: host or device [H][W] int32;
 * count_out: host, number of components (may be NULL). */
int agents_labels(agents_ctx* ctx, const float* c_dev, float threshold, int32_t* labels_out,
                  int32_t* count_out);

/* Options of solve().  Defaults (agents_default_solve_opts): sigma0 = 1, b = 1/2,
 * c = 1e-4 (Section 3.2); max_ls = 30 Armijo trials; tol = 0 (run all k_out steps). */
typedef struct {
  int32_t k_out;    /* multiplier (outer ADMM) steps                                  */
  int32_t k_in;     /* DAL iterations per eps-step                                     */
  int32_t max_ls;   /* Armijo trials per DAL iteration                                 */
  double sigma0;    /* first Armijo step                                               */
  double ls_b;      /* Armijo factor b in (0,1)                                        */
  double ls_c;      /* Armijo constant c in (0,1)                                      */
  double tol;       /* stop when max(|c^j-c^{j-1}|/|c^j|, |L~_j-L~_{j-1}|/|L~_{j-1}|) < tol */
} agents_solve_opts;

typedef struct {
  int32_t outer_done;      /* multiplier steps run                                      */
  int32_t inner_done;      /* DAL iterations run in total                               */
  int32_t trials;          /* Armijo trials (forward sweeps without store) in total     */
  int32_t stalls;          /* DAL iterations that found no admissible step              */
  int32_t stationary;      /* eps-steps ended because no component of D could move
                              (the variational inequality of the Remark on convergence
                              criteria holds)                                           */
  int64_t forward_steps;   /* explicit Euler steps executed (all sweeps)                */
  int64_t adjoint_steps;   /* adjoint steps executed                                    */
  int64_t tv_sweeps;       /* pd_tv_step + alm_update + objective sweeps executed       */
  double final_res;        /* res of the last multiplier step                           */
  double final_obj;        /* L~(c, v, mu) after the last multiplier step               */
  double final_gap;        /* gamma dx dy |v - G c|^2 of the last multiplier step       */
  double final_sigma;      /* Armijo step carried to the next DAL iteration (pass it as
                              sigma0 to continue a solve across calls)                  */
  int64_t kernel_launches; /* CUDA kernels this call launched                           */
} agents_solve_info;

void agents_default_solve_opts(agents_solve_opts* o);

/* Algorithm 2 (with Algorithm 1 inside, exactly as solve()) for n images at once, each in
 * its own context (any mix of sizes, channel counts and window radii; all with the same
 * nsteps, traj_mode 0, on one device).  Every Euler / adjoint step of all images is one
 * persistent launch per (radius, channels) class over a job list of (image, tile) pairs;
 * the Armijo searches run as per-image state machines on the device, so the launch
 * sequences of a DAL sweep and of an Armijo round are replayed as CUDA graphs
 * (use_graph != 0) with one host synchronisation per round for the whole batch.  Images
 * that reach opts->tol stop while the others continue.  autotune != 0 picks the tile shape
 * of each class by timing (cached per process); with autotune = 0 every image's result is
 * bitwise that of solve().  eps_io[i], mu_io[i] (host or device) as in solve(); c_out[i]
 * (host or device, may be NULL, or c_out itself NULL); infos: host array of n records
 * (may be NULL; kernel_launches is -1, launches being shared by the batch; forward_steps
 * counts every recomputed sweep).  Work is ordered after the first context's stream; the
 * call returns when it is done.  Returns AGENTS_EINVAL for n < 1, NULL contexts or
 * buffers, invalid opts, mixed nsteps or devices, or a checkpointed context;
 * AGENTS_EDIVERGED when an image's objective became NaN/Inf (that image stops, the others
 * finish and every output is written); AGENTS_ECUDA / AGENTS_ENOMEM with the message in
 * agents_last_error(ctxs[0]).  The paper solves one image at a time; this is its solve
 * applied to many images in one pass. */
int agents_solve_batch(int32_t n, agents_ctx* const* ctxs, const agents_solve_opts* opts,
                       int32_t autotune, int32_t use_graph, double* const* eps_io,
                       float* const* mu_io, float* const* c_out, agents_solve_info* infos);

/* One record per DAL iteration of the last solve() on a context. */
typedef struct {
  int32_t outer;    /* multiplier step j (1-based)                                       */
  int32_t trials;   /* Armijo trials                                                      */
  int32_t status;   /* 0: step accepted; 1: no admissible step (stall); 2: stationary     */
  int32_t reserved;
  double L0;        /* L~ at the current control                                          */
  double L;         /* L~ at the accepted control (L0 if none)                            */
  double gnorm2;    /* dt sum_n |P D^n|^2 over the components the box does not block      */
  double tau;       /* accepted step (0 if none)                                          */
} agents_iter_record;

/* Copy up to `capacity` records of the last solve() into out (host); *count receives the
 * number of records available.  out may be NULL to query the count. */
int agents_solve_log(const agents_ctx* ctx, agents_iter_record* out, int32_t capacity,
                     int32_t* count);

/* One record per multiplier step of the last solve() on a context: the Section 4.1
 * quantities the stopping test and the convergence plots use. */
typedef struct {
  int32_t outer;       /* multiplier step j (1-based)                                     */
  int32_t inner_done;  /* DAL iterations of this step's eps-step                          */
  double L;            /* L~(c^j, v^j, mu^j)                                              */
  double K;            /* K(c^j) = dx dy sum_i [|(G c^j)_i| + alpha/2 |c^j_i - c0_i|^2]   */
  double r;            /* |v^j - G c^j|                                                   */
  double s;            /* rho |G^T (v^j - v^{j-1})|                                       */
  double gap;          /* gamma dx dy |v^j - G c^j|^2                                     */
  double rel_dc;       /* |c^j - c^{j-1}| / |c^j|                                         */
  double res;          /* max(rel_dc, |L~_j - L~_{j-1}| / |L~_{j-1}|)                     */
  double sigma;        /* Armijo step carried into the next DAL iteration                 */
} agents_outer_record;

/* Copy up to `capacity` multiplier-step records of the last solve() into out (host);
 * *count receives the number available; out may be NULL to query the count. */
int agents_solve_outer_log(const agents_ctx* ctx, agents_outer_record* out, int32_t capacity,
                           int32_t* count);

/* Algorithm 1 on its own (Section 3): the direct-adjoint loop with projected two-way
 * Armijo search on the terminal cost L~(c(T), 0, 0) = dx dy sum_i [rho/2 |G c_i|^2 +
 * alpha/2 |c_i - c0_i|^2], which is J of Eq. cost_functional when the context was created
 * with rho = 1.  Runs at most opts->k_in iterations and stops early when the relative
 * change of the cost in an iteration is below opts->tol (the stationarity criterion of
 * the Remark on convergence criteria; tol = 0 disables it) or when the control is
 * stationary or no step is admissible.  opts->k_out is ignored.  eps_io: host or device
 * [T][2], in/out; c_out: host or device [H][W][C] = c(T; eps*) (may be NULL).
 * info->final_obj is the cost after the last accepted step. */
int dal_solve(agents_ctx* ctx, const agents_solve_opts* opts, double* eps_io, float* c_out,
              agents_solve_info* info);

/* Algorithm 2 (ADMM) with Algorithm 1 (DAL + projected two-way Armijo) as the eps-step.
 * The Armijo test is L~(Pi_E(eps + tau D)) < L~(eps) and
 * L~(Pi_E(eps + tau D)) <= L~(eps) - c tau |P D|^2, |P D|^2 = dt sum_n |P D^n|^2, where
 * P D zeroes the components of D that push a control already on a bound of E outward;
 * an eps-step ends when no component is free (stationary) or no trial passes (stall).
 *   c^(0) = c(T; eps^(0)),  v^(0) = argmin_v L(c^(0), v, mu^(0));
 *   for j = 1..k_out: k_in DAL iterations on L~(c(T; eps), v^(j-1), mu^(j-1));
 *     c^(j) = c(T; eps^(j));  v^(j) = shrink(G c^(j) - mu^(j-1)/rho);
 *     mu^(j) = mu^(j-1) + gamma (v^(j) - G c^(j)).
 * eps_io: host or device [T][2] float64, the initial control in (eps^(0); fill with 57
 * for the paper's start, Section 3.2) and the optimised control out.
 * mu_io: host or device [H][W][2][C], mu^(0) in (zeros for a cold start), mu out.
 * v_out, c_out: host or device outputs [H][W][2][C] and [H][W][C] (may be NULL).
 * labels_out: host or device [H][W] int32 cluster labels of c (threshold 0.02; may be NULL).
 * info: host (may be NULL).  Returns AGENTS_EDIVERGED if an objective or residual
 * becomes NaN/Inf; the outputs then hold the last finite iterate. */
int solve(agents_ctx* ctx, const agents_solve_opts* opts, double* eps_io, float* mu_io,
          float* v_out, float* c_out, int32_t* labels_out, agents_solve_info* info);

/* Objective and terminal adjoint for callers that cannot allocate device memory.
 * The paper has no counterpart: this is a variant of agents_objective for hosts that own
 * all device memory (they reserve their budget up front and hand out only pre-allocated
 * buffers) or that must not call cudaMalloc on a latency-critical path, because it can
 * synchronise the whole device.  It needs no context: every input and output comes from
 * the caller, and its only scratch, the float64 per-block partial sums of the reduction,
 * lives in a 256 KiB static device array that every GPU loading the library holds until
 * the process exits.  It calls no cudaMalloc, cudaFree or allocating library routine.
 *   obj_dev (device, one float64) = the same objective value agents_objective returns:
 *     the complete-square penalty of v - G c + mu/rho, plus the TV norm of v, plus the
 *     fidelity term alpha/2 |c - c0|^2, summed over pixels and scaled by dx dy;
 *   lambda_dev (device [H][W][C], may be NULL) = minus its derivative in c, the terminal
 *     adjoint agents_objective writes;
 *   c_dev, c0_dev: device [H][W][C]; v_dev, mu_dev: device [H][W][2][C]; every field is
 *     device memory, 16-byte aligned, and holds at least that many floats (the library
 *     cannot check sizes: a short buffer is read out of bounds);
 *   alpha, rho > 0; tv_mode as in agents_params; cuda_stream as in agents_init.
 * Limit: ceil(W / 128) * ceil(H / 8) <= 32768 reduction blocks (each block covers
 * 128 x 8 pixels), e.g. 4096 x 8192; the pixel count 33,554,432 is reached only when W
 * is a multiple of 128 and H a multiple of 8, and narrow images reach the block limit at
 * fewer pixels.  Larger images, host pointers and other bad arguments return
 * AGENTS_EINVAL with a message in agents_last_error(NULL).
 * Set-up: the first call on each device (with that device current) loads the library's
 * device code there, which allocates the static array and can synchronise the device;
 * make that first call during set-up, before any stream capture.  Every call looks up the
 * array's address in the current device context (no address is cached across calls, so
 * a device reset or another context of the same device is handled).
 * All calls share the array, so calls whose work overlaps on the GPU (different streams,
 * no ordering between them) race and must not be issued; calls on one stream are ordered
 * and safe.  Nothing in the array needs clearing between calls: each call writes every
 * partial it reads.  Returns after queueing the work (stream-ordered). */
int agents_objective_noalloc(int32_t height, int32_t width, int32_t channels, double alpha,
                             double rho, int32_t tv_mode, const float* c_dev,
                             const float* c0_dev, const float* v_dev, const float* mu_dev,
                             double* obj_dev, float* lambda_dev, void* cuda_stream);

/* Measurement utility (no counterpart in the paper): launch one kernel of independent
 * float32 FMA chains on cuda_stream -- scalar FFMA (packed = 0) or packed FFMA2 on float2
 * (packed != 0) -- with `blocks` blocks of 256 threads, each thread doing `iters`
 * iterations of 16 FMAs, no memory traffic.  *flops_out (host) receives the flop count
 * of the launch (an FMA counts 2).  Timed with events on that stream, it gives the
 * measured FP32 rate that the agent sweeps' roofline fractions are taken against.
 * sink_dev: device memory of blocks * 256 floats (written only in a case that never
 * occurs; it keeps the chains live).  AGENTS_EINVAL on a bad argument, AGENTS_ECUDA if
 * the launch fails. */
int agents_fp32_probe(int32_t packed, int32_t blocks, int32_t iters, float* sink_dev,
                      void* cuda_stream, double* flops_out);

#ifdef __cplusplus
}
#endif

#endif /* AGENTS_H_ */
