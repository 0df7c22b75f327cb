/*
 * dmpc.h - C-ABI of the GB300 DiffMPC hot path: batched, differentiable solves of
 *
 *   OCP:  argmin_{z=(x,u)} sum_{t=0}^{T} c_t^x(x_t) + sum_{t=0}^{T-1} c_t^u(u_t)
 *         s.t. f_t(x_{t+1}, x_t, u_t) = 0,  x_0 = x_s          (paper Sec. 1 and Sec. 3)
 *
 * by SQP (Algorithm 2) whose QPs are solved with the Schur complement S (Eq. 8-10) and
 * preconditioned conjugate gradient (Algorithm 4), and gradients by the implicit function
 * theorem (Eq. 3, Eq. 7, Algorithm 3).  All compute runs in CUDA kernels for sm_103a.
 *
 * Conventions
 *  - Pointers passed to dmpc_solve / dmpc_vjp / dmpc_qp_inspect are DEVICE pointers
 *    (cudaMalloc'd or torch CUDA tensors) owned by the caller, float32, OCPs packed one
 *    after another at the element offsets returned by dmpc_layout().  The library owns only
 *    its workspace and the warm-start buffers kept on the device between calls.
 *  - Per OCP with K = T+1 knots, n = K nx + T nu, m = K nx:
 *      z      (n)  = (x_0, u_0, x_1, u_1, ..., x_{T-1}, u_{T-1}, x_T)        (Sec. 3.1)
 *      lambda (m)  = (lambda_0, ..., lambda_T); lambda_0 multiplies x_0 - x_s = 0,
 *                    lambda_{t+1} multiplies f_t = 0; Lagrangian c + lambda^T g (Eq. 1)
 *      x_s    (nx), x_ref (K nx) (reference states; NULL means zero)
 *      theta  (p)  = [model params (p_s) | T x per-knot params (p_k) | diag Q (nx) |
 *                     diag R (nu) | diag Q_T (nx)],  p = p_s + T p_k + 2 nx + nu
 *    Costs: c_t^x(x) = 1/2 (x - x_ref,t)^T diag(Q) (x - x_ref,t)  (diag(Q_T) at t = T),
 *           c_t^u(u) = 1/2 u^T diag(R) u.
 *  - Models (f_t = x_{t+1} - Phi_t(x_t, u_t), Phi one RK4 / Euler step, or affine):
 *      LQ           nx, nu in {(2,1),(3,2),(4,1),(8,4),(16,8)} ((16,8): 32-thread teams or the cluster
 *                   form); p_s = 0; per knot
 *                   p_k = nx*nx + nx*nu + nx: Abar_t (row-major), Bbar_t, c_t
 *      PENDULUM     nx 2, nu 1, params (m, L)                 RK4
 *      CARTPOLE     nx 4, nu 1, params (m_pole, L), m_cart 1  RK4
 *      KIN_BICYCLE  nx 4, nu 2, params (wheelbase)            RK4
 *      SINGLE_TRACK nx 6, nu 2, params (mu, C_alpha)          RK4 (Fiala tyres)
 *      RIGID_BODY12 nx 12, nu 4, params (m, Jx, Jy, Jz)       RK4
 *      ATTITUDE     nx 3, nu 3, params (J1, J2, J3)           forward Euler
 *      SINGLE_TRACK_RATE  nx 8, nu 2, params (mu, C_alpha): the vehicle with control-rate
 *                   augmentation (App. B.3): state (x, delta, F_x), input their rates;
 *                   x_{t+1} = Phi_t(x_t, (delta_t, F_x,t)) by RK4, (delta, F_x)_{t+1} =
 *                   (delta, F_x)_t + dt u_t, so diag R weighs the control rates; not mixed
 *                   with other models in one batch
 *  - Calls are asynchronous on the handle's CUDA stream and return a dmpc_err for argument
 *    and launch errors.  Numerical outcomes are per OCP in status_out (bit flags below); a
 *    failed OCP never aborts the batch and the device never traps.
 *  - Thread safety: a handle must not be used by two host threads at once.  Calls on one
 *    handle are ordered by its stream.
 */
#ifndef DMPC_H
#define DMPC_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dmpc_handle dmpc_handle;

typedef enum {
  DMPC_OK = 0,
  DMPC_E_ARG = 1,          /* invalid argument (null pointer, bad size, unknown model) */
  DMPC_E_OOM = 2,          /* device allocation failed */
  DMPC_E_BUDGET = 3,       /* request exceeds a memory budget */
  DMPC_E_CUDA = 4,         /* a CUDA call failed; see dmpc_last_error */
  DMPC_E_STATE = 5,        /* call out of order (e.g. vjp before any solve) */
  DMPC_E_UNSUPPORTED = 6   /* model / size combination not compiled in */
} dmpc_err;

/* per-OCP status bits (status_out) */
#define DMPC_S_OK 0
#define DMPC_S_PCG_MAXITER 1     /* a PCG solve hit pcg_max_iters before the tolerance */
#define DMPC_S_NONFINITE 2       /* a non-finite value appeared in z, lambda or PCG scalars */
#define DMPC_S_LS_MINSTEP 4      /* no step size passed the decrease test: smallest alpha taken */
#define DMPC_S_BAD_INPUT 8       /* non-finite cost weight or model parameter */
#define DMPC_S_PCG_BREAKDOWN 16  /* p^T S p <= 0 in PCG (S not positive definite numerically) */
#define DMPC_S_CHOL_FAIL 32      /* a diagonal Schur block failed Cholesky (diagonal fallback used) */
#define DMPC_S_FP64_RESCUE 64    /* informational: a PCG solve whose FP32 iteration stagnated or broke
                                    down was finished in extended precision (FP64 or double-float) */
#define DMPC_S_HESS_INDEF 128    /* exact-Hessian vjp: the exact reduced Hessian was not positive definite
                                    at some knot (a Riccati pivot block failed Cholesky), so this OCP's
                                    gradient is the Gauss-Newton one instead */
#define DMPC_S_SYNC_TIMEOUT 256  /* cluster form: a wait on another CTA of the OCP's thread-block cluster ran
                                    out of time (4 s); the results of this OCP are not valid */

typedef enum {
  DMPC_MODEL_LQ = 0,
  DMPC_MODEL_PENDULUM = 1,
  DMPC_MODEL_CARTPOLE = 2,
  DMPC_MODEL_KIN_BICYCLE = 3,
  DMPC_MODEL_SINGLE_TRACK = 4,
  DMPC_MODEL_RIGID_BODY12 = 5,
  DMPC_MODEL_ATTITUDE = 6,
  DMPC_MODEL_SINGLE_TRACK_RATE = 7  /* SINGLE_TRACK with control-rate augmentation (App. B.3) */
} dmpc_model;

/* Integrator of a continuous model (dmpc_ocp_desc.integrator). */
typedef enum {
  DMPC_INTEGRATOR_DEFAULT = 0,   /* the model's explicit step (RK4; Euler for attitude; affine LQ) */
  DMPC_INTEGRATOR_TRAPEZOID = 1  /* implicit trapezoidal rule f_t = x_{t+1} - x_t - dt/2 (F(x_t, u_t)
                                    + F(x_{t+1}, u_t)), so A^+ = I - dt/2 dF/dx (Eq. 4, 10);
                                    pendulum and cart-pole; not with exact_hessian */
} dmpc_integrator;

/* One OCP of a batch (the OCP statement of Sec. 3): model, sizes, horizon, step. */
typedef struct {
  int model;      /* dmpc_model */
  int nx, nu;     /* state / input dimension (must match the model) */
  int T;          /* horizon, 1 <= T <= 4096 */
  float dt;       /* integrator step (ignored by LQ) */
  int integrator; /* dmpc_integrator; 0 = the model's own */
} dmpc_ocp_desc;

/* Solver options.  dmpc_default_options() fills the defaults noted here. */
typedef struct {
  int sqp_iters;       /* SQP iterations per solve (Algorithm 2); default 1 */
  int line_search;     /* 1: line search of Algorithm 5; 0: full steps (alpha = 1); default 0 */
  int n_alpha;         /* number of candidate step sizes, <= 8; default 5 */
  float alpha[8];      /* candidates in decreasing order; default {1, 0.7, 0.3, 0.1, 0.01} */
  float ls_eta;        /* decrease-test constant eta of Eq. 14; default 0.4 */
  float feas_tol;      /* ||g||_1 <= feas_tol (m + ||x||_1) counts as feasible (penalty 0); 1e-5 */
  float pcg_tol;       /* PCG stops when sqrt(r^T Phi^-1 r / gamma^T Phi^-1 gamma) <= pcg_tol; 1e-9 */
  int pcg_max_iters;   /* PCG iteration cap per solve; default 1000 */
  float ru_delta;      /* reliable-update trigger (FP64 true residual when eta drops by delta^2); 0.1 */
  int warm_start;      /* 1: with z_init == NULL, start from this handle's previous solution and
                          multipliers, and warm-start the adjoint PCG from the previous one; default 1 */
  int store_schur;     /* 1: solve keeps the blocks at the returned z for vjp; 0: vjp recomputes; default 0 */
  int team_threads;    /* threads per OCP: 32, 64, 128 or 256; 0 = chosen from the horizon */
  int teams_per_block; /* OCPs per thread block; 0 = chosen from batch size and shared memory */
  int pcg_precision;   /* 0: FP32 PCG iteration with FP64 reliable updates and a double-float rescue
                          when it stagnates; 1: double-float PCG iteration throughout (about 48-bit
                          arithmetic from FP32 instructions; single-warp teams with nx <= 4, the
                          others behave as 0); default 0 */
  int exact_hessian;   /* 1: dmpc_vjp uses the exact Hessian of the Lagrangian in the KKT matrix (the
                          dynamics curvature weighted by the forward multipliers, Sec. 3.4), so the
                          gradient is exact for nonlinear dynamics (an OCP whose exact reduced Hessian
                          is not positive definite gets the Gauss-Newton gradient and status bit
                          DMPC_S_HESS_INDEF); 0: Gauss-Newton (the paper's default); enlarges the
                          workspace by (nx+nu)^2 doubles per knot; default 0 */
  int pcg_variant;     /* 0: Algorithm 4 as printed (two dependent reductions per iteration); 1: the same
                          iteration reorganised after Chronopoulos and Gear (one fused reduction of r^T u
                          and (S u)^T u per iteration, S p by recurrence; equal in exact arithmetic);
                          single-warp teams (nx <= 4, K <= 64), the others behave as 0; default 0 */
  int cluster_ctas;    /* OCPs whose workspace does not fit in one thread block's shared memory (12-state
                          rigid body) and OCPs with nx >= 16 (LQ nx 16): 0 = run each on a thread-block
                          cluster when one fits (its Schur
                          blocks, preconditioner and PCG solves distributed over the shared memory of the
                          cluster's CTAs, about 40 knots per CTA, fewer where shared memory holds fewer:
                          25 for LQ nx 16, nu 8), 1 = never (one team from global memory),
                          2..8 = clusters of that many CTAs (at most 42 knots per CTA for nx 12, 32 for
                          nx 16, and what one CTA's shared memory holds, else one team);
                          applies with team_threads = 0; default 0 */
} dmpc_options;

/* Fill *opt with the defaults above. */
void dmpc_default_options(dmpc_options* opt);

/* Create a handle for `batch` OCPs (descs[0..batch-1], copied).  opt may be NULL (defaults).
 * cuda_stream: a cudaStream_t (NULL = default stream).  Allocates the device workspace and
 * warm-start buffers.  Errors: DMPC_E_ARG, DMPC_E_UNSUPPORTED, DMPC_E_OOM, DMPC_E_CUDA.
 * On error *out is NULL. */
dmpc_err dmpc_create_problem_batch(const dmpc_ocp_desc* descs, int batch, const dmpc_options* opt,
                                   void* cuda_stream, dmpc_handle** out);

/* Element offsets of each OCP in the packed arrays; every pointer may be NULL, each
 * non-NULL array has batch+1 entries (the last is the total length). */
dmpc_err dmpc_layout(const dmpc_handle* h, long long* z_off, long long* lam_off, long long* theta_off,
                     long long* xs_off, long long* xref_off);

/* Forward pass (Algorithm 2): opt.sqp_iters SQP iterations for every OCP of the batch.
 *   x_s, theta (required), x_ref (NULL = 0): inputs.  The kernel keeps device copies of
 *     them in the handle for the next dmpc_vjp, so the caller may free them on return.
 *   z_init (NULL: warm start from the previous solution if opt.warm_start, else the cold
 *     start x_t = x_s, u_t = 0), lam_init (NULL: previous multipliers or 0).
 *   z_out (required), lam_out (nullable): solution and multipliers.
 *   status_out (nullable, batch ints), pcg_iters_out (nullable, batch x sqp_iters ints:
 *   PCG iterations per QP), alpha_out (nullable, batch x sqp_iters floats: chosen step). */
dmpc_err dmpc_solve(dmpc_handle* h, const float* x_s, const float* theta, const float* x_ref,
                    const float* z_init, const float* lam_init, float* z_out, float* lam_out,
                    int* status_out, int* pcg_iters_out, float* alpha_out);

/* Backward pass (Algorithm 3, Eq. 3 and 7) at the last solution of this handle:
 *   dl_dz (n per OCP, required) -> dl_dtheta (p per OCP, required), dl_dxs (nx per OCP,
 *   required), lamt_out (adjoint multipliers, m per OCP, nullable), status_out (nullable),
 *   pcg_iters_out (nullable, batch ints).  KKT matrix: Gauss-Newton (Sec. 3.4) at the
 *   returned z.  Error DMPC_E_STATE if no solve preceded it. */
dmpc_err dmpc_vjp(dmpc_handle* h, const float* dl_dz, float* dl_dtheta, float* dl_dxs, float* lamt_out,
                  int* status_out, int* pcg_iters_out);

/* The plain one-launch-per-step form of the same method, for comparison: identical arguments,
 * results and resident state as dmpc_solve / dmpc_vjp (they may be mixed on one handle), but
 * every step (linearise, Schur blocks, preconditioner, each PCG operation of Algorithm 4,
 * recovery, line search) is a separate kernel launch over the batch and the per-OCP workspace
 * (the S and Phi^-1 blocks included) lives in HBM.  The launches of one call form a CUDA graph
 * (captured on the handle's first plain call, and again after a tiling change) in which each PCG
 * solve is a conditional WHILE node: it repeats eight PCG iterations until no OCP is still
 * iterating, decided on the device, with no host synchronisation.  Asynchronous on the handle's
 * stream.  Stored-Schur mode is not used. */
dmpc_err dmpc_solve_plain(dmpc_handle* h, const float* x_s, const float* theta, const float* x_ref,
                          const float* z_init, const float* lam_init, float* z_out, float* lam_out,
                          int* status_out, int* pcg_iters_out, float* alpha_out);
dmpc_err dmpc_vjp_plain(dmpc_handle* h, const float* dl_dz, float* dl_dtheta, float* dl_dxs, float* lamt_out,
                        int* status_out, int* pcg_iters_out);

/* Serving (continuous batching).  A handle's OCPs act as slots: the shapes given at creation
 * are each slot's capacity, and a slot can later hold any OCP that fits it.
 *   dmpc_set_ocps: re-describe slots index[0..n-1] (host arrays) with descs[i]; reset[i] != 0
 *     (host, nullable) makes the slot's next solve start cold instead of from its resident
 *     iterate.  Shapes must fit the slot (n, m, p, x_ref length and workspace) else
 *     DMPC_E_BUDGET; a single-model handle keeps its model.  Ordered on the handle's stream.
 *   dmpc_solve_subset: run opt.sqp_iters SQP iterations (Algorithm 2) on the slots listed in the
 *     DEVICE array index[0..n-1] (distinct slot numbers in [0, batch): the kernel reads them as
 *     given, so the caller guarantees this), each continuing from its resident iterate (or cold
 *     when reset);
 *     arrays are the handle-wide packed arrays of dmpc_layout (only listed slots are read or
 *     written).  With sqp_iters = 1 every call advances each listed problem by one SQP
 *     iteration, so requests can join between calls (continuous batching).
 *   dmpc_solve_subset_plain: the same on the plain one-launch-per-step form.
 *   dmpc_device_bytes: device memory owned by the handle (for budget-based admission). */
dmpc_err dmpc_set_ocps(dmpc_handle* h, int n, const int* index, const dmpc_ocp_desc* descs, const int* reset);
dmpc_err dmpc_solve_subset(dmpc_handle* h, const int* index, int n, const float* x_s, const float* theta,
                           const float* x_ref, float* z_out, float* lam_out, int* status_out, int* pcg_iters_out,
                           float* alpha_out);
dmpc_err dmpc_solve_subset_plain(dmpc_handle* h, const int* index, int n, const float* x_s, const float* theta,
                                 const float* x_ref, float* z_out, float* lam_out, int* status_out,
                                 int* pcg_iters_out, float* alpha_out);
long long dmpc_device_bytes(const dmpc_handle* h);

/* Diagnostic: build and solve ONE QP at (z, lam) for every OCP (Eq. 4, 8-11, Algorithm 4)
 * and write a record per OCP at record + rec_off[b] (rec_off from dmpc_inspect_offsets):
 *   A_t (T nx nx), B_t (T nx nu), C_t (T nx), g (K nx: x_0 - x_s, f_0..f_{T-1}),
 *   D, O, Pd, Po (K nx nx each; S_spd and Phi^-1 block rows, O_k couples k to k-1),
 *   gamma_spd (K nx), lambda+ (K nx), z+ (n), PCG iterations (1), of them in the extended-
 *   precision rescue (1).  lam may be NULL (0). */
dmpc_err dmpc_qp_inspect(dmpc_handle* h, const float* x_s, const float* theta, const float* x_ref,
                         const float* z, const float* lam, float* record);
dmpc_err dmpc_inspect_offsets(const dmpc_handle* h, long long* rec_off /* batch+1 */);

/* Allocation-free forward solve for callers that cannot allocate device memory when they
 * solve: a controller in a hard real-time loop restricted to memory reserved at start-up, a
 * plug-in inside a framework whose allocator owns the device, or a process at its memory limit.
 * The paper has no counterpart; it is the same forward pass as dmpc_solve (same kernels) for a
 * uniform batch (every OCP has shape *desc), without a handle.
 *   - Allocates nothing: no cudaMalloc/cudaFree or allocating library call.  Its scratch (record
 *     table, work list, and the per-team workspace when an OCP does not fit in shared memory)
 *     is one fixed device array of DMPC_NOALLOC_SCRATCH_BYTES that every GPU loading the library
 *     holds until process exit.  Requests whose scratch would exceed it return DMPC_E_BUDGET.
 *   - The first call on each device looks up that array's device address (once per device, with
 *     the device current); make the first call on a device before any stream capture.
 *   - Every call shares the array and overwrites it; calls that overlap on the GPU (different
 *     streams, or different host threads) race.  Serialise them on one stream.
 *   - No warm start and no dmpc_vjp: z_init / lam_init (nullable) give the initial guess, else
 *     the cold start.  Arguments are as in dmpc_solve; opt may be NULL (defaults);
 *     cuda_stream is a cudaStream_t (NULL = default stream).  Asynchronous on that stream. */
#define DMPC_NOALLOC_SCRATCH_BYTES (4u << 20)
dmpc_err dmpc_solve_noalloc(const dmpc_ocp_desc* desc, int batch, const dmpc_options* opt, void* cuda_stream,
                            const float* x_s, const float* theta, const float* x_ref, const float* z_init,
                            const float* lam_init, float* z_out, float* lam_out, int* status_out,
                            int* pcg_iters_out, float* alpha_out);

/* Measurement probes (the paper has no counterpart): the denominators the benchmark reports the
 * fused kernel against.  Both run synchronously on the current device, allocate a few bytes of
 * their own, time themselves with CUDA events (best of several repetitions) and are not meant
 * for a solve loop.
 *   dmpc_probe_fp32_peak: FP32 FMA throughput of the whole device in TFLOP/s (2 FLOP per FMA;
 *     eight independent FMA chains per thread, two 1024-thread blocks per SM); *ms_out
 *     (nullable) receives the timed launch's duration.
 *   dmpc_probe_pcg_floor: microseconds per iteration of the fused kernel's single-warp PCG inner
 *     loop (Algorithm 4 with nx = 4 and two knots per lane: two block-tridiagonal products, two
 *     warp reductions, the scalar divisions and the vector updates), one warp alone on the GPU,
 *     `iters` iterations (1 .. 2^24).  A PCG solve of k iterations takes at least k times it.
 * Errors: DMPC_E_ARG (null output, iters out of range), DMPC_E_OOM, DMPC_E_CUDA. */
dmpc_err dmpc_probe_fp32_peak(double* tflops_out, double* ms_out);
dmpc_err dmpc_probe_pcg_floor(int iters, double* us_per_iter_out);

/* Make (z, lam) with the inputs (x_s, theta, x_ref) the handle's resident solution, as if a
 * dmpc_solve had returned them: the next dmpc_vjp differentiates at that point (Algorithm 3
 * linearises at the given z, with lam as the multipliers).  Lets one handle serve several
 * solves of an autograd graph (a closed-loop rollout): each backward step restores the solution
 * its forward step returned.  All pointers are device pointers in the dmpc_layout packing,
 * x_ref may be NULL; lam is the float multiplier output of dmpc_solve.  Stored Schur blocks
 * (store_schur) are dropped, so the next vjp recomputes them.  Asynchronous on the stream.
 * Errors: DMPC_E_ARG, DMPC_E_CUDA. */
dmpc_err dmpc_set_solution(dmpc_handle* h, const float* z, const float* lam, const float* x_s,
                           const float* theta, const float* x_ref);

/* Change the stream used by later calls. */
dmpc_err dmpc_set_stream(dmpc_handle* h, void* cuda_stream);

/* Override the tiling: threads per OCP (32/64/128/256) and OCPs per block (>= 1).  An explicit
 * tiling runs every OCP on one team (no cluster form); (0, 0) restores the automatic choice made
 * at creation, the cluster form included. */
dmpc_err dmpc_set_tiling(dmpc_handle* h, int team_threads, int teams_per_block);

/* Current tiling and per-team workspace: team threads, teams per block, grid size, dynamic
 * shared memory bytes per block (0 when the workspace is in global memory). */
dmpc_err dmpc_get_tiling(const dmpc_handle* h, int* team_threads, int* teams_per_block, int* grid,
                         long long* smem_bytes);

/* Cluster form of the handle (Algorithm 4 distributed over a thread-block cluster; see
 * dmpc_options.cluster_ctas): CTAs per cluster, knots of the S and Phi^-1 blocks each CTA holds
 * in shared memory, and clusters per launch; all 0 when the handle runs one team per OCP.
 * Each pointer may be NULL.  In the cluster form CTA 0 of a cluster runs every other step of
 * the OCP from its global workspace, and every CTA takes part in its PCG solves. */
dmpc_err dmpc_get_cluster(const dmpc_handle* h, int* ctas_per_cluster, int* knots_per_cta, int* clusters);

/* The cluster shape the library takes for OCPs of nx states, nu inputs and at most `knots` knots
 * (T + 1) under dmpc_options.cluster_ctas = cluster_ctas, on a device whose CTAs may use
 * smem_per_cta bytes of shared memory (the opt-in limit: 232448 on GB300): CTAs per cluster, knots
 * of the S and Phi^-1 blocks (Eq. 8-10) each CTA holds, and the dynamic shared memory of one CTA.
 * All 0 when no shape fits the thread and shared-memory limits.  Host arithmetic only: touches no
 * GPU and needs none.  Whether a handle takes the shape also depends on its model having a cluster
 * kernel (12-state rigid body, LQ with nx 16) and on its one-team workspace; dmpc_get_cluster
 * reports what a handle took.  Each output pointer may be NULL.  DMPC_E_ARG: nx, nu or knots < 1,
 * cluster_ctas outside 0..8, smem_per_cta < 0. */
dmpc_err dmpc_cluster_shape(int nx, int nu, int knots, int cluster_ctas, long long smem_per_cta,
                            int* ctas_per_cluster, int* knots_per_cta, long long* smem_bytes);

/* Release the handle and its device memory (synchronises its stream). NULL is ignored. */
void dmpc_destroy(dmpc_handle* h);

/* Last error message of the handle (or of the last failed create when h is NULL). */
const char* dmpc_last_error(const dmpc_handle* h);

const char* dmpc_version(void);

#ifdef __cplusplus
}
#endif
#endif /* DMPC_H */
