/*
 * bidomain.h -- C-ABI of the GB300 Newton-Krylov BDDC / FETI-DP deluxe
 * solver for the segregated implicit Bidomain time step.
 *
 * Method: Huynh, Pavarino, Scacchi, "Parallel Newton-Krylov BDDC and FETI-DP
 * deluxe solvers for implicit time discretizations of the cardiac Bidomain
 * equations" (arXiv 2101.02959).  Each entry point cites the section and
 * equation that defines the operation it performs.
 *
 * Conventions shared by every call:
 *   - Every function returns an int status: BD_OK (0) or a negative BD_ERR_*.
 *     No exception crosses this boundary and no device trap is used; device
 *     failures (a non-positive pivot, a NaN, an exhausted wait) are recorded
 *     in a device flag and reported by the next call that synchronises.
 *   - Nodal vectors have length n_node (node ids lexicographic over the used
 *     grid nodes, x fastest) and are float64.  Two-field vectors (u_i, u_e or
 *     residual / correction pairs) are SoA: the u_i block then the u_e block,
 *     2*n_node doubles.
 *   - Interface vectors (length n_iface) hold two dofs per interface node in
 *     increasing node id, u_i then u_e.  Lagrange-multiplier vectors have
 *     length n_lambda.
 *   - on_device = 1: the pointers are CUDA device pointers; on_device = 0:
 *     host pointers (the library copies them through its own device buffers,
 *     inside the call).  The caller owns every pointer it passes; none is
 *     retained after the call returns.
 *   - All device work is enqueued on the stream given to bidomain_setup;
 *     calls that return data to the host or report statistics synchronise it.
 *   - A handle is not thread-safe; use one handle per host thread.
 */
#ifndef BIDOMAIN_H
#define BIDOMAIN_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define BD_OK 0
#define BD_ERR_ARG (-1)              /* invalid argument or unsupported option */
#define BD_ERR_NOT_SPD (-2)          /* a Cholesky pivot was <= 0 (e.g. tau > 0.37 ms) */
#define BD_ERR_KRYLOV_MAXIT (-3)     /* Krylov stopped at ksp_max_it */
#define BD_ERR_KRYLOV_DIVERGED (-4)  /* ||M^-1 r|| > dtol ||M^-1 b|| */
#define BD_ERR_NEWTON (-5)           /* Newton or its line search failed */
#define BD_ERR_NAN (-6)              /* NaN / Inf met in a residual or a norm */
#define BD_ERR_TIMEOUT (-7)          /* a device-side wait exhausted its budget; the handle's device
                                        work may still be running: destroy the handle */
#define BD_ERR_CUDA (-8)             /* a CUDA runtime call failed */
#define BD_ERR_NOMEM (-9)            /* device allocation failed */
#define BD_ERR_STATE (-10)           /* call made in the wrong order (e.g. no Jacobian yet) */
#define BD_ERR_SCRATCH (-11)         /* too large for the static scratch of schur_apply_noalloc */

/* ---- option values ----------------------------------------------------- */
#define BD_BDDC 0
#define BD_FETIDP 1
#define BD_PCG 0
#define BD_GMRES 1
#define BD_PRIMAL_V 0   /* vertex values (Section 6, Test 3 "V") */
#define BD_PRIMAL_VE 1  /* vertex values and edge averages ("V+E") */
#define BD_PRIMAL_VEF 2 /* vertex values, edge and face averages ("V+E+F", Section 6, Table 7) */
#define BD_SCALING_DELUXE 0
#define BD_SCALING_RHO 1
#define BD_FP64 0       /* every step in float64 */
#define BD_MIXED 1      /* local factors, Schur and deluxe blocks in float32;
                           Newton, Krylov vectors, dots and coarse in float64 */

/* index arrays for bd_plan_index_sets / bidomain_index_sets */
#define BD_IDX_ELEM_SUB 0      /* subdomain of each element (n_elem) */
#define BD_IDX_NODE_MULT 1     /* |N_x| of each node (n_node) */
#define BD_IDX_IFACE_NODES 2   /* interface nodes, sorted */
#define BD_IDX_CLS_TYPE 3      /* 0 vertex, 1 edge, 2 face, per class */
#define BD_IDX_CLS_PTR 4       /* CSR pointer of class nodes (n_cls + 1) */
#define BD_IDX_CLS_NODES 5     /* class nodes, sorted inside each class */
#define BD_IDX_CLS_SUB_PTR 6   /* CSR pointer of N_C (n_cls + 1) */
#define BD_IDX_CLS_SUBS 7      /* subdomains sharing each class */
#define BD_IDX_CLS_DUAL_START 8 /* first global dual dof of each class */
#define BD_IDX_SUB_NODE_PTR 9  /* CSR pointer of local nodes (n_sub + 1) */
#define BD_IDX_SUB_NODES 10    /* local nodes: interior then interface, each sorted */
#define BD_IDX_SUB_NINT 11     /* number of interior nodes per subdomain */
#define BD_IDX_SUB_DUAL_PTR 12 /* CSR pointer of local dual dofs */
#define BD_IDX_SUB_DUAL 13     /* global transformed dual dof of each local dual dof */
#define BD_IDX_SUB_PRIMAL_PTR 14
#define BD_IDX_SUB_PRIMAL 15   /* global primal dof of each local primal dof */
#define BD_IDX_GAUGE 16        /* {gauge node, gauge primal dof} */

typedef struct bd_plan bd_plan;
typedef struct bd_handle bd_handle;

/* Structured grid of n[0] x n[1] x n[2] Q1 hexahedra, split into blocks of
 * s[0] x s[1] x s[2] elements (Section 4.1).  elem_mask (host, nullable): one
 * byte per grid element, x fastest, 1 = keep; each block is split into
 * node-connected components.
 * geometry BD_GEOM_BOX (0, what a zero-filled struct gives): the grid spans
 *   [0,l0]x[0,l1]x[0,l2] cm; the slab fibres of Section 6.
 * geometry BD_GEOM_ELLIPSOID: the truncated ellipsoid of Section 6, a grid
 *   uniform in (phi, theta, r) over [phi0,phi1]x[theta0,theta1]x[0,1] (l is
 *   ignored) mapped by x = a(r) cos(theta) cos(phi), y = b(r) cos(theta) sin(phi),
 *   z = c(r) sin(theta) with a(r) = a1 + r (a2 - a1), likewise b and c
 *   (axes = a1, a2, b1, b2, c1, c2 in cm, all positive; -pi/2 < theta0 <
 *   theta1 < pi/2); isoparametric Q1 elements, fibres rotating 120 degrees
 *   with the depth r.  Stimulus boxes are then given in (phi, theta, r).
 * Invalid sizes or ranges give BD_ERR_ARG. */
#define BD_GEOM_BOX 0
#define BD_GEOM_ELLIPSOID 1
typedef struct {
  int n[3];
  double l[3];
  int s[3];
  const unsigned char *elem_mask;
  int geometry;
  double axes[6];
  double phi[2], theta[2];
} bd_mesh;

/* Conductivity coefficients (S/cm) along fibre, cross-fibre and sheet normal
 * (Section 2, Table 1).  Slab fibres rotate by 120 degrees through the depth,
 * counter-clockwise from the epicardium (z = l2) to the endocardium (z = 0). */
typedef struct {
  double sigma_i[3];
  double sigma_e[3];
} bd_conductivity;

/* Rogers-McCulloch parameters (Section 2, Table 1); chi_cm = chi * Cm in
 * mF/cm^3; potentials in mV measured from rest. */
typedef struct {
  double G, eta1, eta2, vth, vp, chi_cm;
} bd_ionic;

/* Transmembrane stimulus of amplitude amp (mA/cm^3) on the nodes inside the
 * box {x0,x1,y0,y1,z0,z1} of the grid's coordinates (cm for a box; phi, theta,
 * r for the ellipsoid), active for t_on <= t_{n+1} < t_off (ms). */
typedef struct {
  double amp, t_on, t_off;
  double box[6];
} bd_stimulus;

/* Solver options; defaults (bd_options_default) are the tolerances of the
 * paper's Section 6 table: KSP rtol 1e-8, atol 1e-10, dtol 1e4; SNES rtol
 * 1e-4, atol 1e-8, stol 1e-8; BDDC, PCG, V+E, FP64. */
typedef struct {
  int method;        /* BD_BDDC | BD_FETIDP */
  int krylov;        /* BD_PCG | BD_GMRES */
  int primal;        /* BD_PRIMAL_V | BD_PRIMAL_VE | BD_PRIMAL_VEF */
  int precision;     /* BD_FP64 | BD_MIXED */
  int gmres_restart; /* GMRES restart length (default 30) */
  int ksp_max_it;    /* default 1000 */
  int newton_max_it; /* default 50 */
  int use_graphs;    /* 1: replay the Krylov iteration as a captured CUDA graph */
  double ksp_rtol, ksp_atol, ksp_dtol;
  double snes_rtol, snes_atol, snes_stol;
  /* learned initial guess (not in the paper): 1 = predict u^0 with the
   * per-subdomain MLP once two previous states exist; it is trained online with
   * Adam (learning rate mlp_lr) on the steps before mlp_train_steps and used
   * from mlp_warmup training steps on, only when its residual is below the
   * previous-step residual (the fallback); tolerances stay anchored to the
   * fallback residual. */
  int learned_guess, mlp_train_steps, mlp_warmup, mlp_epochs;
  double mlp_lr;
  /* BD_MIXED only: 1 = the rank-k Schur updates of the factorisations run on
   * the tensor cores (tcgen05, TF32 split in hi + lo parts, FP32 accumulation);
   * 2 = also the rows below every 128-column panel, solved as one tensor-core
   * product with the inverse of the panel's factored diagonal block */
  int use_tensor_cores;
  /* 1 = chord Newton: factorise the Jacobian at the first Newton iterate of a
   * time step and reuse it for the later iterations of that step (every iterate
   * is still tested with the exact FP64 residual; when the line search finds no
   * decrease along a lagged direction, the Jacobian is formed at the current
   * iterate and the iteration repeated); 0 = factorise at every Newton iterate
   * (the paper's setting, the default). */
  int lag_jacobian;
  /* scaling of the dual variables (Section 4.2): BD_SCALING_DELUXE (default) or
   * BD_SCALING_RHO (delta_j = sigma_M^(j) / sum over N_x of sigma_M^(k), sigma_M the
   * largest principal conductivity of the medium; 1 / |N_x| here, where every
   * subdomain has the same conductivities) */
  int scaling;
  /* BD_BDDC only: rebuild the preconditioner (transformed local matrices, deluxe
   * blocks, coarse problem) at every precond_every-th Jacobian evaluation, counted
   * from setup; in between, the Krylov solve applies the current Schur operator
   * with the older preconditioner (not in the paper, which rebuilds it each time).
   * 1 = every evaluation (the default).  Values below 1, or above 1 with
   * BD_FETIDP, whose operator contains the preconditioner's local solves, give
   * BD_ERR_ARG.  Evaluations inside bidomain_autotune rebuild it and do not count. */
  int precond_every;
} bd_options;

typedef struct {
  int its;        /* Krylov iterations */
  int reason;     /* BD_OK or BD_ERR_KRYLOV_* */
  double res0;    /* ||M^-1 b|| */
  double res;     /* final ||M^-1 r|| */
  double cond;    /* Lanczos estimate of cond(M^-1 A) (PCG only, else 0) */
} bd_solve_stats;

typedef struct {
  int newton_its;   /* Newton iterations of this step */
  int krylov_its;   /* Krylov iterations summed over them */
  int reason;       /* BD_OK or the failure code */
  int pad;
  double res0;      /* ||F(u^n) - G|| */
  double res_final; /* ||F(u^{n+1}) - G|| */
  double cond_max;  /* largest Lanczos estimate met in the step */
  int guess_used;   /* 1 when Newton started from the learned guess */
  int pad2;
  double res_guess; /* ||F(u_guess) - G|| (0 when no guess was formed) */
  double mlp_loss;  /* training loss of this step (0 when not training) */
} bd_step_stats;

typedef struct {
  int n_node, n_elem, n_sub, n_cls;
  int n_iface, n_dual, n_primal, n_lambda;
  int gauge_node, gauge_primal;
} bd_sizes;

/* ---- host-only plan (no GPU) ------------------------------------------- */

/* Section 4.1: grid, subdomains, N_x, face/edge/vertex classes, primal set
 * (primal = BD_PRIMAL_V, BD_PRIMAL_VE or BD_PRIMAL_VEF) and dof maps, built on the host.
 * Fails with BD_ERR_ARG when a subdomain has no primal constraint or the
 * partition has no vertex (no gauge). */
int bd_plan_create(const bd_mesh *mesh, int primal, bd_plan **out);
int bd_plan_sizes(const bd_plan *plan, bd_sizes *out);
/* Copies index array `which` (BD_IDX_*) into out[0..cap); *len receives its
 * length.  Returns BD_ERR_ARG if cap < *len (nothing copied past cap). */
int bd_plan_index_sets(const bd_plan *plan, int which, int64_t *out, int64_t cap, int64_t *len);
void bd_plan_destroy(bd_plan *plan);

/* ---- solver handle ------------------------------------------------------ */

int bd_options_default(bd_options *opt);

/* Builds the plan, assembles the Q1 stiffness A_i, A_e and lumped mass M
 * (Section 3a), the subassembled local stencils of every subdomain (local
 * forms a^(j), Section 4.1) and allocates every device buffer.  stream: a
 * cudaStream_t (NULL = the library creates its own).  tau in ms. */
int bidomain_setup(const bd_mesh *mesh, const bd_conductivity *cond, const bd_ionic *ionic,
                   double tau, const bd_options *opt, void *stream, bd_handle **out);
int bidomain_sizes(const bd_handle *h, bd_sizes *out);
int bidomain_index_sets(const bd_handle *h, int which, int64_t *out, int64_t cap, int64_t *len);

/* State (u_i, u_e, w) at time t (ms); t sets the step counter n = round(t/tau).
 * With the learned initial guess, the history of earlier states it reads is kept
 * when n equals the handle's own step counter (the caller hands back the state of
 * the current step, e.g. after a host round trip) and restarts otherwise. */
int bidomain_set_state(bd_handle *h, const double *ui, const double *ue, const double *w,
                       double t, int on_device);
int bidomain_get_state(bd_handle *h, double *ui, double *ue, double *w, double *t, int on_device);

/* One decoupled backward-Euler step (Section 3b): Step 1 gating update, then
 * Newton (Section 3c) on F(u) = G with the configured Krylov method and
 * preconditioner, then the gauge shift that gives u_e zero lumped-mass mean.
 * stats may be NULL.  Advances t by tau. */
int bidomain_step(bd_handle *h, const bd_stimulus *stim, bd_step_stats *stats);

/* Step 1 alone (Section 3b): w_next = (w + tau eta2 v / v_p) / (1 + tau eta2),
 * v = ui - ue.  Nodal vectors. */
int bidomain_gating(bd_handle *h, const double *ui, const double *ue, const double *w,
                    double *w_next, int on_device);

/* F(u) - G of Step 2 (Section 3b) at u = (ui, ue) with w_next, previous
 * potentials (ui_n, ue_n) and the stimulus evaluated at t_next.
 * r: 2*n_node (SoA). */
int bidomain_residual(bd_handle *h, const bd_stimulus *stim, double t_next, const double *ui,
                      const double *ue, const double *w_next, const double *ui_n,
                      const double *ue_n, double *r, int on_device);

/* Jacobian of Section 3c at (ui, ue, w_next): updates the local matrices,
 * factorises them, forms the local Schur complements, deluxe blocks and the
 * coarse problem (Sections 4.1-4.4).  Required before the three calls below
 * and before krylov_solve.  Counts as a Jacobian evaluation of the
 * precond_every schedule: between rebuilds only the local factors and Schur
 * complements are updated. */
int bidomain_linearize(bd_handle *h, const double *ui, const double *ue, const double *w_next,
                       int on_device);

/* S_hat x = sum_j R_j^T S_Gamma^(j) R_j x (Section 4.1, eq. schursys);
 * interface vectors; the gauge entry of y is 0. */
int schur_apply(bd_handle *h, const double *x, double *y, int on_device);

/* z = M^-1_BDDC r = Rt_D^T St^-1 Rt_D r (Section 4.4) with deluxe scaling
 * (Section 4.2); interface vectors. */
int bddc_apply(bd_handle *h, const double *r, double *z, int on_device);

/* mu = M^-1_FETI-DP lambda = B_D St B_D^T lambda (Section 4.3); multiplier
 * vectors (fully redundant multipliers u_j - u_m, j < m, per dual dof). */
int fetidp_apply(bd_handle *h, const double *lambda, double *mu, int on_device);

/* y = F lambda = B St^-1 B^T lambda (Section 4.3, eq. lagrangesystem). */
int fetidp_operator(bd_handle *h, const double *lambda, double *y, int on_device);

/* Solves the Jacobian system J s = f (Section 3c, eq. Jacobiansystem) by the
 * configured Krylov method on the interface system (BDDC) or the multiplier
 * system (FETI-DP), then recovers the interior (Section 4.1).  f, s: 2*n_node
 * (SoA).  The u_e correction at the gauge node is 0.  stats may be NULL. */
int krylov_solve(bd_handle *h, const double *f, double *s, int on_device, bd_solve_stats *stats);

/* ---- coarse problem of the current Jacobian (Section 4.4) --------------------------
 * S_PiPi = sum_j R_Pi^T S_PiPi^(j) R_Pi as assembled for the preconditioner, in FP64,
 * as CSR over the global primal dofs (columns ascending; the gauge row and column are
 * the unit vector), and its solve as every preconditioner application performs it: the
 * explicit inverse followed by `nref` steps of FP64 iterative refinement
 * z += X (c - S_PiPi z) (nref < 0: the handle's own count).  Up to 320 coarse unknowns
 * the inverse is brought to FP64 once per Jacobian (Newton-Schulz) and refined once per
 * solve; above, it is kept in the local precision (FP32 in BD_MIXED, refined 4 times per
 * solve; FP64 in BD_FP64, refined once).  Host buffers; the handle must be linearised. */
int bidomain_coarse_size(bd_handle *h, int *n_primal, int *nnz);
int bidomain_coarse_matrix(bd_handle *h, int *rowptr, int *col, double *val);
int bidomain_coarse_solve(bd_handle *h, const double *c, double *z, int nref);

/* ---- autotuner (not in the paper) ----------------------------------------------
 * Times the whole factorisation sequence of bidomain_linearize (CUDA events,
 * best of two after a warm-up) at the current Jacobian for every combination of
 * outer block width {128, 256, 512} (columns per long-K trailing update; panels
 * are 128 columns), number of subdomain groups the batch is factorised in
 * {1, 2, 4} and, in BD_MIXED, the arithmetic: SIMT FP32 (tensor_cores = 0), the
 * rank-k updates on the tensor cores (1), or also the rows below every panel solved on
 * the tensor cores as one product with the inverse of the 128 x 128 diagonal block (2);
 * keeps the fastest for the handle and leaves the Jacobian factorised with it.
 * Requires bidomain_linearize (or a step) first.  Results are identical up to rounding
 * for every choice. */
typedef struct {
  int outer_panel, groups, tensor_cores, candidates;
  double best_ms, default_ms;
} bd_tune_result;
int bidomain_autotune(bd_handle *h, bd_tune_result *out);

/* ---- learned initial guess (not in the paper) ------------------------------
 * The per-subdomain MLP maps local traces of the last three states (6 per
 * node: v^n, v^n - v^{n-1}, v^{n-1} - v^{n-2}, u_e^n and its two differences,
 * all / 100 mV, padded to the largest subdomain) to the increment u^{n+1} - u^n
 * at its nodes (2 per node).  Layers: n_in -> 256 -> 256 -> n_out, ReLU,
 * bfloat16 weights, float32 accumulation.  Parameters are packed float32:
 * W1 (256 x n_in), b1, W2 (256 x 256), b2, W3 (n_out x 256), b3. */
int bidomain_mlp_sizes(bd_handle *h, int *n_in, int *n_hidden, int *n_out, int *batch);
/* set = 1: upload the packed parameters from host memory (and refresh the
 * bfloat16 copies); set = 0: download them. */
int bidomain_mlp_params(bd_handle *h, float *w, int set);
/* Loss sum(mask (y - t)^2) / sum(mask) and its packed gradient for host
 * inputs X (batch x n_in), targets T and mask (batch x n_out). */
int bidomain_mlp_loss_grad(bd_handle *h, const float *X, const float *T, const float *mask, double *loss,
                           float *grad);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8, bias correction; Kingma and Ba,
 * Algorithm 1) of the packed parameters with the packed host gradient `grad` and
 * learning rate lr: the update the online training applies after each backward pass. */
int bidomain_mlp_adam_step(bd_handle *h, const float *grad, double lr);
/* Back to the untrained network: the initial weights (the fixed seeded He-uniform
 * draw of bidomain_setup), zero Adam moments and step count, no training steps
 * counted, and no state history. */
int bidomain_mlp_reset(bd_handle *h);

/* ---- no-allocation variant ------------------------------------------------
 * The paper has no counterpart: this is a deployment variant of schur_apply.
 * It computes the same y = S_hat x, but keeps its scratch (the per-subdomain
 * products S_Gamma^(j) R_j x before they are summed onto the interface) in a
 * fixed device array compiled into the library instead of memory obtained
 * with cudaMalloc.  It is meant for callers that must not allocate device
 * memory when they apply the operator: code running under a fixed device-
 * memory budget, or inside a host framework that owns every allocation.
 *   - x, y: device pointers to interface vectors (n_iface doubles).
 *   - The handle must have been linearised (BD_ERR_STATE otherwise), and the
 *     device current at the call must be the one the handle was set up on
 *     (BD_ERR_STATE otherwise: the array's address differs from device to device).
 *   - Capacity: the sum over subdomains of their interface unknowns must not
 *     exceed 524288 doubles (4 MiB); larger problems get BD_ERR_SCRATCH.
 *     Every GPU that loads the library holds this 4 MiB until the process exits.
 *   - The first call on a device looks up the array's device address with
 *     that device current; make that first call before any stream capture.
 *   - Every call shares the one array and overwrites all of it that it reads,
 *     so nothing needs clearing between calls; calls that overlap on the GPU
 *     (other streams, other threads) race on it.
 *   - No cudaMalloc, cudaFree or allocating library routine is called.
 *     The call synchronises the handle's stream. */
int schur_apply_noalloc(bd_handle *h, const double *x, double *y);

/* ---- instrumentation (no counterpart in the paper) ------------------------- */

/* Kernel classes timed by bidomain_profile_read. */
#define BD_PROF_RANKK 0  /* rank-k updates of the batched partial Cholesky (Schur formation) */
#define BD_PROF_PANEL 1  /* diagonal-block factorisation and panel solves */
#define BD_PROF_GEMV 2   /* dense local matvecs of every Krylov iteration (S_Gamma, S_DD^-1, Psi) */
#define BD_PROF_RESID 3  /* Newton residual F(u) - G */
/* Regions of a step, each timed as a whole (with enable = 2 also while the Krylov
 * iterations replay as CUDA graphs): */
#define BD_PROF_LINEARIZE 4  /* the Jacobian and every factorisation (Sections 4.1-4.4) */
#define BD_PROF_KRYLOV 5     /* one Krylov solve (PCG or GMRES, all iterations) */
#define BD_PROF_TRSV 6       /* interior condensation / recovery triangular solves */
#define BD_PROF_MLP 7        /* learned initial guess: prediction and online training */
#define BD_PROF_STEP 8       /* one whole bidomain_step */

/* enable = 1 records a CUDA event pair on the handle's stream around every
 * launch of the kernel classes and around every region above (and clears the
 * totals); enable = 2 records the regions only; 0 stops recording.  Per-launch
 * events are not recorded inside captured CUDA graphs. */
int bidomain_profile(bd_handle *h, int enable);
/* out[4] = {launches, total milliseconds, algorithmic flops, algorithmic bytes}
 * summed over the launches of class `which` since profiling was enabled.
 * Synchronises the stream. */
int bidomain_profile_read(bd_handle *h, int which, double *out);
/* Kernel launches issued by this library in this process so far. */
int64_t bidomain_launch_count(void);

int bidomain_destroy(bd_handle *h);
const char *bidomain_strerror(int status);
/* The message of the last failure recorded on handle h (the failing CUDA call or
 * argument check), or, with h == NULL, of the last failure on this thread before a
 * handle existed (bd_plan_create, bidomain_setup).  Empty when there is none.  The
 * pointer stays valid until the next call on the same handle or thread. */
const char *bidomain_last_error(const bd_handle *h);

#ifdef __cplusplus
}
#endif
#endif /* BIDOMAIN_H */
