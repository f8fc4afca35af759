/*
 * nhmf -- matrix-free compressible neo-Hookean finite-strain elasticity on structured
 * Q_p hexahedral meshes of the unit cube, for one NVIDIA GB300 (sm_103a).
 *
 * The operations follow the paper's statement of the problem (arXiv 2505.15535):
 *   - energy Psi = mu/2 (tr C - 3 - 2 ln J) + lambda (ln J)^2          (Eq. hypref)
 *   - residual R(u)_i = int P(F) : Grad phi_i dV, P = dPsi/dF          (Eq. F)
 *   - tangent  W_i = K(u; du, phi_i) = int Grad du : L : Grad phi_i dV (Eq. DF, Eq. L;
 *     Algorithm 1 "Given u, du / Return W")
 *   - Q_p elements with (p+1)^3 Gauss points per element               (Section 2.2, 2.4)
 *   - operator diagonal (used by Jacobi / Chebyshev smoothing)         (Section 2.3)
 *
 * Discretisation readings fixed by this library:
 *   mesh      Omega = [0,1]^3 split into N^3 cubes of side h = 1/N; Q_p on GLL nodes;
 *             M = pN + 1 nodes per direction; (p+1)-point Gauss-Legendre rule.
 *   vectors   caller-owned DEVICE arrays of 3*M^3 entries, component-major:
 *             entry c*M^3 + i + M*(j + M*k) is component c at node (i, j, k), x fastest.
 *   Dirichlet the constrained operator is A du = P_f K(u) P_f du + P_D du (identity rows and
 *             columns on the constrained set D); residual rows on D are zero.
 *             Presets: NHMF_BC_NONE (raw operator), NHMF_BC_CLAMP_X0 (all components on
 *             x = 0), NHMF_BC_COMPRESSION (all components on z = 0, u_z on z = 1).
 *
 * Asynchrony: every call enqueues its kernels on `stream` (a cudaStream_t passed as void*;
 * NULL = legacy default stream) and returns without waiting, unless its comment says it
 * synchronises.  One context must not be used from two host threads at the same time.
 *
 * Errors: calls return an nhmf_status; no call aborts the process or traps on the device.
 * Kernels that meet det F <= 0 or a non-finite value record it in a device status word that
 * nhmf_check_status() (and every synchronising call) turns into NHMF_ERR_NONPOS_J /
 * NHMF_ERR_NONFINITE.  Every device-side wait is bounded: a tensor-core convolution whose
 * completion wait runs out records that too (NHMF_ERR_CUDA, "tensor-core completion wait
 * timed out") and returns.  nhmf_last_error() returns a text description of the last failure.
 */
#ifndef NHMF_H
#define NHMF_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  NHMF_OK = 0,
  NHMF_ERR_ARG = 1,           /* invalid argument (null pointer, bad size, bad enum) */
  NHMF_ERR_CUDA = 2,          /* a CUDA runtime call or kernel launch failed */
  NHMF_ERR_OOM = 3,           /* device allocation failed */
  NHMF_ERR_NONPOS_J = 4,      /* det F <= 0 at some quadrature point */
  NHMF_ERR_NONFINITE = 5,     /* NaN or Inf met */
  NHMF_ERR_BREAKDOWN = 6,     /* Krylov breakdown (p^T A p <= 0) */
  NHMF_ERR_NOT_CONVERGED = 7, /* iteration limit reached */
  NHMF_ERR_STATE = 8          /* call out of order (e.g. apply before set_linearization) */
} nhmf_status;

enum { NHMF_FP64 = 0, NHMF_FP32 = 1, NHMF_DF64 = 2 };      /* arithmetic of an apply */
enum { NHMF_ON_THE_FLY = 0, NHMF_CACHED = 1, NHMF_SPATIAL = 2 }; /* point-code strategies */
enum { NHMF_BC_NONE = 0, NHMF_BC_CLAMP_X0 = 1, NHMF_BC_COMPRESSION = 2 };
enum { NHMF_CACHE_FP64 = 1, NHMF_CACHE_FP32 = 2, NHMF_CACHE_DF64 = 4, NHMF_CACHE_SPATIAL = 8 };
/* bit mask for set_linearization */

typedef struct nhmf_ctx nhmf_ctx;

enum { NHMF_MODEL_COMPRESSIBLE = 0, NHMF_MODEL_SPLIT = 1 };

typedef struct {
  int n_el;       /* N, elements per direction, >= 1 */
  int degree;     /* p, 1..4 */
  double mu;      /* shear modulus, > 0 */
  double lambda;  /* second constant, >= 0: the Lame constant lambda of Eq. hypref (the energy
                     uses lambda (ln J)^2), or the bulk modulus kappa of Eq. hypcomplex */
  int bc;         /* NHMF_BC_* preset */
  double top_uz;  /* prescribed u_z on z = 1 for NHMF_BC_COMPRESSION (solver only) */
  int model;      /* NHMF_MODEL_COMPRESSIBLE: Psi = mu/2 (tr C - 3 - 2 ln J) + lambda (ln J)^2
                     (Eq. hypref); NHMF_MODEL_SPLIT: Psi = mu/2 (tr Cbar - 3)
                     + kappa/2 ((J^2 - 1)/2 - ln J), Cbar = J^(-2/3) C (Eq. hypcomplex), which
                     supports the NHMF_ON_THE_FLY and NHMF_SPATIAL strategies */
} nhmf_params;

/* Create a context for one mesh/material on the current CUDA device.  Allocates the
 * context's own device buffers (linearisation copy, status word) and, on the first context
 * of a device, resolves the device address of the static scratch array of
 * nhmf_linear_solve_noalloc, which loads that array (6.3 MB) on the device until the process
 * exits.  Synchronous. */
nhmf_status nhmf_create(const nhmf_params* params, nhmf_ctx** out);

/* Free the context and every device buffer it owns.  Synchronises the device. */
void nhmf_destroy(nhmf_ctx* ctx);

/* Number of DoFs, 3*(p*N+1)^3. */
size_t nhmf_num_dofs(const nhmf_ctx* ctx);

/* Text of the last error on this context (static storage owned by the context). */
const char* nhmf_last_error(const nhmf_ctx* ctx);

/* Fix the linearisation point u (device, FP64, 3*M^3; read only, may be freed after the
 * call) for later tangent/diagonal calls: copies u into the context and, for each bit of
 * `cache_mask`, builds the per-quadrature-point cache of the cached strategy (Section 3.2
 * "partial assembly"): F^-1 (9 values) and ln J (1 value) per point, computed in FP64 and
 * stored in FP64 (NHMF_CACHE_FP64), FP32 (NHMF_CACHE_FP32) and/or as double-float pairs
 * (NHMF_CACHE_DF64, for the NHMF_DF64 apply, layout as FP64 with a (hi, lo) FP32 pair per
 * value) and/or the 36-value FP64 cache of NHMF_SPATIAL (NHMF_CACHE_SPATIAL: J c in Voigt
 * order 11, 22, 33, 23, 13, 12 as the upper triangle of a 6x6 matrix (21), tau (6, Voigt),
 * F^-1 (9, row-major); layout [36][E*(p+1)^3]); 10*E*(p+1)^3 values
 * each, layout [10][E*(p+1)^3] with elements in colour-major order, except the FP32 cache,
 * whose elements are in natural order ex + N (ey + N ez) (the FP32 apply runs over all
 * elements at once), and which for p <= 2 on meshes of N >= 64 is tiled by 32 elements,
 * [E/32][10][(p+1)^3][32], for the one-thread-per-element kernel.  Also allocates the FP32 apply's element-local result buffer
 * (3*E*(p+1)^3 floats) on first call.  Synchronises and returns NHMF_ERR_NONPOS_J if
 * det F <= 0 anywhere. */
nhmf_status nhmf_set_linearization(nhmf_ctx* ctx, const double* u, int cache_mask, void* stream);

/* v = A(u) du with u the current linearisation point.  Strategies: NHMF_ON_THE_FLY
 * (Algorithm 1: F, F^-1, ln J recomputed at every point), NHMF_CACHED (F^-1 and ln J read from
 * the point cache), NHMF_SPATIAL (Algorithm 2, partial assembly in the current configuration,
 * Eq. DF:cur: per point J c (21 values, minor and major symmetry), the Kirchhoff stress
 * tau = J sigma (6) and F^-1 (9) are read from the NHMF_CACHE_SPATIAL cache, and
 * G = [J c : sym(grad du) + grad du tau] F^-T with grad du = Grad du F^-1; FP64 only).  `precision` NHMF_FP64: du, v are double*; NHMF_FP32: du,
 * v are float* and all arithmetic after the cache build runs in FP32 with FP32 accumulation;
 * NHMF_DF64 (cached strategy only): du, v are double* and the arithmetic is double-float (pairs
 * of FP32 numbers, about 48 significant bits) on the FP32 pipe, reading the NHMF_CACHE_DF64
 * point cache.
 * du and v are device arrays of 3*M^3 entries and must not overlap.  Asynchronous.
 * NHMF_ERR_STATE if no linearisation point (or no cache of that precision) is set. */
nhmf_status nhmf_tangent_apply(nhmf_ctx* ctx, int precision, int strategy, const void* du,
                               void* v, void* stream);

/* Tangent application at a given linearisation point (Algorithm 1: given u and du, return
 * W): v = A(u) du, on the fly in FP64, reading u directly.  u, du, v: device FP64
 * [3][M^3], u as in nhmf_set_linearization, du and v as in nhmf_tangent_apply.  No point
 * cache is built and the stored linearisation point (if any) is neither needed nor changed.
 * Asynchronous on `stream`; det F <= 0 at a point is recorded in the status word
 * (nhmf_check_status).  NHMF_ERR_ARG for null pointers or v aliasing u or du. */
nhmf_status nhmf_tangent_apply_at(nhmf_ctx* ctx, const double* u, const double* du, double* v, void* stream);

/* r = R(u) (Eq. F, no traction) in FP64 for the device vector u; rows on D are zero.
 * Synchronises and returns NHMF_ERR_NONPOS_J if det F <= 0 at a point, NHMF_ERR_NONFINITE if
 * u holds a non-finite value or the stress overflows. */
nhmf_status nhmf_residual(nhmf_ctx* ctx, const double* u, double* r, void* stream);

/* d = diag(A(u)) in FP64 at the current linearisation point (1 on D).  Asynchronous. */
nhmf_status nhmf_diagonal(nhmf_ctx* ctx, double* d, void* stream);

/* Heterogeneous material: per-element factors f_e > 0 multiplying mu and lambda (kappa) on
 * element e (the paper's test material has inclusions 100x stiffer than the matrix,
 * Section 3.1).  `factors` is a device array of N^3 doubles in natural element order
 * ex + N (ey + N ez), copied into the context; NULL restores the homogeneous material.  Every
 * operator (residual, tangent apply of every strategy and precision, diagonal, solvers and
 * the multigrid levels, whose coarse elements take the mean of their eight children) uses
 * them.  Synchronises. */
nhmf_status nhmf_set_material_factors(nhmf_ctx* ctx, const double* factors, void* stream);

/* Synchronise `stream`, read and clear the device status word.  Returns NHMF_OK,
 * NHMF_ERR_NONPOS_J, NHMF_ERR_NONFINITE, NHMF_ERR_BREAKDOWN or NHMF_ERR_CUDA (a bounded
 * tensor-core wait ran out). */
nhmf_status nhmf_check_status(nhmf_ctx* ctx, void* stream);

/* ------------------------------------------------------------------ solvers
 * Newton's method with load steps (Section 2.1-2.3): at Newton iterate u, solve
 * A(u) du = b with b = -R(u) on free rows and b = g - u on constrained rows (g the
 * prescribed values of the current load step; the Dirichlet increment is lifted through
 * the unconstrained operator, b_f -= K(u) (g - u)_D), then u += theta du with theta halved
 * while det F <= 0 is met.  A load step converges when ||b|| <= newton_rtol * ||b_0||, b_0
 * the right-hand side of its first iteration.
 * Linear solvers (all on the device; scalars stay on the device and the host reads the
 * residual norm every `check_every` iterations):
 *   NHMF_SOLVER_JACOBI_CG  FP64 CG preconditioned by the inverse operator diagonal
 *                          (the plain baseline);
 *   NHMF_SOLVER_MIXED_FCG  FP64 flexible CG whose preconditioner is an FP32 Jacobi-CG on the
 *                          FP32 apply (FP64 residuals, dot products and updates outside);
 *   NHMF_SOLVER_LEARNED_FCG FP64 flexible CG preconditioned by the trained U-Net, z = N(r);
 *                          falls back to Jacobi-CG from the current iterate on stagnation;
 *   NHMF_SOLVER_MIXED_LEARNED FP64 multi-preconditioned CG with two search directions per
 *                          iteration, the FP32 inner Jacobi-CG of MIXED_FCG and N(r), combined
 *                          by a 2x2 Galerkin step and A-orthogonalised against the previous
 *                          pair; same fallback;
 *   NHMF_SOLVER_GMG        FP64 flexible CG preconditioned by one geometric-multigrid V-cycle
 *                          (Section 2.3): levels N, N/2, ... (halving while N is even and
 *                          N/2 >= 2) with degree p, then degree 1 on the coarsest mesh when
 *                          p > 1; level operators at the linearisation point interpolated
 *                          to each level, Chebyshev smoothing on the inverse diagonal
 *                          (smoother_degree steps on [lmax/smoother_range, 1.2 lmax], lmax from
 *                          12 power iterations in the V-cycle's precision), transfer by
 *                          interpolation and its transpose, Jacobi-CG on the coarsest level
 *                          (to 1e-6 in an FP64 V-cycle, 1e-4 in an FP32 one);
 *   NHMF_SOLVER_MIXED_GMG  the same V-cycle in FP32 (FP32 applies, smoothers, transfers)
 *                          inside FP64 flexible CG;
 *   NHMF_SOLVER_MIXED_GMG_LEARNED the FP32 V-cycle V plus the trained U-Net N on the residual
 *                          the V-cycle leaves, z = V(r) + omega c with c = N(t), t = r - A V(r),
 *                          and the A-optimal step omega = (c.t) / (c.A c) (A by FP32 applies),
 *                          inside FP64 flexible CG; the network is trained on pairs
 *                          recorded by MIXED_GMG solves (record_pairs); falls back to
 *                          Jacobi-CG from the current iterate on stagnation as the learned
 *                          solvers do. */
enum { NHMF_SOLVER_JACOBI_CG = 0, NHMF_SOLVER_MIXED_FCG = 1, NHMF_SOLVER_LEARNED_FCG = 2,
       NHMF_SOLVER_MIXED_LEARNED = 3, NHMF_SOLVER_GMG = 4, NHMF_SOLVER_MIXED_GMG = 5,
       NHMF_SOLVER_MIXED_GMG_LEARNED = 6 };
#define NHMF_MAX_STEPS 64

typedef struct {
  int solver;           /* NHMF_SOLVER_* */
  int strategy;         /* NHMF_ON_THE_FLY or NHMF_CACHED for every apply of the solve */
  int load_steps;       /* S >= 1 */
  int first_step;       /* 1-based first load step to run (resume), default 1 */
  int last_step;        /* last load step to run, default S */
  double compression;   /* compression preset: u_z = -compression * s / S on z = 1 */
  double newton_rtol;   /* default 1e-8 */
  int newton_max_iter;  /* per load step, default 20 */
  int max_backtracks;   /* halvings of the Newton step on det F <= 0, default 8 */
  double linear_rtol;   /* default 1e-6 (relative to ||b||) */
  int linear_max_iter;  /* default 20000 */
  double inner_rtol;    /* mixed: FP32 inner CG relative tolerance, default 1e-3 */
  int inner_max_iter;   /* mixed: FP32 inner CG iteration cap, default 1000 */
  int check_every;      /* iterations between host convergence reads, default 10 */
  int record_pairs;     /* with a U-Net, store training pairs in the network's pair store
                           (default 0): JACOBI_CG, Newton (b, du) and CG (r_j, x* - x_j);
                           MIXED_GMG, the pairs of MIXED_GMG_LEARNED's correction,
                           (r_j - A V(r_j), x* - x_j - V(r_j)), at the first k FCG iterations
                           of each linear solve (k = cg_pair_every) */
  int cg_pair_every;    /* JACOBI_CG: pairs at iterations j = k, 4k, 16k (k = this), default 8 */
  int learned_stall_window;     /* learned solvers: fall back to Jacobi-CG when the residual */
  double learned_stall_factor;  /* drops by less than this factor over this many iterations
                                   (defaults 10 and 0.9), or after linear_max_iter/4 iterations */
  int synthetic_pairs;  /* with record_pairs: per Newton iterate, also store this many pairs
                           (K(u) e, e) for random fields e at one lattice scale each (from
                           the coarsest lattice to nodal white noise), default 0 */
  unsigned long long seed;      /* counter-based generator seed of those fields, default 1 */
  int smoother_degree;          /* GMG: Chebyshev steps per pre-/post-smoothing, default 3 */
  double smoother_range;        /* GMG: lmax / lmin of the Chebyshev interval, default 15 */
  int outer_apply;              /* arithmetic of the FP64 outer applies of the flexible solvers
                                   (every solver but JACOBI_CG): NHMF_FP64 (default) or NHMF_DF64,
                                   the FP64-accurate double-float apply on the FP32 pipe (cached
                                   strategy only; its point cache is built at each Newton
                                   linearisation).  Residuals, right-hand sides and the reported
                                   true residual stay native FP64. */
} nhmf_solve_opts;

typedef struct {
  int steps_done;
  int newton_iters[NHMF_MAX_STEPS];
  long long linear_iters[NHMF_MAX_STEPS];  /* outer Krylov iterations (FP64 applies) */
  long long inner_iters[NHMF_MAX_STEPS];   /* FP32 inner iterations (mixed) */
  int fallbacks[NHMF_MAX_STEPS];           /* learned: linear solves that fell back */
  double rel_residual[NHMF_MAX_STEPS];     /* final ||b|| / ||b_0|| of each step */
  double seconds[NHMF_MAX_STEPS];
  long long total_linear_iters, total_inner_iters;
  double total_seconds;
} nhmf_solve_stats;

/* Fill `opts` with the defaults listed above (solver JACOBI_CG, strategy CACHED, S = 1). */
void nhmf_solve_opts_default(nhmf_solve_opts* opts);

/* Run load steps first_step..last_step of Newton's method on the context's problem.  u
 * (device, FP64, 3*M^3) holds the initial state (the converged state of step first_step-1)
 * and receives the result; the linearisation point ends at the final u.  Allocates the
 * solver's work vectors in the context on first use.  Synchronises.  Returns
 * NHMF_ERR_NOT_CONVERGED if a load step misses its tolerance, NHMF_ERR_NONPOS_J if
 * backtracking cannot keep det F > 0, NHMF_ERR_BREAKDOWN on p^T A p <= 0. */
nhmf_status nhmf_solve(nhmf_ctx* ctx, const nhmf_solve_opts* opts, double* u, nhmf_solve_stats* stats,
                       void* stream);

/* Solve A(u) x = b at the current linearisation point with opts->solver, from x = 0, to
 * ||b - A x|| <= opts->linear_rtol ||b||.  b, x: device FP64, 3*M^3.  `iters` receives the
 * outer iterations, `inner_iters` the FP32 inner ones, `rel_res` the final relative
 * residual (recomputed with an FP64 apply).  Synchronises. */
nhmf_status nhmf_linear_solve(nhmf_ctx* ctx, const nhmf_solve_opts* opts, const double* b, double* x,
                              long long* iters, long long* inner_iters, double* rel_res, void* stream);

/* FP64 Jacobi-CG solve of A(u) x = b that allocates no memory (the paper has no
 * counterpart; this is a deployment variant of nhmf_linear_solve with solver
 * NHMF_SOLVER_JACOBI_CG).  For callers that cannot allocate device memory once running:
 * code whose device memory is owned by a pool or budget, loops that must avoid the
 * implicit device synchronisation of cudaMalloc/cudaFree, or hosts that forbid allocation
 * after start-up.  The context must already exist and hold a linearisation point (and an
 * FP64 point cache for NHMF_CACHED); both of those may allocate, at set-up time.
 *   Scratch: one file-scope device array of 6.3 MB (six FP64 vectors of up to 131,072
 *   entries, reduction partials, scalars).  nhmf_create looks up its device address
 *   (cudaGetSymbolAddress) on the first context of each device, with that device current,
 *   which loads the array there; it stays until the process exits.  A call must run with
 *   the context's device current (NHMF_ERR_STATE otherwise).  Problems with more than
 *   131,072 DoFs are rejected with NHMF_ERR_ARG and a message naming the limit.
 *   Every call shares the array and it keeps the last call's contents (the call clears
 *   what must start at zero): calls that overlap on the GPU, from any context or stream,
 *   race and must be serialised by the caller.
 * Arguments: strategy NHMF_ON_THE_FLY or NHMF_CACHED; rtol > 0 relative to ||b||; max_iter
 * >= 1; b, x distinct device FP64 arrays of 3*M^3 (x == b is NHMF_ERR_ARG); iters and
 * rel_res (the true relative residual, recomputed with an FP64 apply) are host outputs.
 * Synchronises. */
nhmf_status nhmf_linear_solve_noalloc(nhmf_ctx* ctx, int strategy, double rtol, int max_iter, const double* b,
                                      double* x, long long* iters, double* rel_res, void* stream);

/* ------------------------------------------------------------------ learned preconditioner
 * A 3-level convolutional U-Net on the nodal grid (16 channels, 3x3x3 convolutions, ReLU,
 * stride-2 down and transposed-convolution up paths with additive skips; 3 input and 3
 * output channels = the displacement components), BF16 weights and activations with FP32
 * accumulation on the tensor cores (tcgen05 for the stride-1 and transposed stride-2
 * convolutions, mma.sync for the stride-2 down convolution and the weight gradients), FP32
 * master weights trained by Adam.  It maps a
 * residual r (scaled to unit RMS) to a correction; as a preconditioner z = N(r) scaled back
 * and zeroed on constrained DoFs.  Requires p*N divisible by 4 and at most 784.
 * Parameters: a flat FP32 array, layer by layer (in, e0, d1, e1, d2, m2, u1, t1, u0, t0,
 * out), each weight tensor then its bias; conv/down weights W[out][in][3][3][3], up
 * weights U[in][out][3][3][3] (taps ordered dz, dy, dx from -1).
 * Pair store: each pair is the normalised input and target, FP32 [2][3][M^3]. */
nhmf_status nhmf_unet_create(nhmf_ctx* ctx, int pair_capacity);           /* allocates; sync */
size_t nhmf_unet_num_params(const nhmf_ctx* ctx);
int nhmf_unet_num_pairs(const nhmf_ctx* ctx);
/* Copy the flat parameters from / to host memory (n must equal num_params); set resets
 * the Adam moments.  Synchronous. */
nhmf_status nhmf_unet_set_params(nhmf_ctx* ctx, const float* host_params, size_t n);
nhmf_status nhmf_unet_get_params(nhmf_ctx* ctx, float* host_params, size_t n);
/* y = N(x) for device FP32 planar x, y of 3*M^3 (no scaling, no masking).  Asynchronous. */
nhmf_status nhmf_unet_forward(nhmf_ctx* ctx, const float* x, float* y, void* stream);
/* Loss ||f (N(x) - e)||^2 / ||f e||^2 (f = 1 on free DoFs) and its gradient with respect to
 * the parameters (copied to grads_host if not null).  Synchronises. */
nhmf_status nhmf_unet_loss_grad(nhmf_ctx* ctx, const float* x, const float* e, double* loss, float* grads_host,
                                void* stream);
/* z = preconditioner(r) for device FP64 r, z (3*M^3).  Asynchronous. */
nhmf_status nhmf_unet_precondition(nhmf_ctx* ctx, const double* r, double* z, void* stream);
/* Append the pair (r / rms(r), e / rms(e)) to the pair store (dropped when full). */
nhmf_status nhmf_unet_record_pair(nhmf_ctx* ctx, const double* r, const double* e, void* stream);
/* `epochs` passes of Adam (learning rate lr) over the stored pairs in order, one pair per
 * step; returns the mean loss of the first and of the last epoch.  Synchronises. */
nhmf_status nhmf_unet_train(nhmf_ctx* ctx, int epochs, double lr, double* loss_first, double* loss_last,
                            void* stream);

/* Kernel timing.  While enabled, every operator call records a CUDA event pair on its
 * stream around its element kernels (FP64 and double-float: the eight colour launches, not the
 * vector memset or the Dirichlet-row fix; FP32: the element-local launch and the node gather).  nhmf_profile_read() synchronises those events, returns the summed
 * elapsed milliseconds and the number of element-kernel launches recorded for one operator
 * kind (NHMF_KIND_*), and clears that kind's record. */
enum { NHMF_KIND_APPLY = 0, NHMF_KIND_CACHE = 1, NHMF_KIND_RESIDUAL = 2, NHMF_KIND_DIAGONAL = 3 };
nhmf_status nhmf_profile_enable(nhmf_ctx* ctx, int enable);
nhmf_status nhmf_profile_read(nhmf_ctx* ctx, int kind, double* elapsed_ms, long long* launches);

/* Measured FMA throughput of the current device in TFLOP/s (FMA = 2 FLOP) for precision
 * NHMF_FP64 or NHMF_FP32: the ALU roofline denominator of the apply kernels (not an operation
 * of the paper).  Independent FMA chains in every thread of 8 blocks of 256 threads per SM,
 * best of three timed launches after one warm-up (CUDA events).  Allocates and frees a few
 * bytes; synchronises the device. */
nhmf_status nhmf_measure_fma_peak(int precision, double* tflops);

/* ------------------------------------------------------------------ diagnostics
 * Fault injection on the host: the solvers' failure paths, exercised without a device fault.
 * Flags, OR-able; each applies to the next call where it can act and then clears itself:
 *   NHMF_INJECT_NAN_DU        the next Newton update of nhmf_solve carries a NaN: the trial
 *                             residual reports it, and nhmf_solve returns NHMF_ERR_NONFINITE
 *                             with u as after the last accepted update;
 *   NHMF_INJECT_CG_STALL      the preconditioner of the next flexible Krylov solve (mixed,
 *                             multigrid and learned solvers) returns z = 0 throughout: the
 *                             solve breaks down and finishes with Jacobi-CG (one fallback);
 *   NHMF_INJECT_UNET_GARBAGE  the next learned solve replaces every network output with a
 *                             fixed pseudo-random field: the solve stalls and falls back to
 *                             Jacobi-CG (the correction on the V-cycle instead takes a step
 *                             near zero and converges without it).
 * nhmf_create also takes flags from the environment variable NHMF_INJECT, a comma-separated
 * list of nan_in_du, cg_stall, unet_garbage. */
enum {
  NHMF_INJECT_NAN_DU = 1,
  NHMF_INJECT_CG_STALL = 2,
  NHMF_INJECT_UNET_GARBAGE = 4,
  NHMF_INJECT_UNKNOWN = 1 << 30
};
nhmf_status nhmf_set_inject(nhmf_ctx* ctx, unsigned flags);
/* The injection flags still pending (a flag clears when it fires). */
unsigned nhmf_inject_pending(const nhmf_ctx* ctx);
/* Flags of a spec in the NHMF_INJECT syntax (NULL or "" gives 0); NHMF_INJECT_UNKNOWN is set
 * when a name is not recognised.  Host only: needs no device. */
unsigned nhmf_parse_inject(const char* spec);

/* Metrics: with a path set, calls append one JSON object per line to that file - one per
 * Newton iteration and one per load step of nhmf_solve, one per nhmf_linear_solve, and one per
 * nhmf_tangent_apply (which then synchronises to time itself with CUDA events).  Every object
 * has "event"; the other keys name their units (seconds, ms, GDoF/s) or are counts and
 * relative residuals.  NULL or "" closes the file.  nhmf_create also opens the file named by
 * the environment variable NHMF_METRICS_JSONL.  NVTX ranges (apply, residual, diagonal,
 * set_linearization, solve, load step, Newton iteration, linear solve, U-Net training) are
 * always emitted; without a profiler attached they cost a function call each. */
nhmf_status nhmf_set_metrics_log(nhmf_ctx* ctx, const char* path);

#ifdef __cplusplus
}
#endif

#endif /* NHMF_H */
