/*
 * nrs.h -- C ABI of libnrs, the GB300 (sm_103a) implementation of the
 * nearest-neighbour (NEAREST) regularized stokeslet method of Gallagher &
 * Smith, "Passively parallel regularized stokeslets".
 *
 * One time step of the swimming problem (Sec. 4) is:
 *   kinematics  -> nearest neighbours (Sec. 3, the argmin defining n-hat)
 *   -> segments of nu -> assembly of A_s (Sec. 3, eq. nnrsbie; Sec. 4 step 1)
 *   -> rigid-body border (Sec. 4 step 2) -> factor + solve (Sec. 4 step 3)
 *   -> state update of Y = [X0; B] (Sec. 4).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Every pointer argument is owned by the caller.  "device" pointers are CUDA
 *   device memory on the context's device; "host" pointers are ordinary host
 *   memory.  Nothing is retained after a call returns, except where stated.
 * - Points are rows of 4 doubles: force points (x, y, z, 0), quadrature
 *   points (x, y, z, w) with w the quadrature (area) weight.  Bodies occupy
 *   contiguous ranges given by n_off / q_off.
 * - Unknowns and rows: 3m+j for force point m (all bodies) and component j,
 *   then 6 per free body in body order: columns [U(3), Omega(3)], rows
 *   [force balance(3), moment balance(3)].  n = 3 N + 6 F.
 * - Matrices are column-major with leading dimension lda >= n.
 * - All work is enqueued on the context's stream and is asynchronous unless a
 *   host output is requested.  Argument errors are detected before any work is
 *   enqueued and leave outputs untouched.  Device-detected failures (no
 *   convergence, non-finite values, a bounded device wait that ran out) are
 *   recorded in a device status word and returned by the next call that
 *   synchronises (nrs_solve with a report, nrs_step with a report,
 *   nrs_sync).
 * - No call aborts, traps or throws.  Errors return a negative nrs_status;
 *   nrs_last_error() gives a message.
 */
#ifndef NRS_H
#define NRS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    NRS_OK = 0,
    NRS_EINVAL = -1,      /* bad argument (size, null pointer, layout)     */
    NRS_ENOMEM = -2,      /* device allocation failed                      */
    NRS_ECUDA = -3,       /* CUDA runtime error                            */
    NRS_ESINGULAR = -4,   /* exactly zero pivot in the factorisation       */
    NRS_ENOCONV = -5,     /* refinement did not reach the tolerance        */
    NRS_ENONFINITE = -6,  /* NaN/Inf met in the matrix or the iterates     */
    NRS_ETIMEOUT = -7     /* a bounded device-side wait ran out            */
} nrs_status;

/* Precision of the LU factor used as the preconditioner. */
typedef enum {
    NRS_FP64 = 0,  /* plain path: FP64 factor                                     */
    NRS_FP32 = 1,  /* FP32 explicit inverse (Gauss-Jordan), updates on FP32 CUDA cores */
    NRS_TF32 = 2,  /* FP32 explicit inverse, updates on the tensor cores (TF32)       */
    NRS_BF16 = 3   /* reserved: no BF16 factorisation is built; nrs_create and nrs_factor
                      reject it with NRS_EINVAL */
} nrs_prec;

/* Body kinds (Sec. 4: swimmers are free; walls are static). */
enum { NRS_FREE = 0, NRS_PRESCRIBED = 1, NRS_STATIC = 2 };

typedef struct nrs_ctx nrs_ctx;

/* Problem description, read only during nrs_create (host memory). */
typedef struct {
    int32_t nbodies;
    const int64_t *n_off;  /* host [nbodies+1]: force-point ranges per body      */
    const int64_t *q_off;  /* host [nbodies+1]: quadrature-point ranges per body */
    const int32_t *kind;   /* host [nbodies]: NRS_FREE / NRS_PRESCRIBED / NRS_STATIC */
    const int32_t *rigid;  /* host [nbodies] or NULL: 1 if the body-frame shape never changes
                              (its nearest-neighbour map is then computed once and kept) */
    const double *U;       /* host [nbodies*3] or NULL: prescribed translation velocity */
    const double *Omega;   /* host [nbodies*3] or NULL: prescribed angular velocity     */
    double eps;            /* regularisation parameter epsilon (> 0)  */
    double mu;             /* viscosity (> 0)                         */
    int32_t nn_global;     /* 0: nearest neighbour per body in the body frame;
                              1: over all force points in the lab frame */
    int32_t factor_prec;   /* nrs_prec used by nrs_step                */
    int32_t nb;            /* LU block size (0 = default 64; 32/64/128) */
    double tol;            /* refinement stops when ||dx||_inf <= tol ||x||_inf, or when the
                              next correction, predicted from the observed rate, is far
                              below that (0 = 1e-12) */
    int32_t max_outer;     /* refinement steps (0 = 20)          */
    int32_t max_inner;     /* GMRES iterations per step (0 = 30) */
    int32_t reuse_factor;  /* nrs_step: 0 = factor at every stage; 1 = keep the factor (the
                              FP32 inverse or the FP64 LU) across stages as the preconditioner
                              and refactor only when the previous solve needed more than
                              reuse_max_inner GMRES iterations or after reuse_max_stages
                              stages.  The FP64 residual always uses the current matrix. */
    int32_t reuse_max_inner;   /* 0 = 8  */
    int32_t reuse_max_stages;  /* 0 = 16 */
    int32_t warm_start;    /* nrs_step: start each solve from the previous stage's solution */
    int32_t solve_mode;    /* 0: with an explicit-inverse factor (FP32/TF32) and max_inner <= 64,
                              the whole refinement of one right-hand side is one cooperative
                              launch (no host round trip inside a solve); 1: host-driven loop
                              (one synchronisation per GMRES iteration), the FP64 path's mode */
    double inner_tol;      /* GMRES tolerance of each refinement step, relative to the
                              preconditioned residual (0 = 1e-4).  Very ill-conditioned
                              systems need a tighter one: the preconditioned residual then
                              says little about the true residual. */
    int32_t factor_input;  /* the FP32 matrix the mixed-precision factorisation inverts:
                              0 = evaluated in FP32 (differences x_m - X_q in FP64), so the
                              factorisation starts at once while the FP64 assembly runs on a
                              low-priority stream beside it; 1 = the FP64 entries rounded to
                              FP32 (one FP64 pass first).  Very ill-conditioned systems (kappa
                              near 1/u_fp32^2) need 1: the FP32 evaluation's extra error then
                              spoils the preconditioner. */
    int32_t graph;         /* 1: nrs_step records the whole step into a CUDA graph and replays it
                              (from the second call on: the first call builds the nearest-
                              neighbour maps of the rigid bodies).  The recording is keyed by
                              the six shape pointers, dt and whether a report is asked for; a
                              call with another key records again, so callers reuse the same
                              shape buffers.  Needs factor_prec FP32/TF32, solve_mode 0,
                              reuse_factor 0, max_inner <= 64 (else nrs_create returns
                              NRS_EINVAL); the learned start and phase timing run the step
                              without the graph.  backward_err is reported as computed in the
                              graph. */
    int32_t factor_schedule; /* FP32/TF32 factorisation (Gauss-Jordan explicit inverse):
                              0 = automatic: as 4 with TF32 from n = 8192 on, else as 2;
                              1 = with TF32 on a device with tensor memory, the whole
                              inversion as ONE cooperative launch taking every SM (the chain
                              of diagonal inverses on one CTA, the updates on the others,
                              hand-offs by counters in global memory), else as 2; 2 = one
                              level of 64-column blocks, separate kernels on three streams
                              (the chain of diagonal inverses on one of them); 1 and 2 give
                              the same result bit for bit; 3 = two levels (TF32, n >= 512):
                              256-column blocks whose column panel is eliminated in 64-column
                              steps, then one rank-256 tensor-core update of the rest of the
                              matrix (a persistent tcgen05 kernel) from split-TF32 operands
                              (hi hi + hi lo + lo hi, kind::tf32); 4 = as 3 with the update's
                              operands as FP16 pairs (kind::f16: twice the tensor rate and
                              half the operand bytes of TF32), every operand row scaled by a
                              power of two that puts its largest entry in [2^14, 2^15) and
                              unscaled exactly in the update.  Other values: NRS_EINVAL. */
    int32_t residual;      /* the refinement's residual b - A x: 0 = to about u^2 (every
                              product's rounded value summed exactly as a fixed-point
                              integer, the products' rounding errors in FP64, rounded once
                              at the end; see nrs_residual): the residual precision of
                              three-precision GMRES-IR, which reaches working accuracy in
                              the solution up to kappa(A) ~ 1/u; 1 = plain FP64 (the
                              solution is then only accurate to about kappa(A) u) */
    int32_t arnoldi;       /* the matrix-vector products A v of the GMRES iterations inside
                              the refinement (the one-launch mode, solve_mode 0): 0 = with the
                              FP64 matrix (FP64 pipe); 1 = with a float-pair copy of A
                              (hi = fl32(a), lo = fl32(a - hi), about 48 bits) that the
                              assembly writes beside the FP64 matrix (8 more bytes per entry
                              on the device), in double-float arithmetic on the FP32 pipe.
                              The residual always uses the FP64 matrix, so the answer keeps
                              its accuracy; the products' relative error (about 2^-46) only
                              slows the refinement where kappa(A) 2^-46 is not small.  Other
                              values: NRS_EINVAL. */
} nrs_problem_desc;

typedef struct {
    int32_t outer;          /* refinement steps taken                         */
    int32_t inner;          /* total GMRES iterations                         */
    int32_t converged;      /* 1 if the tolerance was met                     */
    int32_t status;         /* nrs_status of the device status word           */
    double backward_err;    /* ||b - A x||_inf / (||A||_inf ||x||_inf + ||b||_inf) */
    double last_update;     /* ||dx||_inf / ||x||_inf of the last step         */
} nrs_solve_report;

typedef struct {
    nrs_solve_report stage[2];
    double ms_total;        /* device time of the step (CUDA events)          */
    int32_t factorizations; /* factorisations done in this step (0..2)        */
    int32_t start[2];       /* start of each stage's refinement: 0 = M^{-1} b (cold),
                               1 = the previous stage's solution (warm_start),
                               2 = the MLP prediction (nrs_mlp_config)          */
    double mlp_rel_err;     /* relative RMS error sqrt(sum (y - t)^2 / sum t^2) of the
                               MLP on the targets of the step's last training stage,
                               before that stage's updates (a held-out error);
                               -1 if the step did not train                     */
    int32_t retried[2];     /* 1 if the stage's refinement did not converge and the stage
                               was factored again (see nrs_step) and solved again */
} nrs_step_report;

/* Body-frame inputs of one stage (device memory):
 *   xi    [N*4]  force points (x,y,z,0) in each body's frame
 *   Xiw   [Q*4]  quadrature points (x,y,z,w) in each body's frame
 *   xidot [N*4]  prescribed deformation velocity of the force points, body frame */
typedef struct {
    const double *xi;
    const double *Xiw;
    const double *xidot;
} nrs_shapes;

/* Create a context for one problem on the current CUDA device; all work is
 * enqueued on ``stream`` (a cudaStream_t, NULL = legacy default stream).
 * Allocates every device workspace (matrices of n x n in FP64 and in the
 * factor precision, pivots, Krylov basis).  Returns NRS_EINVAL for an empty
 * body table, non-increasing offsets, a body with quadrature points but no
 * force points, eps <= 0 or mu <= 0; NRS_ENOMEM if the workspaces do not fit. */
nrs_status nrs_create(nrs_ctx **out, const nrs_problem_desc *desc, void *stream);

/* Release every device workspace of the context (synchronises its stream). */
nrs_status nrs_destroy(nrs_ctx *ctx);

/* Message of the last failed call on this context ("" if none). */
const char *nrs_last_error(const nrs_ctx *ctx);

/* Problem sizes: N force points, Q quadrature points, F free bodies, n unknowns. */
nrs_status nrs_sizes(const nrs_ctx *ctx, int64_t *N, int64_t *Q, int64_t *F, int64_t *n);

/* Rigid-body state Y = [X0; B] (Sec. 4) per body: x0 [nbodies*3], B
 * [nbodies*9] row-major with the body basis vectors as columns.  Host
 * pointers.  nrs_set_state copies in; nrs_get_state synchronises and copies out. */
nrs_status nrs_set_state(nrs_ctx *ctx, const double *x0, const double *B);
nrs_status nrs_get_state(nrs_ctx *ctx, double *x0, double *B);

/* External force and moment on each free body (host [F*6], NULL = zero),
 * the right-hand side of the force/moment balance rows. */
nrs_status nrs_set_external(nrs_ctx *ctx, const double *ext);

/* Kinematics (Sec. 4): lab-frame clouds x = x0 + B xi, X = x0 + B Xi (w
 * copied) from the context's state, and the right-hand side b: for force
 * point m of body b, B xidot_m, plus U + Omega x (x_m - x0) for a prescribed
 * body, zero for a static one; then the external force/moment per free body.
 * Outputs (device): x [N*4], Xw [Q*4], b [n]. */
nrs_status nrs_kinematics(nrs_ctx *ctx, const nrs_shapes *shapes, double *x, double *Xw,
                          double *b);

/* Nearest neighbours (Sec. 3, n-hat(q) = argmin_n |x[n] - X[q]|) and the
 * segments of nu.  x [N*4], Xw [Q*4] device; per body (nn_global = 0) the
 * search runs over the body's own force points, otherwise over all of them.
 * Ties go to the lowest index: the decision is taken on the FP64 value
 * ((dx*dx + dy*dy) + dz*dz) after an FP32 filter with a proven margin, so the
 * indices equal those of an exhaustive FP64 search bit for bit.
 * Outputs (device, each may be NULL): nn [Q] (global force index),
 * seg_ptr [N+1] and perm [Q] (quadrature points of segment n, ascending q,
 * at perm[seg_ptr[n] .. seg_ptr[n+1])).  The context keeps the segments for
 * nrs_assemble. */
nrs_status nrs_nearest_build(nrs_ctx *ctx, const double *x, const double *Xw, int32_t *nn,
                             int32_t *seg_ptr, int32_t *perm);

/* Assembly (Sec. 3 eq. nnrsbie; Sec. 4 steps 1-2) from lab-frame x [N*4] and
 * Xw [Q*4] (device) with the segments of the last nrs_nearest_build:
 *   A[3m+j, 3n+k] = (1/(8 pi mu)) sum_{q in seg(n)} S^eps_jk(x_m - X_q) w_q,
 *   S^eps_jk(r) = (delta_jk (|r|^2 + 2 eps^2) + r_j r_k) / (|r|^2 + eps^2)^{3/2},
 * then the rigid-body border of every free body (columns -I and [x_m - x0]x,
 * rows W_n I and [R_n]x with W_n = sum_{seg n} w_q, R_n = sum_{seg n} w_q (X_q - x0)).
 * The FP64 matrix is kept in the context; if A64 is not NULL it is also
 * copied there (device, column-major, lda >= n). */
nrs_status nrs_assemble(nrs_ctx *ctx, const double *x, const double *Xw, double *A64,
                        int64_t lda);

/* Factor the assembled matrix in precision ``prec`` (Sec. 4 step 3).
 * NRS_FP64: block LU of the FP64 matrix with row pivoting inside each 64 x 64
 * diagonal block.  NRS_FP32/TF32: explicit inverse of an FP32 copy by
 * blocked Gauss-Jordan elimination (pivoting inside each diagonal block),
 * which preconditions the FP64 refinement of nrs_solve.
 * info (host, may be NULL) receives 0 or the 1-based column of the first
 * exactly-zero pivot; that case also returns NRS_ESINGULAR.  Synchronises
 * when info is requested.  Every device-side wait of the factorisation (the
 * pivot-step slots of the diagonal-block inverse, the counters of the fused
 * schedule) is bounded: one that runs out sets the context's status word,
 * returned as NRS_ETIMEOUT by the next nrs_sync or solve report. */
nrs_status nrs_factor(nrs_ctx *ctx, int32_t prec, int32_t *info);

/* Solve A x = b (device b, x [n*nrhs], column-major) by GMRES-based iterative
 * refinement (Carson & Higham 2018): residual b - A x with the FP64 matrix
 * (nrs_residual), correction by GMRES preconditioned with the factor, x += d.
 * x0 (device [n*nrhs] or NULL) is the starting guess, else x0 = LU^{-1} b.
 * report (host, may be NULL; one per right-hand side) synchronises and
 * returns the device status (NRS_ENOCONV when max_outer steps did not reach
 * the tolerance). */
nrs_status nrs_solve(nrs_ctx *ctx, const double *b, double *x, int32_t nrhs, const double *x0,
                     nrs_solve_report *report);

/* r = b - A x with the context's FP64 matrix (that of the last assembly):
 * the residual of the refinement's outer step (Carson & Higham 2018).  With
 * desc.residual = 0 it is accurate to about u^2 ||A||_inf ||x||_inf (u =
 * 2^-53): each product A_ij x_j is rounded in FP64, the rounded products are
 * summed EXACTLY as a 192-bit fixed-point integer anchored at a power of two
 * above ||A||_inf ||x||_inf, the products' rounding errors (one fused
 * multiply-add each) are summed in FP64, and b minus the two sums is rounded
 * once.  With desc.residual = 1 it is a plain FP64 product.  b, x, r: device
 * [n] doubles; r may be b or x.  Asynchronous on the context's stream.
 * Errors: NRS_EINVAL for a NULL pointer or before the first assembly. */
nrs_status nrs_residual(nrs_ctx *ctx, const double *b, const double *x, double *r);

/* One explicit-midpoint (RK2) step of dY/dt = F(Y, t) (Sec. 4): stage 1 at
 * the shapes ``s0`` (time t), stage 2 at ``s_half`` (time t + dt/2), each
 * stage = kinematics, nearest neighbours (kept for rigid bodies), assembly,
 * factor (desc.factor_prec), solve; then dX0/dt = U, dB/dt = [Omega]x B with B
 * re-orthonormalised by modified Gram-Schmidt after each stage.  The state
 * stays on the device.  sol (device [2*n] or NULL) receives both stages'
 * solutions.  report (host or NULL) synchronises.  With an FP32/TF32 factor,
 * a stage whose refinement does not converge is factored again once -- by the
 * one-level elimination where the factor was the two-level one, else from the
 * other FP32 input (factor_input), or fresh where the factor was reused -- and
 * solved again (report->retried); NRS_ENOCONV if that fails too. */
nrs_status nrs_step(nrs_ctx *ctx, const nrs_shapes *s0, const nrs_shapes *s_half, double dt,
                    double *sol, nrs_step_report *report);

/* ---- adaptive Dormand-Prince stepping ------------------------------------
 * The paper integrates the swimming IVP dY/dt = F(Y, t), Y = [X0; B], with
 * MATLAB's ode45, the Dormand-Prince 5(4) pair with step-size control
 * (Sec. 4).  This is that integrator on the device, one stage evaluation
 * (kinematics, nearest neighbours, assembly, factor or reuse, solve, as in
 * nrs_step) per call: the caller supplies the body-frame shapes at the time
 * nrs_dp_next_time names, because the beat kinematics are an input.
 * Stage states Y_i = Y_n + h sum_j a_ij K_j (B re-orthonormalised by modified
 * Gram-Schmidt), K_i = (U, [Omega]x B) from the stage's solution; after the
 * seventh stage the error norm max_c |h sum_j (b5_j - b4_j) K_j,c| /
 * (atol + rtol max(|Y_n,c|, |Y_n+1,c|)) over the state's components decides:
 * err <= 1 accepts Y_n+1 (the seventh stage's state; its rates start the next
 * step), otherwise the step is retried; either way h <- h min(5 or 1,
 * max(0.2, 0.9 err^(-1/5))), clamped to [h_min, h_max] and to the interval's
 * end.  The context's state is the stage state during a step and Y_n+1 after
 * an accepted one.  Not in graph mode; nrs_step overwrites the integrator's
 * saved state (call nrs_dp_start again after it).  Tracers are not carried. */
typedef struct {
    double t;               /* time of the last accepted state                    */
    double h;               /* step size of the step in progress                  */
    double err;             /* error norm of the last completed trial             */
    int32_t stage;          /* next stage to evaluate (0: the first step's first) */
    int32_t accepted, rejected;  /* steps accepted and rejected so far            */
    int32_t last_accepted;  /* 1 if the last completed trial was accepted         */
    int32_t done;           /* 1 once t reached t_end                             */
} nrs_dp_info;

/* Begin an integration from the context's state at t0 to t_end with initial
 * step h0, tolerances rtol (> 0) and atol (>= 0), step bounds 0 < h_min <=
 * h_max.  NRS_EINVAL for bad arguments or a context in graph mode. */
nrs_status nrs_dp_start(nrs_ctx *ctx, double t0, double t_end, double h0, double rtol, double atol,
                        double h_min, double h_max);

/* Time at which the next nrs_dp_stage needs the body-frame shapes. */
nrs_status nrs_dp_next_time(const nrs_ctx *ctx, double *t_stage);

/* Evaluate the next stage with the shapes at nrs_dp_next_time; sol (device
 * [n] or NULL) receives the stage's solution; info (host or NULL) the
 * integrator's state after the call.  The seventh stage synchronises (the
 * error norm is read on the host).  NRS_ENOCONV when a step is rejected at
 * h_min, or a stage's refinement fails; NRS_EINVAL when no integration is in
 * progress (or it is done). */
nrs_status nrs_dp_stage(nrs_ctx *ctx, const nrs_shapes *s, double *sol, nrs_dp_info *info);

/* The integrator's state (host). */
nrs_status nrs_dp_info_get(const nrs_ctx *ctx, nrs_dp_info *info);

/* The rank-64 update of the Gauss-Jordan inverse on its own (the kernel that
 * nrs_factor runs once per 64-column block):
 *   M[i, j] -= sum_{c < 64} C[i*64 + c] * Rt[j*64 + c]      for 0 <= i, j < n,
 * M column-major (device, lda >= n), C and Rt row-major n x 64 (device, 16-byte
 * aligned).  prec = NRS_FP32 runs it on the CUDA cores, NRS_TF32 on the tensor
 * cores (tcgen05, TF32 operands, FP32 accumulation).  Enqueued on the context's
 * stream.  NRS_EINVAL for bad sizes, misaligned panels or a precision without
 * a kernel on this device. */
nrs_status nrs_rank64_update(nrs_ctx *ctx, float *M, int64_t lda, int64_t n, const float *C,
                             const float *Rt, int32_t prec);

/* Wait for the context's stream and return the device status word. */
nrs_status nrs_sync(nrs_ctx *ctx);

/* Counters since the context was created (host outputs, each may be NULL):
 * factorisations done (nrs_factor and inside nrs_step), and the solves whose
 * outcome reached the host (nrs_solve, eager nrs_step) with their total
 * refinement steps and GMRES iterations (a step replayed from a CUDA graph
 * keeps its solve statistics on the device and does not count here), and the
 * stages nrs_step factored and solved again after a refinement that did not
 * converge.  Plain reads of host state: no synchronisation. */
nrs_status nrs_counters(const nrs_ctx *ctx, int64_t *factorizations, int64_t *solves,
                        int64_t *outer, int64_t *inner, int64_t *retries);

/* Residuals b - A x that the refinement of those solves formed (host
 * outputs, each may be NULL): `exact` at the residual precision the context
 * was created with (extended, Sec. 4's three-precision refinement, or FP64),
 * `working` in working precision from the float-pair copy or the FP64 matrix
 * (formed while the normwise backward error is at least 1e-8, whether the
 * step then kept it or formed the exact one as well).  Each refinement step
 * keeps one of them, so exact + working >= the counted refinement steps.
 * Plain reads of host state: no synchronisation. */
nrs_status nrs_residual_counters(const nrs_ctx *ctx, int64_t *exact, int64_t *working);

/* Fluid velocity at field points (Sec. 3: the NEAREST boundary integral
 * evaluated off the body, the quantity the paper's particle-tracking
 * examples integrate):
 *   u(x_p) = (1/(8 pi mu)) sum_q S^eps(x_p - X_q) w_q f_{n(q)},
 * each term evaluated as the FP64 assembly evaluates it (correctly rounded
 * square root and division, no fused multiply-add), the sum over q in
 * contiguous ranges whose partial sums are added in ascending order
 * (deterministic).
 *   Xw [Q*4]  device, lab-frame quadrature points (x, y, z, w) as nrs_kinematics
 *             writes them, or NULL for those of the last nrs_step stage
 *   xp [P*4]  device, field points (x, y, z, unused)
 *   f         device, the force density: 3 values per force point (the first
 *             3N unknowns of a solution)
 *   u [P*4]   device output (u_x, u_y, u_z, 0)
 * n(q) is the nearest-neighbour map of the last nrs_nearest_build or
 * nrs_step.  NRS_EINVAL before there is one (or, with Xw NULL, before the
 * first nrs_step).  The first call with a larger P allocates the partial-sum
 * workspace (synchronises). */
nrs_status nrs_velocity(nrs_ctx *ctx, const double *Xw, const double *xp, int64_t P, const double *f,
                        double *u);

/* Passive tracers carried by the flow: nrs_step advances them with the
 * bodies by the same explicit midpoint, x_half = x + dt/2 u(x; stage 1),
 * x_new = x + dt u(x_half; stage 2), u from nrs_velocity with each stage's
 * geometry and force density.  xp: host [P*4] (x, y, z, anything; column 3
 * is kept); P = 0 removes them.  Allocates the tracer workspaces and
 * synchronises; a step recorded as a CUDA graph is recorded again. */
nrs_status nrs_set_tracers(nrs_ctx *ctx, const double *xp, int64_t P);

/* Synchronise and copy the tracers' current positions out (host [P*4]). */
nrs_status nrs_get_tracers(nrs_ctx *ctx, double *xp);

/* Largest problem nrs_nearest_build_static accepts. */
#define NRS_STATIC_MAX_N 65536       /* force points      */
#define NRS_STATIC_MAX_Q 1048576     /* quadrature points */
#define NRS_STATIC_MAX_BODIES 1024   /* bodies            */

/* Nearest neighbours and segments of nu, as nrs_nearest_build computes them
 * (same kernels, same bit-exact result), for callers that cannot allocate
 * device memory: code running inside a memory pool or arena it does not own,
 * time-critical loops where cudaMalloc would synchronise the device,
 * processes that reserved all device memory up front.  The paper has no
 * counterpart: this is a deployment variant of nrs_nearest_build.
 *
 * No context, no cudaMalloc/cudaFree, no allocating library call.  The
 * caller passes the inputs and outputs; the scratch (segment counters, the
 * block task table, the body offsets, a status word; about 0.4 MB) lives in
 * file-scope device arrays of fixed size that every GPU loading the library
 * holds until the process exits.
 *   x [N*4], Xw [Q*4]      device, as for nrs_nearest_build (body frame for
 *                          global == 0, lab frame for global != 0)
 *   nbodies, n_off, q_off  host offsets as in nrs_problem_desc
 *   nn [Q], seg_ptr [N+1], perm [Q]   device outputs
 *   status                 device int32 or NULL, caller-owned: receives, in
 *                          stream order, the call's device status word -- 0,
 *                          or 4 (non-finite input: those quadrature points get
 *                          nn < 0 and belong to no segment).  The library
 *                          cannot report it through its return value without
 *                          synchronising; read it after the stream work.
 *   stream                 cudaStream_t (NULL = legacy default stream)
 * Returns NRS_EINVAL for sizes above NRS_STATIC_MAX_N / _Q / _BODIES or bad
 * offsets, before any work is enqueued; NRS_ECUDA if a copy or clear of the
 * scratch or a launch fails.  The first call on a device looks up
 * the scratch's device address (cudaGetSymbolAddress) with that device
 * current.  Every call copies n_off and q_off from the caller's (pageable)
 * host memory with cudaMemcpyAsync, so no call may be captured into a CUDA
 * graph: a replay would read host buffers that may be gone.  Every call shares
 * the same scratch, which keeps the last call's contents (each call clears
 * what must start at zero): calls that overlap on the GPU -- on different
 * streams, or from several threads -- race and must be serialised by the
 * caller. */
nrs_status nrs_nearest_build_static(const double *x, const double *Xw, int32_t nbodies,
                                    const int64_t *n_off, const int64_t *q_off, int32_t global,
                                    int32_t *nn, int32_t *seg_ptr, int32_t *perm, int32_t *status,
                                    void *stream);

/* ---- learned starting guess -------------------------------------------------
 * The paper has no learned component: this is an extension of the refinement
 * of Sec. 4 step 3, whose start vector it predicts from the stage's geometry.
 * It never changes what the refinement converges to.
 *
 * A point-wise MLP, 17 -> 64 -> SiLU -> 64 -> SiLU -> 3 (SiLU(z) = z/(1+e^-z)),
 * maps the features of force point m of body b (body frame) to B^T f_m / F:
 *   0-2 xi_m/L, 3-5 xidot_m/V, 6 s = (m - n_off[b]) / max(1, N_b - 1),
 *   7 W_m / mean over body b of W, 8-10 one-hot kind (free, prescribed, static),
 *   11-13 B^T U / V, 14-16 B^T Omega L / V,
 * (U, Omega) = the previous stage's solution (free body), the prescribed
 * motion (prescribed body) or zero (static body); W_m = sum of the
 * quadrature weights of segment m (Sec. 3).  Scales L, V, F: given by
 * nrs_mlp_config, or taken from the first training sample as L = max |xi_m|,
 * V = max |b_m| over the force rows of the right-hand side, F = RMS of |f_m|.
 * Parameters (FP32, NRS_MLP_PARAMS): W1 [64][17] row-major, b1 [64],
 * W2 [64][64], b2 [64], W3 [3][64], b3 [3].  Loss: mean squared error over
 * points and components.  Optimiser: Adam (beta1 0.9, beta2 0.999, eps 1e-8).
 * Sums over points run in a fixed order: results are deterministic. */
#define NRS_MLP_IN 17
#define NRS_MLP_HID 64
#define NRS_MLP_OUT 3
#define NRS_MLP_PARAMS (NRS_MLP_HID * NRS_MLP_IN + NRS_MLP_HID + NRS_MLP_HID * NRS_MLP_HID + \
                        NRS_MLP_HID + NRS_MLP_OUT * NRS_MLP_HID + NRS_MLP_OUT)

/* Load the MLP state (host arrays of NRS_MLP_PARAMS floats): parameters, and
 * the Adam moments (NULL = zero) after t Adam steps (t >= 0).  The first
 * nrs_mlp_* call on a context allocates the MLP workspaces (about 1 KB per
 * force point).  NRS_EINVAL for a NULL params or t < 0. */
nrs_status nrs_mlp_set_params(nrs_ctx *ctx, const float *params, const float *adam_m,
                              const float *adam_v, int32_t t);

/* Synchronise and copy the MLP state out (host; each may be NULL): parameters,
 * Adam moments, the step count and the scales (L, V, F; zeros if not set). */
nrs_status nrs_mlp_get_params(nrs_ctx *ctx, float *params, float *adam_m, float *adam_v,
                              int32_t *t, double *scales);

/* Use the MLP inside nrs_step.  train_iters > 0: after each stage's solve,
 * that many Adam steps (learning rate lr) on the stage's features and solved
 * f.  predict != 0: each stage's refinement starts from the prediction
 * (f_m = F B y_m; (U, Omega) of the previous stage) or from the cold start
 * M^{-1} b, whichever has the smaller ||b - A x||_inf; and after a stage
 * that started from the prediction and needed more GMRES iterations than the
 * running mean of the cold-started stages plus 2, the prediction is skipped
 * for the next 8 stages.  The prediction replaces warm_start while enabled.
 * scales (host [3] or NULL): L, V, F; NULL keeps the current ones, or takes
 * them from the first training sample.  NRS_EINVAL when parameters were not
 * set, lr <= 0 with training, or prediction without scales or training. */
nrs_status nrs_mlp_config(nrs_ctx *ctx, int32_t train_iters, int32_t predict, float lr,
                          const double *scales);

/* One evaluation on caller data (device): X [npts*17] features, Y [npts*3]
 * outputs; with T [npts*3] targets also the loss (host double, may be NULL;
 * synchronises) and, if G [NRS_MLP_PARAMS] is not NULL, the gradient of the
 * loss with respect to the parameters.  1 <= npts <= N of the context. */
nrs_status nrs_mlp_eval(nrs_ctx *ctx, const float *X, const float *T, int64_t npts, float *Y,
                        float *G, double *loss);

/* One Adam step with the gradient G (device [NRS_MLP_PARAMS]). */
nrs_status nrs_mlp_adam(nrs_ctx *ctx, const float *G, float lr);

/* Features X (device [N*17]) of the shapes s (xi, xidot used) with the
 * context's state, the W_n of the last nrs_assemble and previous rigid
 * velocities vprev (device [6F] or NULL = zero); with sol (device [n]) also
 * the targets T (device [N*3]).  Needs the scales (nrs_mlp_config). */
nrs_status nrs_mlp_features(nrs_ctx *ctx, const nrs_shapes *s, const double *vprev,
                            const double *sol, float *X, float *T);

/* Start vector x0 (device [n]) from predictions Y (device [N*3]): f_m = F B y_m
 * with the context's B, then (U, Omega) = vprev (device [6F] or NULL = zero). */
nrs_status nrs_mlp_start(nrs_ctx *ctx, const float *Y, const double *vprev, double *x0);

/* ---- batches of independent problems ----------------------------------------
 * Many problems of uneven size stepped together (the paper solves one problem
 * at a time; this is how a GB300 is filled with many smaller ones).  Each
 * problem is an nrs_ctx owned by the batch, on a stream of its own.  From the
 * second nrs_batch_step on, the steps of ALL problems are recorded into one
 * CUDA graph and replayed by one cudaGraphLaunch per batch step: the problems
 * are split into K chains by longest-processing-time-first on an estimate of
 * their step time (the problems of a chain run in sequence, the chains
 * concurrently), and every refinement is one cooperative launch of G CTAs
 * with K * G at most the co-resident CTA count of that kernel.  The graph is
 * keyed by all shape pointers, dt and whether reports are asked for; reuse
 * the same shape buffers between steps to replay it. */
typedef struct nrs_batch nrs_batch;

/* Create a batch of count problems (host array of descriptions, read during
 * the call).  Every description must allow the recorded step: factor_prec
 * FP32 or TF32, solve_mode 0, reuse_factor 0, max_inner <= 64 (else
 * NRS_EINVAL); its graph field is ignored.  stream: the caller's cudaStream_t
 * (NULL = legacy default stream), on which nrs_batch_step's work is ordered.
 * Starts with K = min(count, 4) chains. */
nrs_status nrs_batch_create(nrs_batch **out, const nrs_problem_desc *descs, int32_t count,
                            void *stream);
/* Destroy the batch and all its contexts (synchronises). */
nrs_status nrs_batch_destroy(nrs_batch *b);
const char *nrs_batch_last_error(const nrs_batch *b);

/* The context of problem i, for nrs_set_state / nrs_get_state /
 * nrs_set_external / nrs_sizes.  The batch owns it: do not destroy it, and do
 * not step it on its own while the batch is in use. */
nrs_status nrs_batch_context(nrs_batch *b, int32_t i, nrs_ctx **ctx);

/* One RK2 step of every problem: s0[i], s_half[i] as for nrs_step (device
 * shapes), sol (host array of count device pointers [2 n_i], or NULL; an
 * entry may be NULL), reports (host array of count, or NULL; synchronises).
 * The first call runs the problems' steps one after the other without the
 * graph.  Returns the worst status over the problems. */
nrs_status nrs_batch_step(nrs_batch *b, const nrs_shapes *s0, const nrs_shapes *s_half, double dt,
                          double *const *sol, nrs_step_report *reports);

/* Set K (1 <= K <= count) and G (K * G <= co-resident CTAs of the solve
 * kernel) and re-plan; chain_of (host [count] or NULL) receives each
 * problem's chain.  The next step records the graph again. */
nrs_status nrs_batch_config(nrs_batch *b, int32_t chains, int32_t grid, int32_t *chain_of);

/* Autotune (K, G): time one replayed batch step for each K in {1, 2, 4, 8,
 * 16} (<= count) and G in {SMs, SMs/2, SMs/4} (capped by the co-residency
 * bound), keep the fastest.  Every trial starts from the batch's state at
 * the call, which is restored afterwards.  Needs one nrs_batch_step first.
 * cache_path (or NULL): text file of "<key> <K> <G> <ms>" lines; the key
 * names the device and the sorted problem sizes.  A cached entry is used
 * without timing (ms_out = -1); a new result is appended. */
nrs_status nrs_batch_tune(nrs_batch *b, const nrs_shapes *s0, const nrs_shapes *s_half, double dt,
                          const char *cache_path, int32_t *chains_out, int32_t *grid_out,
                          double *ms_out);

/* Current K, G and the number of kernels in the recorded graph (0 if none). */
nrs_status nrs_batch_info(const nrs_batch *b, int32_t *chains, int32_t *grid,
                          int64_t *graph_kernels);

/* Longest-processing-time-first plan on its own (host only, no device):
 * order = problems by decreasing cost (ties: lower index first), each given
 * to the chain with the least cost so far (ties: lower chain). */
nrs_status nrs_batch_plan(const double *cost, int32_t count, int32_t chains, int32_t *chain_of,
                          int32_t *order);

/* Phases of the step, as timed by nrs_get_timing. */
enum {
    NRS_PH_KINEMATICS = 0, /* body frame -> lab frame, right-hand side          */
    NRS_PH_NEAREST = 1,    /* nearest-neighbour search                          */
    NRS_PH_SEGMENTS = 2,   /* segments of nu, gather, segment moments           */
    NRS_PH_ASSEMBLE = 3,   /* the A_s assembly kernel                           */
    NRS_PH_BORDER = 4,     /* rigid-body rows and columns                       */
    NRS_PH_CONVERT = 5,    /* copy / precision conversion of A for the factor   */
    NRS_PH_LU_PANEL = 6,   /* diagonal-block factor, row exchange, triangular panels */
    NRS_PH_LU_UPDATE = 7,  /* trailing updates A22 -= L21 U12                   */
    NRS_PH_TRSV = 8,       /* triangular solves with the factor                 */
    NRS_PH_GEMV = 9,       /* FP64 residual / Arnoldi matrix-vector products    */
    NRS_PH_KRYLOV = 10,    /* orthogonalisation, Givens, updates, norms         */
    NRS_PH_UPDATE = 11,    /* explicit-midpoint state update                    */
    NRS_PH_LU_DIAG = 12,   /* next diagonal block: its update and inverse (timed on the
                              factorisation's second stream, overlapping the others) */
    NRS_PH_ASSEMBLE32 = 13, /* the FP32 copy of A_s for the factorisation (mixed path); the
                              FP64 assembly then runs on a third stream, overlapping the
                              factorisation (timed there) */
    NRS_NPHASE = 14
};

/* Enable (1) or disable (0) per-phase timing with CUDA events recorded on the
 * context's stream around each phase's kernels.  Enabling clears the totals. */
nrs_status nrs_set_timing(nrs_ctx *ctx, int32_t enable);

/* Synchronise and return the per-phase totals since timing was enabled (host
 * arrays of NRS_NPHASE: milliseconds and number of timed spans; either may be
 * NULL) and the number of kernels launched since the context was created (or
 * since timing was last enabled), then clear the totals. */
nrs_status nrs_get_timing(nrs_ctx *ctx, double *ms, int64_t *spans, int64_t *launches);

/* The timed spans since timing was enabled, in the order they were recorded,
 * as a trace: phase[i] (an NRS_PH_* value) and begin_ms[i], end_ms[i]
 * (milliseconds from the begin of the first span; spans on the factorisation's
 * side streams overlap those on the main stream).  Host arrays of `capacity`
 * entries (any may be NULL); the first min(capacity, *count) spans are
 * written and *count is set to the number recorded.  Synchronises; clears
 * nothing, so call it before nrs_get_timing. */
nrs_status nrs_get_trace(nrs_ctx *ctx, int32_t *phase, double *begin_ms, double *end_ms,
                         int64_t capacity, int64_t *count);

#ifdef __cplusplus
}
#endif

#endif /* NRS_H */
