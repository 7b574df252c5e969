/*
 * wrmg.h -- C ABI of the GB300 space-time waveform-relaxation multigrid library.
 *
 * The library solves the space-time Taylor-Hood discretisation of the
 * incompressible Navier-Stokes equations (Eq. nsfem; DG(q) in time, Def.
 * "Temporal discretisation", Eq. dgintime) on the unit square,
 *
 *     u_t + conv (u.grad) u + grad p - nu lap u = f,   div u = 0,
 *
 * with Q_{k+1}^2 / Q_k elements on a uniform n x n quadrilateral mesh and N
 * time slabs solved all at once, by inexact Newton with FGMRES preconditioned
 * by V(2,2) waveform-relaxation multigrid cycles (Sec. 3, Algorithm Vcycle).
 * The paper's form u_t + R u.grad u + grad phi - lap u = 0 is conv = R, nu = 1.
 *
 * Vectors.  Every vector argument is a caller-owned DEVICE pointer (cudaMalloc
 * or a torch CUDA tensor) to FP64 data of length wr_ndofs(ctx, level) in the
 * canonical layout
 *
 *     index = ((slab * (q+1) + a) * S + field_offset + y * nf + x)
 *
 * with S = 2 nv^2 + np^2, nv = n(k+1)+1 and np = nk+1 nodes per direction,
 * fields u_x (offset 0), u_y (offset nv^2), Phi (offset 2 nv^2), x fastest,
 * a = 0..q the temporal DoF of the slab (Lagrange basis at the right-Radau
 * points; a = q is the slab end value).  The discrete pressure Phi follows the
 * paper's sign +(Phi, div psi), i.e. it approximates minus the strong-form p.
 * Exceptions: functions ending in _host take host pointers.
 *
 * Streams.  All work is enqueued on the CUDA stream given to wr_create.  Calls
 * that return host scalars (norms, iteration counts) synchronise that stream;
 * the others only enqueue.  A context must not be used from two host threads
 * at once.
 *
 * Errors.  Every call returns a status (WR_OK on success).  No exception
 * crosses the ABI; wr_last_error returns a description of the last failure.
 * After WR_ERR_CUDA the context should be destroyed.
 *
 * Ownership.  A wr_ctx owns the level hierarchy, the linearisation point on
 * every level, the stored patch factors, the Chebyshev eigen-estimates and the
 * Krylov workspace; wr_destroy frees them.  The caller owns every vector.
 */
#ifndef WRMG_H
#define WRMG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define WR_OK 0
#define WR_ERR_ARG 1            /* invalid argument (size, level, null pointer, unsupported k/q) */
#define WR_ERR_NOMEM 2          /* device allocation failed                                     */
#define WR_ERR_CUDA 3           /* a CUDA call or kernel launch failed                          */
#define WR_ERR_NOT_CONVERGED 4  /* Newton or FGMRES reached its iteration limit                 */
#define WR_ERR_TIMEOUT 5        /* a bounded device wait gave up                                */
#define WR_ERR_NAN 6            /* a norm became NaN or Inf                                     */
#define WR_ERR_STATE 7          /* call order violated (e.g. smoother before wr_linearise)      */
#define WR_ERR_CANCELLED 8      /* a served request was cancelled (wr_server_cancel)            */

/* problem data (wr_problem.kind) */
#define WR_TAYLOR_GREEN 0  /* decaying Taylor-Green (Chorin) vortex, f = 0, exact Dirichlet data (conv = 1)  */
#define WR_POLY 1          /* manufactured u = (y^2, x^2)(1+t) (or steady), p = x+y-1, with matching f       */
#define WR_FOURIER 2       /* no-slip walls, u(0) = 0, f = sum amp_j curl(sin(mx_j pi x) sin(my_j pi y))     */
#define WR_LID 3           /* lid-driven cavity (Sec. 4): u = (1, 0) on the open top edge, 0 on the other walls
                              and the top corners, u(0) = 0, f = 0                                         */
/* The heat equation (Def. heat): u_t - nu lap u = 0, natural boundary conditions, continuous Q_k
 * (k = 1, 2, 3) x DG(q) (q = 0..3, the degrees of Sec. 5); one scalar field, canonical index
 * (slab (q+1) + a) S + y nv + x with nv = n k + 1, S = nv^2; vertex-star (open-star) patches;
 * n_coarse = 2, or 1 (required for k = 3, q = 3, whose 2x2 coarse block, 196 x 196 in FP64, does
 * not fit in shared memory; wr_create returns WR_ERR_ARG for it).  The problem is linear:
 * wr_solve with newton_maxit = 1, ew = 0 and eta_fixed = the FGMRES tolerance is the paper's
 * FGMRES-WRMG solve (Sec. 5).  Only the FP64 smoother exists for it. */
#define WR_HEAT 4          /* u(0) = sin(pi x) + cos(2 pi y) (Sec. 5)                                      */
#define WR_HEAT_EIGEN 5    /* u(0) = cos(pi x): u = exp(-nu pi^2 t) cos(pi x) exactly                      */

/* arithmetic of the stored patch factors and of the smoother (wr_options.precision) */
#define WR_FP64 0  /* FP64 factors and smoother (the plain method)                        */
#define WR_FP32 1  /* FP32 factorisation, factors and smoother                              */
#define WR_BF16 2  /* FP32 factorisation, BF16-stored factors, FP32 smoother arithmetic      */

/* the patch matrix of the Vanka+star relaxation (wr_options.patch_assembly; Sec. 3
 * defines the patch by its DoFs and leaves the matrix to the assembled operator) */
#define WR_PATCH_SUBMATRIX 0  /* A_i = J[P_i, P_i], the principal submatrix of the assembled J   */
#define WR_PATCH_LOCAL 1      /* the space-time Jacobian assembled over the patch's own 2x2
                                 cells, restricted to P_i (diagonal and subdiagonal blocks)      */
/* the additive scatter's weights (wr_options.scatter_weight) */
#define WR_WEIGHT_ONE 0           /* y = sum_i R_i^T y_i (plain additive Schwarz)               */
#define WR_WEIGHT_MULTIPLICITY 1  /* y = sum_i R_i^T (y_i / number of patches holding the DoF)  */

/* the slab factors of step (b) (wr_options.store_factors): stored at linearisation
 * and streamed by every smoother apply, or recomputed in place: every apply on a
 * recomputing level rebuilds the convection element matrices and the factors of
 * a window of recompute_slabs slabs into one shared window buffer, applies them,
 * and moves to the next window (the forward substitution carries the jump state
 * across windows).  Results are bitwise those of the stored form. */
#define WR_RECOMPUTE 0   /* every smoothed level recomputes                                      */
#define WR_STORE 1       /* every smoothed level stores                                          */
#define WR_STORE_AUTO 2  /* the fewest finest levels recompute such that the context fits
                            memory_budget_mb (wr_estimate_bytes with memory_budget_mb = 0
                            assumes every level stored)                                          */

typedef struct wr_ctx wr_ctx;

typedef struct {
    int n_fine;     /* cells per direction on the finest level (n_coarse times a power of 2) */
    int n_coarse;   /* cells per direction on the direct-solve level: 2, or 3 when k = 1
                       (heat: 1 or 2)                                                        */
    int k;          /* Taylor-Hood order: velocity Q_{k+1}, pressure Q_k; k = 1 or 2
                       (heat: Q_k, k = 1, 2, 3)                                              */
    int q;          /* DG(q) in time; q = 0 or 1 (heat: 0..3)                                */
    int n_slabs;    /* N time slabs of width T / N                                           */
    double T, nu, conv;
    int kind;       /* WR_TAYLOR_GREEN, WR_POLY, WR_FOURIER, WR_LID, WR_HEAT or WR_HEAT_EIGEN */
    int steady;     /* WR_POLY only: time-constant u = (y^2, x^2)                            */
    int n_modes;    /* WR_FOURIER: number of modes (<= 8), host arrays below                 */
    const int *mx, *my;
    const double *amp;
    double t0;      /* time at the start of slab 0: the slabs cover [t0, t0 + T] (0)           */
} wr_problem;

typedef struct {
    int precision;          /* WR_FP64 (default), WR_FP32 or WR_BF16 factors and smoother         */
    int cheb_steps;         /* Chebyshev steps per relaxation (2: V(2,2))                        */
    double cheb_lo, cheb_hi;/* Chebyshev interval [cheb_lo lam, cheb_hi lam] (0.25, 1.05)       */
    int eig_steps;          /* Arnoldi steps of the eigen-estimate (10)                         */
    double newton_rtol;     /* stop when ||F|| <= newton_rtol ||F_0|| (1e-8)                     */
    int newton_maxit;       /* (20)                                                              */
    int ew;                 /* 1: Eisenstat-Walker forcing terms; 0: fixed eta_fixed             */
    double eta_fixed;       /* (1e-4)                                                            */
    int gmres_restart;      /* (30)                                                              */
    int gmres_maxit;        /* total FGMRES iterations per Newton step (200)                     */
    int patch_assembly;     /* WR_PATCH_SUBMATRIX (default) or WR_PATCH_LOCAL                    */
    int scatter_weight;     /* WR_WEIGHT_ONE (default) or WR_WEIGHT_MULTIPLICITY                 */
    int store_factors;      /* WR_STORE (default), WR_RECOMPUTE or WR_STORE_AUTO                  */
    int recompute_slabs;    /* slabs per recompute window (0: ceil(N / 16))                      */
    int memory_budget_mb;   /* WR_STORE_AUTO: device MiB the context may take (0: 92% of the
                               device's free memory at wr_create)                              */
    int autotune;           /* 1 (default): at the first linearisation, time the smoother-apply
                               tile variants on every level's stored factors and keep the
                               fastest (cached per shape for the process); 0: fixed tiles     */
    int apply_tile;         /* -1 (default): the autotuner's (or the fixed) choice; 0 .. 4 force
                               a smoother-apply tile on every level (0-2: one CTA per patch,
                               1, 2 or 3 CTAs per SM; 3: one warp per patch; 4: one warp per
                               patch, each slab's block bulk-copied to shared memory two slabs
                               ahead (Q2/Q1 DG(0); tile 3 elsewhere))                         */
    double newton_divtol;   /* stop (WR_ERR_NOT_CONVERGED) once ||F|| > newton_divtol ||F_0|| (1e6; 0: never) */
    int newton_stall;       /* stop once FGMRES has used gmres_maxit in this many consecutive
                               Newton steps (3; 0: never)                                     */
    int time_parallel;      /* parallel-in-time patch solve (Sec. 5's partitioned forward
                               substitution): 1 on the smoothed levels whose patches fill at
                               most half of the GPU, 2 on every stored level (4 chunks), 0
                               (default) off.  Each level's slabs split into chunks swept
                               at once from zero states, the chunk-boundary states chained
                               by transfer matrices built at linearisation, and the chunks
                               swept again from their incoming states                        */
} wr_options;

typedef struct {
    int newton_its;            /* Newton steps taken                                       */
    int gmres_its[64];         /* FGMRES iterations of each Newton step                    */
    double residual_norms[65]; /* ||F|| before each Newton step and at the end             */
    double setup_ms;           /* time in wr_linearise, summed                             */
    double krylov_ms;          /* time in FGMRES, summed                                   */
    int vcycles;               /* V-cycles applied                                          */
} wr_stats;

/* Fills *o with the defaults listed above. */
void wr_default_options(wr_options *o);

/* Creates a context: level hierarchy n_fine, n_fine/2, ..., n_coarse with the
 * same time mesh on every level (Sec. 3, semi-coarsening) and all device
 * storage for the stored-factor smoother.  cuda_stream is a cudaStream_t (NULL
 * = default stream).  Host arrays in *p are copied.  Errors: WR_ERR_ARG for
 * unsupported sizes, WR_ERR_NOMEM if the hierarchy does not fit. */
int wr_create(wr_ctx **out, const wr_problem *p, const wr_options *o, void *cuda_stream);
/* Device bytes wr_create would allocate for (*p, *o), without allocating. */
int wr_estimate_bytes(const wr_problem *p, const wr_options *o, int64_t *out);
int wr_destroy(wr_ctx *c);
/* Description of the last failure of context c; with c = NULL, of the last
 * failed call of this host thread that takes no context
 * (wr_apply_jacobian_static), or "null context" if there was none. */
const char *wr_last_error(const wr_ctx *c);

/* Levels are numbered 0 (coarsest, n_coarse) .. L (finest). */
int wr_num_levels(const wr_ctx *c, int *out);
int wr_ndofs(const wr_ctx *c, int level, int64_t *out);
/* Bytes of device memory the context holds. */
int wr_device_bytes(const wr_ctx *c, int64_t *out);
/* Smoothed level (1 .. num_levels - 1): *stored = 1 if its factors are stored,
 * 0 if recomputed per apply; *window_slabs = the slabs per recompute window (N when stored). */
int wr_factor_storage(const wr_ctx *c, int level, int *stored, int *window_slabs);
/* The smoother-apply tile of a smoothed level chosen by the autotuner (0 .. 2), or -1
 * before the first linearisation or with autotune = 0 (the fixed tile of k is used). */
int wr_apply_tile(const wr_ctx *c, int level, int *variant);

/* Global indices (host array, capacity >= 2 (2k+3)^2 (q+1) + (2k-1)^2 (q+1))
 * of Vanka+star patch `patch` (= J (n+1) + I for vertex (I, J)) on `slab` of
 * `level` (Sec. 3, NS relaxation; Fig. patches): velocity DoFs in the closure of
 * the 2x2-cell vertex star, pressure DoFs of the open star, each at every
 * temporal DoF of the slab; order: temporal DoF a, then u_x nodes (y-major),
 * u_y nodes, pressure nodes; Dirichlet nodes dropped. *len receives the count. */
int wr_patch_dofs(const wr_ctx *c, int level, int64_t patch, int slab, int64_t *idx_host, int *len);

/* U = Dirichlet data g at every temporal node on the boundary, zero elsewhere. */
int wr_initial_guess(wr_ctx *c, double *U);

/* F = F(U), the nonlinear space-time residual of Eq. nsfem on the finest level
 * (Dirichlet rows: U - g).  Sum-factorised, matrix-free, FP64. */
int wr_residual(wr_ctx *c, const double *U, double *F);

/* Linearises about W (finest level): injects W to every coarser level,
 * assembles and factors every (patch, slab) block A_nn = J(W)[P_i, P_i] of the
 * waveform patch systems (Eq. waveform_patch_solve; principal submatrices of
 * the assembled space-time Jacobian), factors the coarse slab blocks and runs
 * the 10-step Arnoldi eigen-estimate of M^{-1} J on every smoothed level. */
int wr_linearise(wr_ctx *c, const double *W);
/* Same without the eigen-estimates (they keep their previous values). */
int wr_linearise_no_eig(wr_ctx *c, const double *W);
int wr_get_lambda(const wr_ctx *c, int level, double *lam);
int wr_set_lambda(wr_ctx *c, int level, double lam);

/* y = J(W_level) x: the Newton linearisation of Eq. nsfem about the level's
 * linearisation point, with Dirichlet rows and columns replaced by the
 * identity.  Sum-factorised matrix-free FP64 (kernel (e)). x and y must not alias. */
int wr_apply_jacobian(wr_ctx *c, int level, const double *x, double *y);

/* y = M^{-1} r = sum_i R_i^T A_i^{-1} R_i r: the waveform Vanka+star relaxation
 * (per-patch gather, forward substitution over slabs with the stored slab
 * factors, additive scatter).  level >= 1.  r and y must not alias. */
int wr_patch_apply(wr_ctx *c, int level, const double *r, double *y);

/* One relaxation: cheb_steps Chebyshev steps for J x = b preconditioned by
 * wr_patch_apply; zero_guess != 0 ignores (and overwrites) x. level >= 1. */
int wr_smooth(wr_ctx *c, int level, const double *b, double *x, int zero_guess);

/* xc = R xf = P^T xf from level fine_level to fine_level - 1 (Sec. 3,
 * P = I (x) blockdiag(P_u, P_phi)); Dirichlet entries zero. */
int wr_restrict(wr_ctx *c, int fine_level, const double *xf, double *xc);
/* xf += P xc. */
int wr_prolong_add(wr_ctx *c, int fine_level, const double *xc, double *xf);

/* x = exact solve with level 0's J (block forward substitution over slabs,
 * pressure pinned at vertex (0, 0) per temporal DoF, then made mean-free). */
int wr_coarse_solve(wr_ctx *c, const double *b, double *x);

/* x = one V(2,2) cycle (Algorithm Vcycle) for J_fine x = b from a zero guess. */
int wr_vcycle(wr_ctx *c, const double *b, double *x);
/* The same with HOST b and x: copies b in and x out on the context stream. */
int wr_vcycle_host(wr_ctx *c, const double *b_host, double *x_host);

/* Subtracts from every temporal DoF's pressure its mean int Phi (the null
 * space of J under all-Dirichlet velocity). Works on the finest level. */
int wr_project_pressure(wr_ctx *c, double *x);

/* Newton-FGMRES-WRMG solve from U_inout (call wr_initial_guess first for the
 * standard start) until ||F|| <= newton_rtol ||F_0||.  stats may be NULL.
 * Returns WR_ERR_NOT_CONVERGED if newton_maxit is reached. */
int wr_solve(wr_ctx *c, double *U_inout, wr_stats *stats);
/* The same with a HOST U (copied in and out). */
int wr_solve_host(wr_ctx *c, double *U_host, wr_stats *stats);

/* Sets the velocity that the slab-0 jump term of the residual takes as u(t0)
 * (Eq. nsfem's U_0^-): u0 is a device spatial block of the finest level (S = 2 nv^2
 * + np^2 doubles, canonical field order; its pressure part is ignored), copied;
 * NULL restores the problem's own initial data (the exact u(t0), or zero). */
int wr_set_initial_state(wr_ctx *c, const double *u0);

/* The timestepping comparator (Sec. 5): the context must have n_slabs = 1 (one
 * time element of width T starting at the problem's t0); step i solves that
 * element moved to [t0 + i T, t0 + (i + 1) T] with Newton-FGMRES-WRMG, taking as
 * initial state the end state of step i - 1 (the last temporal DoF of its slab;
 * step 0 takes the state of wr_set_initial_state, or the problem's own data).
 * U: device array of n_steps one-slab solutions in sequence (n_steps (q+1) S
 * doubles, together the canonical layout of the n_steps-slab problem); it is
 * overwritten (each step starts from its boundary lift).  st (may be NULL):
 * newton_its, vcycles, setup_ms and krylov_ms summed over the steps;
 * gmres_its[i] = FGMRES iterations of step i and residual_norms[i] = its final
 * ||F|| (i < 64).  Returns the first failing step's status, else WR_OK; the
 * context keeps the state of the last step (wr_set_initial_state resets it). */
int wr_solve_timestepping(wr_ctx *c, int n_steps, double *U, wr_stats *st);

/* ------------------------------------------------------------------ batching
 * A wr_batch holds many independent space-time solves (uneven meshes, slab
 * counts, viscosities and forcings; one k and one q for the whole batch) and
 * advances them in lock step: every stage of the V-cycle is one launch for all
 * members (the smoother one persistent launch over every member's patches),
 * Newton and FGMRES keep per-member scalars, and members that converge leave
 * the active set.  Member vectors are caller-owned device pointers in the
 * canonical layout of that member's finest level.  The paper solves one
 * problem at a time; batching is a service of this library. */
typedef struct wr_batch wr_batch;
int wr_batch_create(wr_batch **out, int n, const wr_problem *ps, const wr_options *o, void *cuda_stream);
int wr_batch_destroy(wr_batch *b);
const char *wr_batch_last_error(const wr_batch *b);
int wr_batch_ndofs(const wr_batch *b, int member, int64_t *out);
int wr_batch_device_bytes(const wr_batch *b, int64_t *out);
/* U[m] = Dirichlet data of member m (like wr_initial_guess). */
int wr_batch_initial_guess(wr_batch *b, double *const *U);
/* Linearises every member about W[m] (factors and eigen-estimates). */
int wr_batch_linearise(wr_batch *b, double *const *W);
int wr_batch_get_lambda(const wr_batch *b, int member, int level, double *lam);
/* x[m] = one V(2,2) cycle of member m for right-hand side b[m] (all members at once). */
int wr_batch_vcycle(wr_batch *b, double *const *bin, double *const *xout);
/* One V(2,2) cycle of every member on the batch's internal right-hand side
 * (the last b given to wr_batch_vcycle); for throughput measurements. */
int wr_batch_vcycle_resident(wr_batch *b);
/* enable != 0 (the default): every batched V-cycle runs as one CUDA graph, captured
 * anew whenever the active members or the Chebyshev intervals change (the cycle's
 * kernels and arguments are the eager ones, so results are bitwise the same);
 * 0: every kernel is launched eagerly. */
int wr_batch_set_graphs(wr_batch *b, int enable);
/* Newton-FGMRES-WRMG solve of every member from U[m] (in/out); st may be NULL
 * or an array of n wr_stats.  WR_ERR_NOT_CONVERGED if any member hits newton_maxit. */
int wr_batch_solve(wr_batch *b, double *const *U, wr_stats *st);

/* ------------------------------------------------------------------ serving
 * A wr_server solves a stream of independent space-time problems.  Requests
 * wait in arrival (FIFO) order; the head request is admitted as soon as fewer
 * than max_inflight solves run and its device bytes (wr_estimate_bytes plus its
 * solution vector) fit in what remains of mem_budget_bytes.  Each admitted
 * request runs on its own host thread, CUDA stream and context (allocated on
 * admission, freed on completion), so the solves in flight overlap on the GPU
 * and a completion admits the next request at once.  Smaller requests run on
 * higher-priority streams (one level per factor 4 in DoFs), so the GPU starts their
 * kernels first when SMs free up.  A request larger than
 * the whole budget completes with WR_ERR_NOMEM.  Results are the same as a
 * wr_solve of that problem alone (deterministic kernels, per-stream state).
 * The paper solves one problem at a time; serving is a service of this library.
 *   o: the options every request is solved with (NULL: wr_default_options).
 *   The server uses the device current at wr_server_create. */
typedef struct wr_server wr_server;
int wr_server_create(wr_server **out, int64_t mem_budget_bytes, int max_inflight, const wr_options *o);
/* The same server with per-cycle batching (continuous batching): an in-flight
 * slot (max_cohorts of them) holds a cohort instead of one request.  When a slot
 * is free the head request is admitted together with the queued requests of the
 * same k and q behind it, in arrival order, up to max_members and the remaining
 * budget, and the cohort is solved as one lock-step batch (wr_batch: one launch per
 * stage of every V-cycle, Newton step and FGMRES iteration for all its members,
 * V-cycles replayed as CUDA graphs) on the slot's stream.  Cohorts in different
 * slots overlap on the device; requests that arrive meanwhile form the next cohort
 * as soon as a slot and memory free up.  Each member completes (and is pollable)
 * the moment it leaves its cohort, so its latency is its own; a cohort's memory is
 * released when its last member leaves.  Results equal the solve alone up to
 * rounding (1e-10: the apply tiles are tuned per cohort).  Heat-equation and
 * DG(2)/DG(3) requests, which the batch engine does not take, run one per slot as
 * in wr_server_create.  Cancelling a running member takes effect at its cohort's
 * next Newton step.  max_members = 1 is wr_server_create. */
int wr_server_create_batched(wr_server **out, int64_t mem_budget_bytes, int max_cohorts, int max_members,
                             const wr_options *o);
/* Waits for the solves in flight; requests still queued complete with WR_ERR_STATE. */
int wr_server_destroy(wr_server *sv);
/* Queues *p (copied, forcing modes included); U0_host is NULL (start from the
 * Dirichlet data, like wr_initial_guess) or a host iterate of the finest
 * level's length (copied).  *ticket identifies the request for wr_server_poll. */
int wr_server_submit(wr_server *sv, const wr_problem *p, const double *U0_host, uint64_t *ticket);
/* wait == 0: WR_ERR_STATE while the request is queued or running.  Once it has
 * completed (wait != 0 blocks until then): copies the host solution into U_host
 * (may be NULL), its statistics into *st and its latency, submission to
 * completion in ms, into *latency_ms (either may be NULL), forgets the ticket
 * and returns the solve's status (WR_OK, WR_ERR_NOT_CONVERGED, WR_ERR_NOMEM...).
 * Unknown tickets: WR_ERR_ARG. */
int wr_server_poll(wr_server *sv, uint64_t ticket, int wait, double *U_host, wr_stats *st, double *latency_ms);
/* Largest device bytes admitted at once and largest number of solves in flight so far
 * (cohorts, in batched mode). */
int wr_server_stats(wr_server *sv, int64_t *peak_bytes, int *peak_inflight);
/* Largest cohort solved as one batch so far (0 in per-request mode). */
int wr_server_peak_cohort(wr_server *sv, int *out);
/* Cancels a request: a queued one completes at once, a running one at its next
 * Newton step or FGMRES iteration; either way with WR_ERR_CANCELLED (poll it as
 * usual).  A completed request is unaffected.  Unknown tickets: WR_ERR_ARG. */
int wr_server_cancel(wr_server *sv, uint64_t ticket);

/* ------------------------------------------------------------------ failure detection
 * Host-side fault injection and a self-test of the device-side bounded waits; the
 * GPU is never faulted, trapped or hung.  Neither has a counterpart in the paper. */
/* The nth device allocation made by a context or batch from now on fails with
 * WR_ERR_NOMEM, as if the device were full (0 switches the injection off). */
int wr_inject_alloc_failure(int64_t nth);
/* Runs the smoother kernels' bounded wait on an mbarrier that nothing completes,
 * in a one-warp kernel on cuda_stream: *timed_out = 1 when the wait gave up (as it
 * must), *waited_ms = how long it waited (about the 2 s limit). */
int wr_selftest_bounded_wait(void *cuda_stream, int *timed_out, double *waited_ms);

/* Total kernel launches made by this library in this process (all contexts). */
int wr_launch_count(int64_t *out);

/* enable != 0 starts recording CUDA events on the context stream around every
 * launch of the smoother-apply kernel (gather + forward substitution over
 * slabs, steps (a)+(c)), per level; it clears earlier records. */
int wr_profile(wr_ctx *c, int enable);
/* Sum of the recorded smoother-apply kernel durations on `level` (ms) and the
 * number of launches recorded; synchronises the stream. */
int wr_profile_smoother(wr_ctx *c, int level, double *total_ms, int *launches);

/* y = J(W) x on the n_fine mesh that *p describes, like wr_apply_jacobian on
 * the finest level, but with no context and no device allocation: for callers
 * that cannot call cudaMalloc (an application that owns all device memory
 * through its own pool, or a latency-critical loop that must not pay for the
 * allocator's implicit synchronisation).  The paper has no counterpart; this
 * is a service of the library.
 *   W, x, y: caller-owned device pointers, canonical layout, FP64, length
 *   n_slabs (q+1) (2 nv^2 + np^2); x and y must not alias.  Of *p, n_fine, k,
 *   q, n_slabs, T, nu and conv are used, and kind is checked: it must be a
 *   Navier-Stokes kind (WR_TAYLOR_GREEN, WR_POLY, WR_FOURIER or WR_LID; the
 *   heat kinds are refused), none of which changes J.  Work is enqueued on
 *   cuda_stream, which must belong to the current device (else WR_ERR_ARG).
 * Scratch: a fixed 64 MiB array of this library's static device memory (8 Mi
 *   doubles), held by every GPU that loads the library until the process exits.
 *   Problems that need more, i.e. n_slabs n_fine^2 (q+1) (2 (k+2)^2 + (k+1)^2)
 *   > 8 Mi, are rejected with WR_ERR_ARG before any work is enqueued (other
 *   WR_ERR_ARG causes: null or aliased pointers, unsupported k, q or kind, a
 *   stream of another device).
 * The first call on a device looks up the array's device address on that device
 *   (cudaGetSymbolAddress); make that first call before any stream capture.
 * Every call shares the array: calls that overlap on the GPU (other streams,
 *   other threads) race and must be serialised by the caller.  The array keeps
 *   the last call's contents; each call writes every entry it reads first, so
 *   nothing needs clearing.
 * Returns WR_OK, WR_ERR_ARG, or WR_ERR_CUDA (launch failure); after a failure
 *   wr_last_error(NULL) describes it (per host thread). */
int wr_apply_jacobian_static(const wr_problem *p, const double *W, const double *x, double *y, void *cuda_stream);

/* Sum of the recorded durations of the J(W) x element kernel on `level` (ms; the
 * Jacobian applications of Chebyshev residuals, restricted residuals and FGMRES, timed
 * by CUDA events once wr_profile has enabled recording), the number of launches, and
 * the FP64 operations of one launch (the sum-factorised algorithm's count, a
 * multiply-add counting 2; NULL to skip).  Synchronises the stream. */
int wr_profile_jacobian(wr_ctx *c, int level, double *total_ms, int *launches, double *flops_per_launch);

/* FP64 FMA throughput of this GPU, measured by a register-only kernel
 * (TFLOP/s); the denominator for FP64-ALU-bound kernels. */
int wr_measure_fp64_tflops(void *cuda_stream, double *out);

#ifdef __cplusplus
}
#endif
#endif
