/*
 * helm.h -- C ABI of the GB300 ECS-Helmholtz solver (libhelm.so).
 *
 * The library solves H u = b for the indefinite Helmholtz operator
 *     H u = -(Laplacian + phi(x)) u,  phi = k(x)^2                 (Section 2, eq. "helmctu0";
 *                                                                  variable k: Section 4, eq. "Helgen")
 * discretised by the Shortley-Weller second difference (Section 3, eq. "shortwell") on a
 * vertex-centred grid whose ends are continued by exterior-complex-scaled (ECS) layers with
 * mesh width h e^{i theta_gamma} (Section 2, the linear ECS map; Section 3, eq. "ecsgrid").
 * It uses right-preconditioned Bi-CGSTAB or IDR(s) (Section 6.2) with one multigrid V-cycle
 * on a complex-shifted-Laplacian (CSL, Section 5.2, eq. "helmctucsl") or complex-stretched-
 * grid (CSG, Section 5.3, eqs. "CSL-CSG" and "lapctucsg") preconditioner per matvec.
 *
 * Conventions for every entry point:
 *   - Vectors are DEVICE pointers on the current CUDA device, complex interleaved
 *     (re, im) of the element type given by helm_dtype, holding every unknown (interior and
 *     layer nodes; Dirichlet nodes are not stored), index i + Nx*(j + Ny*l), x fastest.
 *     They must be 16-byte aligned (8-byte for HELM_C64) and must not alias unless stated.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  Work is enqueued on it;
 *     calls return before the GPU finishes unless stated.  helm_solve synchronises the
 *     stream once at the end to return its statistics.
 *   - The caller owns b, x and every array it passes.  The library owns the context, the
 *     multigrid hierarchy and all workspace, released by helm_destroy.  helm_create allocates
 *     the operator and the hierarchy; the first helm_solve with a given (method, s) allocates
 *     its Krylov workspace and captures its graphs (a different (method, s) replaces them).
 *     Nothing else allocates device memory.
 *   - No call aborts, traps or throws: every call returns a helm_status.  Argument errors are
 *     detected on the host before anything is launched.  A context is not thread-safe.
 */
#ifndef HELM_H
#define HELM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  HELM_OK = 0,
  HELM_ERR_ARG = 1,       /* invalid argument (sizes, kinds, NULL pointers, misalignment) */
  HELM_ERR_OOM = 2,       /* device allocation failed in helm_create */
  HELM_ERR_CUDA = 3,      /* a CUDA runtime call failed; see helm_last_error() */
  HELM_ERR_BREAKDOWN = 4, /* Krylov breakdown: rho, (r^, v), |t|^2 or omega became zero */
  HELM_ERR_MAXIT = 5,     /* matvec cap reached (or true-residual restarts exhausted) */
  HELM_ERR_NAN = 6,       /* a norm or inner product was not finite */
  HELM_ERR_TIMEOUT = 7,   /* a bounded device-side wait gave up */
  HELM_ERR_BUSY = 8       /* reserved */
} helm_status;

typedef enum { HELM_C64 = 0 /* complex float32 */, HELM_C128 = 1 /* complex float64 */ } helm_dtype;

enum { HELM_PC_NONE = 0, HELM_PC_CSL = 1, HELM_PC_CSG_UNIFORM = 2, HELM_PC_CSG_INTERIOR = 3 };
enum { HELM_SM_JACOBI = 0, HELM_SM_RBGS = 1, HELM_SM_ILU = 2 };
enum { HELM_BICGSTAB = 0, HELM_IDR = 1, HELM_GMRES = 2 };
/* largest GMRES restart length (helm_solve_opts.s) */
#define HELM_GMRES_MAX_M 128

/* Grid of one instance (Section 3, eq. "ecsgrid", extended per axis).  Along axis a the
 * interior holds n_int[a] nodes at 0, h, ..., extent[a] (h = extent/(n_int-1)); a side with
 * n_layer[a][side] = m > 0 continues with m ECS nodes of width h e^{i theta_gamma} and a
 * Dirichlet node after them; a side with m = 0 is a Dirichlet wall (its end node is not an
 * unknown).  A side with m = -1 carries the first-order Sommerfeld condition du/dn = -i k u
 * (Section 2, eq. "sommerfeld1"; the paper's east / north edges of MP2 and MP3, all four edges of
 * MP1's Sommerfeld rows): its end node is an unknown whose row takes a mirrored ghost node,
 * u_g = u_{N-1} - 2 i k h u_N on a high side and u_g = u_1 - 2 i k h u_0 on a low side, with
 * k = sqrt(phi) >= 0 there (also in the preconditioner, whose shift or stretch applies as
 * elsewhere).  Coarsening keeps those nodes: coarse unknown c is fine unknown 2c + 1, or 2c on an
 * axis with a Sommerfeld low side, and it stops at the first level where a Sommerfeld high side's
 * node would not be kept (n - 1 - offset odd).  Levels coarsened with offset 0 run the
 * one-kernel-per-component V-cycle and take no Galerkin operators (HELM_ERR_ARG).  Unknowns per
 * axis: n_int - 2 + (m_lo > 0 ? m_lo + 1 : m_lo < 0 ? 1 : 0) + (m_hi > 0 ? m_hi + 1 : m_hi < 0 ? 1
 * : 0).
 * ecs_ramp = R > 1 replaces the sharp turn by a gradual one (the smooth ECS transition of the
 * paper's remark in Section 7): the m-th layer width counted from the turning point (m = 1, 2,
 * ...) is h e^{i theta_gamma min(m, R) / R}, so the contour turns by theta_gamma / R per width over
 * the first R widths; R = 0 or 1 is the sharp contour. */
typedef struct {
  int dim;              /* 1, 2 or 3 */
  int n_int[3];         /* >= 2 (>= 3 for a side without layer); unused axes ignored */
  int n_layer[3][2];    /* every side >= -1 (-1: Sommerfeld) */
  double extent[3];     /* > 0 */
  double theta_gamma;   /* ECS angle in radians, 0 <= theta_gamma < pi/2 */
  int ecs_ramp;         /* 0..1048576 */
} helm_grid;

/* Wave number k(x) (Section 2, eq. "helmctu0"; variable k: Section 4, eq. "Helgen"): the operator
 * uses phi = k(x)^2 at the real node positions (the layers continue the real coordinate: along axis
 * a the unknown with interior-node index j sits at j h, layer nodes at -m h and extent + m h).
 * When phi (a HOST array) is given it is used as it stands; otherwise `kind` says how to form it on
 * the device during helm_create:
 *   HELM_K_CONST       k = k0 everywhere (a zero-initialised struct);
 *   HELM_K_GAUSS_BUMP  k = k0 (1 + amp exp(-|x - centre|^2 / width2)), centre in the same absolute
 *                      coordinates as the nodes (width2 > 0);
 *   HELM_K_FIELD       k = field[p], a DEVICE array of N real values (x fastest, 8-byte aligned)
 *                      borrowed during helm_create only; a non-finite entry makes helm_create return
 *                      HELM_ERR_ARG.  The solve server does not take this kind (its requests are
 *                      built later, on its own thread): pass phi instead. */
enum { HELM_K_CONST = 0, HELM_K_GAUSS_BUMP = 1, HELM_K_FIELD = 2 };
typedef struct {
  double k0;
  const double* phi;    /* HOST pointer to N real values of k^2 (x fastest), read during helm_create
                           only; NULL: see kind */
  const double* phi_im; /* HOST pointer to N values or NULL: the imaginary part of phi, for k read at
                           the complex node positions of the layers (the analytic continuation of
                           k); it must come with phi.  The uniform-interior shortcut of a level is
                           kept only where it vanishes (the interior nodes are real) */
  int kind;             /* HELM_K_*, used when phi is NULL */
  double amp, width2;   /* HELM_K_GAUSS_BUMP */
  double centre[3];     /* HELM_K_GAUSS_BUMP */
  const double* field;  /* HELM_K_FIELD: DEVICE pointer to N values of k */
} helm_kspec;

/* Preconditioner M and the V(nu1, nu2)-cycle that approximates M^{-1} (Section 5;
 * components of Section 6.1: full-weighting restriction, bilinear/trilinear prolongation,
 * rediscretised coarse operators, damped Jacobi or red-black Gauss-Seidel smoothing, and a
 * direct solve on the coarsest level). */
typedef struct {
  int kind;             /* HELM_PC_*: NONE = identity; CSL: M = -(L + shift * phi);
                           CSG_UNIFORM: every width times e^{i theta_beta}, M = -(L_beta + phi);
                           CSG_INTERIOR: only interior widths scaled */
  double theta_beta;    /* CSG angle */
  double shift_re, shift_im; /* CSL shift beta^2 */
  int nu1, nu2;         /* 0..8 sweeps */
  int smoother;         /* HELM_SM_JACOBI, HELM_SM_RBGS or HELM_SM_ILU (ILU(0), Section 6.1: 1D and
                           2D grids, the one-kernel-per-component V-cycle; see helm_create) */
  double omega;         /* Jacobi damping, 0 < omega <= 1 */
  int max_levels;       /* >= 1; a coarsest level that needs the dense inverse (variable k) must
                           have at most HELM_COARSE_MAX_UNKNOWNS unknowns (else helm_create:
                           HELM_ERR_ARG) */
  int coarse_max;       /* stop coarsening once every axis has <= coarse_max unknowns */
  helm_dtype mg_dtype;  /* HELM_C64: whole V-cycle in complex FP32; HELM_C128: FP64 */
  int flags;            /* HELM_PF_*; 0 = defaults */
} helm_precond;

/* The coarsest level is solved exactly.  With a constant k there and more than 512 unknowns, by
 * separation of variables: per-axis eigendecompositions of the Shortley-Weller matrices, computed
 * in FP64 on the host at helm_create, applied as one transform per axis (any size).  Otherwise its
 * dense inverse is built at helm_create by Gauss-Jordan in FP64 (one block up to 512 unknowns, the
 * whole GPU above) and applied as a dense matrix-vector product in the V-cycle precision; this
 * limits such levels to HELM_COARSE_MAX_UNKNOWNS unknowns (4 GiB in FP64 during create). */
#define HELM_COARSE_MAX_UNKNOWNS 16384

/* helm_precond.flags: HELM_PF_UNFUSED runs every V-cycle component as its own kernel (the
 * same arithmetic as the default fused kernels; for testing the fusion); HELM_PF_NO_PDL
 * launches the solve-path kernels without programmatic dependent launch (same kernels);
 * HELM_PF_NO_AUTOTUNE skips the autotuner of helm_create, which times the large, small, square, wide
 * and one-warp tiles of the fused 2D kernels on every fused level and then whole V-cycles for every
 * admissible depth of the one-block tail kernel, keeps the fastest, and caches the choices for the
 * process (tiles by precision, smoother and level shape; depth by precision, smoother and
 * hierarchy); without it tiles follow a block-count rule and the tail a point budget.  When the
 * environment variable HELM_TUNE_CACHE names a file, the process reads earlier decisions from it
 * and appends its new ones, so that another process (say, one under a profiler) makes the same.  Tiles
 * change the speed only (every point is computed by the same formulas); the tail depth also
 * changes the summation order inside the small levels, i.e. the rounding. */
enum { HELM_PF_UNFUSED = 1, HELM_PF_NO_PDL = 2, HELM_PF_NO_AUTOTUNE = 4, HELM_PF_GALERKIN = 8 };
/* HELM_PF_GALERKIN (2D or 3D, omega-Jacobi or ILU(0); else helm_create: HELM_ERR_ARG): every coarse
 * level's operator is R A P -- the full weighting R times the finer level's operator A times the
 * (bi/tri)linear interpolation P of the V-cycle, a 9-point (2D) or 27-point (3D) stencil built at
 * helm_create in FP64 -- instead of the Shortley-Weller operator rediscretised on the coarse widths
 * (Section 6.1 lists both). */

/* Krylov solve options.  The stopping rule is ||r_m|| / ||b|| < tol on the recurrence
 * residual (Section 6.2, with d_0 = b since x_0 = 0), then b - H x is recomputed in FP64;
 * if it misses tol the method restarts from x (at most max_restarts times).
 * HELM_GMRES is restarted right-preconditioned GMRES(m) (the paper's remark on testing GMRES,
 * Section 7), m = s: each Arnoldi step is one preconditioned matvec, orthogonalised against the
 * basis by classical Gram-Schmidt applied twice; the residual norm of the least-squares problem
 * (from complex Givens rotations) plays the recurrence residual.  A cycle ends at m steps, when
 * that norm meets tol, or at maxmv; then x += M^{-1} V y and the true residual starts the next
 * cycle.  Cycles continue until the true residual meets tol or maxmv is reached; only a cycle
 * whose estimate met tol while the true residual did not counts against max_restarts.  Device
 * memory: m + 1 basis vectors besides the common work vectors. */
typedef struct {
  int method;           /* HELM_BICGSTAB, HELM_IDR or HELM_GMRES */
  int s;                /* IDR shadow dimension, 1..8; GMRES restart length m, 1..HELM_GMRES_MAX_M */
  double tol;           /* > 0 */
  int maxmv;            /* cap on preconditioned matvecs (V-cycle + H apply), >= 1 */
  int max_restarts;     /* >= 0 */
  const void* shadow;   /* IDR: HOST pointer to s x N complex128 raw random vectors (row j =
                           vector j), orthonormalised by the library; required for IDR.  The
                           orthonormalised copy is cached per context and keyed on this
                           pointer: pass a different pointer to change the shadow space */
  double* history;      /* optional DEVICE array of maxmv doubles: entry m-1 receives the
                           recurrence residual / ||b|| after preconditioned matvec m (the
                           convergence history of the paper's Figure "krylov"); NULL = off */
  int host_loop;        /* 0: the loop runs on the device (conditional WHILE graph node);
                           1: the host launches the captured iteration once per iteration and
                           reads the convergence flag after each (same kernels, one
                           synchronisation per iteration; lets kernel profilers see every
                           launch of the loop) */
} helm_solve_opts;

typedef struct {
  helm_status status;
  int iters;            /* Bi-CGSTAB iterations or IDR steps */
  int matvecs;          /* preconditioned matvecs */
  int restarts;
  double rel_res_recur; /* last recurrence residual / ||b|| */
  double rel_res_true;  /* ||b - H x|| / ||b|| recomputed in FP64 */
  long kernels;         /* kernel launches the solve executed on the device */
  int vcycles;          /* V-cycles applied: one per preconditioned matvec, plus one per GMRES cycle
                           for its update x += M^{-1} V y; 0 without a preconditioner */
  double seconds;       /* host wall time from the start of the solve to its statistics being read
                           (a served request: summed over its right-hand sides) */
  int history_len;      /* entries written to opts.history (0 when it was NULL) */
} helm_solve_info;

typedef struct helm_ctx helm_ctx;

/* Builds the grid, the FP64 operator H and the preconditioner hierarchy on the current
 * device (setup kernels on `stream`, then synchronises).  Returns HELM_ERR_ARG for invalid
 * sizes/kinds, HELM_ERR_OOM if device memory runs out (nothing is leaked).
 * HELM_SM_ILU: the ILU(0) factors of every level above the coarsest are computed here (FP64,
 * stored in mg_dtype; the level's own stencil pattern, unknowns in natural order).  It takes 1D
 * and 2D grids whose finest level has at most 7,264 (complex64) or 3,632 (complex128) rows along
 * y (a ring of 4 values per row in one block's 227 KB of shared memory), else HELM_ERR_ARG; each
 * smoothing step runs its two triangular solves as one single-block launch over the wavefronts
 * i + 2j (their n0 + 2 n1 - 2 steps are sequential), so the V-cycle is far slower than with the
 * point smoothers. */
helm_status helm_create(const helm_grid* grid, const helm_kspec* k, const helm_precond* pc,
                        void* stream, helm_ctx** out);

/* Number of unknowns N of the instance (0 if ctx is NULL). */
long helm_size(const helm_ctx* ctx);

/* Device bytes held by the context. */
size_t helm_workspace_bytes(const helm_ctx* ctx);

/* y = H x (eq. "helmctu0" discretised by eq. "shortwell").  dtype HELM_C128: x, y complex128,
 * FP64 arithmetic.  dtype HELM_C64: x complex64 read and y complex128 written, FP64
 * arithmetic (the upcast is exact).  x and y must not alias. */
helm_status helm_apply(helm_ctx* ctx, helm_dtype dtype, const void* x, void* y, void* stream);

/* z = one V(nu1, nu2)-cycle on the preconditioner from a zero initial guess, z ~ M^{-1} r
 * (Section 5.1; M is CSL or CSG, Sections 5.2-5.3).  r is complex128 (a Krylov vector).
 * pc: NULL, or the preconditioner the context was created with -- its hierarchy is built once, in
 * helm_create, so another kind, parameter, cycle, smoother, depth, precision or coarse-operator
 * choice returns HELM_ERR_ARG (create a context for it).  dtype is z's element type: the
 * hierarchy's mg_dtype, or HELM_C128 with an FP32 hierarchy, in which case the cycle runs in FP32
 * and its last kernel writes z widened to complex128 (the precision boundary of the mixed solver;
 * the widening is exact).  HELM_C64 with an FP64 hierarchy returns HELM_ERR_ARG.  For HELM_PC_NONE,
 * z = r converted to dtype.  r and z must not alias. */
helm_status helm_vcycle(helm_ctx* ctx, const helm_precond* pc, helm_dtype dtype, const void* r, void* z,
                        void* stream);

/* Single multigrid component on level `lvl` of the hierarchy (element type = mg_dtype), for
 * testing each kernel against a reference:
 *   HELM_OP_APPLY     out = M_lvl a
 *   HELM_OP_RESIDUAL  out = b - M_lvl a
 *   HELM_OP_SMOOTH    a <- `count` smoothing sweeps on M_lvl a = b (in place; out unused)
 *   HELM_OP_SMOOTH0   a <- the first sweep from a zero guess, then count-1 sweeps
 *   HELM_OP_RESTRICT  out (level lvl+1) = full weighting of a (level lvl)
 *   HELM_OP_PROLONG   a (level lvl) += bilinear interpolation of b (level lvl+1)
 *   HELM_OP_COARSE    out = M_coarsest^{-1} a (lvl must be the coarsest level)
 *   HELM_OP_DOWN      the fused first half of a V(1,1) level (2D, nu1 = 1, not the coarsest):
 *                     a = one smoothing sweep from the zero guess on M_lvl a = b, and
 *                     out (level lvl+1) = full weighting of b - M_lvl a, in one kernel
 *   HELM_OP_TO_STORED   out = a (natural order) in level lvl's storage order
 *   HELM_OP_FROM_STORED out = a (in level lvl's storage order) in natural order
 * Vectors are in natural order (x fastest), unless HELM_OP_STORED is or'ed into `op` (SMOOTH,
 * SMOOTH0, APPLY, RESIDUAL, RESTRICT, PROLONG: every vector in its level's storage order).  The
 * storage order is natural except on the red-black levels of a 3D FP32 hierarchy above the
 * coarsest level (and above the one-block tail): there each row of n0 points holds its even x
 * indices first, then its odd ones ("x-split"), so that the points of one colour in a row are
 * contiguous.  The V-cycle converts at its boundary; this interface is for tests and timing. */
enum { HELM_OP_APPLY = 0, HELM_OP_RESIDUAL = 1, HELM_OP_SMOOTH = 2, HELM_OP_SMOOTH0 = 3,
       HELM_OP_RESTRICT = 4, HELM_OP_PROLONG = 5, HELM_OP_COARSE = 6, HELM_OP_DOWN = 7,
       HELM_OP_TO_STORED = 8, HELM_OP_FROM_STORED = 9, HELM_OP_STORED = 0x100 };
helm_status helm_level_op(helm_ctx* ctx, int op, int lvl, void* a, const void* b, void* out,
                          int count, void* stream);

/* Number of multigrid levels and the unknowns per axis of level lvl (n[3]). */
int helm_num_levels(const helm_ctx* ctx);
helm_status helm_level_shape(const helm_ctx* ctx, int lvl, int* n);

/* Solves H x = b from x = 0 (b, x complex128, device, no aliasing).  Returns the final
 * status (also in info->status); x always holds the last iterate.  The whole Krylov loop runs
 * on the device (one graph launch per solve, a conditional WHILE node around one iteration);
 * the host synchronises once at the end to read the statistics. */
helm_status helm_solve(helm_ctx* ctx, const void* b, void* x, const helm_solve_opts* opts,
                       helm_solve_info* info, void* stream);

/* Solves n independent instances H_i x_i = b_i at once (a batch of uneven grids, k fields and
 * preconditioners): every instance's device-resident solve (as in helm_solve, opts[i]) runs on
 * its own stream, ordered after `stream` and joined back into it, so the instances overlap on the
 * GPU; the host only reads each instance's statistics when its loop has finished.  ctxs must be n
 * distinct contexts (a context holds one solve's workspace); b[i], x[i] follow helm_solve; opts
 * has n entries, so every instance has its own method, shadow space and tolerances.  Streams get
 * priorities longest work first (unknowns x the method's cost per matvec), so that the instances
 * that finish last start first and the short ones fill the gaps.
 * infos (n entries, may be NULL) receives every instance's statistics.  Returns HELM_OK when all
 * instances converged, else the first non-OK instance status (every x[i] still holds that
 * instance's last iterate); argument errors are reported before anything is launched.  The result
 * of each instance is bitwise the result helm_solve gives it alone. */
helm_status helm_solve_batch(helm_ctx* const* ctxs, const void* const* b, void* const* x, int n,
                             const helm_solve_opts* opts, helm_solve_info* infos, void* stream);

/* Solves n independent instances H_i x_i = b_i with Bi-CGSTAB (opts->method must be HELM_BICGSTAB;
 * one opts for all; no history) as ONE group: every kernel of an iteration -- the Krylov updates
 * and inner products, and each level of the V-cycles -- is a single launch over all instances'
 * blocks, driven by a device table of per-instance descriptors (operator, buffers, the blocks each
 * instance owns).  The instances iterate in lockstep in one captured loop graph whose WHILE node
 * runs while any of them is unfinished; an instance that has converged skips the later launches
 * (one flag read per block).  Launches per iteration: 6 Krylov kernels, 2 x (2 L + up to 3)
 * V-cycle kernels (L = the largest number of fused levels) and one condition kernel, whatever n.
 * Requirements (else HELM_ERR_ARG, checked on the host): n >= 1 distinct contexts on the current
 * device, 2D grids, a CSL or CSG preconditioner with V(1,1) cycles on rediscretised fused levels
 * (no HELM_PF_UNFUSED or HELM_PF_GALERKIN) and a dense coarsest inverse, one smoother kind (not
 * HELM_SM_ILU) and one
 * mg_dtype for all.  Grids, k fields, preconditioner parameters and sizes may all differ.
 * Each instance keeps its own block decomposition and reduction order, so its iterates, statistics
 * and solution are bitwise those helm_solve gives it alone; infos[i].kernels is the group's total
 * launch count.  Synchronises `stream` at the end. */
helm_status helm_solve_group(helm_ctx* const* ctxs, const void* const* b, void* const* x, int n,
                             const helm_solve_opts* opts, helm_solve_info* infos, void* stream);

/* ---- serving --------------------------------------------------------------------------------
 * A server admits solve requests of any grid, k field and preconditioner against a device-memory
 * budget and runs up to max_active of them at once, each on its own stream with its own context
 * (continuous batching: a request submitted while others run starts as soon as a slot and the
 * budget allow, and its work overlaps theirs on the GPU).  Requests start in submission order
 * unless helm_server_set_policy says otherwise.
 * Each request's result is bitwise what helm_solve gives it alone.  A server is thread-safe for
 * submit / poll / wait / stats; a worker thread owned by the server does the device work. */
typedef struct {
  helm_grid grid;
  helm_kspec k;          /* k.phi (HOST) is copied at submit */
  helm_precond pc;
  helm_solve_opts opts;  /* opts.shadow (HOST, IDR) is copied at submit; history and host_loop ignored */
  const void* b;         /* HOST complex128, nrhs x N entries (right-hand side after right-hand
                            side); copied at submit */
  void* x;               /* HOST complex128, nrhs x N entries; written before the request
                            completes and must stay valid until then */
  int nrhs;              /* right-hand sides, 1 .. HELM_MAX_RHS (0 counts as 1); they are solved
                            one after another on the request's context, whose operator,
                            hierarchy and Krylov workspace stay on the device in between.  The
                            completed request's statistics add up iterations, matvecs, restarts
                            and kernels over its right-hand sides and keep the largest residuals;
                            a failing right-hand side ends the request with its status */
} helm_request;
#define HELM_MAX_RHS 64
typedef struct helm_server helm_server;

/* Device bytes a request holds while it runs (operator, hierarchy, coarse inverse, Krylov
 * workspace, b and x); the server admits against this estimate.  0 for invalid arguments. */
size_t helm_estimate_bytes(const helm_grid* grid, const helm_precond* pc, const helm_solve_opts* opts);

helm_status helm_server_create(size_t budget_bytes, int max_active, helm_server** out);
/* Admission order.  HELM_SERVE_FIFO (the default): submission order, a request that does not fit
 * the free budget waits and so do the ones behind it.  HELM_SERVE_SMALLEST_FIRST: the queued
 * request with the least work (unknowns x right-hand sides) that fits the free budget, except that
 * a request passed over 2 x max_active times is admitted next.  Either way the requests running at
 * once get stream priorities smallest work first.  The policy changes when requests run, never
 * their results. */
enum { HELM_SERVE_FIFO = 0, HELM_SERVE_SMALLEST_FIRST = 1 };
helm_status helm_server_set_policy(helm_server* s, int policy);
/* HELM_ERR_OOM if the request alone exceeds the budget; *ticket identifies it afterwards. */
helm_status helm_server_submit(helm_server* s, const helm_request* req, uint64_t* ticket);
/* HELM_ERR_BUSY while queued or running; otherwise the request's final status, with its
 * statistics and the submission-to-completion latency in seconds. */
helm_status helm_server_poll(helm_server* s, uint64_t ticket, helm_solve_info* info, double* latency_s);
helm_status helm_server_wait(helm_server* s, uint64_t ticket, helm_solve_info* info, double* latency_s);
helm_status helm_server_stats(helm_server* s, int* queued, int* active, size_t* used_bytes);
/* Finishes every queued and running request, then releases the server. */
void helm_server_destroy(helm_server* s);

/* r = b - H x and *rel_out = ||r|| / ||b|| (0 when b = 0), FP64, without allocating anything.
 * The paper has no counterpart: this is the true-residual computation that helm_solve runs
 * after its Krylov loop, offered to callers that cannot allocate device memory -- processes
 * whose device memory belongs to another allocator that reserved the device up front, and
 * latency-critical loops that cannot afford cudaMalloc, which may synchronise the device.
 * The caller passes every input and output: b, x, r (complex128, N entries) and rel_out (one
 * double), all DEVICE pointers, 16-byte aligned (rel_out 8), r aliasing neither b nor x.
 * Its scratch (per-block partial sums and a completion counter) is a file-scope static
 * device array of 64 KiB + 256 B that every device which loads libhelm.so keeps until the
 * process exits; it bounds N to at most 4,194,304 unknowns (HELM_ERR_ARG beyond).
 * The context's device must be current (else HELM_ERR_ARG).  Each call made outside a stream
 * capture looks up that array's device address with the device current (cudaGetSymbolAddress),
 * so a call after a device reset finds the reloaded array; a call made while `stream` is being
 * captured reuses the address of an earlier call on that device, so make the first call on each
 * device before any stream capture (a first call inside one returns HELM_ERR_ARG).
 * Every call shares the one array and zeroes its counter on `stream` before the kernel:
 * calls whose kernels overlap on the GPU (two streams, or two host threads) race and give
 * wrong results; serialise them.  Asynchronous: *rel_out is valid once `stream` reaches it. */
helm_status helm_residual_noalloc(helm_ctx* ctx, const void* b, const void* x, void* r,
                                  double* rel_out, void* stream);

/* Multigrid as a stationary solver of the preconditioner's own equation M u = f (M = the
 * finest preconditioner operator; Section 7, remark on choosing the CSL and CSG parameters):
 * from u = 0, each cycle sets u <- u + V(f - M u) with one V-cycle V.  *cycles receives the
 * number of cycles after which ||f - M u|| <= reduction ||f|| (0 when f = 0), or -1 when that
 * does not happen within max_cycles or the ratio exceeds 1e6 or stops being finite.  hist
 * (HOST, optional, max_cycles doubles) receives ||f - M u|| / ||f|| after each cycle run.
 * f and u are complex128 DEVICE vectors of N (16-byte aligned, not aliased); the context needs a
 * CSL or CSG preconditioner with an FP64 hierarchy (mg_dtype HELM_C128), else HELM_ERR_ARG.
 * Allocates 2 N complex128 of scratch on `stream` and synchronises it once per cycle. */
helm_status helm_mg_iterate(helm_ctx* ctx, const void* f, void* u, int max_cycles, double reduction,
                            int* cycles, double* hist, void* stream);

/* The automatic parameter choice of the same remark.  The parameter is the imaginary part of
 * the CSL shift (start->kind HELM_PC_CSL) or the CSG angle theta_beta (the CSG kinds).  Trial t
 * uses the parameter p_t = p_{t-1} * factor (p_0 = the start's, one multiplication per trial),
 * builds the hierarchy with it in FP64 (without the autotuner) and runs helm_mg_iterate with right-hand side f (complex128
 * DEVICE vector of N, seeded by the caller); trials continue while multigrid converges within
 * max_cycles, up to max_trials (1..64).  *out = the start with the last converging parameter;
 * params / cycles (HOST, optional, max_trials entries) record each trial's parameter and cycle
 * count (-1 = did not converge); *trials = trials run.  Returns HELM_ERR_MAXIT (and *out = the
 * start) when the start itself does not converge, HELM_ERR_ARG for factor outside (0, 1) or an
 * identity preconditioner, or the error of helm_create. */
helm_status helm_select_precond(const helm_grid* grid, const helm_kspec* k, const helm_precond* start,
                                const void* f, int max_cycles, double reduction, double factor,
                                int max_trials, helm_precond* out, double* params, int* cycles,
                                int* trials, void* stream);

/* Releases everything the context holds (synchronises the device first).  NULL is a no-op. */
void helm_destroy(helm_ctx* ctx);

const char* helm_status_str(helm_status s);

/* Text of the last CUDA error seen by this thread (empty if none). */
const char* helm_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* HELM_H */
