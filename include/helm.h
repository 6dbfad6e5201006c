/*
 * helm.h -- C ABI of the GB300 (sm_103a) solver for the Helmholtz equation with
 * exterior-complex-scaled (ECS) absorbing layers, preconditioned by the complex
 * stretched grid (CSG) operator inverted with one GMRES(s)-smoothed multigrid
 * V-cycle, inside an outer flexible GMRES (binary64 least squares, solution and true
 * residual; the Krylov basis in binary64 or double-float, helm_opts.outer_basis).
 *
 * Method: B. Reps, W. Vanroose, H. bin Zubair, "GMRES-based multigrid for the complex
 * scaled preconditioner for the indefinite Helmholtz equation", arXiv:1012.5379.
 *   - problem  H u = -(Laplacian + phi) u = chi                (Sec. 1, Eq. helm)
 *   - grids    interior spacing h e^{i theta_beta}, layer spacing h e^{i theta_gamma}
 *              (Sec. 2, Eq. csggrid; layers on both sides per Remark 2.2)
 *   - operator three-point non-uniform second difference per axis, Kronecker sum in
 *              d dimensions, M = L^CSG - phi, H = L^ECS - phi   (Sec. 2, Eq. csg_dis,
 *              Lemma 2.1)
 *   - smoother GMRES(s) on every level, V(nu1, nu2) cycle, rediscretised coarse
 *              operators (Sec. 3.1, Prop. 3.1)
 *   - outer    flexible GMRES, one V-cycle per iteration from a zero guess (Sec. 5)
 *
 * Conventions for every entry point:
 *   - Complex vectors are interleaved (re, im) arrays of n^dim complex numbers in
 *     natural order: x fastest, then y, then z (C order of an (n,)*dim array).
 *   - Device pointers must be allocated on the current CUDA device; the caller owns
 *     them.  Host pointers are plain (pinned or pageable) host memory.
 *   - `stream` is a cudaStream_t passed as void*; NULL means the legacy default
 *     stream.  All device work is enqueued on it.
 *   - Return value: HELM_OK (0) or a negative HELM_E* code; helm_last_error() gives a
 *     thread-local message for the last failure on the calling thread.  No C++
 *     exception crosses this boundary.
 *   - Handles are not thread-safe: one host thread at a time per handle.
 */
#ifndef HELM_H
#define HELM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define HELM_OK 0
#define HELM_EINVAL -1   /* invalid argument (sizes, angles, tolerance, NULL pointer) */
#define HELM_ENOMEM -2   /* device allocation failed or serving budget exceeded */
#define HELM_ENOCONV -3  /* maxit reached before tol; x holds the last iterate */
#define HELM_ENUMERIC -4 /* NaN/Inf in a residual norm */
#define HELM_ETIMEOUT -5 /* a bounded wait ran out (serving wait; a V-cycle kernel's wait for its
                            tile copies, after which the handle's results are invalid) */
#define HELM_ECUDA -6    /* CUDA runtime error */
#define HELM_EAGAIN -7   /* serving: request not finished yet */

/* preconditioner precision */
#define HELM_C64 1   /* complex FP32 storage and arithmetic (FP32 accumulation) */
#define HELM_C128 2  /* complex FP64 */
#define HELM_CAUTO 3 /* helm_setup picks: HELM_C128 when the finest grid has at most
                        HELM_AUTO_C128_POINTS unknowns (n^dim), else HELM_C64.  Small grids
                        cost little more in FP64 (their V-cycle is launch-latency bound), and
                        some small problems are sensitive to the FP32 rounding of the
                        preconditioner: with bound states (Benchmark 3 of Sec. 5, nu = 7 on
                        64^2) the complex64 V-cycle costs 40% more outer iterations. */
#define HELM_AUTO_C128_POINTS 16384

typedef struct helm_handle helm_handle;

/* Grid: the unit interval per axis, n interior nodes, spacing h = 1/(n+1); u = 0 on
 * the outer edge of the layers.  n must be >= 3 and coarsening proceeds while n+1 is
 * even and n > coarsest_n (so n = 2^L - 1 gives L-1 levels down to 3).
 * ecs_frac: layer width on each side as a fraction of the box, 0 < ecs_frac < 0.5
 * (0 < ecs_frac < 1 with ecs_sides = HELM_ECS_HIGH).
 * theta_gamma: ECS layer angle in radians, 0 <= theta_gamma < pi/2.
 * ecs_sides: HELM_ECS_BOTH puts a layer at both ends of every axis (Remark 2.2);
 * HELM_ECS_HIGH only at the far end (x = 1), with u = 0 on the near edge x = 0 of the
 * interior (Benchmark 3 of Sec. 5: Dirichlet south and west edges, ECS north and
 * east).  A zero-initialised grid takes HELM_ECS_BOTH. */
typedef struct {
  int dim;            /* 2 or 3 */
  int n;              /* interior nodes per axis (same on every axis) */
  double ecs_frac;    /* default 0.125 */
  double theta_gamma; /* default 0.5 */
  int ecs_sides;      /* HELM_ECS_BOTH or HELM_ECS_HIGH, default HELM_ECS_BOTH */
} helm_grid;
#define HELM_ECS_BOTH 0
#define HELM_ECS_HIGH 1

/* Options.  Zero-initialised fields take the defaults in brackets. */
typedef struct {
  int nu1;          /* pre-smoothing GMRES(s) sweeps per level      [1] */
  int nu2;          /* post-smoothing sweeps per level               [1] */
  int s;            /* GMRES steps per sweep, 1..4                   [3] */
  int coarsest_n;   /* stop coarsening at this size or below         [3] */
  int precond_prec; /* HELM_C64, HELM_C128 or HELM_CAUTO             [HELM_C64] */
  int restart;      /* outer FGMRES restart length m, 0 = none       [0] */
  int maxit;        /* max preconditioner applications per solve     [400] */
  double csl_eps;   /* complex shift of the preconditioner: M = L - (1 + i csl_eps) phi
                     * (Sec. 1, Sec. 2: the complex shifted Laplacian of Erlangga, Oosterlee
                     * and Vuik); 0 = the complex stretched grid alone; with theta_beta = 0
                     * and csl_eps > 0 the preconditioner is M^CSL.  Finite, >= 0.  [0] */
  int smoother;     /* HELM_SMOOTHER_GMRES: GMRES(s) sweeps (Sec. 3);
                     * HELM_SMOOTHER_POLY: the third-degree polynomial smoother of Sec. 4
                     * (three Richardson steps per sweep, weights from helm_poly_smoother per
                     * level; constant k, csl_eps = 0, s ignored).  [HELM_SMOOTHER_GMRES] */
  int outer_basis;  /* arithmetic of the outer FGMRES Krylov basis v_i, of w = H z_j and of the
                     * orthogonalisation h_ij = <v_i, w>, u = w - sum h_ij v_i (Sec. 5):
                     * HELM_BASIS_F64: binary64 throughout;
                     * HELM_BASIS_DF: double-float, each real a pair of binary32 (hi + lo, 47
                     *   significant bits) multiplied and summed with error-free transformations
                     *   on the FP32 pipe; an inner product of n points errs by at most about
                     *   (4 + K) 2^-45 sum |v_i||w_i|, K the points one thread sums
                     *   (ceil(n / 77,824) on 152 SMs), which is inside binary64's
                     *   recursive-summation bound n u sum |v_i||w_i| (u = 2^-53) for n >= 2048;
                     *   with a complex64 preconditioner w = H z_j is formed in double-float too;
                     * HELM_BASIS_AUTO: double-float for grids of more than HELM_AUTO_C128_POINTS
                     *   unknowns solved to tol >= HELM_BASIS_DF_MIN_TOL, binary64 otherwise.  On
                     *   small grids the orthogonalisation costs little either way, and problems
                     *   with bound states are sensitive to any rounding there (Benchmark 3 of
                     *   Sec. 5, nu = 7 on 64^2: 79 outer iterations with binary64, 80 with
                     *   double-float); on the larger grids the two take the same counts.
                     * The Hessenberg matrix, the Givens rotations, the least-squares solution, the
                     * stored z_j, the solution x (updated in double-float with a double-float
                     * basis and a complex64 preconditioner) and the true residual b - H x that
                     * decides convergence are held in binary64 in every mode.  [HELM_BASIS_AUTO] */
} helm_opts;
#define HELM_SMOOTHER_GMRES 0
#define HELM_SMOOTHER_POLY 1
#define HELM_BASIS_AUTO 0
#define HELM_BASIS_F64 1
#define HELM_BASIS_DF 2
#define HELM_BASIS_DF_MIN_TOL 1e-9
/* The Krylov basis length m = min(restart, maxit) (maxit without restart) is at most
 * HELM_MAX_BASIS; helm_setup returns HELM_EINVAL above it. */
#define HELM_MAX_BASIS 1536

typedef struct {
  int iters;           /* preconditioner applications (outer iterations) */
  int restarts;        /* completed FGMRES cycles */
  double rel_res_est;  /* Arnoldi estimate |g_{j+1}| / ||b|| at exit */
  double rel_res_true; /* ||b - H x|| / ||b|| recomputed in FP64 at exit */
  int status;          /* HELM_OK, HELM_ENOCONV or HELM_ENUMERIC */
  int basis;           /* the arithmetic the solve's Krylov basis ran in: HELM_BASIS_F64 or
                        * HELM_BASIS_DF (what HELM_BASIS_AUTO resolved to) */
} helm_info;

/* Build the CSG hierarchy (Sec. 3.1, Prop. 3.1) and the ECS operator H for one
 * problem, and allocate its workspace on the current device.
 *   phi:  device pointer to n^dim floats holding phi = k(x)^2 at the interior nodes
 *         (natural order), or NULL for a constant wavenumber `k` (phi = k^2).  The
 *         field is copied; coarse levels sample it at their nodes.
 *   theta_beta: CSG interior angle in radians, 0 <= theta_beta < pi/2 (Sec. 2).
 *   opts may be NULL (all defaults).  opts->csl_eps > 0 (constant k only) adds the
 *         complex shift of the CSL variant: M = L - (1 + i csl_eps) k^2 on every level,
 *         the stretched-grid angle applying as well (theta_beta = 0: pure CSL).
 *   grid->ecs_sides = HELM_ECS_HIGH places the layers at the far end of every axis
 *         only (Dirichlet near edges, Benchmark 3 of Sec. 5); the hierarchy, the
 *         kernels and every other call are unchanged.
 * Errors: HELM_EINVAL (dim, n, angles, ecs_frac, ecs_sides, opts out of range,
 * csl_eps with a phi field), HELM_ENOMEM, HELM_ECUDA.  The call synchronises `stream`
 * before returning. */
int helm_setup(const helm_grid* grid, const float* phi, double k, double theta_beta,
               const helm_opts* opts, void* stream, helm_handle** out);

/* Release a handle and all device memory it owns (NULL is a no-op). */
void helm_destroy(helm_handle* h);

/* z ~ (M^CSG)^{-1} r by one V(nu1, nu2) cycle from a zero initial guess (Sec. 3.2,
 * Sec. 5).  r and z are device arrays of n^dim complex numbers in precision `prec`
 * (HELM_C64: float pairs, HELM_C128: double pairs), independent of the handle's
 * internal precision (converted on the way in and out).  Asynchronous on `stream`. */
int helm_precond_apply(helm_handle* h, const void* r, void* z, int prec, void* stream);

/* w = M^CSG v (prec = HELM_C64/HELM_C128, which = 0) or w = H v (which = 1) on the
 * finest level (Sec. 2, Eq. csg_dis).  Asynchronous on `stream`.  Exposed for
 * verification of the stencil. */
int helm_apply_operator(helm_handle* h, int which, const void* v, void* w, int prec, void* stream);

/* Solve H x = b with right-preconditioned FGMRES(m) (Sec. 5) to
 * ||b - H x|| / ||b|| <= tol, recomputed in FP64.
 *   b: device, n^dim complex128 (read only).
 *   x: device, n^dim complex128; on entry the initial guess, on exit the solution.
 *   info: filled on return (may be NULL).
 * Blocks the calling thread until the solve finishes (it reads convergence flags
 * from the device each iteration).  Returns HELM_OK, HELM_ENOCONV (maxit reached,
 * x holds the last iterate), HELM_ENUMERIC, HELM_EINVAL, HELM_ETIMEOUT or HELM_ECUDA. */
int helm_solve(helm_handle* h, const double* b, double* x, double tol, helm_info* info,
               void* stream);

/* As helm_solve, but b and x are HOST arrays: b is copied to the device, the solve
 * runs from a zero initial guess, and the solution is copied back into x.  Each call
 * allocates two device buffers of n^dim complex128 values for the copies and frees them
 * before it returns (HELM_ENOMEM if they cannot be allocated); page-locked host arrays
 * make the copies asynchronous. */
int helm_solve_host(helm_handle* h, const double* b_host, double* x_host, double tol,
                    helm_info* info, void* stream);

/* Solve `count` independent problems together: every V-cycle level is one launch
 * over all problems that have that level, and the outer FGMRES steps of all
 * problems share launches.  Problems may differ in n, k, phi and theta_beta, but
 * must share dim, precond_prec, nu1, nu2 and s, and have n + 1 a power of two.  Each
 * problem's result is bitwise the same as when it is solved alone (reductions are
 * per problem in a fixed order).
 *   b[i], x[i]: device arrays as in helm_solve for handle hs[i].
 *   infos: array of `count` (may be NULL).
 * Returns HELM_OK if every problem converged, HELM_ENOCONV / HELM_ENUMERIC if at
 * least one did not (see infos[i].status), or an argument/CUDA error. */
int helm_batch_solve(helm_handle* const* hs, int count, const double* const* b,
                     double* const* x, double tol, helm_info* infos, void* stream);

/* As helm_batch_solve, but b[i] and x[i] are HOST arrays: every b[i] is copied to
 * the device, the problems are solved together from zero initial guesses, and
 * every solution is copied back into x[i].  Allocates (and frees) device staging
 * buffers for the vectors. */
int helm_batch_solve_host(helm_handle* const* hs, int count, const double* const* b_host,
                          double* const* x_host, double tol, helm_info* infos, void* stream);

/* ---------------------------------------------------------------------------------
 * Serving: continuous batching of solves (the workload of Sec. 5 as a service).
 * A worker thread owns the device.  Between outer FGMRES iterations it admits queued
 * requests while the device-memory budget allows (in arrival order, except that a
 * request an idle slot or the free budget can serve may pass a waiting head a bounded
 * number of times), iterates every
 * admitted problem of a dimension together (one launch per V-cycle level and outer
 * kernel for all of them; 2D and 3D on separate streams, so their kernels overlap),
 * and retires problems as they converge.  Idle problem slots of the same shape are
 * reused.  A result is bitwise the same whatever other requests shared its launches.
 * The paper has no counterpart: this is the deployment interface of the solver.
 * --------------------------------------------------------------------------------- */
typedef struct helm_server helm_server;

typedef struct {
  size_t budget_bytes; /* device memory the server's problem slots may hold    [120 GiB] */
  int max_active;      /* problems iterated at once, 0 = bounded by the budget [0] */
  int precond_prec;    /* HELM_C64 or HELM_C128                                [HELM_C64] */
  int restart;         /* FGMRES restart of every request                       [40] */
  int maxit;           /* max outer iterations of every request                 [400] */
  int nu1, nu2, s;     /* V(nu1, nu2) with GMRES(s)                             [1, 1, 3] */
  double ecs_frac;     /* layer width of every request's grid                   [0.125] */
  double theta_gamma;  /* layer angle                                           [0.5] */
} helm_serve_opts;

typedef struct {
  long long submitted, completed, rejected;
  int queued, active, peak_active;
  size_t bytes_in_use, peak_bytes;
  int handles_created, handles_reused;
  long long group_builds;  /* problem groups (re)built on membership changes (whole library) */
  long long graph_builds;  /* V-cycle CUDA graphs captured and instantiated (whole library) */
  double build_s;          /* host seconds spent in both */
} helm_serve_counters;

/* Start a server on the current device (opts may be NULL: all defaults). */
int helm_serve_start(const helm_serve_opts* opts, helm_server** out);

/* Queue a solve of H x = b: grid (dim, n) with n + 1 a power of two, constant
 * wavenumber k, CSG angle theta_beta, tolerance tol.  b_host and x_host are HOST
 * arrays of n^dim complex128 (interleaved re, im; x fastest) that the server BORROWS:
 * the caller keeps b unchanged and both alive until the ticket completes; the solution
 * is written into x_host.  Page-locked buffers (cudaHostAlloc) let their copies
 * overlap with other requests' work; pageable ones are copied synchronously by the
 * worker.  Returns a ticket; never blocks on the device.  HELM_EINVAL for invalid
 * arguments or a stopping server. */
int helm_serve_submit(helm_server* s, int dim, int n, double k, double theta_beta, const double* b_host,
                      double* x_host, double tol, long long* ticket);

/* If the request is finished (its solution is in x_host): fill info and latency_s
 * (submit to completion, seconds; both may be NULL), release the ticket and return
 * its status (HELM_OK, HELM_ENOCONV, HELM_ENUMERIC, or HELM_ENOMEM when the request
 * can never fit the budget).  HELM_EAGAIN while pending. */
int helm_serve_poll(helm_server* s, long long ticket, helm_info* info, double* latency_s);

/* As helm_serve_poll, waiting at most timeout_s seconds (HELM_ETIMEOUT). */
int helm_serve_wait(helm_server* s, long long ticket, double timeout_s, helm_info* info, double* latency_s);

/* Counters of the server (a consistent snapshot). */
int helm_serve_stats(helm_server* s, helm_serve_counters* out);

/* Finish every queued and admitted request, then stop the worker and free the
 * device memory of all problem slots.  Unclaimed results are discarded. */
int helm_serve_stop(helm_server* s);

/* Bytes of device memory the handle holds. */
int helm_workspace_bytes(const helm_handle* h, size_t* bytes);

/* Levels of the hierarchy and their sizes (sizes may be NULL). */
int helm_levels(const helm_handle* h, int* nlevels, int* sizes, int max_sizes);

/* The handle's preconditioner precision, HELM_C64 or HELM_C128 (what HELM_CAUTO
 * resolved to).  Batched solves need handles of one precision. */
int helm_precond_precision(const helm_handle* h, int* prec);

/* The third-degree polynomial smoother (Sec. 4) of one level: real spacing h,
 * constant k, CSG angle theta_beta, layer angle theta_gamma, dimension dim.  p has
 * p(0) = 1, p(t1) = p(t2) = 0 and p(t0) = e^{i phi} at the vertices of the spectrum's
 * bounding triangle (Prop. 3.1); phi is chosen by the first- and second-order
 * stability conditions (Sec. 4.3, 4.4; the midpoint of the longest admissible arc on
 * a 0.05 degree grid, 0 where the first-order condition holds for every phi).
 * Writes phi (radians) and w[0..5] = re, im of the three Richardson weights of
 * p(t) = (1 - w1 t)(1 - w2 t)(1 - w3 t), ordered by real, then imaginary part (the
 * order the V-cycle applies them in).  Host only (no device work).  HELM_EINVAL if
 * no stable polynomial exists (theta_beta too small for this k and h, Sec. 4.5). */
int helm_poly_smoother(double k, double h, double theta_beta, double theta_gamma, int dim, double* phi,
                       double* w);

/* Stencil coefficients of one axis of the grid (Sec. 2, Eq. csggrid and the
 * three-point difference of Eq. csg_dis): the complex spacings h_i = z(x_{i+1}) - z(x_i)
 * of the stretched map (angle theta_beta inside, theta_gamma in the layers placed as
 * ecs_sides says, width ecs_frac) and, at interior node i = 0..n-1,
 * (L u)_i = a_i u_{i-1} + d_i u_i + c_i u_{i+1} with L ~ -d^2/dz^2.  a, d, c are host
 * arrays of n complex numbers as (re, im) double pairs, owned by the caller.  Host only
 * (no device work): this is the setup's own geometry, exported so that it can be
 * checked without a GPU.  HELM_EINVAL on a NULL array, n < 1, angles outside
 * [0, pi/2) or ecs_frac outside the range helm_grid states. */
int helm_axis_coefficients(int n, double ecs_frac, int ecs_sides, double theta_gamma, double theta_beta,
                           double* a, double* d, double* c);

/* One V(nu1, nu2) cycle, z ~ (M^CSG)^{-1} r, for a small grid without allocating any
 * device memory.  For callers that cannot let a library call cudaMalloc: programs
 * whose device memory is reserved up front by a pooling allocator, and
 * latency-critical loops that cannot afford the implicit device synchronisation of
 * cudaMalloc/cudaFree.  The paper has no counterpart: this is an interface variant
 * of helm_precond_apply.
 *   grid, theta_beta, opts: as for helm_setup (constant wavenumber k only; opts may be
 *     NULL; restart and maxit are ignored; precond_prec selects the arithmetic;
 *     csl_eps must be 0, smoother HELM_SMOOTHER_GMRES and grid->ecs_sides
 *     HELM_ECS_BOTH: HELM_EINVAL otherwise).
 *   r, z: device arrays of n^dim complex numbers in precision `prec`, natural order.
 * All working memory lives in one fixed 4 MiB device array inside the library, which
 * every GPU that loads the library holds until the process exits.  Grids whose
 * hierarchy does not fit are rejected with HELM_EINVAL and a message giving the
 * bytes needed: 2D n <= 127 and 3D n <= 31 fit in HELM_C64, 2D n <= 127 and 3D n <= 15
 * in HELM_C128; the coarsest level may hold at most 32 unknowns.
 * The first call on a device resolves the array's device address (once per device,
 * with that device current); make that first call before any stream capture.  Each
 * call clears the array, copies a few kilobytes of set-up data from host stack memory
 * (which synchronises `stream`) and enqueues three kernels on `stream`.  Every call
 * shares the one array: calls whose kernels overlap on the GPU (other streams, other
 * host threads) race and corrupt each other; serialise them on one stream.
 * The whole cycle runs in a single CTA, so it is meant for small grids. */
int helm_precond_apply_noalloc(const helm_grid* grid, double k, double theta_beta,
                               const helm_opts* opts, const void* r, void* z, int prec,
                               void* stream);

/* ---------------------------------------------------------------------------------
 * Launch tuning.  The paper has no counterpart: these choose launch parameters of the
 * V-cycle passes on this GPU.  Tuned choices live in a process-wide table keyed by
 * pass, dimension, level pitch P = n + 1, precision and Arnoldi step; every handle with
 * such a level uses them, and a choice depends on nothing else, so a problem's result
 * is the same alone and in any batch.  helm_setup reads the table once per process
 * from $HELM_TUNING or, if that is unset, tuning.json beside the library (absent: the
 * built-in defaults).  A table written on another kind of device is not used.
 * --------------------------------------------------------------------------------- */

/* Tune the launch choices of one problem's V-cycle on the current device: the tiles
 * per CTA of the 2D passes (Arnoldi steps, residual + restriction, prolongation), and
 * for 3D complex64 levels of pitch 128..1024 the TMA-fed Arnoldi pass of each step
 * (off, or on with 2..8 plane slots in flight, 2 or 4 points per thread in y, and the
 * level shared as one piece per resident CTA or as 1, 2 or 4 z pieces per column).
 * Every candidate is timed over whole V-cycles (reps cycles, best of three trials) by
 * coordinate descent from the defaults, finest level first, and kept when it makes the
 * V-cycle more than 0.5% faster.  grid, phi, k, theta_beta, opts as for helm_setup
 * (restart and maxit ignored).  The choices enter the process's table; with path
 * non-NULL the whole table, plus a record of this run, is written there as JSON.
 * default_ms / tuned_ms (may be NULL) receive the milliseconds per V-cycle before and
 * after.  Blocks until done; allocates a handle and two vectors for the duration.
 * Errors as helm_setup, HELM_EINVAL for the polynomial smoother or an unwritable path. */
int helm_autotune(const helm_grid* grid, const float* phi, double k, double theta_beta, const helm_opts* opts,
                  int reps, const char* path, double* default_ms, double* tuned_ms, void* stream);

/* Replace the process's tuned choices with the JSON table at `path` (NULL: $HELM_TUNING,
 * else tuning.json beside the library).  Host only.  HELM_EINVAL if the file is missing
 * or malformed (the current table is then kept). */
int helm_tuning_load(const char* path);

/* The tuned choice of pass "arnoldi", "restrict", "prolong", "persist" or "zplanes" on a
 * level of dimension dim and pitch P in precision prec (HELM_C64 / HELM_C128) for Arnoldi
 * step J (0 for the other passes): writes its 4 integers into v and returns 1, or
 * returns 0 when the table has none (the built-in default applies).  v: 2D passes
 * {tiles per CTA}; 3D Arnoldi {TMA-fed pass on, plane slots, z pieces per column (0: one
 * share per resident CTA), points per thread in y}; "persist" {persistent segment on};
 * "zplanes" (3D levels without the TMA-fed passes) {planes each CTA marches: 2, 4, 8 or
 * 16}.  Host only. */
int helm_tuning_get(const char* pass, int dim, int P, int prec, int J, int* v);

/* Spin limit of the grid-wide barrier between the passes of the persistent V-cycle
 * segments (the small grid-wide levels of every V-cycle run as one cooperative launch
 * per half cycle; a CTA waits at most this long for the others, then the launch
 * returns and the solve reports HELM_ETIMEOUT).  Process-wide, [0, 60] seconds, default
 * 1.  The paper has no counterpart: this bounds a wait of this GPU implementation (a
 * limit of 0 makes every waiting CTA give up at once, which tests the error path). */
int helm_set_barrier_timeout(double seconds);

/* The outer multi-dot of FGMRES (Sec. 5: the inner products h_ij = <v_i, w> of the
 * Arnoldi step) on caller data: h[i] = sum_p conj(V_i[p]) w[p], i = 0..nvec-1, through
 * the same pass a solve runs, with V and w first stored in the basis arithmetic `basis`
 * (HELM_BASIS_F64 or HELM_BASIS_DF, see helm_opts.outer_basis).  For checking the
 * orthogonalisation's accuracy apart from a solve.
 *   V:  device array of nvec vectors of npts complex128 (interleaved re, im), vector i at
 *       V + 2 i npts; w: device array of npts complex128.  Both are read only.
 *   h:  HOST array of 2 nvec doubles (complex128 results).
 *   1 <= nvec <= HELM_MAX_BASIS + 1, 1 <= npts <= 2^34.  The call allocates a
 *   workspace of about (nvec + 1) npts 16 bytes, runs on `stream` and synchronises it.
 * Errors: HELM_EINVAL (arguments), HELM_ENOMEM, HELM_ECUDA. */
int helm_multidot(int basis, const double* V, int nvec, size_t npts, const double* w, double* h, void* stream);

/* Kernels this library has launched in the process so far (all handles, all
 * streams).  The paper has no counterpart: this is launch accounting for
 * benchmarks. */
unsigned long long helm_launch_count(void);

/* Start timing every kernel launch whose class name starts with `prefix` ("" = all
 * classes) with CUDA events on its launching stream.  Class names: "vc.arnoldi.l0",
 * "vc.restrict.l0", "vc.prolong.l0", "vc.update.l0" (finest level), the same with
 * ".lc" (coarser grid-wide levels), "vc.coarse", "out.apply_h", "out.dots",
 * "out.vnew", "out.cycle_end", "io.*".  Process-wide, not thread-safe; the paper has
 * no counterpart (benchmark instrumentation). */
int helm_profile_begin(const char* prefix);

/* Stop timing, wait for the recorded events and write a JSON object
 * {"class": {"launches": n, "ms": total, "bytes": algorithmic bytes, "flops": ...}}
 * into buf (NUL-terminated, truncated to cap).  Returns HELM_OK, or HELM_EINVAL if
 * buf is NULL or cap is 0. */
int helm_profile_end(char* buf, size_t cap);

/* Thread-local text of the last error on the calling thread ("" if none). */
const char* helm_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* HELM_H */
