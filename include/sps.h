/*
 * sps.h -- C ABI of the GB300 (sm_103a) tensor-product spline smoothing solver.
 *
 * The library fits a tensor-product B-spline s(x) = sum_k alpha_k phi_k(x) to
 * scattered data (x_i, y_i) in R^P x R by solving the penalised normal
 * equations (Phi'Phi + lambda Lambda) alpha = Phi'y (Siebenborn & Wagner,
 * arXiv:1901.00654, Section 2.2, the linear system after the smoothing
 * spline problem) with the multigrid-preconditioned conjugate gradient method
 * of Algorithm 8, whose preconditioner is the V-cycle of Algorithm 7 with the
 * damped Jacobi smoother of Algorithm 6.  Every operator is applied matrix
 * free on the GPU: Phi v and Phi'u by the Khatri-Rao products of Algorithms 3
 * and 4 (fused into one point operator), Lambda v and the grid transfers by
 * the Kronecker structure of Algorithm 2.
 *
 * Conventions shared by every call:
 *  - Coefficients are stored row-major over the multi-index (j_1, ..., j_P)
 *    with the LAST dimension fastest; j_p = 0 .. N_p + q - 1 where N_p is the
 *    number of knot intervals of dimension p on that grid level.  Basis
 *    function j_p is the cardinal B-spline on [lo + (j_p - q) h, lo + (j_p + 1) h]
 *    (extended uniform knots, h = (hi - lo) / N_p).
 *  - Points are passed as an n x P row-major array (x[i*P + p]).
 *  - `mem` says where a buffer lives: SPS_MEM_HOST (ordinary or pinned host
 *    memory) or SPS_MEM_DEVICE (device memory of the plan's GPU).
 *  - `stream` is a cudaStream_t (NULL = the legacy default stream).  Calls
 *    that return results in host memory synchronise that stream before
 *    returning; calls with device outputs are asynchronous with respect to the
 *    host except where stated.
 *  - Every call returns 0 (SPS_OK) or a negative SPS_E* code; no call aborts
 *    or throws.  sps_last_error() gives a message for the calling thread's
 *    most recent failure.
 *  - Ownership: the caller owns every buffer it passes; the plan owns all of
 *    its device memory until sps_destroy.  The library copies what it keeps.
 *  - Level numbers follow the paper: g = 1 is the coarsest grid, g = G (the
 *    `levels` argument of sps_plan_create) the finest.
 */
#ifndef SPS_H
#define SPS_H

#include <stdint.h>

#if defined(__GNUC__)
#define SPS_API __attribute__((visibility("default")))
#else
#define SPS_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---- */
#define SPS_OK            0
#define SPS_EINVAL       -1  /* invalid argument (P, q, N_p, levels, lambda, sizes, pointers) */
#define SPS_EDOM         -2  /* a point lies outside [lo, hi] or is not finite */
#define SPS_ENOMEM       -3  /* device or host allocation failed */
#define SPS_ESTATE       -4  /* call out of order (e.g. solve before set_points) */
#define SPS_EBREAKDOWN   -5  /* CG breakdown: p'Ap <= 0 or a non-finite scalar */
#define SPS_ENOCONV      -6  /* max_iter reached; coef holds the last iterate */
#define SPS_ETIMEOUT     -7  /* a device-side loop hit its iteration cap */
#define SPS_ECUDA        -8  /* a CUDA runtime call failed */
#define SPS_EEMPTY       -9  /* no data points (n = 0) */
#define SPS_EINTERNAL   -10  /* a kernel found its launch inconsistent with its input
                                (a library bug) and skipped work; results are invalid */

/* ---- enums ---- */
#define SPS_F32 0            /* float  inputs */
#define SPS_F64 1            /* double inputs */
#define SPS_MEM_HOST   0
#define SPS_MEM_DEVICE 1
#define SPS_PREC_FP64  0     /* every step in FP64 (plain method): basis values,
                                products, sums, the assembled coarse and
                                intermediate-level matrices, the coarse solve */
#define SPS_PREC_MIXED 1     /* FP32 V-cycle and FP32 point operator inside an FP64
                                flexible PCG with FP64 residual replacement */

#define SPS_MAX_DIM    5     /* P <= 5 */
#define SPS_MAX_LEVELS 12

typedef struct sps_plan sps_plan;       /* opaque; owned by the library */

typedef struct sps_options {
    int    precision;      /* SPS_PREC_FP64 (default) or SPS_PREC_MIXED */
    int    nu1, nu2;       /* pre/post Jacobi sweeps per level (default 1, 1) */
    double omega;          /* Jacobi damping; <= 0 (default): per level
                              1.8 / lambda_hat, lambda_hat an upper estimate of
                              lambda_max(D_g^-1 A_g) by Lanczos (top Ritz value
                              plus its residual bound) */
    int    power_iters;    /* Lanczos steps for lambda_hat (default 20, at most 32) */
    int    max_iter;       /* outer iteration cap (default 20000) */
    int    warm_start;     /* 1: coef passed to sps_solve is the initial guess */
    int    tile;           /* tile side in cells, 0 = automatic per P */
    double replace_ratio;  /* MIXED: recompute the FP64 residual when |r| has
                              dropped by this factor since the last recompute
                              (default 1e-2) */
    int    hybrid;         /* 1 (default): levels between the coarsest and the
                              finest whose assembled (2q+1)^P-stencil matrix is
                              cheaper to apply than a point sweep are assembled
                              once in sps_set_points (same matrix A_g); 0: every
                              level matrix free */
    int    graphs;         /* 1 (default): each PCG iteration after the first is
                              replayed from a CUDA graph captured once per set-up;
                              0: launched kernel by kernel */
    int    precondition;   /* 1 (default): the multigrid V-cycle of Algorithm 7;
                              0: none, i.e. plain CG, the comparison method of
                              Section 4 (Table 2, Fig. 2) */
    int    autotune;       /* 1: on the plan's first sps_set_points, time the
                              point operator of every matrix-free level with
                              tile sides ts/2, ts, 2ts (and, for P = 3, 4, both
                              lane layouts per run) and keep
                              the fastest; the operator is the same matrix.
                              0 (default): fixed tile side per P */
    int    lanes_r;        /* apply of the point operator for P = 3, 4 (FP32,
                              and FP64 on levels with precomputed basis values):
                              dimensions of a run's (q+1)^P coefficients held in
                              one lane's registers, 2 (4^(P-2) lanes per run,
                              16 sums each) or 3 (4^(P-3) lanes, 64 sums);
                              0 (default): FP32 2 for P = 3, else 3.  Ignored
                              for other P; the autotuner may change it */
    int    coarse_cg;      /* coarse grid solver on level 1 (Section 3.2, coarse grid
                              solver): 0 (default) the dense inverse of the assembled
                              A_1, formed from its Jacobi-scaled form (K_1 <= 4096);
                              1 an inner matrix-free Jacobi-preconditioned CG on A_1
                              (no assembly, no K_1 limit), run for coarse_iters
                              iterations per coarse solve.  The inner CG makes the
                              V-cycle a nonlinear preconditioner, so the outer
                              iteration then uses the flexible (Polak-Ribiere) beta */
    int    coarse_iters;   /* inner CG iterations per coarse solve (default 32) */
    int64_t max_device_bytes; /* 0 (default): no limit; else the plan's device memory
                              (plan buffers, point data and call temporaries) may not
                              exceed this many bytes: an allocation beyond it fails
                              with SPS_ENOMEM before cudaMalloc is called */
} sps_options;

typedef struct sps_result {
    int    status;         /* SPS_OK, SPS_ENOCONV or SPS_EBREAKDOWN */
    int    iterations;     /* outer CG iterations (operator applies on level G) */
    double rel_res;        /* |r| / |Phi'y| of the recursive residual at exit */
    double rel_res_true;   /* |Phi'y - A alpha| / |Phi'y| recomputed in FP64 at exit */
    int    fp64_applies;   /* FP64 applies on level G (MIXED: residual replacements, plus
                              one per iteration after a fallback to the FP64 outer
                              operator, which an FP32 breakdown triggers) */
    double solve_ms;       /* wall time of sps_solve (host clock) */
} sps_result;

/* Fill *opt with the defaults listed above (where the paper leaves a parameter
 * unstated -- nu1, nu2, omega, the stopping rule -- these are this library's readings). */
SPS_API void sps_default_options(sps_options* opt);

/* Create a plan for P-dimensional cubic (q = 3) tensor-product splines.
 *  intervals[P]: knot intervals N_p of the finest grid, each a power of two,
 *                N_p >= 2^(levels-1) so the coarsest grid has >= 1 interval.
 *  lo, hi [P]:   domain Omega = prod [lo_p, hi_p] (NULL -> 0 and 1).
 *  levels:       number of grid levels G >= 1 (Section 3.2, hierarchy); the
 *                coarsest has K_1 = prod (N_p / 2^(G-1) + 3) <= 4096 coefficients
 *                when it is solved densely (sps_options.coarse_cg = 0), and
 *                P * log2(max_p N_p) <= 26.
 *  lambda:       smoothing parameter >= 0 (0 gives the least-squares spline,
 *                which is SPD only when every basis support holds enough data;
 *                otherwise the solve reports SPS_EBREAKDOWN).
 *  q:            the spline degree; only cubic splines (q = 3) are built, the
 *                degree of every workload here (any other q: SPS_EINVAL).
 *  opt:          NULL for defaults.
 * Allocates the per-level coefficient vectors on the current CUDA device.
 * Errors: SPS_EINVAL, SPS_ENOMEM, SPS_ECUDA. */
SPS_API int sps_plan_create(sps_plan** out, int P, int q, const int* intervals, const double* lo,
                    const double* hi, int levels, double lambda, const sps_options* opt);

/* Load the data (x_i, y_i), i < n: copies them to the device, validates that
 * every coordinate is finite and inside [lo_p, hi_p] and every response is
 * finite, sorts the points by the
 * Morton key of their finest knot cell (stable), builds the per-level work
 * lists, computes diag(A_g) (Algorithm 5 plus the penalty diagonal), the
 * right-hand side Phi'y (Algorithm 3), the coarse matrix and its inverse, and
 * omega.  x: n x P row-major, y: n, both of `dtype`, in `mem`.
 * The caller may free x and y once the call returns.  Synchronises `stream`.
 * Host inputs (mem = SPS_MEM_HOST) pass through a device copy that the call
 * allocates and frees (cudaFree synchronises the device); callers on a
 * latency-critical path pass device buffers instead.
 * Errors: SPS_EINVAL, SPS_EEMPTY (n == 0), SPS_EDOM (a coordinate outside the
 * domain, or a coordinate or response not finite), SPS_ENOMEM, SPS_EBREAKDOWN
 * (the Lanczos estimate for omega found no positive eigenvalue), SPS_ECUDA,
 * SPS_EINTERNAL. */
SPS_API int sps_set_points(sps_plan* plan, int64_t n, const void* x, const void* y, int dtype, int mem,
                   void* stream);

/* Solve (Phi'Phi + lambda Lambda) alpha = Phi'y to |r| <= tol |Phi'y| by
 * Algorithm 8 (FP64) or its mixed-precision flexible variant.  coef: K_G
 * doubles in `mem` (input = initial guess when opt.warm_start; output = alpha).
 * res may be NULL.  Synchronises `stream`.
 * Errors: SPS_ESTATE (no points), SPS_EINVAL, SPS_ENOCONV (max_iter reached,
 * or a residual that is not finite after the iteration stopped; res is filled
 * and coef holds the last iterate), SPS_EBREAKDOWN (p'Ap <= 0 or a non-finite
 * step), SPS_ECUDA, SPS_EINTERNAL. */
SPS_API int sps_solve(sps_plan* plan, double* coef, int mem, double tol, sps_result* res, void* stream);

/* Change lambda, the penalty weight of Section 2.2, of a plan; takes effect at
 * the next sps_set_points (which
 * recomputes the right-hand side, diagonals, coarse matrix and damping).
 * Lets a pool of plans of one grid shape serve problems with different
 * lambda without new allocations.  Errors: SPS_EINVAL. */
SPS_API int sps_set_lambda(sps_plan* plan, double lambda);

/* Release the plan and all of its device memory.  NULL is accepted.  (Plan
 * lifetime: no counterpart in the paper.) */
SPS_API int sps_destroy(sps_plan* plan);

/* Thread-local message of the last failure (never NULL; no counterpart in the paper). */
SPS_API const char* sps_last_error(void);

/* Launch shape of the batched solver (not a step of the paper's method).  The
 * costliest problems of a batch are solved each by a thread-block cluster of
 * `cluster` CTAs (their loops split across the CTAs, dot products through
 * distributed shared memory), the rest by one CTA each. */
typedef struct sps_batch_shape {
    int    cluster;        /* CTAs per cluster: 1 (no clusters), 2, 4 or 8 */
    int    big;            /* the `big` costliest problems go to clusters; -1: those
                              whose cost exceeds the batch's total cost per CTA */
    double predicted_ms;   /* sps_tune_batch: simulated batch time of this shape */
} sps_batch_shape;

/* Solve `count` independent problems in ONE persistent kernel launch captured
 * in a CUDA graph, running the mixed-precision flexible PCG of Algorithm 8
 * with the FP32 V-cycle of Algorithm 7 inside the kernel.  Problems are taken
 * from device queues in decreasing cost order: first the costliest by
 * thread-block clusters, then the rest by single CTAs.  The shape is the one
 * sps_tune_batch chose for a batch of the same problems (same count and, per
 * problem, P, K and n) if it was tuned, else clusters of 2 CTAs for the problems
 * costing more than the batch's total cost per CTA.  Results agree with
 * sps_solve to the solve's tolerance (the summation order differs).  plans[i]
 * must have P <= 3, the dense coarse solver and points set; coefs[i] receives
 * K_G(i) doubles in `mem`; tol is shared; results may be NULL (else `count`
 * entries).  Each plan's buffers are used, so a plan must not be in another
 * call at the same time.  Returns the first non-OK status among the problems
 * (all are attempted).  Synchronises `stream`. */
SPS_API int sps_solve_batch(sps_plan* const* plans, int count, double* const* coefs, int mem, double tol,
                            sps_result* results, void* stream);

/* sps_solve_batch (many problems of Algorithm 8 in one launch; not in the
 * paper) with an explicit launch shape (shape may be NULL: as
 * sps_solve_batch); *used (may be NULL) receives the shape that ran (a cluster
 * size that cannot be resident on the device falls back to 1). */
SPS_API int sps_solve_batch_shape(sps_plan* const* plans, int count, double* const* coefs, int mem, double tol,
                                  const sps_batch_shape* shape, sps_result* results, sps_batch_shape* used,
                                  void* stream);

/* Autotuner of the batched solver's shape (not in the paper): solves the batch once for every
 * cluster size 1, 2, 4, 8 with every problem on a team of that size, keeps
 * each problem's measured time per size, and picks the cluster size and the
 * number of problems solved by clusters whose simulated batch time (the two
 * device queues replayed with the measured times) is the shortest.  The pick
 * is returned in *best and used by later sps_solve_batch calls on the same
 * problems; coefs receive the coefficients of the last tuning solve.
 * Errors: as sps_solve_batch. */
SPS_API int sps_tune_batch(sps_plan* const* plans, int count, double* const* coefs, int mem, double tol,
                           sps_batch_shape* best, void* stream);

/* The model the batch autotuner minimises (host only; the batched solver has
 * no counterpart in the paper): the makespan in ms of the persistent queues
 * of sps_solve_batch_shape for measured per-problem times, t1[i] on a single
 * CTA and tc[i] on a team of `cluster` CTAs (host arrays of n).  `grid` CTAs
 * form grid / cluster teams, which take the first `big` problems of `order`
 * (a permutation of 0 .. n-1, costliest first) with times tc; a team that
 * finds that queue empty splits into single CTAs, which take the remaining
 * problems in order with times t1.  cluster = 1: single CTAs take every
 * problem (big is ignored).  cluster in {1, 2, 4, 8}, grid >= cluster,
 * 0 <= big <= n; SPS_EINVAL otherwise. */
SPS_API int sps_simulate_batch(const int* order, const double* t1, const double* tc, int n, int cluster, int big,
                               int grid, double* makespan_ms);

/* Values s(x_j) = sum_k alpha_k phi_k(x_j) of the spline with coefficients
 * `coef` at m query points: Algorithm 4 (transposed Khatri-Rao product) with
 * the query points in place of the data, on the finest grid of the plan
 * (Sections 2.1, 2.2) -- how a fitted smoothing spline is used to predict.
 * coef: K_G doubles (the layout of sps_solve); xq: m x P row-major, dtype
 * SPS_F32 or SPS_F64; out: m doubles; all three in `mem`.  Needs only
 * sps_plan_create (no points).  A point on x = hi belongs to the last cell.
 * Errors: SPS_EINVAL; SPS_EDOM if a query point is outside [lo, hi] or not
 * finite (its value is NaN, the others are evaluated).  m = 0 does nothing.
 * Synchronises `stream`. */
SPS_API int sps_evaluate(sps_plan* plan, const double* coef, int64_t m, const void* xq, int dtype, double* out,
                         int mem, void* stream);

/* Launch shape of level `level`'s point operator (after sps_set_points):
 * tile side in cells and, for the FP32 apply, the dimensions held in one
 * lane's registers (2 or 3; 0 = the default for P).  Not a step of the
 * paper's method: it reports what sps_options.autotune chose.
 * Errors: SPS_EINVAL (NULL or level out of range). */
SPS_API int sps_get_tuning(const sps_plan* plan, int level, int* tile, int* lanes_r);

/* Device memory the plan holds now, in bytes (its buffers and point data).
 * Not a step of the paper's method: serving admits requests by it.
 * Errors: SPS_EINVAL (NULL argument). */
SPS_API int sps_plan_device_bytes(const sps_plan* plan, int64_t* bytes);

/* ---------------- component entry points (each one step of the solve) ----------------
 * All vectors are doubles in `mem`; `prec` selects the FP64 kernels
 * (SPS_PREC_FP64) or the FP32 kernels of the mixed mode (SPS_PREC_MIXED, inputs
 * rounded to FP32 and results widened).  They require sps_set_points and
 * synchronise `stream` when an output is in host memory. */

/* K_g = prod_p (N_p^(g) + q), the number of coefficients on level g (1 <= g <= G;
 * Section 3.2 hierarchy, Table 1 for the finest level). */
SPS_API int sps_coef_count(const sps_plan* plan, int level, int64_t* K);

/* u = (Phi_g'Phi_g + lambda Lambda_g) v on level g, with all n points
 * (Section 3.2, hierarchy; Algorithms 2-4).  v, u: K_g. */
SPS_API int sps_apply(sps_plan* plan, int level, int prec, const double* v, double* u, int mem, void* stream);

/* u = Phi_g'(Phi_g v) alone: the fused point operator of Algorithms 3 and 4
 * (no penalty), on level g with all n points.  v, u: K_g. */
SPS_API int sps_point_apply(sps_plan* plan, int level, int prec, const double* v, double* u, int mem,
                            void* stream);

/* u = Lambda_g v (penalty alone, Section 2.2; Kronecker sums of Algorithm 2). */
SPS_API int sps_penalty_apply(sps_plan* plan, int level, int prec, const double* v, double* u, int mem,
                      void* stream);

/* d = diag(Phi_g'Phi_g + lambda Lambda_g) (Algorithm 5 plus the penalty diagonal). */
SPS_API int sps_diag(sps_plan* plan, int level, double* d, int mem, void* stream);

/* b = Phi_G'y (Algorithm 3 with the responses). */
SPS_API int sps_rhs(sps_plan* plan, double* b, int mem, void* stream);

/* f = I_{g-1}^{g} c (prolongation, Section 2.4 subdivision matrix, Kronecker
 * form); c: K_{g-1}, f: K_g, 2 <= g <= G. */
SPS_API int sps_prolong(sps_plan* plan, int level, int prec, const double* c, double* f, int mem, void* stream);

/* c = (I_{g-1}^{g})' f (restriction, Section 3.2 grid transfer); f: K_g, c: K_{g-1}. */
SPS_API int sps_restrict(sps_plan* plan, int level, int prec, const double* f, double* c, int mem, void* stream);

/* e = A_1^{-1} r on the coarsest level (Section 3.2, coarse grid solver), by the
 * plan's coarse solver (sps_options.coarse_cg).  In FP64 plans the dense path
 * is the GEMV with the inverse followed by one step of iterative refinement
 * with the assembled A_1 (FP64 residual). */
SPS_API int sps_coarse_solve(sps_plan* plan, const double* r, double* e, int mem, void* stream);

/* Assembled operator A_g = Phi_g'Phi_g + lambda Lambda_g of level g as the
 * solver holds it (Section 3.2, hierarchy; Algorithm 5 for the diagonal):
 *  g = 1 with the dense coarse solver: the dense K_1 x K_1 matrix, row-major;
 *  an intermediate level assembled in stencil form (sps_options.hybrid): the
 *  offset-major stencil out[s * K_g + k] = A_g(k, k + offset_s), s < 7^P, with
 *  offset_s the base-7 digits of s minus 3 (last dimension fastest); entries
 *  whose column falls outside the grid are 0.
 * *entries receives the number of doubles (0 when the level is applied matrix
 * free; out is then untouched); out may be NULL to query the count.  Values
 * are those the solver uses (FP64 plans: FP64; mixed plans keep FP32 stencils,
 * returned widened).  Errors: SPS_ESTATE, SPS_EINVAL. */
SPS_API int sps_level_matrix(sps_plan* plan, int level, double* out, int64_t* entries, int mem, void* stream);

/* z = one V-cycle (Algorithm 7) from zero applied to r on level G. */
SPS_API int sps_vcycle(sps_plan* plan, int prec, const double* r, double* z, int mem, void* stream);

/* The stable sort of the points: perm[i] = original index of the i-th sorted
 * point and key[i] its Morton key (either pointer may be NULL); n entries.
 * The cell of a point follows from the B-spline supports (Section 2.1); the
 * sort by cell is this library's work decomposition, not the paper's. */
SPS_API int sps_get_sort(sps_plan* plan, int64_t* perm, uint64_t* key, int mem, void* stream);

/* Jacobi damping omega_g of Algorithm 6 (not given in the paper) for g = 1..G
 * (omega[g-1]); host memory. */
SPS_API int sps_get_omega(const sps_plan* plan, double* omega);

/* Override omega_g of Algorithm 6 (host array of G values, all > 0). */
SPS_API int sps_set_omega(sps_plan* plan, const double* omega);

/* Host part of the Jacobi damping estimate (Section 3.2, smoothing iteration;
 * Algorithm 6's omega is not given in the paper): from m Lanczos coefficients
 * of D_g^-1/2 A_g D_g^-1/2 -- alpha[j] and beta2[j] = beta_j^2, j < m, host
 * arrays -- theta, the largest eigenvalue of the tridiagonal T_m (diagonal
 * alpha, off-diagonal beta_0 .. beta_{m-2}), and lambda_hat = theta +
 * beta_{m-1} |s_m| (s the unit eigenvector of T_m for theta), the upper
 * estimate of lambda_max that sps_set_points turns into omega_g = 1.8 /
 * lambda_hat.  Host-only (no device work).  SPS_EINVAL for null pointers or
 * m outside 1..32, SPS_EBREAKDOWN for non-finite input or theta <= 0. */
SPS_API int sps_lanczos_estimate(const double* alpha, const double* beta2, int m, double* theta,
                                 double* lambda_hat);

/* Measurement hook (no counterpart in the paper).  Kernel timing of the point
 * operator of Algorithms 3 and 4 (the dominant kernel): between
 * sps_profile_begin and sps_profile_end every launch of the point operator in
 * its apply mode is bracketed by CUDA events on its stream (at most 8192
 * launches are timed).  sps_profile_end synchronises those events and returns
 * the summed duration in ms and the number of timed launches. */
SPS_API int sps_profile_begin(void);
SPS_API int sps_profile_end(double* point_apply_ms, uint64_t* point_apply_launches);

/* ---------------- no-allocation variant ----------------
 * The paper has no counterpart of this entry point; it exists for callers
 * that must not allocate device memory: code running inside another
 * framework whose caching allocator has reserved the GPU's memory, or
 * latency-critical loops where cudaMalloc/cudaFree (and cudaFree's implicit
 * device-wide synchronisation) are not acceptable.  It computes the same
 * u = scale * Lambda v as sps_penalty_apply, but for a grid passed directly
 * (no plan, which would allocate) and with its temporaries in one fixed
 * device array of 6 * SPS_NOALLOC_MAX_COEF doubles (12 MiB) that every GPU
 * which loads the library holds until the process exits.
 *  P, intervals[P], lo/hi[P] (NULL -> 0, 1): the grid, as in sps_plan_create
 *  (intervals need not be powers of two here); K = prod (N_p + 3) must be
 *  <= SPS_NOALLOC_MAX_COEF, larger grids are rejected with SPS_EINVAL.
 *  v, u: K doubles in DEVICE memory (u is overwritten); stream: cudaStream_t.
 *  u must not overlap v (SPS_EINVAL).
 * It calls no cudaMalloc, cudaFree or allocating library routine.  All calls
 * share the one scratch array, so calls that overlap on the GPU (other
 * streams or host threads) race; the scratch needs no clearing because every
 * step writes the entries it later reads.  The first call on a device sets up
 * (looks up the scratch address with cudaGetSymbolAddress and uploads the
 * cubic element matrices to constant memory); make that first call before any
 * stream capture.  Under CUDA's default lazy module loading the 12 MiB array
 * is taken on a device at that first call, not when the library loads (with
 * CUDA_MODULE_LOADING=EAGER: at load): a caller about to hand the GPU's memory
 * to another allocator makes one call first.  The set-up is not redone after
 * cudaDeviceReset: do not use the entry point on a device after a reset.
 * Errors: SPS_EINVAL, SPS_ECUDA. */
#define SPS_NOALLOC_MAX_COEF 262144
SPS_API int sps_penalty_apply_noalloc(int P, const int* intervals, const double* lo, const double* hi,
                                      double scale, const double* v, double* u, void* stream);

/* Number of CUDA kernels this library has launched in this process so far
 * (measurement hook; no counterpart in the paper). */
SPS_API int sps_launch_count(uint64_t* count);

/* Timing probe (no counterpart in the paper; the roofline denominator of the
 * point operator): measured FMA throughput of the device in FMA/s for FP32
 * (fp=0) or FP64 (fp=1), from a register-resident FMA loop over all SMs. */
SPS_API int sps_probe_fma_rate(int fp, double* fma_per_s, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* SPS_H */
