/*
 * mlmc.h -- C ABI of libmlmc: multilevel Monte Carlo estimation of
 * x = exp(t A) v on one GPU (GB300, sm_103a).
 *
 * Method: Acebron, Herrero, Monteiro, "A highly parallel algorithm for
 * computing the action of a matrix exponential on a vector based on a
 * multilevel Monte Carlo method".
 *   - A = D - T splitting, Sec. 2.1, Eq. 1;
 *   - Strang level approximation, Eq. 2, with dt_l = t / 2^l (Sec. 2.2);
 *   - path law: continuous-time Markov chain with exponential holding times
 *     of rate L_jj and jumps j -> k with probability |a_jk| / L_jj
 *     (Sec. 3, Eq. 12);
 *   - coupled fine/coarse walks on one path (Fig. 1, Algorithm 2);
 *   - telescoping estimator and sample sizes, Eq. 8-11, Algorithm 1.
 *
 * Conventions for every entry point
 *   - The return value is an mlmc_status; nothing throws across the ABI.
 *     On failure mlmc_last_error() returns a message for the calling thread.
 *   - Matrices are canonical CSR: row_ptr int64 [n+1] with row_ptr[0] = 0,
 *     col int32 [nnz] strictly increasing within each row (so no duplicate
 *     entries), vals float64 [nnz].  A missing diagonal entry means a_ii = 0.
 *     nnz must be below 2^31.
 *   - "Host or device" pointers may be either: the library copies through
 *     unified addressing.  Pinned host memory makes those copies faster.
 *   - All GPU work is ordered on the plan's stream (the `cuda_stream`
 *     argument of mlmc_plan_create, a cudaStream_t; NULL = legacy default
 *     stream).  Entry points that return results to the caller synchronise
 *     that stream before returning.
 *   - A plan is not thread safe: one host thread at a time per plan.
 */
#ifndef MLMC_H
#define MLMC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    MLMC_OK = 0,
    MLMC_ERR_INVALID_ARG = 1,   /* bad sizes, pointers, CSR structure, NaN/Inf */
    MLMC_ERR_CUDA = 2,          /* a CUDA runtime call failed */
    MLMC_ERR_OOM = 3,           /* device allocation failed */
    MLMC_ERR_NOT_CONVERGED = 4, /* budget exhausted; x and stats still written */
    MLMC_ERR_WALK_LIMIT = 5,    /* a walk exceeded max_jumps_per_walk */
    MLMC_ERR_NUMERIC = 6,       /* a non-finite weight was produced */
    MLMC_ERR_EXCHANGE = 7       /* a sharded solve's exchange callback failed */
} mlmc_status;

enum { MLMC_FP64 = 0, MLMC_FP32_KAHAN = 1 };   /* walk arithmetic */
enum { MLMC_BACKWARD = 0, MLMC_FORWARD = 1 };  /* estimator mode */
enum { MLMC_PLAIN = 0, MLMC_LEARNED = 1 };     /* jump proposal */

/* Level schedule and budgets (Algorithm 1 inputs).
 *   l0                coarsest level; -1 selects Eq. 16,
 *                     l0 = ceil(log2(2 t max_i max(|d_i|, L_ii))), >= 0
 *   num_levels        initial number of levels L - l0 + 1 (Algorithm 1 uses 5)
 *   max_levels        the controller adds levels up to this many
 *   pilot_walks       walks per row per level in the pilot run
 *   precision         MLMC_FP64 or MLMC_FP32_KAHAN
 *   mode              MLMC_BACKWARD (Algorithm 2 from every row) or
 *                     MLMC_FORWARD (the full-vector representation, Eq. 5:
 *                     walks on A^T from starts drawn ~|v_s|, each adding
 *                     sign(v_s) (W/w_s)|v_s| e^E to x[end]; W/w_s corrects
 *                     the integer start weights w_s = ceil(|v_s|/max|v| 2^20),
 *                     so the estimate is exact in expectation).  In forward
 *                     mode pilot_walks and max_walks_per_row are per row of
 *                     A and are multiplied by n (total walks).
 *   proposal          MLMC_PLAIN at creation (mlmc_plan_set_proposal switches
 *                     the plan to MLMC_LEARNED)
 *   max_jumps_per_walk  a walk that would exceed it stops, contributes 0 and
 *                     makes the call return MLMC_ERR_WALK_LIMIT
 *   max_walks_per_row sample budget per level (per row)
 *   time_budget_s     wall-clock budget of one mlmc_expmv call
 *   walks_per_lane    work granularity of the walk kernel (0 = automatic)
 *   block_threads     threads per block of the walk kernel (0 = automatic)
 *   l2_persist        1 (default): the walk kernels read the row records and
 *                     alias entries through an L2 access-policy window
 *                     (persisting hits, streaming misses), and plan creation
 *                     raises this process's persisting-L2 set-aside to cover
 *                     the tables up to the device maximum (never lowering it;
 *                     the set-aside belongs to the process's CUDA context and
 *                     ends with it); the hit ratio is set-aside / window.
 *                     0: plain caching.
 *   launch_reps       walks per launch: backward mode, replicas per row of one
 *                     walk launch; forward mode, walks of one launch
 *                     (0 = automatic: max(32, 2^31/n) replicas per row, or
 *                     2^31 walks; a smaller value splits a request into more
 *                     launches with the same walks and results). */
typedef struct {
    int32_t l0;
    int32_t num_levels;
    int32_t max_levels;
    int32_t precision;
    int32_t mode;
    int32_t proposal;
    int64_t pilot_walks;
    int64_t max_jumps_per_walk;
    int64_t max_walks_per_row;
    double time_budget_s;
    int32_t walks_per_lane;
    int32_t block_threads;
    int32_t l2_persist;
    int32_t launch_reps;
} mlmc_schedule;

/* Per-level statistics of the last mlmc_expmv call.
 *   level            l; dt_l = t / 2^l
 *   walks_per_row    M_l
 *   mean_norm2       ||m_l||_2^2 of the level's mean correction vector
 *   var              V_l: total variance of one sample (one walk from every
 *                    row), sum_i Var(Y_i), unbiased estimate
 *   cost_events_per_walk  mean events (holding-time draws = jumps + 1)
 *   jumps            total jumps taken at this level
 *   seconds          GPU time of this level's walk launches (CUDA events on
 *                    the plan's stream)
 *   launches         walk kernel launches at this level (a top-up is split
 *                    into launches of about 2^31 walks)
 *   still_walks      walks that ended without a jump */
typedef struct {
    int32_t level;
    int32_t pad;
    int64_t walks_per_row;
    double mean_norm2;
    double var;
    double cost_events_per_walk;
    int64_t jumps;
    double seconds;
    int64_t launches;
    int64_t still_walks;
} mlmc_level_stats;

/* One replayed walk (mlmc_trace): the state at s = 1, the number of jumps,
 * the product of jump signs phi, an FNV-1a hash of the states entered by
 * each jump (offset basis 2166136261, prime 16777619, over the 32-bit state
 * indices), the contribution y, and a status (0 ok, 1 jump limit).  `pad`
 * holds the start state in forward mode (0 in backward mode). */
typedef struct {
    int32_t end;
    int32_t jumps;
    int32_t sign;
    uint32_t hash;
    double y;
    int32_t status;
    int32_t pad;
} mlmc_walk_record;

typedef struct mlmc_plan mlmc_plan;

/* Fill *sched with the defaults: l0 = -1 (Eq. 16), num_levels = 5,
 * max_levels = 12, FP64, backward, plain, pilot_walks = 64,
 * max_jumps_per_walk = 1<<20, max_walks_per_row = 1<<34,
 * time_budget_s = 600, automatic launch shape. */
mlmc_status mlmc_schedule_default(mlmc_schedule *sched);

/* Create a plan for x = exp(t A) v (Sec. 2.1-3).  Copies the CSR matrix
 * (host or device pointers) to the device, validates it, and builds on the
 * device the per-row split quantities of Eq. 1 and the alias tables of the
 * jump law of Eq. 12.
 *   out        receives the plan (owned by the caller; free with
 *              mlmc_plan_destroy)
 *   n          matrix order, 1 <= n < 2^31
 *   nnz        stored entries, must equal row_ptr[n]
 *   t          time (the paper's beta), t >= 0, finite
 *   sched      NULL for the defaults
 *   rel_tol    target relative RMS error of mlmc_expmv, > 0
 *   cuda_stream  cudaStream_t for all work of the plan
 * Errors: INVALID_ARG for a bad CSR (row_ptr not monotone or not ending at
 * nnz, a column out of range or not strictly increasing, a non-finite
 * value), t < 0, n or nnz out of range; OOM; CUDA. */
mlmc_status mlmc_plan_create(mlmc_plan **out, int64_t n, int64_t nnz, const int64_t *row_ptr,
                             const int32_t *col, const double *vals, double t,
                             const mlmc_schedule *sched, double rel_tol, void *cuda_stream);

/* Rebuild the split quantities and alias tables from the plan's resident
 * copy of A (the same kernels as at creation).  Asynchronous on the plan's
 * stream. */
mlmc_status mlmc_plan_rebuild(mlmc_plan *plan);

/* Importance-sampling proposal for the jumps (the learned part; the paper
 * has no counterpart beyond its jump law, Eq. 12).  With h (n positive
 * finite floats, host or device, e.g. an estimate of x) every row's jump
 * law becomes the defensive mixture
 *   q_ij = (1 - alpha) |a_ij| h_j / sum_k |a_ik| h_k + alpha |a_ij| / L_ii,
 * sampled by alias tables built on the device, and every jump adds
 * log(k_ij / q_ij) to the walk's exponent, so every estimate stays unbiased
 * for any h > 0.  alpha in (0, 1].  Later walks of the plan (mlmc_expmv,
 * mlmc_mlmcl, mlmc_trace, mlmc_trace_noalloc) use the proposal; h = NULL
 * returns to the plain law.  The table build is asynchronous; h is read
 * once (the call synchronises the plan's stream to validate it). */
mlmc_status mlmc_plan_set_proposal(mlmc_plan *plan, const float *h, double alpha);

/* What a proposal tilts (mlmc_plan_set_tilt, mlmc_learn_tilt).
 * MLMC_TILT_TIME (mlmc_learn_tilt only, with both others): laws that change
 * with time (mlmc_plan_set_tilt_pieces) are candidates too. */
enum { MLMC_TILT_JUMPS = 1, MLMC_TILT_CLOCKS = 2, MLMC_TILT_TIME = 4 };

/* Proposal with the jumps alone tilted (tilt = MLMC_TILT_JUMPS: exactly
 * mlmc_plan_set_proposal) or with the holding times tilted as well
 * (tilt = MLMC_TILT_JUMPS | MLMC_TILT_CLOCKS: the h-transform of the walk;
 * the paper has no counterpart, its clocks run at the rates L_ii of Sec. 3,
 * Eq. 12).  With tilted clocks the walk holds row i for an
 * Exp(t lambda_i) time with
 *   lambda_i = sum_{j != i} |a_ij| h_j / h_i, clamped to [L_ii/1024, max(L_ii, 2/t)]
 * (0 where L_ii = 0), weights its path by exp(t int (a_ii + lambda_X) ds)
 * instead of exp(t int d_X ds), and every jump out of row i adds
 * log(L_ii / lambda_i) + log(k/q) to the exponent.  Every level then
 * estimates, without bias, the Strang product (Eq. 2) of the split
 * D' = diag(a_ii + lambda_i), T' = diag(lambda) - (A - diag(a)); like the
 * paper's split it tends to exp(tA)v as the level grows, and the
 * controller's level corrections and bias test apply unchanged.  With h
 * close to the solution the path weights nearly telescope to h(start)/h(end):
 * this removes the variance that long holding times in rows with large
 * t d_ii give the paper's walk (the hubs of a scale-free graph).  h, alpha
 * and the synchronisation as mlmc_plan_set_proposal; h = NULL returns to the
 * plain walk.  Tables: the proposal entries plus row records of the rates
 * lambda (48 bytes per row and 32 per entry in all). */
mlmc_status mlmc_plan_set_tilt(mlmc_plan *plan, const float *h, double alpha, int32_t tilt);

/* A tilted proposal that changes with time (the paper has none; it extends
 * mlmc_plan_set_tilt with MLMC_TILT_JUMPS | MLMC_TILT_CLOCKS).  The scaled
 * time s in [0, 1] is cut into `pieces` equal pieces [p/K, (p+1)/K); piece p
 * has its own law from h + p n (h: K x n positive finite floats, host or
 * device, piece-major): rates lambda_p, jump law q_p, d_p = t (a_ii +
 * lambda_p), per-jump log(L/lambda_p) + log(k/q_p) as mlmc_plan_set_tilt
 * defines them.  A pending jump time s that reaches the piece's end b is
 * carried into the next piece at its rate, s -> b + (s - b) (1/lambda_next)
 * / (1/lambda_now) in the walk's precision (the unused part of the
 * exponential clock; infinite when a rate is 0), and the grid weights of
 * Eq. 2 take each grid interval's own piece at both of its ends, so a grid
 * point on a boundary gets the mean of the two pieces' d.  Every level still
 * estimates, without bias, a Strang-type product that tends to exp(tA)v with
 * weak order 2.  With h_p close to exp((1 - s_p) tA) v, the zero-variance
 * h(s), the path weights telescope where a single h can only average over
 * time.  K = 1 is mlmc_plan_set_tilt with tilted clocks.  K must be a power
 * of two <= 16 and <= 2^l0 (every boundary a grid point of every level
 * walked; mlmc_mlmcl / mlmc_trace / mlmc_trace_noalloc refuse levels whose
 * grid misses one), on a backward-mode plan without a source term;
 * intermediate times (mlmc_expmv_times) and batches refuse such a proposal.
 * Tables: K sets (entries, row records, rates) plus one still threshold per
 * row.  h = NULL returns to the plain walk.  Synchronises. */
mlmc_status mlmc_plan_set_tilt_pieces(mlmc_plan *plan, const float *h, int32_t pieces, double alpha);

/* The installed proposal's time pieces (1 for mlmc_plan_set_tilt's laws,
 * 0 without a proposal or plan). */
int32_t mlmc_plan_tilt_pieces(const mlmc_plan *plan);

/* The tilted clocks' tables (after mlmc_plan_set_tilt with
 * MLMC_TILT_CLOCKS), as mlmc_export_tables exports the plain ones: lambda,
 * dl = t (a_ii + lambda), inv_rate = 1/(t lambda) (n doubles), their FP32
 * copies (n floats), and for FP32 plans the still thresholds of the FP32
 * walk (n int32; -1 for FP64 plans and rows that are not screened).  Any
 * pointer may be NULL.  Synchronises. */
mlmc_status mlmc_export_tilt(const mlmc_plan *plan, double *lam, double *dl, double *inv_rate,
                             float *inv_rate32, float *dl32, int32_t *still32);

/* The same for time piece `piece` of a proposal with time pieces (piece 0
 * is mlmc_export_tilt); still32 is the row's threshold for the whole law. */
mlmc_status mlmc_export_tilt_piece(const mlmc_plan *plan, int32_t piece, double *lam, double *dl,
                                   double *inv_rate, float *inv_rate32, float *dl32,
                                   int32_t *still32);

/* The h of the plan's proposal (n floats, host or device; K x n with K =
 * mlmc_plan_tilt_pieces time pieces), e.g. to give every rank of a sharded
 * solve the proposal one rank learned.  Synchronises. */
mlmc_status mlmc_export_h(const mlmc_plan *plan, float *h);

/* Checkpoint and resume of a solve (the paper has no counterpart).  The
 * state of the last mlmc_expmv / mlmc_expmv_entry / mlmc_expmv_sum call is
 * small: per level the row sums of Y, the totals (sum Y^2, jumps, walks) and
 * M_l, plus v and the seed.  mlmc_plan_save_state writes it to host memory
 * (buf NULL or cap too small: *bytes receives the size needed, and a too
 * small cap is an error); mlmc_plan_load_state restores it into a plan made
 * from the same matrix size, t, l0, precision and mode, with the same source
 * and proposal settings (anything else is INVALID_ARG).  mlmc_expmv_resume
 * continues a saved or interrupted mlmc_expmv (for example one that returned
 * MLMC_ERR_NOT_CONVERGED at its time budget) with a fresh budget: no pilot,
 * and each level's walks continue from index M_l, so with the counter-based
 * generator no walk is repeated and the samples are those an uninterrupted
 * solve would draw.  x: host or device, n doubles.  All three synchronise. */
mlmc_status mlmc_plan_save_state(const mlmc_plan *plan, void *buf, size_t cap, size_t *bytes);
mlmc_status mlmc_plan_load_state(mlmc_plan *plan, const void *buf, size_t bytes);
mlmc_status mlmc_expmv_resume(mlmc_plan *plan, double *x);

/* Source term of an inhomogeneous system du/dt = A u + F with constant F
 * (Sec. 5: the solution exp(tA) u0 + int_0^t exp(sA) F ds, the integral by
 * Simpson's rule on each level's time grid, evaluated along the same walks as
 * the exponential; Algorithm 3).  With f (n finite doubles, host or device)
 * every later walk of the plan (mlmc_expmv, mlmc_expmv_entry,
 * mlmc_expmv_sum, mlmc_mlmcl, mlmc_trace, mlmc_trace_noalloc) adds to its
 * sample t/(3N) sum_k w_k sign(t_k) eta(t_k) F[X(t_k)] over the N + 1 grid
 * points of its level (w = 1, 4, 2, ..., 4, 1; eta the Strang weight of
 * Eq. 2 at t_k) and, above l0, subtracts the same sum of level l-1 (N/2
 * steps of 2t/N), so mlmc_expmv returns the solution u(t) with u0 = v.
 * The closed form of the geometric sum over each holding segment keeps the
 * cost per walk independent of N.  Needs a backward-mode plan with l0 >= 1
 * (Simpson needs an even number of steps on every level) and no proposal;
 * mlmc_mlmcl / mlmc_trace then need level >= 1 (>= 2 when coarse).  Batches
 * do not take plans with a source.  f = NULL removes the source term.
 * Synchronises the plan's stream (f is validated on the host). */
mlmc_status mlmc_plan_set_source(mlmc_plan *plan, const double *f);

/* The proposal tables, exported like mlmc_export_tables (positions
 * row_ptr[i] + b for bucket b < deg_i), plus lr_keep / lr_alias = log(k/q)
 * of the kept and alias columns.  Any pointer may be NULL.  Synchronises. */
mlmc_status mlmc_export_proposal(const mlmc_plan *plan, uint32_t *thr, int32_t *keep_col,
                                 uint8_t *keep_neg, int32_t *alias_col, uint8_t *alias_neg,
                                 float *lr_keep, float *lr_alias);

/* The proposal tables of time piece `piece` (piece 0 is
 * mlmc_export_proposal). */
mlmc_status mlmc_export_proposal_piece(const mlmc_plan *plan, int32_t piece, uint32_t *thr,
                                       int32_t *keep_col, uint8_t *keep_neg, int32_t *alias_col,
                                       uint8_t *alias_neg, float *lr_keep, float *lr_alias);

/* x = exp(t A) v by Algorithm 1: a pilot of pilot_walks per row on levels
 * l0..l0+num_levels-1, Giles' sample sizes M_l (Eq. 11, read as
 * M_l = ceil(2/eps^2 sqrt(V_l/C_l) sum_k sqrt(V_k C_k)), eps = rel_tol ||x||),
 * top-up walks, and a new level while the bias estimate
 * max(||m_L||, ||m_{L-1}||/4)/3 exceeds eps/sqrt(2).
 *   v, x   host or device pointers to n doubles (may not alias)
 *   seed   Philox key; the same seed reproduces the same walks
 * Synchronises the plan's stream.  NOT_CONVERGED still writes x. */
mlmc_status mlmc_expmv(mlmc_plan *plan, const double *v, double *x, uint64_t seed);

/* The solution at intermediate times (Sec. 5 and Fig. 7: the paper reads the
 * heat equation's solution at the grid times of one run, and Algorithm 3
 * evaluates the Strang weight eta at every grid time of a walk):
 * x(t_k) = exp(t_k A) v for t_k = t k / n_times, k = 1..n_times, from the
 * same walks as mlmc_expmv.  A walk's sample for t_k is formed from its
 * prefix up to the fine grid point k N / n_times, exactly as its final
 * sample is from the whole path (exponents over the grid points up to it,
 * half weights at both ends, the coarse rule on the even points, v at the
 * state there); so each level's sum at t_k estimates the level-l Strang
 * product of k N/n_times steps, and the sum over levels telescopes like
 * Eq. 8.  The controller (Algorithm 1) sets M_l for the final time.
 *   x_times  host or device, n_times x n doubles, row k-1 holds x(t_k) (the
 *            last row is mlmc_expmv's x)
 *   n_times  a power of two, 2 <= n_times <= 2^l0, and at most 16 (FP32
 *            plans) or 8 (FP64 plans)
 * Backward-mode plans without a source term, not sharded.  Time sums use
 * (n_times - 1) x n doubles per level (allocated on the first call, for
 * n_times = 16).  Synchronises; NOT_CONVERGED still writes x_times. */
mlmc_status mlmc_expmv_times(mlmc_plan *plan, const double *v, double *x_times, int32_t n_times,
                             uint64_t seed);

/* mlmc_trace with the intermediate-time samples of every walk as well:
 * y_times (device, n*reps*(n_times-1) doubles) receives, for the record at
 * index r, its samples for k = 1..n_times-1 at y_times[r*(n_times-1) + k-1].
 * n_times as for mlmc_expmv_times with `level` in place of l0 (level - 1 when
 * coarse).  A walk stopped at the jump limit keeps the samples of the times
 * it passed and has 0 at the later ones.  Synchronises. */
mlmc_status mlmc_trace_times(mlmc_plan *plan, int32_t level, int32_t coarse, int64_t rep_begin,
                             int64_t reps, const double *v, uint64_t seed, int32_t n_times,
                             mlmc_walk_record *rec, double *y_times);

/* One entry x_i = (exp(t A) v)_i: Algorithm 2 as printed, walks from row i
 * only, with the controller of Algorithm 1 on the scalar (eps = rel_tol
 * |x_i|).  v: host or device, n doubles; xi: host.  This is what the paper's
 * tables measure for the heat equation (a single point). */
mlmc_status mlmc_expmv_entry(mlmc_plan *plan, int64_t i, const double *v, double *xi,
                             uint64_t seed);

/* The scalar 1^T exp(t A) v (with v = 1: the total communicability of
 * Eq. 24), to relative error rel_tol on the scalar: walks from every row,
 * eps = rel_tol |1^T x|.  total: host. */
mlmc_status mlmc_expmv_sum(mlmc_plan *plan, const double *v, double *total, uint64_t seed);

/* Statistics of the last mlmc_expmv / _entry / _sum: up to `cap` levels
 * into out (host), the level count into *n_levels and the estimated relative
 * RMS error sqrt(sum_l V_l/M_l)/|target| into *est_rel_err (either pointer
 * may be NULL). */
mlmc_status mlmc_stats(const mlmc_plan *plan, mlmc_level_stats *out, int32_t cap,
                       int32_t *n_levels, double *est_rel_err);

/* MLMCL of Algorithm 2 for every row: walks rep_begin .. rep_begin+reps-1
 * of each row at level `level` (N = 2^level steps of dt = t/N); `coarse`
 * nonzero adds the coupled level-1 weight on the same path and returns the
 * difference P_l - P_{l-1}.
 *   v        device pointer, n doubles (the right-hand side)
 *   sum_y    device pointer, n doubles: sum_y[i] += sum over the walks of Y
 *   totals   device pointer, 5 doubles: [0] += sum Y^2, [1] += jumps,
 *            [2] += walks, [3] += walks that hit the jump limit,
 *            [4] += walks that ended without a jump
 * Asynchronous on the plan's stream; uses the plan's precision.
 * Forward-mode plans: reps counts walks (not per row), rep_begin is the first
 * walk index, and each walk adds to sum_y at its end state; the call reads
 * the start-weight total back and so synchronises. */
mlmc_status mlmc_mlmcl(mlmc_plan *plan, int32_t level, int32_t coarse, int64_t rep_begin,
                       int64_t reps, const double *v, uint64_t seed, double *sum_y,
                       double *totals);

/* Replay walks rep_begin .. rep_begin+reps-1 of every row at one level and
 * record each (the same kernel and launch shape as mlmc_mlmcl, with
 * recording on).  rec: device pointer, n*reps records, index row*reps +
 * (rep - rep_begin); forward-mode plans: reps records, index g - rep_begin
 * for walk g.  Synchronises. */
mlmc_status mlmc_trace(mlmc_plan *plan, int32_t level, int32_t coarse, int64_t rep_begin,
                       int64_t reps, const double *v, uint64_t seed, mlmc_walk_record *rec);

/* mlmc_trace without device allocation.  The paper has no counterpart: this
 * is a library service.  mlmc_trace takes its scratch (per-row sums, launch
 * totals, the work counter, an FP32 copy of v) from cudaMalloc and gives it
 * back with cudaFree, and cudaFree synchronises the whole device.  A caller
 * whose device memory is reserved up front by another allocator, or that
 * cannot let a device-wide synchronisation stall its other streams, calls
 * this instead: it records the same walks with the same kernel, and its
 * scratch is a static device array of about 3 MB that every GPU loading the
 * library holds until the process exits.
 *   Arguments, record layout and results are those of mlmc_trace; rec and v
 *   are device pointers owned by the caller.
 *   n (the plan's order) must not exceed 262144 (2^18) rows, else
 *   MLMC_ERR_INVALID_ARG with a message naming the limit.
 *   The plan's device must be the current device.  The first call on a
 *   device looks up the array's device address (cudaGetSymbolAddress) and
 *   keeps it for the device's current context; a failed lookup is not kept
 *   (the next call tries again), and a call in a new context of the device
 *   (after cudaDeviceReset) looks it up again.  Make the first call on a
 *   device before any stream capture.
 *   Asynchronous on the plan's stream; makes no allocation.  Every call on a
 *   device shares the array and it keeps the previous call's contents; the
 *   call clears what must start at zero.  Calls whose GPU work overlaps (on
 *   different streams, or from different plans on one device) race on it. */
mlmc_status mlmc_trace_noalloc(mlmc_plan *plan, int32_t level, int32_t coarse, int64_t rep_begin,
                               int64_t reps, const double *v, uint64_t seed,
                               mlmc_walk_record *rec);

/* ---------------------------------------------------------------------
 * Sharded solves: one problem over several ranks (one GPU each).  The
 * paper's MPI runs (Sec. 4, Tables 6-7) give every process its share of the
 * walks and reduce the level sums between levels; here every rank holds
 * the whole plan (matrix, tables, proposal) and walks its part of each
 * level's new walk indices, and the counter-based generator makes a walk's
 * draws depend only on its index, so the union of the ranks' walks is
 * exactly the walks a one-rank solve draws.  Before each controller
 * decision (after the pilot, after each round of top-ups) the per-level row
 * sums and totals of all ranks are summed by the caller's exchange, and
 * every rank then takes the same decisions from the same numbers.
 * --------------------------------------------------------------------- */

/* Sum buf[0..count) over all ranks, in place, on every rank (an
 * all-reduce of doubles; buf is the buffer given to mlmc_plan_set_shard).
 * Called by the host thread that runs the solve, after the plan's stream
 * has been synchronised; it must finish the reduction before it returns.
 * Return 0 on success; anything else ends the solve with
 * MLMC_ERR_EXCHANGE. */
typedef int32_t (*mlmc_exchange_fn)(int64_t count, void *ctx);

/* Doubles the exchange buffer of a sharded plan must hold:
 * max_levels * (n + 8) + 1.  Returns -1 for a NULL plan. */
int64_t mlmc_shard_buffer_doubles(const mlmc_plan *plan);

/* The walk indices [*lo, *hi) of `extra` new ones that rank `rank` of
 * `world` takes: an even split in rank order, the first extra % world ranks
 * one more.  Host only (no device work). */
mlmc_status mlmc_shard_range(int64_t extra, int32_t rank, int32_t world, int64_t *lo, int64_t *hi);

/* Make later mlmc_expmv / mlmc_expmv_entry / mlmc_expmv_sum calls of this
 * plan one rank of a sharded solve (world = 1 or exchange = NULL: back to
 * an unsharded plan).
 *   rank, world  0 <= rank < world <= 65536; every rank makes the same
 *                calls with the same v, seed, schedule and proposal
 *   exchange     the all-reduce above; ctx is passed to it
 *   buf, cap     the exchange buffer, host or device memory owned by the
 *                caller, at least mlmc_shard_buffer_doubles(plan) doubles
 * Each rank's pilot and top-up walks of a level are its shard_range of the
 * level's new walk indices.  The time budget is checked at the exchanges
 * only (a top-up is not cut short) and a rank past its deadline stops every
 * rank at the next one.  Saved states and mlmc_expmv_resume are not
 * available on sharded plans.  mlmc_stats reports the whole solve. */
mlmc_status mlmc_plan_set_shard(mlmc_plan *plan, int32_t rank, int32_t world,
                                mlmc_exchange_fn exchange, void *ctx, double *buf, int64_t cap);

/* ---------------------------------------------------------------------
 * Batches: many problems solved together.  A problem is a plan with one
 * right-hand side; a plan may appear several times (several right-hand
 * sides of one matrix) and plans may differ in size and in t.
 * --------------------------------------------------------------------- */
typedef struct mlmc_batch mlmc_batch;

/* Create a batch over plans[0..count-1] (not owned; they must outlive the
 * batch, share one device and one precision).  sched supplies the level
 * schedule and budgets (NULL = the first plan's); each plan keeps its own
 * l0.  rel_tol is the per-problem target.  cuda_stream is the caller's
 * stream: mlmc_batch_expmv orders its work after work queued there.
 * Creation runs the launch-shape autotuner (walks per lane of a work item
 * from {4, 16, 64} per problem-size bucket n < 1e4, < 1e5, >= 1e5, then
 * threads per block of the round kernel from {128, 256}; a few short trial
 * launches of the round kernel on the batch's own problems) and captures the
 * CUDA graph of one round. */
mlmc_status mlmc_batch_create(mlmc_batch **out, mlmc_plan *const *plans, int32_t count,
                              const mlmc_schedule *sched, double rel_tol, void *cuda_stream);

/* x_k = exp(t_k A_k) v_k for every problem k, by Algorithm 1 run for all
 * problems in lockstep rounds.  A round is one launch of one captured
 * graph: the round's table of (problem, level, replica range) segments is
 * uploaded, one persistent walk kernel walks every segment (warps pull
 * (segment, row, chunk) items from a global counter and run the
 * single-plan walk on the segment's tables), the batched reductions follow,
 * and the host synchronises once.  v[k], x[k]: host or
 * device pointers to n_k doubles; seeds[k]: Philox key of problem k (the
 * walks are those a single-plan solve with that seed draws, with the plan's
 * jump law: its proposal when one is set).  Returns
 * NOT_CONVERGED if any problem stopped on a budget (every x is still
 * written). */
mlmc_status mlmc_batch_expmv(mlmc_batch *batch, const double *const *v, double *const *x,
                             const uint64_t *seeds);

/* Per-level statistics of problem `problem` after mlmc_batch_expmv (as
 * mlmc_stats; seconds is 0: the launches of different problems overlap). */
mlmc_status mlmc_batch_stats(const mlmc_batch *batch, int32_t problem, mlmc_level_stats *out,
                             int32_t cap, int32_t *n_levels, double *est_rel_err);

/* Rounds, GPU seconds of the rounds and number of converged problems of the
 * last mlmc_batch_expmv; any pointer may be NULL. */
mlmc_status mlmc_batch_info(const mlmc_batch *batch, int64_t *rounds, double *gpu_seconds,
                            int32_t *converged);

/* The autotuner's walks per lane for the three size buckets (cap >= 3) and,
 * with cap >= 4, the round kernel's threads per block in entry 3. */
mlmc_status mlmc_batch_autotune(const mlmc_batch *batch, int32_t *walks_per_lane, int32_t cap);

void mlmc_batch_destroy(mlmc_batch *batch);

/* ---------------------------------------------------------------------
 * The learned proposal's network (not in the paper): a 16 -> 64 -> 64 -> 1
 * MLP, BF16 weights and activations on the tensor cores (tcgen05, FP32
 * accumulation in tensor memory), FP32 master weights, Adam.  Inputs are
 * per-node features (n x 16 BF16, device), output z (n FP32, device); the
 * proposal uses h = exp(z).
 * --------------------------------------------------------------------- */
typedef struct mlmc_mlp mlmc_mlp;

/* Create an MLP with seeded initial weights; all work on cuda_stream. */
mlmc_status mlmc_mlp_create(mlmc_mlp **out, uint64_t seed, void *cuda_stream);
void mlmc_mlp_destroy(mlmc_mlp *mlp);

/* Number of FP32 parameters (packed: W1[16][64] row = input, b1[64],
 * W2[64][64] row = input, b2[64], w3[64], b3). */
int32_t mlmc_mlp_param_count(void);

/* Kernels the MLP has launched on its stream since creation (launch
 * accounting; the feature, target and proposal kernels of
 * mlmc_learn_proposal / mlmc_learn_tilt count on the plan). */
int64_t mlmc_mlp_launch_count(const mlmc_mlp *mlp);

/* Set (set != NULL) and/or read (get != NULL) the packed FP32 parameters
 * (host or device pointers).  Synchronises. */
mlmc_status mlmc_mlp_params(mlmc_mlp *mlp, const float *set, float *get);

/* z = MLP(x) for n rows: x device bf16 [n][16], z device float [n]. */
mlmc_status mlmc_mlp_forward(mlmc_mlp *mlp, const uint16_t *x, int64_t n, float *z);

/* Loss mean_i (z_i - y_i)^2 over the n rows and its gradient with respect
 * to the packed parameters (forward and backward kernels of the training
 * step; loss and grad may be host or device pointers). */
mlmc_status mlmc_mlp_loss_grad(mlmc_mlp *mlp, const uint16_t *x, const float *y, int64_t n,
                               float *loss, float *grad);

/* `steps` Adam steps (learning rate lr) on uniform minibatches of `batch`
 * rows of (x, y); *final_loss (host, may be NULL) gets the last batch loss. */
mlmc_status mlmc_mlp_train(mlmc_mlp *mlp, const uint16_t *x, const float *y, int64_t n,
                           int32_t steps, int32_t batch, float lr, uint64_t seed,
                           float *final_loss);

/* Learn and install a proposal: `pilot_walks` walks per row at l0 under the
 * plain law give per-row estimates x-hat; the MLP is trained on per-node
 * features (degree, t L_ii, t d_i, v, k^m v for m = 1..4 with k the jump
 * law, neighbour degree statistics, and the third-order Taylor value
 * sum_{m<=3} (t|A|)^m |v| / m!) to predict log(|x-hat| + 1e-3 max|x-hat|), and h = exp(MLP) is installed with
 * mlmc_plan_set_proposal(plan, h, alpha).  v: host or device, n doubles. */
mlmc_status mlmc_learn_proposal(mlmc_plan *plan, mlmc_mlp *mlp, const double *v, uint64_t seed,
                                int64_t pilot_walks, int32_t steps, int32_t batch, float lr,
                                double alpha, float *final_loss);

/* mlmc_learn_proposal generalised: `tilt` as in mlmc_plan_set_tilt, and
 * `rounds` (1..8) pilot-train-install rounds, each round after the first
 * drawing a pilot of 4 * pilot_walks walks per row (walk indices after the
 * earlier rounds' ones) with the proposal installed by the previous one.  With tilted clocks the MLP's
 * target is a log(|x-hat| + 1e-3 max|x-hat|) + (1 - a) log(|v| + 1e-3
 * max|v|) (the zero-variance h of a walk at scaled time s is exp((1-s)tA)v,
 * from x at the start to v at the end); the first pilots walk with the
 * tilts of h0 = T_3^a |v|^(1-a) for a = 1/2, 3/4 and 1, T_3 the third-order
 * Taylor value of exp(t|N|)|v| (N the off-diagonal part; the paper's walk
 * would give pilot estimates with the heavy tails the tilt removes), and
 * the form whose pilot measured the smallest variance gives the first
 * round's targets and their exponent a.  The MLP's
 * training rows are weighted by degree (row i counted 1 + floor(deg_i /
 * mean degree) times, at most 4n rows): the few rows with many
 * off-diagonals set the laws of every row around them.  Every pilot
 * measures the per-walk variance of the law it walks with (the rows' sample
 * variances averaged over the rows), and one more pilot of 4 * pilot_walks
 * walks per row measures the last round's tilt; the law with the smallest
 * measured variance is the one installed (for MLMC_TILT_JUMPS the paper's
 * walk is a candidate too: then the plan is left with the plain walk; with
 * tilted clocks the three warm starts are).  The
 * pilots draw from a stream keyed by a hash of `seed`, never the one
 * mlmc_expmv draws from with the same seed, so the installed law does not
 * depend on the walks that estimate x.  final_loss is the last round's.
 * With tilt = MLMC_TILT_JUMPS | MLMC_TILT_CLOCKS | MLMC_TILT_TIME and
 * l0 >= 1, one more law is walked and measured after the last round's: K =
 * min(8, 2^l0) time pieces (mlmc_plan_set_tilt_pieces) with h_p the same
 * Taylor value at the time left in the middle of piece p, sum_{m<=3}
 * ((1 - s_p) t|N|)^m |v| / m! (+ 1e-3 max|v|); walked last, its tables are
 * already built when it is the law installed.  It costs more per walk (its
 * carry-overs, K table sets), so it is installed only when its variance
 * times its pilot's walk time per walk (CUDA events around the launch) is
 * below the best law's: the work to reach a given error.
 * Backward-mode plans only. */
mlmc_status mlmc_learn_tilt(mlmc_plan *plan, mlmc_mlp *mlp, const double *v, uint64_t seed,
                            int64_t pilot_walks, int32_t steps, int32_t batch, float lr,
                            double alpha, int32_t tilt, int32_t rounds, float *final_loss);

/* What the plan's last mlmc_learn_tilt / mlmc_learn_proposal measured, in
 * pilot order: *count (may be NULL) pilot variances; var[k] (host, the
 * first min(cap, count)) = the per-walk variance at l0 of pilot k.  Jumps
 * only: rounds + 1 pilots (the paper's walk, then the tilt trained in each
 * round).  Tilted clocks: rounds + 3 (the warm starts a = 1/2, 3/4, 1, then
 * the tilt trained in each round), plus the time-piece law last when
 * MLMC_TILT_TIME is set and l0 >= 1.  *chosen
 * (may be NULL) = the index of the law installed (-1 before any learning). */
mlmc_status mlmc_plan_learn_report(const mlmc_plan *plan, int32_t *chosen, double *var, int32_t cap,
                                   int32_t *count);

/* Copy the device tables to host arrays (any pointer may be NULL):
 *   l_ii, dl (= t d_i), inv_rate (1/(t L_ii), +inf when L_ii = 0): n doubles
 *   inv_rate32, dl32: n floats (the FP32 copies the FP32 walk uses)
 *   deg: n int32 (off-diagonal count)
 *   thr, keep_col, alias_col: nnz entries at positions row_ptr[i] + b for
 *   bucket b < deg_i; keep_neg/alias_neg: nnz bytes (1 = negative a_ij).
 * Synchronises the plan's stream. */
mlmc_status mlmc_export_tables(const mlmc_plan *plan, double *l_ii, double *dl, double *inv_rate,
                               float *inv_rate32, float *dl32, int32_t *deg, uint32_t *thr,
                               int32_t *keep_col, uint8_t *keep_neg, int32_t *alias_col,
                               uint8_t *alias_neg);

/* Plan facts: n, nnz, the chosen l0, and t. Any pointer may be NULL. */
/* The L2 access-policy window of the plan's walk kernels (l2_persist):
 * bytes of the window (0 when off or unsupported) and the fraction of it
 * kept persisting.  Either pointer may be NULL. */
mlmc_status mlmc_plan_l2_window(const mlmc_plan *plan, int64_t *bytes, double *hit_ratio);

mlmc_status mlmc_plan_info(const mlmc_plan *plan, int64_t *n, int64_t *nnz, int32_t *l0,
                           double *t);

/* Free the plan and all its device memory (NULL is a no-op). */
void mlmc_plan_destroy(mlmc_plan *plan);

/* Message for the last failure on the calling thread ("" if none). */
const char *mlmc_last_error(void);

/* Kernels launched on the plan's stream since creation (all of this
 * library's kernels, for launch accounting). */
int64_t mlmc_launch_count(const mlmc_plan *plan);

#ifdef __cplusplus
}
#endif

#endif /* MLMC_H */
