/*
 * mpk.h - C ABI of the GB300 level-blocked matrix power kernel (MPK) library.
 *
 * What it computes (arXiv 2309.02228, "Algebraic Temporal Blocking for Sparse Iterative
 * Solvers on Multi-Core CPUs"):
 *   - Sec. 3, Alg. 1: the MPK, y_p = A^p x for p = 1..p_m into p_m vectors, here generalised
 *     to the three-term recurrence y_k = a_k (A y_{k-1}) + b_k y_{k-1} + c_k y_{k-2} that covers
 *     the monomial basis, the Newton basis of Sec. 4 (a=1, b=-theta_k, c=0) and the Chebyshev
 *     basis of the polynomial smoother of Sec. 5.3 (three-term Chebyshev recursion).
 *   - Sec. 3: temporal cache blocking by the level structure of a BFS on the graph of A and a
 *     cache-size parameter C (levels grouped so that the working set of a p-deep wavefront
 *     fits the cache); here the cache is the GPU's L2.
 *   - Sec. 4, Alg. 3(c): s-step GMRES (MPK, block orthogonalisation, TSQR, convergence check),
 *     with the MPK in the Newton basis.
 * The paper is a CPU (OpenMP) study; this library is a single-GPU (sm_103a) design of the same
 * method.  Everything runs in the library's own CUDA kernels; the host code only orders launches.
 *
 * Conventions for every entry point:
 *   - Pointers named d_* or documented "device" are device pointers; "host" ones are host.
 *   - Sizes are element counts.  Indices are 32-bit (Sec. 2.2: 32-bit integers), so
 *     n < 2^31 and nnz < 2^31.
 *   - Calls are asynchronous on the given stream unless stated otherwise; a NULL stream means
 *     the legacy default stream.  Every call returns an mpk_status; no exception crosses the ABI.
 *   - Errors detected on the device (a dependency wait that ran out) are latched in the plan
 *     and returned by mpk_plan_sync(), which also clears them.
 *   - The caller owns every buffer it passes; a plan owns its own device copies.
 *   - One plan must not be used from two streams at the same time: it holds the workspace and
 *     the dependency flags of its launches.
 */
#ifndef MPK_GB300_H
#define MPK_GB300_H

#include <stdint.h>
#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    MPK_OK = 0,
    MPK_ERR_ARG = 1,            /* invalid argument (null pointer, size, flag combination) */
    MPK_ERR_CUDA = 2,           /* a CUDA runtime call failed */
    MPK_ERR_OOM = 3,            /* device allocation failed */
    MPK_ERR_TIMEOUT = 4,        /* a bounded device-side wait ran out; results are invalid */
    MPK_ERR_BREAKDOWN = 5,      /* Cholesky of a Gram matrix met a non-positive pivot */
    MPK_ERR_NOT_CONVERGED = 6,  /* solver stopped at its iteration limit */
    MPK_ERR_UNIMPLEMENTED = 7,  /* a combination this build does not support */
    MPK_ERR_BUDGET = 8,         /* serving: the request can never fit the memory budget */
    MPK_ERR_NOT_READY = 9       /* serving: nothing completed yet */
} mpk_status;

typedef enum { MPK_F32 = 0, MPK_F64 = 1 } mpk_dtype;

/* A square sparse matrix in CRS/CSR form (Sec. 2.2, Alg. 1: val[nnz], col[nnz],
 * rowPtr[n+1]).  DEVICE pointers, caller-owned; columns need not be sorted; duplicate
 * entries are kept (and summed by the SpMV).  mpk_plan_create copies what it needs, so the
 * arrays may be freed once it returns (after a stream synchronise). */
typedef struct {
    int64_t n;
    int64_t nnz;
    const int32_t *row_ptr;   /* n+1 entries, row_ptr[0] = 0, non-decreasing */
    const int32_t *col;       /* nnz entries in [0, n) */
    const void *val;          /* nnz entries of type dtype */
    mpk_dtype dtype;
} mpk_csr;

/* Plan options (mpk_plan_opts_default fills the defaults). */
typedef struct {
    int64_t l2_budget_bytes;  /* level-group budget, the analogue of the paper's cache size
                                 C (Sec. 4: C = 85 / 200 MB on its CPUs).  0 = half the L2. */
    int32_t p_blk;            /* blocking depth the groups are sized for and the longest
                                 segment one blocked launch runs (the paper's p_opt,
                                 Sec. 3); 0 = p_max. */
    int32_t root_rule;        /* 0 = George-Liu pseudo-peripheral root from row 0,
                                 1 = row 0 */
    int32_t n_sweeps;         /* George-Liu re-root sweeps (default 2) */
    int32_t assume_symmetric; /* 1 = the pattern is structurally symmetric; skips building
                                 A^T for the BFS and the dependency closure */
    int32_t chunk_slices;     /* 32-row slices per blocked task (default 8) */
    int32_t keep_f32;         /* keep an FP32 copy of the values (MPK in FP32) */
    int32_t keep_f64;         /* keep an FP64 copy of the values (MPK / residual in FP64) */
    int32_t ctas_per_sm;      /* persistent CTAs per SM for the blocked kernel (0 = auto:
                                 3 CTA-task CTAs, or as many warp-task CTAs as fit) */
    uint32_t wait_timeout_us; /* bound on every device-side dependency wait (default 2e6) */
    int32_t schedule;         /* blocked task order: 0 = level-group wavefront (step t runs
                                 group t-k+1 at power k), 1 = lag-greedy (default: a power
                                 advances once its dependencies were issued slack_tasks
                                 tickets earlier) */
    int32_t slack_tasks;      /* lag-greedy slack in tasks; 0 = the number of resident CTAs
                                 (CTA tasks), 128 per SM (warp tasks) or three per resident
                                 warp (lane tasks) */
    int32_t block_threads;    /* compute threads per CTA of the blocked kernel: 128 or 256
                                 (default); one control warp is added */
    int32_t stage;            /* CTA-task kernel only: stage each task's matrix block
                                 (columns and values) in shared memory with bulk asynchronous
                                 copies: -1 auto (on unless a 32-row slice exceeds a slot),
                                 0 off */
    int32_t kernel;           /* blocked kernel: 0 = warp tasks (every warp takes
                                 tasks from a ticket dispenser and waits on per-block
                                 completion counters), 1 = CTA tasks fed by a control warp,
                                 2 = warp tasks in static round robin, 3 = ready-first warp
                                 tasks (no schedule: a warp claims, highest power first, the
                                 next chunk of a power whose dependencies are complete, else
                                 the next chunk of power 1; claimed tasks never wait; chunks
                                 are dealt to interleaved shards, each with its own cursors),
                                 4 = lane tasks (the default; single right-hand side, not
                                 MPK_GS2; other calls run kernel 0): tasks of task_units
                                 sub-slices of
                                 32 / lanes_per_row rows, in lag-greedy order, dealt round
                                 robin to the CTAs and inside a CTA to whichever warp is free
                                 (a shared-memory counter: no global atomic per task), waiting
                                 on per-block completion counters; lanes_per_row > 1 selects
                                 this kernel for single right-hand sides whatever the value of
                                 kernel; 6 = owner shares (single right-hand side, one lane
                                 per row, not MPK_GS2; other calls run kernel 0): every level
                                 group is split into one share per CTA, CTA c owning share c
                                 of every group for every power; warp groups of a CTA each run
                                 one power through the groups in the level-group wavefront
                                 (Sec. 3), each task waiting on per-CTA progress counters of
                                 the CTAs whose shares its rows read */
    int32_t blocked;          /* mpk_apply without MPK_UNBLOCKED: 1 = always the blocked
                                 kernel, 0 = never, -1 = automatic (default): p >= 2 and a
                                 matrix larger than the L2 cache, and then whichever kernel
                                 the first call for each (precision, p, n_rhs) measures as
                                 faster - that call runs and times both, which synchronises
                                 its stream once; results are identical either way */
    int32_t jacobi;           /* 1 = also keep the Jacobi-scaled matrix A D^-1 (Sec. 5.1,
                                 Eq. (Jacobi): the diagonal preconditioner fused into the SpMV
                                 as a scaling along the columns), D = diag(A), for
                                 MPK_JACOBI: a second copy of the SELL values per kept
                                 precision, b_ij = a_ij / a_jj (computed in FP64), plus
                                 D^-1 in FP64.  A column whose diagonal entry is missing or
                                 zero is not scaled (d_j^-1 := 1).  Also builds what MPK_GS2
                                 needs: a bit mask of the strictly lower entries (in the
                                 caller's row order; one uint32 per 32 stored entries) and
                                 those entries of A D^-1 packed per row into slices of their
                                 own (columns and values, about half the matrix again).
                                 Default 0 */
    int32_t shard_warps;      /* kernel = 3: warps per shard of the ready-first hand-out
                                 (default 4; fewer shards share cursors more, more shards widen
                                 the window between powers) */
    int32_t lanes_per_row;    /* single right-hand side (plain and MPK_JACOBI powers, blocked
                                 and unblocked alike, so both still give identical values):
                                 lanes of a warp that share one row, 1, 2, 4 or 8.  A warp then
                                 covers a sub-slice of 32 / lanes_per_row rows of a SELL-32
                                 slice; each lane sums the row's entries j = part,
                                 part + lanes_per_row, ... (ascending) and the partial sums
                                 are added by a fixed butterfly.  Fewer rows per warp shorten
                                 the rows a task holds (0 = automatic: 1, which measured
                                 fastest on the 27-point benchmark matrices in both
                                 precisions) */
    int32_t task_units;       /* kernel = 4: sub-slices per task (default 1) */
    int32_t task_dispatch;    /* kernel = 4: 0 = tickets dealt round robin to the CTAs, inside
                                 a CTA to whichever warp is free (default); 1 = one ticket
                                 dispenser for the whole grid (a global atomic per task);
                                 2 = static: warp w of W runs tickets w, w + W, w + 2W, ... */
    int32_t owner_lag;        /* kernel = 6: groups between consecutive local powers in the
                                 wavefront (task (g, k) runs in step g + owner_lag (k - 1));
                                 1 (default) is the paper's wavefront, larger values give a
                                 power more time to publish at the cost of a wider window;
                                 0 = 1 */
    int32_t owner_prefetch;   /* kernel = 6: while local power 1 runs group g, the CTA asks the
                                 copy engine to prefetch its share of group g + owner_prefetch
                                 into L2 (cp.async.bulk.prefetch); 0 = off, default 1 */
    int32_t level_order;      /* order of the rows inside a level (Sec. 3 fixes the levels, not
                                 this order): 0 = ascending original index; 1 (default) =
                                 breadth-first: level l's rows by the position of their
                                 earliest-placed neighbour in level l - 1 (in G(A + A^T)), then
                                 by index - the queue order of a breadth-first search that
                                 appends each row's next-level neighbours in ascending index,
                                 which keeps rows that share neighbours together when the
                                 caller's numbering carries no locality (measured on the
                                 randomly permuted 7-point 256^3 matrix: FP32 SpMV 1.55x faster
                                 than with index order).  Built on the device one level after
                                 another. */
} mpk_plan_opts;

typedef struct mpk_plan_s *mpk_plan_t;

/* Statistics of a plan (host struct filled by mpk_plan_stats). */
typedef struct {
    int64_t n, nnz;
    int32_t n_levels, n_groups, n_slices, n_chunks;
    int32_t root;             /* BFS root (original row index) */
    int32_t p_blk;
    int64_t l2_budget_bytes;
    int64_t sell_nnz;         /* stored SELL entries including padding */
    int64_t device_bytes;     /* bytes the plan holds on the device */
    double create_ms;         /* wall time of mpk_plan_create (synchronous part) */
    int32_t bfs_sweeps;       /* BFS runs made by the root search */
    int32_t max_level_rows;
} mpk_plan_info;

/* Coefficients of one MPK call (host memory, read during the call).
 * Power k = 1..p uses a[k-1], b[k-1], c[k-1]; the c term multiplies y_{k-2} (y_{-1} := 0).
 * gamma (optional, p+1 entries): with MPK_FINAL_ONLY the output is sum_k gamma[k] y_k
 * (the polynomial P(A) x of Sec. 5.3, eq. (3)); NULL means the output is y_p. */
typedef struct {
    int32_t p;
    const double *a;
    const double *b;
    const double *c;
    const double *gamma;
} mpk_coeffs;

/* mpk_apply flags */
#define MPK_PERMUTED_IO   0x01u  /* X, Y are in the plan's level order (see mpk_plan_perm) */
#define MPK_FINAL_ONLY    0x02u  /* Y receives one block: y_p, or sum gamma_k y_k */
#define MPK_HOST_IO       0x04u  /* X, Y are HOST pointers; the call copies them in and out
                                    and returns after the result is in Y */
#define MPK_UNBLOCKED     0x08u  /* p back-to-back SpMV launches (Alg. 1) instead of the
                                    blocked schedule; same arithmetic, bit-identical result */
#define MPK_Y0_IS_X       0x10u  /* block 0 of Y already holds x; X is ignored (needs
                                    MPK_PERMUTED_IO, not MPK_FINAL_ONLY) */
#define MPK_RHS_INTERLEAVED 0x20u /* X and Y blocks are row-major n x n_rhs (element (i,r) at
                                    i*n_rhs + r) instead of column-major with leading dim. */
#define MPK_JACOBI        0x80u  /* the powers are those of A D^-1 instead of A (right
                                    Jacobi preconditioning, Sec. 5.1); needs a plan created
                                    with opts.jacobi = 1, else MPK_ERR_ARG */
#define MPK_GS2           0x100u /* the powers are those of the GS2-preconditioned operator
                                    A P^-1 (Sec. 5.1, Alg. GS2: one two-stage Gauss-Seidel
                                    iteration from z^0 = 0 with gamma inner Jacobi-Richardson
                                    iterations; L, D, U split in the caller's row order, a
                                    zero or missing diagonal entry read as 1):
                                      y_k = a_k A P^-1 y_{k-1} + b_k y_{k-1} + c_k y_{k-2}.
                                    Each power runs as gamma + 1 sub-powers over the matrix
                                    (Alg. GS2(b): the gamma inner stages on the Jacobi-scaled
                                    strictly lower part, which they stream from its own packed
                                    copy, then the product with A D^-1); the blocked kernel
                                    schedules the sub-powers like powers, all in one launch.
                                    Add
                                    MPK_GS2_GAMMA(gamma), gamma in 0..15 (0 = Jacobi).  Needs a
                                    plan created with opts.jacobi = 1 and n_rhs = 1
                                    (MPK_ERR_ARG / MPK_ERR_UNIMPLEMENTED otherwise); excludes
                                    MPK_JACOBI; the CTA-task kernel (opts.kernel = 1) runs it
                                    unblocked. */
#define MPK_GS2_GAMMA(g)  ((((uint32_t)(g)) & 15u) << 12)
#define MPK_DEBUG_DROP_FLAG 0x40000000u /* test aid: the blocked task (chunk 0, power 1)
                                    does not publish its flag, so the waits on it run out and
                                    the call reports MPK_ERR_TIMEOUT at mpk_plan_sync */

/* Default options. */
mpk_status mpk_plan_opts_default(mpk_plan_opts *o);

/* Build a plan for A (Sec. 3 pre-processing), entirely on the device:
 *   1. BFS levels of the graph of A + A^T from the root (George-Liu search or row 0);
 *      unreached rows continue from the lowest-index unvisited row one level higher;
 *   2. rows ordered by (level, original index): perm, iperm, level_ptr;
 *   3. B = P A P^T with columns ascending per row, values in FP32 and/or FP64;
 *   4. level groups: consecutive levels joined while
 *        p_blk*(4*rows + (4+w)*nnz) + (p_blk+1)*w*rows <= l2_budget_bytes
 *      (w = value bytes of the MPK precision), a level over budget being a group of its own;
 *   5. SELL-32 slices inside each group, tasks of chunk_slices slices, per-task dependency
 *      ranges and the dependency flags.
 * p_max: largest number of powers a single mpk_apply will request (1..63).
 * A: device CSR (see mpk_csr).  opts may be NULL (defaults).  stream: used for all work; the
 * call synchronises it before returning (the host needs the level counts).
 * On success *out is a new plan; on failure *out is NULL and nothing is leaked. */
mpk_status mpk_plan_create(const mpk_csr *A, int32_t p_max, const mpk_plan_opts *opts,
                           cudaStream_t stream, mpk_plan_t *out);

mpk_status mpk_plan_destroy(mpk_plan_t plan);

/* Fill *st (host). */
mpk_status mpk_plan_stats(mpk_plan_t plan, mpk_plan_info *st);

/* Copy the level structure out (DEVICE output buffers, any may be NULL):
 *   perm[n]          original row at level-order position r
 *   iperm[n]         level-order position of original row i
 *   level[n]         BFS level of original row i
 *   level_ptr[n_levels+1], group_ptr[n_groups+1] (group_ptr indexes levels).
 * Asynchronous on stream. */
mpk_status mpk_plan_perm(mpk_plan_t plan, int32_t *perm, int32_t *iperm, int32_t *level,
                         int32_t *level_ptr, int32_t *group_ptr, cudaStream_t stream);

/* Copy the permuted matrix B = P A P^T out (DEVICE outputs: row_ptr[n+1], col[nnz], val[nnz]
 * of type dtype; the plan must keep that precision).  Asynchronous on stream. */
mpk_status mpk_plan_csr(mpk_plan_t plan, mpk_dtype dtype, int32_t *row_ptr, int32_t *col,
                        void *val, cudaStream_t stream);

/* Replace the values of the plan's matrix by those of a matrix with the SAME pattern
 * (device CSR in the original order), keeping the level structure.  Asynchronous. */
mpk_status mpk_plan_update_values(mpk_plan_t plan, const mpk_csr *A, cudaStream_t stream);

/* Matrix power kernel (Sec. 3, Alg. 1 / blocked):
 *   y_0 = x,  y_k = a_k (A y_{k-1}) + b_k y_{k-1} + c_k y_{k-2}   (k = 1..p, y_{-1} = 0)
 * for n_rhs right-hand sides at once.
 *   co     coefficients (host), 1 <= co->p <= 63
 *   dtype  arithmetic and storage type of X and Y (the plan must keep that precision); the
 *          row sums accumulate in dtype
 *   X      n x n_rhs input block (column-major, leading dimension ldx >= n; or row-major with
 *          MPK_RHS_INTERLEAVED)
 *   Y      output: p+1 blocks y_0..y_p (block k at Y + k*ldy*n_rhs elements), or with
 *          MPK_FINAL_ONLY one block; ldy >= n
 *   flags  MPK_* above
 * Blocked launches run the level-group wavefront with device-side dependency flags; results
 * are bit-identical to MPK_UNBLOCKED on the same plan.  Asynchronous on stream (except with
 * MPK_HOST_IO). */
mpk_status mpk_apply(mpk_plan_t plan, const mpk_coeffs *co, mpk_dtype dtype, const void *X,
                     int64_t ldx, void *Y, int64_t ldy, int32_t n_rhs, uint32_t flags,
                     cudaStream_t stream);

/* Wait for the plan's work on stream and report (then clear) a latched device error:
 * MPK_OK or MPK_ERR_TIMEOUT.  Synchronous. */
mpk_status mpk_plan_sync(mpk_plan_t plan, cudaStream_t stream);

/* Allocation-free final-power MPK.  This entry point is the library's own addition: the
 * paper has no counterpart.
 *
 * For callers that must not allocate device memory once set up: code that runs under a
 * fixed device-memory budget (a serving loop that sized itself at start), and code on a
 * latency-critical path, where cudaMalloc may synchronise the device and its time is
 * unbounded.  mpk_apply allocates its workspace lazily, on the first call that needs it;
 * this call never does.
 *
 * Computes the same result as mpk_apply(plan, co, dtype, X, n, Y, n, 1,
 * MPK_FINAL_ONLY | MPK_UNBLOCKED | flags, stream), with the same kernels:
 * Y = y_p, or sum_k gamma_k y_k when co->gamma is set (the recurrence of mpk_apply above),
 * for ONE right-hand side, by p back-to-back SpMV launches (the plan's unblocked row
 * function: one row per lane, or lanes_per_row lanes sharing a row).
 *   co     coefficients (host), 1 <= co->p <= 63
 *   dtype  MPK_F64 or MPK_F32 (the plan must keep that precision)
 *   X      device vector of n elements (original row order, or level order with
 *          MPK_PERMUTED_IO); read only
 *   Y      device vector of n elements, written (same order as X); must not overlap X
 *   flags  0, MPK_PERMUTED_IO and/or MPK_JACOBI; anything else is MPK_ERR_ARG
 * Scratch: a fixed array of MPK_NOALLOC_SCRATCH_BYTES per device, static in the library and
 * shared by every plan and thread of the process.  A call needs 3 vectors of n elements with
 * MPK_PERMUTED_IO, else 5, each rounded up to 256 bytes: at 32 MiB, n <= 1,398,080 (FP64,
 * level order) or 838,848 (FP64, original order); in FP32 n <= 2,796,160 or 1,677,696.  A larger plan returns
 * MPK_ERR_ARG before any work, with a message on stderr naming the bytes it would need.
 * Nothing in the scratch needs to start at zero or be cleared between calls.
 * Races: calls on one device that can overlap in time (other streams, other host threads,
 * other plans) share the one scratch array and corrupt each other's results.  Keep such
 * calls ordered: one stream, or events between streams.
 * Set-up: the first call on each device, with that device current, looks up the array's
 * address (cudaGetSymbolAddress) and keeps it; make that first call before any stream capture
 * begins on the device.  The kept address does not survive a reset of the device's primary
 * context (cudaDeviceReset): call mpk_noalloc_forget() after such a reset, before the next
 * call.  Asynchronous on stream. */
#define MPK_NOALLOC_SCRATCH_BYTES (32u << 20)
mpk_status mpk_apply_final_noalloc(mpk_plan_t plan, const mpk_coeffs *co, mpk_dtype dtype,
                                   const void *X, void *Y, uint32_t flags, cudaStream_t stream);
/* Drops the scratch addresses kept by mpk_apply_final_noalloc for every device, so that the
 * next call on each device looks its array up again (needed after cudaDeviceReset, whose
 * context reset moves the array).  Not to be called while such calls may run on other
 * threads.  Always MPK_OK.  No counterpart in the paper. */
mpk_status mpk_noalloc_forget(void);

/* Ritz values (Sec. 4: the Newton shifts are "eigenvalue information" from a few steps of
 * standard GMRES): the eigenvalues of the k x k leading block of an upper Hessenberg matrix,
 * by the implicitly double-shifted QR iteration.  H: HOST, column-major with leading
 * dimension ldh >= k (entries below the subdiagonal are ignored); wr, wi: HOST arrays of k
 * receiving real and imaginary parts (complex pairs consecutive, positive imaginary part
 * first).  MPK_ERR_NOT_CONVERGED after 60 k steps without convergence; MPK_ERR_ARG for NULLs,
 * k < 1 or non-finite entries.  Synchronous, host only (no device work). */
mpk_status mpk_hessenberg_eigvals(const double *H, int64_t ldh, int32_t k, double *wr, double *wi);

/* Host helpers for coefficient triples (host arrays of length p). */
/* Chebyshev basis on [alpha, beta]: y_k = T_k((A - c0 I)/d) x, c0 = (alpha+beta)/2,
 * d = (beta-alpha)/2 (three-term recursion; Sec. 5.3 Chebyshev smoother). */
mpk_status mpk_coeffs_chebyshev(double alpha, double beta, int32_t p, double *a, double *b,
                                double *c);
/* Newton basis y_k = (A - theta_k I) y_{k-1} (Sec. 4). */
mpk_status mpk_coeffs_newton(const double *theta, int32_t p, double *a, double *b, double *c);
/* First `count` of `n` real values in Leja order (first = largest modulus; each next one
 * maximises the product of distances to those chosen; ties -> smaller value); used for the
 * Newton shifts from Ritz values (Sec. 4).  Host arrays. */
mpk_status mpk_leja_order(const double *values, int32_t n, int32_t count, double *out);

/* ------------------------------------------------------------------------------------------
 * Autotuner.  No counterpart in the paper, which sets its blocking depth p_opt and cache size C
 * by hand per machine (Sec. 3, Sec. 4).  On this part the best plan options depend on the
 * precision and the number of right-hand sides, so they are measured for one call shape.
 * ---------------------------------------------------------------------------------------- */
typedef struct {
    int32_t n_trials;       /* candidates timed */
    int32_t best_index;     /* position of the best in the candidate list (0 = the base) */
    double best_ms;         /* median time per mpk_apply call with the best options */
    double base_ms;         /* the same with the base options */
} mpk_tune_info;

/* Times mpk_apply(co, dtype, n_rhs, flags) on plans of A built with a fixed list of nine
 * candidate options derived from `base` (NULL: mpk_plan_opts_default): the base itself; p back-to-back
 * SpMVs (blocked = 0); the lane-task kernel with a slack of two and of four tickets per
 * resident warp, and with two slices per task; the warp-task kernel with chunks of 4 and 8
 * slices; the lane-task kernel with level groups sized for a quarter of L2 and for all of it
 * (lanes_per_row stays the base's).  Each
 * candidate runs two untimed calls and `reps` timed ones (CUDA events on `stream`, median).
 * A: DEVICE CSR as for mpk_plan_create; p = co->p <= MPK_MAX_P; flags: any mpk_apply flags
 * but MPK_HOST_IO, MPK_Y0_IS_X, MPK_UNBLOCKED and the debug flag (MPK_ERR_ARG).  The tuner
 * allocates one plan at a time and device input (all ones) and output buffers of the call's
 * shape, all freed before it returns; synchronous on `stream`.  *best receives the fastest
 * candidate's options (pass them to mpk_plan_create); info (host) may be NULL.  Every
 * candidate computes bit-identical results, so the choice affects only speed. */
mpk_status mpk_autotune(const mpk_csr *A, int32_t p, const mpk_coeffs *co, mpk_dtype dtype,
                        int32_t n_rhs, uint32_t flags, const mpk_plan_opts *base, int32_t reps,
                        mpk_plan_opts *best, mpk_tune_info *info, cudaStream_t stream);

/* ------------------------------------------------------------------------------------------
 * s-step GMRES (Sec. 4, Alg. 3(a)+(c)) with FP64 iterative refinement.
 * ---------------------------------------------------------------------------------------- */
typedef struct {
    int32_t s;              /* block size = MPK powers per block (default 8) */
    int32_t restart;        /* restart length m (default 48) */
    double tol;             /* stop when ||b - A x||_2 <= tol ||b||_2 (FP64; default 1e-8) */
    double inner_tol;       /* inner solve tolerance relative to its rhs (default 1e-5) */
    int32_t max_outer;      /* refinement steps, one restart cycle each (default 1000); the
                               solve also stops (MPK_ERR_NOT_CONVERGED) after 50 steps without
                               a new best true residual */
    int32_t inner_cycles;   /* restart cycles per inner solve (default 1) */
    int32_t max_iters;      /* cap on inner iterations in total (default 100000) */
    mpk_dtype basis;        /* MPK_F32: FP32 matrix + basis, FP64 Gram/Cholesky/H/x/r;
                               MPK_F64: everything in FP64 */
    int32_t bcgs_passes;    /* block classical Gram-Schmidt sweeps (1 or 2; default 1) */
    const double *shifts;   /* host, s values, or NULL: Ritz values of a first plain GMRES
                               cycle, Leja-ordered (Sec. 4) */
    uint32_t mpk_flags;     /* extra mpk_apply flags for the basis MPK: MPK_UNBLOCKED runs
                               s back-to-back SpMVs (the baseline solver) */
    int32_t poly_degree;    /* d > 0: GMRES-polynomial preconditioning of degree d (Sec. 5.2,
                               Eq. (poly_precon)).  The first restart cycle (plain GMRES on A)
                               supplies the polynomial q of its first d + 1 steps
                               (x_{d+1} - x_0 = q(A) r0); later cycles run GMRES(restart) with
                               single columns on A q(A) (right preconditioning: one MPK of d
                               powers plus one SpMV per column) and add q(A) V y to x.  q is
                               applied in root form, q(A) x = sum_k (1/theta_{k+1})
                               prod_{i<=k} (I - A/theta_i) x, with the Leja-ordered harmonic
                               Ritz values theta of those steps (a symmetric A is assumed: real
                               roots; without a positive definite pencil no polynomial is
                               used).  d <= min(63, restart - 1); default 0 (off) */
    int32_t poly_f64;       /* 1 (default): apply A q(A) with the FP64 matrix values even with
                               an FP32 basis (q evaluated in FP32 loses digits quickly with the
                               degree); 0: in the basis precision */
    int32_t jacobi;         /* k = 1: right Jacobi preconditioning (Sec. 5.1, Eq. (Jacobi)),
                               one sweep from zero = the diagonal scaling D^-1: every Krylov
                               operator application is one of A D^-1 (MPK_JACOBI; with
                               poly_degree the polynomial is built for A D^-1 too), and each
                               correction u is added as x += D^-1 u.
                               k >= 2 (up to 64): k Jacobi sweeps from zero as the right
                               preconditioner, P^-1 = D^-1 p(A D^-1) with the Neumann
                               polynomial p(t) = sum_{j<k} (1 - t)^j (the sweeps' closed form);
                               cycles run single columns on A D^-1 p(A D^-1), one final-only
                               MPK of k - 1 powers plus one SpMV per column, applied in FP64
                               unless poly_f64 = 0; excludes poly_degree.  info.poly_degree
                               reports k - 1 and poly_interval {0, 0}.
                               The true residual b - A x is unchanged by right preconditioning,
                               so tol keeps its meaning.  Needs a plan created with
                               opts.jacobi = 1.  Default 0 */
    int32_t gs2;            /* 1: right preconditioning by one two-stage Gauss-Seidel
                               iteration from zero (Sec. 5.1, Alg. GS2) with gs2_gamma inner
                               Jacobi-Richardson iterations: the s-step basis is that of
                               A P^-1 (MPK_GS2, every power gs2_gamma + 1 sub-powers, blocked
                               like powers), the first cycle's Ritz values are those of
                               A P^-1, and each correction u is added as x += P^-1 u,
                               evaluated in FP64.  Needs a plan created with opts.jacobi = 1;
                               excludes jacobi and poly_degree.  Default 0 */
    int32_t gs2_gamma;      /* inner iterations of GS2, 0..15 (default 1, as in the paper's
                               GS2 experiments) */
    double *trace_hist;     /* HOST, trace_cap doubles, or NULL: receives, for the first
                               restart cycle in the s-step (Newton) basis, the residual
                               estimate |g_{c+1}| / ||r|| after each column c's Givens
                               rotation (Alg. 3(c)'s convergence check), r the cycle's
                               right-hand side; info.trace_len counts the entries */
    int32_t trace_cap;      /* capacity of trace_hist */
    double *trace_H;        /* HOST, (restart + 1) x restart doubles, column-major, or NULL:
                               that cycle's Arnoldi Hessenberg (before the rotations), zero past
                               its last column */
} mpk_gmres_opts;

typedef struct {
    int32_t iters;          /* inner iterations (Krylov columns) in total */
    int32_t outer;          /* refinement steps taken */
    int32_t restarts;       /* restart cycles in total */
    int32_t status;         /* mpk_status of the solve */
    double rel_residual;    /* true ||b - A x|| / ||b|| in FP64 at exit */
    double shifts[64];      /* shifts used (first s entries) */
    double ms_total, ms_mpk, ms_ortho, ms_other;   /* CUDA-event timings per phase */
    int32_t poly_degree;    /* degree of the polynomial preconditioner used (0: none) */
    double poly_interval[2];/* smallest and largest root of the polynomial */
    int32_t trace_len;      /* entries written to opts.trace_hist */
    int32_t breakdowns;     /* CholQR breakdowns met (each one's cycle keeps the columns
                               before the failing block; the following cycles run at s / 2) */
    int32_t s_final;        /* block size of the last cycle */
} mpk_gmres_info;

mpk_status mpk_gmres_opts_default(mpk_gmres_opts *o);

/* Solve A x = b.  A: a plan holding the precision(s) the options need (FP64 values always,
 * for the residual; FP32 too when basis = MPK_F32) and p_max >= s.  b, x: DEVICE FP64
 * vectors of length n in the original order; x holds the initial guess on entry and the
 * solution on exit.  info (host) may be NULL.
 * Each outer step computes r = b - A x in FP64, runs one restart cycle of s-step GMRES on
 * A d = r in the basis precision (to inner_tol relative to ||r||, or to tol overall with an
 * FP64 basis) and adds d to x; it stops when ||b - A x|| <= tol ||b||.  Without shifts, the
 * first cycle is plain GMRES(m) (classical Gram-Schmidt, two sweeps) whose Ritz values (the
 * real parts of the eigenvalues of its k x k Arnoldi Hessenberg, mpk_hessenberg_eigvals),
 * Leja-ordered, give the Newton shifts.  A Cholesky breakdown ends the cycle at the last good block and halves
 * s for later cycles; at s = 1 it returns MPK_ERR_BREAKDOWN.
 * Synchronous on stream (the host reads a few status words per block).  Returns MPK_OK,
 * MPK_ERR_NOT_CONVERGED (limits reached; x holds the best iterate), MPK_ERR_BREAKDOWN, or an
 * argument / CUDA error. */
mpk_status sstep_gmres_solve(mpk_plan_t A, const double *b, double *x, const mpk_gmres_opts *o,
                             mpk_gmres_info *info, cudaStream_t stream);

/* ------------------------------------------------------------------------------------------
 * s-step CG with FP64 iterative refinement.  The paper names s-step CG as the short-recurrence
 * method whose solver speedup should approach the MPK's, its orthogonalisation being minimal
 * (Sec. 4, discussion of the s-step GMRES results; Sec. 7); the steps are the standard
 * communication-avoiding CG: per outer iteration s Newton powers on p and s - 1 on r give
 * Y = [p, .., rho_s(A) p, r, .., rho_{s-1}(A) r] (one two-rhs MPK call of s powers on the
 * pair (p, r), so the matrix is read s times, not 2s - 1); one FP64 Gram matrix G = Y^T Y;
 * s CG steps on coordinate vectors of length 2s + 1 with the change of basis B (A Y = Y B);
 * then x += Y x', r = Y r', p = Y p'.
 * ---------------------------------------------------------------------------------------- */
typedef struct {
    int32_t s;              /* CG steps per outer iteration = powers of the p basis (1..15,
                               default 8) */
    double tol;             /* stop when ||b - A x||_2 <= tol ||b||_2 (FP64; default 1e-8) */
    double inner_tol;       /* inner solve tolerance relative to its rhs (default 1e-5) */
    int32_t max_outer;      /* refinement steps (default 1000); the solve also stops
                               (MPK_ERR_NOT_CONVERGED) after 50 steps without a new best true
                               residual */
    int32_t max_iters;      /* CG steps in total (default 100000) */
    mpk_dtype basis;        /* MPK_F32 (default): FP32 matrix values, basis and coordinate
                               recovery, FP64 Gram matrix, coefficients, x and true residual;
                               MPK_F64: everything in FP64 */
    const double *shifts;   /* host, s Newton shifts, or NULL: the first refinement step is a
                               setup phase of 4 s plain CG steps whose Ritz values (eigenvalues
                               of the Lanczos tridiagonal of its coefficients) are Leja-ordered */
    uint32_t mpk_flags;     /* extra mpk_apply flags for the basis MPKs: MPK_UNBLOCKED runs
                               back-to-back SpMVs (the baseline) */
    int32_t replace;        /* residual replacement period k (default 1; 0 = off): at the start
                               of every k-th outer iteration after the first, the basis
                               r-column is replaced by the FP64 true residual b - A x (rounded
                               to the basis precision; p is kept), one FP64 SpMV per k outer
                               iterations (van der Vorst and Ye; Carson and Demmel for s-step
                               methods).  It bounds the drift of the recurrence residual in an
                               FP32 basis, so the inner solve runs to 0.5 tol ||b|| directly
                               instead of inner_tol and the CG iterates are not restarted */
} mpk_cg_opts;

typedef struct {
    int32_t iters;          /* CG steps in total (setup phase included) */
    int32_t outer;          /* refinement steps taken */
    int32_t status;         /* mpk_status of the solve */
    int32_t s_used;         /* s at exit (halved after a breakdown) */
    double rel_residual;    /* true ||b - A x|| / ||b|| in FP64 at exit */
    double shifts[16];      /* shifts used (first s entries) */
    double ms_total, ms_mpk, ms_gram, ms_other;   /* CUDA-event timings per phase */
} mpk_cg_info;

mpk_status mpk_cg_opts_default(mpk_cg_opts *o);

/* Solve A x = b for a symmetric positive definite A.  A: a plan holding FP64 values (for the
 * residual), FP32 values too when basis = MPK_F32, and p_max >= s.  b, x: DEVICE FP64 vectors
 * of length n in the original order; x holds the initial guess on entry and the solution on
 * exit; info (host) may be NULL.  Each refinement step computes r = b - A x in FP64 and runs
 * s-step CG on A d = r in the basis precision until its recurrence residual is below
 * inner_tol ||r|| (0.5 tol ||b|| with an FP64 basis or residual replacement), adding the
 * correction to x as it goes.
 * A non-positive p^T A p in the coordinate recurrence (an indefinite A, or a numerically
 * singular basis) ends that outer iteration at its last good step and halves s; at s = 1 the
 * solve returns MPK_ERR_BREAKDOWN.  Synchronous on stream (the host reads a few status words
 * per outer iteration).  Returns MPK_OK, MPK_ERR_NOT_CONVERGED (x holds the last iterate),
 * MPK_ERR_BREAKDOWN, or an argument / CUDA error. */
mpk_status sstep_cg_solve(mpk_plan_t A, const double *b, double *x, const mpk_cg_opts *o,
                          mpk_cg_info *info, cudaStream_t stream);

/* Measured FMA rate of this device: `tflops` (host) receives 2 x FMAs / s in TFLOP/s of a
 * kernel whose threads run eight independent FMA chains of type dtype (best of three timed
 * launches of about 20 ms each, CUDA events on `stream`, after one warm-up launch).  The
 * paper has no counterpart: it is the arithmetic roofline against which the measurement
 * reports a kernel bound by FMA issue (the FP64 MPK on this part) rather than by memory.
 * Synchronous; allocates a small output buffer. */
mpk_status mpk_fma_peak(mpk_dtype dtype, double *tflops, cudaStream_t stream);

/* ------------------------------------------------------------------------------------------
 * Batched MPK over many systems (Sec. 3's level-blocked MPK, run for many matrices at once).
 * The systems' task graphs are concatenated into one block-diagonal graph and run by one
 * persistent launch: many small, uneven systems - each alone too small to fill the GPU, its
 * wavefront short and narrow - share the device, and the pipeline does not drain between
 * systems.  Every system's values equal its own mpk_apply's bit for bit (the same row
 * function as the unblocked power kernel).
 * ---------------------------------------------------------------------------------------- */
typedef struct mpk_batch_s *mpk_batch_t;

/* plans: HOST array of count plans (each keeping values of `dtype`, all on the current
 * device; a plan must outlive the batch and must not be used by another call while the
 * batch runs).  p: the powers every mpk_batch_apply runs (1..63).  Builds the union's task
 * graph and schedule (synchronous on stream).  MPK_ERR_ARG on bad arguments. */
mpk_status mpk_batch_create(const mpk_plan_t *plans, int32_t count, int32_t p, mpk_dtype dtype,
                            cudaStream_t stream, mpk_batch_t *out);

/* For every system i: y_k = a_k A_i y_{k-1} + b_k y_{k-1} + c_k y_{k-2}, k = 1..p, all powers
 * out, in the plan's level order.  co: HOST array of count coefficient sets (each with p
 * triples; gamma ignored).  X, Y: HOST arrays of count DEVICE pointers; Y[i] holds (p + 1)
 * blocks of n_i values (power k at Y[i] + k n_i), X[i] n_i values copied into block 0 (or,
 * with MPK_Y0_IS_X, block 0 of Y[i] already holds x and X may be NULL).  flags: MPK_PERMUTED_IO
 * (required), MPK_Y0_IS_X, MPK_UNBLOCKED (each system by its own p back-to-back SpMV
 * launches instead, the baseline).  Asynchronous on stream.  When the per-system records
 * (matrices, vector pointers, coefficients) differ from the previous call they are uploaded,
 * which first synchronises the stream; a call with the same records neither copies nor
 * synchronises, so it can be captured in a CUDA graph after one ordinary call, and every
 * replay is a fresh launch.  Waits are bounded; mpk_batch_sync reports MPK_ERR_TIMEOUT. */
mpk_status mpk_batch_apply(mpk_batch_t batch, const mpk_coeffs *co, const void *const *X,
                           void *const *Y, uint32_t flags, cudaStream_t stream);
/* Synchronises stream; returns and clears a latched device error of the batch's launches. */
mpk_status mpk_batch_sync(mpk_batch_t batch, cudaStream_t stream);
mpk_status mpk_batch_destroy(mpk_batch_t batch);

/* ------------------------------------------------------------------------------------------
 * The orthogonalisation steps of the solvers on their own: the same kernels, callable on the
 * caller's tall-skinny blocks (all pointers DEVICE, column-major, FP64 results).  Asynchronous
 * on the stream; each call allocates (and frees, stream-ordered) a small partial-sum buffer.
 *
 * Precision of every Gram product in a basis of FP32 values: the products are summed in FP32
 * over at most 32 terms per lane, those block sums over the lanes by a fixed FP32 tree of at
 * most eight levels, and the results in FP64 in a fixed order, so for each entry
 *     |G^ - G| <= (40 u32 + m u64) (|X|^T |Y|),   u32 = 2^-24, u64 = 2^-53,
 * with m the FP64 additions (about n / 1024); about 2.4e-6 relative to |X|^T |Y| for the sizes
 * of this library's workloads.  An FP64 basis sums in FP64 throughout.  Results do not
 * depend on timing (fixed summation order).
 * ---------------------------------------------------------------------------------------- */

/* Block classical Gram-Schmidt's projection coefficients and CholQR's Gram (Sec. 4,
 * Alg. 3(c), BOrtho and TSQR): G = X^T Y for X n x K (leading dimension ldx >= n) and Y n x S
 * (ldy >= n), both of type dtype; G: K x S FP64, column-major (G[a + b K]).
 * 1 <= K <= 145, 1 <= S <= 16.  n = 0 writes zeros.  MPK_ERR_ARG on bad sizes or NULLs. */
mpk_status mpk_gram(mpk_dtype dtype, const void *X, int64_t ldx, int32_t K, const void *Y,
                    int64_t ldy, int32_t S, int64_t n, double *G, cudaStream_t stream);

/* Block update of the orthogonalisation (Sec. 4, Alg. 3(c)): W <- (W - Q C) Rinv in place,
 * row by row in dtype, with Q n x K1 (ldq >= n; K1 = 0 skips the projection and Q, C may be
 * NULL), W n x S (ldw >= n), C K1 x S FP64 column-major, Rinv S x S FP64 column-major of which
 * the upper triangle (rows <= columns) is used - BCGS's projection W - Q C, then CholQR's
 * W R^-1.  0 <= K1 <= 129, 1 <= S <= 16.  G (may be NULL): receives W^T W of the new W
 * (S x S FP64), fused into the update for S <= 8 as in the solver, a separate Gram otherwise. */
mpk_status mpk_block_update(mpk_dtype dtype, const void *Q, int64_t ldq, int32_t K1, void *W,
                            int64_t ldw, int32_t S, const double *C, const double *Rinv,
                            int64_t n, double *G, cudaStream_t stream);

/* The Gram matrix of s-step CG's basis storage (see sstep_cg_solve): Y holds s + 1 pairs of
 * interleaved vectors, pair k at Y + 2 k ldv with its two values for row i at 2i and 2i + 1;
 * G = Y^T Y over the M = 2s + 2 storage columns in pair order (column 2k + q is slot q of pair
 * k), written as the full M x M FP64 matrix, column-major.  1 <= s <= 15; Y 16-byte aligned,
 * ldv >= n rounded up to even (FP32: ldv even).  MPK_ERR_ARG otherwise. */
mpk_status mpk_gram_pairs(mpk_dtype dtype, const void *Y, int64_t ldv, int32_t s, int64_t n,
                          double *G, cudaStream_t stream);

/* ------------------------------------------------------------------------------------------
 * Serving: a continuously batched stream of s-step GMRES solves on one GPU.
 * ---------------------------------------------------------------------------------------- */
typedef struct {
    int64_t hbm_budget_bytes;   /* device memory the server may hold for requests */
    int32_t max_active;         /* requests advanced concurrently (slots) */
    int32_t n_streams;          /* CUDA streams the slots are spread over */
    mpk_gmres_opts gmres;       /* solver options applied to every request */
} mpk_server_opts;

typedef struct mpk_server_s *mpk_server_t;

typedef struct {
    int64_t id;                 /* the id returned by mpk_server_submit */
    int32_t status;             /* mpk_status of the solve */
    int32_t iters, outer;
    double rel_residual;
    double t_submit_ms, t_start_ms, t_done_ms;   /* host clock, ms since server creation */
} mpk_server_result;

mpk_status mpk_server_opts_default(mpk_server_opts *o);
mpk_status mpk_server_create(const mpk_server_opts *o, mpk_server_t *out);
/* Queue a solve of A x = b.  A: HOST CSR arrays (int32 row_ptr/col, FP64 val); b: HOST FP64,
 * n entries; x_out: HOST FP64 buffer of n entries that receives the solution when the result
 * is reported.  The server copies A and b before returning.  *id receives the request id.
 * Returns MPK_ERR_BUDGET if the request alone exceeds the memory budget. */
mpk_status mpk_server_submit(mpk_server_t srv, int64_t n, int64_t nnz, const int32_t *row_ptr,
                             const int32_t *col, const double *val, const double *b,
                             double *x_out, int64_t *id);
/* Copy up to max_results finished results into out (host); *n_out receives the count.
 * Non-blocking: drives the server one round (admission, progress) and returns. */
mpk_status mpk_server_poll(mpk_server_t srv, mpk_server_result *out, int32_t max_results,
                           int32_t *n_out);
/* Number of requests queued or in flight. */
mpk_status mpk_server_pending(mpk_server_t srv, int64_t *n_pending);
mpk_status mpk_server_destroy(mpk_server_t srv);

/* Human-readable name of a status. */
const char *mpk_status_str(mpk_status s);

/* Library build identifier (e.g. "mpk_gb300 sm_103a"). */
const char *mpk_version(void);

#ifdef __cplusplus
}
#endif
#endif /* MPK_GB300_H */
