/*
 * hylu.h -- C ABI of a GB300 (sm_103a) implementation of the numeric phase of
 * HYLU, a hybrid up-looking sparse LU solver (X. Chen, "HYLU: Hybrid Parallel
 * Sparse LU Factorization", Sec. 2).
 *
 * Plain C types only: sizes are int32/int64, matrices are CSR arrays, device
 * buffers are raw pointers into the memory of the current CUDA device and
 * streams are passed as `void*` holding a cudaStream_t (NULL = legacy default
 * stream).  Every entry point returns HYLU_OK (0), a warning (> 0) or an error
 * (< 0).  There is no CPU fallback: numeric work runs only in this library's
 * CUDA kernels, and a call made without a usable CUDA device returns
 * HYLU_ERR_CUDA.
 *
 * Threads and streams: handles are independent (except for the one scratch
 * array that every hylu_solve_static call shares), so different host threads
 * may drive different handles at the same time.  Calls on ONE handle must
 * not overlap on the host, and because a handle's factor storage, solve
 * workspace and device counters are shared by its calls, the caller orders
 * its device work too: calls on one handle made on different streams race
 * unless those streams are synchronized with each other.
 *
 * Data conventions (used by every call below):
 *   - A is n x n CSR: rowptr int64[n+1] (rowptr[0] = 0), col int32[nnz]
 *     strictly increasing within each row, values float64[nnz].
 *   - Preprocessing (Sec. 2.1) gives row/column permutations and scalings:
 *     Ahat(i,k) = dr[rowperm[i]] * A(rowperm[i], colperm[k]) * dc[colperm[k]],
 *     rowperm/colperm map new index -> original index, dr/dc are indexed by
 *     original row/column.
 *   - The numeric phase factors Ahat * Pi = L * U (L unit lower, U upper); Pi
 *     only exchanges columns inside the diagonal block of a supernode
 *     (supernode diagonal pivoting, Sec. 2.2); piv[p] = column label at
 *     position p.
 */
#ifndef HYLU_H
#define HYLU_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---- */
#define HYLU_OK 0
#define HYLU_WARN_PERTURBED 1         /* a small pivot was perturbed (Sec. 2.2) */
#define HYLU_WARN_REFINE_STALLED 2    /* refinement stopped above the target  */
#define HYLU_ERR_ARG (-1)             /* null/invalid argument                */
#define HYLU_ERR_PATTERN (-2)         /* unsorted, duplicate or out-of-range column */
#define HYLU_ERR_STRUCT_SINGULAR (-3) /* no perfect matching on the nonzeros  */
#define HYLU_ERR_NOMEM (-4)           /* device or host allocation failed     */
#define HYLU_ERR_CUDA (-5)            /* a CUDA call failed / no device       */
#define HYLU_ERR_DEVICE_TIMEOUT (-6)  /* a bounded device wait expired        */
#define HYLU_ERR_STATE (-7)           /* call out of order (e.g. solve before factor) */
#define HYLU_ERR_INTERNAL (-8)        /* plan inconsistency (a bug)           */
#define HYLU_ERR_TOO_LARGE (-9)       /* size above a fixed library limit     */

/* ---- options ---- */
#define HYLU_ORDER_AMD 0
#define HYLU_ORDER_ND 1
#define HYLU_ORDER_NATURAL 2
#define HYLU_ORDER_USER 3
#define HYLU_ORDER_AUTO 4   /* AMD and nested dissection both; the plan with the lower estimated
                               factorization time is kept (see hylu_analyze) */

typedef struct hylu_handle hylu_handle; /* opaque, owned by the library */

typedef struct {
    int ordering;          /* HYLU_ORDER_*; default AMD (Sec. 2.1)                    */
    int static_pivot;      /* 1: maximum-product matching on the values (Sec. 2.1)    */
    int scale;             /* 1: apply the matching's row/column scalings             */
    int sn_max;            /* largest supernode, in rows (default 256)                 */
    int nd_leaf;           /* nested dissection: subgraphs this small use AMD          */
    double pivot_tau;      /* pivots below pivot_tau * max|Ahat| are perturbed (sqrt eps) */
    double refine_tol;     /* refinement target on the backward error (1e-12)          */
    int refine_maxit;      /* refinement corrections at most (10)                      */
    int refine;            /* 0: only after a perturbation (Sec. 2.3); 1: always       */
    long long spin_limit;  /* iterations of a device wait before HYLU_ERR_DEVICE_TIMEOUT */
    int rows_per_task;     /* reserved (rows are claimed one per warp)                 */
    int debug;             /* 1: extra host checks                                     */
    double amd_dense;      /* AMD: rows denser than max(16, amd_dense*sqrt(n)) go last (2) */
    int timing;            /* 1: time the factor and solve kernels with CUDA events     */
    int precision;         /* 0: FP64 factors; 1: FP32 factors (scaling and the small-pivot
                              check in FP64) with FP64 iterative refinement on every solve */
    double heavy_ratio;    /* rows whose update work is at least heavy_ratio x the mean row (and
                              at least 1e6 flops) are claimed first, from a queue of their own,
                              by two warps of every block; 0 disables (32) */
    int gemm_min_rows;     /* precision form (precision = 1): supernodes of at least this many rows
                              take the updates of their diagonal block and U tail from source
                              supernodes of at least min(16, gemm_min_rows) rows as split-BF16
                              tensor-core GEMM tasks (Sec. 2.2, Fig. 1c, sup-sup); 0 disables (64).
                              Ignored for FP64 factors. */
    int solve_seq_rows;    /* substitution, bulk-sequential (Sec. 2.3, Fig. 3): a chain of two or
                              more consecutive light levels (at most this many rows, see
                              hylu_export_solve_segments) is solved level after level by one
                              thread block with block barriers instead of the level watermark's
                              hand-off; 0 solves every level in bulk (default 8) */
} hylu_options;

typedef struct {
    int32_t n;
    int64_t nnz_a;          /* entries of A                                 */
    int64_t nnz_lu;         /* entries of the unpadded symbolic L+U pattern */
    int64_t nnz_store;      /* stored entries (padded pattern)              */
    int32_t nnodes;         /* supernodes + standalone rows                 */
    int32_t nsupernodes;    /* nodes of more than one row                   */
    int32_t rows_in_supernodes;
    int32_t max_supernode;
    int32_t ntasks;         /* tasks of the factor kernel: rows plus supernode tail tasks */
    double flops;           /* unpadded symbolic flop count (Sec. 2.1)      */
    double flops_padded;    /* flops on the padded pattern                  */
    int32_t nperturb;       /* perturbed pivots of the last factorization   */
    int32_t refine_iters;   /* corrections of the last solve                */
    double backward_error;  /* of the last solve: ||b-Ax||inf/(||A||inf ||x||inf + ||b||inf) */
    int32_t device_status;  /* 0 or a HYLU_ERR_* raised on the device       */
    int32_t failed_node;    /* node where a device wait expired, else -1    */
    double analyze_ms;
    double factor_kernel_ms; /* last factorization kernel (opt.timing = 1), else -1 */
    double solve_kernel_ms;  /* last substitution kernels (opt.timing = 1), else -1  */
    int32_t nheavy;          /* rows the factor kernel claims first (see heavy_ratio) */
    int32_t factor_levels;   /* dependency levels of the factor kernel's tasks (critical-path length) */
    int32_t fwd_levels;      /* node levels of the forward / backward substitution (for a batch, */
    int32_t bwd_levels;      /*   the largest over its instances)                                 */
    /* the padded flops by kernel (Sec. 2.1 counts them during the symbolic
     * factorization; Sec. 2.2, Fig. 1 names the kernels); they add up to
     * flops_padded */
    double flops_row_row;      /* updates from standalone source rows                  */
    double flops_sup_row;      /* updates from source supernodes into standalone rows  */
    double flops_sup_sup;      /* updates from source supernodes into supernode rows   */
    double flops_in_supernode; /* supernode rows against the earlier rows of their own
                                  diagonal block (the in-supernode factorization)     */
    int32_t ordering;          /* HYLU_ORDER_* the plan was built with (HYLU_ORDER_AUTO
                                  resolves to AMD or ND; a batch whose systems chose
                                  differently reports HYLU_ORDER_AUTO)                */
    double analyze_phase_ms[4]; /* analysis wall time by phase: [0] matching and
                                   scaling, [1] ordering, [2] symbolic factorization,
                                   supernodes and schedules, [3] value map (a batch:
                                   summed over its systems)                           */
    int32_t gemm_destinations;  /* precision form: GEMM destinations (see gemm_min_rows), 0 when the
                                   tensor-core sup-sup path is off                     */
    int32_t gemm_tasks;         /* its tensor-core GEMM tasks per factorization           */
    double gemm_flops;          /* useful FP32 flops of those tasks (2 per multiply-add of
                                   L_{D,S} U_{S,T}); 6 BF16 products carry each          */
    int32_t tuned;              /* 1 after hylu_tune                                      */
    int32_t factor_blocks_per_sm; /* blocks per SM of the factor / substitution launches   */
    int32_t solve_blocks_per_sm;
    int32_t heavy_queue;        /* 1: heavy rows are claimed first (see heavy_ratio)       */
    int32_t solve_seq_rows;     /* the bulk-sequential threshold in use (hylu_tune may set 0) */
    int32_t solve_segments[2];  /* segments of light levels of the forward / backward
                                   substitution in use (0 before the first factorization) */
} hylu_info;

/* Fill *opt with the defaults listed above.  Returns HYLU_ERR_ARG on NULL. */
int hylu_default_options(hylu_options* opt);

/* Preprocessing (Sec. 2.1): static pivoting with scaling (maximum-product
 * matching on `vals`, host memory), fill-reducing ordering (AMD, nested
 * dissection, natural, or `user_perm` = new -> original index when
 * opt->ordering == HYLU_ORDER_USER), symbolic factorization, supernode
 * detection (consecutive rows with identical U structure, Sec. 2.2) and the
 * task schedule (Sec. 2.2.1).  All inputs are host arrays owned by the caller
 * and are copied; `vals` is only read for the matching (may be NULL when
 * opt->static_pivot == 0; with static pivoting, a NaN or infinite value
 * returns HYLU_ERR_ARG).
 * On success *out is a new handle (free it with
 * hylu_destroy).  Errors: HYLU_ERR_ARG, HYLU_ERR_PATTERN,
 * HYLU_ERR_STRUCT_SINGULAR, HYLU_ERR_NOMEM.  Runs on the host only.
 * HYLU_ORDER_AUTO analyses under both AMD and nested dissection and keeps
 * the plan whose estimated factorization time is lower: the larger of its
 * flops at 1.06e12 flop/s (the measured FP64 rate of a GB300) and its
 * dependency levels at 21 us each (the measured cost of one level along the
 * factor kernel's chain); info.ordering reports the choice.  Any other
 * ordering value outside 0..4 returns HYLU_ERR_ARG.
 * n = 0 (an empty system) is accepted: hylu_factor, hylu_refactor,
 * hylu_solve, hylu_solve_transpose, hylu_grad_values, hylu_tune and the
 * exports then return HYLU_OK without touching the device, and their device
 * pointers may be NULL. */
int hylu_analyze(int32_t n, int64_t nnz, const int64_t* rowptr, const int32_t* col,
                 const double* vals, const int32_t* user_perm, const hylu_options* opt,
                 hylu_handle** out);

/* Numeric factorization (Sec. 2.2, Fig. 1): d_vals is a DEVICE array of the
 * nnz values of A in the CSR order given to hylu_analyze.  The first call
 * uploads the plan and allocates the factor storage on the current device;
 * later calls reuse it.  Asynchronous on `stream`; the library copies d_vals
 * (device to device) so the caller may reuse it once the stream has passed
 * this call.  Device-side failures (a wait that expired) are reported by
 * hylu_get_info / the next synchronizing call. */
int hylu_factor(hylu_handle* h, const double* d_vals, void* stream);

/* Repeated solve with an identical pattern (Sec. 3.2): same as hylu_factor
 * with new values; keeps the matching, scalings and ordering of the analysis
 * and recomputes the pivot choices inside supernodes.  Requires a previous
 * hylu_factor (else HYLU_ERR_STATE). */
int hylu_refactor(hylu_handle* h, const double* d_vals, void* stream);

/* Forward/backward substitution (Sec. 2.3): solves A x = b for nrhs right-hand
 * sides stored column by column with leading dimension ld >= n, both DEVICE
 * arrays (d_b is read only, d_x written; they may not overlap).  When a pivot
 * was perturbed (or opt.refine == 1) the solution is refined in FP64 on the
 * original A (Sec. 2.3) until the backward error reaches opt.refine_tol, stops
 * halving, or opt.refine_maxit corrections were made; this synchronizes the
 * stream.  Returns HYLU_WARN_REFINE_STALLED if the target was not reached.
 * Workspace: the first call with more right-hand sides (or a larger ld) than
 * any before allocates device buffers for it (about 2 n nrhs + 2 ld nrhs
 * doubles); earlier buffers stay allocated until hylu_destroy, so a captured
 * graph that points at them stays valid. */
int hylu_solve(hylu_handle* h, const double* d_b, double* d_x, int nrhs, int ld, void* stream);

/* Transpose solve A^T x = b with the same factors (U^T then L^T), same
 * arguments and refinement rule as hylu_solve. */
int hylu_solve_transpose(hylu_handle* h, const double* d_b, double* d_x, int nrhs, int ld,
                         void* stream);

/* Adjoint scatter for differentiating x = A^{-1} b with respect to the
 * entries of A (a torch.autograd backward, for instance): with lam = A^{-T} g
 * from hylu_solve_transpose and x the forward solution, writes
 * d_dvals[q] = -sum_r lam_r[i] * x_r[j] for every entry q = (i, j) of A, in
 * the CSR order given to hylu_analyze (dL/dA restricted to A's pattern;
 * dL/db is lam itself).  All DEVICE arrays; lam and x hold nrhs columns of
 * leading dimension ld >= n.  Asynchronous on `stream`. */
int hylu_grad_values(hylu_handle* h, const double* d_lam, const double* d_x, double* d_dvals, int nrhs,
                     int ld, void* stream);

/* ---- batched form (many value sets of one pattern, many patterns) ----
 * Analyse k independent systems (system s: CSR n[s], rowptr[s], col[s],
 * vals[s] host arrays, same conventions as hylu_analyze) to be factored with
 * nsets value sets each.  The handle holds one block-diagonal plan of the
 * k * nsets instances; instance q = v * k + s (value set v of system s).
 * hylu_factor / hylu_refactor then take d_vals = all instances' values
 * concatenated in instance order, and hylu_solve right-hand sides of length
 * N = sum over instances of n[s] (instance q at rows hylu_batch_layout's
 * row_base[q]): every instance is factored in ONE persistent launch and
 * solved in one launch sequence.  The k systems are analysed on host threads.
 * Every system needs n >= 1: an empty system in a batch is refused with
 * HYLU_ERR_ARG (a single empty system is accepted by hylu_analyze). */
int hylu_analyze_batch(int32_t k, const int32_t* n, const int64_t* const* rowptr, const int32_t* const* col,
                       const double* const* vals, int32_t nsets, const hylu_options* opt, hylu_handle** out);

/* Layout of a batch handle (HOST arrays, any may be NULL): row_base int32[k*nsets]
 * first row of each instance in the combined system, val_base int64[k*nsets]
 * offset of each instance's values in d_vals.  *total_n gets N. */
int hylu_batch_layout(hylu_handle* h, int32_t* row_base, int64_t* val_base, int32_t* total_n);

/* Capture refactorization of d_vals followed by the substitution of d_b into
 * d_x (nrhs columns, leading dimension ld) as a CUDA graph on `stream`,
 * replayed by hylu_graph_launch.  A graph cannot branch on the host, so the
 * iterative refinement of Sec. 2.3 is recorded as a FIXED number of
 * `corrections` (0..16) FP64 steps after the solve (residual r = b - A x on
 * the original A, solve A d = r, x += d), whatever the backward error; one
 * more residual pass follows, so that hylu_get_info after a replay reports
 * the backward error of the replay's final x (over the whole system of the
 * handle: for a batch, the block-diagonal system of all its instances) and
 * refine_iters = corrections.  Two corrections take a solution whose pivots
 * were perturbed (relative size ~1.5e-8) to about 1e-16 on well-conditioned
 * systems.  Requires a previous hylu_factor and hylu_solve with at least
 * nrhs right-hand sides (so that nothing is allocated during capture), and
 * a created stream (the legacy default stream cannot be captured:
 * HYLU_ERR_ARG).  The pointers are baked into the graph; the values behind
 * them are read afresh by every replay (the kernels' readiness generations
 * live in device memory and advance on each replay), so new values written
 * into d_vals / d_b between replays are factored and solved. */
int hylu_graph_capture(hylu_handle* h, const double* d_vals, const double* d_b, double* d_x, int nrhs, int ld,
                       int corrections, void* stream);
int hylu_graph_launch(hylu_handle* h, void* stream);

/* Autotune the handle on d_vals by short timed trials (refactorizes several
 * times; synchronizes; allocates two n-vectors for the duration): blocks per
 * SM (1..4) of the factor launch (fixed at one for the tensor-core variant of
 * the precision form), the heavy-row queue on or off at that grid, and blocks
 * per SM of the substitution launches, with the handle's solve_seq_rows and
 * with every level in bulk (solve_seq_rows = 0).  The chosen point stays in
 * the handle (hylu_info reports it: tuned, factor_blocks_per_sm,
 * solve_blocks_per_sm, heavy_queue, solve_seq_rows), the factors of d_vals
 * are left in place, and *blocks_per_sm receives the factor launch's
 * setting.  The substitution is timed with as many right-hand sides as the
 * handle's solves used so far (1 to 8). */
int hylu_tune(hylu_handle* h, const double* d_vals, int* blocks_per_sm, void* stream);

/* Synchronize the handle's last stream and report sizes, flop counts,
 * perturbations, refinement results and any device-side status. */
int hylu_get_info(hylu_handle* h, hylu_info* info);

/* Copy preprocessing outputs to caller-owned HOST arrays (any may be NULL):
 * rowperm/colperm int32[n], dr/dc float64[n], sn_start int32[nnodes+1]. */
int hylu_export_perm(hylu_handle* h, int32_t* rowperm, int32_t* colperm, double* dr, double* dc,
                     int32_t* sn_start);

/* Claim schedule of the factor kernel (HOST arrays, any may be NULL; for
 * analysis and tests): order int32[info.ntasks] (entries < n are rows, entry
 * n + t is tail task t), heavy int32[info.nheavy] (the heavy-row queue),
 * task_node int32[info.ntasks - n] (the supernode each tail task solves). */
int hylu_export_schedule(hylu_handle* h, int32_t* order, int32_t* heavy, int32_t* task_node);

/* Diagnostics: the tables of the tensor-core sup-sup update that a
 * precision-form factorization of `h` would use with gemm_min_rows =
 * min_rows (see GemmPlan in the sources), as one flat int64 HOST array:
 * a header of 10 numbers (destinations, (destination, source) pairs, tail
 * map entries, GEMM tasks, diag tasks, claim-order length, levels, L slots,
 * smallest source supernode of a pair, A elements per split term) followed by
 * the arrays in a fixed order.  buf == NULL:
 * *len receives the length; otherwise *len is the capacity on entry.  Host
 * only.  HYLU_ERR_INTERNAL when the pattern is not closed under the
 * supernode tails (never for a plan of this library). */
int hylu_export_gemm_plan(hylu_handle* h, int min_rows, int64_t* buf, int64_t* len);

/* Bulk-sequential partition of the forward (backward = 0) or backward
 * (backward = 1) substitution for solve_seq_rows = max_rows (Sec. 2.3,
 * Fig. 3), as int32 in HOST memory.  A level of one instance is light when it
 * holds at most max_rows rows, no node of more rows, and at most 1024 max_rows
 * entries of work (its rows' L lists, or its nodes' U tails times their rows,
 * plus the squares of its node sizes); a segment is a maximal chain of two or
 * more consecutive light levels, solved by one thread block; the other rows
 * are solved in bulk.  In the forward direction a bulk row with at least
 * 2048 L entries has its list split into chunks of about 1024 entries (the
 * rectangular blocks of Sec. 2.3 with their nonzeros spread evenly), each
 * claimed on its own once the levels of its entries complete; the row adds
 * their sums (the one-right-hand-side substitution; with several right-hand
 * sides rows sum their whole lists).  Layout: a header [ntask, nseg, nlevels,
 * nrows, nsnodes, nchunks], then task (ntask: the bulk rows in claim order,
 * and n + c for chunk c before the rows of its level), meta (3 nseg:
 * instance, first level, last level; segments sorted by first level), seg_off
 * (nseg + 1, into the level table), lvl_row (nlevels + 1, into rows), lvl_node
 * (nlevels + 1, into snodes), rows (nrows: the segments' rows, level by level,
 * node by node), snodes (nsnodes: the segments' nodes of more than one row),
 * then per chunk its row, first and end entry (in the row's L list) and the
 * level it waits for (4 arrays of nchunks), and each row's chunk offsets
 * (n + 1).  buf = NULL returns the length in *len; HYLU_ERR_ARG when *len is
 * too small (*len then holds the length needed).  Host work only. */
int hylu_export_solve_segments(hylu_handle* h, int backward, int max_rows, int32_t* buf, int64_t* len);

/* Padded storage pattern in CSR form (HOST arrays, any may be NULL):
 * rowptr int64[n+1], col int32[info.nnz_store]; columns sorted per row. */
int hylu_export_pattern(hylu_handle* h, int64_t* rowptr, int32_t* col);

/* Factor values on the padded pattern (HOST arrays, synchronizes): vals
 * float64[nnz_store] in the CSR order of hylu_export_pattern, piv int32[n].
 * Entry (i, c): L(i, position c) if c is below the first row of i's node,
 * position c (L if c < i, U if c >= i) inside i's own supernode block, and
 * U(i, label c) past the end of i's node. */
int hylu_export_factors(hylu_handle* h, double* vals, int32_t* piv);

/* Release device and host memory of the handle (NULL is accepted). */
int hylu_destroy(hylu_handle* h);

/* Substitution that allocates nothing (no counterpart in the paper: this is
 * an interface for callers that must not allocate).  Some callers cannot let
 * a library call cudaMalloc on their behalf: a program that reserves the whole
 * device memory up front for its own pool (a framework's caching allocator),
 * where an extra cudaMalloc fails or fragments that pool, and latency-bound
 * loops, where cudaMalloc's implicit device-wide synchronization is not
 * acceptable.  hylu_solve allocates its work vectors on first use; this call
 * instead keeps them in one fixed array compiled into the library
 * (2 * HYLU_STATIC_SOLVE_MAX_N doubles = 4 MiB, held on every device that
 * loads the library until the process exits).
 *
 * Solves A x = b for ONE right-hand side with the factors of the last
 * hylu_factor/hylu_refactor on `h` (which must have completed its own
 * allocations earlier: this call does not allocate them).  d_b is read, d_x
 * written, both DEVICE arrays of n doubles.  No iterative refinement is
 * applied (use hylu_solve when a pivot was perturbed).  Asynchronous on
 * `stream`; nothing is synchronized, so a failure of the factorization on
 * the device (HYLU_ERR_DEVICE_TIMEOUT) does not show here: read it with
 * hylu_get_info before trusting the result.
 *
 * Errors: HYLU_ERR_STATE when `h` is not factored, or holds FP32 factors
 * (opt.precision = 1: their solution is only FP32-accurate without the FP64
 * refinement that hylu_solve applies); HYLU_ERR_ARG for NULL pointers (n > 0)
 * or when the current device is not the one `h` was factored on.  A factored
 * empty system (n = 0) returns HYLU_OK without device work.
 *
 * Limits and sharing: n above HYLU_STATIC_SOLVE_MAX_N returns
 * HYLU_ERR_TOO_LARGE before any device work.  The array is shared by every
 * call in the process and keeps the last call's contents (all of it is
 * rewritten before it is read, so nothing needs clearing); two calls whose
 * work overlaps on the GPU -- on different streams, or on different handles
 * -- race on it and must be ordered by the caller.  The first call on each
 * device looks up the array's device address (cudaGetSymbolAddress, with that
 * device current); make that first call before any stream capture.  The
 * address is cached for the process: after a cudaDeviceReset of a device
 * (which also ends every handle on it) do not call this function again. */
#define HYLU_STATIC_SOLVE_MAX_N 262144
int hylu_solve_static(hylu_handle* h, const double* d_b, double* d_x, void* stream);

/* Checkpoint of an analysis (no counterpart in the paper, whose repeated-solve
 * mode, Sec. 3.2, reuses the preprocessing only within one run).  The host
 * analysis of hylu_analyze / hylu_analyze_batch (matching, scalings,
 * ordering, symbolic pattern, supernodes, schedules) costs seconds on large
 * patterns and depends on nothing but the pattern, the values given to it and
 * the options; these two calls let a later process skip it.
 *
 * hylu_plan_save writes the handle's plan, batch layout and options into the
 * caller-owned HOST buffer `buf` as one flat byte image (little-endian, with
 * a version and an FNV-1a checksum).  With buf == NULL, *bytes receives the
 * size needed; otherwise *bytes is the capacity on entry and the size written
 * on return (HYLU_ERR_ARG, with *bytes set to the size needed, when the
 * buffer is too small).  Host only; the handle need not be factored.
 *
 * hylu_plan_load makes a new handle from such an image (the caller keeps
 * `buf`; the library copies what it needs).  opt == NULL keeps the saved
 * options; otherwise the numeric options (pivot_tau, refinement, precision,
 * spin_limit, timing, debug) come from *opt and the analysis options
 * (ordering, static_pivot, scale, sn_max, nd_leaf, amd_dense, heavy_ratio)
 * stay the saved ones.  The new handle behaves as the saved one did after
 * its analysis: hylu_factor first, then the solves.  Errors: HYLU_ERR_ARG
 * (NULL pointers, bytes <= 0, opt->precision not 0 or 1), HYLU_ERR_PATTERN
 * (not an image of this version: wrong magic, version or byte order, bad
 * checksum, truncated, or sizes and index ranges that do not fit together),
 * HYLU_ERR_NOMEM.  The checks catch damaged images, not crafted ones: load
 * only images this library wrote. */
int hylu_plan_save(hylu_handle* h, void* buf, int64_t* bytes);
int hylu_plan_load(const void* buf, int64_t bytes, const hylu_options* opt, hylu_handle** out);

/* Diagnostics: when the handle was analysed with (opt.debug & 2), copy the
 * per-row trace of the last factorization to the HOST array out[4 * n]:
 * for row i, out[4i] = claim time, out[4i+1] = updates from earlier nodes
 * done, out[4i+2] = published (a supernode row with a U tail: its
 * diagonal-block step published), all in ns of %globaltimer; out[4i+3] =
 * for the last row of a supernode with a U tail, the time its tail tasks
 * completed the node, else (ns waited on other nodes << 32) | ns waited on
 * the own supernode.  HYLU_ERR_STATE when tracing is off. */
int hylu_debug_trace(hylu_handle* h, unsigned long long* out);

/* Diagnostics of the tensor-core sup-sup path after a factorization
 * (synchronizes; HOST arrays, any may be NULL): pair_cnt int32[pairs] (rows
 * that wrote their multipliers for each pair), gd_done int32[destinations]
 * (GEMM tasks finished), walk_done int32[n] (factor generation at which each
 * row's walk ended), status int32[16] (the device status words); with
 * tracing on (opt.debug & 2), block_prog int32[4 * *nblocks]: per GEMM block
 * the last task claimed, its stage (1 claimed, 2 waited, 3-6 per K chunk:
 * loads issued, operands staged, products issued, products done, 7-8
 * epilogue), the chunk and a spare word (*nblocks = 0 without tracing).
 * HYLU_ERR_STATE when the path is off or nothing was factored. */
int hylu_debug_gemm(hylu_handle* h, int32_t* pair_cnt, int32_t* gd_done, int32_t* walk_done, int32_t* status,
                    int32_t* block_prog, int32_t* nblocks);

/* Diagnostics: when the handle was analysed with (opt.debug & 4), copy the
 * completion time (ns of %globaltimer) of every node in the last forward
 * (out[2 * node]) and backward (out[2 * node + 1]) substitution to the HOST
 * array out[2 * nnodes].  HYLU_ERR_STATE when that tracing is off. */
int hylu_debug_solve_trace(hylu_handle* h, unsigned long long* out);

/* Diagnostics: resident blocks per SM on the current device of the FP64
 * factor kernel (out4[0]), of the FP32 one (out4[1]) and of its tensor-core
 * variant (out4[2]); out4[3] = that variant's registers per thread * 10000 +
 * shared bytes per block / 16. */
int hylu_debug_occupancy(int* out4);

/* Number of kernel launches this library has issued since it was loaded (a
 * graph replay counts the kernels recorded in it; recording counts none). */
int64_t hylu_launch_count(void);

/* Measure the FP64 fused multiply-add throughput of the current device (the
 * roofline of the FP64 numeric kernels: the factorization is bound by the
 * FP64 pipe on GB300).  Runs a short register-resident DFMA kernel on
 * `stream` and synchronizes it; *gflops receives FLOP/s / 1e9 (2 per FMA). */
int hylu_measure_fp64_peak(double* gflops, void* stream);

/* The tensor-core tile engine of the precision form's sup-sup update (Sec.
 * 2.2, Fig. 1c), applied to plain dense matrices so that it can be checked on
 * its own: C -= A B with A (m x k, row stride lda), B (k x n, ldb) and C
 * (m x n, ldc) FP32 row-major DEVICE arrays.  Each operand is split into
 * nsplit (2 or 3) BF16 terms and the products run as tcgen05 MMAs with FP32
 * accumulation in tensor memory (3 term products for nsplit 2, about 2^-16
 * relative accuracy; 6 for nsplit 3, about FP32 accuracy).  Allocates its
 * split copies of A, synchronizes `stream` and frees them; returns
 * HYLU_ERR_ARG for bad sizes, HYLU_ERR_CUDA when the driver offers no TMA
 * tensor-map encoder, HYLU_ERR_DEVICE_TIMEOUT when a bounded wait expired. */
int hylu_split_gemm(const float* d_a, const float* d_b, float* d_c, int m, int n, int k, int lda, int ldb,
                    int ldc, int nsplit, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* HYLU_H */
