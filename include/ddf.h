/*
 * ddf.h - C ABI of the GB300 DDF library (libddf.so).
 *
 * DDF ("Vectorizing Sparse Matrix Codes with Dependency Driven Trace
 * Analysis", Cetinic, Cheshmi, Dehnavi) is an inspector-executor method.  The
 * inspector reads only the sparsity pattern of a CSR matrix and mines it for
 * codelets (Sec. III, Alg. 1); the executor runs those codelets (Sec. IV-B).
 * The paper's user calls are DDF_Inspector(A.pattern(), Kernel) and
 * Kernel_Vectorized(clist, A, x, y) (Listing 2).  This library exposes the
 * same split for the two kernels of the paper, SpMV (y = A x) and SpTRSV
 * (L x = b, forward substitution on a lower triangle with its diagonal):
 *
 *     ddf_inspect(csr, kind)  -> device-resident plan (the codelet list)
 *     ddf_spmv(plan, x, y)       ddf_sptrsv(plan, b, x)
 *
 * Conventions
 *   - Plain C, no exceptions cross the ABI; every call returns ddf_status.
 *   - Integer indices are int32 (rowptr, colidx); values and vectors are
 *     IEEE binary64.  Row i of a CSR matrix holds columns colidx[rowptr[i] ..
 *     rowptr[i+1]-1], strictly increasing, each in [0, n_cols).
 *   - Pointers passed in are borrowed: they are read during the call (or, for
 *     device pointers given to the execute calls, by the kernels that call
 *     enqueues) and never freed by the library.  A plan owns every device
 *     buffer it allocates; ddf_plan_destroy releases them.
 *   - ddf_stream_t is a cudaStream_t (NULL = the legacy default stream).
 *     The execute calls are asynchronous on that stream and do not
 *     synchronise the host.  ddf_inspect synchronises the stream it is given
 *     a few times (to read back sizes) before it returns.
 *   - Argument and CSR validation errors are returned by the call.  Errors
 *     that only the device can see (a dependency wait that ran out) are
 *     latched in the plan's status word and returned by ddf_get_status.
 *   - A plan is not safe for concurrent use from two streams: it carries
 *     scratch state (the solve's work ticket and status word).
 */
#ifndef DDF_H
#define DDF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define DDF_API __attribute__((visibility("default")))
#else
#define DDF_API
#endif

typedef struct ddf_plan_s* ddf_plan_t;
typedef void* ddf_stream_t;

typedef enum {
    DDF_OK = 0,
    DDF_ERR_ARG = 1,            /* NULL pointer, negative size, bad option      */
    DDF_ERR_NOT_SQUARE = 2,     /* SpTRSV needs n_rows == n_cols               */
    DDF_ERR_UNSORTED = 3,       /* rowptr not monotone or columns not increasing */
    DDF_ERR_OUT_OF_RANGE = 4,   /* a column outside [0, n_cols)                 */
    DDF_ERR_NOT_LOWER = 5,      /* SpTRSV: an entry above the diagonal          */
    DDF_ERR_MISSING_DIAG = 6,   /* SpTRSV: a row whose last entry is not L_ii    */
    DDF_ERR_ZERO_DIAG = 7,      /* SpTRSV: L_ii == 0                            */
    DDF_ERR_WRONG_KIND = 8,     /* execute call does not match the plan's kind  */
    DDF_ERR_OOM = 9,            /* device allocation failed                      */
    DDF_ERR_CUDA = 10,          /* a CUDA runtime call failed                    */
    DDF_ERR_TIMEOUT = 11,       /* SpTRSV: a dependency wait exceeded its limit  */
    DDF_ERR_NOT_CONVERGED = 12, /* reserved for iterative refinement            */
    DDF_ERR_TOO_LARGE = 13      /* size beyond what an entry point supports      */
} ddf_status;

typedef enum { DDF_SPMV = 1, DDF_SPTRSV = 2 } ddf_kind;

/* Storage types of plan values and of low-precision vectors. */
typedef enum { DDF_F64 = 0, DDF_F32 = 1, DDF_BF16 = 2 } ddf_dtype;

/* Codelet types (Sec. III-B): BLAS = f, g, h strided; PSC I = f, g strided and
 * h(i0,i1) = h0 + delta*i0 + s[i1] with one offset array s for all rows;
 * PSC II = the remaining runs, executed with per-nonzero column offsets. */
typedef enum { DDF_BLAS = 0, DDF_PSC1 = 1, DDF_PSC2 = 2 } ddf_codelet_type;
enum { DDF_ALLOW_BLAS = 1, DDF_ALLOW_PSC1 = 2, DDF_ALLOW_PSC2 = 4, DDF_ALLOW_ALL = 7 };

/* A CSR matrix.  on_device != 0: the three arrays are device pointers on the
 * current device; otherwise host pointers.  values may be NULL for
 * ddf_inspect (pattern only, Listing 2); the plan's values are then set by
 * ddf_update_values before the first execute call. */
typedef struct {
    int32_t n_rows, n_cols;
    int64_t nnz;
    const int32_t* rowptr;  /* [n_rows + 1], rowptr[0] = 0, rowptr[n_rows] = nnz */
    const int32_t* colidx;  /* [nnz] */
    const double* values;   /* [nnz] or NULL */
    int32_t on_device;
    int32_t reserved;
} ddf_csr;

/* Inspector and executor options; ddf_opts_default fills the defaults. */
typedef struct {
    int32_t window_t;       /* t: rows per mining region (Alg. 1, GetConsecutiveIterations), 1..512 */
    int32_t allowed_types;  /* DDF_ALLOW_* mask; PSC II is required (default DDF_ALLOW_ALL)          */
    int64_t w_op;           /* Eq. 1 weight of one operation |p|          (default 8 bytes)  */
    int64_t w_codelet;      /* Eq. 1 per-codelet constant                 (default 32 bytes) */
    int64_t w_index;        /* Eq. 1 weight of one offset-array entry     (default 4 bytes)  */
    int64_t spin_cap_ns;    /* SpTRSV: longest wait on one dependency     (default 2e9 ns)   */
    int32_t unit_nnz;       /* executor work unit: target nonzeros per warp (default 256)     */
    int32_t store_dtype;    /* DDF_F64 (default), or DDF_F32 / DDF_BF16 for the mixed-precision
                               executors (the plan then also keeps a low-precision copy)     */
    int32_t coarsen_rows;   /* SpTRSV partitions (Sec. IV-A, LBC-style coarsening):
                               0 = level sets of G; R in 1..DDF_COARSEN_MAX_ROWS = the
                               non-empty (block of R consecutive rows, level) pairs, in block
                               then level order.  A coarsened plan is solved one block per
                               CTA, dependencies inside a block through shared memory
                               (default DDF_COARSEN_DEFAULT_ROWS = 0: level sets)             */
    int32_t lower_of_input; /* SpTRSV: 0 (default) = the input is the lower-triangular L; 1 =
                               the input is a square matrix A and L is its lower triangle,
                               each row's entries with column <= row (a prefix of the sorted
                               row), read in place without a copy.  Every row of A must then
                               hold its diagonal.  ddf_update_values takes A's values.  Must
                               be 0 for SpMV                                                   */
    int32_t reserved[6];
} ddf_opts;

#define DDF_COARSEN_MAX_ROWS 16384
#define DDF_COARSEN_DEFAULT_ROWS 0

/* Plan statistics (counts per codelet type are indexed by ddf_codelet_type). */
typedef struct {
    int32_t kind, n_rows, n_cols, depth;  /* depth = number of partitions (levels for SpTRSV) */
    int64_t nnz;                          /* stored entries of the inspected matrix          */
    int64_t points;                       /* iteration points (SpTRSV: off-diagonal entries) */
    int64_t ncodelets[3];
    int64_t ops[3];                       /* iteration points covered by each type (Fig. 9)  */
    int64_t rows[3];                      /* rows covered by each type                        */
    int64_t nunits;                       /* executor work units                              */
    int64_t bytes_exec;                   /* algorithmic bytes of one execute call            */
    int64_t max_row_len;
    int64_t levels;                       /* SpTRSV: depth of G (longest path + 1)          */
    int64_t blocks;                       /* SpTRSV: row blocks of a coarsened plan, else 0   */
    int64_t reserved[4];
} ddf_plan_stats_t;

/* Fill *o with the defaults listed above.  Never fails for a non-NULL o. */
DDF_API void ddf_opts_default(ddf_opts* o);

/*
 * Inspector (Alg. 1).  Reads the pattern of A (and its values when present),
 * validates it, and builds a device-resident plan on the current device:
 *   kind == DDF_SPMV:   one partition with every row; codelets are runs of
 *                       consecutive rows (Sec. IV-A, SpMV has no dependencies).
 *   kind == DDF_SPTRSV: A must be square and lower triangular with every
 *                       diagonal entry present, last in its row and nonzero.
 *                       The dependency DAG's level sets are the partitions
 *                       (findDependencies, partitionIterationSpace); codelets
 *                       are runs of rows inside one level; the off-diagonal
 *                       values are copied in that level order.
 * o may be NULL (defaults).  On success *out receives the plan; on error *out
 * is set to NULL and nothing is left allocated.  Synchronises stream s.
 */
DDF_API ddf_status ddf_inspect(const ddf_csr* A, ddf_kind kind, const ddf_opts* o, ddf_stream_t s,
                       ddf_plan_t* out);

/* Replace the plan's values with a new array of the same pattern (nnz entries
 * in the original CSR order), without re-inspection.  The inspector reads only
 * the pattern and the executor the values (Listing 2: DDF_Inspector is given
 * A.pattern(), the vectorised kernel A itself), so one inspection serves every
 * matrix of that pattern, the amortisation of its cost in Sec. V-C.  values is
 * a device pointer when on_device != 0; it is read during the call and may be
 * freed afterwards.  The plan stores the values in its executor layout (level
 * order for SpTRSV; for SpMV, CSR order except rows executed in value tiles,
 * whose values are point-major).  SpTRSV: fails with DDF_ERR_ZERO_DIAG when a
 * new diagonal entry is 0 (synchronises s in that case only to report it);
 * DDF_ERR_ARG for a NULL plan or values, DDF_ERR_OOM / DDF_ERR_CUDA when a
 * staging copy of host values cannot be made. */
DDF_API ddf_status ddf_update_values(ddf_plan_t p, const double* values, int32_t on_device,
                             ddf_stream_t s);

/* SpMV executor (Sec. IV-B, the executor of Listing 3): y = A x with
 * y_i = sum_k A_ik x_k as the CSR code of Fig. 1a computes it, each codelet of
 * the plan run by the generic code of its type (Sec. III-B: BLAS, PSC I,
 * PSC II).  x [n_cols] and y [n_rows] are FP64 device pointers, caller-owned;
 * y is overwritten (rows without entries get 0) and must not overlap x.
 * Launches one kernel per codelet type and layout present on s (BLAS and
 * PSC I rows of at most 256 points run one lane per row; the rest
 * in warp work units) and returns without synchronising.  Returns
 * DDF_ERR_WRONG_KIND for a SpTRSV plan, DDF_ERR_ARG for NULL vectors or a plan
 * without values. */
DDF_API ddf_status ddf_spmv(ddf_plan_t p, const double* x, double* y, ddf_stream_t s);

/* SpTRSV executor (Sec. IV-B over the partitions of Sec. IV-A): solves
 * L x = b by forward substitution, x_i = (b_i - sum_{j<i} L_ij x_j) / L_ii.
 * b and x are FP64 device pointers of n_rows entries, caller-owned, and must
 * not overlap.  The partitions of findDependencies / partitionIterationSpace
 * (level sets of the dependency graph G, or their coarsened form) run in
 * order and the codelets of one partition together, linked by per-row ready
 * flags instead of a barrier (x itself: an entry is ready once it no longer
 * holds the fill pattern written at the start of the call).  Asynchronous on
 * s.  Every dependency wait is bounded by spin_cap_ns; a wait that runs out
 * latches DDF_ERR_TIMEOUT in the plan's status word (read it with
 * ddf_get_status) and the solve finishes with NaN in the affected rows
 * instead of hanging.  Returns DDF_ERR_WRONG_KIND for a SpMV plan and
 * DDF_ERR_ARG for NULL or overlapping vectors. */
DDF_API ddf_status ddf_sptrsv(ddf_plan_t p, const double* b, double* x, ddf_stream_t s);

/*
 * Mixed-precision SpMV (a later form of the executor of Sec. IV-B; the paper
 * runs its codelets in double precision, Listing 3): the plan must have been inspected with store_dtype DDF_F32 or
 * DDF_BF16.  y = A x with the values in that type, x and y device vectors of
 * vec_dtype (DDF_F32 or DDF_BF16), every product and sum in FP32.  Same
 * codelets and kernels per type as ddf_spmv.
 */
DDF_API ddf_status ddf_spmv_lowp(ddf_plan_t p, const void* x, void* y, ddf_dtype vec_dtype, ddf_stream_t s);

/*
 * Mixed-precision SpTRSV with iterative refinement.  The plan (kind
 * DDF_SPTRSV, store_dtype DDF_F32 or DDF_BF16) keeps the FP64 values as well.
 * x0 = solve(b) in low precision (FP32 vectors, FP32 sums); then repeatedly
 * r = b - L x in FP64, stop once ||r||_2 <= tol ||b||_2, else d = solve(r) in
 * low precision and x += d in FP64.  The residual and the update are the only
 * FP64 steps.  b and x are FP64 device vectors.  *iters receives the number
 * of corrections applied, *relres the last relative residual (either may be
 * NULL).  Synchronises s once per refinement step.  Returns
 * DDF_ERR_NOT_CONVERGED when max_iter corrections do not reach tol (x then
 * holds the last iterate) and DDF_ERR_TIMEOUT when a solve's wait ran out.
 */
DDF_API ddf_status ddf_sptrsv_refine(ddf_plan_t p, const double* b, double* x, double tol, int32_t max_iter,
                                     ddf_stream_t s, int32_t* iters, double* relres);

/*
 * Batched inspection: `count` independent matrices (each a ddf_csr as for
 * ddf_inspect, host or device arrays, possibly of different sizes) are
 * inspected as one block-diagonal matrix.  Matrix i occupies rows and columns
 * starting at the sum of the sizes of matrices 0..i-1; multi-RHS vectors of
 * the batch are laid out the same way.  For DDF_SPTRSV every matrix must be
 * square and lower triangular; the level sets then mix rows of all matrices,
 * which widens every level.  Everything else is as in ddf_inspect.
 */
DDF_API ddf_status ddf_inspect_batch(const ddf_csr* mats, int32_t count, ddf_kind kind, const ddf_opts* o,
                                     ddf_stream_t s, ddf_plan_t* out);

/*
 * Multi-RHS SpMV: Y = A X for nrhs (1..32) right-hand sides.  X is
 * [n_cols][nrhs] and Y [n_rows][nrhs], row-major, device memory, of dtype
 * DDF_F64 (FP64 values and sums) or DDF_F32 (the plan's FP32 values, FP32
 * sums; the plan needs store_dtype DDF_F32).  Runs the SpMV plan's codelets
 * (Sec. III-B) with one warp per matrix row at a time.  When nrhs is 16 bytes
 * times a power of two from 2 to 16 (FP32: 8, 16, 32; FP64: 4, 8, 16, 32)
 * and X and Y start on 16-byte boundaries, a lane moves 16 bytes of a row of
 * X and one load of the warp fetches the X rows of several points; otherwise
 * lane k owns right-hand side k.  Either way the summation order is fixed.
 */
DDF_API ddf_status ddf_spmm(ddf_plan_t p, const void* X, void* Y, int32_t nrhs, ddf_dtype dtype, ddf_stream_t s);

/*
 * Multi-RHS SpTRSV: solves L X = B for nrhs (1..32) right-hand sides, layouts
 * and dtypes as in ddf_spmm (B and X must not overlap).  Rows run in the
 * plan's level order (the partitions of Sec. IV-A) with per-element ready
 * flags as in ddf_sptrsv, one warp per row at a time, lanes laid out as in
 * ddf_spmm; each warp of a persistent grid takes the next work units (rows
 * of one level) from a ticket.
 * Plain launches only (no cooperative launch), so the call can be recorded
 * in a CUDA graph.
 */
DDF_API ddf_status ddf_sptrsm(ddf_plan_t p, const void* B, void* X, int32_t nrhs, ddf_dtype dtype,
                              ddf_stream_t s);

/*
 * A batch's SpMV and SpTRSV in one persistent launch (after the fill of Xs
 * that marks its rows unsolved): Y = A X on the SpMV plan pa and L Xs = B on
 * the SpTRSV plan pl, both typically from ddf_inspect_batch, with nrhs
 * (1..32) right-hand sides; layouts and dtypes as in ddf_spmm / ddf_sptrsm
 * (DDF_F32 needs both plans stored in FP32).  The warps of the launch take
 * tickets: first the solve's work units, in level order, then the SpMV's
 * work items, so the products run on the warps the solve's narrow deep
 * levels leave idle.  Results equal those of ddf_spmm and ddf_sptrsm on the
 * same operands.  Xs must not overlap X, Y or B, and Y must not overlap X or
 * B (DDF_ERR_ARG).  DDF_ERR_WRONG_KIND unless pa is DDF_SPMV and pl
 * DDF_SPTRSV.  Solve errors (DDF_ERR_TIMEOUT) are latched in pl's status
 * word (ddf_get_status).  Plain launches only, so the call can be recorded
 * in a CUDA graph.
 */
DDF_API ddf_status ddf_batch_run(ddf_plan_t pa, const void* X, void* Y, ddf_plan_t pl, const void* B, void* Xs,
                                 int32_t nrhs, ddf_dtype dtype, ddf_stream_t s);

/*
 * Autotuner for the multi-RHS executors.  Kind DDF_SPMV: rebuilds the plan's
 * work units for each candidate tile size (target nonzeros per unit: 64 ..
 * 2048) and times ddf_spmm; kind DDF_SPTRSV: times ddf_sptrsm for each
 * candidate number of work units a warp takes per ticket (1 .. 8).  Timing uses CUDA
 * events on the given operands; the fastest candidate is kept and returned
 * in *best_unit_nnz (may be NULL).  Overwrites the output operand.
 * Synchronises s.
 */
DDF_API ddf_status ddf_tune(ddf_plan_t p, const void* in, void* out, int32_t nrhs, ddf_dtype dtype,
                            ddf_stream_t s, int32_t* best_unit_nnz);

/*
 * GPU recalibration of the cost model (Eq. 1, Sec. III-C).  The paper fits the
 * model's weights to CPU timings (Fig. 5); here the weights are chosen on the
 * GPU: the matrix A (with values) is inspected for `kind` with each of six
 * weight sets (w_op, w_codelet, w_index) = (8, 32, 4) (the default byte
 * costs), (8, 8, 4), (8, 128, 4), (8, 32, 1), (8, 32, 16) and (1, 3, 1) (the
 * paper's CPU form), the executor is timed on each plan (CUDA events, the
 * fastest of three runs after a warm-up, a vector of ones as input), and the
 * fastest set is written into *o (its other fields are kept and used for
 * every inspection).  *pick (may be NULL) receives the index of the chosen
 * set.  DDF_ERR_ARG without values or for another kind; inspection and
 * executor errors are returned as they are.  Allocates and frees its own
 * vectors; synchronises s.
 */
DDF_API ddf_status ddf_tune_cost(const ddf_csr* A, ddf_kind kind, ddf_opts* o, ddf_stream_t s, int32_t* pick);

/* Synchronise s, then return and clear the plan's device status word: the
 * errors only the executor can see while it runs the partitions of Sec. IV-A
 * in order (DDF_ERR_TIMEOUT: a dependency wait ran out).  DDF_OK when none
 * occurred; DDF_ERR_CUDA when the stream itself reported an error. */
DDF_API ddf_status ddf_get_status(ddf_plan_t p, ddf_stream_t s);

/* Plan statistics (host struct st, caller-owned): counts of codelets, rows
 * and operations per type (the breakdown of Fig. 9 in Sec. V-A), the number
 * of partitions and of levels of G (Sec. IV-A), and the executor's
 * algorithmic bytes per call.  Synchronous (computed on the first call from a
 * host copy of the descriptors).  DDF_ERR_ARG for NULL arguments. */
DDF_API ddf_status ddf_plan_stats(ddf_plan_t p, ddf_plan_stats_t* st);

/*
 * Export the plan in canonical form for checking: the codelet list cList of
 * Alg. 1 with, for each codelet, the access functions of Sec. III-A (f: row,
 * g: value offset, h: column) in the strided form of Sec. III-D, and the
 * partitions of Sec. IV-A.  Buffers are host memory owned by the caller:
 *   records [ncodelets][12] int64: part, type, q0, m, n, f_str, rho, g_str,
 *            gamma, h0, delta, sigma (n = -1 for PSC II; rho, gamma, delta,
 *            sigma are 0 where undefined, e.g. for one-row codelets);
 *   seq [n_rows] int32: the partition sequence (row at each position);
 *   part_ptr [depth + 1] int32: first position of each partition;
 *   gs [n_rows] int64: g(q, 0), the offset of each position's first value in
 *            CSR order for SpMV and in the level-ordered copy for SpTRSV.
 * Any output pointer may be NULL to skip it; *ncodelets and *depth always
 * receive the sizes.  Synchronous.
 */
DDF_API ddf_status ddf_plan_export(ddf_plan_t p, int64_t* records, int64_t* ncodelets, int32_t* seq,
                           int32_t* part_ptr, int32_t* depth, int64_t* gs);

/*
 * Plan serialisation (reuse of an inspection across runs, the amortisation
 * of Sec. V-C).  ddf_plan_save with buf == NULL stores the required size in
 * *len; otherwise it writes the plan (descriptors, work units, level order,
 * the plan's copies of indices and values, low-precision copies) into buf,
 * which must hold *len >= that size bytes, and returns DDF_ERR_ARG with the
 * size in *len when it is too small.  ddf_plan_load rebuilds a device plan
 * on the current device from such a buffer without re-inspection; it checks
 * the header, the sizes and a checksum and returns DDF_ERR_ARG on any
 * mismatch.  The buffer is host-endian.  Both synchronise (save: the plan's
 * stream; load: s).  The checksum detects corruption, not tampering, so load
 * also runs ddf_plan_validate on the rebuilt plan and returns its status
 * (and no plan) when a check fails.
 */
DDF_API ddf_status ddf_plan_save(ddf_plan_t p, void* buf, size_t* len);
DDF_API ddf_status ddf_plan_load(const void* buf, size_t len, ddf_stream_t s, ddf_plan_t* out);

/*
 * Check every index an executor derives from the plan against the arrays it
 * addresses (Sec. III's access functions: for each codelet the rows f(i0),
 * the value extents g(i0, i1) and the columns h(i0, i1); the work units; the
 * level pointers; the coarsened block and chunk tables; for SpTRSV the rows
 * of the inspected matrix kept for ddf_update_values, each of which must
 * fill exactly its position's extent), and for SpTRSV that
 * every column names a row below the diagonal that an earlier partition
 * (Algorithm 1's level or block schedule) solves.  Returns DDF_OK,
 * DDF_ERR_ARG (a malformed descriptor, unit or table), DDF_ERR_OUT_OF_RANGE
 * (an index outside its array) or DDF_ERR_NOT_LOWER (a dependency on a row
 * not yet solved).  Runs on the plan's stream and synchronises it; the plan
 * is not modified.  Inspection builds plans that pass by construction.
 */
DDF_API ddf_status ddf_plan_validate(ddf_plan_t p);

/* Release every device buffer of the plan (stream-ordered on the stream the
 * plan was inspected on, after the work queued there; the call does not
 * wait for it).  NULL is ignored. */
DDF_API void ddf_plan_destroy(ddf_plan_t p);

/* Static description of a status code. */
DDF_API const char* ddf_status_string(ddf_status st);

/* Number of kernel launches the last execute call on this plan enqueued. */
DDF_API int32_t ddf_last_launches(ddf_plan_t p);

/* Total number of kernels this library has launched in the process so far
 * (inspector, executors and their helpers).  Thread-safe. */
DDF_API int64_t ddf_kernel_launches(void);

/*
 * Test hook for failure detection (not part of the method): overwrite one
 * column of the plan's level-ordered SpTRSV copy so that the entry at
 * position k of that copy names row `col`.  Pointing a row at a later row
 * makes its dependency wait run out, which exercises the bounded waits and
 * DDF_ERR_TIMEOUT without faulting the GPU.  Returns DDF_ERR_ARG when k or
 * col is out of range.  Synchronous.
 */
DDF_API ddf_status ddf_debug_set_dependency(ddf_plan_t p, int64_t k, int32_t col);

/*
 * Test hook for failure detection (not part of the method): the library's
 * next k device allocations succeed and the one after them fails as if the
 * device were out of memory, so the call making it returns DDF_ERR_OOM after
 * releasing what it had allocated.  One-shot; k < 0 disarms the hook.
 * Process-wide, host-side only (no device fault is involved).  Always
 * returns DDF_OK.
 */
DDF_API ddf_status ddf_debug_fail_alloc(int64_t k);

/*
 * Lower-triangular solve that allocates nothing (this entry point has no
 * counterpart in the paper; it serves callers of this library that must not
 * allocate device memory: code running inside a memory-pool or allocator
 * hook, where calling cudaMalloc would re-enter the allocator; services with
 * a fixed device-memory budget; and latency-critical loops that cannot afford
 * the device-wide synchronisation cudaMalloc and cudaFree may imply).
 *
 * Solves L x = b by forward substitution directly on the caller's CSR lower
 * triangle (device pointers: rowptr [n+1], colidx [nnz], values [nnz], b and x
 * [n]; columns increasing, the diagonal last in each row), without a plan.
 * Its scratch (a work ticket, a status word and one ready flag per row) lives
 * in a file-scope device array of DDF_NOALLOC_MAX_ROWS + 64 words (4 MiB)
 * that every GPU which loads the library holds until the process exits.
 * n > DDF_NOALLOC_MAX_ROWS returns DDF_ERR_TOO_LARGE before any device work.
 *
 * Every call looks up the device address of that array in the current
 * context (cudaGetSymbolAddress, with the device current; the lookup itself
 * allocates nothing).  The very first lookup in a context loads the library's
 * module, and loading the module is what creates the array: a caller that
 * must not allocate later makes one call with n == 0 first, as a warm-up (it
 * does the look-up and returns DDF_OK without touching the GPU otherwise).
 * Every call shares the array: its header is cleared at the start of each
 * call, and rows are flagged with a per-call number, so stale flags of
 * earlier calls are never mistaken for new ones; calls that overlap on the
 * GPU (two streams, two threads) race and must not be issued.  The call
 * copies the status to the host and synchronises stream s, so it cannot be
 * recorded in a CUDA graph.  It returns the solve's status:
 * DDF_ERR_MISSING_DIAG / DDF_ERR_NOT_LOWER / DDF_ERR_ZERO_DIAG for a
 * malformed row (detected on the device; such rows are skipped, never read
 * out of bounds), DDF_ERR_TIMEOUT when a dependency wait exceeds
 * spin_cap_ns (nanoseconds).
 */
#define DDF_NOALLOC_MAX_ROWS (1 << 20)
DDF_API ddf_status ddf_sptrsv_csr_noalloc(int32_t n, int64_t nnz, const int32_t* rowptr,
                                          const int32_t* colidx, const double* values,
                                          const double* b, double* x, int64_t spin_cap_ns,
                                          ddf_stream_t s);

#ifdef __cplusplus
}
#endif

#endif /* DDF_H */
