/*
 * spmv.h -- C ABI of the GB300 sparse matrix-vector library for finite-volume CFD matrices.
 *
 * What it computes (the paper's hot path and what is grown around it):
 *   y = A x for a square sparse matrix A from an unstructured finite-volume mesh, where the
 *   sparsity pattern drives indirect gathers of x (Sec. 2; Sec. 4.3 "naive implementation").
 *   Pre-processing, applied once per matrix: optional (reverse) Cuthill-McKee reordering
 *   (Sec. 4.1), conversion to sliced ELLPACK with S rows per slice stored column-major inside
 *   a slice (Sec. 4.2), and the per-slice first/last column of x that the slice reads
 *   (Sec. 5.1, col_start / col_end).  Around the SpMV: multi-right-hand-side products,
 *   Jacobi-preconditioned CG in FP64, CG with FP32 inner solves and FP64 iterative
 *   refinement, and a continuous-batching solve server (none of these are in the paper).
 *
 * Conventions for every entry point:
 *   - Every call returns an spmv_status_t and never aborts the process.
 *   - "Device pointer" means memory of the current CUDA device; "host pointer" means
 *     ordinary (optionally pinned) host memory.
 *   - stream is a cudaStream_t passed as void* (NULL = the legacy default stream).  Calls
 *     marked "async" only enqueue work on that stream; calls marked "sync" return after the
 *     work is complete.
 *   - Vectors of a reordered matrix live in the reordered ("internal") numbering; convert
 *     with spmv_permute.
 *   - Index type int32 (row_ptr, col_idx), so nnz < 2^31.
 */
#ifndef GB300_SPMV_H
#define GB300_SPMV_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct spmv_matrix_s *spmv_matrix_t;
typedef struct spmv_server_s *spmv_server_t;

typedef enum {
    SPMV_OK = 0,
    SPMV_ERR_INVALID_ARG = 1,   /* null pointer, negative size, unsupported option value   */
    SPMV_ERR_INVALID_CSR = 2,   /* row_ptr not monotone, column out of range, unsorted/dup  */
    SPMV_ERR_OOM = 3,           /* a device allocation failed                               */
    SPMV_ERR_BUDGET = 4,        /* a server request can never fit the memory budget        */
    SPMV_ERR_CUDA = 5,          /* any other CUDA runtime error                             */
    SPMV_ERR_NOT_CONVERGED = 6, /* CG reached its iteration cap                             */
    SPMV_ERR_TIMEOUT = 7,       /* a bounded device-side wait or a solve deadline expired   */
    SPMV_ERR_PENDING = 8,       /* server request not finished yet                          */
    SPMV_ERR_UNSUPPORTED = 9,   /* operation not available for this handle's precision     */
    SPMV_ERR_CANCELLED = 10     /* a server request was cancelled before it finished        */
} spmv_status_t;

/* reorder */
#define SPMV_REORDER_NONE 0
#define SPMV_REORDER_RCM 1 /* reverse Cuthill-McKee (Sec. 4.1 uses CM; same bandwidth) */
#define SPMV_REORDER_CM 2

/* precision: which value arrays the handle stores */
#define SPMV_PREC_FP64 0 /* FP64 values (12 bytes per non-zero with the int32 column)       */
#define SPMV_PREC_FP32 1 /* FP32 values only (8 bytes per non-zero)                         */
#define SPMV_PREC_DUAL 2 /* FP64 and FP32 values: FP64 and FP32 products, mixed-precision CG */

/* variant of the SpMV kernel */
#define SPMV_VARIANT_AUTO 0
#define SPMV_VARIANT_CSR 1         /* thread per CSR row, x gathered from global memory (Sec. 4.3) */
#define SPMV_VARIANT_SELL 2        /* sliced ELLPACK, A streamed, x kept resident in L2        */
#define SPMV_VARIANT_SELL_WINDOW 3 /* sliced ELLPACK, x staged per CTA in a shared-memory window (Sec. 5.1) */
#define SPMV_VARIANT_SELL_BULK 4   /* sliced ELLPACK, x kept resident in L2, the matrix streamed
                                    * into a ring of shared-memory stages by bulk asynchronous
                                    * copies (one CTA per SM; falls back to SELL when a slice
                                    * does not fit a stage).  Same summation order as SELL. */

typedef struct {
    int slice_height;    /* S, rows per slice: 32, 64, 128 or 256 (0 = default 64)            */
    int block;           /* threads per CTA for the SpMV kernels that take one slice-lane per
                          * thread: 64..1024, multiple of 32 (0 = 256).  The FP64 kernel that
                          * strides over the slice-lanes with five entries in flight (chosen when
                          * the widest slice needs fewer load rounds that way) uses 256. */
    int variant;         /* SPMV_VARIANT_*                                                   */
    int reorder;         /* SPMV_REORDER_*                                                   */
    int precision;       /* SPMV_PREC_*                                                      */
    int autotune;        /* 1: time the candidate (S, block, variant) on this matrix and keep the fastest */
    int peripheral;      /* 1: George-Liu pseudo-peripheral start node for (R)CM             */
    int window_words;    /* SELL_WINDOW capacity in x entries per CTA (0 = largest that fits) */
    int index_bits;      /* 0 = 16 when every slice spans < 65,535 columns, else 32;
                          * 32 = always int32 columns; 16 = 16-bit where possible.  16-bit
                          * columns are offsets from the slice's col_start (Sec. 5.1). */
    int sigma;           /* 0 = off; else a power of two in [32, 4096]: after the reordering,
                          * rows are sorted by decreasing length (stable) inside windows of
                          * sigma rows, so the slices pad less (the rows are renumbered: use
                          * spmv_permute / spmv_get_permutation as for a reordering). */
    int checks;          /* 1: after the conversion, verify its structures on the device
                          * (spmv_verify) and fail with SPMV_ERR_INVALID_CSR on any violation;
                          * 0 = off (default).  Costs one pass over the matrix at creation. */
    int spmm_form;       /* kernel form of the multi-vector products whose rows are gathered
                          * in 32-byte pieces (SPMV_SPMM_*): AUTO = tuned when autotune is on,
                          * else the measured default (UNROLLED).  Every form gives the same
                          * bits. */
    int pq_ctas;         /* CG product grid: CTAs per SM (0 = tuned when autotune is on, else
                          * 4; 2..4 explicit).  The grid fixes the reduction order of p.q. */
    int pq_unroll;       /* CG product entries in flight per lane: 0 = tuned / automatic, 2, 5 */
    int gather_bytes;    /* cg_solve_multi: bytes of a row of P each product lane gathers
                          * (0 = tuned when autotune is on, else 32; 16 or 32) */
    int chain_form;      /* spmv_apply_chain with this handle as B (SPMV_CHAIN_*): AUTO =
                          * tuned on the first call when autotune is on, else TWO */
} spmv_options_t;

/* forms of the operator chain y = B (C x) (spmv_options_t.chain_form of B); both give the
 * same y bit for bit */
#define SPMV_CHAIN_AUTO 0
#define SPMV_CHAIN_FUSED 1 /* one kernel: each entry b_if evaluates row f of C on the spot */
#define SPMV_CHAIN_TWO 2   /* two sliced products through a temporary t = C x (C->n_rows
                            * entries) that B's handle allocates on first use and keeps */

/* forms of the 256-bit multi-vector product (spmv_options_t.spmm_form) */
#define SPMV_SPMM_AUTO 0
#define SPMV_SPMM_WIDE 1      /* one warp per group of rows, two entries per step          */
#define SPMV_SPMM_WIDE_PIPE 2 /* the same, the next two entries' values and columns loaded
                               * while the current rows of X are gathered                   */
#define SPMV_SPMM_WIDE_GS4 3  /* grid-stride over row blocks, 4 CTAs per SM, the next block's
                               * matrix data prefetched into L2                              */
#define SPMV_SPMM_WIDE_GS6 4  /* the same at 6 CTAs per SM                                   */
#define SPMV_SPMM_UNROLLED 5  /* one warp per group of rows, the body unrolled for the slice's
                               * width (up to 10), the row's matrix loads all in flight; the
                               * default when not tuned                                      */

/* Invariants verified by spmv_verify, one bit each in its result:                      */
#define SPMV_CHECK_SLICE_PTR 1  /* slice pointers start at 0, grow by multiples of S, end at
                                 * the entry count                                         */
#define SPMV_CHECK_ROW 2        /* each CSR row fits its slice and its columns increase    */
#define SPMV_CHECK_COLUMN 4     /* sliced entries equal the CSR columns in [0, n_cols);
                                 * padding is -1                                            */
#define SPMV_CHECK_VALUE 8      /* sliced values equal the CSR values bit for bit; padding 0 */
#define SPMV_CHECK_RANGE 16     /* every column lies in its slice's [col_start, col_end)   */
#define SPMV_CHECK_REL16 32     /* 16-bit offsets decode to the columns; 0xFFFF = padding  */
#define SPMV_CHECK_PERM 64      /* the renumbering is a permutation                         */

/* Fills *opt with the defaults (S = 64, block = 256, AUTO variant, no reordering, FP64,
 * no autotuning, peripheral start on, automatic column index width, no checks).  Returns SPMV_ERR_INVALID_ARG if opt is NULL. */
spmv_status_t spmv_default_options(spmv_options_t *opt);

/* Human-readable name of a status code (static string, never NULL). */
const char *spmv_status_string(spmv_status_t status);

/*
 * spmv_create -- sync.  Builds a matrix handle from CSR (Sec. 4.2 input; Sec. 4.1 reordering;
 * Sec. 4.2 sliced ELLPACK; Sec. 5.1 per-slice column range).
 *   n_rows, n_cols >= 0 (rectangular operators such as the divergence and gradient matrices of
 *   the operator-based formulation, Sec. 2, are allowed when opt->reorder is NONE and
 *   opt->sigma is 0; reordering and CG need n_rows == n_cols); nnz >= 0; row_ptr
 *   int32[n_rows+1] with row_ptr[0] = 0 and row_ptr[n_rows] = nnz; col_idx int32[nnz], strictly
 *   increasing inside each row, in [0, n_cols); values double[nnz].
 *   inputs_on_device: 0 = the three arrays are host pointers, 1 = device pointers.
 *   The arrays are copied; the caller keeps ownership and may free them after return.
 *   opt may be NULL (defaults).  On success *out owns every device buffer of the matrix.
 * Errors: INVALID_ARG (null pointers, n_rows != n_cols, bad options), INVALID_CSR (the checks
 * above, run on the device), OOM, CUDA.  On error *out is set to NULL.
 */
spmv_status_t spmv_create(int32_t n_rows, int32_t n_cols, int64_t nnz, const int32_t *row_ptr,
                          const int32_t *col_idx, const double *values, int inputs_on_device,
                          const spmv_options_t *opt, void *stream, spmv_matrix_t *out);

/* Frees every device buffer of the handle (synchronizes the device first).  NULL is a no-op. */
spmv_status_t spmv_destroy(spmv_matrix_t A);

/* Sizes and choices of a handle.  Any output pointer may be NULL. */
typedef struct {
    int32_t n_rows;
    int64_t nnz;
    int32_t slice_height;    /* S actually used                                  */
    int32_t block;           /* CTA size actually used                           */
    int32_t variant;         /* kernel variant actually used                     */
    int32_t precision;
    int32_t reorder;
    int32_t n_slices;
    int64_t sell_entries;    /* stored sliced-ELLPACK entries, padding included   */
    int32_t bandwidth;       /* max |row - col| in the internal numbering         */
    int32_t max_slice_span;  /* max over slices of col_end - col_start            */
    int32_t window_words;    /* shared-memory window capacity (SELL_WINDOW), else 0 */
    size_t device_bytes;     /* device memory owned by the handle                 */
    int32_t index_bits;      /* 32 or 16 (column indices streamed by the kernels) */
    int32_t n_cols;
    int32_t spmm_form[2][4]; /* SPMV_SPMM_* used by the multi-vector product, per precision
                              * (0 FP64, 1 FP32) and lanes per row (1, 2, 4, 8: k = 4, 8, 16,
                              * 32 FP64 or 8, 16, 32, 64 FP32) */
    int32_t pq_ctas;         /* CG product grid: CTAs per SM                        */
    int32_t pq_unroll;       /* CG product entries in flight per lane (FP64 handle)  */
    int32_t gather_bytes;    /* cg_solve_multi product: bytes gathered per lane      */
    int32_t chain_form[2];   /* SPMV_CHAIN_* of spmv_apply_chain(_f32) with this B      */
} spmv_info_t;
spmv_status_t spmv_get_info(spmv_matrix_t A, spmv_info_t *info);

/* sync.  perm_host int32[n_rows]: perm[new] = old (identity when not reordered). */
spmv_status_t spmv_get_permutation(spmv_matrix_t A, int32_t *perm_host);

/* sync.  CSR of the matrix in the internal numbering (rows sorted by column), host arrays of
 * n_rows+1, nnz and nnz entries.  values may be NULL for an FP32-only handle. */
spmv_status_t spmv_export_csr(spmv_matrix_t A, int32_t *row_ptr, int32_t *col_idx, double *values);

/* sync.  Sliced-ELLPACK arrays (Sec. 4.2) to host memory: slice_ptr int64[n_slices+1],
 * col int32[sell_entries] (padding = -1), values double[sell_entries] (padding = 0.0; may be
 * NULL), col_start / col_end int32[n_slices] (Sec. 5.1; may be NULL). */
spmv_status_t spmv_export_sell(spmv_matrix_t A, int64_t *slice_ptr, int32_t *col, double *values,
                               int32_t *col_start, int32_t *col_end);

/*
 * spmv_apply -- async.  y = A x (overwrites y) in the internal numbering (Sec. 4.3 / 5.2).
 * x_dev, y_dev: device double[n_rows] (FP64 / DUAL handles), 16-byte aligned; must not
 * overlap.
 * Summation order per row: ascending column, fused multiply-add from +0.0.
 */
spmv_status_t spmv_apply(spmv_matrix_t A, const double *x_dev, double *y_dev, void *stream);

/*
 * spmv_apply_host -- sync.  y = A x with x_host (double[n_cols]) and y_host (double[n_rows]) in
 * host memory, internal numbering, FP64 / DUAL handles.  The rows are cut into up to 8 runs of
 * slices; x goes to the device in increasing column order on `stream`, each run's product
 * starts as soon as the columns its slices read (Sec. 5.1 col_end) have arrived, and its rows
 * of y return to the host while later runs compute.  Page-locked host buffers make the copies
 * asynchronous DMA; pageable ones work, staged by the CUDA runtime.  The handle keeps device copies
 * of x and y (counted in device_bytes) and streams of its own.  y is bit-identical to
 * spmv_apply's.  Returns after y is on the host.  Calls on one handle from several host
 * threads must be serialised by the caller.
 */
spmv_status_t spmv_apply_host(spmv_matrix_t A, const double *x_host, double *y_host,
                              void *stream);

/*
 * spmv_apply_host_async -- async.  The same product, enqueued without waiting: `stream` reaches
 * the end of the call's work once y_host holds the result; until then the caller must not
 * change x_host or read y_host.  x, the product and y move in one piece each (no runs);
 * successive calls use three device staging sets in turn (3 x (n_cols + n_rows) doubles,
 * allocated on the first host call and counted in device_bytes), so calls issued on different
 * streams overlap (the copy of one call's x with an earlier call's y and with the products); a
 * staging set is reused only after its previous call is done with it.
 */
spmv_status_t spmv_apply_host_async(spmv_matrix_t A, const double *x_host, double *y_host,
                                    void *stream);

/* async.  y = alpha (A x) + beta y (the accumulating form of the paper's task signature, whose
 * result vector is read and written, Sec. 3.2): t = the row sum in column order, then
 * y_i = fma(alpha, t, beta * y_i), or alpha * t when beta == 0 (y is then not read, so it may
 * hold NaN).  x: double[n_cols], y: double[n_rows], 16-byte aligned, not overlapping.
 * FP64 / DUAL handles; the _f32 form takes FP32 vectors and scalars (FP32 / DUAL handles). */
spmv_status_t spmv_apply_axpby(spmv_matrix_t A, double alpha, const double *x_dev, double beta,
                               double *y_dev, void *stream);
spmv_status_t spmv_apply_axpby_f32(spmv_matrix_t A, float alpha, const float *x_dev, float beta,
                                   float *y_dev, void *stream);

/* async.  y = A32 x with FP32 values, vector and accumulation (FP32 / DUAL handles). */
spmv_status_t spmv_apply_f32(spmv_matrix_t A, const float *x_dev, float *y_dev, void *stream);

/* async.  Naive CSR kernel (thread per row, x gathered from global memory; Sec. 4.3),
 * kept as the baseline the sliced kernels are compared with.  FP64 / DUAL handles. */
spmv_status_t spmv_apply_csr(spmv_matrix_t A, const double *x_dev, double *y_dev, void *stream);

/*
 * spmv_apply_multi -- async.  Y = A X for k right-hand sides, X and Y row-major
 * (n_rows x k, entry (i, c) at i*k + c), device memory, FP64, 16-byte aligned, not
 * overlapping.  1 <= k <= 64.  Each gathered row of X is reused for all k columns: when k is a
 * power-of-two multiple of 32 bytes and X and Y are 32-byte aligned, each lane gathers 32 bytes
 * of a row with one 256-bit load; other power-of-two k use 8- or 16-byte vector loads.  Column
 * c equals spmv_apply on column c bit for bit.
 */
spmv_status_t spmv_apply_multi(spmv_matrix_t A, int k, const double *X_dev, double *Y_dev,
                               void *stream);
/* async.  FP32 version of spmv_apply_multi (FP32 / DUAL handles). */
spmv_status_t spmv_apply_multi_f32(spmv_matrix_t A, int k, const float *X_dev, float *Y_dev,
                                   void *stream);

/*
 * spmv_apply_chain -- async.  y = B (C x) for an operator chain (the operator-based formulation
 * evaluates a time step as chains of sparse products, Sec. 2): each entry b_if of B meets
 * t_f = sum_j c_fj x_j over row f of C in column order with fused multiply-add from +0.0, and
 * y_i = sum_f b_if t_f in B's column order, so y equals spmv_apply(B, spmv_apply(C, x)) bit for
 * bit.  Two forms compute it (B's chain_form option): one fused kernel that never writes C x
 * (it evaluates each row of C once per entry of B naming it), or the two sliced products
 * through a temporary t = C x kept by B's handle (allocated on the first call of that form,
 * counted in device_bytes).  Unset (AUTO), the two products run -- measured faster on GB300,
 * where t stays in L2 between them -- or, with autotune on, the first call times both forms
 * (synchronizing the stream) and keeps the faster for B.  Requires B's columns = C's rows
 * (B->n_cols == C->n_rows) and neither handle renumbered (no reorder, no sigma); FP64 values.
 * x: device double[C n_cols]; y: device double[B n_rows], 16-byte aligned, not overlapping x.
 */
spmv_status_t spmv_apply_chain(spmv_matrix_t B, spmv_matrix_t C, const double *x_dev,
                               double *y_dev, void *stream);

/* async.  FP32 version of spmv_apply_chain (FP32 / DUAL handles), with its own form choice:
 * y equals spmv_apply_f32(B, spmv_apply_f32(C, x)) bit for bit. */
spmv_status_t spmv_apply_chain_f32(spmv_matrix_t B, spmv_matrix_t C, const float *x_dev,
                                   float *y_dev, void *stream);

/* async.  Converts a vector between the caller's numbering and the internal one:
 * direction 0: out[new] = in[perm[new]]; direction 1: out[perm[new]] = in[new].
 * elem_bytes 4 or 8; in/out device arrays of n_rows elements, must not overlap. */
spmv_status_t spmv_permute(spmv_matrix_t A, int direction, int elem_bytes, const void *in_dev,
                           void *out_dev, void *stream);

/*
 * spmv_verify -- sync.  Verifies on the device that the handle's sliced ELLPACK arrays, slice
 * column ranges (Sec. 5.1), 16-bit offsets and renumbering hold the invariants listed above
 * (SPMV_CHECK_*), i.e. that every product kernel reads inside its arrays and reproduces the
 * CSR row sums.  *violations (may be NULL) receives the bits of the violated invariants.
 * Returns SPMV_OK when none is violated, SPMV_ERR_INVALID_CSR otherwise.  Not in the paper:
 * a device-side substitute for a memory checker.
 */
spmv_status_t spmv_verify(spmv_matrix_t A, int *violations, void *stream);

/*
 * spmv_diag_checks -- sync.  Self-test of spmv_verify: plants one fault at a time in device
 * copies of the handle's arrays (a column out of range, a changed value, a slice pointer off
 * by one, a wrong 16-bit offset, a column range that excludes its columns, a repeated row in
 * the renumbering; those that apply to the handle) and runs the checks on each copy.  The
 * handle is not modified.  *planted and *detected receive one bit per fault (1, 2, 4, 8, 16,
 * 32 in that order).  Returns SPMV_ERR_INVALID_ARG for a handle with fewer than 2 rows or no
 * stored entry.
 */
spmv_status_t spmv_diag_checks(spmv_matrix_t A, int *planted, int *detected, void *stream);

/*
 * spmv_device_status -- sync (waits for the stream).  Returns SPMV_ERR_TIMEOUT when a kernel
 * launched on the handle gave up one of its bounded waits since the handle was created or since
 * the last call (the staged product of SPMV_VARIANT_SELL_BULK waits on shared-memory barriers
 * for at most one second; a product that gave up left part of y unwritten), else SPMV_OK.  The
 * record is cleared.  INVALID_ARG for a NULL handle.
 */
spmv_status_t spmv_device_status(spmv_matrix_t A, void *stream);

/*
 * spmv_diag_bulk_timeout -- sync.  Self-test of the staged product's bounded waits: runs one
 * SPMV_VARIANT_SELL_BULK product of the handle (x = 0 in a scratch buffer; FP64 values when the
 * handle has them, else FP32) in which the first warp never copies its first slice, so that its
 * wait runs out after one second; the warp records the fact, waits for its other copies and
 * exits, while the rest of the product completes.  Returns SPMV_ERR_TIMEOUT when the expired
 * wait was recorded (the expected outcome; the record is cleared and the handle stays usable),
 * SPMV_ERR_CUDA when it was not, SPMV_ERR_UNSUPPORTED when the handle's slices do not fit the
 * staged product, INVALID_ARG for a NULL or empty handle.
 */
spmv_status_t spmv_diag_bulk_timeout(spmv_matrix_t A, void *stream);

/* ------------------------------ conjugate gradients ------------------------------------ */
typedef struct {
    double rtol;          /* stop when ||b - A x||_2 <= rtol ||b||_2 (default 1e-10)            */
    int max_iter;         /* CG iteration cap (FP64) or cap per inner solve (mixed); default 20000 */
    int mixed;            /* 0: FP64 Jacobi-PCG; 1: FP32 inner PCG + FP64 refinement (DUAL)   */
    double inner_rtol;    /* mixed: relative residual reduction of each inner solve (1e-4)    */
    int max_outer;        /* mixed: refinement steps cap (default 20)                          */
    int use_x0;           /* 1: x_dev holds the starting guess; 0: start from x = 0            */
    int persistent;       /* 1: one cooperative kernel per solve; 0: CUDA-graph batches of iterations */
    int check_every;      /* graph path: iterations per graph launch between host checks (16) */
    double timeout_s;     /* wall-clock limit of the solve, 0 = none                           */
    int adaptive_inner;   /* mixed: 1 = each inner solve stops at max(inner_rtol,
                           * 0.5 rtol ||b|| / ||r||), the reduction still missing (default 1) */
} cg_options_t;

typedef struct {
    int iterations;          /* CG iterations (mixed: inner iterations in total)        */
    int outer_iterations;    /* mixed: refinement steps; FP64: recurrence restarts      */
    double rel_residual;     /* ||b - A x||_2 / ||b||_2 recomputed in FP64 at the end   */
    spmv_status_t status;
} cg_result_t;

spmv_status_t cg_default_options(cg_options_t *opt);

/*
 * cg_solve -- sync.  Solves A x = b for SPD A by Jacobi-preconditioned CG (FP64), or with
 * opt->mixed by FP32 inner Jacobi-PCG and FP64 iterative refinement (residual, norms and the
 * update of x in FP64).  b_dev, x_dev: device double[n_rows] in the internal numbering.
 * Requires a square matrix (else INVALID_ARG) with a non-zero diagonal entry in every row.
 * Returns NOT_CONVERGED / TIMEOUT with
 * x_dev holding the last iterate; result (may be NULL) is filled in every case.
 */
spmv_status_t cg_solve(spmv_matrix_t A, const double *b_dev, double *x_dev, const cg_options_t *opt,
                       cg_result_t *result, void *stream);

/*
 * cg_solve_multi -- sync.  Solves A X = B for k right-hand sides at once: k Jacobi-PCG
 * recurrences (FP64, or with opt->mixed the FP32-inner / FP64 refinement of cg_solve, with the
 * same inner tolerance rule) advanced in lock-step, each iteration one multi-vector product
 * Q = A P in which every streamed matrix entry gathers one row of P for all k columns.  Not in
 * the paper, whose linear solver is SpMV-bound (Sec. 2): batching the systems that share a
 * matrix reads the matrix once per iteration instead of k times.  Each column keeps its own
 * step lengths and its own stop (a converged column keeps its x and drops out of the updates)
 * and restarts from its true residual as cg_solve does (at most twice).
 *   k: 1..32.  B_dev, X_dev: device double[n_rows * k], row-major (entry (i, c) at i*k + c),
 *   internal numbering, not overlapping.  X holds x0 when opt->use_x0, else it is
 *   overwritten (the solve starts from 0).  results: cg_result_t[k] (may be NULL): per column
 *   the iterations (mixed: inner iterations in total), the restarts (mixed: refinement steps),
 *   the true relative residual recomputed in FP64, and the column's status.
 *   opt->persistent: each recurrence runs as one cooperative kernel instead of CUDA-graph
 *   batches of check_every iterations; the results are identical bit for bit.
 * Returns SPMV_OK when every column converged, else the first failing column's status
 * (NOT_CONVERGED, TIMEOUT); INVALID_ARG, UNSUPPORTED (no FP64 values; mixed without FP32
 * values), OOM, CUDA as cg_solve.  The handle keeps the work arrays (five of n_rows * kp
 * doubles, kp = k rounded up to 8, 16 or 32, plus four of n_rows * kp floats for mixed),
 * counted in device_bytes.
 */
spmv_status_t cg_solve_multi(spmv_matrix_t A, int k, const double *B_dev, double *X_dev,
                             const cg_options_t *opt, cg_result_t *results, void *stream);

/*
 * spmv_diag_cg_timing -- sync.  Diagnostic of where an FP64 CG iteration's time goes on this
 * handle (not in the paper): the recurrence runs on b = 1 with no stopping test, and CUDA events
 * on `stream` time ms_out[0] one CUDA-graph batch of `iters` iterations, per iteration;
 * ms_out[1] the same kernels launched directly on the stream, per iteration; ms_out[2..4] the
 * product, the x/r sweep and the p sweep each between events of their own, per launch;
 * ms_out[5] a read-back of the scalar block to the host (the solve's convergence check), per
 * read.  ms_out: host double[6].  1 <= iters <= 4096.  Overwrites the handle's solve state.
 * INVALID_ARG for an empty or rectangular handle, UNSUPPORTED without FP64 values.
 */
spmv_status_t spmv_diag_cg_timing(spmv_matrix_t A, int iters, double *ms_out, void *stream);

/*
 * spmv_diag_barrier_timeout -- sync.  Self-test of the failure path of the persistent CG
 * kernel's bounded waits (not in the paper): launches `ctas` co-resident CTAs (1 <= ctas <= SM
 * count) on the kernel's grid barrier configured to expect one CTA more than exist, so no
 * wait is ever released; every CTA gives up after limit_s seconds (0 < limit_s <= 10) and
 * records the timeout.  Returns SPMV_ERR_TIMEOUT when the device reported the timeout as
 * designed, SPMV_ERR_CUDA otherwise.  Nothing faults or hangs.
 */
spmv_status_t spmv_diag_barrier_timeout(int ctas, double limit_s, void *stream);

/* ------------------------------ allocation-free solve ----------------------------------- */
/* Largest system (rows) that cg_solve_csr_noalloc accepts. */
#define SPMV_NOALLOC_MAX_ROWS 65536

/*
 * cg_solve_csr_noalloc -- sync.  The paper has no counterpart to this entry point.  It is for
 * callers that cannot allocate device memory when they solve, and therefore cannot create a
 * matrix handle (spmv_create allocates): for example a plugin inside a host application that
 * owns and pools all GPU memory itself, or a real-time loop whose memory is fixed in advance.
 * It solves A x = b by FP64 Jacobi-preconditioned CG (the iteration of cg_solve, with a
 * thread-per-row CSR product) directly on caller-owned device CSR arrays, and calls no
 * cudaMalloc, cudaFree or other allocating routine.  Its work vectors and reduction scratch
 * live in one fixed array inside the library (4 * SPMV_NOALLOC_MAX_ROWS doubles plus about
 * 33 KB of partial sums and scalars, about 2.1 MB).
 *   n <= SPMV_NOALLOC_MAX_ROWS, else SPMV_ERR_INVALID_ARG with no device work.  row_ptr_dev,
 *   col_idx_dev, values_dev: device CSR with the layout and checks of spmv_create (checked on
 *   the device: SPMV_ERR_INVALID_CSR, x untouched; a zero or missing diagonal is also
 *   INVALID_CSR).  b_dev, x_dev: device double[n]; x_dev holds x0 when opt->use_x0, else it is
 *   overwritten starting from 0.  opt->mixed and opt->persistent give SPMV_ERR_UNSUPPORTED.
 *   The call returns after the solve is complete (it waits on `stream`).
 * Set-up: the first call on a device (and the first after that device's context is replaced,
 * e.g. by cudaDeviceReset) looks up the array's device address (cudaGetSymbolAddress) with
 * that device current.  With the CUDA runtime's default lazy module loading, that first call
 * is also when the device reserves the array's 2.1 MB, which it then holds until the process
 * exits (with CUDA_MODULE_LOADING=EAGER it is reserved when the library is loaded).  A call
 * with n = 0 performs the set-up alone and returns SPMV_OK: make it on each device before the
 * application pools the device's memory, and before any stream capture begins.
 * All calls share the one array, which keeps the last call's contents; each call clears what
 * it needs at its start.  Calls that overlap on the GPU (other streams, other host threads)
 * race on the array and must be serialised by the caller.
 */
spmv_status_t cg_solve_csr_noalloc(int32_t n, int64_t nnz, const int32_t *row_ptr_dev,
                                   const int32_t *col_idx_dev, const double *values_dev,
                                   const double *b_dev, double *x_dev, const cg_options_t *opt,
                                   cg_result_t *result, void *stream);

/* ------------------------------ row-block partition with halo exchange ------------------ */
/*
 * A square matrix split into n_parts contiguous row blocks, one per GPU (or per process), for
 * matrices that do not fit one device or solves spread over several.  Not in the paper (its
 * kernel runs on one FPGA); after an RCM order (Sec. 4.1) each block's rows read columns of
 * their own block and of the neighbouring blocks only, so the exchange before each product is
 * a small halo.  Part p owns rows [row_begin[p], row_begin[p + 1]).  Its extended vector
 * x_ext = [halo below (n_halo_lo) | own entries (n_local) | halo above (n_halo_hi)] holds the
 * halo entries in increasing global column order, and its matrix is stored with columns
 * renumbered into x_ext monotonically, so each of its rows is the whole matrix's row in the
 * same column order: the parts' products concatenated equal spmv_apply on the whole matrix
 * bit for bit.  Exchange: part p sends to each part q (q ascending) the entries of its own x
 * that q's halo reads (send lists: own rows in increasing order), and receives from each q one
 * contiguous run of its halo (q ascending: the runs below its rows fill the low halo, those
 * above the high halo).
 */
typedef struct spmv_part_s *spmv_part_t;

typedef struct {
    int32_t n_parts, part;
    int32_t row_begin, row_end;  /* own rows (global numbering)                      */
    int32_t n_local;             /* row_end - row_begin                              */
    int32_t n_halo_lo;           /* halo entries with global column < row_begin      */
    int32_t n_halo_hi;           /* halo entries with global column >= row_end       */
    int32_t n_ext;               /* n_halo_lo + n_local + n_halo_hi                  */
    int64_t nnz_local;
    int32_t send_total;          /* entries this part sends per exchange             */
    int32_t recv_total;          /* n_halo_lo + n_halo_hi                            */
    size_t device_bytes;
} spmv_part_info_t;

/*
 * spmv_partition_create -- sync.  Part `part` of the partition of the square CSR matrix
 * (n rows, host arrays with the layout and checks of spmv_create, global numbering -- apply an
 * RCM order before partitioning, e.g. with spmv_get_permutation / spmv_export_csr of a
 * reordered handle).  row_begin: host int32[n_parts + 1], 0 = row_begin[0] <= ... <=
 * row_begin[n_parts] = n.  1 <= n_parts <= 4096.  on_device = 0 builds only the host-side plan
 * (halo, send lists, the part's CSR in the x_ext numbering: no CUDA call is made, for hosts
 * without a GPU); on_device = 1 also builds the part's device handle (opt as for spmv_create;
 * reorder and sigma must stay off so the global column order is kept).  Errors: INVALID_ARG,
 * INVALID_CSR (checked on the host), OOM, CUDA.
 */
spmv_status_t spmv_partition_create(int32_t n, int64_t nnz, const int32_t *row_ptr,
                                    const int32_t *col_idx, const double *values, int n_parts,
                                    const int32_t *row_begin, int part, int on_device,
                                    const spmv_options_t *opt, void *stream, spmv_part_t *out);
spmv_status_t spmv_partition_destroy(spmv_part_t P);
spmv_status_t spmv_partition_info(spmv_part_t P, spmv_part_info_t *info);

/* Host copies of the exchange plan (any output may be NULL): send_counts[n_parts] and
 * recv_counts[n_parts] (entries sent to / received from each part, 0 for itself),
 * send_rows[send_total] (own rows to send, local numbering, grouped by destination part
 * ascending), halo_cols[recv_total] (the halo's global columns, ascending). */
spmv_status_t spmv_partition_lists(spmv_part_t P, int32_t *send_counts, int32_t *recv_counts,
                                   int32_t *send_rows, int32_t *halo_cols);

/* Host copy of the part's CSR: row_ptr[n_local + 1], col_idx[nnz_local] (x_ext numbering),
 * values[nnz_local] (may be NULL). */
spmv_status_t spmv_partition_local_csr(spmv_part_t P, int32_t *row_ptr, int32_t *col_idx,
                                       double *values);

/* async.  send_dev[i] = x_own_dev[send_rows[i]] for the whole send list (device double
 * arrays: x_own of n_local entries -- the own part of an x_ext -- and send of send_total). */
spmv_status_t spmv_partition_pack(spmv_part_t P, const double *x_own_dev, double *send_dev,
                                  void *stream);

/* async.  y = A_part x_ext: x_ext device double[n_ext] with its halo in place, y device
 * double[n_local] (16-byte aligned, not overlapping). */
spmv_status_t spmv_partition_apply(spmv_part_t P, const double *x_ext_dev, double *y_dev,
                                   void *stream);

/* Transport callbacks of cg_solve_partitioned, called on the calling host thread with the
 * stream synchronised; each returns 0 on success.  exchange: send the part's send buffer
 * (device double[send_total], grouped by destination ascending) and fill recv (device
 * double[recv_total]) with the runs received from every other part, ascending.  allreduce:
 * replace values_host[0..count) by their sum over all parts. */
typedef int (*spmv_exchange_fn)(const double *send_dev, double *recv_dev, void *ctx);
typedef int (*spmv_allreduce_fn)(double *values_host, int count, void *ctx);

/*
 * cg_solve_partitioned -- sync, called by every part at once.  FP64 Jacobi-PCG of the
 * partitioned system: each part keeps its own rows of x, r, p, q; per iteration one halo
 * exchange of p and two scalar all-reduces (p.q; then r.(D^-1 r) and r.r), the recurrence of
 * cg_solve (its true-residual restarts excepted).  b_dev, x_dev: device double[n_local]; x
 * holds x0 when opt->use_x0.  result->rel_residual is the true ||b - A x|| / ||b|| over all
 * parts.  NOT_CONVERGED at the iteration cap; INVALID_CSR when any part has a row without a
 * non-zero diagonal; opt->mixed / persistent: UNSUPPORTED; a failing callback: CUDA.
 */
spmv_status_t cg_solve_partitioned(spmv_part_t P, const double *b_dev, double *x_dev,
                                   const cg_options_t *opt, cg_result_t *result,
                                   spmv_exchange_fn exchange, spmv_allreduce_fn allreduce,
                                   void *ctx, void *stream);

/* ------------------------------ continuous-batching server ------------------------------ */
typedef struct {
    uint64_t submitted, completed, rejected;
    int active_slots;        /* solves currently on the device                 */
    int queued;              /* admitted to the queue, waiting for memory/slot */
    size_t bytes_in_use;     /* device bytes held by active solves             */
    size_t peak_bytes;
    double p50_latency_s, p99_latency_s; /* over completed requests               */
    uint64_t cancelled;      /* requests that ended as SPMV_ERR_CANCELLED      */
    /* seconds summed over finished requests, per phase on the slot threads: setup (conversion
     * to sliced ELLPACK, copies of A and b), solve (cg_solve), teardown (copy of x, frees) */
    double setup_s, solve_s, teardown_s;
} spmv_server_stats_t;

/* Creates a server with a device-memory budget (bytes) and at most max_slots solves in flight.
 * Admission: a free slot takes the first queued request (in arrival order) whose estimated
 * footprint fits what the budget has left, so a large request waiting for memory does not
 * block smaller ones behind it; a request passed over 16 times is admitted next.
 * The server allocates from a stream-ordered memory pool of its own that keeps up to the
 * budget mapped after requests free it (released when the server is destroyed). */
spmv_status_t spmv_server_create(size_t hbm_budget_bytes, int max_slots, spmv_server_t *out);

/* Enqueues a solve of A x = b (host CSR + host b, copied before return).  opt->mixed selects
 * the precision; opt->persistent is ignored: the server launches every solve's kernels
 * directly on its slot's stream, so that concurrent solves overlap on the GPU (cooperative
 * launches from several streams do not, and a CUDA graph per one-off handle costs more to
 * build and destroy than it saves); the result is identical either way.
 * *ticket identifies the request.  BUDGET if it can never fit. */
spmv_status_t spmv_server_submit(spmv_server_t s, int32_t n, int64_t nnz, const int32_t *row_ptr,
                                 const int32_t *col_idx, const double *values, const double *b,
                                 const cg_options_t *opt, uint64_t *ticket);

/* PENDING until the request is done; then copies x (host double[n], original numbering) and
 * the result, releases the request and returns its status. */
spmv_status_t spmv_server_poll(spmv_server_t s, uint64_t ticket, double *x_host,
                               cg_result_t *result);

spmv_status_t spmv_server_get_stats(spmv_server_t s, spmv_server_stats_t *stats);

/* Requests whose estimated device footprint (the admission estimate) is at least `bytes` run
 * their kernels on a stream of the device's highest priority, so that when solves compete for
 * the SMs the large ones -- the tail of the latency distribution -- are scheduled first; 0
 * (the default) runs every request at the default priority.  Applies to requests admitted
 * after the call.  Results are unchanged (each request's kernels and reductions are the same
 * whatever stream runs them).  Server-side only: no counterpart in the paper. */
spmv_status_t spmv_server_set_priority_bytes(spmv_server_t s, size_t bytes);

/* Cancels a request.  A queued request never starts; a running solve stops at its next
 * convergence check (after each CUDA-graph batch of check_every iterations; a small system
 * running as one persistent kernel stops when that kernel returns), with none of its kernels
 * left in flight, and frees its device memory.  Either way the request then reports
 * SPMV_ERR_CANCELLED through poll, which leaves x_host untouched.  A request that had already
 * finished keeps its own status.  Returns SPMV_OK for any ticket not yet polled,
 * SPMV_ERR_INVALID_ARG otherwise.  Server-side only: no counterpart in the paper. */
spmv_status_t spmv_server_cancel(spmv_server_t s, uint64_t ticket);

/* Stops the worker, frees every request (finished or not) and the server. */
spmv_status_t spmv_server_destroy(spmv_server_t s);

#ifdef __cplusplus
}
#endif
#endif /* GB300_SPMV_H */
