/*
 * sp2ell.h -- C ABI of the GB300 (sm_103a) library for SP2 density-matrix purification
 * on thresholded ELLPACK sparse matrices.
 *
 * The method is the one the paper studies on multi-core CPUs: the SP2-Basic loop of the
 * ExaSP2 proxy application, whose phases are the ELLPACK matrix-matrix multiply X*X
 * ("SP2 Loop X2"), a norm ("SP2 Loop Norm") and the update ("SP2 Loop Misc")
 * (Section "Performance Evaluation using an ExaSP2 Application"), on the ELLPACK storage
 * of the allocation listing (arrays nnz[N], index[N*M], value[N*M]; Section
 * "Micro-Kernel Performance Evaluation - NUMA Aware Data").  The SP2 recursion itself
 * is the published one (Niklasson 2002, cited in the Introduction).
 *
 * Conventions
 *   - Every function returns int: SP2_OK (0) or a negative SP2E_* code.  A failing call
 *     leaves a message for sp2_last_error_string() (thread-local).
 *   - Arguments are checked before any launch; no exception crosses the ABI.
 *   - `stream` is a cudaStream_t passed as void* (NULL = the legacy default stream).
 *     Calls that return host scalars or a status that depends on device results
 *     synchronise that stream; the others are asynchronous.
 *   - All matrices are square, n x n, n >= 1.  Device arrays are row-major ELLPACK:
 *       idx[i*width + s], val[i*width + s] for s < nnz[i] hold row i's entries;
 *       slots s >= nnz[i] are never read and their contents are unspecified.
 *     A row never holds the same column twice.  Rows written by the library are sorted
 *     by ascending column.
 *   - One handle must not be used from two streams at the same time.  The library uses
 *     the current CUDA device; matrices must live on it.
 */
#ifndef SP2ELL_H
#define SP2ELL_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- status codes */
#define SP2_OK 0
#define SP2E_ARG (-1)        /* invalid argument (null pointer, bad size, aliasing, NaN/negative tau) */
#define SP2E_OVERFLOW (-2)   /* an output row needs more slots than the output width */
#define SP2E_NOMEM (-3)      /* device or pinned-host allocation failed */
#define SP2E_CUDA (-4)       /* a CUDA runtime call or kernel launch failed */
#define SP2E_NOTCONV (-5)    /* SP2 reached max_iter without meeting its stop rule */
#define SP2E_NONFINITE (-6)  /* a NaN or Inf appeared in an input or a reduction */
#define SP2E_TIMEOUT (-7)    /* a bounded device-side wait gave up */

/* ---------------------------------------------------------------- value types */
#define SP2_F64 0            /* double values */
#define SP2_F32 1            /* float values */

/*
 * ELLPACK matrix descriptor (plain struct, passed by pointer).
 *   n      rows (= columns)
 *   width  slots per row (the paper's M); library-allocated widths are multiples of 32
 *   dtype  SP2_F64 or SP2_F32: element type of val
 *   owner  1 when ellpack_create allocated the arrays (ellpack_destroy frees them),
 *          0 when they are borrowed from the caller (ellpack_wrap; never freed here)
 *   idx    device int32[n*width]
 *   val    device double[n*width] or float[n*width]
 *   nnz    device int32[n]
 */
typedef struct ellpack_t {
  int32_t n;
  int32_t width;
  int32_t dtype;
  int32_t owner;
  int32_t *idx;
  void *val;
  int32_t *nnz;
} ellpack_t;

/* Library version (major*10000 + minor*100 + patch). */
int sp2_version(void);

/* Message of the last failing call on this thread ("" if none). */
const char *sp2_last_error_string(void);

/* Returns to the driver the device memory the library keeps for reuse on the current
 * device (its stream-ordered allocations come from a library-owned pool that keeps freed
 * memory).  Synchronises the device.  Errors: SP2E_CUDA. */
int sp2_release_memory(void);

/*
 * Allocates an n x n ELLPACK matrix of the given width and dtype on the current device
 * (stream-ordered allocation on `stream`) and sets every nnz[i] to 0.  width >= 1 is
 * rounded up to a multiple of 32.  Errors: SP2E_ARG, SP2E_NOMEM, SP2E_CUDA.
 */
int ellpack_create(int32_t n, int32_t width, int32_t dtype, void *stream, ellpack_t *out);

/* Fills `out` with caller-owned device arrays (borrowed: never freed by the library).
 * width need not be a multiple of 32.  Errors: SP2E_ARG. */
int ellpack_wrap(int32_t n, int32_t width, int32_t dtype, int32_t *idx, void *val, int32_t *nnz,
                 ellpack_t *out);

/* Frees the arrays of a library-owned matrix (stream-ordered) and zeroes the descriptor;
 * a borrowed matrix is only zeroed.  Errors: SP2E_ARG, SP2E_CUDA. */
int ellpack_destroy(ellpack_t *m, void *stream);

/* Copies host arrays (same layout: idx[n*width], val[n*width], nnz[n]) to the device
 * matrix, asynchronously; host buffers must stay valid until the stream reaches the
 * copy (use pinned memory for overlap).  Errors: SP2E_ARG, SP2E_CUDA. */
int ellpack_upload(ellpack_t *m, const int32_t *h_idx, const void *h_val, const int32_t *h_nnz,
                   void *stream);

/* Copies the device matrix to host arrays of the same layout and synchronises the
 * stream.  Errors: SP2E_ARG, SP2E_CUDA. */
int ellpack_download(const ellpack_t *m, int32_t *h_idx, void *h_val, int32_t *h_nnz, void *stream);

/* The same copies, enqueued on `stream` without waiting: the host arrays hold the matrix
 * once the stream's work up to this point has completed (pinned host memory lets the
 * copies run beside kernels of other streams).  Errors: SP2E_ARG, SP2E_CUDA. */
int ellpack_download_async(const ellpack_t *m, int32_t *h_idx, void *h_val, int32_t *h_nnz, void *stream);

/* Device-to-device copy of rows: dst row i <- src row i (values converted when the
 * dtypes differ).  Same n; dst must not share arrays with src; dst->width may be smaller
 * than src->width as long as every row fits, else SP2E_OVERFLOW (those rows are left
 * unwritten).  Synchronises `stream`.  Errors: SP2E_ARG, SP2E_OVERFLOW, SP2E_CUDA. */
int ellpack_copy(const ellpack_t *src, ellpack_t *dst, void *stream);

/*
 * Thresholded ELLPACK matrix-matrix multiply (the paper's "ELLPACK X2" operation,
 * Section "Performance Evaluation using System Matrices"), BLAS gemm convention:
 *
 *     C <- drop_tau(alpha * A * B + beta * C)
 *
 *   pattern(C_i) = union over k in cols(A_i) of cols(B_k), plus the old cols(C_i) when
 *   beta != 0; an entry is kept iff |v| > tau (tau == 0 keeps every structural entry,
 *   exact zeros included); rows of C come out sorted by column.  The comparison with
 *   tau is made in the matrices' own precision.
 *   A, B, C must share n and dtype.  A and B may be the same matrix; C must not alias A
 *   or B (SP2E_ARG).  tau must be >= 0 and finite.
 *   required_width (optional, host): receives the largest post-threshold row length.
 *   Returns SP2E_OVERFLOW if some row needs more than C->width slots; C's contents are
 *   then unspecified and *required_width tells the width to allocate.  Synchronises
 *   `stream` (the status depends on device results).
 *   Errors: SP2E_ARG, SP2E_OVERFLOW, SP2E_NOMEM, SP2E_CUDA.
 */
int ellpack_multiply(const ellpack_t *A, const ellpack_t *B, ellpack_t *C, double alpha, double beta,
                     double tau, void *stream, int32_t *required_width);

/*
 * One row block of a thresholded product, for a product whose rows are spread over
 * several GPUs (the row-block split of the multiply; the paper's NUMA-aware placement of
 * row blocks, Section "Micro-Kernel Performance Evaluation - NUMA Aware Data", carried to
 * one block per GPU):
 *
 *     Out_r <- drop_tau(alpha * A_r * B + beta * C_r),   r = row0 .. row0 + A->n - 1
 *
 *   A, C and Out hold the block's rows (local row i is global row row0 + i) with global
 *   column indices; B has the global row count (B->n = the product's column count) and
 *   must hold every row k that A's entries name (local rows and the halo rows received
 *   from other GPUs); its other rows are never read and may be empty.  C may be NULL when
 *   beta == 0.  Keep rule, sorted rows and summation order as ellpack_multiply, so the
 *   blocks of a product are bitwise the rows of the whole product.
 *   trace, frobenius2 (optional, host): the block's share of tr(Out) (entries
 *   (i, row0 + i)) and of ||Out||_F^2, to be summed over the blocks.
 *   required_width (optional, host) and SP2E_OVERFLOW as for ellpack_multiply.
 *   Synchronises `stream`.  Errors: SP2E_ARG, SP2E_OVERFLOW, SP2E_NOMEM, SP2E_CUDA.
 */
int ellpack_multiply_block(const ellpack_t *A, int32_t row0, const ellpack_t *B, const ellpack_t *C, ellpack_t *Out,
                           double alpha, double beta, double tau, int32_t *required_width, double *trace,
                           double *frobenius2, void *stream);

/* The rest of the row-block split: the block's share of the set-up and of the traces.
 * Each takes the block's rows (local row i is global row row0 + i, global columns).
 *   ellpack_gershgorin_block: the Gershgorin bounds of the block's discs (the diagonal of
 *     local row i is column row0 + i); the global bounds are the minimum and maximum over
 *     the blocks.  Errors: SP2E_ARG, SP2E_NONFINITE, SP2E_CUDA.
 *   sp2_x0_block: X0's rows of the block from the global bounds, as sp2_x0 (the block's
 *     rows of drop_tau((emax I - H) / (emax - emin)), diagonal at column row0 + i).
 *     Errors: SP2E_ARG, SP2E_NOMEM, SP2E_CUDA.
 *   ellpack_stats_block: the block's share of tr X and of ||X||_F^2 (= tr X^2 for a
 *     symmetric X), the "SP2 Loop Norm" quantities (Section "Performance Evaluation using
 *     an ExaSP2 Application") to be summed over the blocks.  Errors: SP2E_ARG,
 *     SP2E_NONFINITE, SP2E_NOMEM, SP2E_CUDA.
 * All three synchronise `stream`. */
int ellpack_gershgorin_block(const ellpack_t *H, int32_t row0, double *emin, double *emax, void *stream);
int sp2_x0_block(const ellpack_t *H, int32_t row0, double emin, double emax, double tau, ellpack_t *X0,
                 void *stream);
int ellpack_stats_block(const ellpack_t *X, int32_t row0, double *trace, double *frobenius2, void *stream);

/* The halo of a row block: the distinct columns k that X's stored entries name outside the
 * block's rows row0 .. row0 + X->n - 1 (columns outside 0 .. ncols - 1 ignored), written
 * in ascending order to rows (device int32[ncols], caller-owned); *count (host) receives
 * how many.  These are the rows of X the block's product needs from other GPUs.
 * Synchronises `stream`.  Errors: SP2E_ARG, SP2E_NOMEM, SP2E_CUDA. */
int ellpack_halo_rows(const ellpack_t *X, int32_t row0, int32_t ncols, int32_t *rows, int32_t *count, void *stream);

/*
 * A <- drop_tau(alpha * A + beta * B) (the "SP2 Loop Misc" update, Section "Performance
 * Evaluation using an ExaSP2 Application"): pattern is the union of the two rows, keep
 * rule as in ellpack_multiply, rows sorted.  A and B share n and dtype and must not be
 * the same matrix.  Returns SP2E_OVERFLOW (A unspecified, *required_width set) if a
 * row does not fit A->width.  Synchronises `stream`.
 */
int ellpack_add(ellpack_t *A, const ellpack_t *B, double alpha, double beta, double tau, void *stream,
                int32_t *required_width);

/* tr A = sum_i A_ii, accumulated in FP64 in a fixed order (the "SP2 Loop Norm"
 * quantity).  Synchronises `stream`.  Errors: SP2E_ARG, SP2E_CUDA, SP2E_NONFINITE. */
int ellpack_trace(const ellpack_t *A, double *out, void *stream);

/* Squared Frobenius norm sum_ij A_ij^2 in FP64 (equal to tr A^2 for symmetric A).
 * Synchronises `stream`. */
int ellpack_frobenius2(const ellpack_t *A, double *out, void *stream);

/*
 * tr A and sum_ij A_ij^2, like ellpack_trace and ellpack_frobenius2 (same kernels, same
 * fixed summation order, so the same results), for callers that cannot allocate device
 * memory: for example a host application that reserves all of the GPU's memory for its
 * own pool at start-up and forbids any further allocation, or a latency-critical loop
 * where an allocation call and the synchronisation it may bring are not acceptable.
 * This entry point allocates nothing.  Its scratch is a fixed array of
 * SP2_NOALLOC_MAX_N * 16 + 256 bytes (1 MiB + 256 B) in the library's device image,
 * held by every GPU that loads the library until the process exits; n above
 * SP2_NOALLOC_MAX_N is rejected with SP2E_ARG.  The first call on a device looks up the
 * array's device address (cudaGetSymbolAddress) with that device current; make that
 * first call before any stream capture.  All calls share the one array: calls that
 * overlap on the GPU (other streams, other host threads) race and must not be issued.
 * The paper has no counterpart; it exists only for such callers.
 * trace (required) and frobenius2 (optional) are host pointers.  Synchronises `stream`.
 * Errors: SP2E_ARG, SP2E_CUDA, SP2E_NONFINITE.
 */
#define SP2_NOALLOC_MAX_N 65536
int ellpack_trace_noalloc(const ellpack_t *A, double *trace, double *frobenius2, void *stream);

/* Gershgorin bounds of H: e_min = min_i (H_ii - sum_{j!=i} |H_ij|),
 * e_max = max_i (H_ii + sum_{j!=i} |H_ij|), FP64.  Synchronises `stream`. */
int ellpack_gershgorin(const ellpack_t *H, double *emin, double *emax, void *stream);

/* ---------------------------------------------------------------- profiling */
/* Kernel classes timed by the profiler. */
#define SP2_PROF_SPGEMM 0   /* the first pass of the SpGEMM over every row (dominant) */
#define SP2_PROF_LARGE 1    /* the bins of deferred rows (window, 2^14-slot table, dense row) */
#define SP2_PROF_REDUCE 2   /* ordered trace/norm reductions */
#define SP2_PROF_OTHER 3    /* everything else (X0, conversions, add, Gershgorin) */
#define SP2_PROF_SYMM 4     /* symmetric products: lower-bound starts and the mirror of U */
#define SP2_PROF_CASCADE 5  /* the later first passes of a cascade (loose compact, full rows),
                               over the rows the earlier passes passed on */
#define SP2_PROF_CLASSES 6

typedef struct sp2_profile {
  int64_t launches;                   /* kernels launched by the library while enabled */
  int32_t count[SP2_PROF_CLASSES];    /* timed launches per class */
  double total_ms[SP2_PROF_CLASSES];  /* summed CUDA-event durations per class */
} sp2_profile;

/* Starts (and resets) the profiler of the calling process: from now on every kernel
 * launch is counted and the launches of the classes above are bracketed by CUDA events
 * recorded on the launching stream.  Errors: SP2E_CUDA. */
int sp2_profile_start(void);

/* Stops the profiler, waits for the recorded events and fills *out (may be NULL).
 * Errors: SP2E_CUDA. */
int sp2_profile_stop(sp2_profile *out);

/* Measured multiply-add rate of the current device in `dtype` (SP2_F64: DFMA, SP2_F32:
 * FFMA): a grid of 8 CTAs per SM runs independent fused multiply-add chains; one untimed
 * launch, then `reps` (1..1000) launches timed with CUDA events on `stream`.  *tflops
 * (host) receives the best rate in TFLOP/s (2 flop per FMA).  It is the ALU roofline that
 * the FP64 product is measured against (the paper has no counterpart: it measures on
 * CPUs).  Errors: SP2E_ARG, SP2E_NOMEM, SP2E_CUDA.  Synchronises `stream`. */
int sp2_fma_peak(int dtype, int reps, double *tflops, void *stream);

/* ---------------------------------------------------------------- learned sizing */
/*
 * Exact structural row counts of A*B (+ C when C is not NULL): counts[i] =
 * |union over k in cols(A_i) of cols(B_k)| (union cols(C_i)), an upper bound of the
 * post-threshold length of row i of the product.  counts: device int32[n];
 * max_count (optional, host) receives the largest.  A row whose columns fall in more than
 * 2048 groups of 32 reports min(n, sum of the lengths of the rows it gathers) instead
 * (still an upper bound).  Errors: SP2E_ARG (sizes or dtypes differ, or B has more than
 * 2^26 - 32 columns).  Synchronises `stream`.
 */
int ellpack_struct_count(const ellpack_t *A, const ellpack_t *B, const ellpack_t *C, int32_t *counts,
                         int32_t *max_count, void *stream);

#define NNZPRED_NPARAMS 5313  /* 16*64 + 64 + 64*64 + 64 + 64 + 1 */
#define NNZPRED_NSTATS 35     /* feature means[16], feature stds[16], target mean, target std,
                                 margin added to the predicted log1p length (0 until calibrated) */

/* A small MLP (16 -> 64 -> 64 -> 1, ReLU, FP32) predicting log1p of the post-threshold
 * length of each row of the next SP2 product from features of the current X. */
typedef struct nnzpred_t {
  float *params;   /* device: W1[64][16], b1[64], W2[64][64], b2[64], w3[64], b3 */
  float *adam_m;   /* device: Adam first moments  [NNZPRED_NPARAMS] */
  float *adam_v;   /* device: Adam second moments [NNZPRED_NPARAMS] */
  float *stats;    /* device: standardisation statistics [NNZPRED_NSTATS] */
  int64_t steps;   /* optimiser steps taken */
} nnzpred_t;

/*
 * Features of every row i of X (device float[n*16], row-major) for the product that the
 * SP2 step with `branch` (1 X^2, 2 2X - X^2) and drop tolerance tau will compute:
 *  0 log1p nnz_i, 1 log1p sum_k nnz_k, 2 log1p max_k nnz_k, 3 log1p min_k nnz_k,
 *  4 log10 max_k|x_ik|, 5 log10 ||x_i||_2, 6 log10 sum_k|x_ik|, 7 log10 |x_ii|,
 *  8 log10 sum_k |x_ik| max_j|x_kj|, 9 log1p #{|x_ik| > 10 tau}, 10 log1p #{|x_ik| > 100 tau},
 *  11 log10 tau, 12 branch == 2, 13 log1p (sum_k |x_ik| nnz_k / sum_k |x_ik|), 14 one, 15 zero
 * (k over the stored entries of row i).  Asynchronous.
 */
int nnzpred_features(const ellpack_t *X, double tau, int32_t branch, float *feat, void *stream);

/* Allocates the predictor (device) and initialises its weights from `seed` (uniform
 * +-sqrt(6/fan_in), biases 0, identity statistics).  Synchronises `stream`. */
int nnzpred_create(nnzpred_t *p, uint64_t seed, void *stream);
int nnzpred_destroy(nnzpred_t *p, void *stream);

/* Standardisation statistics from a training set: features feat[n*16] and exact row
 * lengths count[n] (device); the model works on standardised log1p(count). */
int nnzpred_set_stats(nnzpred_t *p, const float *feat, const int32_t *count, int64_t n, void *stream);

/* Gradient of the mean squared error over the n samples into grad[NNZPRED_NPARAMS]
 * (device) and the loss into *loss (host, optional).  Synchronises `stream`. */
int nnzpred_grad(const nnzpred_t *p, const float *feat, const int32_t *count, int64_t n, float *grad, float *loss,
                 void *stream);

/* `steps` Adam steps (lr, betas 0.9/0.999) on mini-batches of `batch` samples drawn by a
 * counter-based hash; *final_loss (host, optional) = loss of the last batch. */
int nnzpred_train(nnzpred_t *p, const float *feat, const int32_t *count, int64_t n, int32_t steps, int32_t batch,
                  float lr, float *final_loss, void *stream);

/* Predicted row lengths pred[n] (device float) from feat[n*16]: expm1(max(y + margin, 0))
 * with y the network's log1p length.  Asynchronous. */
int nnzpred_predict(const nnzpred_t *p, const float *feat, int64_t n, float *pred, void *stream);

/* Calibration: sets the margin to the smallest m >= 0 such that at least a fraction
 * `quantile` (in (0, 1]) of the n samples have log1p(count) <= y + m, so that the
 * predictions err on the long side for that share of the rows (a network fitted to the
 * mean under-predicts about half of them).  *margin (host, optional) receives it.
 * Synchronises `stream`.  Errors: SP2E_ARG, SP2E_NOMEM, SP2E_CUDA. */
int nnzpred_calibrate(nnzpred_t *p, const float *feat, const int32_t *count, int64_t n, float quantile,
                      float *margin, void *stream);

/* Output width for the product the SP2 step with `branch` and `tau` computes from X:
 * the features of X, the predicted row lengths (into pred, device float[n], optional),
 * and *width (host) = ceil(1.1 x the longest prediction) + 16 rounded up to 32 and capped
 * at n -- the rule sp2_purify uses with sizing 2.  Synchronises `stream`.
 * Errors: SP2E_ARG, SP2E_NOMEM, SP2E_CUDA. */
int nnzpred_width(const nnzpred_t *p, const ellpack_t *X, double tau, int32_t branch, int32_t *width, float *pred,
                  void *stream);

/* Weights and statistics to / from a file. */
int nnzpred_save(const nnzpred_t *p, const char *path, void *stream);
int nnzpred_load(nnzpred_t *p, const char *path, void *stream);

/* ---------------------------------------------------------------- standalone ops */
/*
 * Operations of the BML-style ELLPACK surface around the SP2 path (the paper names the
 * BML library and its ELLPACK format, Sections "Introduction" and "Performance
 * Evaluation using System Matrices"; these are their plain definitions on the stored
 * entries).  Rows stay sorted by column; results are bitwise reproducible.
 */

/* A <- alpha * A on the stored entries (pattern unchanged).  Asynchronous.
 * Errors: SP2E_ARG (alpha not finite). */
int ellpack_scale(ellpack_t *A, double alpha, void *stream);

/* Drops in place the stored entries with |v| <= tau (tau = 0 drops exact zeros); the
 * kept entries keep their order.  Asynchronous.  Errors: SP2E_ARG (tau < 0 or not finite). */
int ellpack_threshold(ellpack_t *A, double tau, void *stream);

/* out3 (host double[3]) = { max |a_ij|, max_i sum_j |a_ij| (infinity norm), ||A||_F },
 * FP64 over the stored entries.  Synchronises `stream`.  Errors: SP2E_ARG,
 * SP2E_NONFINITE (a NaN or Inf entry). */
int ellpack_norms(const ellpack_t *A, double *out3, void *stream);

/* At <- A^T (same n and dtype; At must not share arrays with A), rows sorted by column.
 * *required_width (optional) receives the longest column count of A; SP2E_OVERFLOW
 * (At unchanged) when it exceeds At->width.  Synchronises `stream`. */
int ellpack_transpose(const ellpack_t *A, ellpack_t *At, int32_t *required_width, void *stream);

/* dense (device, row-major n x ld, A's dtype, ld >= n) <- A, zeros elsewhere.
 * Asynchronous.  Errors: SP2E_ARG. */
int ellpack_to_dense(const ellpack_t *A, void *dense, int64_t ld, void *stream);

/* A <- the entries of the dense matrix (device, row-major n x ld, A's dtype) with v != 0
 * (tau = 0) or |v| > tau, in column order.  *required_width (optional) receives the
 * longest row; SP2E_OVERFLOW when a row does not fit A->width (its stored prefix is then
 * unspecified).  Synchronises `stream`. */
int ellpack_from_dense(const void *dense, int64_t ld, double tau, ellpack_t *A, int32_t *required_width,
                       void *stream);

/* ---------------------------------------------------------------- autotuner */
/*
 * The SpGEMM first pass has several variants that compute the same product (spgemm_path
 * 1, 2, 4: column-block accumulator shared by that many warps per row (7: 2 warps, fewer
 * accumulator slots per row, for the upper triangles of symmetric products); 3: one warp
 * per row, two k steps per pass (8: compact, as 7); 9: tiles of 8 consecutive rows sharing
 * one sorted column index, one warp per row; 10..12: per-warp hash table of 2^path
 * slots).  The tuner
 * times them on a real product and keeps the fastest per class (SM count, dtype,
 * floor(log2 n), floor(log2 mean stored row length of A)) in a process-wide host table
 * (thread-safe).  sp2_purify, sp2_step and sp2_purify_batched use the table when
 * spgemm_path is SP2_PATH_TUNED, tuning a class on its first product.  The paper has no
 * counterpart.
 */
#define SP2_PATH_TUNED (-1)
#define SP2_TUNE_CANDIDATES 10  /* 1, 2, 4, 7, 3, 8, 9, 10, 11, 12 in this order */

/* Times every variant on Out <- drop_tau(alpha A*B + beta C) (C may be NULL): one untimed
 * and `reps` timed runs each (CUDA events on `stream`); records the fastest for A's class
 * and returns it in *best_path; times_ms (optional, host float[SP2_TUNE_CANDIDATES])
 * receives the mean time of each.  Out is overwritten with the product (rows that do not
 * fit are left unspecified, as for ellpack_multiply).  Errors: SP2E_ARG, SP2E_NOMEM,
 * SP2E_CUDA.  Synchronises `stream`. */
int sp2_tune_spgemm(const ellpack_t *A, const ellpack_t *B, const ellpack_t *C, ellpack_t *Out, double alpha,
                    double beta, double tau, int32_t reps, int32_t *best_path, float *times_ms, void *stream);

/* Host-only table access (no GPU work).  sms = 0 in lookup means the current device;
 * *path = -1 when the class has no entry. */
int sp2_tune_record(int32_t sms, int32_t dtype, int32_t n, double mean_row_nnz, int32_t path, float ms);
int sp2_tune_lookup(int32_t sms, int32_t dtype, int32_t n, double mean_row_nnz, int32_t *path);
int sp2_tune_clear(void);
int sp2_tune_size(int32_t *entries);
/* Text file, one class per line ("sms dtype log2_n log2_mean_row path ms"); load merges
 * into the table (an entry replaces the same class).  SP2E_ARG for an unreadable or
 * malformed file (nothing is merged then). */
int sp2_tune_save(const char *path);
int sp2_tune_load(const char *path);

/* ---------------------------------------------------------------- SP2 */

#define SP2_PREC_F64 0      /* every step in FP64 */
#define SP2_PREC_MIXED 1    /* FP32 products and updates with FP64 traces, branch and tests
                               until err_n < switch_tol (or the FP32 loop stalls); then X is
                               promoted to FP64 and at least n_fp64_tail FP64 iterations run,
                               continuing until the FP64 stop rule holds */
#define SP2_PREC_F32 2      /* the FP32 loop of SP2_PREC_MIXED alone (no FP64 tail) */

#define SP2_STATS_CAP 256   /* per-iteration records kept in sp2_stats */

typedef struct sp2_options {
  int32_t precision;    /* SP2_PREC_F64 or SP2_PREC_MIXED */
  int32_t max_iter;     /* cap on updates (default 100) */
  int32_t stall_rule;   /* 1: stop once |trX - trX2| < stall_arm has been seen and
                           err_n >= stall_ratio * err_{n-2} */
  int32_t n_fp64_tail;  /* MIXED: minimum FP64 iterations after the switch (default 2) */
  int32_t max_width;    /* cap on the working width (0 = n); SP2E_OVERFLOW beyond it */
  int32_t spgemm_path;  /* SpGEMM first pass: 0 automatic (symmetric products, the
                           default: the cascade of route_rows, whose tight pass is the F64
                           path 7 / F32 path 8 form; full rows: F64 path 4, F32 path 3);
                           1, 2, 4 = column-block accumulator shared by that
                           many warps per row (7: 2 warps, compact blocks); 3 = column
                           blocks, one warp per row, two k steps per pass (8: compact);
                           9 = row tiles sharing a column index; 10..12 = per-warp hash
                           table of 2^k slots; SP2_PATH_TUNED = the autotuner's choice */
  double tau;           /* drop tolerance (default 1e-5) */
  double switch_tol;    /* MIXED: leave the FP32 loop once err_n < switch_tol (0 = automatic:
                           max(tol, 1e-4)); the FP32 stall rule also ends it */
  int32_t graph;        /* sp2_purify_batched: 1 = the loop runs as one CUDA graph with a
                           conditional WHILE node (default); 0 = host-stepped */
  int32_t sizing;       /* sp2_purify output widths: 0 heuristic (4x the longest row of X,
                           regrow on overflow), 1 exact structural counts before every
                           multiply, 2 1.1 x the predictor's longest row + 16 (after an
                           overflow the multiply is repeated at the exact width it counted) */
  const nnzpred_t *predictor;  /* for sizing 2 */
  double stall_arm;     /* the stall rule arms once |trX - trX2| < stall_arm (default 0.1) */
  int32_t symmetric;    /* 1 (default): H must be exactly symmetric (checked: SP2E_ARG
                           otherwise); every product computes its upper triangle and mirrors
                           it (the same result bit for bit, about half the products).
                           0: full rows, no check */
  double stall_ratio;   /* the armed stall rule fires once err_n >= stall_ratio * err_{n-2};
                           in (0, 1], default 1 (two updates brought no reduction); below 1
                           it also ends a slow monotone drift at the floor tau sets */
  int32_t route_rows;   /* automatic first pass (spgemm_path 0) of a symmetric product: a
                           cascade of passes, each over the rows that outgrew the previous
                           one's accumulator blocks: tight compact, loose compact, full rows,
                           then the deferred-row bins (below 2048 rows the full-row pass
                           alone, one launch instead of three).  1 = each row keeps a flag (on the
                           device) with the level it last needed, and later updates start it
                           there (default); 0 = every row starts at the cascade's first level */
  int32_t small_path;   /* 1 (default): FP64 runs (precision F64, spgemm_path 0, sizing 0, no
                           width cap below n) of at most 2048 rows take the loop in one
                           cooperative launch, each row built in a dense shared-memory
                           accumulator, until an iterate has a row longer than 64 entries;
                           the host-stepped loop continues from there.  The same rows bit
                           for bit, traces added in another order.  0: always the
                           host-stepped loop */
  double level_up_frac; /* the cascade starts at the tight compact level (fewest blocks per
                           row, most rows per SM); once its first pass passes on more than
                           this fraction of the rows in an update, it starts one level higher
                           (loose, then full rows) for the rest of the run.  > 0; default 1
                           (>= 1 keeps the tight start) */
} sp2_options;

typedef struct sp2_stats {
  int32_t iterations;                   /* updates applied */
  int32_t status;                       /* 0 err < tol, 1 stall rule, 2 max_iter */
  int32_t fp32_iterations;              /* MIXED: updates made in FP32 */
  int32_t regrows;                      /* multiplies repeated after a width overflow */
  int32_t struct_passes;                /* structural-count passes run */
  int32_t tuned;                        /* product classes tuned during the run (SP2_PATH_TUNED) */
  int32_t width_max;                    /* largest output width used */
  double pred_log_mae;                  /* sizing 2: mean |log1p(pred) - log1p(actual)| per row */
  double pred_under_frac;               /* sizing 2: fraction of rows longer than predicted */
  double emin, emax;                    /* Gershgorin bounds */
  double time_ms;                       /* wall time of the call */
  double trX[SP2_STATS_CAP];            /* per visited X_n (n = 0..iterations) */
  double trX2[SP2_STATS_CAP];           /* tr X_n^2, taken as ||X_n||_F^2 */
  double err[SP2_STATS_CAP];            /* |trX - trX2| / n */
  int32_t branch[SP2_STATS_CAP];        /* per update: 1 = X^2, 2 = 2X - X^2 */
  int64_t nnz_total[SP2_STATS_CAP];     /* per visited X_n */
  int32_t max_row_nnz[SP2_STATS_CAP];   /* per visited X_n */
  int32_t rows_level1[SP2_STATS_CAP];   /* per update: rows the tight compact pass passed
                                           on to the loose one (cascade) */
  int32_t rows_level2[SP2_STATS_CAP];   /* per update: rows passed on to the full-row pass */
  int32_t rows_deferred[SP2_STATS_CAP]; /* per update: rows handed to the deferred-row bins */
  int32_t rows_routed[SP2_STATS_CAP];   /* per update: rows whose route flag sent them past
                                           the cascade's first pass unstarted */
  int32_t level[SP2_STATS_CAP];         /* per update: the level the cascade of a symmetric
                                           product started at (0 tight, 1 loose, 2 full
                                           rows); -1 for other first passes (and for the
                                           updates of the one-launch loop) */
  int32_t small_iterations;             /* updates made by the one-launch loop (small_path);
                                           the host-stepped loop made the rest */
  int32_t pad;
} sp2_stats;

/*
 * SP2 initial guess (the "Init Misc" phase, Section "Performance Evaluation using an
 * ExaSP2 Application"): Gershgorin bounds of H, then
 *   X0 = drop_tau((e_max I - H) / (e_max - e_min)).
 * H F64.  X0 F64, X0->n == H->n, X0->width >= H->width + 1.  Row order of X0: the kept
 * entries of H's row left of the diagonal, the diagonal (always present unless it falls
 * below tau), then those right of it (sorted whenever H's row is sorted).  emin/emax
 * (optional, host) receive the bounds.  Synchronises `stream`.
 * Errors: SP2E_ARG (also e_max <= e_min), SP2E_NONFINITE, SP2E_CUDA.
 */
int sp2_x0(const ellpack_t *H, double tau, ellpack_t *X0, double *emin, double *emax, void *stream);

/* One SP2 iteration: in/out record of sp2_step. */
typedef struct sp2_step_info {
  double trX, trX2;        /* in when have_traces == 1 (else computed): tr X, ||X||_F^2 */
  int32_t have_traces;     /* in */
  int32_t branch;          /* out: 1 = X^2, 2 = 2X - X^2 */
  double err;              /* out: |trX - trX2| / n of the input X */
  double trXn, trXn2;      /* out: tr X', ||X'||_F^2 of the result */
  int64_t nnz_total;       /* out: stored entries of X' */
  int32_t max_row_nnz;     /* out: longest row of X' */
  int32_t required_width;  /* out: longest post-threshold row (valid on overflow too) */
  int32_t spgemm_path;     /* in: SpGEMM first pass, as sp2_options.spgemm_path */
  int32_t rows_deferred;   /* out: rows the first pass (for spgemm_path 0 of a symmetric
                              product: the last pass of the cascade) handed to the
                              deferred-row bins (the shared-memory window, then the
                              2^14-slot table): rows that outgrew its accumulator, and with
                              the one-warp passes rows of X longer than 512 entries */
  int32_t rows_dense;      /* out: rows handed further to the dense global-row pass */
  int32_t spgemm_path_used; /* out: the first-pass variant that ran (the tuner's choice
                               for SP2_PATH_TUNED) */
  int32_t symmetric;       /* in: 1 = X is exactly symmetric (not checked): the product's
                              upper triangle is computed and mirrored */
  int32_t compact_level;   /* in: symmetric product with spgemm_path 0: the level its
                              cascade of first passes starts at, 0 tight (the default),
                              1 loose, 2 full rows */
} sp2_step_info;

/*
 * One SP2 iteration on X (the "SP2 Loop X2 / Norm / Misc" phases): with
 *   trX = tr X, trX2 = ||X||_F^2 (= tr X^2 for symmetric X),
 *   X' = drop_tau(2X - X*X) if |2 trX - trX2 - nocc| < |trX2 - nocc|, else drop_tau(X*X),
 * computed in one fused pass whose epilogue also yields tr X' and ||X'||_F^2 (FP64).
 * X and X' share n and dtype and must not share arrays.  Returns SP2E_OVERFLOW when a
 * row of X' needs more than Xn->width slots (info->required_width tells how many).
 * Synchronises `stream`.  Errors: SP2E_ARG, SP2E_OVERFLOW, SP2E_NONFINITE, SP2E_CUDA.
 */
int sp2_step(const ellpack_t *X, ellpack_t *Xn, double nocc, double tau, sp2_step_info *info, void *stream);

/* Fills *opt with the defaults (F64, max_iter 100, stall rule on, tail 2, tau 1e-5,
 * symmetric products, route flags on, the cascade kept at the tight start). */
void sp2_options_default(sp2_options *opt);

/*
 * SP2 purification (SP2-Basic, Section "Performance Evaluation using an ExaSP2
 * Application"; recursion of Niklasson 2002):
 *   e_min, e_max = Gershgorin bounds of H
 *   X_0 = drop_tau((e_max I - H) / (e_max - e_min))  (diagonal always in the pattern)
 *   for n = 0, 1, ...:  trX = tr X_n, trX2 = ||X_n||_F^2,  err_n = |trX - trX2| / N
 *       stop if err_n < tol, or (stall_rule) |trX - trX2| < 0.1 has been seen and
 *       err_n >= err_{n-2}, or n == max_iter
 *       X_{n+1} = drop_tau(2X_n - X_n^2) if |2 trX - trX2 - nocc| < |trX2 - nocc|,
 *                 else drop_tau(X_n^2)
 * H: symmetric, F64 (an F32 H is accepted and promoted).  nocc in (0, n).  tol > 0.
 * opt may be NULL (defaults).  On success *D receives a new library-owned F64 matrix
 * (release with ellpack_destroy) and *stats (optional) the per-iteration record.
 * Returns SP2_OK, or SP2E_NOTCONV with D still set when max_iter was reached.
 * Errors: SP2E_ARG, SP2E_NOMEM, SP2E_CUDA, SP2E_OVERFLOW (max_width too small),
 * SP2E_NONFINITE, SP2E_TIMEOUT (small_path: a grid barrier of the one-launch loop saw no
 * progress for about a second); after an error *stats holds the iterations recorded before
 * it.  Synchronises `stream` (with small_path, `stream` must not be under graph capture).
 */
int sp2_purify(const ellpack_t *H, double nocc, double tol, const sp2_options *opt, ellpack_t *D,
               sp2_stats *stats, void *stream);

/*
 * Batched SP2: `count` independent purifications (Hamiltonians of any sizes) in one
 * device-resident loop.  The matrices are stacked block-diagonally so that every SpGEMM
 * launch covers all rows of all matrices still running; each matrix keeps its own
 * traces, branch, stop rule (the rules of sp2_purify) and, in SP2_PREC_MIXED, its own
 * FP32 -> FP64 switch, all decided on the device.  With opt->graph (default) the loop is
 * one CUDA graph with a conditional WHILE node, launched once.
 * H[m]: F64 matrices (host array of descriptors); nocc[m] in (0, H[m].n); tol > 0.
 * On success D[m] receives a new library-owned F64 matrix each (release with
 * ellpack_destroy) and stats[m] (optional) the per-iteration record of matrix m.
 * Returns SP2E_NOTCONV (D still set) if some matrix reached max_iter.  If a row
 * outgrows the working width the loop restarts wider (stats[m].regrows counts it).
 * The products are shared by the batch: the per-update row counts of stats[m] stay 0.
 * Errors: SP2E_ARG, SP2E_NOMEM, SP2E_CUDA, SP2E_OVERFLOW, SP2E_NONFINITE.  Synchronises
 * `stream` (NULL: a private stream is used for the graph).
 */
int sp2_purify_batched(const ellpack_t *H, const double *nocc, int32_t count, double tol, const sp2_options *opt,
                       ellpack_t *D, sp2_stats *stats, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* SP2ELL_H */
