// common.cuh -- internal declarations shared by the translation units of libsp2ell.
//
// Storage: row-major ELLPACK (the allocation listing of Section "Micro-Kernel Performance
// Evaluation - NUMA Aware Data": nnz[N], index[N*M], value[N*M]).  Row i's entries are
// slots i*w .. i*w+nnz[i]-1; padding slots are never read.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <cstddef>
#include <mutex>

#include "sp2ell.h"

namespace sp2 {

// ------------------------------------------------------------------ errors
void set_error(const char *fmt, ...);
int fail(int code, const char *fmt, ...);
int cuda_fail(cudaError_t e, const char *what, const char *file, int line);

#define SP2_CUDA(call)                                                             \
  do {                                                                             \
    cudaError_t e_ = (call);                                                       \
    if (e_ != cudaSuccess) return ::sp2::cuda_fail(e_, #call, __FILE__, __LINE__); \
  } while (0)

#define SP2_TRY(call)          \
  do {                         \
    int rc_ = (call);          \
    if (rc_ != SP2_OK) return rc_; \
  } while (0)

inline cudaStream_t as_stream(void *s) { return reinterpret_cast<cudaStream_t>(s); }

int num_sms();
// Ordinal of the current device, clamped to the 64 per-device cache entries.
int current_device();

// One-time per-device set-up of a launcher (kernel attributes, occupancy), safe against
// first calls made at the same time from several host threads: the set-up runs under a
// lock, and a failed set-up is retried on the next call.  value[dev] holds what the
// set-up stored (read after device_once returned SP2_OK).
struct DeviceOnce {
  std::mutex mu;
  bool done[64] = {false};
  int value[64] = {0};
};
template <typename F>
int device_once(DeviceOnce &o, int dev, F &&setup) {
  std::lock_guard<std::mutex> lk(o.mu);
  if (!o.done[dev]) {
    const int rc = setup(o.value[dev]);
    if (rc != 0) return rc;
    o.done[dev] = true;
  }
  return 0;
}
inline int round_up(int x, int m) { return ((x + m - 1) / m) * m; }
inline size_t round_up_sz(size_t x, size_t m) { return ((x + m - 1) / m) * m; }

// ------------------------------------------------------------------ profiling
// note_launch() after every kernel launch; prof_begin/prof_end bracket one launch of a
// class with CUDA events when the profiler is on (no-ops otherwise).
void note_launch();
void prof_begin(int cls, cudaStream_t s);
void prof_end(int cls, cudaStream_t s);

// ------------------------------------------------------------------ views
template <typename T>
struct EllView {  // read-only view
  int n, w;
  const int *__restrict__ idx;
  const T *__restrict__ val;
  const int *__restrict__ nnz;
};

template <typename T>
struct EllOut {  // writable view
  int n, w;
  int *idx;
  T *val;
  int *nnz;
};

template <typename T>
inline EllView<T> view(const ellpack_t *m) {
  return EllView<T>{m->n, m->width, m->idx, static_cast<const T *>(m->val), m->nnz};
}
template <typename T>
inline EllOut<T> outview(const ellpack_t *m) {
  return EllOut<T>{m->n, m->width, m->idx, static_cast<T *>(m->val), m->nnz};
}

int check_matrix(const ellpack_t *m, const char *name);
inline size_t dtype_size(int dt) { return dt == SP2_F64 ? sizeof(double) : sizeof(float); }

// ------------------------------------------------------------------ device memory
// Stream-ordered allocation helpers (cudaMallocAsync pool of the current device).
int dev_alloc(void **p, size_t bytes, cudaStream_t s);
void dev_free(void *p, cudaStream_t s);

// Grow-only scratch kept per device for the large-row fallback of the multiply:
// `slots` dense rows of n accumulators (T) and n marks (int, initialised to -1).
int fallback_scratch(int n, int dtype, int slots, void **acc, int **mark, cudaStream_t s);

// ------------------------------------------------------------------ per-step reductions
// Result of one multiply / trace pass, reduced in a fixed order (deterministic).
struct StepResult {
  double tr;           // sum of diagonal entries of the output
  double fro;          // sum of squares of the output entries
  long long nnz_total; // stored entries
  int max_nnz;         // longest row
  int overflow_rows;   // rows that did not fit the output width
  int max_count;       // longest post-threshold row, fitted or not
  int n_fallback;      // rows deferred from the per-warp tables to the 2^14-slot table
  int nonfinite;       // 1 if tr or fro is not finite
  int n_fallback2;     // rows deferred further to the dense global-row kernel
  int n_heavy;         // of n_fallback: rows sent on for the length of their row of A alone
  int n_routed;        // rows whose route flag sent them past the first pass unstarted
  int n_level1;        // rows the tight compact pass passed on to the loose one
  int n_level2;        // rows passed on to the full-row pass
};

// Device control block of one multiply launch.
struct SpgemmCtl {
  int overflow_rows;
  int max_count;
  int n_fallback;   // count of the first deferred-row list
  int n_fallback2;  // count of the second deferred-row list
  int n_fallbackw;  // count of the rows the window bin passes on
  int n_heavy;      // rows of the first list deferred for the length of their row of A
  int n_routed;     // rows the first pass of a cascade sent on unstarted (route flag)
  int n_level1;     // count of the list of the loose compact pass of a cascade
  int n_level2;     // count of the list of the full-row pass of a cascade
};

// Bitonic network over the 32*E keys a warp holds, E per lane in lane-major order
// (element lane*E + t): exchanges at distances below E stay in a lane's registers, the
// others pair lanes lane ^ (j / E) by shuffle.  Ascending on exit.
template <typename K, int E>
__device__ __forceinline__ void warp_bitonic(K (&a)[E], int lane) {
  static_assert(E == 1 || E == 2 || E == 4 || E == 8 || E == 16, "E: 1, 2, 4, 8 or 16 keys per lane");
  constexpr int LOGP = 5 + (E >= 2) + (E >= 4) + (E >= 8) + (E >= 16);
#pragma unroll
  for (int lk = 1; lk <= LOGP; ++lk) {
    const int k = 1 << lk;
#pragma unroll
    for (int lj = lk - 1; lj >= 0; --lj) {
      const int j = 1 << lj;
      if (j < E) {
#pragma unroll
        for (int t = 0; t < E; ++t) {
          if (t & j) continue;
          const int u = t | j;
          const bool asc = ((lane * E + t) & k) == 0;
          const K x = a[t], y = a[u];
          const bool sw = asc ? (x > y) : (x < y);
          a[t] = sw ? y : x;
          a[u] = sw ? x : y;
        }
      } else {
        const int m = j / E;
        const bool lower = (lane & m) == 0;
#pragma unroll
        for (int t = 0; t < E; ++t) {
          const K x = a[t];
          const K y = __shfl_xor_sync(0xffffffffu, x, m);
          const bool asc = ((lane * E + t) & k) == 0;
          const bool lo = x < y;
          a[t] = (asc == lower) ? (lo ? x : y) : (lo ? y : x);
        }
      }
    }
  }
}

// rowstat[r] = {diagonal value, sum of squares} of output row r (post-threshold).
// Reduces rowstat and out.nnz over n rows, copies ctl counters, into *res (device).
void launch_reduce_rows(const double2 *rowstat, const int *nnz, int n, const SpgemmCtl *ctl,
                        StepResult *res, cudaStream_t s);

// ------------------------------------------------------------------ kernels (host launchers)
// Multiply driver: out = drop_tau(alpha * A*B + beta * Add); Add may be null (beta ignored),
// may equal A (SP2 update 2X - X^2), or equal out (in-place BLAS form).
// Writes rowstat (n entries) and fills ctl; does not synchronise.
// Batched multiplies: the matrices of a batch are stacked as one block-diagonal ELLPACK
// (columns offset by each matrix's first row); each row reads its matrix's alpha, beta
// and active flag (rows of inactive matrices are left untouched, rowstat included).
struct BatchView {
  const int *row_mat = nullptr;   // per row: matrix id (null: one matrix, scalar alpha/beta)
  const double *alpha = nullptr;  // per matrix
  const double *beta = nullptr;   // per matrix (0: no addend)
  const int *active = nullptr;    // per matrix
};

// Upper-triangle mode of a symmetric product (X*X, X symmetric): row i accumulates only
// the columns j >= i.  tp[i*A.w + t] is the first position of row k = A.idx[i, t] of B
// with a column >= i (that source row is read from there on); tpd[i] is the same
// position in the addend row i.  Null pointers: full rows.
// Rows of one first pass of a cascade: all rows (list null) or the rows of a device list
// whose count a previous pass left at *count; level = the pass's compact level (0 tight,
// 1 loose, 2 full rows), compared with the per-row route flags.
struct PassRows {
  const int *list = nullptr;
  const int *count = nullptr;
  int level = 0;
};

// Symmetric products of fewer rows than this run the full-row first pass alone (cascade
// level 2, one launch): there a product takes tens of microseconds, and the two list passes
// of the cascade, launched whether or not any row reaches them, would cost more than the
// faster compact passes save.  (Measured on the N = 1024 banded SP2 as one graph: 7312
// iterations/s with three first-pass launches per product, about 7500 with one.)
constexpr int kCascadeMinRows = 2048;
inline int cascade_start(int n, bool upper, int compact_level) {
  if (!upper || n < kCascadeMinRows) return 2;
  return compact_level < 0 ? 0 : (compact_level > 2 ? 2 : compact_level);
}

// The SP2 loop of a small FP64 matrix in one cooperative launch (small.cu): X0 (n rows,
// width >= n) in, Y (n rows, width >= n) as the second buffer; the last iterate is in X0 or Y
// (*final_buf 0 or 1).  Fills the per-iterate records of *stats up to *iterations.  *status
// as sp2_stats.status, 3 for a non-finite trace, or 4 when an iterate grew a row too long for
// the one-launch loop: the host-stepped loop then continues from iterate *iterations (whose
// traces are recorded, its branch not yet taken) with the stall rule's *armed state; 5 when
// the context cannot launch the grid cooperatively (nothing ran).
// Errors: SP2E_TIMEOUT (a grid barrier waited too long), SP2E_CUDA.
constexpr int kSmallMaxN = 2048;
int small_purify(ellpack_t *X0, ellpack_t *Y, double nocc, double tol, const sp2_options &opt, int *iterations,
                 int *status, int *final_buf, int *armed, sp2_stats *stats, cudaStream_t s);

struct Upper {
  const int *tp = nullptr;
  const int *tpd = nullptr;
};

struct MultiplyArgs {
  const ellpack_t *A, *B, *Add;
  ellpack_t *Out;
  double alpha, beta, tau;
  int path;  // first pass: 0 automatic, 1..4 column blocks, 10..12 hash table
  BatchView bv{};              // per-row coefficients for batched multiplies
  int *fb_prealloc = nullptr;  // 3*n ints for the deferred-row lists (null: allocated per call)
  // X*X (+ X) with X symmetric (A == B, Add null or A): compute the upper triangle and
  // mirror it (bitwise the same result as full rows, about half the products)
  bool sym = false;
  // path 0 of a symmetric product: a cascade of first passes from this level on (0 the
  // tight compact variant, 1 the loose one, 2 the full-row variants), each over the rows
  // that outgrew the previous one; the rows that outgrow the full-row pass go to the bins
  int compact_level = 0;
  // per-row route flags (n bytes, or null) of the automatic first passes: the level a row
  // starts at.  A pass skips (passes on unstarted) a row flagged above its level, and
  // flags a row that outgrows its blocks with the next level, so that later products
  // start it there
  unsigned char *route = nullptr;
  void *sym_prealloc = nullptr;  // scratch of the symmetric product (null: allocated per call)
  size_t sym_prealloc_bytes = 0;
  Upper up{};  // set internally for the upper-triangle pass
};
// Scratch of a symmetric product with n rows, input width aw and output width ow.
inline size_t sym_scratch_bytes(int n, int aw, int ow, int dtype) {
  auto a256 = [](size_t b) { return ((b + 255) / 256) * 256; };
  const size_t es = dtype == SP2_F64 ? 8 : 4;
  return a256(es * (size_t)n * ow) + a256(4 * (size_t)n * ow) + a256(4 * (size_t)n) + a256(4 * (size_t)n * aw) +
         a256(4 * (size_t)n) + a256(4 * (3 * (size_t)n + 1));
}
// Symmetric product passes (symm.cu): first positions of the upper triangle; mirroring
// the upper rows U into full rows of Out (work: 3n+1 ints), rowstat of the full rows.
int upper_start_async(const ellpack_t *X, int *tp, int *tpd, cudaStream_t s);
// Entries of X without a bitwise-equal mirror entry (0: X is exactly symmetric); synchronises.
int symmetry_defects(const ellpack_t *X, long long *defects, cudaStream_t s);
int mirror_async(const ellpack_t *U, ellpack_t *Out, const BatchView &bv, int *work, double2 *rowstat, SpgemmCtl *ctl,
                 cudaStream_t s);
int multiply_async(const MultiplyArgs &a, double2 *rowstat, SpgemmCtl *ctl, cudaStream_t s);

// A <- drop_tau(alpha*A + beta*B), rowstat/ctl as above.
int add_async(ellpack_t *A, const ellpack_t *B, double alpha, double beta, double tau, double2 *rowstat,
              SpgemmCtl *ctl, cudaStream_t s);

// rowstat of an existing matrix (diag, sum of squares); the diagonal of local row r is
// column r + row0 (row0 > 0: A holds rows row0 .. of a larger matrix).
int rowstat_async(const ellpack_t *A, double2 *rowstat, cudaStream_t s, int row0 = 0);

// Gershgorin bounds into dev_bounds[0..1] = {emin, emax} (row0 as for rowstat_async: the
// bounds of the discs of rows row0 .. of a larger matrix).
int gershgorin_async(const ellpack_t *H, double *dev_bounds, cudaStream_t s, int row0 = 0);

// X0 = drop_tau((emax I - H)/(emax - emin)), bounds read from dev_bounds on the device.
// X->width >= H->width + 1, X->dtype == SP2_F64, H F64.
int x0_async(const ellpack_t *H, const double *dev_bounds, double tau, ellpack_t *X, cudaStream_t s, int row0 = 0);

// Element-type conversion (same n).  Rows longer than dst->width are left unwritten and
// counted in *overflow (device int, may be null).
int convert_async(const ellpack_t *src, ellpack_t *dst, cudaStream_t s, int *overflow = nullptr);

// Copies src into dst (same dtype; dst->width >= src row lengths; rows copied as is).
int copy_async(const ellpack_t *src, ellpack_t *dst, cudaStream_t s);

// Learned sizing (nnzpred.cu): structural counts of A*B (+C) into counts[n] with their
// maximum in *dmax (device); row features; predicted row lengths; prediction error
// {sum |log1p(pred) - log1p(actual)|, rows above prediction} into out2[2]; max of v.
int struct_count_async(const ellpack_t *A, const ellpack_t *B, const ellpack_t *C, int *counts, int *dmax,
                       cudaStream_t s);
int features_async(const ellpack_t *X, double tau, int branch, float *rmax_scratch, float *feat, cudaStream_t s);
int predict_async(const nnzpred_t *p, const float *feat, long long n, float *pred, cudaStream_t s);
// out2[0] = sum over rows of |log1p(pred) - log1p(actual)|, out2[1] = rows with actual > pred;
// out2 holds kPredErrDoubles doubles (the rest is scratch for the blocks' partial sums)
constexpr int kPredErrDoubles = 2 + 2 * 256;
int pred_error_async(const float *pred, const int *actual, long long n, double *out2, cudaStream_t s);
int max_float_async(const float *v, long long n, float *out, cudaStream_t s);
// Output width from the predictor's longest row: 10 % and 16 slots of margin.
inline long long predicted_width(float max_pred) { return (long long)ceil(1.10 * (double)max_pred) + 16; }

// Autotuner (tune.cu): mean stored row length of X (synchronises); the table entry for
// the class of a multiply (false if absent); timing every first-pass variant on the
// multiply `a`, recording the fastest in the table.
int mean_row_nnz(const ellpack_t *X, double *mean, cudaStream_t s);
bool tune_find(int dtype, int n, double mean_nnz, int *path);
int tune_multiply(MultiplyArgs a, double mean_nnz, double2 *rowstat, SpgemmCtl *ctl, int reps, int *best,
                  float *times, cudaStream_t s);

}  // namespace sp2
