// ops.cu -- standalone ELLPACK operations of a BML-like matrix library: scale, drop
// threshold, norms, transpose, and conversion to and from dense row-major arrays.
//
// All use one warp per row; a row's stored entries stay sorted by column.  Reductions
// take a fixed order (per-row values, then one CTA over the rows), so every result is
// bitwise reproducible.
#include <math.h>

#include "common.cuh"

namespace sp2 {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kOpsThreads = 256;

int grid_warps_rows(long long rows) {
  long long b = (rows * 32 + kOpsThreads - 1) / kOpsThreads;
  const long long cap = (long long)num_sms() * 16;
  return (int)(b < 1 ? 1 : (b < cap ? b : cap));
}

__device__ __forceinline__ unsigned lanes_below() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

template <typename T>
__global__ void scale_kernel(EllOut<T> A, T alpha) {
  const int lane = threadIdx.x & 31;
  const int warps = (gridDim.x * blockDim.x) >> 5;
  for (int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < A.n; r += warps) {
    const int k = min(A.nnz[r], A.w);
    for (int s = lane; s < k; s += 32) A.val[(size_t)r * A.w + s] *= alpha;
  }
}

// In-place drop: keep |v| > tau (the row order is kept; one ballot per 32 entries).
template <typename T>
__global__ void threshold_kernel(EllOut<T> A, T tau) {
  const int lane = threadIdx.x & 31;
  const int warps = (gridDim.x * blockDim.x) >> 5;
  const unsigned lt = lanes_below();
  for (int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < A.n; r += warps) {
    const int k = min(A.nnz[r], A.w);
    int *ri = A.idx + (size_t)r * A.w;
    T *rv = A.val + (size_t)r * A.w;
    int out = 0;
    for (int s0 = 0; s0 < k; s0 += 32) {
      const int s = s0 + lane;
      int j = 0;
      T v = T(0);
      bool keep = false;
      if (s < k) {
        j = ri[s];
        v = rv[s];
        keep = fabs((double)v) > (double)tau;
      }
      const unsigned m = __ballot_sync(kFull, keep);
      __syncwarp();  // every lane has read its entry before any is overwritten
      if (keep) {
        const int p = out + __popc(m & lt);
        ri[p] = j;
        rv[p] = v;
      }
      out += __popc(m);
      __syncwarp();
    }
    if (lane == 0) A.nnz[r] = out;
  }
}

// Per row: max |a_ij| and sum_j |a_ij| into rows[r] = {max, sum, sum of squares}.
template <typename T>
__global__ void rownorm_kernel(EllView<T> A, double *__restrict__ rows) {
  const int lane = threadIdx.x & 31;
  const int warps = (gridDim.x * blockDim.x) >> 5;
  for (int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < A.n; r += warps) {
    const int k = min(A.nnz[r], A.w);
    double mx = 0.0, sm = 0.0, sq = 0.0;
    for (int s = lane; s < k; s += 32) {
      const double v = fabs((double)A.val[(size_t)r * A.w + s]);
      mx = fmax(mx, v);
      sm += v;
      sq = fma(v, v, sq);
    }
    for (int o = 16; o > 0; o >>= 1) {
      mx = fmax(mx, __shfl_xor_sync(kFull, mx, o));
      sm += __shfl_xor_sync(kFull, sm, o);
      sq += __shfl_xor_sync(kFull, sq, o);
    }
    if (lane == 0) {
      rows[3 * (size_t)r] = mx;
      rows[3 * (size_t)r + 1] = sm;
      rows[3 * (size_t)r + 2] = sq;
    }
  }
}

// One CTA: out = {max_r max, max_r sum, sqrt(sum_r squares)}; thread t takes rows t, t+T, ...
// in order, then a fixed tree.
__global__ void norms_reduce_kernel(const double *__restrict__ rows, int n, double *__restrict__ out) {
  __shared__ double s_mx[kOpsThreads], s_in[kOpsThreads], s_sq[kOpsThreads];
  double mx = 0.0, in = 0.0, sq = 0.0;
  for (int r = threadIdx.x; r < n; r += kOpsThreads) {
    mx = fmax(mx, rows[3 * (size_t)r]);
    in = fmax(in, rows[3 * (size_t)r + 1]);
    sq += rows[3 * (size_t)r + 2];
  }
  s_mx[threadIdx.x] = mx;
  s_in[threadIdx.x] = in;
  s_sq[threadIdx.x] = sq;
  __syncthreads();
  for (int h = kOpsThreads / 2; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h) {
      s_mx[threadIdx.x] = fmax(s_mx[threadIdx.x], s_mx[threadIdx.x + h]);
      s_in[threadIdx.x] = fmax(s_in[threadIdx.x], s_in[threadIdx.x + h]);
      s_sq[threadIdx.x] += s_sq[threadIdx.x + h];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[0] = s_mx[0];
    out[1] = s_in[0];
    out[2] = sqrt(s_sq[0]);
  }
}

// Transpose, pass 1: entries per column (integer atomics: exact).
template <typename T>
__global__ void col_count_kernel(EllView<T> A, int ncol, int *__restrict__ cnt) {
  const int lane = threadIdx.x & 31;
  const int warps = (gridDim.x * blockDim.x) >> 5;
  for (int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < A.n; r += warps) {
    const int k = min(A.nnz[r], A.w);
    for (int s = lane; s < k; s += 32) {
      const int j = A.idx[(size_t)r * A.w + s];
      if ((unsigned)j < (unsigned)ncol) atomicAdd(cnt + j, 1);
    }
  }
}

// Transpose, pass 2: entry (r, j) goes to row j of At at a slot taken from a per-column
// cursor; pass 3 sorts each row of At by column (the slots are a permutation, so the
// sorted row is unique whatever order pass 2 filled it in).
template <typename T>
__global__ void col_scatter_kernel(EllView<T> A, EllOut<T> At, int *__restrict__ cursor) {
  const int lane = threadIdx.x & 31;
  const int warps = (gridDim.x * blockDim.x) >> 5;
  for (int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < A.n; r += warps) {
    const int k = min(A.nnz[r], A.w);
    for (int s = lane; s < k; s += 32) {
      const int j = A.idx[(size_t)r * A.w + s];
      if ((unsigned)j >= (unsigned)At.n) continue;
      const int p = atomicAdd(cursor + j, 1);
      if (p < At.w) {
        At.idx[(size_t)j * At.w + p] = r;
        At.val[(size_t)j * At.w + p] = A.val[(size_t)r * A.w + s];
      }
    }
  }
}

// Sort each row by column: rank of an entry = number of entries with a smaller column
// (columns within a row are distinct), computed against the whole row; the row is
// staged in shared memory (rows up to kSortMax entries; longer rows take the same rank
// computation from global memory into a scratch row).
constexpr int kSortWarps = 8, kSortMax = 512;
static_assert(kSortWarps * 32 == kOpsThreads, "the sort runs on the row grid of the other passes");

template <typename T>
__global__ void __launch_bounds__(kSortWarps * 32) row_sort_kernel(EllOut<T> At, const int *__restrict__ cnt,
                                                                   int *__restrict__ scr_i, T *__restrict__ scr_v) {
  __shared__ int si[kSortWarps][kSortMax];
  __shared__ T sv[kSortWarps][kSortMax];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int warps = gridDim.x * kSortWarps;
  for (int r = blockIdx.x * kSortWarps + wid; r < At.n; r += warps) {
    const int k = min(cnt[r], At.w);
    int *ri = At.idx + (size_t)r * At.w;
    T *rv = At.val + (size_t)r * At.w;
    const bool small = k <= kSortMax;
    int *ci = small ? si[wid] : scr_i + (size_t)r * At.w;
    T *cv = small ? sv[wid] : scr_v + (size_t)r * At.w;
    for (int s = lane; s < k; s += 32) {
      ci[s] = ri[s];
      cv[s] = rv[s];
    }
    __syncwarp();
    for (int s = lane; s < k; s += 32) {
      const int c = ci[s];
      int rank = 0;
      for (int t = 0; t < k; ++t) rank += ci[t] < c;
      ri[rank] = c;
      rv[rank] = cv[s];
    }
    if (lane == 0) At.nnz[r] = k;
    __syncwarp();
  }
}

template <typename T>
__global__ void to_dense_kernel(EllView<T> A, T *__restrict__ dense, long long ld) {
  const int lane = threadIdx.x & 31;
  const int warps = (gridDim.x * blockDim.x) >> 5;
  for (int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < A.n; r += warps) {
    const int k = min(A.nnz[r], A.w);
    for (int s = lane; s < k; s += 32) {
      const int j = A.idx[(size_t)r * A.w + s];
      if ((unsigned)j < (unsigned)ld) dense[(size_t)r * ld + j] = A.val[(size_t)r * A.w + s];
    }
  }
}

// Dense row r -> ELLPACK row: keep v != 0 (tau == 0) or |v| > tau, in column order;
// rows longer than the width are counted (their stored prefix is unspecified).
template <typename T>
__global__ void from_dense_kernel(const T *__restrict__ dense, long long ld, int ncol, T tau, EllOut<T> A,
                                  int *__restrict__ ctl) {
  const int lane = threadIdx.x & 31;
  const int warps = (gridDim.x * blockDim.x) >> 5;
  const unsigned lt = lanes_below();
  int wmax = 0, wover = 0;
  for (int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < A.n; r += warps) {
    const T *row = dense + (size_t)r * ld;
    int out = 0;
    for (int c0 = 0; c0 < ncol; c0 += 32) {
      const int c = c0 + lane;
      const T v = c < ncol ? row[c] : T(0);
      const bool keep = c < ncol && (tau == T(0) ? v != T(0) : fabs((double)v) > (double)tau);
      const unsigned m = __ballot_sync(kFull, keep);
      if (keep) {
        const int p = out + __popc(m & lt);
        if (p < A.w) {
          A.idx[(size_t)r * A.w + p] = c;
          A.val[(size_t)r * A.w + p] = v;
        }
      }
      out += __popc(m);
    }
    if (lane == 0) A.nnz[r] = min(out, A.w);
    wmax = max(wmax, out);
    wover += out > A.w;
  }
  if (lane == 0) {
    if (wmax) atomicMax(ctl, wmax);
    if (wover) atomicAdd(ctl + 1, wover);
  }
}

__global__ void int_max_kernel(const int *__restrict__ c, int n, int *__restrict__ out) {
  int m = 0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) m = max(m, c[i]);
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(kFull, m, o));
  if ((threadIdx.x & 31) == 0 && m) atomicMax(out, m);
}

int sync_read(void *host, const void *dev, size_t bytes, cudaStream_t s, const char *who) {
  cudaError_t e = cudaMemcpyAsync(host, dev, bytes, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, who, __FILE__, __LINE__);
  return SP2_OK;
}

}  // namespace
}  // namespace sp2

using namespace sp2;

extern "C" int ellpack_scale(ellpack_t *A, double alpha, void *stream) {
  SP2_TRY(check_matrix(A, "ellpack_scale"));
  if (!isfinite(alpha)) return fail(SP2E_ARG, "ellpack_scale: alpha not finite");
  cudaStream_t s = as_stream(stream);
  if (A->dtype == SP2_F64) scale_kernel<double><<<grid_warps_rows(A->n), kOpsThreads, 0, s>>>(outview<double>(A), alpha);
  else scale_kernel<float><<<grid_warps_rows(A->n), kOpsThreads, 0, s>>>(outview<float>(A), (float)alpha);
  note_launch();
  SP2_CUDA(cudaGetLastError());
  return SP2_OK;
}

extern "C" int ellpack_threshold(ellpack_t *A, double tau, void *stream) {
  SP2_TRY(check_matrix(A, "ellpack_threshold"));
  if (!(tau >= 0.0) || !isfinite(tau)) return fail(SP2E_ARG, "ellpack_threshold: tau must be finite and >= 0");
  cudaStream_t s = as_stream(stream);
  if (A->dtype == SP2_F64)
    threshold_kernel<double><<<grid_warps_rows(A->n), kOpsThreads, 0, s>>>(outview<double>(A), tau);
  else
    threshold_kernel<float><<<grid_warps_rows(A->n), kOpsThreads, 0, s>>>(outview<float>(A), (float)tau);
  note_launch();
  SP2_CUDA(cudaGetLastError());
  return SP2_OK;
}

extern "C" int ellpack_norms(const ellpack_t *A, double *out3, void *stream) {
  SP2_TRY(check_matrix(A, "ellpack_norms"));
  if (!out3) return fail(SP2E_ARG, "ellpack_norms: out is NULL");
  cudaStream_t s = as_stream(stream);
  double *rows = nullptr;
  SP2_TRY(dev_alloc((void **)&rows, sizeof(double) * (3 * (size_t)A->n + 3), s));
  if (A->dtype == SP2_F64) rownorm_kernel<double><<<grid_warps_rows(A->n), kOpsThreads, 0, s>>>(view<double>(A), rows);
  else rownorm_kernel<float><<<grid_warps_rows(A->n), kOpsThreads, 0, s>>>(view<float>(A), rows);
  note_launch();
  double *res = rows + 3 * (size_t)A->n;
  norms_reduce_kernel<<<1, kOpsThreads, 0, s>>>(rows, A->n, res);
  note_launch();
  int rc = SP2_OK;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) rc = cuda_fail(e, "ellpack_norms", __FILE__, __LINE__);
  if (rc == SP2_OK) rc = sync_read(out3, res, 3 * sizeof(double), s, "ellpack_norms");
  dev_free(rows, s);
  SP2_TRY(rc);
  if (!isfinite(out3[0]) || !isfinite(out3[1]) || !isfinite(out3[2]))
    return fail(SP2E_NONFINITE, "ellpack_norms: non-finite entries");
  return SP2_OK;
}

extern "C" int ellpack_transpose(const ellpack_t *A, ellpack_t *At, int32_t *required_width, void *stream) {
  SP2_TRY(check_matrix(A, "ellpack_transpose: A"));
  SP2_TRY(check_matrix(At, "ellpack_transpose: At"));
  if (A->n != At->n || A->dtype != At->dtype) return fail(SP2E_ARG, "ellpack_transpose: n or dtype differ");
  if (A->idx == At->idx || A->val == At->val || A->nnz == At->nnz)
    return fail(SP2E_ARG, "ellpack_transpose: At aliases A");
  cudaStream_t s = as_stream(stream);
  const int n = A->n;
  int *cnt = nullptr;
  SP2_TRY(dev_alloc((void **)&cnt, sizeof(int) * 2 * (size_t)n, s));
  int *cursor = cnt + n;
  int rc = SP2_OK;
  cudaError_t e = cudaMemsetAsync(cnt, 0, sizeof(int) * 2 * (size_t)n, s);
  if (e != cudaSuccess) rc = cuda_fail(e, "ellpack_transpose", __FILE__, __LINE__);
  const int grid = grid_warps_rows(n);
  if (rc == SP2_OK) {
    if (A->dtype == SP2_F64) col_count_kernel<double><<<grid, kOpsThreads, 0, s>>>(view<double>(A), n, cnt);
    else col_count_kernel<float><<<grid, kOpsThreads, 0, s>>>(view<float>(A), n, cnt);
    note_launch();
  }
  // the longest column decides whether At fits
  int hmax = 0;
  if (rc == SP2_OK) {
    int *dmax = nullptr;
    rc = dev_alloc((void **)&dmax, sizeof(int), s);
    if (rc == SP2_OK) {
      e = cudaMemsetAsync(dmax, 0, sizeof(int), s);
      if (e == cudaSuccess) {
        int_max_kernel<<<grid, kOpsThreads, 0, s>>>(cnt, n, dmax);
        note_launch();
        e = cudaGetLastError();
      }
      rc = e == cudaSuccess ? sync_read(&hmax, dmax, sizeof(int), s, "ellpack_transpose")
                            : cuda_fail(e, "ellpack_transpose", __FILE__, __LINE__);
      dev_free(dmax, s);
    }
  }
  if (required_width) *required_width = hmax;
  if (rc == SP2_OK && hmax > At->width) {
    dev_free(cnt, s);
    return fail(SP2E_OVERFLOW, "ellpack_transpose: a column holds %d entries, At width is %d", hmax, At->width);
  }
  void *scr = nullptr;
  if (rc == SP2_OK && hmax > kSortMax)  // scratch rows for the sort of long rows
    rc = dev_alloc(&scr, (sizeof(int) + dtype_size(At->dtype)) * (size_t)n * At->width, s);
  if (rc == SP2_OK) {
    int *scr_i = static_cast<int *>(scr);
    void *scr_v = scr ? static_cast<void *>(static_cast<int *>(scr) + (size_t)n * At->width) : nullptr;
    if (A->dtype == SP2_F64) {
      col_scatter_kernel<double><<<grid, kOpsThreads, 0, s>>>(view<double>(A), outview<double>(At), cursor);
      row_sort_kernel<double><<<grid, kSortWarps * 32, 0, s>>>(
          outview<double>(At), cnt, scr_i, static_cast<double *>(scr_v));
    } else {
      col_scatter_kernel<float><<<grid, kOpsThreads, 0, s>>>(view<float>(A), outview<float>(At), cursor);
      row_sort_kernel<float><<<grid, kSortWarps * 32, 0, s>>>(
          outview<float>(At), cnt, scr_i, static_cast<float *>(scr_v));
    }
    note_launch();
    note_launch();
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) rc = cuda_fail(e, "ellpack_transpose", __FILE__, __LINE__);
  }
  if (scr) dev_free(scr, s);
  dev_free(cnt, s);
  return rc;
}

extern "C" int ellpack_to_dense(const ellpack_t *A, void *dense, int64_t ld, void *stream) {
  SP2_TRY(check_matrix(A, "ellpack_to_dense"));
  if (!dense) return fail(SP2E_ARG, "ellpack_to_dense: dense is NULL");
  if (ld < A->n) return fail(SP2E_ARG, "ellpack_to_dense: ld = %lld < n = %d", (long long)ld, A->n);
  cudaStream_t s = as_stream(stream);
  SP2_CUDA(cudaMemsetAsync(dense, 0, dtype_size(A->dtype) * (size_t)A->n * (size_t)ld, s));
  if (A->dtype == SP2_F64)
    to_dense_kernel<double><<<grid_warps_rows(A->n), kOpsThreads, 0, s>>>(view<double>(A), static_cast<double *>(dense), ld);
  else
    to_dense_kernel<float><<<grid_warps_rows(A->n), kOpsThreads, 0, s>>>(view<float>(A), static_cast<float *>(dense), ld);
  note_launch();
  SP2_CUDA(cudaGetLastError());
  return SP2_OK;
}

extern "C" int ellpack_from_dense(const void *dense, int64_t ld, double tau, ellpack_t *A, int32_t *required_width,
                                  void *stream) {
  SP2_TRY(check_matrix(A, "ellpack_from_dense"));
  if (!dense) return fail(SP2E_ARG, "ellpack_from_dense: dense is NULL");
  if (ld < A->n) return fail(SP2E_ARG, "ellpack_from_dense: ld = %lld < n = %d", (long long)ld, A->n);
  if (!(tau >= 0.0) || !isfinite(tau)) return fail(SP2E_ARG, "ellpack_from_dense: tau must be finite and >= 0");
  cudaStream_t s = as_stream(stream);
  int *ctl = nullptr;
  SP2_TRY(dev_alloc((void **)&ctl, 2 * sizeof(int), s));
  int h[2] = {0, 0};
  int rc = SP2_OK;
  cudaError_t e = cudaMemsetAsync(ctl, 0, 2 * sizeof(int), s);
  if (e == cudaSuccess) {
    if (A->dtype == SP2_F64)
      from_dense_kernel<double><<<grid_warps_rows(A->n), kOpsThreads, 0, s>>>(static_cast<const double *>(dense), ld,
                                                                              A->n, tau, outview<double>(A), ctl);
    else
      from_dense_kernel<float><<<grid_warps_rows(A->n), kOpsThreads, 0, s>>>(static_cast<const float *>(dense), ld,
                                                                             A->n, (float)tau, outview<float>(A), ctl);
    note_launch();
    e = cudaGetLastError();
  }
  rc = e == cudaSuccess ? sync_read(h, ctl, sizeof(h), s, "ellpack_from_dense")
                        : cuda_fail(e, "ellpack_from_dense", __FILE__, __LINE__);
  dev_free(ctl, s);
  SP2_TRY(rc);
  if (required_width) *required_width = h[0];
  if (h[1] > 0)
    return fail(SP2E_OVERFLOW, "ellpack_from_dense: %d row(s) need %d slots, width is %d", h[1], h[0], A->width);
  return SP2_OK;
}
