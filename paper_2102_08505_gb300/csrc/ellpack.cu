// ellpack.cu -- matrix lifetime, transfers, reductions (trace, norm, Gershgorin),
// the SP2 initial guess X0 and element-type conversion.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <mutex>
#include <vector>

#include "common.cuh"

namespace sp2 {

// ------------------------------------------------------------------ errors
static thread_local char g_err[512] = "";

void set_error(const char *fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

int fail(int code, const char *fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return code;
}

int cuda_fail(cudaError_t e, const char *what, const char *file, int line) {
  const char *base = strrchr(file, '/');
  set_error("CUDA error %s (%s) in %s at %s:%d", cudaGetErrorName(e), cudaGetErrorString(e), what,
            base ? base + 1 : file, line);
  return e == cudaErrorMemoryAllocation ? SP2E_NOMEM : SP2E_CUDA;
}

int current_device() {
  int dev = 0;
  cudaGetDevice(&dev);
  return (dev < 0 || dev >= 64) ? 0 : dev;
}

int num_sms() {
  static DeviceOnce once;
  int dev = 0;
  cudaGetDevice(&dev);
  const int slot = (dev < 0 || dev >= 64) ? 0 : dev;
  device_once(once, slot, [&](int &v) {
    v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    if (v < 1) v = 1;
    return 0;
  });
  return once.value[slot];
}

int check_matrix(const ellpack_t *m, const char *name) {
  if (!m) return fail(SP2E_ARG, "%s is NULL", name);
  if (m->n < 1) return fail(SP2E_ARG, "%s: n = %d must be >= 1", name, m->n);
  if (m->width < 1) return fail(SP2E_ARG, "%s: width = %d must be >= 1", name, m->width);
  if (m->dtype != SP2_F64 && m->dtype != SP2_F32) return fail(SP2E_ARG, "%s: unknown dtype %d", name, m->dtype);
  if (!m->idx || !m->val || !m->nnz) return fail(SP2E_ARG, "%s: null array pointer", name);
  if ((long long)m->n * (long long)m->width > (1LL << 40)) return fail(SP2E_ARG, "%s: n*width too large", name);
  return SP2_OK;
}

// ------------------------------------------------------------------ device memory
// The library's stream-ordered allocations come from its own pool per device, which keeps
// freed memory for reuse (release threshold: unlimited) instead of handing it back to the
// driver at every synchronisation; sp2_release_memory() returns it.
namespace {
std::mutex g_pool_mu;
cudaMemPool_t g_pool[64] = {};

int library_pool(cudaMemPool_t *pool) {
  int dev = 0;
  SP2_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return fail(SP2E_ARG, "device ordinal %d out of range", dev);
  std::lock_guard<std::mutex> lk(g_pool_mu);
  if (!g_pool[dev]) {
    cudaMemPoolProps props;
    memset(&props, 0, sizeof(props));
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t p = nullptr;
    SP2_CUDA(cudaMemPoolCreate(&p, &props));
    uint64_t keep = UINT64_MAX;
    SP2_CUDA(cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &keep));
    g_pool[dev] = p;
  }
  *pool = g_pool[dev];
  return SP2_OK;
}
}  // namespace

int dev_alloc(void **p, size_t bytes, cudaStream_t s) {
  *p = nullptr;
  if (bytes == 0) bytes = 16;
  cudaMemPool_t pool = nullptr;
  SP2_TRY(library_pool(&pool));
  cudaError_t e = cudaMallocFromPoolAsync(p, bytes, pool, s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return fail(e == cudaErrorMemoryAllocation ? SP2E_NOMEM : SP2E_CUDA, "device allocation of %zu bytes failed: %s",
                bytes, cudaGetErrorString(e));
  }
  return SP2_OK;
}

void dev_free(void *p, cudaStream_t s) {
  if (p) cudaFreeAsync(p, s);
}

namespace {
struct FallbackScratch {
  void *acc = nullptr;
  int *mark = nullptr;
  size_t acc_bytes = 0, mark_elems = 0;
};
std::mutex g_scratch_mu;
FallbackScratch g_scratch[64];
}  // namespace

int fallback_scratch(int n, int dtype, int slots, void **acc, int **mark, cudaStream_t s) {
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) return fail(SP2E_ARG, "device ordinal %d out of range", dev);
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  FallbackScratch &f = g_scratch[dev];
  size_t need_acc = (size_t)slots * (size_t)n * dtype_size(dtype);
  size_t need_mark = (size_t)slots * (size_t)n;
  if (f.acc_bytes < need_acc || f.mark_elems < need_mark) {
    // the scratch outlives streams: allocate it synchronously, once per growth
    SP2_CUDA(cudaStreamSynchronize(s));
    if (f.acc) cudaFree(f.acc);
    if (f.mark) cudaFree(f.mark);
    f.acc = nullptr;
    f.mark = nullptr;
    f.acc_bytes = f.mark_elems = 0;
    SP2_CUDA(cudaMalloc(&f.acc, need_acc));
    SP2_CUDA(cudaMalloc((void **)&f.mark, need_mark * sizeof(int)));
    SP2_CUDA(cudaMemset(f.acc, 0, need_acc));
    SP2_CUDA(cudaMemset(f.mark, 0xFF, need_mark * sizeof(int)));
    SP2_CUDA(cudaDeviceSynchronize());
    f.acc_bytes = need_acc;
    f.mark_elems = need_mark;
  }
  *acc = f.acc;
  *mark = f.mark;
  return SP2_OK;
}

// ------------------------------------------------------------------ reductions
// One CTA reduces n rows in a fixed order: thread t sums rows t, t+T, ...; then a tree.
constexpr int kReduceThreads = 1024;

__global__ void __launch_bounds__(kReduceThreads) reduce_rows_kernel(const double2 *__restrict__ rowstat,
                                                                     const int *__restrict__ nnz, int n,
                                                                     const SpgemmCtl *__restrict__ ctl,
                                                                     StepResult *__restrict__ res) {
  __shared__ double s_tr[kReduceThreads], s_fro[kReduceThreads];
  __shared__ long long s_nnz[kReduceThreads];
  __shared__ int s_max[kReduceThreads];
  double tr = 0.0, fro = 0.0;
  long long tot = 0;
  int mx = 0;
  for (int r = threadIdx.x; r < n; r += kReduceThreads) {
    double2 v = rowstat[r];
    tr += v.x;
    fro += v.y;
    int k = nnz[r];
    tot += k;
    mx = max(mx, k);
  }
  s_tr[threadIdx.x] = tr;
  s_fro[threadIdx.x] = fro;
  s_nnz[threadIdx.x] = tot;
  s_max[threadIdx.x] = mx;
  __syncthreads();
  for (int h = kReduceThreads / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) {
      s_tr[threadIdx.x] += s_tr[threadIdx.x + h];
      s_fro[threadIdx.x] += s_fro[threadIdx.x + h];
      s_nnz[threadIdx.x] += s_nnz[threadIdx.x + h];
      s_max[threadIdx.x] = max(s_max[threadIdx.x], s_max[threadIdx.x + h]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    StepResult o;
    o.tr = s_tr[0];
    o.fro = s_fro[0];
    o.nnz_total = s_nnz[0];
    o.max_nnz = s_max[0];
    o.overflow_rows = ctl ? ctl->overflow_rows : 0;
    o.max_count = ctl ? ctl->max_count : s_max[0];
    o.n_fallback = ctl ? ctl->n_fallback : 0;
    o.n_fallback2 = ctl ? ctl->n_fallback2 : 0;
    o.n_heavy = ctl ? ctl->n_heavy : 0;
    o.n_routed = ctl ? ctl->n_routed : 0;
    o.n_level1 = ctl ? ctl->n_level1 : 0;
    o.n_level2 = ctl ? ctl->n_level2 : 0;
    o.nonfinite = (isfinite(o.tr) && isfinite(o.fro)) ? 0 : 1;
    *res = o;
  }
}

void launch_reduce_rows(const double2 *rowstat, const int *nnz, int n, const SpgemmCtl *ctl, StepResult *res,
                        cudaStream_t s) {
  prof_begin(SP2_PROF_REDUCE, s);
  reduce_rows_kernel<<<1, kReduceThreads, 0, s>>>(rowstat, nnz, n, ctl, res);
  note_launch();
  prof_end(SP2_PROF_REDUCE, s);
}

// rowstat of a stored matrix: warp per row.
template <typename T>
__global__ void rowstat_kernel(EllView<T> A, int row0, double2 *__restrict__ rowstat) {
  const int lane = threadIdx.x & 31;
  const int warps = (gridDim.x * blockDim.x) >> 5;
  for (int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < A.n; r += warps) {
    const int k = min(A.nnz[r], A.w);
    double d = 0.0, f = 0.0;
    for (int s = lane; s < k; s += 32) {
      const int j = A.idx[(size_t)r * A.w + s];
      const double v = (double)A.val[(size_t)r * A.w + s];
      if (j == r + row0) d += v;
      f += v * v;
    }
    for (int o = 16; o > 0; o >>= 1) {
      d += __shfl_xor_sync(0xffffffffu, d, o);
      f += __shfl_xor_sync(0xffffffffu, f, o);
    }
    if (lane == 0) rowstat[r] = make_double2(d, f);
  }
}

static int grid_for_rows(int n, int warps_per_block) {
  long long blocks = ((long long)n + warps_per_block - 1) / warps_per_block;
  long long cap = (long long)num_sms() * 16;
  return (int)(blocks < cap ? (blocks < 1 ? 1 : blocks) : cap);
}

int rowstat_async(const ellpack_t *A, double2 *rowstat, cudaStream_t s, int row0) {
  int grid = grid_for_rows(A->n, 8);
  if (A->dtype == SP2_F64)
    { rowstat_kernel<double><<<grid, 256, 0, s>>>(view<double>(A), row0, rowstat); note_launch(); }
  else
    { rowstat_kernel<float><<<grid, 256, 0, s>>>(view<float>(A), row0, rowstat); note_launch(); }
  SP2_CUDA(cudaGetLastError());
  return SP2_OK;
}

// Gershgorin: per-block min/max partials, then one CTA reduces them in order.
template <typename T>
__global__ void gershgorin_rows_kernel(EllView<T> H, int row0, double2 *__restrict__ part) {
  __shared__ double s_lo[8], s_hi[8];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  double lo = INFINITY, hi = -INFINITY;
  const int warps = (gridDim.x * blockDim.x) >> 5;
  for (int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < H.n; r += warps) {
    const int k = min(H.nnz[r], H.w);
    double d = 0.0, rad = 0.0;
    for (int s = lane; s < k; s += 32) {
      const int j = H.idx[(size_t)r * H.w + s];
      const double v = (double)H.val[(size_t)r * H.w + s];
      if (j == r + row0) d += v; else rad += fabs(v);
    }
    for (int o = 16; o > 0; o >>= 1) {
      d += __shfl_xor_sync(0xffffffffu, d, o);
      rad += __shfl_xor_sync(0xffffffffu, rad, o);
    }
    const double l = d - rad, h = d + rad;
    lo = (isnan(l) || isnan(lo)) ? NAN : fmin(lo, l);  // fmin/fmax would drop a NaN
    hi = (isnan(h) || isnan(hi)) ? NAN : fmax(hi, h);
  }
  if (lane == 0) { s_lo[wid] = lo; s_hi[wid] = hi; }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
      lo = (isnan(lo) || isnan(s_lo[w])) ? NAN : fmin(lo, s_lo[w]);
      hi = (isnan(hi) || isnan(s_hi[w])) ? NAN : fmax(hi, s_hi[w]);
    }
    part[blockIdx.x] = make_double2(lo, hi);
  }
}

__global__ void minmax_reduce_kernel(const double2 *__restrict__ part, int m, double *__restrict__ out) {
  __shared__ double s_lo[256], s_hi[256];
  double lo = INFINITY, hi = -INFINITY;
  bool bad = false;
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    double2 v = part[i];
    if (isnan(v.x) || isnan(v.y)) bad = true;
    lo = fmin(lo, v.x);
    hi = fmax(hi, v.y);
  }
  s_lo[threadIdx.x] = bad ? NAN : lo;
  s_hi[threadIdx.x] = hi;
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) {
      double a = s_lo[threadIdx.x], b = s_lo[threadIdx.x + h];
      s_lo[threadIdx.x] = (isnan(a) || isnan(b)) ? NAN : fmin(a, b);
      s_hi[threadIdx.x] = fmax(s_hi[threadIdx.x], s_hi[threadIdx.x + h]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) { out[0] = s_lo[0]; out[1] = isnan(s_lo[0]) ? NAN : s_hi[0]; }
}

int gershgorin_async(const ellpack_t *H, double *dev_bounds, cudaStream_t s, int row0) {
  int grid = grid_for_rows(H->n, 8);
  double2 *part = nullptr;
  SP2_TRY(dev_alloc((void **)&part, sizeof(double2) * grid, s));
  if (H->dtype == SP2_F64)
    { gershgorin_rows_kernel<double><<<grid, 256, 0, s>>>(view<double>(H), row0, part); note_launch(); }
  else
    { gershgorin_rows_kernel<float><<<grid, 256, 0, s>>>(view<float>(H), row0, part); note_launch(); }
  { minmax_reduce_kernel<<<1, 256, 0, s>>>(part, grid, dev_bounds); note_launch(); }
  cudaError_t e = cudaGetLastError();
  dev_free(part, s);
  if (e != cudaSuccess) return cuda_fail(e, "gershgorin kernels", __FILE__, __LINE__);
  return SP2_OK;
}

// X0 = drop_tau((emax I - H) / (emax - emin)), warp per row.  Output order: the kept
// entries with column < i (in H's order), the diagonal, then the kept entries with
// column > i -- sorted whenever H's row is sorted.  The diagonal is always stored
// unless it falls below tau.
__global__ void x0_kernel(EllView<double> H, const double *__restrict__ bounds, double tau, int row0,
                          EllOut<double> X) {
  const int lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  const double emin = bounds[0], emax = bounds[1];
  const double inv = 1.0 / (emax - emin);
  const int warps = (gridDim.x * blockDim.x) >> 5;
  for (int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < H.n; r += warps) {
    const int k = min(H.nnz[r], H.w);
    const int dc = r + row0;  // column of the diagonal entry of local row r
    // pass 1: counts of kept entries below / above the diagonal, diagonal presence
    int n_lo = 0, has_diag = 0;
    double dval = emax * inv;  // value if H has no diagonal entry
    for (int b = 0; b < k; b += 32) {
      const int s = b + lane;
      int j = -1;
      double x = 0.0;
      if (s < k) {
        j = H.idx[(size_t)r * H.w + s];
        const double h = H.val[(size_t)r * H.w + s];
        x = (j == dc) ? (emax - h) * inv : -h * inv;
        if (j == dc) dval = x;
      }
      const bool keep = (s < k) && j != dc && (tau == 0.0 || fabs(x) > tau);
      n_lo += __popc(__ballot_sync(0xffffffffu, keep && j < dc));
      has_diag |= __any_sync(0xffffffffu, j == dc);
    }
    // the diagonal value lives in one lane; broadcast it
    {
      unsigned m = 0;
      for (int b = 0; b < k; b += 32) {
        const int s = b + lane;
        const bool isd = s < k && H.idx[(size_t)r * H.w + s] == dc;
        m = __ballot_sync(0xffffffffu, isd);
        if (m) { dval = __shfl_sync(0xffffffffu, dval, __ffs(m) - 1); break; }
      }
    }
    const bool keep_diag = (tau == 0.0 || fabs(dval) > tau);
    // pass 2: write
    int lo_pos = 0, hi_pos = n_lo + (keep_diag ? 1 : 0);
    for (int b = 0; b < k; b += 32) {
      const int s = b + lane;
      int j = -1;
      double x = 0.0;
      if (s < k) {
        j = H.idx[(size_t)r * H.w + s];
        const double h = H.val[(size_t)r * H.w + s];
        x = -h * inv;
      }
      const bool keep = (s < k) && j != dc && (tau == 0.0 || fabs(x) > tau);
      const unsigned mlo = __ballot_sync(0xffffffffu, keep && j < dc);
      const unsigned mhi = __ballot_sync(0xffffffffu, keep && j > dc);
      if (keep) {
        const int pos = (j < dc) ? lo_pos + __popc(mlo & lt) : hi_pos + __popc(mhi & lt);
        X.idx[(size_t)r * X.w + pos] = j;
        X.val[(size_t)r * X.w + pos] = x;
      }
      lo_pos += __popc(mlo);
      hi_pos += __popc(mhi);
    }
    if (lane == 0) {
      if (keep_diag) {
        X.idx[(size_t)r * X.w + n_lo] = dc;
        X.val[(size_t)r * X.w + n_lo] = dval;
      }
      X.nnz[r] = hi_pos;
    }
    (void)has_diag;
  }
}

int x0_async(const ellpack_t *H, const double *dev_bounds, double tau, ellpack_t *X, cudaStream_t s, int row0) {
  if (H->dtype != SP2_F64 || X->dtype != SP2_F64) return fail(SP2E_ARG, "x0: F64 matrices expected");
  if (X->width < H->width + 1) return fail(SP2E_ARG, "x0: output width too small");
  int grid = grid_for_rows(H->n, 8);
  { x0_kernel<<<grid, 256, 0, s>>>(view<double>(H), dev_bounds, tau, row0, outview<double>(X)); note_launch(); }
  SP2_CUDA(cudaGetLastError());
  return SP2_OK;
}

// ------------------------------------------------------------------ conversion / copy
template <typename S, typename D>
__global__ void convert_kernel(EllView<S> a, EllOut<D> b, int *__restrict__ overflow) {
  const int lane = threadIdx.x & 31;
  const int warps = (gridDim.x * blockDim.x) >> 5;
  for (int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < a.n; r += warps) {
    const int k0 = min(a.nnz[r], a.w);
    if (k0 > b.w) {  // row does not fit: counted, left unwritten
      if (lane == 0 && overflow) atomicAdd(overflow, 1);
      continue;
    }
    const int k = k0;
    for (int s = lane; s < k; s += 32) {
      b.idx[(size_t)r * b.w + s] = a.idx[(size_t)r * a.w + s];
      b.val[(size_t)r * b.w + s] = (D)a.val[(size_t)r * a.w + s];
    }
    if (lane == 0) b.nnz[r] = k;
  }
}

int convert_async(const ellpack_t *src, ellpack_t *dst, cudaStream_t s, int *overflow) {
  int grid = grid_for_rows(src->n, 8);
  if (src->dtype == SP2_F64 && dst->dtype == SP2_F32)
    { convert_kernel<double, float><<<grid, 256, 0, s>>>(view<double>(src), outview<float>(dst), overflow); note_launch(); }
  else if (src->dtype == SP2_F32 && dst->dtype == SP2_F64)
    { convert_kernel<float, double><<<grid, 256, 0, s>>>(view<float>(src), outview<double>(dst), overflow); note_launch(); }
  else if (src->dtype == SP2_F64)
    { convert_kernel<double, double><<<grid, 256, 0, s>>>(view<double>(src), outview<double>(dst), overflow); note_launch(); }
  else
    { convert_kernel<float, float><<<grid, 256, 0, s>>>(view<float>(src), outview<float>(dst), overflow); note_launch(); }
  SP2_CUDA(cudaGetLastError());
  return SP2_OK;
}

int copy_async(const ellpack_t *src, ellpack_t *dst, cudaStream_t s) { return convert_async(src, dst, s, nullptr); }

}  // namespace sp2

// ==================================================================== C ABI
using namespace sp2;

extern "C" int sp2_version(void) { return 10000; }

extern "C" const char *sp2_last_error_string(void) { return sp2::g_err; }

extern "C" int ellpack_create(int32_t n, int32_t width, int32_t dtype, void *stream, ellpack_t *out) {
  if (!out) return fail(SP2E_ARG, "ellpack_create: out is NULL");
  memset(out, 0, sizeof(*out));
  if (n < 1 || width < 1) return fail(SP2E_ARG, "ellpack_create: n=%d width=%d must be >= 1", n, width);
  if (dtype != SP2_F64 && dtype != SP2_F32) return fail(SP2E_ARG, "ellpack_create: unknown dtype %d", dtype);
  int w = round_up(width, 32);
  if ((long long)n * w > (1LL << 40)) return fail(SP2E_ARG, "ellpack_create: n*width too large");
  cudaStream_t s = as_stream(stream);
  void *idx = nullptr, *val = nullptr, *nnz = nullptr;
  size_t cells = (size_t)n * (size_t)w;
  int rc = dev_alloc(&idx, cells * sizeof(int32_t), s);
  if (rc == SP2_OK) rc = dev_alloc(&val, cells * dtype_size(dtype), s);
  if (rc == SP2_OK) rc = dev_alloc(&nnz, (size_t)n * sizeof(int32_t), s);
  if (rc != SP2_OK) {
    dev_free(idx, s); dev_free(val, s); dev_free(nnz, s);
    return rc;
  }
  cudaError_t e = cudaMemsetAsync(nnz, 0, (size_t)n * sizeof(int32_t), s);
  if (e != cudaSuccess) {
    dev_free(idx, s); dev_free(val, s); dev_free(nnz, s);
    return cuda_fail(e, "cudaMemsetAsync", __FILE__, __LINE__);
  }
  out->n = n;
  out->width = w;
  out->dtype = dtype;
  out->owner = 1;
  out->idx = (int32_t *)idx;
  out->val = val;
  out->nnz = (int32_t *)nnz;
  return SP2_OK;
}

extern "C" int ellpack_wrap(int32_t n, int32_t width, int32_t dtype, int32_t *idx, void *val, int32_t *nnz,
                            ellpack_t *out) {
  if (!out) return fail(SP2E_ARG, "ellpack_wrap: out is NULL");
  memset(out, 0, sizeof(*out));
  ellpack_t m;
  m.n = n; m.width = width; m.dtype = dtype; m.owner = 0; m.idx = idx; m.val = val; m.nnz = nnz;
  SP2_TRY(check_matrix(&m, "ellpack_wrap"));
  *out = m;
  return SP2_OK;
}

extern "C" int ellpack_destroy(ellpack_t *m, void *stream) {
  if (!m) return fail(SP2E_ARG, "ellpack_destroy: NULL");
  if (m->owner) {
    cudaStream_t s = as_stream(stream);
    dev_free(m->idx, s);
    dev_free(m->val, s);
    dev_free(m->nnz, s);
  }
  memset(m, 0, sizeof(*m));
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "ellpack_destroy", __FILE__, __LINE__);
  return SP2_OK;
}

extern "C" int ellpack_upload(ellpack_t *m, const int32_t *h_idx, const void *h_val, const int32_t *h_nnz,
                              void *stream) {
  SP2_TRY(check_matrix(m, "ellpack_upload"));
  if (!h_idx || !h_val || !h_nnz) return fail(SP2E_ARG, "ellpack_upload: null host pointer");
  cudaStream_t s = as_stream(stream);
  size_t cells = (size_t)m->n * (size_t)m->width;
  SP2_CUDA(cudaMemcpyAsync(m->idx, h_idx, cells * sizeof(int32_t), cudaMemcpyHostToDevice, s));
  SP2_CUDA(cudaMemcpyAsync(m->val, h_val, cells * dtype_size(m->dtype), cudaMemcpyHostToDevice, s));
  SP2_CUDA(cudaMemcpyAsync(m->nnz, h_nnz, (size_t)m->n * sizeof(int32_t), cudaMemcpyHostToDevice, s));
  return SP2_OK;
}

extern "C" int ellpack_download_async(const ellpack_t *m, int32_t *h_idx, void *h_val, int32_t *h_nnz,
                                      void *stream) {
  SP2_TRY(check_matrix(m, "ellpack_download_async"));
  if (!h_idx || !h_val || !h_nnz) return fail(SP2E_ARG, "ellpack_download_async: null host pointer");
  cudaStream_t s = as_stream(stream);
  size_t cells = (size_t)m->n * (size_t)m->width;
  SP2_CUDA(cudaMemcpyAsync(h_idx, m->idx, cells * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  SP2_CUDA(cudaMemcpyAsync(h_val, m->val, cells * dtype_size(m->dtype), cudaMemcpyDeviceToHost, s));
  SP2_CUDA(cudaMemcpyAsync(h_nnz, m->nnz, (size_t)m->n * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  return SP2_OK;
}

extern "C" int ellpack_download(const ellpack_t *m, int32_t *h_idx, void *h_val, int32_t *h_nnz, void *stream) {
  SP2_TRY(check_matrix(m, "ellpack_download"));
  if (!h_idx || !h_val || !h_nnz) return fail(SP2E_ARG, "ellpack_download: null host pointer");
  cudaStream_t s = as_stream(stream);
  size_t cells = (size_t)m->n * (size_t)m->width;
  SP2_CUDA(cudaMemcpyAsync(h_idx, m->idx, cells * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  SP2_CUDA(cudaMemcpyAsync(h_val, m->val, cells * dtype_size(m->dtype), cudaMemcpyDeviceToHost, s));
  SP2_CUDA(cudaMemcpyAsync(h_nnz, m->nnz, (size_t)m->n * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  SP2_CUDA(cudaStreamSynchronize(s));
  return SP2_OK;
}

// rowstat pass + ordered reduction, result copied to the host.
static int stored_reduction(const ellpack_t *A, StepResult *host_res, cudaStream_t s) {
  double2 *rowstat = nullptr;
  StepResult *dres = nullptr;
  SP2_TRY(dev_alloc((void **)&rowstat, sizeof(double2) * (size_t)A->n, s));
  int rc = dev_alloc((void **)&dres, sizeof(StepResult), s);
  if (rc != SP2_OK) { dev_free(rowstat, s); return rc; }
  rc = rowstat_async(A, rowstat, s);
  if (rc == SP2_OK) {
    launch_reduce_rows(rowstat, A->nnz, A->n, nullptr, dres, s);
    cudaError_t e = cudaMemcpyAsync(host_res, dres, sizeof(StepResult), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) rc = cuda_fail(e, "trace reduction", __FILE__, __LINE__);
  }
  dev_free(rowstat, s);
  dev_free(dres, s);
  return rc;
}

extern "C" int ellpack_trace(const ellpack_t *A, double *out, void *stream) {
  SP2_TRY(check_matrix(A, "ellpack_trace"));
  if (!out) return fail(SP2E_ARG, "ellpack_trace: out is NULL");
  StepResult r;
  SP2_TRY(stored_reduction(A, &r, as_stream(stream)));
  *out = r.tr;
  if (!isfinite(r.tr)) return fail(SP2E_NONFINITE, "ellpack_trace: non-finite trace");
  return SP2_OK;
}

extern "C" int ellpack_frobenius2(const ellpack_t *A, double *out, void *stream) {
  SP2_TRY(check_matrix(A, "ellpack_frobenius2"));
  if (!out) return fail(SP2E_ARG, "ellpack_frobenius2: out is NULL");
  StepResult r;
  SP2_TRY(stored_reduction(A, &r, as_stream(stream)));
  *out = r.fro;
  if (!isfinite(r.fro)) return fail(SP2E_NONFINITE, "ellpack_frobenius2: non-finite norm");
  return SP2_OK;
}

extern "C" int ellpack_gershgorin(const ellpack_t *H, double *emin, double *emax, void *stream) {
  SP2_TRY(check_matrix(H, "ellpack_gershgorin"));
  if (!emin || !emax) return fail(SP2E_ARG, "ellpack_gershgorin: null output");
  cudaStream_t s = as_stream(stream);
  double *db = nullptr;
  SP2_TRY(dev_alloc((void **)&db, 2 * sizeof(double), s));
  int rc = gershgorin_async(H, db, s);
  double hb[2] = {0, 0};
  if (rc == SP2_OK) {
    cudaError_t e = cudaMemcpyAsync(hb, db, sizeof(hb), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) rc = cuda_fail(e, "gershgorin copy", __FILE__, __LINE__);
  }
  dev_free(db, s);
  SP2_TRY(rc);
  *emin = hb[0];
  *emax = hb[1];
  if (!isfinite(hb[0]) || !isfinite(hb[1])) return fail(SP2E_NONFINITE, "ellpack_gershgorin: non-finite bound");
  return SP2_OK;
}

// ------------------------------------------------------------------ halo rows
// The rows a block's entries name outside the block, ascending: a flag per column, then a
// two-level stable compaction (per-CTA counts, one CTA's scan, per-CTA ordered writes).
constexpr int kHaloPer = 4096;  // flags per CTA of the compaction
template <typename T>
__global__ void halo_mark_kernel(EllView<T> X, int row0, int ncols, unsigned char *__restrict__ flag) {
  const int warps = (gridDim.x * blockDim.x) >> 5, lane = threadIdx.x & 31;
  for (int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < X.n; r += warps) {
    const int k = min(X.nnz[r], X.w);
    for (int s = lane; s < k; s += 32) {
      const int j = X.idx[(size_t)r * X.w + s];
      if ((unsigned)j < (unsigned)ncols && (j < row0 || j >= row0 + X.n)) flag[j] = 1;
    }
  }
}

__global__ void __launch_bounds__(256) halo_count_kernel(const unsigned char *__restrict__ flag, int ncols,
                                                         int *__restrict__ part) {
  __shared__ int s[256];
  const int base = blockIdx.x * kHaloPer;
  int c = 0;
  for (int i = threadIdx.x; i < kHaloPer && base + i < ncols; i += 256) c += flag[base + i];
  s[threadIdx.x] = c;
  __syncthreads();
  for (int h = 128; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h) s[threadIdx.x] += s[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = s[0];
}

// Exclusive scan of the m per-CTA counts in place; the total into part[m].
__global__ void __launch_bounds__(1024) halo_scan_kernel(int *__restrict__ part, int m) {
  __shared__ int s[1024];
  int carry = 0;
  for (int c0 = 0; c0 < m; c0 += 1024) {
    const int i = c0 + (int)threadIdx.x;
    const int v = i < m ? part[i] : 0;
    s[threadIdx.x] = v;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {  // Hillis-Steele inclusive scan
      const int y = (int)threadIdx.x >= o ? s[threadIdx.x - o] : 0;
      __syncthreads();
      s[threadIdx.x] += y;
      __syncthreads();
    }
    if (i < m) part[i] = carry + s[threadIdx.x] - v;
    const int tot = s[1023];
    __syncthreads();
    carry += tot;
  }
  if (threadIdx.x == 0) part[m] = carry;
}

__global__ void __launch_bounds__(256) halo_write_kernel(const unsigned char *__restrict__ flag, int ncols,
                                                         const int *__restrict__ part, int *__restrict__ rows) {
  __shared__ int s_warp[8];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int base = blockIdx.x * kHaloPer;
  int pos = part[blockIdx.x];
  for (int c0 = 0; c0 < kHaloPer; c0 += 256) {
    const int i = base + c0 + (int)threadIdx.x;
    const bool on = c0 + (int)threadIdx.x < kHaloPer && i < ncols && flag[i];
    const unsigned m = __ballot_sync(0xffffffffu, on);
    if (lane == 0) s_warp[wid] = __popc(m);
    __syncthreads();
    int before = 0, total = 0;
    for (int w = 0; w < 8; ++w) {
      if (w < wid) before += s_warp[w];
      total += s_warp[w];
    }
    if (on) rows[pos + before + __popc(m & ((1u << lane) - 1u))] = i;
    pos += total;
    __syncthreads();
  }
}

extern "C" int ellpack_halo_rows(const ellpack_t *X, int32_t row0, int32_t ncols, int32_t *rows, int32_t *count,
                                 void *stream) {
  SP2_TRY(check_matrix(X, "ellpack_halo_rows"));
  if (!rows || !count) return fail(SP2E_ARG, "ellpack_halo_rows: null output");
  if (row0 < 0 || ncols < 1 || (long long)row0 + X->n > (long long)ncols)
    return fail(SP2E_ARG, "ellpack_halo_rows: rows %d .. %lld outside 0 .. %d", row0, (long long)row0 + X->n - 1,
                ncols - 1);
  cudaStream_t s = as_stream(stream);
  const int ctas = (ncols + kHaloPer - 1) / kHaloPer;
  unsigned char *flag = nullptr;
  int *part = nullptr;
  SP2_TRY(dev_alloc((void **)&flag, (size_t)ncols, s));
  int rc = dev_alloc((void **)&part, sizeof(int) * ((size_t)ctas + 1), s);
  int h = 0;
  if (rc == SP2_OK) {
    cudaError_t e = cudaMemsetAsync(flag, 0, (size_t)ncols, s);
    if (e == cudaSuccess) {
      const int grid = grid_for_rows(X->n, 8);
      if (X->dtype == SP2_F64) halo_mark_kernel<double><<<grid, 256, 0, s>>>(view<double>(X), row0, ncols, flag);
      else halo_mark_kernel<float><<<grid, 256, 0, s>>>(view<float>(X), row0, ncols, flag);
      halo_count_kernel<<<ctas, 256, 0, s>>>(flag, ncols, part);
      halo_scan_kernel<<<1, 1024, 0, s>>>(part, ctas);
      halo_write_kernel<<<ctas, 256, 0, s>>>(flag, ncols, part, rows);
      note_launch(); note_launch(); note_launch(); note_launch();
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, part + ctas, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) rc = cuda_fail(e, "ellpack_halo_rows", __FILE__, __LINE__);
  }
  dev_free(flag, s);
  dev_free(part, s);
  SP2_TRY(rc);
  *count = h;
  return SP2_OK;
}

extern "C" int ellpack_gershgorin_block(const ellpack_t *H, int32_t row0, double *emin, double *emax, void *stream) {
  SP2_TRY(check_matrix(H, "ellpack_gershgorin_block"));
  if (!emin || !emax) return fail(SP2E_ARG, "ellpack_gershgorin_block: null output");
  if (row0 < 0) return fail(SP2E_ARG, "ellpack_gershgorin_block: row0 = %d must be >= 0", row0);
  cudaStream_t s = as_stream(stream);
  double *db = nullptr;
  SP2_TRY(dev_alloc((void **)&db, 2 * sizeof(double), s));
  int rc = gershgorin_async(H, db, s, row0);
  double hb[2] = {0, 0};
  if (rc == SP2_OK) {
    cudaError_t e = cudaMemcpyAsync(hb, db, sizeof(hb), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) rc = cuda_fail(e, "gershgorin copy", __FILE__, __LINE__);
  }
  dev_free(db, s);
  SP2_TRY(rc);
  *emin = hb[0];
  *emax = hb[1];
  if (!isfinite(hb[0]) || !isfinite(hb[1])) return fail(SP2E_NONFINITE, "ellpack_gershgorin_block: non-finite bound");
  return SP2_OK;
}

extern "C" int ellpack_stats_block(const ellpack_t *X, int32_t row0, double *trace, double *frobenius2,
                                   void *stream) {
  SP2_TRY(check_matrix(X, "ellpack_stats_block"));
  if (!trace || !frobenius2) return fail(SP2E_ARG, "ellpack_stats_block: null output");
  if (row0 < 0) return fail(SP2E_ARG, "ellpack_stats_block: row0 = %d must be >= 0", row0);
  cudaStream_t s = as_stream(stream);
  double2 *rowstat = nullptr;
  StepResult *dres = nullptr;
  SP2_TRY(dev_alloc((void **)&rowstat, sizeof(double2) * (size_t)X->n, s));
  int rc = dev_alloc((void **)&dres, sizeof(StepResult), s);
  StepResult h{};
  if (rc == SP2_OK) rc = rowstat_async(X, rowstat, s, row0);
  if (rc == SP2_OK) {
    launch_reduce_rows(rowstat, X->nnz, X->n, nullptr, dres, s);
    cudaError_t e = cudaMemcpyAsync(&h, dres, sizeof(h), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) rc = cuda_fail(e, "ellpack_stats_block", __FILE__, __LINE__);
  }
  dev_free(rowstat, s);
  dev_free(dres, s);
  SP2_TRY(rc);
  *trace = h.tr;
  *frobenius2 = h.fro;
  if (!isfinite(h.tr) || !isfinite(h.fro)) return fail(SP2E_NONFINITE, "ellpack_stats_block: non-finite result");
  return SP2_OK;
}

extern "C" int ellpack_copy(const ellpack_t *src, ellpack_t *dst, void *stream) {
  SP2_TRY(check_matrix(src, "ellpack_copy: src"));
  SP2_TRY(check_matrix(dst, "ellpack_copy: dst"));
  if (src->n != dst->n) return fail(SP2E_ARG, "ellpack_copy: sizes differ");
  if (src->idx == dst->idx || src->val == dst->val || src->nnz == dst->nnz)
    return fail(SP2E_ARG, "ellpack_copy: src and dst share arrays");
  cudaStream_t s = as_stream(stream);
  int *dov = nullptr;
  SP2_TRY(dev_alloc((void **)&dov, sizeof(int), s));
  int hov = 0;
  cudaError_t e = cudaMemsetAsync(dov, 0, sizeof(int), s);
  int rc = e == cudaSuccess ? convert_async(src, dst, s, dov) : cuda_fail(e, "ellpack_copy", __FILE__, __LINE__);
  if (rc == SP2_OK) {
    e = cudaMemcpyAsync(&hov, dov, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) rc = cuda_fail(e, "ellpack_copy", __FILE__, __LINE__);
  }
  dev_free(dov, s);
  SP2_TRY(rc);
  if (hov > 0) return fail(SP2E_OVERFLOW, "ellpack_copy: %d row(s) longer than dst width %d", hov, dst->width);
  return SP2_OK;
}

extern "C" int sp2_release_memory(void) {
  int dev = 0;
  SP2_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return fail(SP2E_ARG, "device ordinal %d out of range", dev);
  std::lock_guard<std::mutex> lk(g_pool_mu);
  if (g_pool[dev]) {
    SP2_CUDA(cudaDeviceSynchronize());
    SP2_CUDA(cudaMemPoolTrimTo(g_pool[dev], 0));
  }
  return SP2_OK;
}
