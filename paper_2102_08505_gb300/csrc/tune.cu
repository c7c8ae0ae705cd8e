// tune.cu -- autotuner of the SpGEMM first pass.
//
// The first-pass variants (column blocks with 1, 2 or 4 warps per row, the one-warp
// two-k-step variant, the compact forms of both for symmetric products, the row tiles
// with a shared column index, per-warp hash tables of 2^10..2^12 slots) compute the same
// product;
// which is fastest depends on the device, the element type, the matrix size and the row
// lengths.  The tuner times every variant on a real product, keeps the fastest in a
// table keyed by (SM count, dtype, floor(log2 n), floor(log2 mean row length of A)), and
// serves later multiplies of the same class from the table.  The table lives in host
// memory, is shared by all threads (mutex), and can be saved to and loaded from a text
// file so that a deployment tunes once.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "common.cuh"

namespace sp2 {
namespace {

constexpr int kCandidates[] = {1, 2, 4, 7, 3, 8, 9, 10, 11, 12};
constexpr int kNumCandidates = sizeof(kCandidates) / sizeof(kCandidates[0]);
static_assert(kNumCandidates == SP2_TUNE_CANDIDATES, "candidate count");

struct Entry {
  int sms, dtype, lg_n, lg_w, path;
  float ms;
};

std::mutex g_mu;
std::vector<Entry> g_table;

int bucket_n(long long n) {
  int b = 0;
  while ((1LL << (b + 1)) <= n) ++b;
  return b;
}

int bucket_w(double mean) { return mean < 1.0 ? 0 : (int)floor(log2(mean)); }

bool same_key(const Entry &e, int sms, int dtype, int lg_n, int lg_w) {
  return e.sms == sms && e.dtype == dtype && e.lg_n == lg_n && e.lg_w == lg_w;
}

void record(int sms, int dtype, int lg_n, int lg_w, int path, float ms) {
  std::lock_guard<std::mutex> lk(g_mu);
  for (auto &e : g_table)
    if (same_key(e, sms, dtype, lg_n, lg_w)) {
      e.path = path;
      e.ms = ms;
      return;
    }
  g_table.push_back({sms, dtype, lg_n, lg_w, path, ms});
}

bool lookup(int sms, int dtype, int lg_n, int lg_w, int *path) {
  std::lock_guard<std::mutex> lk(g_mu);
  for (const auto &e : g_table)
    if (same_key(e, sms, dtype, lg_n, lg_w)) {
      *path = e.path;
      return true;
    }
  return false;
}

bool valid_candidate(int p) {
  for (int c : kCandidates)
    if (c == p) return true;
  return false;
}

__global__ void nnz_sum_kernel(const int *__restrict__ nnz, int n, int w, unsigned long long *__restrict__ out) {
  unsigned long long s = 0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) s += (unsigned)min(nnz[i], w);
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0 && s) atomicAdd(out, s);
}

}  // namespace

int mean_row_nnz(const ellpack_t *X, double *mean, cudaStream_t s) {
  unsigned long long *d = nullptr;
  SP2_TRY(dev_alloc((void **)&d, sizeof(unsigned long long), s));
  unsigned long long h = 0;
  cudaError_t e = cudaMemsetAsync(d, 0, sizeof(*d), s);
  if (e == cudaSuccess) {
    const int blocks = std::min((X->n + 255) / 256, num_sms() * 4);
    nnz_sum_kernel<<<blocks < 1 ? 1 : blocks, 256, 0, s>>>(X->nnz, X->n, X->width, d);
    note_launch();
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d, sizeof(h), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  dev_free(d, s);
  if (e != cudaSuccess) return cuda_fail(e, "mean_row_nnz", __FILE__, __LINE__);
  *mean = (double)h / (double)X->n;
  return SP2_OK;
}

// Times every candidate on the multiply `a` (its output is rewritten by each; all give
// the product), `reps` timed runs each after one untimed run; records the fastest.
int tune_multiply(MultiplyArgs a, double mean_nnz, double2 *rowstat, SpgemmCtl *ctl, int reps, int *best,
                  float *times, cudaStream_t s) {
  if (reps < 1) reps = 1;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  SP2_CUDA(cudaEventCreate(&e0));
  cudaError_t ce = cudaEventCreate(&e1);
  if (ce != cudaSuccess) {
    cudaEventDestroy(e0);
    return cuda_fail(ce, "tune: event", __FILE__, __LINE__);
  }
  struct Ev {
    cudaEvent_t a, b;
    ~Ev() { cudaEventDestroy(a); cudaEventDestroy(b); }
  } ev{e0, e1};
  int bp = 0;
  float bms = 0.f;
  for (int c = 0; c < kNumCandidates; ++c) {
    a.path = kCandidates[c];
    SP2_TRY(multiply_async(a, rowstat, ctl, s));
    SP2_CUDA(cudaEventRecord(e0, s));
    for (int r = 0; r < reps; ++r) SP2_TRY(multiply_async(a, rowstat, ctl, s));
    SP2_CUDA(cudaEventRecord(e1, s));
    SP2_CUDA(cudaEventSynchronize(e1));
    float ms = 0.f;
    SP2_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    ms /= (float)reps;
    if (times) times[c] = ms;
    if (bp == 0 || ms < bms) {
      bp = kCandidates[c];
      bms = ms;
    }
  }
  record(num_sms(), a.A->dtype, bucket_n(a.A->n), bucket_w(mean_nnz), bp, bms);
  *best = bp;
  return SP2_OK;
}

bool tune_find(int dtype, int n, double mean_nnz, int *path) {
  return lookup(num_sms(), dtype, bucket_n(n), bucket_w(mean_nnz), path);
}

}  // namespace sp2

using namespace sp2;

extern "C" int sp2_tune_spgemm(const ellpack_t *A, const ellpack_t *B, const ellpack_t *C, ellpack_t *Out,
                               double alpha, double beta, double tau, int32_t reps, int32_t *best_path,
                               float *times_ms, void *stream) {
  SP2_TRY(check_matrix(A, "sp2_tune_spgemm: A"));
  SP2_TRY(check_matrix(B, "sp2_tune_spgemm: B"));
  SP2_TRY(check_matrix(Out, "sp2_tune_spgemm: Out"));
  if (C) SP2_TRY(check_matrix(C, "sp2_tune_spgemm: C"));
  if (!best_path) return fail(SP2E_ARG, "sp2_tune_spgemm: best_path is NULL");
  if (A->n != B->n || Out->n != A->n || (C && C->n != A->n)) return fail(SP2E_ARG, "sp2_tune_spgemm: sizes differ");
  if (A->dtype != B->dtype || Out->dtype != A->dtype || (C && C->dtype != A->dtype))
    return fail(SP2E_ARG, "sp2_tune_spgemm: dtypes differ");
  if (Out->idx == A->idx || Out->idx == B->idx || (C && Out->idx == C->idx))
    return fail(SP2E_ARG, "sp2_tune_spgemm: Out aliases an operand");
  if (!(tau >= 0.0) || !isfinite(tau) || !isfinite(alpha) || !isfinite(beta))
    return fail(SP2E_ARG, "sp2_tune_spgemm: bad alpha, beta or tau");
  if (reps < 1 || reps > 1000) return fail(SP2E_ARG, "sp2_tune_spgemm: reps must be in [1, 1000]");
  cudaStream_t s = as_stream(stream);
  double mean = 0.0;
  SP2_TRY(mean_row_nnz(A, &mean, s));
  double2 *rowstat = nullptr;
  SpgemmCtl *ctl = nullptr;
  SP2_TRY(dev_alloc((void **)&rowstat, sizeof(double2) * (size_t)A->n, s));
  int rc = dev_alloc((void **)&ctl, sizeof(SpgemmCtl), s);
  if (rc == SP2_OK) {
    MultiplyArgs a{A, B, (C && beta != 0.0) ? C : nullptr, Out, alpha, beta, tau, 0};
    int best = 0;
    rc = tune_multiply(a, mean, rowstat, ctl, reps, &best, times_ms, s);
    if (rc == SP2_OK) *best_path = best;
  }
  if (ctl) dev_free(ctl, s);
  dev_free(rowstat, s);
  return rc;
}

extern "C" int sp2_tune_record(int32_t sms, int32_t dtype, int32_t n, double mean_row_nnz, int32_t path, float ms) {
  if (sms < 1) return fail(SP2E_ARG, "sp2_tune_record: sms must be >= 1");
  if (dtype != SP2_F64 && dtype != SP2_F32) return fail(SP2E_ARG, "sp2_tune_record: unknown dtype %d", dtype);
  if (n < 1 || !(mean_row_nnz >= 0.0) || !isfinite(mean_row_nnz)) return fail(SP2E_ARG, "sp2_tune_record: bad n or mean");
  if (!valid_candidate(path)) return fail(SP2E_ARG, "sp2_tune_record: path %d is not a tunable variant", path);
  record(sms, dtype, bucket_n(n), bucket_w(mean_row_nnz), path, ms);
  return SP2_OK;
}

extern "C" int sp2_tune_lookup(int32_t sms, int32_t dtype, int32_t n, double mean_row_nnz, int32_t *path) {
  if (!path) return fail(SP2E_ARG, "sp2_tune_lookup: path is NULL");
  if (n < 1 || !(mean_row_nnz >= 0.0)) return fail(SP2E_ARG, "sp2_tune_lookup: bad n or mean");
  if (sms == 0) sms = num_sms();
  int p = -1;
  *path = lookup(sms, dtype, bucket_n(n), bucket_w(mean_row_nnz), &p) ? p : -1;
  return SP2_OK;
}

extern "C" int sp2_tune_clear(void) {
  std::lock_guard<std::mutex> lk(g_mu);
  g_table.clear();
  return SP2_OK;
}

extern "C" int sp2_tune_size(int32_t *entries) {
  if (!entries) return fail(SP2E_ARG, "sp2_tune_size: entries is NULL");
  std::lock_guard<std::mutex> lk(g_mu);
  *entries = (int32_t)g_table.size();
  return SP2_OK;
}

extern "C" int sp2_tune_save(const char *path) {
  if (!path) return fail(SP2E_ARG, "sp2_tune_save: path is NULL");
  std::vector<Entry> t;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    t = g_table;
  }
  std::sort(t.begin(), t.end(), [](const Entry &x, const Entry &y) {
    if (x.sms != y.sms) return x.sms < y.sms;
    if (x.dtype != y.dtype) return x.dtype < y.dtype;
    if (x.lg_n != y.lg_n) return x.lg_n < y.lg_n;
    return x.lg_w < y.lg_w;
  });
  FILE *f = fopen(path, "w");
  if (!f) return fail(SP2E_ARG, "sp2_tune_save: cannot open %s", path);
  bool ok = fprintf(f, "# sp2ell spgemm tuning v1: sms dtype log2_n log2_mean_row path ms\n") > 0;
  for (const auto &e : t)
    ok = ok && fprintf(f, "%d %d %d %d %d %.6g\n", e.sms, e.dtype, e.lg_n, e.lg_w, e.path, (double)e.ms) > 0;
  ok = (fclose(f) == 0) && ok;
  if (!ok) return fail(SP2E_ARG, "sp2_tune_save: write to %s failed", path);
  return SP2_OK;
}

extern "C" int sp2_tune_load(const char *path) {
  if (!path) return fail(SP2E_ARG, "sp2_tune_load: path is NULL");
  FILE *f = fopen(path, "r");
  if (!f) return fail(SP2E_ARG, "sp2_tune_load: cannot open %s", path);
  char line[256];
  std::vector<Entry> in;
  bool header = false, bad = false;
  int lineno = 0;
  while (fgets(line, sizeof(line), f)) {
    ++lineno;
    if (line[0] == '#') {
      if (lineno == 1 && strstr(line, "sp2ell spgemm tuning v1")) header = true;
      continue;
    }
    Entry e;
    double ms = 0.0;
    if (sscanf(line, "%d %d %d %d %d %lf", &e.sms, &e.dtype, &e.lg_n, &e.lg_w, &e.path, &ms) != 6 || e.sms < 1 ||
        (e.dtype != SP2_F64 && e.dtype != SP2_F32) || e.lg_n < 0 || e.lg_n > 31 || e.lg_w < 0 || e.lg_w > 31 ||
        !valid_candidate(e.path)) {
      bad = true;
      break;
    }
    e.ms = (float)ms;
    in.push_back(e);
  }
  fclose(f);
  if (!header) return fail(SP2E_ARG, "sp2_tune_load: %s is not a tuning file", path);
  if (bad) return fail(SP2E_ARG, "sp2_tune_load: %s line %d is malformed", path, lineno);
  for (const auto &e : in) record(e.sms, e.dtype, e.lg_n, e.lg_w, e.path, e.ms);
  return SP2_OK;
}
