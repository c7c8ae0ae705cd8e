// profile.cu -- launch counting and CUDA-event timing of kernel classes, and the FMA-rate
// micro-benchmark that gives the measured arithmetic peak of this GPU.
#include <atomic>
#include <mutex>
#include <vector>

#include "common.cuh"

namespace sp2 {
namespace {
std::atomic<bool> g_on{false};
std::atomic<long long> g_launches{0};
std::mutex g_mu;
struct Pair {
  int cls;
  cudaEvent_t a, b;
};
std::vector<Pair> g_pairs;
thread_local cudaEvent_t t_open[SP2_PROF_CLASSES] = {};
}  // namespace

void note_launch() {
  if (g_on.load(std::memory_order_relaxed)) g_launches.fetch_add(1, std::memory_order_relaxed);
}

// No events while a stream is being captured into a graph (graph bodies of the batched
// loop may not hold event nodes).
static bool capturing(cudaStream_t s) {
  cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &st) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return st != cudaStreamCaptureStatusNone;
}

void prof_begin(int cls, cudaStream_t s) {
  if (!g_on.load(std::memory_order_relaxed) || cls < 0 || cls >= SP2_PROF_CLASSES) return;
  if (capturing(s)) return;
  cudaEvent_t e;
  if (cudaEventCreate(&e) != cudaSuccess) { cudaGetLastError(); return; }
  cudaEventRecord(e, s);
  t_open[cls] = e;
}

void prof_end(int cls, cudaStream_t s) {
  if (!g_on.load(std::memory_order_relaxed) || cls < 0 || cls >= SP2_PROF_CLASSES || !t_open[cls]) return;
  if (capturing(s)) return;
  cudaEvent_t e;
  if (cudaEventCreate(&e) != cudaSuccess) { cudaGetLastError(); return; }
  cudaEventRecord(e, s);
  std::lock_guard<std::mutex> lk(g_mu);
  g_pairs.push_back(Pair{cls, t_open[cls], e});
  t_open[cls] = nullptr;
}

}  // namespace sp2

using namespace sp2;

extern "C" int sp2_profile_start(void) {
  std::lock_guard<std::mutex> lk(g_mu);
  for (auto &p : g_pairs) { cudaEventDestroy(p.a); cudaEventDestroy(p.b); }
  g_pairs.clear();
  g_launches.store(0);
  g_on.store(true);
  return SP2_OK;
}

extern "C" int sp2_profile_stop(sp2_profile *out) {
  g_on.store(false);
  std::lock_guard<std::mutex> lk(g_mu);
  sp2_profile r{};
  r.launches = g_launches.load();
  int rc = SP2_OK;
  for (auto &p : g_pairs) {
    float ms = 0.f;
    cudaError_t e = cudaEventSynchronize(p.b);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, p.a, p.b);
    if (e != cudaSuccess && rc == SP2_OK) rc = cuda_fail(e, "sp2_profile_stop", __FILE__, __LINE__);
    r.count[p.cls] += 1;
    r.total_ms[p.cls] += ms;
    cudaEventDestroy(p.a);
    cudaEventDestroy(p.b);
  }
  g_pairs.clear();
  if (out) *out = r;
  return rc;
}

// ------------------------------------------------------------------ FMA-rate benchmark
// Every thread runs CH independent multiply-add chains of `iters` steps each.  The chains
// are x <- x * m + c with |m| < 1, so values stay finite; the results are stored so that
// the work cannot be removed.  A grid of several CTAs per SM keeps every FMA pipe busy.
namespace sp2 {
namespace {
template <typename T, int CH>
__global__ void __launch_bounds__(256) fma_rate_kernel(T *out, int iters, T m, T c) {
  T x[CH];
#pragma unroll
  for (int u = 0; u < CH; ++u) x[u] = T(threadIdx.x + u) * T(1e-3);
#pragma unroll 1
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int r = 0; r < 8; ++r)
#pragma unroll
      for (int u = 0; u < CH; ++u) x[u] = fma(x[u], m, c);
  }
  T s = T(0);
#pragma unroll
  for (int u = 0; u < CH; ++u) s += x[u];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <typename T, int CH>
int fma_rate(int reps, double *tflops, cudaStream_t s) {
  const int blocks = num_sms() * 8, threads = 256;
  const int iters = sizeof(T) == 8 ? 256 : 4096;
  void *buf = nullptr;
  SP2_TRY(dev_alloc(&buf, sizeof(T) * (size_t)blocks * threads, s));
  cudaEvent_t a = nullptr, b = nullptr;
  int rc = SP2_OK;
  double best = 0.0;
  if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) {
    rc = cuda_fail(cudaGetLastError(), "fma_rate events", __FILE__, __LINE__);
  } else {
    const T m = T(0.999), c = T(1e-3);
    fma_rate_kernel<T, CH><<<blocks, threads, 0, s>>>(static_cast<T *>(buf), iters, m, c);  // warm-up
    note_launch();
    for (int r = 0; r < reps && rc == SP2_OK; ++r) {
      cudaEventRecord(a, s);
      fma_rate_kernel<T, CH><<<blocks, threads, 0, s>>>(static_cast<T *>(buf), iters, m, c);
      note_launch();
      cudaEventRecord(b, s);
      float ms = 0.f;
      cudaError_t e = cudaEventSynchronize(b);
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
      if (e != cudaSuccess) { rc = cuda_fail(e, "fma_rate", __FILE__, __LINE__); break; }
      const double flop = 2.0 * 8.0 * CH * (double)iters * blocks * threads;
      if (ms > 0.f) best = fmax(best, flop / (ms * 1e-3) / 1e12);
    }
  }
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  dev_free(buf, s);
  if (rc == SP2_OK) *tflops = best;
  return rc;
}
}  // namespace
}  // namespace sp2

extern "C" int sp2_fma_peak(int dtype, int reps, double *tflops, void *stream) {
  if (dtype != SP2_F64 && dtype != SP2_F32) return fail(SP2E_ARG, "sp2_fma_peak: unknown dtype %d", dtype);
  if (reps < 1 || reps > 1000) return fail(SP2E_ARG, "sp2_fma_peak: reps = %d must be in 1..1000", reps);
  if (!tflops) return fail(SP2E_ARG, "sp2_fma_peak: tflops is NULL");
  cudaStream_t s = as_stream(stream);
  return dtype == SP2_F64 ? fma_rate<double, 8>(reps, tflops, s) : fma_rate<float, 16>(reps, tflops, s);
}
