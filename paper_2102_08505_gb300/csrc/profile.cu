// profile.cu -- launch counting and CUDA-event timing of kernel classes.
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
