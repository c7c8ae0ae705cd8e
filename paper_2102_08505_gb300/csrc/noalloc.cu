// noalloc.cu -- trace and squared Frobenius norm for callers that cannot allocate
// device memory: the scratch lives in a fixed array in the library's device image.
#include <math.h>

#include <mutex>

#include "common.cuh"

namespace sp2 {
namespace {

// Per-row partial results for up to SP2_NOALLOC_MAX_N rows, then one StepResult.  Every
// GPU that loads the library holds this array until the process exits.
constexpr size_t kRowBytes = sizeof(double2) * (size_t)SP2_NOALLOC_MAX_N;
constexpr size_t kScratchBytes = kRowBytes + 256;
static_assert(sizeof(StepResult) <= 256, "result slot too small");
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_mu;
void *g_addr[64] = {nullptr};

// Device address of the scratch array on the current device, looked up once per device
// (in host code the symbol is only a host-side stand-in, not a device address).
int scratch_address(void **out) {
  int dev = 0;
  SP2_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return fail(SP2E_ARG, "ellpack_trace_noalloc: device ordinal %d out of range", dev);
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[dev]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      return fail(SP2E_CUDA, "ellpack_trace_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
    }
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return SP2_OK;
}

}  // namespace
}  // namespace sp2

using namespace sp2;

extern "C" int ellpack_trace_noalloc(const ellpack_t *A, double *trace, double *frobenius2, void *stream) {
  SP2_TRY(check_matrix(A, "ellpack_trace_noalloc: A"));
  if (!trace) return fail(SP2E_ARG, "ellpack_trace_noalloc: trace is NULL");
  if (A->n > SP2_NOALLOC_MAX_N)
    return fail(SP2E_ARG, "ellpack_trace_noalloc: n = %d exceeds the fixed scratch of %d rows", A->n,
                SP2_NOALLOC_MAX_N);
  void *base = nullptr;
  SP2_TRY(scratch_address(&base));
  cudaStream_t s = as_stream(stream);
  double2 *rowstat = static_cast<double2 *>(base);
  StepResult *res = reinterpret_cast<StepResult *>(static_cast<unsigned char *>(base) + kRowBytes);
  // every row's partial is written before the ordered reduction reads it, and the
  // reduction writes the whole result: nothing in the scratch needs clearing
  SP2_TRY(rowstat_async(A, rowstat, s));
  launch_reduce_rows(rowstat, A->nnz, A->n, nullptr, res, s);
  SP2_CUDA(cudaGetLastError());
  StepResult h;
  SP2_CUDA(cudaMemcpyAsync(&h, res, sizeof(h), cudaMemcpyDeviceToHost, s));
  SP2_CUDA(cudaStreamSynchronize(s));
  *trace = h.tr;
  if (frobenius2) *frobenius2 = h.fro;
  // each requested output follows the rule of its allocating counterpart (ellpack_trace,
  // ellpack_frobenius2): a squared norm that overflows fails only if it was asked for
  if (!isfinite(h.tr)) return fail(SP2E_NONFINITE, "ellpack_trace_noalloc: non-finite trace");
  if (frobenius2 && !isfinite(h.fro))
    return fail(SP2E_NONFINITE, "ellpack_trace_noalloc: non-finite squared Frobenius norm");
  return SP2_OK;
}
