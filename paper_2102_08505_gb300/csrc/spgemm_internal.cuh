// spgemm_internal.cuh -- device helpers shared by the SpGEMM first-pass kernels
// (spgemm.cu, tile.cu) and the launcher of the row-tile first pass.
#pragma once

#include "common.cuh"

namespace sp2 {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

__device__ __forceinline__ double fmadd(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float fmadd(float a, float b, float c) { return fmaf(a, b, c); }

// Drop rule |v| > tau evaluated on the bit patterns: for IEEE values with the sign bit
// cleared the integer order is the numeric order, so the test runs on the integer pipe
// (the FP64 pipe of this GPU is narrow).  A NaN compares above tau and is kept, so it
// reaches the traces and is reported instead of vanishing.
__device__ __forceinline__ long long mag_bits(double v) { return __double_as_longlong(v) & 0x7FFFFFFFFFFFFFFFLL; }
__device__ __forceinline__ int mag_bits(float v) { return __float_as_int(v) & 0x7FFFFFFF; }

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

// At tau = 0 every structural entry is kept, exact zeros included: accumulators start at a
// signalling-NaN pattern that no arithmetic produces, and the first update replaces it.
__device__ __forceinline__ bool is_untouched(double v) {
  return __double_as_longlong(v) == (long long)0xFFF4A5A5A5A5A5A5ULL;
}
__device__ __forceinline__ bool is_untouched(float v) { return __float_as_uint(v) == 0xFFA5A5A5u; }
template <typename T> __device__ __forceinline__ T untouched();
template <> __device__ __forceinline__ double untouched<double>() { return __longlong_as_double((long long)0xFFF4A5A5A5A5A5A5ULL); }
template <> __device__ __forceinline__ float untouched<float>() { return __uint_as_float(0xFFA5A5A5u); }

// Row-tile first pass (tile.cu) over all rows of a.A; rows it cannot hold are appended to
// fb[*fb_count] for the deferred-row bins.
template <typename T>
int launch_tile(const MultiplyArgs &a, double2 *rowstat, SpgemmCtl *ctl, int *fb, int *fb_count, cudaStream_t s);

}  // namespace sp2
