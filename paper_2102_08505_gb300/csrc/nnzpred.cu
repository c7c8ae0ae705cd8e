// nnzpred.cu -- exact structural row counts of a product, row features, and a small
// MLP (16 -> 64 -> 64 -> 1, FP32) that predicts the post-threshold length of each row of
// the next SP2 product, trained on the GPU by the kernels below.
//
// Structural count of row i of A*B (+C): |union over k in cols(A_i) of cols(B_k)|
// (+ cols(C_i)), an upper bound of the kept length.  One warp per row marks the touched
// columns in bitmask blocks of 32 columns reached through a group table (the column-block
// layout of the SpGEMM, without values).
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "common.cuh"

namespace sp2 {
namespace {

constexpr unsigned kFullMask = 0xffffffffu;

// ---------------------------------------------------------------- structural count
// A group-table entry packs (group << 11) | block: groups below 2^21 - 1, so n <= 2^26 - 32.
constexpr int kCntLog2G = 12, kCntG = 1 << kCntLog2G, kCntNB = 2048;  // 2048 blocks of 32 columns
constexpr int kCntBlkBits = 11;
constexpr int kCntMaxN = (1 << 26) - 32;
constexpr int kCntWarps = 8;
constexpr int kCntBytesPerWarp = kCntG * 4 + kCntNB * 4 + 16;

__device__ __forceinline__ int cnt_hash(unsigned g) { return (int)((g * 0x9E3779B1u) >> (32 - kCntLog2G)); }

template <typename T>
__global__ void __launch_bounds__(kCntWarps * 32) struct_count_kernel(EllView<T> A, EllView<T> B, EllView<T> C,
                                                                     int use_c, int *__restrict__ counts,
                                                                     int *__restrict__ max_out) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  unsigned char *base = smem + (size_t)wid * kCntBytesPerWarp;
  unsigned *gtab = reinterpret_cast<unsigned *>(base);
  unsigned *mask = reinterpret_cast<unsigned *>(base + kCntG * 4);
  int *nblk = reinterpret_cast<int *>(base + kCntG * 4 + kCntNB * 4);
  const int ncol = B.n;
  int wmax = 0;
  for (int r = blockIdx.x * kCntWarps + wid; r < A.n; r += gridDim.x * kCntWarps) {
    for (int i = lane; i < kCntG; i += 32) gtab[i] = 0xFFFFFFFFu;
    for (int i = lane; i < kCntNB; i += 32) mask[i] = 0u;
    if (lane == 0) *nblk = 0;
    __syncwarp();
    bool over = false;
    // one source row: set the bits of its columns
    auto mark_row = [&](const int *ri, int nb) {
      for (int q = lane; q < nb; q += 32) {
        const int j = __ldg(ri + q);
        if ((unsigned)j >= (unsigned)ncol) continue;
        const unsigned g = (unsigned)j >> 5;
        int h = cnt_hash(g), b = -1;
        for (int p = 0; p < kCntG; ++p) {
          const unsigned e = ((volatile unsigned *)gtab)[h];
          if (e != 0xFFFFFFFFu && (e >> kCntBlkBits) == g) { b = (int)(e & (kCntNB - 1)); break; }
          if (e == 0xFFFFFFFFu) {
            // take a block number first; the CAS decides which lane's number is kept
            const int nbn = atomicAdd(nblk, 1);
            if (nbn >= kCntNB) break;
            const unsigned old = atomicCAS(gtab + h, 0xFFFFFFFFu, (g << kCntBlkBits) | (unsigned)nbn);
            if (old == 0xFFFFFFFFu) { b = nbn; break; }
            if ((old >> kCntBlkBits) == g) { b = (int)(old & (kCntNB - 1)); break; }
          }
          h = (h + 1) & (kCntG - 1);
        }
        if (b < 0) { over = true; continue; }
        atomicOr(mask + b, 1u << (j & 31));
      }
    };
    const int na = min(A.nnz[r], A.w);
    long long naive = 0;  // sum of the source rows' lengths: a bound without deduplication
    if (use_c) {
      const int nc = min(C.nnz[r], C.w);
      naive += nc;
      mark_row(C.idx + (size_t)r * C.w, nc);
    }
    for (int t = 0; t < na; ++t) {
      const int k = __ldg(A.idx + (size_t)r * A.w + t);
      if ((unsigned)k >= (unsigned)B.n) continue;
      const int nb = min(__ldg(B.nnz + k), B.w);
      naive += nb;
      mark_row(B.idx + (size_t)k * B.w, nb);
    }
    __syncwarp();
    int c = 0;
    const int nb = min(*nblk, kCntNB);
    for (int i = lane; i < nb; i += 32) c += __popc(mask[i]);
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(kFullMask, c, o);
    over = __any_sync(kFullMask, over) || *nblk > kCntNB;
    // rows spanning more than 2048 groups of 32 columns: the undeduplicated sum, capped at
    // the column count (still an upper bound of the structural length)
    if (over) c = (int)(naive < ncol ? naive : ncol);
    if (lane == 0) counts[r] = c;
    wmax = max(wmax, c);
    __syncwarp();
  }
  if (lane == 0 && wmax) atomicMax(max_out, wmax);
}

// ---------------------------------------------------------------- features
template <typename T>
__global__ void rowmax_kernel(EllView<T> X, float *__restrict__ rmax) {
  const int lane = threadIdx.x & 31;
  const int warps = (gridDim.x * blockDim.x) >> 5;
  for (int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < X.n; r += warps) {
    const int k = min(X.nnz[r], X.w);
    float m = 0.f;
    for (int s = lane; s < k; s += 32) m = fmaxf(m, fabsf((float)X.val[(size_t)r * X.w + s]));
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(kFullMask, m, o));
    if (lane == 0) rmax[r] = m;
  }
}

__device__ __forceinline__ float lg10(float x) { return log10f(x + 1e-30f); }

// 16 features per row of X (see nnzpred_features in the header), model-ready transforms.
template <typename T>
__global__ void features_kernel(EllView<T> X, const float *__restrict__ rmax, float ltau, float branch,
                                float tau, float *__restrict__ feat) {
  const int lane = threadIdx.x & 31;
  const int warps = (gridDim.x * blockDim.x) >> 5;
  for (int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < X.n; r += warps) {
    const int k = min(X.nnz[r], X.w);
    float s_nb = 0.f, mx_nb = 0.f, mn_nb = 3.0e38f, mx_v = 0.f, s2 = 0.f, s1 = 0.f, dg = 0.f, bnd = 0.f;
    float c10 = 0.f, c100 = 0.f, wnb = 0.f;
    for (int s = lane; s < k; s += 32) {
      const int j = X.idx[(size_t)r * X.w + s];
      const float v = fabsf((float)X.val[(size_t)r * X.w + s]);
      const bool ok = (unsigned)j < (unsigned)X.n;
      const float nb = ok ? (float)min(X.nnz[j], X.w) : 0.f;
      s_nb += nb;
      mx_nb = fmaxf(mx_nb, nb);
      mn_nb = fminf(mn_nb, nb);
      mx_v = fmaxf(mx_v, v);
      s2 = fmaf(v, v, s2);
      s1 += v;
      if (j == r) dg = v;
      bnd = fmaf(v, ok ? rmax[j] : 0.f, bnd);
      c10 += v > 10.f * tau ? 1.f : 0.f;
      c100 += v > 100.f * tau ? 1.f : 0.f;
      wnb = fmaf(v, nb, wnb);
    }
    for (int o = 16; o > 0; o >>= 1) {
      s_nb += __shfl_xor_sync(kFullMask, s_nb, o);
      mx_nb = fmaxf(mx_nb, __shfl_xor_sync(kFullMask, mx_nb, o));
      mn_nb = fminf(mn_nb, __shfl_xor_sync(kFullMask, mn_nb, o));
      mx_v = fmaxf(mx_v, __shfl_xor_sync(kFullMask, mx_v, o));
      s2 += __shfl_xor_sync(kFullMask, s2, o);
      s1 += __shfl_xor_sync(kFullMask, s1, o);
      dg = fmaxf(dg, __shfl_xor_sync(kFullMask, dg, o));
      bnd += __shfl_xor_sync(kFullMask, bnd, o);
      c10 += __shfl_xor_sync(kFullMask, c10, o);
      c100 += __shfl_xor_sync(kFullMask, c100, o);
      wnb += __shfl_xor_sync(kFullMask, wnb, o);
    }
    if (k == 0) mn_nb = 0.f;
    if (lane < 16) {
      float f;
      switch (lane) {
        case 0: f = log1pf((float)k); break;
        case 1: f = log1pf(s_nb); break;
        case 2: f = log1pf(mx_nb); break;
        case 3: f = log1pf(mn_nb); break;
        case 4: f = lg10(mx_v); break;
        case 5: f = lg10(sqrtf(s2)); break;
        case 6: f = lg10(s1); break;
        case 7: f = lg10(dg); break;
        case 8: f = lg10(bnd); break;
        case 9: f = log1pf(c10); break;
        case 10: f = log1pf(c100); break;
        case 11: f = ltau; break;
        case 12: f = branch; break;
        case 13: f = log1pf(s1 > 0.f ? wnb / s1 : 0.f); break;
        case 14: f = 1.f; break;
        default: f = 0.f; break;
      }
      feat[(size_t)r * 16 + lane] = f;
    }
  }
}

// ---------------------------------------------------------------- MLP
// Parameter layout (floats): W1[64][16], b1[64], W2[64][64], b2[64], w3[64], b3.
constexpr int kIn = 16, kH = 64;
constexpr int kW1 = 0, kB1 = kW1 + kH * kIn, kW2 = kB1 + kH, kB2 = kW2 + kH * kH, kW3 = kB2 + kH, kB3 = kW3 + kH;
static_assert(kB3 + 1 == NNZPRED_NPARAMS, "parameter count");
constexpr int kMlpWarps = 8;

// Normalised input of sample i (standardised with the predictor's statistics).
__device__ __forceinline__ float norm_in(const float *__restrict__ feat, size_t i, int c, const float *mean,
                                         const float *stdv) {
  return (feat[i * 16 + c] - mean[c]) / stdv[c];
}

// Shared-memory copy of the parameters with padded weight rows (W1 rows of 17, W2 rows of
// 65 floats), so that a lane per output unit (forward) and a lane per input column
// (backward) both read distinct banks.
constexpr int kPW1 = 0, kPB1 = kPW1 + kH * (kIn + 1), kPW2 = kPB1 + kH, kPB2 = kPW2 + kH * (kH + 1), kPW3 = kPB2 + kH,
              kPB3 = kPW3 + kH, kPN = kPB3 + 1;

__device__ __forceinline__ int padded(int i) {
  if (i < kB1) return kPW1 + (i / kIn) * (kIn + 1) + i % kIn;
  if (i < kW2) return kPB1 + (i - kB1);
  if (i < kB2) return kPW2 + ((i - kW2) / kH) * (kH + 1) + (i - kW2) % kH;
  return kPB2 + (i - kB2);  // b2, w3, b3 are contiguous in both layouts
}

__device__ __forceinline__ void load_padded(const float *__restrict__ P, float *sP) {
  for (int i = threadIdx.x; i < NNZPRED_NPARAMS; i += blockDim.x) sP[padded(i)] = P[i];
}

// One warp per sample: lane l owns hidden units l and l + 32 of both layers.
struct WarpAct {
  float x[kIn];
  float h1a, h1b, h2a, h2b, y;
};

__device__ __forceinline__ void mlp_forward_warp(const float *sP, const float *xin, float *h1s, WarpAct &act,
                                                 int lane) {
#pragma unroll
  for (int c = 0; c < kIn; ++c) act.x[c] = xin[c];
  const float *w1a = sP + kPW1 + lane * (kIn + 1), *w1b = sP + kPW1 + (lane + 32) * (kIn + 1);
  float a = sP[kPB1 + lane], b = sP[kPB1 + lane + 32];
#pragma unroll
  for (int c = 0; c < kIn; ++c) {
    a = fmaf(w1a[c], act.x[c], a);
    b = fmaf(w1b[c], act.x[c], b);
  }
  act.h1a = fmaxf(a, 0.f);
  act.h1b = fmaxf(b, 0.f);
  h1s[lane] = act.h1a;
  h1s[lane + 32] = act.h1b;
  __syncwarp();
  const float *w2a = sP + kPW2 + lane * (kH + 1), *w2b = sP + kPW2 + (lane + 32) * (kH + 1);
  a = sP[kPB2 + lane];
  b = sP[kPB2 + lane + 32];
#pragma unroll 16
  for (int c = 0; c < kH; ++c) {
    const float h = h1s[c];
    a = fmaf(w2a[c], h, a);
    b = fmaf(w2b[c], h, b);
  }
  act.h2a = fmaxf(a, 0.f);
  act.h2b = fmaxf(b, 0.f);
  float y = fmaf(sP[kPW3 + lane], act.h2a, sP[kPW3 + lane + 32] * act.h2b);
  for (int o = 16; o > 0; o >>= 1) y += __shfl_xor_sync(kFullMask, y, o);
  act.y = y + sP[kPB3];
}

__global__ void __launch_bounds__(kMlpWarps * 32) mlp_predict_kernel(const float *__restrict__ P,
                                                                     const float *__restrict__ stats,
                                                                     const float *__restrict__ feat, long long n,
                                                                     float *__restrict__ pred) {
  __shared__ float sP[kPN];
  __shared__ float h1s[kMlpWarps][kH];
  load_padded(P, sP);
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const float *mean = stats, *stdv = stats + 16;
  const float tmean = stats[32], tstd = stats[33], margin = stats[34];
  for (long long i = (long long)blockIdx.x * kMlpWarps + wid; i < n; i += (long long)gridDim.x * kMlpWarps) {
    float xin[kIn];
#pragma unroll
    for (int c = 0; c < kIn; ++c) xin[c] = norm_in(feat, (size_t)i, c, mean, stdv);
    WarpAct act;
    mlp_forward_warp(sP, xin, h1s[wid], act, lane);
    if (lane == 0) pred[i] = expm1f(fmaxf(act.y * tstd + tmean + margin, 0.f));  // back to a row length
    __syncwarp();
  }
}

// Gradient of the mean over samples of (y - t)^2 / 2, t the standardised log1p target.
// Each warp handles samples; per-block gradients are summed in shared memory (padded
// layout), then added to grad (packed layout, zeroed by the caller).  loss (optional)
// receives the summed squared error / 2.
__global__ void __launch_bounds__(kMlpWarps * 32) mlp_grad_kernel(const float *__restrict__ P,
                                                                  const float *__restrict__ stats,
                                                                  const float *__restrict__ feat,
                                                                  const int *__restrict__ count,
                                                                  const int *__restrict__ sel, long long n,
                                                                  float inv_n, float *__restrict__ grad,
                                                                  float *__restrict__ loss) {
  __shared__ float sP[kPN];
  __shared__ float sG[kPN];
  __shared__ float h1s[kMlpWarps][kH];
  __shared__ float dh2s[kMlpWarps][kH];
  __shared__ float sL;
  load_padded(P, sP);
  for (int i = threadIdx.x; i < kPN; i += blockDim.x) sG[i] = 0.f;
  if (threadIdx.x == 0) sL = 0.f;
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const float *mean = stats, *stdv = stats + 16;
  const float tmean = stats[32], tstd = stats[33];
  for (long long q = (long long)blockIdx.x * kMlpWarps + wid; q < n; q += (long long)gridDim.x * kMlpWarps) {
    const long long i = sel ? sel[q] : q;
    float xin[kIn];
#pragma unroll
    for (int c = 0; c < kIn; ++c) xin[c] = norm_in(feat, (size_t)i, c, mean, stdv);
    WarpAct act;
    mlp_forward_warp(sP, xin, h1s[wid], act, lane);
    const float t = (log1pf((float)count[i]) - tmean) / tstd;
    const float e = act.y - t;
    const float dy = e * inv_n;
    if (lane == 0) atomicAdd(&sL, 0.5f * e * e);
    // layer 3
    atomicAdd(&sG[kPW3 + lane], act.h2a * dy);
    atomicAdd(&sG[kPW3 + lane + 32], act.h2b * dy);
    if (lane == 0) atomicAdd(&sG[kPB3], dy);
    const float d2a = act.h2a > 0.f ? sP[kPW3 + lane] * dy : 0.f;
    const float d2b = act.h2b > 0.f ? sP[kPW3 + lane + 32] * dy : 0.f;
    dh2s[wid][lane] = d2a;
    dh2s[wid][lane + 32] = d2b;
    atomicAdd(&sG[kPB2 + lane], d2a);
    atomicAdd(&sG[kPB2 + lane + 32], d2b);
    __syncwarp();
    // layer 2 weights: dW2[u][c] = dh2[u] * h1[c]; lane covers columns c = lane, lane + 32
    const float h1c0 = h1s[wid][lane], h1c1 = h1s[wid][lane + 32];
    for (int u = 0; u < kH; ++u) {
      const float d = dh2s[wid][u];
      if (d != 0.f) {
        atomicAdd(&sG[kPW2 + u * (kH + 1) + lane], d * h1c0);
        atomicAdd(&sG[kPW2 + u * (kH + 1) + lane + 32], d * h1c1);
      }
    }
    // dh1[c] = sum_u W2[u][c] dh2[u], masked by relu
    float g0 = 0.f, g1 = 0.f;
    for (int u = 0; u < kH; ++u) {
      const float d = dh2s[wid][u];
      g0 = fmaf(sP[kPW2 + u * (kH + 1) + lane], d, g0);
      g1 = fmaf(sP[kPW2 + u * (kH + 1) + lane + 32], d, g1);
    }
    const float d1a = act.h1a > 0.f ? g0 : 0.f;
    const float d1b = act.h1b > 0.f ? g1 : 0.f;
    atomicAdd(&sG[kPB1 + lane], d1a);
    atomicAdd(&sG[kPB1 + lane + 32], d1b);
#pragma unroll
    for (int c = 0; c < kIn; ++c) {
      atomicAdd(&sG[kPW1 + lane * (kIn + 1) + c], d1a * act.x[c]);
      atomicAdd(&sG[kPW1 + (lane + 32) * (kIn + 1) + c], d1b * act.x[c]);
    }
    __syncwarp();
  }
  __syncthreads();
  for (int i = threadIdx.x; i < NNZPRED_NPARAMS; i += blockDim.x) {
    const float g = sG[padded(i)];
    if (g != 0.f) atomicAdd(grad + i, g);
  }
  if (threadIdx.x == 0 && loss) atomicAdd(loss, sL);
}

__global__ void adam_kernel(float *__restrict__ P, const float *__restrict__ G, float *__restrict__ M,
                            float *__restrict__ V, float lr, float b1, float b2, float eps, float c1, float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= NNZPRED_NPARAMS) return;
  const float g = G[i];
  const float m = b1 * M[i] + (1.f - b1) * g;
  const float v = b2 * V[i] + (1.f - b2) * g * g;
  M[i] = m;
  V[i] = v;
  P[i] -= lr * (m / c1) / (sqrtf(v / c2) + eps);
}

// Deterministic initialisation: uniform(-a, a) per parameter from a counter-based hash
// (splitmix64 of seed and index), a = sqrt(6 / fan_in); biases zero.
__device__ __forceinline__ unsigned long long splitmix64(unsigned long long x) {
  x += 0x9E3779B97F4A7C15ULL;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ULL;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBULL;
  return x ^ (x >> 31);
}

__global__ void init_params_kernel(float *__restrict__ P, unsigned long long seed) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= NNZPRED_NPARAMS) return;
  const float u = (float)((splitmix64(seed * 0x100000001B3ULL + (unsigned long long)i) >> 40) * (1.0 / 16777216.0));
  float a = 0.f;
  if (i < kB1) a = sqrtf(6.f / kIn);
  else if (i >= kW2 && i < kB2) a = sqrtf(6.f / kH);
  else if (i >= kW3 && i < kB3) a = sqrtf(6.f / kH);
  P[i] = a * (2.f * u - 1.f);
}

// Mini-batch selection: sample indices from a counter-based hash (epoch, step, i).
__global__ void batch_select_kernel(int *__restrict__ sel, int b, long long n, unsigned long long key) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= b) return;
  sel[i] = (int)(splitmix64(key + (unsigned long long)i) % (unsigned long long)n);
}

// Mean and standard deviation of the 16 features and of the target log1p(count) over
// the training set (one CTA: one warp per quantity, fixed order).
__global__ void feat_stats_kernel(const float *__restrict__ feat, const int *__restrict__ count, long long n,
                                  float *__restrict__ stats) {
  const int c = threadIdx.x >> 5, lane = threadIdx.x & 31;  // 17 warps
  double sum = 0.0, sq = 0.0;
  for (long long i = lane; i < n; i += 32) {
    const double v = c < 16 ? (double)feat[(size_t)i * 16 + c] : log1p((double)count[i]);
    sum += v;
    sq += v * v;
  }
  for (int o = 16; o > 0; o >>= 1) {
    sum += __shfl_xor_sync(kFullMask, sum, o);
    sq += __shfl_xor_sync(kFullMask, sq, o);
  }
  if (lane == 0) {
    const double mean = sum / (double)n;
    const double var = sq / (double)n - mean * mean;
    const double sd = var > 1e-12 ? sqrt(var) : 1.0;
    if (c < 16) { stats[c] = (float)mean; stats[16 + c] = (float)sd; }
    else { stats[32] = (float)mean; stats[33] = (float)sd; stats[34] = 0.f; }
  }
}

// Residuals log1p(count_i) - y_i of the network's log1p lengths (the margin left out).
__global__ void __launch_bounds__(kMlpWarps * 32) mlp_residual_kernel(const float *__restrict__ P,
                                                                     const float *__restrict__ stats,
                                                                     const float *__restrict__ feat,
                                                                     const int *__restrict__ count, long long n,
                                                                     float *__restrict__ res) {
  __shared__ float sP[kPN];
  __shared__ float h1s[kMlpWarps][kH];
  load_padded(P, sP);
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const float *mean = stats, *stdv = stats + 16;
  const float tmean = stats[32], tstd = stats[33];
  for (long long i = (long long)blockIdx.x * kMlpWarps + wid; i < n; i += (long long)gridDim.x * kMlpWarps) {
    float xin[kIn];
#pragma unroll
    for (int c = 0; c < kIn; ++c) xin[c] = norm_in(feat, (size_t)i, c, mean, stdv);
    WarpAct act;
    mlp_forward_warp(sP, xin, h1s[wid], act, lane);
    if (lane == 0) res[i] = log1pf((float)count[i]) - (act.y * tstd + tmean);
    __syncwarp();
  }
}

// Sum over rows of |log1p(pred) - log1p(actual)| and the number of rows whose actual
// length exceeds the prediction: per-thread FP32 sums over a grid-stride slice, a
// fixed-order FP64 tree per block into part[2 * block], then one warp adds the blocks'
// partial sums in block order (deterministic for a fixed grid).
constexpr int kErrBlocks = 256, kErrThreads = 256;
static_assert(kPredErrDoubles >= 2 + 2 * kErrBlocks, "prediction-error scratch");

__global__ void __launch_bounds__(kErrThreads) pred_error_kernel(const float *__restrict__ pred,
                                                                 const int *__restrict__ actual, long long n,
                                                                 double *__restrict__ part) {
  __shared__ double s_e[kErrThreads];
  __shared__ double s_u[kErrThreads];
  float e = 0.f, u = 0.f;
  for (long long i = (long long)blockIdx.x * kErrThreads + threadIdx.x; i < n; i += (long long)gridDim.x * kErrThreads) {
    const float a = (float)actual[i], p = pred[i];
    e += fabsf(log1pf(p) - log1pf(a));
    u += a > p ? 1.f : 0.f;
  }
  s_e[threadIdx.x] = e;
  s_u[threadIdx.x] = u;
  __syncthreads();
  for (int h = kErrThreads / 2; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h) { s_e[threadIdx.x] += s_e[threadIdx.x + h]; s_u[threadIdx.x] += s_u[threadIdx.x + h]; }
    __syncthreads();
  }
  if (threadIdx.x == 0) { part[2 * blockIdx.x] = s_e[0]; part[2 * blockIdx.x + 1] = s_u[0]; }
}

__global__ void pred_error_final_kernel(const double *__restrict__ part, int blocks, double *__restrict__ out) {
  const int lane = threadIdx.x;
  double e = 0.0, u = 0.0;
  for (int b = lane; b < blocks; b += 32) { e += part[2 * b]; u += part[2 * b + 1]; }
  for (int o = 16; o > 0; o >>= 1) {
    e += __shfl_xor_sync(kFullMask, e, o);
    u += __shfl_xor_sync(kFullMask, u, o);
  }
  if (lane == 0) { out[0] = e; out[1] = u; }
}

// Largest of n non-negative floats (as int bits, whose order matches) into *out, which the
// caller zeroes.
__global__ void __launch_bounds__(256) max_float_kernel(const float *__restrict__ v, long long n,
                                                        int *__restrict__ out) {
  __shared__ float s[256];
  float m = 0.f;
  for (long long i = (long long)blockIdx.x * 256 + threadIdx.x; i < n; i += (long long)gridDim.x * 256)
    m = fmaxf(m, v[i]);
  s[threadIdx.x] = m;
  __syncthreads();
  for (int h = 128; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h) s[threadIdx.x] = fmaxf(s[threadIdx.x], s[threadIdx.x + h]);
    __syncthreads();
  }
  if (threadIdx.x == 0 && s[0] > 0.f) atomicMax(out, __float_as_int(s[0]));
}

int grid_warps(long long items, int warps_per_block) {
  long long b = (items + warps_per_block - 1) / warps_per_block;
  long long cap = (long long)num_sms() * 8;
  return (int)(b < 1 ? 1 : (b < cap ? b : cap));
}

}  // namespace

// Structural counts of A*B (+C); launched from the SP2 driver too.
int struct_count_async(const ellpack_t *A, const ellpack_t *B, const ellpack_t *C, int *counts, int *dmax,
                       cudaStream_t s) {
  if (B->n > kCntMaxN) return fail(SP2E_ARG, "structural count: %d columns, above the limit %d", B->n, kCntMaxN);
  SP2_CUDA(cudaMemsetAsync(dmax, 0, sizeof(int), s));
  const int smem = kCntWarps * kCntBytesPerWarp;
  const int grid = grid_warps(A->n, kCntWarps);
  if (A->dtype == SP2_F64) {
    SP2_CUDA(cudaFuncSetAttribute(struct_count_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    struct_count_kernel<double><<<grid, kCntWarps * 32, smem, s>>>(view<double>(A), view<double>(B),
                                                                     C ? view<double>(C) : view<double>(A), C != nullptr,
                                                                     counts, dmax);
  } else {
    SP2_CUDA(cudaFuncSetAttribute(struct_count_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    struct_count_kernel<float><<<grid, kCntWarps * 32, smem, s>>>(view<float>(A), view<float>(B),
                                                                    C ? view<float>(C) : view<float>(A), C != nullptr,
                                                                    counts, dmax);
  }
  note_launch();
  SP2_CUDA(cudaGetLastError());
  return SP2_OK;
}

int features_async(const ellpack_t *X, double tau, int branch, float *rmax_scratch, float *feat, cudaStream_t s) {
  const int grid = grid_warps(X->n, 8);
  const float ltau = tau > 0.0 ? (float)log10(tau) : -30.f;
  if (X->dtype == SP2_F64) {
    rowmax_kernel<double><<<grid, 256, 0, s>>>(view<double>(X), rmax_scratch);
    features_kernel<double><<<grid, 256, 0, s>>>(view<double>(X), rmax_scratch, ltau, branch == 2 ? 1.f : 0.f,
                                                 (float)tau, feat);
  } else {
    rowmax_kernel<float><<<grid, 256, 0, s>>>(view<float>(X), rmax_scratch);
    features_kernel<float><<<grid, 256, 0, s>>>(view<float>(X), rmax_scratch, ltau, branch == 2 ? 1.f : 0.f,
                                                (float)tau, feat);
  }
  note_launch();
  note_launch();
  SP2_CUDA(cudaGetLastError());
  return SP2_OK;
}

int pred_error_async(const float *pred, const int *actual, long long n, double *out2, cudaStream_t s) {
  // out2 holds 2 + 2 * kErrBlocks doubles: the result, then the blocks' partial sums
  long long b = (n + kErrThreads - 1) / kErrThreads;
  const int blocks = (int)(b < kErrBlocks ? (b < 1 ? 1 : b) : kErrBlocks);
  pred_error_kernel<<<blocks, kErrThreads, 0, s>>>(pred, actual, n, out2 + 2);
  pred_error_final_kernel<<<1, 32, 0, s>>>(out2 + 2, blocks, out2);
  note_launch();
  note_launch();
  SP2_CUDA(cudaGetLastError());
  return SP2_OK;
}

int max_float_async(const float *v, long long n, float *out, cudaStream_t s) {
  SP2_CUDA(cudaMemsetAsync(out, 0, sizeof(float), s));
  long long b = (n + 255) / 256;
  const long long cap = (long long)num_sms() * 2;
  max_float_kernel<<<(int)(b < cap ? (b < 1 ? 1 : b) : cap), 256, 0, s>>>(v, n, reinterpret_cast<int *>(out));
  note_launch();
  SP2_CUDA(cudaGetLastError());
  return SP2_OK;
}

int predict_async(const nnzpred_t *p, const float *feat, long long n, float *pred, cudaStream_t s) {
  mlp_predict_kernel<<<grid_warps(n, kMlpWarps), kMlpWarps * 32, 0, s>>>(p->params, p->stats, feat, n, pred);
  note_launch();
  SP2_CUDA(cudaGetLastError());
  return SP2_OK;
}

}  // namespace sp2

using namespace sp2;

static int check_pred(const nnzpred_t *p, const char *who) {
  if (!p || !p->params || !p->stats || !p->adam_m || !p->adam_v) return fail(SP2E_ARG, "%s: predictor not created", who);
  return SP2_OK;
}

extern "C" int ellpack_struct_count(const ellpack_t *A, const ellpack_t *B, const ellpack_t *C, int32_t *counts,
                                    int32_t *max_count, void *stream) {
  SP2_TRY(check_matrix(A, "ellpack_struct_count: A"));
  SP2_TRY(check_matrix(B, "ellpack_struct_count: B"));
  if (C) SP2_TRY(check_matrix(C, "ellpack_struct_count: C"));
  if (!counts) return fail(SP2E_ARG, "ellpack_struct_count: counts is NULL");
  if (A->n != B->n || (C && C->n != A->n)) return fail(SP2E_ARG, "ellpack_struct_count: sizes differ");
  if (A->dtype != B->dtype || (C && C->dtype != A->dtype)) return fail(SP2E_ARG, "ellpack_struct_count: dtypes differ");
  cudaStream_t s = as_stream(stream);
  int *dmax = nullptr;
  SP2_TRY(dev_alloc((void **)&dmax, sizeof(int), s));
  int rc = struct_count_async(A, B, C, counts, dmax, s);
  int h = 0;
  if (rc == SP2_OK) {
    cudaError_t e = cudaMemcpyAsync(&h, dmax, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) rc = cuda_fail(e, "ellpack_struct_count", __FILE__, __LINE__);
  }
  dev_free(dmax, s);
  SP2_TRY(rc);
  if (max_count) *max_count = h;
  return SP2_OK;
}

extern "C" int nnzpred_features(const ellpack_t *X, double tau, int32_t branch, float *feat, void *stream) {
  SP2_TRY(check_matrix(X, "nnzpred_features: X"));
  if (!feat) return fail(SP2E_ARG, "nnzpred_features: feat is NULL");
  if (!(tau >= 0.0) || !isfinite(tau)) return fail(SP2E_ARG, "nnzpred_features: bad tau");
  cudaStream_t s = as_stream(stream);
  float *rmax = nullptr;
  SP2_TRY(dev_alloc((void **)&rmax, sizeof(float) * (size_t)X->n, s));
  int rc = features_async(X, tau, branch, rmax, feat, s);
  dev_free(rmax, s);
  return rc;
}

extern "C" int nnzpred_create(nnzpred_t *p, uint64_t seed, void *stream) {
  if (!p) return fail(SP2E_ARG, "nnzpred_create: NULL");
  memset(p, 0, sizeof(*p));
  cudaStream_t s = as_stream(stream);
  float *buf = nullptr;
  SP2_TRY(dev_alloc((void **)&buf, sizeof(float) * (3 * NNZPRED_NPARAMS + NNZPRED_NSTATS), s));
  p->params = buf;
  p->adam_m = buf + NNZPRED_NPARAMS;
  p->adam_v = buf + 2 * NNZPRED_NPARAMS;
  p->stats = buf + 3 * NNZPRED_NPARAMS;
  SP2_CUDA(cudaMemsetAsync(p->adam_m, 0, sizeof(float) * (2 * NNZPRED_NPARAMS + NNZPRED_NSTATS), s));
  init_params_kernel<<<(NNZPRED_NPARAMS + 255) / 256, 256, 0, s>>>(p->params, (unsigned long long)seed);
  note_launch();
  // identity statistics until training sets them
  float id[NNZPRED_NSTATS];
  for (int i = 0; i < NNZPRED_NSTATS; ++i) id[i] = (i >= 16 && i < 32) || i == 33 ? 1.f : 0.f;
  SP2_CUDA(cudaMemcpyAsync(p->stats, id, sizeof(id), cudaMemcpyHostToDevice, s));
  SP2_CUDA(cudaStreamSynchronize(s));
  p->steps = 0;
  return SP2_OK;
}

extern "C" int nnzpred_destroy(nnzpred_t *p, void *stream) {
  if (!p) return fail(SP2E_ARG, "nnzpred_destroy: NULL");
  if (p->params) dev_free(p->params, as_stream(stream));
  memset(p, 0, sizeof(*p));
  return SP2_OK;
}

extern "C" int nnzpred_set_stats(nnzpred_t *p, const float *feat, const int32_t *count, int64_t n, void *stream) {
  SP2_TRY(check_pred(p, "nnzpred_set_stats"));
  if (!feat || !count || n < 1) return fail(SP2E_ARG, "nnzpred_set_stats: bad arguments");
  feat_stats_kernel<<<1, 17 * 32, 0, as_stream(stream)>>>(feat, count, n, p->stats);
  note_launch();
  SP2_CUDA(cudaGetLastError());
  return SP2_OK;
}

extern "C" int nnzpred_grad(const nnzpred_t *p, const float *feat, const int32_t *count, int64_t n, float *grad,
                            float *loss, void *stream) {
  SP2_TRY(check_pred(p, "nnzpred_grad"));
  if (!feat || !count || !grad || n < 1) return fail(SP2E_ARG, "nnzpred_grad: bad arguments");
  cudaStream_t s = as_stream(stream);
  float *dl = nullptr;
  SP2_TRY(dev_alloc((void **)&dl, sizeof(float), s));
  SP2_CUDA(cudaMemsetAsync(grad, 0, sizeof(float) * NNZPRED_NPARAMS, s));
  SP2_CUDA(cudaMemsetAsync(dl, 0, sizeof(float), s));
  mlp_grad_kernel<<<grid_warps(n, kMlpWarps), kMlpWarps * 32, 0, s>>>(p->params, p->stats, feat, count, nullptr, n,
                                                                      1.f / (float)n, grad, dl);
  note_launch();
  float h = 0.f;
  cudaError_t e = cudaMemcpyAsync(&h, dl, sizeof(float), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  dev_free(dl, s);
  if (e != cudaSuccess) return cuda_fail(e, "nnzpred_grad", __FILE__, __LINE__);
  if (loss) *loss = h / (float)n;
  return SP2_OK;
}

extern "C" int nnzpred_train(nnzpred_t *p, const float *feat, const int32_t *count, int64_t n, int32_t steps,
                             int32_t batch, float lr, float *final_loss, void *stream) {
  SP2_TRY(check_pred(p, "nnzpred_train"));
  if (!feat || !count || n < 1 || steps < 0 || batch < 1) return fail(SP2E_ARG, "nnzpred_train: bad arguments");
  cudaStream_t s = as_stream(stream);
  float *work = nullptr;
  SP2_TRY(dev_alloc((void **)&work, sizeof(float) * (NNZPRED_NPARAMS + 1) + sizeof(int) * (size_t)batch, s));
  float *grad = work, *dl = work + NNZPRED_NPARAMS;
  int *sel = reinterpret_cast<int *>(work + NNZPRED_NPARAMS + 1);
  const float b1 = 0.9f, b2 = 0.999f;
  int rc = SP2_OK;
  for (int t = 0; t < steps && rc == SP2_OK; ++t) {
    const int step = p->steps + t + 1;
    batch_select_kernel<<<(batch + 255) / 256, 256, 0, s>>>(sel, batch, n,
                                                            0xC0FFEEULL * (unsigned long long)step * 0x9E3779B1ULL);
    cudaMemsetAsync(grad, 0, sizeof(float) * (NNZPRED_NPARAMS + 1), s);
    mlp_grad_kernel<<<grid_warps(batch, kMlpWarps), kMlpWarps * 32, 0, s>>>(
        p->params, p->stats, feat, count, sel, batch, 1.f / (float)batch, grad, t + 1 == steps ? dl : nullptr);
    adam_kernel<<<(NNZPRED_NPARAMS + 255) / 256, 256, 0, s>>>(p->params, grad, p->adam_m, p->adam_v, lr, b1, b2,
                                                              1e-8f, 1.f - powf(b1, (float)step),
                                                              1.f - powf(b2, (float)step));
    note_launch();
    note_launch();
    note_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) rc = cuda_fail(e, "nnzpred_train", __FILE__, __LINE__);
  }
  float h = 0.f;
  if (rc == SP2_OK && steps > 0) {
    cudaError_t e = cudaMemcpyAsync(&h, dl, sizeof(float), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) rc = cuda_fail(e, "nnzpred_train", __FILE__, __LINE__);
  }
  dev_free(work, s);
  SP2_TRY(rc);
  p->steps += steps;
  if (final_loss) *final_loss = steps > 0 ? h / (float)batch : 0.f;
  return SP2_OK;
}

extern "C" int nnzpred_predict(const nnzpred_t *p, const float *feat, int64_t n, float *pred, void *stream) {
  SP2_TRY(check_pred(p, "nnzpred_predict"));
  if (!feat || !pred || n < 1) return fail(SP2E_ARG, "nnzpred_predict: bad arguments");
  return predict_async(p, feat, n, pred, as_stream(stream));
}

extern "C" int nnzpred_calibrate(nnzpred_t *p, const float *feat, const int32_t *count, int64_t n, float quantile,
                                 float *margin, void *stream) {
  SP2_TRY(check_pred(p, "nnzpred_calibrate"));
  if (!feat || !count || n < 1) return fail(SP2E_ARG, "nnzpred_calibrate: bad arguments");
  if (!(quantile > 0.f && quantile <= 1.f)) return fail(SP2E_ARG, "nnzpred_calibrate: quantile must be in (0, 1]");
  cudaStream_t s = as_stream(stream);
  float *res = nullptr;
  SP2_TRY(dev_alloc((void **)&res, sizeof(float) * (size_t)n, s));
  mlp_residual_kernel<<<grid_warps(n, kMlpWarps), kMlpWarps * 32, 0, s>>>(p->params, p->stats, feat, count, n, res);
  note_launch();
  std::vector<float> h((size_t)n);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(h.data(), res, sizeof(float) * (size_t)n, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  dev_free(res, s);
  if (e != cudaSuccess) return cuda_fail(e, "nnzpred_calibrate", __FILE__, __LINE__);
  // the k-th smallest residual, k = ceil(quantile * n): at least that share lies at or below it
  size_t k = (size_t)ceil((double)quantile * (double)n);
  if (k < 1) k = 1;
  if (k > (size_t)n) k = (size_t)n;
  std::nth_element(h.begin(), h.begin() + (k - 1), h.end());
  float m = h[k - 1];
  if (!(m > 0.f)) m = 0.f;  // the margin only raises predictions (a NaN residual gives none)
  SP2_CUDA(cudaMemcpyAsync(p->stats + 34, &m, sizeof(float), cudaMemcpyHostToDevice, s));
  SP2_CUDA(cudaStreamSynchronize(s));
  if (margin) *margin = m;
  return SP2_OK;
}

extern "C" int nnzpred_width(const nnzpred_t *p, const ellpack_t *X, double tau, int32_t branch, int32_t *width,
                             float *pred, void *stream) {
  SP2_TRY(check_pred(p, "nnzpred_width"));
  SP2_TRY(check_matrix(X, "nnzpred_width: X"));
  if (!width) return fail(SP2E_ARG, "nnzpred_width: width is NULL");
  if (!(tau >= 0.0) || !isfinite(tau)) return fail(SP2E_ARG, "nnzpred_width: bad tau");
  cudaStream_t s = as_stream(stream);
  const size_t n = (size_t)X->n;
  float *scr = nullptr;  // rmax[n], feat[16n], pred[n] (unless given), max
  SP2_TRY(dev_alloc((void **)&scr, sizeof(float) * (18 * n + 1), s));
  float *rmax = scr, *feat = scr + n, *pr = pred ? pred : scr + 17 * n, *fmax = scr + 18 * n;
  int rc = features_async(X, tau, branch, rmax, feat, s);
  if (rc == SP2_OK) rc = predict_async(p, feat, (long long)n, pr, s);
  if (rc == SP2_OK) rc = max_float_async(pr, (long long)n, fmax, s);
  float h = 0.f;
  if (rc == SP2_OK) {
    cudaError_t e = cudaMemcpyAsync(&h, fmax, sizeof(float), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) rc = cuda_fail(e, "nnzpred_width", __FILE__, __LINE__);
  }
  dev_free(scr, s);
  SP2_TRY(rc);
  long long w = ((predicted_width(h) + 31) / 32) * 32;
  if (w > X->n) w = X->n;
  if (w < 1) w = 1;
  *width = (int32_t)w;
  return SP2_OK;
}

extern "C" int nnzpred_save(const nnzpred_t *p, const char *path, void *stream) {
  SP2_TRY(check_pred(p, "nnzpred_save"));
  if (!path) return fail(SP2E_ARG, "nnzpred_save: path is NULL");
  std::vector<float> h(NNZPRED_NPARAMS + NNZPRED_NSTATS);
  cudaStream_t s = as_stream(stream);
  SP2_CUDA(cudaMemcpyAsync(h.data(), p->params, sizeof(float) * NNZPRED_NPARAMS, cudaMemcpyDeviceToHost, s));
  SP2_CUDA(cudaMemcpyAsync(h.data() + NNZPRED_NPARAMS, p->stats, sizeof(float) * NNZPRED_NSTATS,
                           cudaMemcpyDeviceToHost, s));
  SP2_CUDA(cudaStreamSynchronize(s));
  FILE *f = fopen(path, "wb");
  if (!f) return fail(SP2E_ARG, "nnzpred_save: cannot open %s", path);
  const char magic[8] = {'N', 'N', 'Z', 'P', 'R', 'D', '0', '1'};
  size_t ok = fwrite(magic, 1, 8, f) == 8 && fwrite(h.data(), sizeof(float), h.size(), f) == h.size();
  fclose(f);
  if (!ok) return fail(SP2E_ARG, "nnzpred_save: write failed");
  return SP2_OK;
}

extern "C" int nnzpred_load(nnzpred_t *p, const char *path, void *stream) {
  SP2_TRY(check_pred(p, "nnzpred_load"));
  if (!path) return fail(SP2E_ARG, "nnzpred_load: path is NULL");
  std::vector<float> h(NNZPRED_NPARAMS + NNZPRED_NSTATS);
  FILE *f = fopen(path, "rb");
  if (!f) return fail(SP2E_ARG, "nnzpred_load: cannot open %s", path);
  char magic[8];
  bool ok = fread(magic, 1, 8, f) == 8 && memcmp(magic, "NNZPRD01", 8) == 0 &&
            fread(h.data(), sizeof(float), h.size(), f) == h.size();
  fclose(f);
  if (!ok) return fail(SP2E_ARG, "nnzpred_load: %s is not a predictor file", path);
  cudaStream_t s = as_stream(stream);
  SP2_CUDA(cudaMemcpyAsync(p->params, h.data(), sizeof(float) * NNZPRED_NPARAMS, cudaMemcpyHostToDevice, s));
  SP2_CUDA(cudaMemcpyAsync(p->stats, h.data() + NNZPRED_NPARAMS, sizeof(float) * NNZPRED_NSTATS,
                           cudaMemcpyHostToDevice, s));
  SP2_CUDA(cudaStreamSynchronize(s));
  return SP2_OK;
}
