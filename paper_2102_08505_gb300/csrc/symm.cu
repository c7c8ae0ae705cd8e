// symm.cu -- the symmetric product X*X (+ X) by its upper triangle.
//
// For symmetric X the product C = alpha X*X + beta X is symmetric, and C_ij and C_ji are
// the same sum over the same k in the same (ascending) order.  So each output row i
// computes only its columns j >= i: for a term a_ik * B_k it reads row k of B from the
// first column >= i on, a position found once per product by a lower-bound search
// (upper_start_kernel).  The upper rows U are then mirrored into full rows:
//   count   -- entries (i, j > i) of U per column j: the length L_j of row j's lower part;
//   place   -- row i's U part goes to positions L_i .. of output row i, and every (i, j > i)
//              is scattered to row j's lower part (positions from a per-row cursor);
//   sort    -- each lower part is sorted by column (its columns are distinct, so the order
//              is unique), and the row's diagonal value and sum of squares are recorded.
// The full rows equal, bit for bit, those computed without the symmetry, with about half
// the products.
#include <limits.h>
#include <math.h>

#include "common.cuh"

namespace sp2 {
namespace {

constexpr unsigned kFullM = 0xffffffffu;
constexpr int kSymThreads = 256;
constexpr int kSortWarpMax = 256;    // lower parts up to this length are sorted by one warp in registers
constexpr int kSortMidMax = 512;     // ... up to this length by one warp in registers, in a kernel of their own
constexpr int kSortCtaMax = 4096;    // ... up to this length by one CTA in shared memory

int grid_rows_sym(long long rows) {
  long long b = (rows * 32 + kSymThreads - 1) / kSymThreads;
  const long long cap = (long long)num_sms() * 16;
  return (int)(b < 1 ? 1 : (b < cap ? b : cap));
}

__device__ __forceinline__ bool row_active(const BatchView &bv, int r) {
  return !bv.row_mat || bv.active[bv.row_mat[r]];
}

// tp[r*w + s] = first position of row k = idx[r, s] with a column >= r; tpd[r] = the same
// in row r itself.  One warp per row; each lane a binary search of its entry's row.
template <typename T>
__global__ void upper_start_kernel(EllView<T> X, int *__restrict__ tp, int *__restrict__ tpd) {
  const int lane = threadIdx.x & 31;
  const int warps = (gridDim.x * blockDim.x) >> 5;
  for (int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < X.n; r += warps) {
    const int nr = min(X.nnz[r], X.w);
    for (int s = lane; s < nr; s += 32) {
      const int k = X.idx[(size_t)r * X.w + s];
      int lo = 0;
      if ((unsigned)k < (unsigned)X.n) {
        const int *rk = X.idx + (size_t)k * X.w;
        int hi = min(X.nnz[k], X.w);
        while (lo < hi) {
          const int mid = (lo + hi) >> 1;
          if (rk[mid] < r) lo = mid + 1; else hi = mid;
        }
      }
      tp[(size_t)r * X.w + s] = lo;
    }
    if (lane == 0) {
      const int *rr = X.idx + (size_t)r * X.w;
      int lo = 0, hi = nr;
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (rr[mid] < r) lo = mid + 1; else hi = mid;
      }
      tpd[r] = lo;
    }
  }
}

// cnt[j] += 1 for every entry (i, j > i) of U.
template <typename T>
__global__ void mirror_count_kernel(EllView<T> U, BatchView bv, int *__restrict__ cnt) {
  const int lane = threadIdx.x & 31;
  const int warps = (gridDim.x * blockDim.x) >> 5;
  for (int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < U.n; i += warps) {
    if (!row_active(bv, i)) continue;
    const int nu = min(U.nnz[i], U.w);
    for (int s = lane; s < nu; s += 32) {
      const int j = U.idx[(size_t)i * U.w + s];
      if (j > i && j < U.n) atomicAdd(cnt + j, 1);
    }
  }
}

// Output row i: its U part at positions cnt[i] .. (if the row fits), and each (i, j > i)
// into row j at a position taken from cursor[j] (always below cnt[j]).
template <typename T>
__global__ void mirror_place_kernel(EllView<T> U, EllOut<T> Out, BatchView bv, const int *__restrict__ cnt,
                                    int *__restrict__ cursor, SpgemmCtl *__restrict__ ctl) {
  const int lane = threadIdx.x & 31;
  const int warps = (gridDim.x * blockDim.x) >> 5;
  int wmax = 0, wover = 0;
  for (int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < U.n; i += warps) {
    if (!row_active(bv, i)) continue;
    const int nu = min(U.nnz[i], U.w);
    const int L = cnt[i];
    const int total = L + nu;
    const bool fits = total <= Out.w;
    for (int s = lane; s < nu; s += 32) {
      const int j = U.idx[(size_t)i * U.w + s];
      const T v = U.val[(size_t)i * U.w + s];
      if (fits) {
        Out.idx[(size_t)i * Out.w + L + s] = j;
        Out.val[(size_t)i * Out.w + L + s] = v;
      }
      if (j > i && j < U.n) {
        const int p = atomicAdd(cursor + j, 1);
        if (p < Out.w) {
          Out.idx[(size_t)j * Out.w + p] = i;
          Out.val[(size_t)j * Out.w + p] = v;
        }
      }
    }
    if (lane == 0) {
      Out.nnz[i] = fits ? total : 0;  // an overflowing row is left empty (its content is unspecified)
      if (!fits) ++wover;
      wmax = max(wmax, total);
    }
  }
  if (lane == 0) {
    if (wmax) atomicMax(&ctl->max_count, wmax);
    if (wover) atomicAdd(&ctl->overflow_rows, wover);
  }
}

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFullM, v, o);
  return v;
}

// Sorts the L <= 32*E entries at ri/rv by column (distinct columns): keys (column, old
// position) sorted in registers, then the values gathered from their old positions.  K =
// unsigned: the key packs the column above the PB = log2(32*E) position bits (columns below
// 2^(32-PB): half the shuffles of the 64-bit key); K = unsigned long long: column << 32.
template <typename K, int E>
struct SortKey {
  static constexpr int PB = sizeof(K) == 8 ? 32 : (E == 1 ? 5 : E == 2 ? 6 : E == 4 ? 7 : E == 8 ? 8 : 9);
  static_assert(sizeof(K) == 8 || E <= 16, "32-bit keys for up to 16 entries per lane");
};
template <typename T, int E, typename K>
__device__ __forceinline__ void warp_sort_row(int *ri, T *rv, int L, int lane) {
  constexpr int PB = SortKey<K, E>::PB;
  K a[E];
#pragma unroll
  for (int t = 0; t < E; ++t) {
    const int s = lane * E + t;
    a[t] = s < L ? ((K)(unsigned)ri[s] << PB) | (K)(unsigned)s : ~(K)0;
  }
  warp_bitonic<K, E>(a, lane);
  T v[E];
#pragma unroll
  for (int t = 0; t < E; ++t)
    v[t] = lane * E + t < L ? rv[(unsigned)(a[t] & (((K)1 << PB) - 1))] : T(0);
  __syncwarp();  // every old value is read before any is overwritten
#pragma unroll
  for (int t = 0; t < E; ++t) {
    const int s = lane * E + t;
    if (s < L) {
      ri[s] = (int)(a[t] >> PB);
      rv[s] = v[t];
    }
  }
  __syncwarp();
}
// rowstat[i] = (diagonal, sum of squares) of the full row i, one warp.
template <typename T>
__device__ __forceinline__ void row_stat_warp(const int *ri, const T *rv, int total, int i, int lane,
                                              double2 *rowstat) {
  double d = 0.0, f = 0.0;
  for (int s = lane; s < total; s += 32) {
    const double v = (double)rv[s];
    if (ri[s] == i) d += v;
    f = fma(v, v, f);
  }
  d = warp_sum_d(d);
  f = warp_sum_d(f);
  if (lane == 0) rowstat[i] = make_double2(d, f);
  __syncwarp();
}

// Sorts row i's lower part (positions 0 .. L-1) by column and records rowstat[i].  One
// warp per row, in registers for L <= kSortWarpMax; longer lower parts are left for the
// passes over the flagged rows (list `longs`).
// K: the sort key (unsigned when every column is below 2^24, the 8 position bits of 256
// entries leaving 24 for the column; else unsigned long long), chosen at launch.
template <typename T, typename K>
__global__ void __launch_bounds__(kSymThreads) mirror_sort_kernel(EllOut<T> Out, BatchView bv,
                                                                 const int *__restrict__ cnt,
                                                                 double2 *__restrict__ rowstat,
                                                                 int *__restrict__ longs, int *__restrict__ nlong) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int warps = gridDim.x * (kSymThreads / 32);
  for (int i = blockIdx.x * (kSymThreads / 32) + wid; i < Out.n; i += warps) {
    if (!row_active(bv, i)) continue;
    const int L = cnt[i];
    const int total = Out.nnz[i];
    if (total > Out.w || total < L) {  // the row overflowed: nothing to sort
      if (lane == 0) rowstat[i] = make_double2(0.0, 0.0);
      continue;
    }
    int *ri = Out.idx + (size_t)i * Out.w;
    T *rv = Out.val + (size_t)i * Out.w;
    if (L > kSortWarpMax) {
      if (lane == 0) longs[atomicAdd(nlong, 1)] = i;
      continue;
    }
    if (L > 128) {
      warp_sort_row<T, 8, K>(ri, rv, L, lane);
    } else if (L > 32) {
      if (L > 64) warp_sort_row<T, 4, K>(ri, rv, L, lane);
      else warp_sort_row<T, 2, K>(ri, rv, L, lane);
    } else if (L > 1) {
      warp_sort_row<T, 1, K>(ri, rv, L, lane);
    }
    row_stat_warp(ri, rv, total, i, lane, rowstat);
  }
}

// Flagged rows with kSortWarpMax < L <= kSortMidMax: one warp per row, 16 keys per lane
// (a kernel of its own so that the registers this takes do not limit the common pass).  K as
// in mirror_sort_kernel, with 9 position bits (columns below 2^23 for the 32-bit key).
template <typename T, typename K>
__global__ void __launch_bounds__(kSymThreads) mirror_sort_mid_kernel(EllOut<T> Out, const int *__restrict__ cnt,
                                                                     double2 *__restrict__ rowstat,
                                                                     const int *__restrict__ longs,
                                                                     const int *__restrict__ nlong) {
  const int nl = *nlong;
  const int lane = threadIdx.x & 31;
  const int warps = gridDim.x * (kSymThreads / 32);
  for (int q = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; q < nl; q += warps) {
    const int i = longs[q];
    const int L = cnt[i];
    if (L > kSortMidMax) continue;
    int *ri = Out.idx + (size_t)i * Out.w;
    T *rv = Out.val + (size_t)i * Out.w;
    warp_sort_row<T, 16, K>(ri, rv, L, lane);
    row_stat_warp(ri, rv, Out.nnz[i], i, lane, rowstat);
  }
}

// Long lower parts (L > kSortMidMax): one CTA per row.  Up to kSortCtaMax entries, bitonic in shared memory;
// beyond, each entry's rank (count of smaller columns) places it in the row's slots of U,
// free once the U part has been placed, and the sorted part is copied back.
template <typename T>
__global__ void __launch_bounds__(kSymThreads) mirror_sort_long_kernel(EllOut<T> Out, EllOut<T> Uscr,
                                                                      const int *__restrict__ cnt,
                                                                      double2 *__restrict__ rowstat,
                                                                      const int *__restrict__ longs,
                                                                      const int *__restrict__ nlong) {
  extern __shared__ __align__(16) unsigned char smem[];
  int *sk = reinterpret_cast<int *>(smem);
  T *sv = reinterpret_cast<T *>(smem + sizeof(int) * kSortCtaMax);
  __shared__ double s_d[kSymThreads / 32], s_f[kSymThreads / 32];
  const int nl = *nlong;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int q = blockIdx.x; q < nl; q += gridDim.x) {
    const int i = longs[q];
    const int L = cnt[i];
    if (L <= kSortMidMax) continue;  // the same for the whole CTA: sorted by the warp pass
    const int total = Out.nnz[i];
    int *ri = Out.idx + (size_t)i * Out.w;
    T *rv = Out.val + (size_t)i * Out.w;
    if (L <= kSortCtaMax) {
      int P = 2;
      while (P < L) P <<= 1;
      for (int s = threadIdx.x; s < P; s += blockDim.x) {
        sk[s] = s < L ? ri[s] : INT_MAX;
        sv[s] = s < L ? rv[s] : T(0);
      }
      __syncthreads();
      for (int k = 2; k <= P; k <<= 1)
        for (int jj = k >> 1; jj > 0; jj >>= 1) {
          for (int e = threadIdx.x; e < (P >> 1); e += blockDim.x) {
            const int a = ((e & ~(jj - 1)) << 1) | (e & (jj - 1));
            const int b = a + jj;
            const int x = sk[a], y = sk[b];
            if ((x > y) == ((a & k) == 0)) {
              sk[a] = y; sk[b] = x;
              const T t = sv[a]; sv[a] = sv[b]; sv[b] = t;
            }
          }
          __syncthreads();
        }
      for (int s = threadIdx.x; s < L; s += blockDim.x) {
        ri[s] = sk[s];
        rv[s] = sv[s];
      }
    } else {
      int *ui = Uscr.idx + (size_t)i * Uscr.w;
      T *uv = Uscr.val + (size_t)i * Uscr.w;
      for (int s = threadIdx.x; s < L; s += blockDim.x) {
        const int c = ri[s];
        int rank = 0;
        for (int t = 0; t < L; ++t) rank += ri[t] < c;
        if (rank < Uscr.w) {
          ui[rank] = c;
          uv[rank] = rv[s];
        }
      }
      __syncthreads();
      for (int s = threadIdx.x; s < L; s += blockDim.x) {
        ri[s] = ui[s];
        rv[s] = uv[s];
      }
    }
    __syncthreads();
    double d = 0.0, f = 0.0;
    for (int s = threadIdx.x; s < total; s += blockDim.x) {
      const double v = (double)rv[s];
      if (ri[s] == i) d += v;
      f = fma(v, v, f);
    }
    d = warp_sum_d(d);
    f = warp_sum_d(f);
    if (lane == 0) { s_d[wid] = d; s_f[wid] = f; }
    __syncthreads();
    if (threadIdx.x == 0) {
      double dd = 0.0, ff = 0.0;
      for (int w = 0; w < kSymThreads / 32; ++w) { dd += s_d[w]; ff += s_f[w]; }
      rowstat[i] = make_double2(dd, ff);
    }
    __syncthreads();
  }
}

}  // namespace

int upper_start_async(const ellpack_t *X, int *tp, int *tpd, cudaStream_t s) {
  const int g = grid_rows_sym(X->n);
  prof_begin(SP2_PROF_SYMM, s);
  if (X->dtype == SP2_F64) upper_start_kernel<double><<<g, kSymThreads, 0, s>>>(view<double>(X), tp, tpd);
  else upper_start_kernel<float><<<g, kSymThreads, 0, s>>>(view<float>(X), tp, tpd);
  note_launch();
  prof_end(SP2_PROF_SYMM, s);
  SP2_CUDA(cudaGetLastError());
  return SP2_OK;
}

template <typename T>
static int mirror_t(const ellpack_t *U, ellpack_t *Out, const BatchView &bv, int *work, double2 *rowstat,
                    SpgemmCtl *ctl, cudaStream_t s) {
  const int n = U->n;
  // work: cnt[n], cursor[n], nlong[1] (zeroed here), longs[n]
  int *cnt = work, *cursor = work + n, *nlong = work + 2 * n, *longs = work + 2 * n + 1;
  prof_begin(SP2_PROF_SYMM, s);
  SP2_CUDA(cudaMemsetAsync(work, 0, sizeof(int) * (2 * (size_t)n + 1), s));
  const int g = grid_rows_sym(n);
  mirror_count_kernel<T><<<g, kSymThreads, 0, s>>>(view<T>(U), bv, cnt);
  mirror_place_kernel<T><<<g, kSymThreads, 0, s>>>(view<T>(U), outview<T>(Out), bv, cnt, cursor, ctl);
  static_assert(kSortWarpMax <= 256, "the 32-bit key holds 8 position bits");
  if (Out->n < (1 << 24))
    mirror_sort_kernel<T, unsigned><<<g, kSymThreads, 0, s>>>(outview<T>(Out), bv, cnt, rowstat, longs, nlong);
  else
    mirror_sort_kernel<T, unsigned long long>
        <<<g, kSymThreads, 0, s>>>(outview<T>(Out), bv, cnt, rowstat, longs, nlong);
  note_launch();
  note_launch();
  note_launch();
  static_assert(kSortMidMax <= 512, "the 32-bit key holds 9 position bits");
  if (Out->n < (1 << 23))
    mirror_sort_mid_kernel<T, unsigned>
        <<<num_sms() * 2, kSymThreads, 0, s>>>(outview<T>(Out), cnt, rowstat, longs, nlong);
  else
    mirror_sort_mid_kernel<T, unsigned long long>
        <<<num_sms() * 2, kSymThreads, 0, s>>>(outview<T>(Out), cnt, rowstat, longs, nlong);
  note_launch();
  constexpr int smem = kSortCtaMax * (int)(sizeof(int) + sizeof(T));
  static DeviceOnce once;
  SP2_TRY(device_once(once, current_device(), [&](int &) {
    SP2_CUDA(cudaFuncSetAttribute(mirror_sort_long_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    return SP2_OK;
  }));
  mirror_sort_long_kernel<T><<<num_sms(), kSymThreads, smem, s>>>(outview<T>(Out), outview<T>(U), cnt, rowstat, longs,
                                                                   nlong);
  note_launch();
  prof_end(SP2_PROF_SYMM, s);
  SP2_CUDA(cudaGetLastError());
  return SP2_OK;
}

int mirror_async(const ellpack_t *U, ellpack_t *Out, const BatchView &bv, int *work, double2 *rowstat, SpgemmCtl *ctl,
                 cudaStream_t s) {
  return U->dtype == SP2_F64 ? mirror_t<double>(U, Out, bv, work, rowstat, ctl, s)
                             : mirror_t<float>(U, Out, bv, work, rowstat, ctl, s);
}

}  // namespace sp2

namespace sp2 {
namespace {

__device__ __forceinline__ bool same_bits(double a, double b) { return __double_as_longlong(a) == __double_as_longlong(b); }
__device__ __forceinline__ bool same_bits(float a, float b) { return __float_as_int(a) == __float_as_int(b); }

// Counts the entries (r, k, v) of X without a mirror entry (k, r, v) of the same bits.
template <typename T>
__global__ void symmetry_check_kernel(EllView<T> X, int *__restrict__ bad) {
  const int lane = threadIdx.x & 31;
  const int warps = (gridDim.x * blockDim.x) >> 5;
  int nb = 0;
  for (int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < X.n; r += warps) {
    const int nr = min(X.nnz[r], X.w);
    for (int s = lane; s < nr; s += 32) {
      const int k = X.idx[(size_t)r * X.w + s];
      if ((unsigned)k >= (unsigned)X.n) { ++nb; continue; }
      const int *rk = X.idx + (size_t)k * X.w;
      int lo = 0, hi = min(X.nnz[k], X.w);
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (rk[mid] < r) lo = mid + 1; else hi = mid;
      }
      const bool hit = lo < min(X.nnz[k], X.w) && rk[lo] == r;
      if (!hit) { ++nb; continue; }
      if (!same_bits(X.val[(size_t)r * X.w + s], X.val[(size_t)k * X.w + lo])) ++nb;
    }
  }
  for (int o = 16; o > 0; o >>= 1) nb += __shfl_xor_sync(0xffffffffu, nb, o);
  if (lane == 0 && nb) atomicAdd(bad, nb);
}

}  // namespace

int symmetry_defects(const ellpack_t *X, long long *defects, cudaStream_t s) {
  int *d = nullptr;
  SP2_TRY(dev_alloc((void **)&d, sizeof(int), s));
  int h = 0;
  cudaError_t e = cudaMemsetAsync(d, 0, sizeof(int), s);
  if (e == cudaSuccess) {
    const int g = grid_rows_sym(X->n);
    if (X->dtype == SP2_F64) symmetry_check_kernel<double><<<g, kSymThreads, 0, s>>>(view<double>(X), d);
    else symmetry_check_kernel<float><<<g, kSymThreads, 0, s>>>(view<float>(X), d);
    note_launch();
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  dev_free(d, s);
  if (e != cudaSuccess) return cuda_fail(e, "symmetry check", __FILE__, __LINE__);
  *defects = h;
  return SP2_OK;
}

}  // namespace sp2
