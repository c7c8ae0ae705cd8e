// small.cu -- the SP2 loop of a small FP64 matrix (n <= kSmallMaxN rows) in one cooperative
// launch (SP2-Basic of the ExaSP2 proxy, Section "Performance Evaluation using an ExaSP2
// Application"; recursion of Niklasson 2002).
//
// For a small matrix every product takes a few microseconds, so the host-stepped loop of
// sp2_purify is bound by launches and by the one read of the traces per iteration.  Here all
// iterations run in one kernel: each warp owns rows (row r on warp r mod #warps) and builds
// them in a dense accumulator of n values in shared memory; after each product a barrier
// over the grid (hand-written, bounded: a block that waits about a second without the
// others arriving flags the run as timed out and every block returns) lets every block add
// the per-block trace partials in block order, so every block takes the same branch and stop
// decision without a further barrier.
//
// Each product row is the sum over k in the row's order of (alpha x_ik) x_kj, started from
// beta x_ij: the same terms in the same order as the column-block passes and the mirrored
// upper-triangle products, so the rows come out bitwise those of the host-stepped loop; the
// traces are the same values added in another order.
#include <math.h>
#include <string.h>

#include "spgemm_internal.cuh"

namespace sp2 {
namespace {

constexpr int kSmallWarps = 8;
constexpr int kSmallThreads = kSmallWarps * 32;
constexpr int kSmallMaxBlocks = (kSmallMaxN + kSmallWarps - 1) / kSmallWarps;  // the grid never exceeds it
constexpr long long kBarrierSpins = 1ll << 21;  // a pause and an L2 read each: about a second
// Iterates with a row longer than this continue in the host-stepped loop: one warp per row
// holds the first 64 entries of three source rows in registers, and longer rows run into
// dependent loads and the narrow FP64 pipe of one SM, where the column-block passes over all
// SMs do better.
constexpr int kSmallRowMax = 64;

struct SmallPart {
  double tr, fro;
  long long nnz;
  int maxr, pad;
};

struct SmallState {
  unsigned count, gen;  // grid barrier
  int error;            // 1: a barrier timed out
  int it, status;       // status: 0 err < tol, 1 stall rule, 2 max_iter, 3 non-finite trace,
                        // 4 handed to the host-stepped loop (a row above kSmallRowMax entries)
  int final_buf, armed;
  double trX[SP2_STATS_CAP], trX2[SP2_STATS_CAP], err[SP2_STATS_CAP];
  long long nnz[SP2_STATS_CAP];
  int maxr[SP2_STATS_CAP], branch[SP2_STATS_CAP];
};

struct SmallArgs {
  EllOut<double> buf[2];
  int n;
  double nocc, tol, tau, stall_arm, stall_ratio;
  int max_iter, stall_rule;
  SmallPart *part;
  SmallState *st;
};

// Barrier over the (co-resident, cooperative) grid.  Returns false once any block has timed
// out; every write before it is visible to every block after it.
__device__ bool grid_barrier(SmallState *st) {
  __shared__ int s_ok;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned *gen = &st->gen;
    volatile int *error = &st->error;
    const unsigned g = *gen;
    __threadfence();
    if (atomicAdd(&st->count, 1u) == gridDim.x - 1) {
      atomicExch(&st->count, 0u);
      __threadfence();
      atomicAdd(&st->gen, 1u);
    } else {
      long long spins = 0;
      while (*gen == g) {
        if (*error || ++spins > kBarrierSpins) {
          atomicExch(&st->error, 1);
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
    s_ok = *error == 0;
  }
  __syncthreads();
  return s_ok != 0;
}

__global__ void __launch_bounds__(kSmallThreads) sp2_small_kernel(SmallArgs p) {
  extern __shared__ __align__(16) double smem_acc[];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int n = p.n;
  // dense accumulator of the warp's current row: an untouched column holds a signalling-NaN
  // pattern that no arithmetic produces (structural entries are told from exact zeros)
  double *acc = smem_acc + (size_t)wid * n;
  __shared__ double s_tr[kSmallWarps], s_fro[kSmallWarps];
  __shared__ long long s_nnz[kSmallWarps];
  __shared__ int s_max[kSmallWarps];
  __shared__ double s_trX, s_trX2;
  __shared__ int s_stop, s_up;
  __shared__ double s_ptr[kSmallMaxBlocks], s_pfr[kSmallMaxBlocks];
  __shared__ long long s_pnz[kSmallMaxBlocks];
  __shared__ int s_pmx[kSmallMaxBlocks];
  const int gw = blockIdx.x * kSmallWarps + wid, tw = gridDim.x * kSmallWarps;
  const unsigned lt = lanemask_lt();
  const long long tb = mag_bits(p.tau);
  const double none = untouched<double>();
  SmallState *st = p.st;
  for (int c = lane; c < n; c += 32) acc[c] = none;
  __syncwarp();

  // per-block partials of the rows of the new iterate (diagonal, sum of squares, stored
  // entries, longest row), then the grid barrier and the sum of the partials in block order
  double wtr = 0.0, wfro = 0.0;
  long long wnnz = 0;
  int wmax = 0;
  auto finish_stats = [&]() -> bool {
    if (lane == 0) { s_tr[wid] = wtr; s_fro[wid] = wfro; s_nnz[wid] = wnnz; s_max[wid] = wmax; }
    __syncthreads();
    if (threadIdx.x == 0) {
      SmallPart q{0.0, 0.0, 0, 0, 0};
      for (int w = 0; w < kSmallWarps; ++w) {
        q.tr += s_tr[w];
        q.fro += s_fro[w];
        q.nnz += s_nnz[w];
        q.maxr = max(q.maxr, s_max[w]);
      }
      p.part[blockIdx.x] = q;
    }
    if (!grid_barrier(st)) return false;
    // every block's partials into shared memory at once (L2 reads, the L1 may be stale),
    // then added in block order by one thread
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) {
      s_ptr[b] = __ldcg(&p.part[b].tr);
      s_pfr[b] = __ldcg(&p.part[b].fro);
      s_pnz[b] = __ldcg(&p.part[b].nnz);
      s_pmx[b] = __ldcg(&p.part[b].maxr);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double tr = 0.0, fro = 0.0;
      long long nz = 0;
      int mx = 0;
      for (int b = 0; b < (int)gridDim.x; ++b) {
        tr += s_ptr[b];
        fro += s_pfr[b];
        nz += s_pnz[b];
        mx = max(mx, s_pmx[b]);
      }
      s_trX = tr;
      s_trX2 = fro;
      s_nnz[0] = nz;
      s_max[0] = mx;
    }
    __syncthreads();
    wtr = 0.0; wfro = 0.0; wnnz = 0; wmax = 0;
    return true;
  };

  // X0: statistics of the stored rows
  {
    const EllOut<double> X = p.buf[0];
    for (int r = gw; r < n; r += tw) {
      const int k = min(__ldcg(X.nnz + r), X.w);
      double d = 0.0, f = 0.0;
      for (int s = lane; s < k; s += 32) {
        const int j = __ldcg(X.idx + (size_t)r * X.w + s);
        const double v = __ldcg(X.val + (size_t)r * X.w + s);
        if (j == r) d += v;
        f = fma(v, v, f);
      }
      wtr += warp_sum(d);
      wfro += warp_sum(f);
      wnnz += k;
      wmax = max(wmax, k);
    }
  }
  if (!finish_stats()) return;

  int cur = 0;
  bool armed = false;
  double e1 = 0.0, e2 = 0.0;  // err of the two previous iterates (thread 0 of every block)
  for (int it = 0;; ++it) {
    if (threadIdx.x == 0) {
      const double trX = s_trX, trX2 = s_trX2;
      const double err = fabs(trX - trX2) / (double)n;
      int status = -1;
      if (!isfinite(trX) || !isfinite(trX2)) {
        status = 3;
      } else {
        if (fabs(trX - trX2) < p.stall_arm) armed = true;
        const bool stalled = armed && it >= 2 && err >= p.stall_ratio * e2;
        if (err < p.tol) status = 0;
        else if (p.stall_rule && stalled) status = 1;
        else if (it >= p.max_iter) status = 2;
        else if (s_max[0] > kSmallRowMax) status = 4;  // rows this long go to the host-stepped loop
      }
      const bool up = fabs(2.0 * trX - trX2 - p.nocc) < fabs(trX2 - p.nocc);
      if (blockIdx.x == 0) {
        if (it < SP2_STATS_CAP) {
          st->trX[it] = trX;
          st->trX2[it] = trX2;
          st->err[it] = err;
          st->nnz[it] = s_nnz[0];
          st->maxr[it] = s_max[0];
          if (status < 0) st->branch[it] = up ? 2 : 1;
        }
        if (status >= 0) {
          st->it = it;
          st->status = status;
          st->final_buf = cur;
          st->armed = armed ? 1 : 0;
        }
      }
      e2 = e1;
      e1 = err;
      s_stop = status >= 0;
      s_up = up;
    }
    __syncthreads();
    if (s_stop) return;
    const double alpha = s_up ? -1.0 : 1.0, beta = s_up ? 2.0 : 0.0;
    const EllOut<double> X = p.buf[cur], Y = p.buf[cur ^ 1];
    for (int r = gw; r < n; r += tw) {
      const int na = min(__ldcg(X.nnz + r), X.w);
      const int *xi = X.idx + (size_t)r * X.w;
      const double *xv = X.val + (size_t)r * X.w;
      auto update = [&](int j, double a, double v) {
        if ((unsigned)j < (unsigned)n) {
          const double o = acc[j];
          acc[j] = fma(a, v, is_untouched(o) ? 0.0 : o);
        }
      };
      if (beta != 0.0) {  // the addend first: beta x_rj
        for (int s = lane; s < na; s += 32) update(__ldcg(xi + s), beta, __ldcg(xv + s));
        __syncwarp();
      }
      // source rows in the row's order.  Their (k, alpha x_rk, length) are read 32 at a time,
      // one chunk ahead; the first 64 entries of each source row are fetched into registers
      // three steps before they are used (ring j0/j1/j2), so that the steps do not wait on
      // global loads one after the other
      int ck, cnb, nk, nnb;
      double ca, nca;
      auto load_chunk = [&](int cb, int &kk, double &aa, int &nbb) {
        const int t = cb + lane;
        kk = 0; aa = 0.0; nbb = 0;
        if (t < na) {
          const int k = __ldcg(xi + t);
          if ((unsigned)k < (unsigned)n) {
            kk = k;
            aa = alpha * __ldcg(xv + t);
            nbb = min(__ldcg(X.nnz + k), X.w);
          }
        }
      };
      load_chunk(0, ck, ca, cnb);
      load_chunk(32, nk, nca, nnb);
      int cbase = 0;
      auto fetch = [&](int t, int (&jj)[2], double (&vv)[2], int &nb, double &a, size_t &off) {
        int k;
        if (t < cbase + 32) {
          k = __shfl_sync(kFull, ck, t & 31); a = __shfl_sync(kFull, ca, t & 31); nb = __shfl_sync(kFull, cnb, t & 31);
        } else {
          k = __shfl_sync(kFull, nk, t & 31); a = __shfl_sync(kFull, nca, t & 31); nb = __shfl_sync(kFull, nnb, t & 31);
        }
        off = (size_t)k * X.w;
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          const int q = 32 * u + lane;
          jj[u] = q < nb ? __ldcg(X.idx + off + q) : -1;
          vv[u] = q < nb ? __ldcg(X.val + off + q) : 0.0;
        }
      };
      auto apply = [&](const int (&jj)[2], const double (&vv)[2], int nb, double a, size_t off) {
        update(jj[0], a, vv[0]);
        update(jj[1], a, vv[1]);
        for (int q = 64 + lane; q < nb; q += 32) update(__ldcg(X.idx + off + q), a, __ldcg(X.val + off + q));
        __syncwarp();  // a later source row may update the same columns from other lanes
      };
      int j0[2], j1[2], j2[2];
      double v0[2], v1[2], v2[2];
      int nb0 = 0, nb1 = 0, nb2 = 0;
      double a0 = 0.0, a1 = 0.0, a2 = 0.0;
      size_t o0 = 0, o1 = 0, o2 = 0;
      if (na > 0) fetch(0, j0, v0, nb0, a0, o0);
      if (na > 1) fetch(1, j1, v1, nb1, a1, o1);
      for (int t = 0; t < na; t += 3) {
        if (t + 4 >= cbase + 64) {  // the next chunk becomes current: steps t + 2 .. t + 4 stay in reach
          ck = nk; ca = nca; cnb = nnb;
          cbase += 32;
          load_chunk(cbase + 32, nk, nca, nnb);
        }
        if (t + 2 < na) fetch(t + 2, j2, v2, nb2, a2, o2);
        apply(j0, v0, nb0, a0, o0);
        if (t + 1 >= na) break;
        if (t + 3 < na) fetch(t + 3, j0, v0, nb0, a0, o0);
        apply(j1, v1, nb1, a1, o1);
        if (t + 2 >= na) break;
        if (t + 4 < na) fetch(t + 4, j1, v1, nb1, a1, o1);
        apply(j2, v2, nb2, a2, o2);
      }
      // the row in column order: structural entries that pass the drop rule; the
      // accumulator is reset behind the scan
      int cnt = 0;
      double d = 0.0, f = 0.0;
      for (int c0 = 0; c0 < n; c0 += 32) {
        const int c = c0 + lane;
        bool keep = false;
        double v = 0.0;
        if (c < n) {
          v = acc[c];
          if (!is_untouched(v)) {
            acc[c] = none;
            keep = p.tau == 0.0 || mag_bits(v) > tb;
          }
        }
        const unsigned m = __ballot_sync(kFull, keep);
        if (keep) {
          const int pos = cnt + __popc(m & lt);
          if (pos < Y.w) {
            Y.idx[(size_t)r * Y.w + pos] = c;
            Y.val[(size_t)r * Y.w + pos] = v;
          }
          if (c == r) d += v;
          f = fma(v, v, f);
        }
        cnt += __popc(m);
      }
      __syncwarp();
      if (lane == 0) Y.nnz[r] = min(cnt, Y.w);
      wtr += warp_sum(d);
      wfro += warp_sum(f);
      wnnz += cnt;
      wmax = max(wmax, cnt);
    }
    if (!finish_stats()) return;
    cur ^= 1;
  }
}

}  // namespace

int small_purify(ellpack_t *X0, ellpack_t *Y, double nocc, double tol, const sp2_options &opt, int *iterations,
                 int *status, int *final_buf, int *armed, sp2_stats *stats, cudaStream_t s) {
  const int n = X0->n;
  if (n < 1 || n > kSmallMaxN || X0->dtype != SP2_F64 || Y->dtype != SP2_F64 || Y->n != n)
    return fail(SP2E_ARG, "small_purify: bad buffers");
  const size_t smem = (size_t)kSmallWarps * sizeof(double) * (size_t)n;
  static DeviceOnce once;
  const int dev = current_device();
  SP2_TRY(device_once(once, dev, [&](int &) {
    const size_t most = (size_t)kSmallWarps * sizeof(double) * (size_t)kSmallMaxN;
    SP2_CUDA(cudaFuncSetAttribute(sp2_small_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)most));
    return SP2_OK;
  }));
  int occ = 0;
  SP2_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, sp2_small_kernel, kSmallThreads, smem));
  if (occ < 1) {  // nothing ran: the caller takes the host-stepped loop
    *status = 5;
    return SP2_OK;
  }
  const long long need = ((long long)n + kSmallWarps - 1) / kSmallWarps;
  const long long cap = (long long)num_sms() * occ;
  const int grid = (int)(need < cap ? need : cap);

  SmallPart *part = nullptr;
  SmallState *dst = nullptr;
  SP2_TRY(dev_alloc((void **)&part, sizeof(SmallPart) * (size_t)grid, s));
  int rc = dev_alloc((void **)&dst, sizeof(SmallState), s);
  SmallState *h = nullptr;
  if (rc == SP2_OK) {
    h = static_cast<SmallState *>(malloc(sizeof(SmallState)));
    if (!h) rc = fail(SP2E_NOMEM, "small_purify: host record");
  }
  if (rc == SP2_OK) {
    cudaError_t e = cudaMemsetAsync(dst, 0, sizeof(SmallState), s);
    SmallArgs a;
    a.buf[0] = outview<double>(X0);
    a.buf[1] = outview<double>(Y);
    a.n = n;
    a.nocc = nocc;
    a.tol = tol;
    a.tau = opt.tau;
    a.stall_arm = opt.stall_arm;
    a.stall_ratio = opt.stall_ratio;
    a.max_iter = opt.max_iter;
    a.stall_rule = opt.stall_rule;
    a.part = part;
    a.st = dst;
    void *args[] = {&a};
    bool launched = false;
    if (e == cudaSuccess) {
      e = cudaLaunchCooperativeKernel((const void *)sp2_small_kernel, dim3(grid), dim3(kSmallThreads), args, smem, s);
      if (e == cudaErrorCooperativeLaunchTooLarge || e == cudaErrorNotSupported) {
        // a context that cannot host the whole grid at once (shared SMs, no cooperative
        // launch): nothing ran, the caller takes the host-stepped loop
        (void)cudaGetLastError();
        e = cudaSuccess;
        *status = 5;
      } else {
        launched = true;
        note_launch();
      }
    }
    if (launched && e == cudaSuccess) e = cudaMemcpyAsync(h, dst, sizeof(SmallState), cudaMemcpyDeviceToHost, s);
    if (launched && e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) rc = cuda_fail(e, "sp2_small_kernel", __FILE__, __LINE__);
    if (!launched && rc == SP2_OK) {
      free(h);
      dev_free(part, s);
      dev_free(dst, s);
      return SP2_OK;
    }
  }
  if (rc == SP2_OK) {
    if (h->error) {
      rc = fail(SP2E_TIMEOUT, "sp2_purify: a grid barrier of the one-launch loop timed out");
    } else {
      *iterations = h->it;
      *status = h->status;
      *final_buf = h->final_buf;
      *armed = h->armed;
      const int m = h->it + 1 < SP2_STATS_CAP ? h->it + 1 : SP2_STATS_CAP;
      for (int t = 0; t < m; ++t) {
        stats->trX[t] = h->trX[t];
        stats->trX2[t] = h->trX2[t];
        stats->err[t] = h->err[t];
        stats->nnz_total[t] = h->nnz[t];
        stats->max_row_nnz[t] = h->maxr[t];
        if (t < h->it) {
          stats->branch[t] = h->branch[t];
          stats->level[t] = -1;
        }
      }
    }
  }
  free(h);
  dev_free(part, s);
  dev_free(dst, s);
  return rc;
}

}  // namespace sp2
