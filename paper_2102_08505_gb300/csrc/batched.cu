// batched.cu -- many independent SP2 purifications in one device-resident loop.
//
// The matrices of the batch are stacked as one block-diagonal ELLPACK matrix (the
// columns of matrix m are offset by its first row), so one launch of the SpGEMM covers
// every row of every still-active matrix: the per-row matrix id selects that matrix's
// (alpha, beta) and active flag (BatchView).  After each multiply a segmented FP64
// reduction gives every matrix its tr X and ||X||_F^2, and a control kernel (one thread
// per matrix) applies the SP2 stop rules, the branch of the next step and, in mixed
// precision, the FP32 -> FP64 switch, all on the device.  The whole loop is one CUDA
// graph: a conditional WHILE node whose body holds two half-iterations (X -> Y, Y -> X),
// the control kernel of the second half setting the loop condition.  The host launches
// the graph once and reads the results when it ends.
#include <math.h>
#include <string.h>

#include <chrono>
#include <vector>

#include "common.cuh"

namespace sp2 {
namespace {

constexpr int kCap = SP2_STATS_CAP;

struct MatState {
  double nocc;
  int n;         // rows of this matrix
  int it;        // updates applied
  int phase;     // 0 FP32 loop, 1 FP64 (plain run or tail), 2 done
  int armed;
  int status;    // 0 err < tol, 1 stall rule, 2 max_iter
  int fp32_it;
  int final_buf; // 0: X buffers, 1: Y buffers
  int final_dt;  // SP2_F64 / SP2_F32
  int pending;   // 1: convert its FP32 rows to FP64 at the start of the next half
  int branch;    // branch of the last update: 1 X^2, 2 2X - X^2
  int pad;
};

struct Red {  // per-matrix reduction of the last multiply
  double tr, fro;
  long long nnz;
  int max_nnz;
  int pad;
};

struct Control {
  int max_iter, stall_rule, n_tail, mixed;
  double tol, switch_tol;
  int error;        // 1: width overflow (the loop stops, the host regrows); 2: loop bound hit
  int active_count; // matrices still running after the last control kernel
  int halves;       // half-iterations run so far
  int max_halves;   // hard bound on the loop, whatever the per-matrix state says
  double stall_arm; // the stall rule arms once |trX - trX2| < stall_arm
  double stall_ratio; // ... and fires once err_n >= stall_ratio * err_{n-2}
};

struct Stats {
  double *trX, *trX2, *err;
  int *branch;
  long long *nnz;
  int *maxr;
};

// ---------------------------------------------------------------- kernels
__global__ void stack_kernel(const EllView<double> *__restrict__ mats, const int *__restrict__ off,
                             const int *__restrict__ row_mat, int ntot, EllOut<double> S) {
  const int lane = threadIdx.x & 31;
  const int warps = (gridDim.x * blockDim.x) >> 5;
  for (int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < ntot; r += warps) {
    const int m = row_mat[r];
    const EllView<double> H = mats[m];
    const int i = r - off[m];
    const int k = min(min(H.nnz[i], H.w), S.w);
    for (int s = lane; s < k; s += 32) {
      S.idx[(size_t)r * S.w + s] = H.idx[(size_t)i * H.w + s] + off[m];
      S.val[(size_t)r * S.w + s] = H.val[(size_t)i * H.w + s];
    }
    if (lane == 0) S.nnz[r] = k;
  }
}

// Gershgorin bounds of each matrix: one CTA per matrix, rows in a fixed order.
__global__ void seg_gershgorin_kernel(EllView<double> S, const int *__restrict__ off, double *__restrict__ bounds) {
  __shared__ double s_lo[8], s_hi[8];
  const int m = blockIdx.x;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  double lo = INFINITY, hi = -INFINITY;
  for (int r = off[m] + wid; r < off[m + 1]; r += nw) {
    const int k = min(S.nnz[r], S.w);
    double d = 0.0, rad = 0.0;
    for (int s = lane; s < k; s += 32) {
      const double v = S.val[(size_t)r * S.w + s];
      if (S.idx[(size_t)r * S.w + s] == r) d += v; else rad += fabs(v);
    }
    for (int o = 16; o > 0; o >>= 1) {
      d += __shfl_xor_sync(0xffffffffu, d, o);
      rad += __shfl_xor_sync(0xffffffffu, rad, o);
    }
    const double l = d - rad, h = d + rad;
    lo = (isnan(l) || isnan(lo)) ? NAN : fmin(lo, l);
    hi = (isnan(h) || isnan(hi)) ? NAN : fmax(hi, h);
  }
  if (lane == 0) { s_lo[wid] = lo; s_hi[wid] = hi; }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < nw; ++w) {
      lo = (isnan(lo) || isnan(s_lo[w])) ? NAN : fmin(lo, s_lo[w]);
      hi = (isnan(hi) || isnan(s_hi[w])) ? NAN : fmax(hi, s_hi[w]);
    }
    bounds[2 * m] = lo;
    bounds[2 * m + 1] = hi;
  }
}

// X0 = drop_tau((emax I - H)/(emax - emin)) with each row's own matrix bounds; same row
// layout as the single-matrix kernel (entries left of the diagonal, the diagonal, then
// the entries right of it).
__global__ void x0_batched_kernel(EllView<double> H, const int *__restrict__ row_mat, const double *__restrict__ bounds,
                                  double tau, EllOut<double> X) {
  const int lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  const int warps = (gridDim.x * blockDim.x) >> 5;
  for (int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < H.n; r += warps) {
    const int m = row_mat[r];
    const double emin = bounds[2 * m], emax = bounds[2 * m + 1];
    const double inv = 1.0 / (emax - emin);
    const int k = min(H.nnz[r], H.w);
    int n_lo = 0;
    double dval = emax * inv;
    for (int b = 0; b < k; b += 32) {
      const int s = b + lane;
      int j = -1;
      double x = 0.0;
      if (s < k) {
        j = H.idx[(size_t)r * H.w + s];
        const double h = H.val[(size_t)r * H.w + s];
        x = (j == r) ? (emax - h) * inv : -h * inv;
      }
      const unsigned md = __ballot_sync(0xffffffffu, j == r);
      if (md) dval = __shfl_sync(0xffffffffu, x, __ffs(md) - 1);
      const bool keep = (s < k) && j != r && (tau == 0.0 || fabs(x) > tau);
      n_lo += __popc(__ballot_sync(0xffffffffu, keep && j < r));
    }
    const bool keep_diag = (tau == 0.0 || fabs(dval) > tau);
    int lo_pos = 0, hi_pos = n_lo + (keep_diag ? 1 : 0);
    for (int b = 0; b < k; b += 32) {
      const int s = b + lane;
      int j = -1;
      double x = 0.0;
      if (s < k) {
        j = H.idx[(size_t)r * H.w + s];
        x = -H.val[(size_t)r * H.w + s] * inv;
      }
      const bool keep = (s < k) && j != r && (tau == 0.0 || fabs(x) > tau);
      const unsigned mlo = __ballot_sync(0xffffffffu, keep && j < r);
      const unsigned mhi = __ballot_sync(0xffffffffu, keep && j > r);
      if (keep) {
        const int pos = (j < r) ? lo_pos + __popc(mlo & lt) : hi_pos + __popc(mhi & lt);
        X.idx[(size_t)r * X.w + pos] = j;
        X.val[(size_t)r * X.w + pos] = x;
      }
      lo_pos += __popc(mlo);
      hi_pos += __popc(mhi);
    }
    if (lane == 0) {
      if (keep_diag) {
        X.idx[(size_t)r * X.w + n_lo] = r;
        X.val[(size_t)r * X.w + n_lo] = dval;
      }
      X.nnz[r] = hi_pos;
    }
  }
}

// Rows of the matrices whose FP32 loop just ended: FP32 -> FP64 copy (same buffer parity).
__global__ void switch_convert_kernel(EllView<float> a, EllOut<double> b, const int *__restrict__ row_mat,
                                      const MatState *__restrict__ st) {
  const int lane = threadIdx.x & 31;
  const int warps = (gridDim.x * blockDim.x) >> 5;
  for (int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < a.n; r += warps) {
    if (!st[row_mat[r]].pending) continue;
    const int k = min(min(a.nnz[r], a.w), b.w);
    for (int s = lane; s < k; s += 32) {
      b.idx[(size_t)r * b.w + s] = a.idx[(size_t)r * a.w + s];
      b.val[(size_t)r * b.w + s] = (double)a.val[(size_t)r * a.w + s];
    }
    if (lane == 0) b.nnz[r] = k;
  }
}

// Per-matrix sums of the rows updated by the last multiply (fixed order: deterministic).
__global__ void seg_reduce_kernel(const double2 *__restrict__ rowstat, const int *__restrict__ nnz32,
                                  const int *__restrict__ nnz64, const int *__restrict__ off,
                                  const int *__restrict__ act32, const int *__restrict__ act64, Red *__restrict__ red,
                                  int init_all, const MatState *__restrict__ st) {
  __shared__ double s_tr[256], s_fro[256];
  __shared__ long long s_nnz[256];
  __shared__ int s_max[256];
  const int m = blockIdx.x;
  const bool f32 = init_all ? (st[m].phase == 0) : (act32 && act32[m] != 0);
  const bool f64 = init_all ? (st[m].phase == 1) : (act64 && act64[m] != 0);
  if (!f32 && !f64) return;
  const int *nz = f32 ? nnz32 : nnz64;
  double tr = 0.0, fro = 0.0;
  long long tot = 0;
  int mx = 0;
  for (int r = off[m] + threadIdx.x; r < off[m + 1]; r += blockDim.x) {
    const double2 v = rowstat[r];
    tr += v.x;
    fro += v.y;
    tot += nz[r];
    mx = max(mx, nz[r]);
  }
  s_tr[threadIdx.x] = tr;
  s_fro[threadIdx.x] = fro;
  s_nnz[threadIdx.x] = tot;
  s_max[threadIdx.x] = mx;
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h) {
      s_tr[threadIdx.x] += s_tr[threadIdx.x + h];
      s_fro[threadIdx.x] += s_fro[threadIdx.x + h];
      s_nnz[threadIdx.x] += s_nnz[threadIdx.x + h];
      s_max[threadIdx.x] = max(s_max[threadIdx.x], s_max[threadIdx.x + h]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) red[m] = Red{s_tr[0], s_fro[0], s_nnz[0], s_max[0], 0};
}

// One thread per matrix: stop rules, switch and branch (the rules of sp2_purify).
// half < 0: the initial guess was just reduced; half 0 / 1: the multiply of that half.
__global__ void control_kernel(int count, int half, MatState *__restrict__ st, const Red *__restrict__ red,
                               double *__restrict__ a32, double *__restrict__ b32, int *__restrict__ act32,
                               double *__restrict__ a64, double *__restrict__ b64, int *__restrict__ act64,
                               Control *__restrict__ ctl, const SpgemmCtl *__restrict__ c32,
                               const SpgemmCtl *__restrict__ c64, Stats stats, cudaGraphConditionalHandle handle,
                               int set_condition) {
  __shared__ int s_active;
  if (threadIdx.x == 0) {
    s_active = 0;
    if ((c32 && c32->overflow_rows > 0) || (c64 && c64->overflow_rows > 0)) ctl->error = 1;
    if (half >= 0 && ++ctl->halves > ctl->max_halves && !ctl->error) ctl->error = 2;
  }
  __syncthreads();
  for (int m = threadIdx.x; m < count; m += blockDim.x) {
    MatState s = st[m];
    const bool was_active = half < 0 ? s.phase != 2 : ((act32 && act32[m]) || (act64 && act64[m]));
    s.pending = 0;
    if (was_active && !ctl->error) {
      if (half >= 0) s.it += 1;
      const Red rr = red[m];
      const double err = fabs(rr.tr - rr.fro) / (double)s.n;
      const int it = s.it;
      if (it < kCap) {
        stats.trX[(size_t)m * kCap + it] = rr.tr;
        stats.trX2[(size_t)m * kCap + it] = rr.fro;
        stats.err[(size_t)m * kCap + it] = err;
        stats.nnz[(size_t)m * kCap + it] = rr.nnz;
        stats.maxr[(size_t)m * kCap + it] = rr.max_nnz;
      }
      if (half >= 0) {
        s.final_buf = half == 0 ? 1 : 0;  // the buffer this half wrote
        s.final_dt = s.phase == 0 ? SP2_F32 : SP2_F64;
      }
      if (fabs(rr.tr - rr.fro) < ctl->stall_arm) s.armed = 1;
      const bool stalled = s.armed && it >= 2 && it - 2 < kCap && err >= ctl->stall_ratio * stats.err[(size_t)m * kCap + it - 2];
      bool done = false;
      if (!isfinite(rr.tr) || !isfinite(rr.fro)) {
        done = true;
        s.status = 3;
      } else if (s.phase == 0) {
        if (err < ctl->switch_tol || stalled) {
          if (ctl->n_tail > 0) {
            s.phase = 1;
            s.pending = 1;
            s.fp32_it = it;
          } else {
            done = true;
            s.status = err < ctl->tol ? 0 : 1;
          }
        } else if (it >= ctl->max_iter) {
          done = true;
          s.status = 2;
        }
      } else if (ctl->mixed) {
        if (it - s.fp32_it >= ctl->n_tail) {
          if (err < ctl->tol) { done = true; s.status = 0; }
          else if (stalled) { done = true; s.status = 1; }
        }
        if (!done && it >= ctl->max_iter + ctl->n_tail) { done = true; s.status = 2; }
      } else {
        if (err < ctl->tol) { done = true; s.status = 0; }
        else if (ctl->stall_rule && stalled) { done = true; s.status = 1; }
        else if (it >= ctl->max_iter) { done = true; s.status = 2; }
      }
      if (done) s.phase = 2;
      if (act32) act32[m] = 0;
      if (act64) act64[m] = 0;
      if (!done) {
        const bool up = fabs(2.0 * rr.tr - rr.fro - s.nocc) < fabs(rr.fro - s.nocc);
        s.branch = up ? 2 : 1;
        if (it < kCap) stats.branch[(size_t)m * kCap + it] = s.branch;
        if (s.phase == 0) { a32[m] = up ? -1.0 : 1.0; b32[m] = up ? 2.0 : 0.0; act32[m] = 1; }
        else { a64[m] = up ? -1.0 : 1.0; b64[m] = up ? 2.0 : 0.0; act64[m] = 1; }
        atomicAdd(&s_active, 1);
      }
    } else if (!was_active) {
      if (act32) act32[m] = 0;
      if (act64) act64[m] = 0;
    }
    if (ctl->error) {
      if (act32) act32[m] = 0;
      if (act64) act64[m] = 0;
    }
    st[m] = s;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    ctl->active_count = ctl->error ? 0 : s_active;
    if (set_condition) cudaGraphSetConditional(handle, (ctl->error || s_active == 0) ? 0u : 1u);
  }
}

// Final X of each matrix -> its own F64 matrix (columns back to local indices).
template <typename S>
__global__ void unstack_kernel(EllView<S> src, EllOut<double> dst, int first, int wantbuf, int wantdt,
                               const MatState *__restrict__ st, int m, int buf, int dt) {
  if (st[m].final_buf != wantbuf || st[m].final_dt != wantdt) return;
  (void)buf;
  (void)dt;
  const int lane = threadIdx.x & 31;
  const int warps = (gridDim.x * blockDim.x) >> 5;
  for (int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < dst.n; i += warps) {
    const int r = first + i;
    const int k = min(min(src.nnz[r], src.w), dst.w);
    for (int s = lane; s < k; s += 32) {
      dst.idx[(size_t)i * dst.w + s] = src.idx[(size_t)r * src.w + s] - first;
      dst.val[(size_t)i * dst.w + s] = (double)src.val[(size_t)r * src.w + s];
    }
    if (lane == 0) dst.nnz[i] = k;
  }
}

// ---------------------------------------------------------------- host driver
struct DevBuf {
  std::vector<void *> ptrs;
  cudaStream_t s;
  ~DevBuf() {
    for (void *p : ptrs) dev_free(p, s);
  }
  template <typename P>
  int get(P **p, size_t bytes) {
    void *q = nullptr;
    SP2_TRY(dev_alloc(&q, bytes, s));
    ptrs.push_back(q);
    *p = static_cast<P *>(q);
    return SP2_OK;
  }
};

int grid_rows(long long rows) {
  long long b = (rows + 7) / 8;
  long long cap = (long long)num_sms() * 16;
  return (int)(b < 1 ? 1 : (b < cap ? b : cap));
}

}  // namespace
}  // namespace sp2

using namespace sp2;

extern "C" int sp2_purify_batched(const ellpack_t *H, const double *nocc, int32_t count, double tol,
                                  const sp2_options *opt_in, ellpack_t *D, sp2_stats *stats, void *stream) {
  auto t0 = std::chrono::steady_clock::now();
  if (!H || !nocc || !D) return fail(SP2E_ARG, "sp2_purify_batched: null argument");
  if (count < 1) return fail(SP2E_ARG, "sp2_purify_batched: count = %d must be >= 1", count);
  for (int m = 0; m < count; ++m) memset(&D[m], 0, sizeof(ellpack_t));
  sp2_options opt;
  if (opt_in) opt = *opt_in; else sp2_options_default(&opt);
  if (!(tol > 0.0) || !isfinite(tol)) return fail(SP2E_ARG, "sp2_purify_batched: tol must be finite and > 0");
  if (!(opt.tau >= 0.0) || !isfinite(opt.tau)) return fail(SP2E_ARG, "sp2_purify_batched: bad tau");
  if (opt.precision != SP2_PREC_F64 && opt.precision != SP2_PREC_MIXED && opt.precision != SP2_PREC_F32)
    return fail(SP2E_ARG, "sp2_purify_batched: unknown precision %d", opt.precision);
  if (opt.max_iter < 0 || opt.max_iter + opt.n_fp64_tail >= SP2_STATS_CAP || opt.n_fp64_tail < 0)
    return fail(SP2E_ARG, "sp2_purify_batched: bad max_iter / n_fp64_tail");
  if (!(opt.spgemm_path == SP2_PATH_TUNED || (opt.spgemm_path >= 0 && opt.spgemm_path <= 4) ||
        (opt.spgemm_path >= 7 && opt.spgemm_path <= 12)))
    return fail(SP2E_ARG, "sp2_purify_batched: spgemm_path must be -1, 0..4 or 7..12");
  if (!(opt.stall_arm > 0.0) || !isfinite(opt.stall_arm))
    return fail(SP2E_ARG, "sp2_purify_batched: stall_arm must be > 0");
  if (!(opt.stall_ratio > 0.0 && opt.stall_ratio <= 1.0))
    return fail(SP2E_ARG, "sp2_purify_batched: stall_ratio must be in (0, 1]");
  if (opt.route_rows != 0 && opt.route_rows != 1)
    return fail(SP2E_ARG, "sp2_purify_batched: route_rows must be 0 or 1");
  long long ntot_ll = 0;
  int wh = 1, nmax = 0;
  std::vector<int> off(count + 1, 0);
  std::vector<EllView<double>> views(count);
  for (int m = 0; m < count; ++m) {
    SP2_TRY(check_matrix(&H[m], "sp2_purify_batched: H[m]"));
    if (H[m].dtype != SP2_F64) return fail(SP2E_ARG, "sp2_purify_batched: H[%d] must be F64", m);
    if (!(nocc[m] > 0.0) || !(nocc[m] < (double)H[m].n))
      return fail(SP2E_ARG, "sp2_purify_batched: nocc[%d] = %g outside (0, %d)", m, nocc[m], H[m].n);
    off[m] = (int)ntot_ll;
    ntot_ll += H[m].n;
    wh = H[m].width > wh ? H[m].width : wh;
    nmax = H[m].n > nmax ? H[m].n : nmax;
    views[m] = view<double>(&H[m]);
  }
  if (ntot_ll >= (1LL << 31)) return fail(SP2E_ARG, "sp2_purify_batched: too many rows in total");
  const int ntot = (int)ntot_ll;
  off[count] = ntot;
  const bool mixed = opt.precision == SP2_PREC_MIXED;
  const bool f32only = opt.precision == SP2_PREC_F32;
  const bool use32 = mixed || f32only;
  const bool use64 = !f32only;
  const double switch_tol = opt.switch_tol > 0.0 ? opt.switch_tol : (tol > 1e-4 ? tol : 1e-4);

  cudaStream_t user = as_stream(stream);
  cudaStream_t s = user;
  bool own_stream = false;
  if (opt.graph && s == nullptr) {  // the legacy stream cannot be captured
    SP2_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    own_stream = true;
    SP2_CUDA(cudaStreamSynchronize(nullptr));
  }
  struct StreamGuard {
    cudaStream_t s;
    bool own;
    ~StreamGuard() { if (own) { cudaStreamSynchronize(s); cudaStreamDestroy(s); } }
  } sguard{s, own_stream};

  std::vector<int> row_mat_h(ntot);
  for (int m = 0; m < count; ++m)
    for (int r = off[m]; r < off[m + 1]; ++r) row_mat_h[r] = m;
  std::vector<MatState> st_h(count);
  for (int m = 0; m < count; ++m) {
    MatState z;
    memset(&z, 0, sizeof(z));
    z.nocc = nocc[m];
    z.n = H[m].n;
    z.phase = use32 ? 0 : 1;
    z.final_buf = 0;
    z.final_dt = use32 ? SP2_F32 : SP2_F64;
    st_h[m] = z;
  }

  int width = round_up(opt.max_width > 0 ? opt.max_width : (wh + 1) * 8, 32);
  if (width < round_up(wh + 1, 32)) width = round_up(wh + 1, 32);
  if (width > round_up(nmax, 32)) width = round_up(nmax, 32);
  if (width < wh + 1) width = round_up(wh + 1, 32);
  int regrows = 0, tuned_classes = 0;
  long long body_iters = 0;

  for (;;) {  // (re)start with a larger width after an overflow
    DevBuf db{{}, s};
    EllView<double> *d_views = nullptr;
    int *d_off = nullptr, *d_rowmat = nullptr, *d_fb = nullptr;
    double *d_bounds = nullptr, *d_a32 = nullptr, *d_b32 = nullptr, *d_a64 = nullptr, *d_b64 = nullptr;
    int *d_act32 = nullptr, *d_act64 = nullptr;
    MatState *d_st = nullptr;
    Red *d_red = nullptr;
    Control *d_ctl = nullptr;
    SpgemmCtl *d_c32 = nullptr, *d_c64 = nullptr;
    double2 *d_rowstat = nullptr;
    Stats sd{};
    SP2_TRY(db.get(&d_views, sizeof(EllView<double>) * count));
    SP2_TRY(db.get(&d_off, sizeof(int) * (count + 1)));
    SP2_TRY(db.get(&d_rowmat, sizeof(int) * ntot));
    SP2_TRY(db.get(&d_fb, sizeof(int) * 3 * (size_t)ntot));
    SP2_TRY(db.get(&d_bounds, sizeof(double) * 2 * count));
    SP2_TRY(db.get(&d_a32, sizeof(double) * count));
    SP2_TRY(db.get(&d_b32, sizeof(double) * count));
    SP2_TRY(db.get(&d_a64, sizeof(double) * count));
    SP2_TRY(db.get(&d_b64, sizeof(double) * count));
    SP2_TRY(db.get(&d_act32, sizeof(int) * count));
    SP2_TRY(db.get(&d_act64, sizeof(int) * count));
    SP2_TRY(db.get(&d_st, sizeof(MatState) * count));
    SP2_TRY(db.get(&d_red, sizeof(Red) * count));
    SP2_TRY(db.get(&d_ctl, sizeof(Control)));
    SP2_TRY(db.get(&d_c32, sizeof(SpgemmCtl)));
    SP2_TRY(db.get(&d_c64, sizeof(SpgemmCtl)));
    SP2_TRY(db.get(&d_rowstat, sizeof(double2) * (size_t)ntot));
    // scratch of the symmetric products, allocated here: nothing allocates inside the loop
    unsigned char *d_sym = nullptr;
    const size_t sym_bytes = opt.symmetric ? sym_scratch_bytes(ntot, width, width, SP2_F64) : 0;
    if (opt.symmetric) SP2_TRY(db.get(&d_sym, sym_bytes));
    // The symmetric products run the cascade of first passes from the tight compact level:
    // each row finds its level inside the captured loop, which takes no feedback from the
    // host.  Route flags (route_rows 1), one set per precision, start a row at the level it
    // needed last time.
    unsigned char *d_route32 = nullptr, *d_route64 = nullptr;
    if (opt.route_rows && use32) SP2_TRY(db.get(&d_route32, (size_t)ntot));
    if (opt.route_rows && use64) SP2_TRY(db.get(&d_route64, (size_t)ntot));
    if (d_route32) SP2_CUDA(cudaMemsetAsync(d_route32, 0, (size_t)ntot, s));
    if (d_route64) SP2_CUDA(cudaMemsetAsync(d_route64, 0, (size_t)ntot, s));
    const int level = 0;
    SP2_TRY(db.get(&sd.trX, sizeof(double) * (size_t)count * kCap));
    SP2_TRY(db.get(&sd.trX2, sizeof(double) * (size_t)count * kCap));
    SP2_TRY(db.get(&sd.err, sizeof(double) * (size_t)count * kCap));
    SP2_TRY(db.get(&sd.branch, sizeof(int) * (size_t)count * kCap));
    SP2_TRY(db.get(&sd.nnz, sizeof(long long) * (size_t)count * kCap));
    SP2_TRY(db.get(&sd.maxr, sizeof(int) * (size_t)count * kCap));
    SP2_CUDA(cudaMemcpyAsync(d_views, views.data(), sizeof(EllView<double>) * count, cudaMemcpyHostToDevice, s));
    SP2_CUDA(cudaMemcpyAsync(d_off, off.data(), sizeof(int) * (count + 1), cudaMemcpyHostToDevice, s));
    SP2_CUDA(cudaMemcpyAsync(d_rowmat, row_mat_h.data(), sizeof(int) * ntot, cudaMemcpyHostToDevice, s));
    SP2_CUDA(cudaMemcpyAsync(d_st, st_h.data(), sizeof(MatState) * count, cudaMemcpyHostToDevice, s));
    SP2_CUDA(cudaMemsetAsync(d_act32, 0, sizeof(int) * count, s));
    SP2_CUDA(cudaMemsetAsync(d_act64, 0, sizeof(int) * count, s));
    SP2_CUDA(cudaMemsetAsync(sd.branch, 0, sizeof(int) * (size_t)count * kCap, s));
    Control ch{opt.max_iter, opt.stall_rule, mixed ? opt.n_fp64_tail : 0, mixed ? 1 : 0, tol, switch_tol, 0, 0, 0,
               2 * (opt.max_iter + opt.n_fp64_tail + 8), opt.stall_arm, opt.stall_ratio};
    SP2_CUDA(cudaMemcpyAsync(d_ctl, &ch, sizeof(ch), cudaMemcpyHostToDevice, s));
    SP2_CUDA(cudaMemsetAsync(d_c32, 0, sizeof(SpgemmCtl), s));
    SP2_CUDA(cudaMemsetAsync(d_c64, 0, sizeof(SpgemmCtl), s));

    ellpack_t Hs{}, X64{}, Y64{}, X32{}, Y32{};
    struct Mats {
      ellpack_t *m[5];
      cudaStream_t s;
      ~Mats() {
        for (auto *p : m)
          if (p && p->owner) ellpack_destroy(p, s);
      }
    } mats{{&Hs, &X64, &Y64, &X32, &Y32}, s};
    SP2_TRY(ellpack_create(ntot, wh, SP2_F64, s, &Hs));
    SP2_TRY(ellpack_create(ntot, width, SP2_F64, s, &X64));
    SP2_TRY(ellpack_create(ntot, width, SP2_F64, s, &Y64));
    if (use32) {
      SP2_TRY(ellpack_create(ntot, width, SP2_F32, s, &X32));
      SP2_TRY(ellpack_create(ntot, width, SP2_F32, s, &Y32));
    }
    // a1, a2: stack, bounds per matrix, X0
    stack_kernel<<<grid_rows(ntot), 256, 0, s>>>(d_views, d_off, d_rowmat, ntot, outview<double>(&Hs));
    note_launch();
    seg_gershgorin_kernel<<<count, 256, 0, s>>>(view<double>(&Hs), d_off, d_bounds);
    note_launch();
    std::vector<double> hb(2 * count);
    SP2_CUDA(cudaMemcpyAsync(hb.data(), d_bounds, sizeof(double) * 2 * count, cudaMemcpyDeviceToHost, s));
    SP2_CUDA(cudaStreamSynchronize(s));
    for (int m = 0; m < count; ++m) {
      if (!isfinite(hb[2 * m]) || !isfinite(hb[2 * m + 1])) return fail(SP2E_NONFINITE, "sp2_purify_batched: H[%d] holds a NaN or Inf", m);
      if (!(hb[2 * m + 1] > hb[2 * m])) return fail(SP2E_ARG, "sp2_purify_batched: H[%d] has degenerate bounds", m);
    }
    x0_batched_kernel<<<grid_rows(ntot), 256, 0, s>>>(view<double>(&Hs), d_rowmat, d_bounds, opt.tau,
                                                       outview<double>(&X64));
    note_launch();
    if (opt.symmetric) {  // the upper-triangle products need exactly symmetric matrices
      long long defects = 0;
      SP2_TRY(symmetry_defects(&Hs, &defects, s));
      if (defects)
        return fail(SP2E_ARG, "sp2_purify_batched: some H is not exactly symmetric (%lld entries without a mirror); "
                              "use symmetric = 0", defects);
    }
    if (use32) SP2_TRY(convert_async(&X64, &X32, s));
    // a3 for X0, then the first branch decisions
    SP2_TRY(rowstat_async(use32 ? &X32 : &X64, d_rowstat, s));
    seg_reduce_kernel<<<count, 256, 0, s>>>(d_rowstat, X32.nnz, X64.nnz, d_off, nullptr, nullptr, d_red, 1, d_st);
    note_launch();
    control_kernel<<<1, 256, 0, s>>>(count, -1, d_st, d_red, d_a32, d_b32, d_act32, d_a64, d_b64, d_act64, d_ctl,
                                     nullptr, nullptr, sd, 0, 0);
    note_launch();
    SP2_CUDA(cudaGetLastError());
    // the fallback scratch is sized before any capture (it may reallocate)
    {
      void *acc = nullptr;
      int *mark = nullptr;
      SP2_TRY(fallback_scratch(ntot, SP2_F64, ntot < 64 ? ntot : 64, &acc, &mark, s));
    }

    // SpGEMM variants: fixed, or the tuner's choice for the stacked product's class.  The
    // loop is captured once, so the classes are those of X0 * X0 (tuned here, before the
    // capture, if new; the products written meanwhile are recomputed by the loop).
    int path32 = opt.spgemm_path, path64 = opt.spgemm_path;
    if (opt.spgemm_path == SP2_PATH_TUNED) {
      double mean = 0.0;
      SP2_TRY(mean_row_nnz(&X64, &mean, s));
      auto pick = [&](ellpack_t *cur, ellpack_t *nxt, SpgemmCtl *c, int *path) -> int {
        if (tune_find(cur->dtype, ntot, mean, path)) return SP2_OK;
        MultiplyArgs a{cur, cur, nullptr, nxt, 1.0, 0.0, opt.tau, 0};
        a.sym = opt.symmetric != 0;
        a.compact_level = level;
        a.sym_prealloc = d_sym;
        a.sym_prealloc_bytes = sym_bytes;
        SP2_TRY(tune_multiply(a, mean, d_rowstat, c, 2, path, nullptr, s));
        ++tuned_classes;
        return SP2_OK;
      };
      if (use32) SP2_TRY(pick(&X32, &Y32, d_c32, &path32));
      if (use64) SP2_TRY(pick(&X64, &Y64, d_c64, &path64));
    }
    BatchView bv32{d_rowmat, d_a32, d_b32, d_act32};
    BatchView bv64{d_rowmat, d_a64, d_b64, d_act64};
    auto half = [&](int h, cudaGraphConditionalHandle handle, int set_cond) -> int {
      ellpack_t *cur32 = h == 0 ? &X32 : &Y32, *nxt32 = h == 0 ? &Y32 : &X32;
      ellpack_t *cur64 = h == 0 ? &X64 : &Y64, *nxt64 = h == 0 ? &Y64 : &X64;
      if (mixed) {
        switch_convert_kernel<<<grid_rows(ntot), 256, 0, s>>>(view<float>(cur32), outview<double>(cur64), d_rowmat, d_st);
        note_launch();
      }
      if (use32) {
        MultiplyArgs a{cur32, cur32, cur32, nxt32, 1.0, 0.0, opt.tau, path32};
        a.bv = bv32;
        a.fb_prealloc = d_fb;
        a.sym = opt.symmetric != 0;
        a.compact_level = level;
        if (path32 == 0) a.route = d_route32;
        a.sym_prealloc = d_sym;
        a.sym_prealloc_bytes = sym_bytes;
        SP2_TRY(multiply_async(a, d_rowstat, d_c32, s));
      }
      if (use64) {
        MultiplyArgs a{cur64, cur64, cur64, nxt64, 1.0, 0.0, opt.tau, path64};
        a.bv = bv64;
        a.fb_prealloc = d_fb;
        a.sym = opt.symmetric != 0;
        a.compact_level = level;
        if (path64 == 0) a.route = d_route64;
        a.sym_prealloc = d_sym;
        a.sym_prealloc_bytes = sym_bytes;
        SP2_TRY(multiply_async(a, d_rowstat, d_c64, s));
      }
      seg_reduce_kernel<<<count, 256, 0, s>>>(d_rowstat, use32 ? nxt32->nnz : nullptr, use64 ? nxt64->nnz : nullptr,
                                              d_off, use32 ? d_act32 : nullptr, use64 ? d_act64 : nullptr, d_red, 0,
                                              d_st);
      note_launch();
      control_kernel<<<1, 256, 0, s>>>(count, h, d_st, d_red, d_a32, d_b32, use32 ? d_act32 : nullptr, d_a64, d_b64,
                                       use64 ? d_act64 : nullptr, d_ctl, use32 ? d_c32 : nullptr,
                                       use64 ? d_c64 : nullptr, sd, handle, set_cond);
      note_launch();
      SP2_CUDA(cudaGetLastError());
      return SP2_OK;
    };

    if (opt.graph) {
      cudaGraph_t graph = nullptr;
      cudaGraphExec_t exec = nullptr;
      SP2_CUDA(cudaGraphCreate(&graph, 0));
      struct GraphGuard {
        cudaGraph_t *g;
        cudaGraphExec_t *e;
        ~GraphGuard() {
          if (*e) cudaGraphExecDestroy(*e);
          if (*g) cudaGraphDestroy(*g);
        }
      } gg{&graph, &exec};
      cudaGraphConditionalHandle handle;
      SP2_CUDA(cudaGraphConditionalHandleCreate(&handle, graph, 1, cudaGraphCondAssignDefault));
      cudaGraphNodeParams cp = {cudaGraphNodeTypeConditional};
      cp.conditional.handle = handle;
      cp.conditional.type = cudaGraphCondTypeWhile;
      cp.conditional.size = 1;
      cudaGraphNode_t node;
      SP2_CUDA(cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &cp));
      cudaGraph_t body = cp.conditional.phGraph_out[0];
      // kernels configured outside capture once (attributes, occupancy): run a half with
      // every matrix inactive is not possible here (the state is live), so configure by
      // capturing: the launch helpers only record launches and memsets into the body
      SP2_CUDA(cudaStreamBeginCaptureToGraph(s, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
      int rc = half(0, handle, 0);
      if (rc == SP2_OK) rc = half(1, handle, 1);
      cudaGraph_t captured = nullptr;
      cudaError_t ec = cudaStreamEndCapture(s, &captured);
      SP2_TRY(rc);
      if (ec != cudaSuccess) return cuda_fail(ec, "sp2_purify_batched: capture", __FILE__, __LINE__);
      SP2_CUDA(cudaGraphInstantiate(&exec, graph, 0));
      SP2_CUDA(cudaGraphLaunch(exec, s));
      SP2_CUDA(cudaStreamSynchronize(s));
    } else {
      for (int guard = 0; guard < 2 * (opt.max_iter + opt.n_fp64_tail + 8) + 2; ++guard) {
        SP2_TRY(half(guard & 1, 0, 0));
        Control c;
        SP2_CUDA(cudaMemcpyAsync(&c, d_ctl, sizeof(c), cudaMemcpyDeviceToHost, s));
        SP2_CUDA(cudaStreamSynchronize(s));
        ++body_iters;
        if (c.error || c.active_count == 0) break;
      }
    }
    Control cend;
    SP2_CUDA(cudaMemcpyAsync(&cend, d_ctl, sizeof(cend), cudaMemcpyDeviceToHost, s));
    std::vector<MatState> st_out(count);
    SP2_CUDA(cudaMemcpyAsync(st_out.data(), d_st, sizeof(MatState) * count, cudaMemcpyDeviceToHost, s));
    SP2_CUDA(cudaStreamSynchronize(s));
    if (cend.error == 2) return fail(SP2E_TIMEOUT, "sp2_purify_batched: loop bound of %d half-iterations reached", cend.max_halves);
    if (cend.error) {  // a row outgrew the width: start again wider
      if (width >= round_up(nmax, 32)) return fail(SP2E_OVERFLOW, "sp2_purify_batched: width overflow at %d", width);
      width = round_up(width + width / 2, 32);
      if (width > round_up(nmax, 32)) width = round_up(nmax, 32);
      ++regrows;
      continue;
    }
    // outputs
    int worst = SP2_OK;
    for (int m = 0; m < count; ++m) {
      const int n = off[m + 1] - off[m];
      SP2_TRY(ellpack_create(n, width, SP2_F64, s, &D[m]));
      const int g = grid_rows(n);
      unstack_kernel<double><<<g, 256, 0, s>>>(view<double>(&X64), outview<double>(&D[m]), off[m], 0, SP2_F64, d_st, m, 0, 0);
      unstack_kernel<double><<<g, 256, 0, s>>>(view<double>(&Y64), outview<double>(&D[m]), off[m], 1, SP2_F64, d_st, m, 0, 0);
      if (use32) {
        unstack_kernel<float><<<g, 256, 0, s>>>(view<float>(&X32), outview<double>(&D[m]), off[m], 0, SP2_F32, d_st, m, 0, 0);
        unstack_kernel<float><<<g, 256, 0, s>>>(view<float>(&Y32), outview<double>(&D[m]), off[m], 1, SP2_F32, d_st, m, 0, 0);
      }
      note_launch();
      if (st_out[m].status == 2 && worst == SP2_OK) worst = SP2E_NOTCONV;
      if (st_out[m].status == 3) worst = SP2E_NONFINITE;
    }
    SP2_CUDA(cudaGetLastError());
    if (stats) {
      std::vector<double> trX((size_t)count * kCap), trX2((size_t)count * kCap), er((size_t)count * kCap);
      std::vector<int> br((size_t)count * kCap), mr((size_t)count * kCap);
      std::vector<long long> nz((size_t)count * kCap);
      SP2_CUDA(cudaMemcpyAsync(trX.data(), sd.trX, sizeof(double) * trX.size(), cudaMemcpyDeviceToHost, s));
      SP2_CUDA(cudaMemcpyAsync(trX2.data(), sd.trX2, sizeof(double) * trX2.size(), cudaMemcpyDeviceToHost, s));
      SP2_CUDA(cudaMemcpyAsync(er.data(), sd.err, sizeof(double) * er.size(), cudaMemcpyDeviceToHost, s));
      SP2_CUDA(cudaMemcpyAsync(br.data(), sd.branch, sizeof(int) * br.size(), cudaMemcpyDeviceToHost, s));
      SP2_CUDA(cudaMemcpyAsync(mr.data(), sd.maxr, sizeof(int) * mr.size(), cudaMemcpyDeviceToHost, s));
      SP2_CUDA(cudaMemcpyAsync(nz.data(), sd.nnz, sizeof(long long) * nz.size(), cudaMemcpyDeviceToHost, s));
      SP2_CUDA(cudaStreamSynchronize(s));
      const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
      for (int m = 0; m < count; ++m) {
        sp2_stats &o = stats[m];
        memset(&o, 0, sizeof(o));
        o.iterations = st_out[m].it;
        o.status = st_out[m].status;
        o.fp32_iterations = use32 ? (mixed && st_out[m].fp32_it > 0 ? st_out[m].fp32_it : (f32only ? st_out[m].it : 0)) : 0;
        o.regrows = regrows;
        o.tuned = tuned_classes;
        o.emin = hb[2 * m];
        o.emax = hb[2 * m + 1];
        o.time_ms = ms;
        for (int t = 0; t < kCap; ++t) {
          o.trX[t] = trX[(size_t)m * kCap + t];
          o.trX2[t] = trX2[(size_t)m * kCap + t];
          o.err[t] = er[(size_t)m * kCap + t];
          o.branch[t] = br[(size_t)m * kCap + t];
          o.nnz_total[t] = nz[(size_t)m * kCap + t];
          o.max_row_nnz[t] = mr[(size_t)m * kCap + t];
          // the products of the batch are shared: no per-matrix deferral counts
          o.level[t] = t < o.iterations ? (opt.symmetric && opt.spgemm_path == 0 ? cascade_start(ntot, true, level) : -1)
                                        : 0;
        }
      }
    }
    SP2_CUDA(cudaStreamSynchronize(s));
    if (worst == SP2E_NOTCONV) return fail(SP2E_NOTCONV, "sp2_purify_batched: a matrix reached max_iter");
    if (worst == SP2E_NONFINITE) return fail(SP2E_NONFINITE, "sp2_purify_batched: non-finite traces");
    return SP2_OK;
  }
}
