// sp2.cu -- host-stepped SP2 purification (SP2-Basic of the ExaSP2 proxy, Section
// "Performance Evaluation using an ExaSP2 Application"; recursion of Niklasson 2002).
//
// Per iteration the device does one fused pass: X' = drop_tau(alpha X*X + beta X) with
// (alpha, beta) = (1, 0) for X^2 and (-1, 2) for 2X - X^2, whose epilogue also leaves
// each row's diagonal value and sum of squares; one CTA reduces those in a fixed order
// to tr X' and ||X'||_F^2 = tr X'^2 (X' symmetric).  The host reads that 56-byte result
// once per iteration (the stop test and the branch of the next step need it) and
// launches the next step.  Mixed precision runs the same loop on FP32 values with FP64
// reductions, then converts X to FP64 and runs the FP64 tail iterations.
#include <math.h>
#include <string.h>

#include <chrono>

#include "common.cuh"

namespace sp2 {
namespace {

struct Buffers {
  cudaStream_t s;
  double2 *rowstat = nullptr;
  SpgemmCtl *ctl = nullptr;
  StepResult *dres = nullptr;
  double *bounds = nullptr;
  void *sizing = nullptr;  // counts, maxima, features, predictions (sizing modes 1 and 2)
  unsigned char *route = nullptr;  // per-row route flags of the first pass (route_rows 1)
  ellpack_t X{}, Y{}, Hf{};
  bool hf_owned = false;
  ~Buffers() {
    dev_free(rowstat, s);
    dev_free(ctl, s);
    dev_free(dres, s);
    dev_free(bounds, s);
    dev_free(sizing, s);
    dev_free(route, s);
    if (X.owner) ellpack_destroy(&X, s);
    if (Y.owner) ellpack_destroy(&Y, s);
    if (hf_owned) ellpack_destroy(&Hf, s);
  }
};

int read_result(Buffers &b, StepResult *h) {
  SP2_CUDA(cudaMemcpyAsync(h, b.dres, sizeof(StepResult), cudaMemcpyDeviceToHost, b.s));
  SP2_CUDA(cudaStreamSynchronize(b.s));
  return SP2_OK;
}

// (Re)allocates m with at least `width` slots and the given dtype; contents undefined.
bool valid_path(int p) { return p == SP2_PATH_TUNED || (p >= 0 && p <= 4) || (p >= 7 && p <= 12); }

int ensure(ellpack_t *m, int n, int width, int dtype, cudaStream_t s) {
  if (m->owner && m->width >= width && m->dtype == dtype) return SP2_OK;
  if (m->owner) SP2_TRY(ellpack_destroy(m, s));
  return ellpack_create(n, width, dtype, s, m);
}


}  // namespace
}  // namespace sp2

using namespace sp2;

extern "C" void sp2_options_default(sp2_options *o) {
  if (!o) return;
  memset(o, 0, sizeof(*o));
  o->precision = SP2_PREC_F64;
  o->max_iter = 100;
  o->stall_rule = 1;
  o->n_fp64_tail = 2;
  o->max_width = 0;
  o->spgemm_path = 0;
  o->tau = 1e-5;
  o->switch_tol = 0.0;
  o->graph = 1;
  o->sizing = 0;
  o->predictor = nullptr;
  o->stall_arm = 0.1;
  o->stall_ratio = 1.0;
  o->symmetric = 1;
  o->route_rows = 1;
  o->small_path = 1;
  o->level_up_frac = 1.0;
}

extern "C" int sp2_purify(const ellpack_t *H, double nocc, double tol, const sp2_options *opt_in, ellpack_t *D,
                          sp2_stats *stats, void *stream) {
  auto t0 = std::chrono::steady_clock::now();
  SP2_TRY(check_matrix(H, "sp2_purify: H"));
  if (!D) return fail(SP2E_ARG, "sp2_purify: D is NULL");
  memset(D, 0, sizeof(*D));
  sp2_options opt;
  if (opt_in) opt = *opt_in; else sp2_options_default(&opt);
  const int n = H->n;
  if (!(nocc > 0.0) || !(nocc < (double)n)) return fail(SP2E_ARG, "sp2_purify: nocc=%g must lie in (0, %d)", nocc, n);
  if (!(tol > 0.0) || !isfinite(tol)) return fail(SP2E_ARG, "sp2_purify: tol must be finite and > 0");
  if (!(opt.tau >= 0.0) || !isfinite(opt.tau)) return fail(SP2E_ARG, "sp2_purify: tau must be finite and >= 0");
  if (opt.precision != SP2_PREC_F64 && opt.precision != SP2_PREC_MIXED && opt.precision != SP2_PREC_F32)
    return fail(SP2E_ARG, "sp2_purify: unknown precision %d", opt.precision);
  if (opt.precision == SP2_PREC_F32) {  // the FP32 loop alone
    opt.precision = SP2_PREC_MIXED;
    opt.n_fp64_tail = 0;
  }
  if (opt.max_iter < 0 || opt.max_iter + opt.n_fp64_tail >= SP2_STATS_CAP)
    return fail(SP2E_ARG, "sp2_purify: max_iter + n_fp64_tail must be < %d", SP2_STATS_CAP);
  if (opt.n_fp64_tail < 0) return fail(SP2E_ARG, "sp2_purify: n_fp64_tail < 0");
  if (!valid_path(opt.spgemm_path)) return fail(SP2E_ARG, "sp2_purify: spgemm_path must be -1, 0..4 or 7..12");
  const int max_w = (opt.max_width > 0 && opt.max_width < n) ? opt.max_width : n;
  if (!(opt.switch_tol >= 0.0) || !isfinite(opt.switch_tol)) return fail(SP2E_ARG, "sp2_purify: bad switch_tol");
  if (opt.sizing < 0 || opt.sizing > 2) return fail(SP2E_ARG, "sp2_purify: sizing must be 0, 1 or 2");
  if (!(opt.stall_arm > 0.0) || !isfinite(opt.stall_arm)) return fail(SP2E_ARG, "sp2_purify: stall_arm must be > 0");
  if (!(opt.stall_ratio > 0.0 && opt.stall_ratio <= 1.0))
    return fail(SP2E_ARG, "sp2_purify: stall_ratio must be in (0, 1]");
  if (opt.route_rows != 0 && opt.route_rows != 1) return fail(SP2E_ARG, "sp2_purify: route_rows must be 0 or 1");
  if (opt.small_path != 0 && opt.small_path != 1) return fail(SP2E_ARG, "sp2_purify: small_path must be 0 or 1");
  if (!(opt.level_up_frac > 0.0) || !isfinite(opt.level_up_frac))
    return fail(SP2E_ARG, "sp2_purify: level_up_frac must be finite and > 0");
  if (opt.sizing == 2 && (!opt.predictor || !opt.predictor->params))
    return fail(SP2E_ARG, "sp2_purify: sizing 2 needs a created predictor");
  const double switch_tol = opt.switch_tol > 0.0 ? opt.switch_tol : (tol > 1e-4 ? tol : 1e-4);

  Buffers b;
  b.s = as_stream(stream);
  cudaStream_t s = b.s;
  sp2_stats st;
  memset(&st, 0, sizeof(st));
  if (stats) memset(stats, 0, sizeof(*stats));

  SP2_TRY(dev_alloc((void **)&b.rowstat, sizeof(double2) * (size_t)n, s));
  SP2_TRY(dev_alloc((void **)&b.ctl, sizeof(SpgemmCtl), s));
  SP2_TRY(dev_alloc((void **)&b.dres, sizeof(StepResult), s));
  SP2_TRY(dev_alloc((void **)&b.bounds, 2 * sizeof(double), s));
  if (opt.route_rows) {
    SP2_TRY(dev_alloc((void **)&b.route, (size_t)n, s));
    SP2_CUDA(cudaMemsetAsync(b.route, 0, (size_t)n, s));
  }
  // sizing scratch: max int, max float, counts int[n], rmax float[n], pred float[n],
  // features float[16n], then the prediction-error sums (kPredErrDoubles doubles)
  int *sz_counts = nullptr, *sz_dmax = nullptr;
  double *sz_perr = nullptr;
  float *sz_fmax = nullptr, *sz_rmax = nullptr, *sz_pred = nullptr, *sz_feat = nullptr;
  if (opt.sizing) {
    const size_t off_perr = round_up_sz(16 + sizeof(int) * (size_t)n + sizeof(float) * (size_t)n * 18, 16);
    const size_t bytes = off_perr + sizeof(double) * kPredErrDoubles;
    SP2_TRY(dev_alloc(&b.sizing, bytes, s));
    unsigned char *q = static_cast<unsigned char *>(b.sizing);
    sz_dmax = reinterpret_cast<int *>(q);
    sz_fmax = reinterpret_cast<float *>(q + 8);
    sz_counts = reinterpret_cast<int *>(q + 16);
    sz_rmax = reinterpret_cast<float *>(q + 16 + sizeof(int) * (size_t)n);
    sz_pred = sz_rmax + n;
    sz_feat = sz_pred + n;
    sz_perr = reinterpret_cast<double *>(q + off_perr);
  }
  double mae_sum = 0.0, under_sum = 0.0, rows_seen = 0.0;
  auto exact_width = [&](const ellpack_t *X, bool up, int *w) -> int {
    SP2_TRY(struct_count_async(X, X, up ? X : nullptr, sz_counts, sz_dmax, s));
    int h = 0;
    SP2_CUDA(cudaMemcpyAsync(&h, sz_dmax, sizeof(int), cudaMemcpyDeviceToHost, s));
    SP2_CUDA(cudaStreamSynchronize(s));
    *w = h < 1 ? 1 : h;
    return SP2_OK;
  };

  // F64 copy of H if needed
  const ellpack_t *H64 = H;
  if (H->dtype != SP2_F64) {
    SP2_TRY(ellpack_create(n, H->width, SP2_F64, s, &b.Hf));
    b.hf_owned = true;
    SP2_TRY(convert_async(H, &b.Hf, s));
    H64 = &b.Hf;
  }

  // a1: Gershgorin bounds (read back once: validated and reported)
  SP2_TRY(gershgorin_async(H64, b.bounds, s));
  double hb[2];
  SP2_CUDA(cudaMemcpyAsync(hb, b.bounds, sizeof(hb), cudaMemcpyDeviceToHost, s));
  SP2_CUDA(cudaStreamSynchronize(s));
  st.emin = hb[0];
  st.emax = hb[1];
  if (!isfinite(hb[0]) || !isfinite(hb[1])) return fail(SP2E_NONFINITE, "sp2_purify: H holds a NaN or Inf");
  if (!(hb[1] > hb[0])) return fail(SP2E_ARG, "sp2_purify: degenerate spectral bounds (e_max <= e_min)");

  if (opt.symmetric) {  // the upper-triangle products need an exactly symmetric H
    long long defects = 0;
    SP2_TRY(symmetry_defects(H64, &defects, s));
    if (defects) return fail(SP2E_ARG, "sp2_purify: H is not exactly symmetric (%lld entries without a mirror); "
                                       "use symmetric = 0", defects);
  }

  // a2..a7 for a small FP64 matrix: X0 here, then the loop in one cooperative launch, for as
  // long as the iterates' rows stay short; the host-stepped loop below takes over after that
  bool handed = false;
  int it0 = 0;
  bool armed0 = false;
  StepResult res{};
  if (opt.small_path && opt.precision == SP2_PREC_F64 && opt.spgemm_path == 0 && opt.sizing == 0 &&
      n <= kSmallMaxN && max_w >= n) {
    const int w = n > H64->width + 1 ? n : H64->width + 1;  // every product row fits
    SP2_TRY(ellpack_create(n, w, SP2_F64, s, &b.X));
    SP2_TRY(x0_async(H64, b.bounds, opt.tau, &b.X, s));
    SP2_TRY(ellpack_create(n, w, SP2_F64, s, &b.Y));
    int iters = 0, status = 0, fbuf = 0, arm = 0;
    const int rc = small_purify(&b.X, &b.Y, nocc, tol, opt, &iters, &status, &fbuf, &arm, &st, s);
    if (status == 5 && rc == SP2_OK) {  // not launched: the host-stepped loop from X0
      SP2_TRY(ellpack_destroy(&b.X, s));
      SP2_TRY(ellpack_destroy(&b.Y, s));
      memset(&b.X, 0, sizeof(b.X));
      memset(&b.Y, 0, sizeof(b.Y));
    } else if (status == 4 && rc == SP2_OK) {  // the host-stepped loop continues from iterate iters
      if (fbuf) { ellpack_t t = b.X; b.X = b.Y; b.Y = t; }
      handed = true;
      it0 = iters;
      armed0 = arm != 0;
      res.tr = st.trX[iters];
      res.fro = st.trX2[iters];
      res.nnz_total = st.nnz_total[iters];
      res.max_nnz = st.max_row_nnz[iters];
      res.max_count = res.max_nnz;
      st.small_iterations = iters;
    } else {
      st.iterations = iters;
      st.small_iterations = iters;
      st.status = status == 3 ? 0 : status;
      st.width_max = w;
      st.time_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
      if (stats) *stats = st;
      if (rc != SP2_OK) return rc;
      if (status == 3) return fail(SP2E_NONFINITE, "sp2_purify: non-finite trace at iteration %d", iters);
      // result: the buffer holding the last iterate (width max(n, width of H + 1)) goes to the
      // caller as it is
      ellpack_t *R = fbuf ? &b.Y : &b.X;
      *D = *R;
      memset(R, 0, sizeof(*R));
      st.time_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
      if (stats) *stats = st;
      if (status == 2) return fail(SP2E_NOTCONV, "sp2_purify: max_iter=%d reached (err %.3e)", opt.max_iter,
                                   st.err[iters < SP2_STATS_CAP ? iters : SP2_STATS_CAP - 1]);
      return SP2_OK;
    }
  }

  const bool mixed = opt.precision == SP2_PREC_MIXED;
  if (!handed) {
    // a2: X0 in FP64
    SP2_TRY(ellpack_create(n, H64->width + 1, SP2_F64, s, &b.X));
    SP2_TRY(x0_async(H64, b.bounds, opt.tau, &b.X, s));
    if (mixed) {
      SP2_TRY(ellpack_create(n, b.X.width, SP2_F32, s, &b.Y));
      SP2_TRY(convert_async(&b.X, &b.Y, s));
      ellpack_t t = b.X; b.X = b.Y; b.Y = t;  // X <- F32 copy, Y <- spare F64 buffer
    }
    // a3 for X0: traces from a pass over the stored matrix
    SP2_TRY(rowstat_async(&b.X, b.rowstat, s));
    launch_reduce_rows(b.rowstat, b.X.nnz, n, nullptr, b.dres, s);
    SP2_CUDA(cudaGetLastError());
    SP2_TRY(read_result(b, &res));
  }

  enum Phase { MAIN, TAIL } phase = MAIN;
  bool fp32 = mixed;
  int tail_left = opt.n_fp64_tail;
  bool armed = armed0;
  int it = it0;
  // the record so far reaches the caller on every return from here, errors included
  struct StatsOnExit {
    sp2_stats *dst;
    const sp2_stats *src;
    const int *it;
    ~StatsOnExit() {
      if (dst) {
        *dst = *src;
        dst->iterations = *it;
      }
    }
  } stats_on_exit{stats, &st, &it};
  int status = 0;  // set when the loop stops: 0 err < tol, 1 stall rule, 2 max_iter
  int last_count = res.max_nnz;
  int compact_level = 0;
  // the route flags (the level each row starts at) belong to one precision's passes:
  // cleared when the precision changes
  auto clear_route = [&]() -> int {
    if (b.route) SP2_CUDA(cudaMemsetAsync(b.route, 0, (size_t)n, s));
    return SP2_OK;
  };
  for (;;) {
    if (res.nonfinite) return fail(SP2E_NONFINITE, "sp2_purify: non-finite trace at iteration %d", it);
    const double trX = res.tr, trX2 = res.fro;
    const double err = fabs(trX - trX2) / (double)n;
    if (it < SP2_STATS_CAP) {
      st.trX[it] = trX;
      st.trX2[it] = trX2;
      st.err[it] = err;
      st.nnz_total[it] = res.nnz_total;
      st.max_row_nnz[it] = res.max_nnz;
    }
    // a7: stop rules
    bool stop = false;
    const bool stalled = [&] {
      if (fabs(trX - trX2) < opt.stall_arm) armed = true;
      return armed && it >= 2 && err >= opt.stall_ratio * st.err[it - 2];
    }();
    if (phase == MAIN) {
      bool main_done = false;
      if (fp32) {
        // FP32 loop: leave at switch_tol, at an FP32 stall, or at max_iter
        if (err < switch_tol || stalled) main_done = true;
        else if (it >= opt.max_iter) { main_done = true; status = 2; }
      } else {
        if (err < tol) { main_done = true; status = 0; }
        else if (opt.stall_rule && stalled) { main_done = true; status = 1; }
        else if (it >= opt.max_iter) { main_done = true; status = 2; }
      }
      if (main_done) {
        if (fp32 && tail_left > 0 && status != 2) {
          // a8: promote to FP64 and refine
          SP2_TRY(ensure(&b.Y, n, b.X.width, SP2_F64, s));
          SP2_TRY(convert_async(&b.X, &b.Y, s));
          ellpack_t t = b.X; b.X = b.Y; b.Y = t;
          fp32 = false;
          phase = TAIL;
          SP2_TRY(clear_route());
          st.fp32_iterations = it;
        } else {
          if (fp32 && status != 2) status = err < tol ? 0 : 1;
          stop = true;
        }
      }
    } else {  // TAIL: at least n_fp64_tail FP64 iterations, then the FP64 stop rule
      const int done = it - st.fp32_iterations;
      if (done >= opt.n_fp64_tail) {
        if (err < tol) { status = 0; stop = true; }
        else if (stalled) { status = 1; stop = true; }
      }
      if (!stop && it >= opt.max_iter + opt.n_fp64_tail) { status = 2; stop = true; }
    }
    if (stop) break;

    // a4: branch
    const bool up = fabs(2.0 * trX - trX2 - nocc) < fabs(trX2 - nocc);
    const double alpha = up ? -1.0 : 1.0, beta = up ? 2.0 : 0.0;
    if (it < SP2_STATS_CAP) st.branch[it] = up ? 2 : 1;

    // a5/a6: sized output, multiply with fused update and trace partials
    long long guess = (long long)4 * res.max_nnz;
    if (guess < (long long)(1.25 * last_count)) guess = (long long)(1.25 * last_count);
    if (guess < 64) guess = 64;
    if (opt.sizing == 1) {  // exact structural bound: never overflows
      int w = 0;
      SP2_TRY(exact_width(&b.X, up, &w));
      st.struct_passes++;
      guess = w;
    } else if (opt.sizing == 2) {  // predicted lengths of the product's rows
      SP2_TRY(features_async(&b.X, opt.tau, up ? 2 : 1, sz_rmax, sz_feat, s));
      SP2_TRY(predict_async(opt.predictor, sz_feat, n, sz_pred, s));
      SP2_TRY(max_float_async(sz_pred, n, sz_fmax, s));
      float fm = 0.f;
      SP2_CUDA(cudaMemcpyAsync(&fm, sz_fmax, sizeof(float), cudaMemcpyDeviceToHost, s));
      SP2_CUDA(cudaStreamSynchronize(s));
      guess = predicted_width(fm);
    }
    int width = round_up((int)(guess < max_w ? guess : max_w), 32);
    if (width > n) width = n;
    if (width < 32 && n >= 32) width = 32;
    // SpGEMM variant: fixed, or the tuner's choice for this class of product (a class seen
    // for the first time is tuned once the product fits)
    int lg = opt.spgemm_path;
    bool tune_pending = false;
    const double mean_nnz = (double)res.nnz_total / (double)n;
    if (lg == SP2_PATH_TUNED && !tune_find(b.X.dtype, n, mean_nnz, &lg)) {
      lg = 0;
      tune_pending = true;
    }
    for (;;) {
      SP2_TRY(ensure(&b.Y, n, width, b.X.dtype, s));
      MultiplyArgs a{&b.X, &b.X, beta != 0.0 ? &b.X : nullptr, &b.Y, alpha, beta, opt.tau, lg};
      a.sym = opt.symmetric != 0;
      a.compact_level = compact_level;
      if (lg == 0) a.route = b.route;
      SP2_TRY(multiply_async(a, b.rowstat, b.ctl, s));
      launch_reduce_rows(b.rowstat, b.Y.nnz, n, b.ctl, b.dres, s);
      SP2_CUDA(cudaGetLastError());
      SP2_TRY(read_result(b, &res));
      if (res.overflow_rows == 0) break;
      if (res.max_count > max_w)
        return fail(SP2E_OVERFLOW, "sp2_purify: a row needs %d slots, above the width cap %d", res.max_count, max_w);
      if (opt.sizing == 2) {  // the prediction was short: the failed pass counted the exact lengths
        width = round_up(res.max_count, 32);
      } else {
        width = round_up((int)(1.25 * res.max_count) + 1, 32);
      }
      if (width > max_w) width = round_up(max_w, 32) > n ? n : round_up(max_w, 32);
      if (width < res.max_count) width = res.max_count;
      st.regrows++;
    }
    if (tune_pending) {  // time every variant on this product, then redo it with the fastest
      MultiplyArgs a{&b.X, &b.X, beta != 0.0 ? &b.X : nullptr, &b.Y, alpha, beta, opt.tau, 0};
      a.sym = opt.symmetric != 0;
      SP2_TRY(tune_multiply(a, mean_nnz, b.rowstat, b.ctl, 2, &lg, nullptr, s));
      a.path = lg;
      SP2_TRY(multiply_async(a, b.rowstat, b.ctl, s));
      launch_reduce_rows(b.rowstat, b.Y.nnz, n, b.ctl, b.dres, s);
      SP2_CUDA(cudaGetLastError());
      SP2_TRY(read_result(b, &res));
      st.tuned++;
    }
    if (width > st.width_max) st.width_max = width;
    if (opt.sizing == 2) {  // how far the predictions were from the exact lengths
      SP2_TRY(pred_error_async(sz_pred, b.Y.nnz, n, sz_perr, s));
      double pe[2];
      SP2_CUDA(cudaMemcpyAsync(pe, sz_perr, sizeof(pe), cudaMemcpyDeviceToHost, s));
      SP2_CUDA(cudaStreamSynchronize(s));
      mae_sum += pe[0];
      under_sum += pe[1];
      rows_seen += (double)n;
    }
    last_count = res.max_count;
    if (it < SP2_STATS_CAP) {
      st.rows_level1[it] = res.n_level1;
      st.rows_level2[it] = res.n_level2;
      st.rows_deferred[it] = res.n_fallback;
      st.rows_routed[it] = res.n_routed;
      st.level[it] = (opt.symmetric && lg == 0) ? cascade_start(n, true, compact_level) : -1;
    }
    // the cascade of first passes (automatic for symmetric products) starts at the tight
    // compact level; once its first pass passes on more than level_up_frac of the rows, the
    // cascade starts one level higher for the rest of the run.  Rows passed on for their
    // length alone (FP32, rows of X above 512 entries) are not counted
    if (compact_level < 2 && opt.symmetric && lg == 0 && n >= kCascadeMinRows) {
      const int passed = (compact_level == 0 ? res.n_level1 : res.n_level2) - res.n_heavy;
      if ((double)passed > opt.level_up_frac * (double)n) ++compact_level;
    }
    ellpack_t t = b.X; b.X = b.Y; b.Y = t;
    ++it;
  }
  if (mixed && st.fp32_iterations == 0 && fp32) st.fp32_iterations = it;

  // result: an F64 matrix owned by the caller
  if (b.X.dtype != SP2_F64) {
    SP2_TRY(ensure(&b.Y, n, b.X.width, SP2_F64, s));
    SP2_TRY(convert_async(&b.X, &b.Y, s));
    ellpack_t t = b.X; b.X = b.Y; b.Y = t;
  }
  *D = b.X;
  memset(&b.X, 0, sizeof(b.X));
  SP2_CUDA(cudaStreamSynchronize(s));
  st.iterations = it;
  st.status = status;
  if (rows_seen > 0) {
    st.pred_log_mae = mae_sum / rows_seen;
    st.pred_under_frac = under_sum / rows_seen;
  }
  st.time_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  if (stats) *stats = st;
  if (status == 2) return fail(SP2E_NOTCONV, "sp2_purify: max_iter=%d reached (err %.3e)", opt.max_iter, st.err[it < SP2_STATS_CAP ? it : SP2_STATS_CAP - 1]);
  return SP2_OK;
}

extern "C" int sp2_x0_block(const ellpack_t *H, int32_t row0, double emin, double emax, double tau, ellpack_t *X0,
                            void *stream) {
  SP2_TRY(check_matrix(H, "sp2_x0_block: H"));
  SP2_TRY(check_matrix(X0, "sp2_x0_block: X0"));
  if (H->n != X0->n) return fail(SP2E_ARG, "sp2_x0_block: H and X0 hold different row counts");
  if (H->dtype != SP2_F64 || X0->dtype != SP2_F64) return fail(SP2E_ARG, "sp2_x0_block: F64 matrices expected");
  if (X0->width < H->width + 1) return fail(SP2E_ARG, "sp2_x0_block: X0 width %d < H width + 1", X0->width);
  if (X0->idx == H->idx || X0->val == H->val || X0->nnz == H->nnz) return fail(SP2E_ARG, "sp2_x0_block: X0 aliases H");
  if (row0 < 0) return fail(SP2E_ARG, "sp2_x0_block: row0 = %d must be >= 0", row0);
  if (!(tau >= 0.0) || !isfinite(tau)) return fail(SP2E_ARG, "sp2_x0_block: tau must be finite and >= 0");
  if (!isfinite(emin) || !isfinite(emax) || !(emax > emin))
    return fail(SP2E_ARG, "sp2_x0_block: bounds must be finite with emax > emin");
  cudaStream_t s = as_stream(stream);
  double *db = nullptr;
  SP2_TRY(dev_alloc((void **)&db, 2 * sizeof(double), s));
  const double hb[2] = {emin, emax};
  int rc = SP2_OK;
  cudaError_t e = cudaMemcpyAsync(db, hb, sizeof(hb), cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) rc = cuda_fail(e, "sp2_x0_block bounds", __FILE__, __LINE__);
  if (rc == SP2_OK) rc = x0_async(H, db, tau, X0, s, row0);
  if (rc == SP2_OK) {
    e = cudaStreamSynchronize(s);  // the bounds live in a stack array until the copy is done
    if (e != cudaSuccess) rc = cuda_fail(e, "sp2_x0_block", __FILE__, __LINE__);
  }
  dev_free(db, s);
  return rc;
}

extern "C" int sp2_x0(const ellpack_t *H, double tau, ellpack_t *X0, double *emin, double *emax, void *stream) {
  SP2_TRY(check_matrix(H, "sp2_x0: H"));
  SP2_TRY(check_matrix(X0, "sp2_x0: X0"));
  if (H->n != X0->n) return fail(SP2E_ARG, "sp2_x0: sizes differ");
  if (H->dtype != SP2_F64 || X0->dtype != SP2_F64) return fail(SP2E_ARG, "sp2_x0: F64 matrices expected");
  if (X0->width < H->width + 1) return fail(SP2E_ARG, "sp2_x0: X0 width %d < H width + 1", X0->width);
  if (X0->idx == H->idx || X0->val == H->val || X0->nnz == H->nnz) return fail(SP2E_ARG, "sp2_x0: X0 aliases H");
  if (!(tau >= 0.0) || !isfinite(tau)) return fail(SP2E_ARG, "sp2_x0: tau must be finite and >= 0");
  cudaStream_t s = as_stream(stream);
  double *db = nullptr;
  SP2_TRY(dev_alloc((void **)&db, 2 * sizeof(double), s));
  int rc = gershgorin_async(H, db, s);
  double hb[2] = {0, 0};
  if (rc == SP2_OK) {
    cudaError_t e = cudaMemcpyAsync(hb, db, sizeof(hb), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) rc = cuda_fail(e, "sp2_x0 bounds", __FILE__, __LINE__);
  }
  if (rc == SP2_OK && (!isfinite(hb[0]) || !isfinite(hb[1]))) rc = fail(SP2E_NONFINITE, "sp2_x0: H holds a NaN or Inf");
  if (rc == SP2_OK && !(hb[1] > hb[0])) rc = fail(SP2E_ARG, "sp2_x0: degenerate spectral bounds");
  if (rc == SP2_OK) rc = x0_async(H, db, tau, X0, s);
  if (rc == SP2_OK) {
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) rc = cuda_fail(e, "sp2_x0", __FILE__, __LINE__);
  }
  dev_free(db, s);
  SP2_TRY(rc);
  if (emin) *emin = hb[0];
  if (emax) *emax = hb[1];
  return SP2_OK;
}

extern "C" int sp2_step(const ellpack_t *X, ellpack_t *Xn, double nocc, double tau, sp2_step_info *info,
                        void *stream) {
  SP2_TRY(check_matrix(X, "sp2_step: X"));
  SP2_TRY(check_matrix(Xn, "sp2_step: Xn"));
  if (!info) return fail(SP2E_ARG, "sp2_step: info is NULL");
  if (X->n != Xn->n || X->dtype != Xn->dtype) return fail(SP2E_ARG, "sp2_step: X and Xn differ in n or dtype");
  if (X->idx == Xn->idx || X->val == Xn->val || X->nnz == Xn->nnz) return fail(SP2E_ARG, "sp2_step: Xn aliases X");
  if (!(tau >= 0.0) || !isfinite(tau)) return fail(SP2E_ARG, "sp2_step: tau must be finite and >= 0");
  if (!isfinite(nocc)) return fail(SP2E_ARG, "sp2_step: nocc not finite");
  if (!valid_path(info->spgemm_path)) return fail(SP2E_ARG, "sp2_step: spgemm_path must be -1, 0..4 or 7..12");
  if (info->compact_level < 0 || info->compact_level > 2) return fail(SP2E_ARG, "sp2_step: compact_level must be 0, 1 or 2");
  const int n = X->n;
  Buffers b;
  b.s = as_stream(stream);
  cudaStream_t s = b.s;
  SP2_TRY(dev_alloc((void **)&b.rowstat, sizeof(double2) * (size_t)n, s));
  SP2_TRY(dev_alloc((void **)&b.ctl, sizeof(SpgemmCtl), s));
  SP2_TRY(dev_alloc((void **)&b.dres, sizeof(StepResult), s));
  StepResult res;
  if (!info->have_traces) {
    SP2_TRY(rowstat_async(X, b.rowstat, s));
    launch_reduce_rows(b.rowstat, X->nnz, n, nullptr, b.dres, s);
    SP2_CUDA(cudaGetLastError());
    SP2_TRY(read_result(b, &res));
    if (res.nonfinite) return fail(SP2E_NONFINITE, "sp2_step: non-finite trace of X");
    info->trX = res.tr;
    info->trX2 = res.fro;
  }
  const double trX = info->trX, trX2 = info->trX2;
  info->err = fabs(trX - trX2) / (double)n;
  const bool up = fabs(2.0 * trX - trX2 - nocc) < fabs(trX2 - nocc);
  info->branch = up ? 2 : 1;
  MultiplyArgs a{X, X, up ? X : nullptr, Xn, up ? -1.0 : 1.0, up ? 2.0 : 0.0, tau, info->spgemm_path};
  a.sym = info->symmetric != 0;
  a.compact_level = info->compact_level;
  if (a.path == SP2_PATH_TUNED) {
    double mean = 0.0;
    SP2_TRY(mean_row_nnz(X, &mean, s));
    if (!tune_find(X->dtype, n, mean, &a.path)) SP2_TRY(tune_multiply(a, mean, b.rowstat, b.ctl, 2, &a.path, nullptr, s));
  }
  info->spgemm_path_used = a.path;
  SP2_TRY(multiply_async(a, b.rowstat, b.ctl, s));
  launch_reduce_rows(b.rowstat, Xn->nnz, n, b.ctl, b.dres, s);
  SP2_CUDA(cudaGetLastError());
  SP2_TRY(read_result(b, &res));
  info->trXn = res.tr;
  info->trXn2 = res.fro;
  info->nnz_total = res.nnz_total;
  info->max_row_nnz = res.max_nnz;
  info->required_width = res.max_count;
  info->rows_deferred = res.n_fallback;
  info->rows_dense = res.n_fallback2;
  if (res.overflow_rows > 0)
    return fail(SP2E_OVERFLOW, "sp2_step: %d row(s) need %d slots, Xn width is %d", res.overflow_rows, res.max_count,
                Xn->width);
  if (res.nonfinite) return fail(SP2E_NONFINITE, "sp2_step: non-finite trace of the result");
  return SP2_OK;
}
