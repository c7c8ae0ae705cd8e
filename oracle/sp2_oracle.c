/*
 * sp2_oracle.c -- plain, slow, single-purpose CPU FP64 oracle for SP2 density-matrix
 * purification on thresholded ELLPACK matrices.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may call, link or load this
 * file; it exists so that tests, the smoke check and the CPU baseline leg of the
 * benchmark can check the CUDA library against an independent implementation.  It
 * shares no code, header or constant with the CUDA library.
 *
 * What it follows:
 *   - ELLPACK storage: per matrix an int nnz[N], an int index[N*M] and a double
 *     value[N*M] array (Section "Micro-Kernel Performance Evaluation - NUMA Aware
 *     Data", the allocation listing).  Row i keeps its entries in slots i*M .. i*M+nnz[i]-1
 *     (row-major reading of the N*M arrays).  Slots past nnz[i] are never read.
 *   - The ELLPACK matrix-matrix multiply X*X with small entries dropped ("BML ELLPACK
 *     matrix-matrix multiply", Section "Performance Evaluation using System Matrices").
 *     The paper does not print the algorithm; the oracle is the plain definition:
 *       pattern(C_i) = union over k in cols(A_i) of cols(B_k)   (plus cols(C_i) if beta != 0)
 *       v_ij = alpha * sum_k a_ik * b_kj + beta * c_ij, summed over k in ascending order
 *       keep (j, v_ij) iff |v_ij| > tau; for tau == 0 every structural entry is kept
 *       (exact zeros included); each output row is sorted by column.
 *   - SP2-Basic ("SP2 Loop X2 / Norm / Misc" phases, Section "Performance Evaluation
 *     using an ExaSP2 Application"; only gapped systems are appropriate for SP2, same
 *     section) following the published SP2 recursion (Niklasson 2002, cited in the
 *     Introduction):
 *       Gershgorin bounds e_min, e_max of H
 *       X0 = (e_max I - H) / (e_max - e_min), thresholded
 *       repeat: trX = tr X; P = X*X; trX2 = tr P; err = |trX - trX2| / N
 *               stop if err < tol (or the stall rule fires, or max_iter is reached)
 *               X <- drop(2X - P) if |2 trX - trX2 - nocc| < |trX2 - nocc|, else drop(P)
 *     The paper names SP2 but prints none of its rules, so the following are readings:
 *       - branch: 2X - X^2 is taken iff |2 trX - trX2 - nocc| < |trX2 - nocc| (strict);
 *         a tie takes X^2, which keeps the choice deterministic;
 *       - error: err_n = |trX_n - trX2_n| / N, the trace defect per orbital, because with
 *         tau > 0 the unnormalised defect cannot reach a tolerance such as 1e-10;
 *       - stall rule: armed once |trX - trX2| < stall_arm (0.1), it fires when
 *         err_n >= stall_ratio * err_{n-2} (ratio 1: two updates brought no reduction),
 *         so that a run whose error has reached the floor set by tau ends there; it is
 *         not armed earlier because a gapless H shows that pattern long before the end;
 *       - tr X^2 is the diagonal of the unthresholded product P, taken before the drop;
 *       - keep rule: an entry survives the drop iff |v| > tau (a drop tolerance removes
 *         the small entries; an entry equal to tau is removed); at tau == 0 every
 *         structural entry is kept, exact zeros included, so that the pattern does not
 *         depend on cancellation.
 *
 * Storage readings (the paper fixes only the array sizes): rows are stored row-major
 * (index[i*M + s], consistent with the N*M allocations), each row in ascending column
 * order; padding slots are never read.
 *
 * Compiled with -ffp-contract=off so that every a*b + c is a separately rounded
 * multiply and add, i.e. the arithmetic is exactly what the C source says.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
  int n;        /* rows (= columns) */
  int w;        /* width M: slots per row */
  int *idx;     /* n*w column indices, row-major */
  double *val;  /* n*w values, row-major */
  int *nnz;     /* n stored entries per row */
} orc_ell;

static int g_threads = 1;

void orc_set_threads(int t) { g_threads = t > 0 ? t : 1; }

int orc_get_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

static int cmp_int(const void *a, const void *b) {
  int x = *(const int *)a, y = *(const int *)b;
  return (x > y) - (x < y);
}

/* (column, value) pair used to visit a row of A in ascending column order. */
typedef struct { int k; double a; } kv;
static int cmp_kv(const void *a, const void *b) {
  int x = ((const kv *)a)->k, y = ((const kv *)b)->k;
  return (x > y) - (x < y);
}

/*
 * C_out = drop_tau(alpha * A * B + beta * C) for the rows listed in `rows`
 * (rows == NULL: all rows; output row r holds product row rows[r]).
 * out must have out->n >= nrows and a width out->w.  row_count[r] receives the
 * post-threshold number of entries of output row r even when it exceeds out->w; such
 * rows are left unwritten (nnz set to 0) and the function returns 1.  Returns 0 when
 * every row fitted, -1 on bad arguments (a row or column index outside 0 .. n-1
 * included), -3 when host memory runs out.
 * diag (optional, length nrows): the unthresholded, unscaled sum_k a_ik b_ki of each row.
 */
int orc_spgemm(const orc_ell *A, const orc_ell *B, const orc_ell *C, double alpha,
               double beta, double tau, const int *rows, int nrows, orc_ell *out,
               int *row_count, double *diag) {
  if (!A || !B || !out || tau < 0.0) return -1;
  int n = A->n;
  if (B->n != n) return -1;
  if (beta != 0.0 && (!C || C->n != n)) return -1;
  if (rows == NULL) nrows = n;
  int overflow = 0, nomem = 0, badidx = 0;
#pragma omp parallel num_threads(g_threads) reduction(| : overflow, nomem, badidx)
  {
    double *acc = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double *cv = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    int *mark = (int *)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
    int *list = (int *)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
    kv *arow = (kv *)malloc(sizeof(kv) * (size_t)(A->w > 0 ? A->w : 1));
    const int ok = acc && cv && mark && list && arow;
    if (!ok) nomem = 1;
    /* mark[j] == r  <=>  column j is already in the pattern of output row r */
    if (ok)
      for (int j = 0; j < n; ++j) mark[j] = -1;
#pragma omp for schedule(dynamic, 64)
    for (int r = 0; r < nrows; ++r) {
      if (!ok) continue;
      int i = rows ? rows[r] : r;
      int cnt = 0;
      /* row i of A in ascending column order */
      int na = A->nnz[i];
      for (int s = 0; s < na; ++s) {
        arow[s].k = A->idx[(size_t)i * A->w + s];
        arow[s].a = A->val[(size_t)i * A->w + s];
      }
      qsort(arow, (size_t)na, sizeof(kv), cmp_kv);
      for (int t = 0; t < na; ++t) {
        int k = arow[t].k;
        double a = arow[t].a;
        if (k < 0 || k >= n) { badidx = 1; continue; }
        int nb = B->nnz[k];
        for (int s = 0; s < nb; ++s) {
          int j = B->idx[(size_t)k * B->w + s];
          double b = B->val[(size_t)k * B->w + s];
          if (j < 0 || j >= n) { badidx = 1; continue; }
          if (mark[j] != r) { mark[j] = r; acc[j] = 0.0; cv[j] = 0.0; list[cnt++] = j; }
          acc[j] = acc[j] + a * b;
        }
      }
      if (diag) diag[r] = (mark[i] == r) ? acc[i] : 0.0;
      if (beta != 0.0) {
        int nc = C->nnz[i];
        for (int s = 0; s < nc; ++s) {
          int j = C->idx[(size_t)i * C->w + s];
          if (j < 0 || j >= n) { badidx = 1; continue; }
          if (mark[j] != r) { mark[j] = r; acc[j] = 0.0; cv[j] = 0.0; list[cnt++] = j; }
          cv[j] = C->val[(size_t)i * C->w + s];
        }
      }
      qsort(list, (size_t)cnt, sizeof(int), cmp_int);
      int kept = 0;
      for (int t = 0; t < cnt; ++t) {
        int j = list[t];
        double v = alpha * acc[j] + beta * cv[j];
        if (tau == 0.0 || fabs(v) > tau) list[kept++] = j, acc[j] = v;
      }
      if (row_count) row_count[r] = kept;
      if (kept > out->w) {
        overflow = 1;
        out->nnz[r] = 0;
      } else {
        for (int t = 0; t < kept; ++t) {
          out->idx[(size_t)r * out->w + t] = list[t];
          out->val[(size_t)r * out->w + t] = acc[list[t]];
        }
        out->nnz[r] = kept;
      }
    }
    free(acc); free(cv); free(mark); free(list); free(arow);
  }
  if (nomem) return -3;
  if (badidx) return -1;  /* a column index outside 0 .. n-1: not an n x n matrix */
  return overflow ? 1 : 0;
}

/* out = drop_tau(alpha * A + beta * B); pattern = union of the two patterns. */
int orc_add(const orc_ell *A, const orc_ell *B, double alpha, double beta, double tau,
            orc_ell *out, int *row_count) {
  if (!A || !B || !out || A->n != B->n || tau < 0.0) return -1;
  int n = A->n;
  int overflow = 0;
  double *av = (double *)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
  double *bv = (double *)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
  int *mark = (int *)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
  int *list = (int *)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
  if (!av || !bv || !mark || !list) { free(av); free(bv); free(mark); free(list); return -3; }
  for (int j = 0; j < n; ++j) mark[j] = -1;
  for (int i = 0; i < n; ++i) {
    int cnt = 0;
    for (int s = 0; s < A->nnz[i]; ++s) {
      int j = A->idx[(size_t)i * A->w + s];
      if (j < 0 || j >= n) { free(av); free(bv); free(mark); free(list); return -1; }
      if (mark[j] != i) { mark[j] = i; av[j] = 0.0; bv[j] = 0.0; list[cnt++] = j; }
      av[j] = A->val[(size_t)i * A->w + s];
    }
    for (int s = 0; s < B->nnz[i]; ++s) {
      int j = B->idx[(size_t)i * B->w + s];
      if (j < 0 || j >= n) { free(av); free(bv); free(mark); free(list); return -1; }
      if (mark[j] != i) { mark[j] = i; av[j] = 0.0; bv[j] = 0.0; list[cnt++] = j; }
      bv[j] = B->val[(size_t)i * B->w + s];
    }
    qsort(list, (size_t)cnt, sizeof(int), cmp_int);
    int kept = 0;
    for (int t = 0; t < cnt; ++t) {
      int j = list[t];
      double v = alpha * av[j] + beta * bv[j];
      if (tau == 0.0 || fabs(v) > tau) { list[kept++] = j; av[j] = v; }
    }
    if (row_count) row_count[i] = kept;
    if (kept > out->w) { overflow = 1; out->nnz[i] = 0; continue; }
    for (int t = 0; t < kept; ++t) {
      out->idx[(size_t)i * out->w + t] = list[t];
      out->val[(size_t)i * out->w + t] = av[list[t]];
    }
    out->nnz[i] = kept;
  }
  free(av); free(bv); free(mark); free(list);
  return overflow ? 1 : 0;
}

/* out = drop_tau(A): keep (j, a_ij) iff |a_ij| > tau (tau == 0 keeps every entry). */
int orc_drop(const orc_ell *A, double tau, orc_ell *out) {
  if (!A || !out || out->n != A->n || out->w < A->w || tau < 0.0) return -1;
  for (int i = 0; i < A->n; ++i) {
    int kept = 0;
    for (int s = 0; s < A->nnz[i]; ++s) {
      double v = A->val[(size_t)i * A->w + s];
      if (tau == 0.0 || fabs(v) > tau) {
        out->idx[(size_t)i * out->w + kept] = A->idx[(size_t)i * A->w + s];
        out->val[(size_t)i * out->w + kept] = v;
        kept++;
      }
    }
    out->nnz[i] = kept;
  }
  return 0;
}

/* tr A = sum_i A_ii (a missing diagonal entry counts as zero). */
double orc_trace(const orc_ell *A) {
  double t = 0.0;
  for (int i = 0; i < A->n; ++i)
    for (int s = 0; s < A->nnz[i]; ++s)
      if (A->idx[(size_t)i * A->w + s] == i) t = t + A->val[(size_t)i * A->w + s];
  return t;
}

/* Gershgorin disc bounds: e_min = min_i (H_ii - R_i), e_max = max_i (H_ii + R_i),
 * R_i = sum_{j != i} |H_ij|. */
int orc_gershgorin(const orc_ell *H, double *emin, double *emax) {
  if (!H || H->n <= 0) return -1;
  double lo = INFINITY, hi = -INFINITY;
  for (int i = 0; i < H->n; ++i) {
    double d = 0.0, r = 0.0;
    for (int s = 0; s < H->nnz[i]; ++s) {
      int j = H->idx[(size_t)i * H->w + s];
      double v = H->val[(size_t)i * H->w + s];
      if (j == i) d = v; else r = r + fabs(v);
    }
    if (d - r < lo) lo = d - r;
    if (d + r > hi) hi = d + r;
  }
  *emin = lo;
  *emax = hi;
  return 0;
}

/* X0 = drop_tau((e_max I - H) / (e_max - e_min)); rows sorted by column; the diagonal
 * is present in the pattern even where H has no diagonal entry.  out->w >= H->w + 1. */
int orc_x0(const orc_ell *H, double emin, double emax, double tau, orc_ell *out) {
  if (!H || !out || out->n != H->n || out->w < H->w + 1 || !(emax > emin)) return -1;
  int n = H->n;
  double *v = (double *)malloc(sizeof(double) * (size_t)(H->w + 1));
  int *c = (int *)malloc(sizeof(int) * (size_t)(H->w + 1));
  kv *row = (kv *)malloc(sizeof(kv) * (size_t)(H->w + 1));
  if (!v || !c || !row) { free(v); free(c); free(row); return -3; }
  for (int i = 0; i < n; ++i) {
    int cnt = 0, has_diag = 0;
    for (int s = 0; s < H->nnz[i]; ++s) {
      int j = H->idx[(size_t)i * H->w + s];
      double h = H->val[(size_t)i * H->w + s];
      double x;
      if (j == i) { x = (emax - h) / (emax - emin); has_diag = 1; }
      else x = (0.0 - h) / (emax - emin);
      row[cnt].k = j; row[cnt].a = x; cnt++;
    }
    if (!has_diag) { row[cnt].k = i; row[cnt].a = emax / (emax - emin); cnt++; }
    qsort(row, (size_t)cnt, sizeof(kv), cmp_kv);
    int kept = 0;
    for (int t = 0; t < cnt; ++t)
      if (tau == 0.0 || fabs(row[t].a) > tau) { c[kept] = row[t].k; v[kept] = row[t].a; kept++; }
    for (int t = 0; t < kept; ++t) {
      out->idx[(size_t)i * out->w + t] = c[t];
      out->val[(size_t)i * out->w + t] = v[t];
    }
    out->nnz[i] = kept;
  }
  free(v); free(c); free(row);
  return 0;
}

/* ------------------------------------------------------------------ SP2 loop */

typedef struct {
  int iterations;     /* number of updates applied */
  int status;         /* 0 converged (err < tol), 1 stopped by stall rule, 2 max_iter reached,
                         -1 bad arguments, -3 out of host memory */
  int max_iter;       /* capacity of the per-iteration arrays below */
  double emin, emax;  /* Gershgorin bounds */
  double *trX;        /* per visited X_n: tr X_n                         [max_iter+1] */
  double *trX2;       /* per visited X_n: tr X_n^2 (diagonal of X_n*X_n)  [max_iter+1] */
  double *err;        /* per visited X_n: |trX - trX2| / N               [max_iter+1] */
  int *branch;        /* per update: 1 = X^2, 2 = 2X - X^2                [max_iter]   */
  long long *nnz_total; /* per visited X_n: total stored entries          [max_iter+1] */
  int *max_row_nnz;   /* per visited X_n                                  [max_iter+1] */
} orc_sp2_stats;

static void ell_free(orc_ell *m) { free(m->idx); free(m->val); free(m->nnz); m->idx = 0; m->val = 0; m->nnz = 0; }

/* Allocates an n x w matrix; returns 0, or ORC_NOMEM (nothing left allocated). */
#define ORC_NOMEM (-3)
static int ell_alloc(int n, int w, orc_ell *m) {
  m->n = n; m->w = w;
  m->idx = (int *)malloc(sizeof(int) * (size_t)n * (size_t)w);
  m->val = (double *)malloc(sizeof(double) * (size_t)n * (size_t)w);
  m->nnz = (int *)calloc((size_t)n, sizeof(int));
  if (!m->idx || !m->val || !m->nnz) { ell_free(m); return ORC_NOMEM; }
  return 0;
}

static void row_stats(const orc_ell *m, long long *tot, int *mx) {
  long long t = 0; int x = 0;
  for (int i = 0; i < m->n; ++i) { t += m->nnz[i]; if (m->nnz[i] > x) x = m->nnz[i]; }
  *tot = t; *mx = x;
}

/* Runs an ELLPACK product into a freshly sized matrix *out (width grown until it fits).
 * Returns 0, ORC_NOMEM, or -1 if the product rejects its arguments. */
static int spgemm_fit(const orc_ell *A, const orc_ell *B, const orc_ell *C, double alpha,
                      double beta, double tau, int w_guess, double *diag, orc_ell *out) {
  int n = A->n;
  int *cnt = (int *)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
  if (!cnt) return ORC_NOMEM;
  int w = w_guess < 1 ? 1 : (w_guess > n ? n : w_guess);
  for (;;) {
    if (ell_alloc(n, w, out) != 0) { free(cnt); return ORC_NOMEM; }
    int rc = orc_spgemm(A, B, C, alpha, beta, tau, NULL, n, out, cnt, diag);
    if (rc == 0) { free(cnt); return 0; }
    ell_free(out);
    if (rc < 0) { free(cnt); return rc; }
    int need = 0;
    for (int i = 0; i < n; ++i) if (cnt[i] > need) need = cnt[i];
    w = need;
  }
}

/* Sized by the longest union of two rows (at most nnz_A(i) + nnz_B(i)), not by the stored
 * widths, so that the widths of an iteration's matrices do not compound. */
static int add_fit(const orc_ell *A, const orc_ell *B, double alpha, double beta, double tau,
                   orc_ell *out) {
  int w = 1;
  for (int i = 0; i < A->n; ++i)
    if (A->nnz[i] + B->nnz[i] > w) w = A->nnz[i] + B->nnz[i];
  if (w > A->n) w = A->n;
  if (ell_alloc(A->n, w, out) != 0) return ORC_NOMEM;
  int rc = orc_add(A, B, alpha, beta, tau, out, NULL);
  if (rc < 0) ell_free(out);
  return rc < 0 ? rc : 0;
}

/*
 * SP2 purification of H.  On return *D holds the density matrix (library-allocated
 * arrays, release with orc_free_ell).  Stall rule (if stall_arm > 0): armed once
 * |trX - trX2| < stall_arm (0.1 in the method's reading); fires when
 * err_n >= stall_ratio * err_{n-2} (stall_ratio 1 in the method's reading: two updates
 * brought no reduction; a ratio below 1 also ends a slow monotone drift).
 */
int orc_sp2(const orc_ell *H, double nocc, double tol, double tau, int max_iter, double stall_arm,
            double stall_ratio, orc_ell *D, orc_sp2_stats *st) {
  if (!H || !D || !st || max_iter < 0 || tau < 0.0) return -1;
  if (!(stall_ratio > 0.0 && stall_ratio <= 1.0)) return -1;
  int n = H->n;
  double emin, emax;
  orc_gershgorin(H, &emin, &emax);
  st->emin = emin; st->emax = emax;
  orc_ell X;
  if (ell_alloc(n, H->w + 1, &X) != 0) { st->status = ORC_NOMEM; return ORC_NOMEM; }
  int rc = orc_x0(H, emin, emax, tau, &X);
  if (rc != 0) { ell_free(&X); st->status = rc; return rc; }
  int armed = 0;
  st->status = 2;
  int it = 0;
  for (;; ++it) {
    double trX = orc_trace(&X);
    long long xt; int xmax;
    row_stats(&X, &xt, &xmax);
    /* first width tried: 8x the longest row of X (spgemm_fit grows it to the exact count) */
    orc_ell P;
    rc = spgemm_fit(&X, &X, NULL, 1.0, 0.0, 0.0, 8 * xmax, NULL, &P);
    if (rc != 0) { ell_free(&X); st->status = rc; return rc; }
    double trX2 = orc_trace(&P);
    double err = fabs(trX - trX2) / (double)n;
    if (it <= st->max_iter) {
      st->trX[it] = trX; st->trX2[it] = trX2; st->err[it] = err;
      row_stats(&X, &st->nnz_total[it], &st->max_row_nnz[it]);
    }
    if (err < tol) { st->status = 0; ell_free(&P); break; }
    if (stall_arm > 0.0) {
      if (fabs(trX - trX2) < stall_arm) armed = 1;
      if (armed && it >= 2 && err >= stall_ratio * st->err[it - 2]) { st->status = 1; ell_free(&P); break; }
    }
    if (it >= max_iter) { st->status = 2; ell_free(&P); break; }
    orc_ell Xn;
    if (fabs(2.0 * trX - trX2 - nocc) < fabs(trX2 - nocc)) {
      st->branch[it] = 2;
      rc = add_fit(&P, &X, -1.0, 2.0, tau, &Xn);    /* 2X - X^2 */
    } else {
      st->branch[it] = 1;
      rc = ell_alloc(n, P.w, &Xn);                   /* X^2, thresholded */
      if (rc == 0) orc_drop(&P, tau, &Xn);
    }
    ell_free(&P);
    ell_free(&X);
    if (rc != 0) { st->status = rc; return rc; }
    X = Xn;
  }
  st->iterations = it;
  *D = X;
  return 0;
}

void orc_free_ell(orc_ell *m) { if (m) ell_free(m); }
