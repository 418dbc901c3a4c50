/*
 * Plain CPU FP64 oracle for the SISSO l0-regularization step.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the package smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code with
 * the CUDA path.
 *
 * What it computes (paper Sec. 2.4): for every n-tuple of the m input
 * features, a least-squares fit of the features to the target, scored by the
 * squared deviation; the best tuples are returned.  Per tuple it follows the
 * steps the paper lists in Sec. 2.4: assemble the descriptor matrix in
 * scratch space, QR-factorise it with Householder reflections, compute the
 * least-squares fit, compute the score.  Readings taken where the paper is
 * silent:
 *   - the fit has an intercept; centring every column and the target by the
 *     task mean removes it exactly, so the QR runs on centred columns;
 *   - multi-task (Sec. 3.1, same descriptor, per-task coefficients): each
 *     task is fitted on its own rows; PER_TASK ranks each task separately by
 *     its SSE, SHARED ranks by the pooled mean SSE sum_t SSE_t / N;
 *   - tuples are combinations without repetition, ascending indices
 *     (C(m, n) of them, Sec. 3.1 counts);
 *   - equal scores are ordered by the lexicographically smaller tuple;
 *   - a tuple is ineligible (rank deficient) when
 *     rho = min_j |R_jj| / ||a_j|| < rho_min, a_j the centred column.
 *
 * Norms use the scaled two-pass sum of squares (max |v| first, then the sum
 * of (v/max)^2).  Plain loops, FP64, no BLAS.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_MAX_DIM 16

/* ---------------------------------------------------------------- norms -- */
static double norm2_scaled(const double *v, int64_t n) {
  double scale = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    double a = fabs(v[i]);
    if (a > scale) scale = a;
  }
  if (scale == 0.0) return 0.0;
  double ssq = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    double r = v[i] / scale;
    ssq += r * r;
  }
  return scale * sqrt(ssq);
}

/* ------------------------------------------------------------ centring -- */
/* Centre each column of task rows [lo, hi) and the target by their mean
 * (two-pass: mean, then subtract).  xc is [m][n_t], yc is [n_t]. */
static void centre_task(const double *X, const double *y, int64_t n_total,
                        int64_t m, int64_t lo, int64_t hi, double *xc,
                        double *yc, double *colnorm) {
  int64_t nt = hi - lo;
  for (int64_t j = 0; j < m; ++j) {
    const double *col = X + j * n_total + lo;
    double s = 0.0;
    for (int64_t i = 0; i < nt; ++i) s += col[i];
    double mean = s / (double)nt;
    double *dst = xc + j * nt;
    for (int64_t i = 0; i < nt; ++i) dst[i] = col[i] - mean;
    colnorm[j] = norm2_scaled(dst, nt);
  }
  double s = 0.0;
  for (int64_t i = 0; i < nt; ++i) s += y[lo + i];
  double mean = s / (double)nt;
  for (int64_t i = 0; i < nt; ++i) yc[i] = y[lo + i] - mean;
}

/* ------------------------------------------------------- Householder LSQ -- */
/* A: n x d, column-major (column c at A + c*n), overwritten.
 * b: n, overwritten with Q^T b.  Returns SSE = ||(Q^T b)[d:]||^2.
 * R diagonal is written to rdiag[0..d-1]. */
static double householder_lsq(double *A, int64_t n, int d, double *b,
                              double *rdiag) {
  for (int j = 0; j < d; ++j) {
    double *aj = A + (int64_t)j * n;
    int64_t len = n - j;
    double sigma = norm2_scaled(aj + j, len);
    if (sigma == 0.0) { /* nothing to reflect; R_jj = 0 */
      rdiag[j] = 0.0;
      continue;
    }
    double x0 = aj[j];
    double alpha = (x0 >= 0.0) ? -sigma : sigma;
    /* v = x - alpha e1; H = I - beta v v^T with beta = 1 / (sigma (sigma + |x0|)) */
    double v0 = x0 - alpha;
    double beta = 1.0 / (sigma * (sigma + fabs(x0)));
    /* apply to later columns */
    for (int c = j + 1; c < d; ++c) {
      double *ac = A + (int64_t)c * n;
      double s = v0 * ac[j];
      for (int64_t i = j + 1; i < n; ++i) s += aj[i] * ac[i];
      s *= beta;
      ac[j] -= s * v0;
      for (int64_t i = j + 1; i < n; ++i) ac[i] -= s * aj[i];
    }
    /* apply to b */
    {
      double s = v0 * b[j];
      for (int64_t i = j + 1; i < n; ++i) s += aj[i] * b[i];
      s *= beta;
      b[j] -= s * v0;
      for (int64_t i = j + 1; i < n; ++i) b[i] -= s * aj[i];
    }
    aj[j] = alpha;
    rdiag[j] = alpha;
  }
  double sse = 0.0;
  for (int64_t i = d; i < n; ++i) sse += b[i] * b[i];
  return sse;
}

/* Score one tuple on one task: copy centred columns to scratch, QR, SSE.
 * Returns SSE; *rho = min_j |R_jj| / ||a_j|| (0 when a column is zero). */
static double score_tuple_task(const double *xc, const double *yc, int64_t nt,
                               const double *colnorm, const int32_t *tup, int d,
                               double *scratchA, double *scratchb,
                               double *rho) {
  double rdiag[ORACLE_MAX_DIM];
  for (int c = 0; c < d; ++c)
    memcpy(scratchA + (int64_t)c * nt, xc + (int64_t)tup[c] * nt,
           sizeof(double) * (size_t)nt);
  memcpy(scratchb, yc, sizeof(double) * (size_t)nt);
  double sse = householder_lsq(scratchA, nt, d, scratchb, rdiag);
  double r = INFINITY;
  for (int c = 0; c < d; ++c) {
    double cn = colnorm[tup[c]];
    double q = (cn > 0.0) ? fabs(rdiag[c]) / cn : 0.0;
    if (q < r) r = q;
  }
  *rho = r;
  return sse;
}

/* --------------------------------------------------------------- top-k -- */
typedef struct {
  int k, d, n;
  double *score;   /* [k] ascending */
  int32_t *tup;    /* [k][d] */
} topk_t;

static int tuple_less(const int32_t *a, const int32_t *b, int d) {
  for (int c = 0; c < d; ++c) {
    if (a[c] != b[c]) return a[c] < b[c];
  }
  return 0;
}

/* (score, tuple) strictly less than entry i of the list */
static int entry_less(double s, const int32_t *t, const topk_t *L, int i) {
  if (s < L->score[i]) return 1;
  if (s > L->score[i]) return 0;
  return tuple_less(t, L->tup + (int64_t)i * L->d, L->d);
}

static void topk_push(topk_t *L, double s, const int32_t *t) {
  if (L->n == L->k && !entry_less(s, t, L, L->k - 1)) return;
  int pos = (L->n < L->k) ? L->n : L->k - 1;
  while (pos > 0 && entry_less(s, t, L, pos - 1)) {
    L->score[pos] = L->score[pos - 1];
    memcpy(L->tup + (int64_t)pos * L->d, L->tup + (int64_t)(pos - 1) * L->d,
           sizeof(int32_t) * (size_t)L->d);
    --pos;
  }
  L->score[pos] = s;
  memcpy(L->tup + (int64_t)pos * L->d, t, sizeof(int32_t) * (size_t)L->d);
  if (L->n < L->k) L->n++;
}

/* ------------------------------------------------------- public entries -- */
typedef struct {
  int n_tasks;
  int64_t m, n_total;
  const int64_t *offsets;
  double **xc, **yc, **colnorm;
} centred_t;

static int centred_make(centred_t *C, const double *X, const double *y,
                        const int64_t *offsets, int n_tasks, int64_t m) {
  C->n_tasks = n_tasks;
  C->m = m;
  C->n_total = offsets[n_tasks];
  C->offsets = offsets;
  C->xc = (double **)calloc((size_t)n_tasks, sizeof(double *));
  C->yc = (double **)calloc((size_t)n_tasks, sizeof(double *));
  C->colnorm = (double **)calloc((size_t)n_tasks, sizeof(double *));
  if (!C->xc || !C->yc || !C->colnorm) return 2;
  for (int t = 0; t < n_tasks; ++t) {
    int64_t lo = offsets[t], hi = offsets[t + 1];
    int64_t nt = hi - lo;
    C->xc[t] = (double *)malloc(sizeof(double) * (size_t)(m * nt));
    C->yc[t] = (double *)malloc(sizeof(double) * (size_t)nt);
    C->colnorm[t] = (double *)malloc(sizeof(double) * (size_t)m);
    if (!C->xc[t] || !C->yc[t] || !C->colnorm[t]) return 2;
    centre_task(X, y, C->n_total, m, lo, hi, C->xc[t], C->yc[t],
                C->colnorm[t]);
  }
  return 0;
}

static void centred_free(centred_t *C) {
  for (int t = 0; t < C->n_tasks; ++t) {
    if (C->xc) free(C->xc[t]);
    if (C->yc) free(C->yc[t]);
    if (C->colnorm) free(C->colnorm[t]);
  }
  free(C->xc);
  free(C->yc);
  free(C->colnorm);
}

static int validate(const int64_t *offsets, int n_tasks, int64_t m, int d) {
  if (n_tasks < 1 || m < 1 || d < 1 || d > ORACLE_MAX_DIM || d > m) return 1;
  if (offsets[0] != 0) return 1;
  for (int t = 0; t < n_tasks; ++t)
    if (offsets[t + 1] - offsets[t] < d + 2) return 1;
  return 0;
}

/* Score explicit tuples.  tuples: [n_tuples][d] ascending 0-based indices.
 * out_sse, out_rho: [n_tuples][n_tasks]. */
int oracle_l0_score(const double *X, const double *y, const int64_t *offsets,
                    int n_tasks, int64_t m, int d, int64_t n_tuples,
                    const int32_t *tuples, double *out_sse, double *out_rho,
                    int n_threads) {
  if (validate(offsets, n_tasks, m, d)) return 1;
  centred_t C;
  memset(&C, 0, sizeof(C));
  if (centred_make(&C, X, y, offsets, n_tasks, m)) {
    centred_free(&C);
    return 2;
  }
  int64_t nmax = 0;
  for (int t = 0; t < n_tasks; ++t)
    if (offsets[t + 1] - offsets[t] > nmax) nmax = offsets[t + 1] - offsets[t];
#ifdef _OPENMP
  if (n_threads > 0) omp_set_num_threads(n_threads);
#pragma omp parallel
#endif
  {
    double *A = (double *)malloc(sizeof(double) * (size_t)(nmax * d));
    double *b = (double *)malloc(sizeof(double) * (size_t)nmax);
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 64)
#endif
    for (int64_t q = 0; q < n_tuples; ++q) {
      const int32_t *tup = tuples + q * d;
      for (int t = 0; t < n_tasks; ++t) {
        int64_t nt = offsets[t + 1] - offsets[t];
        double rho;
        out_sse[q * n_tasks + t] = score_tuple_task(
            C.xc[t], C.yc[t], nt, C.colnorm[t], tup, d, A, b, &rho);
        out_rho[q * n_tasks + t] = rho;
      }
    }
    free(A);
    free(b);
  }
  centred_free(&C);
  return 0;
}

/* Least-squares coefficients of one tuple on one task (intercept first):
 * out_coef[0] = beta_0, out_coef[1..d] = beta for the tuple's columns.
 * Back-substitution R beta = (Q^T yc)[0:d]; beta_0 = mean(y) - sum beta_j mean(x_j). */
int oracle_l0_coefs(const double *X, const double *y, const int64_t *offsets,
                    int n_tasks, int64_t m, int d, int task,
                    const int32_t *tup, double *out_coef) {
  if (validate(offsets, n_tasks, m, d) || task < 0 || task >= n_tasks) return 1;
  int64_t n_total = offsets[n_tasks];
  int64_t lo = offsets[task], hi = offsets[task + 1], nt = hi - lo;
  double *A = (double *)malloc(sizeof(double) * (size_t)(nt * d));
  double *b = (double *)malloc(sizeof(double) * (size_t)nt);
  if (!A || !b) { free(A); free(b); return 2; }
  double means[ORACLE_MAX_DIM], rdiag[ORACLE_MAX_DIM];
  for (int c = 0; c < d; ++c) {
    const double *col = X + (int64_t)tup[c] * n_total + lo;
    double s = 0.0;
    for (int64_t i = 0; i < nt; ++i) s += col[i];
    means[c] = s / (double)nt;
    for (int64_t i = 0; i < nt; ++i) A[(int64_t)c * nt + i] = col[i] - means[c];
  }
  double s = 0.0;
  for (int64_t i = 0; i < nt; ++i) s += y[lo + i];
  double ymean = s / (double)nt;
  for (int64_t i = 0; i < nt; ++i) b[i] = y[lo + i] - ymean;
  householder_lsq(A, nt, d, b, rdiag);
  double beta[ORACLE_MAX_DIM];
  for (int r = d - 1; r >= 0; --r) {
    double acc = b[r];
    for (int c = r + 1; c < d; ++c) acc -= A[(int64_t)c * nt + r] * beta[c];
    beta[r] = acc / rdiag[r];
  }
  double b0 = ymean;
  for (int c = 0; c < d; ++c) b0 -= beta[c] * means[c];
  out_coef[0] = b0;
  for (int c = 0; c < d; ++c) out_coef[1 + c] = beta[c];
  free(A);
  free(b);
  return 0;
}

/* Exhaustive l0 search.  shared_mode 0 = PER_TASK (n_out = n_tasks),
 * 1 = SHARED (n_out = 1).  Outputs: out_tuples [n_out][k][d] (-1 padding),
 * out_score [n_out][k] (+inf padding), out_rmse [n_out][k],
 * out_n_eligible [n_out]. */
int oracle_l0_fit(const double *X, const double *y, const int64_t *offsets,
                  int n_tasks, int64_t m, int d, int k, int shared_mode,
                  double rho_min, int n_threads, int32_t *out_tuples,
                  double *out_score, double *out_rmse,
                  int64_t *out_n_eligible) {
  if (validate(offsets, n_tasks, m, d) || k < 1) return 1;
  centred_t C;
  memset(&C, 0, sizeof(C));
  if (centred_make(&C, X, y, offsets, n_tasks, m)) {
    centred_free(&C);
    return 2;
  }
  int n_out = shared_mode ? 1 : n_tasks;
  int64_t n_total = offsets[n_tasks];
  int64_t nmax = 0;
  for (int t = 0; t < n_tasks; ++t)
    if (offsets[t + 1] - offsets[t] > nmax) nmax = offsets[t + 1] - offsets[t];

  int nthr = 1;
#ifdef _OPENMP
  if (n_threads > 0) omp_set_num_threads(n_threads);
  nthr = omp_get_max_threads();
#endif
  topk_t *lists = (topk_t *)calloc((size_t)(nthr * n_out), sizeof(topk_t));
  int64_t *elig = (int64_t *)calloc((size_t)(nthr * n_out), sizeof(int64_t));
  for (int q = 0; q < nthr * n_out; ++q) {
    lists[q].k = k;
    lists[q].d = d;
    lists[q].n = 0;
    lists[q].score = (double *)malloc(sizeof(double) * (size_t)k);
    lists[q].tup = (int32_t *)malloc(sizeof(int32_t) * (size_t)(k * d));
  }

#ifdef _OPENMP
#pragma omp parallel
#endif
  {
    int tid = 0;
#ifdef _OPENMP
    tid = omp_get_thread_num();
#endif
    double *A = (double *)malloc(sizeof(double) * (size_t)(nmax * d));
    double *b = (double *)malloc(sizeof(double) * (size_t)nmax);
    double *sse_t = (double *)malloc(sizeof(double) * (size_t)n_tasks);
    double *rho_t = (double *)malloc(sizeof(double) * (size_t)n_tasks);
    int32_t tup[ORACLE_MAX_DIM];
    /* parallel over the first index; the rest enumerated lexicographically */
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 1)
#endif
    for (int64_t first = 0; first <= m - d; ++first) {
      tup[0] = (int32_t)first;
      for (int c = 1; c < d; ++c) tup[c] = (int32_t)(first + c);
      for (;;) {
        int eligible = 1;
        double total = 0.0;
        for (int t = 0; t < n_tasks; ++t) {
          int64_t nt = offsets[t + 1] - offsets[t];
          sse_t[t] = score_tuple_task(C.xc[t], C.yc[t], nt, C.colnorm[t], tup,
                                      d, A, b, &rho_t[t]);
          if (!(rho_t[t] >= rho_min)) eligible = 0;
          total += sse_t[t];
        }
        if (shared_mode) {
          /* SHARED: ineligible when rank deficient in any task */
          if (eligible) {
            elig[tid * n_out]++;
            topk_push(&lists[tid * n_out], total / (double)n_total, tup);
          }
        } else {
          /* PER_TASK: each task ranks on its own */
          for (int t = 0; t < n_tasks; ++t) {
            if (rho_t[t] >= rho_min) {
              elig[tid * n_out + t]++;
              topk_push(&lists[tid * n_out + t], sse_t[t], tup);
            }
          }
        }
        /* next tuple with the same first index, lexicographic */
        int c = d - 1;
        while (c >= 1 && tup[c] == (int32_t)(m - d + c)) --c;
        if (c < 1) break;
        tup[c]++;
        for (int e = c + 1; e < d; ++e) tup[e] = tup[e - 1] + 1;
      }
    }
    free(A);
    free(b);
    free(sse_t);
    free(rho_t);
  }

  /* merge per-thread lists */
  for (int o = 0; o < n_out; ++o) {
    topk_t fin;
    fin.k = k;
    fin.d = d;
    fin.n = 0;
    fin.score = (double *)malloc(sizeof(double) * (size_t)k);
    fin.tup = (int32_t *)malloc(sizeof(int32_t) * (size_t)(k * d));
    int64_t ne = 0;
    for (int th = 0; th < nthr; ++th) {
      topk_t *L = &lists[th * n_out + o];
      for (int i = 0; i < L->n; ++i)
        topk_push(&fin, L->score[i], L->tup + (int64_t)i * d);
      ne += elig[th * n_out + o];
    }
    out_n_eligible[o] = ne;
    int64_t nt = shared_mode ? n_total : (offsets[o + 1] - offsets[o]);
    for (int i = 0; i < k; ++i) {
      if (i < fin.n) {
        out_score[(int64_t)o * k + i] = fin.score[i];
        double msd = shared_mode ? fin.score[i] : fin.score[i] / (double)nt;
        out_rmse[(int64_t)o * k + i] = sqrt(msd);
        memcpy(out_tuples + ((int64_t)o * k + i) * d,
               fin.tup + (int64_t)i * d, sizeof(int32_t) * (size_t)d);
      } else {
        out_score[(int64_t)o * k + i] = INFINITY;
        out_rmse[(int64_t)o * k + i] = INFINITY;
        for (int c = 0; c < d; ++c) out_tuples[((int64_t)o * k + i) * d + c] = -1;
      }
    }
    free(fin.score);
    free(fin.tup);
  }
  for (int q = 0; q < nthr * n_out; ++q) {
    free(lists[q].score);
    free(lists[q].tup);
  }
  free(lists);
  free(elig);
  centred_free(&C);
  return 0;
}

int oracle_max_dim(void) { return ORACLE_MAX_DIM; }
