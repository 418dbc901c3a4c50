// l0_select.cu -- grid top-K' merge, FP64 re-fit of the candidates from the
// raw columns, final ranking and the candidate-pool certificate.
#include <cfloat>

#include "l0_kernels.cuh"

namespace l0 {

namespace {

// ------------------------------------------------------------------ merge --
// Stream n entries (s, k) through the CTA list: one entry per thread per
// round, fold after every round (redo the round on overflow).
template <typename R>
__device__ void stream_entries(CtaList<R> &L, const R *s, const u64 *k, int n) {
  for (int base = 0; base < n; base += blockDim.x) {
    const int i = base + threadIdx.x;
    R sv = r_inf<R>();
    u64 kv = ~0ull;
    if (i < n) { sv = s[i]; kv = k[i]; }
    int redo = 0;
    do {
      if (i < n && cta_list_admits<R>(L, sv, kv)) cta_list_push<R>(L, sv, kv);
      __syncthreads();
      if (++redo > L0_MAX_REDO) break;
    } while (cta_list_fold<R>(L, nullptr));
  }
}

// exclusive prefix sum of one int per thread over the CTA (blockDim a
// multiple of 32, at most 1024); *total gets the sum.  ws: [32] shared.
__device__ int block_excl_scan(int v, int *ws, int *total) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  int inc = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int t = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += t;
  }
  if (lane == 31) ws[w] = inc;
  __syncthreads();
  if (w == 0) {
    int x = lane < nw ? ws[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += t;
    }
    if (lane < nw) ws[lane] = x;   // inclusive warp totals
  }
  __syncthreads();
  const int before = (w > 0 ? ws[w - 1] : 0) + inc - v;
  *total = ws[nw - 1];
  __syncthreads();   // ws is free again
  return before;
}

// Gather the prefix (score <= cut) of n_lists sorted lists into shared
// memory (up to cap entries), sort once, keep the first K.  Returns the
// number kept, or -1 when more than cap entries qualified (nothing written).
// With at most blockDim lists, thread l finds list l's prefix (all searches
// in flight together), a scan places the prefixes, and each thread copies
// entries found by a search of the placements; otherwise one warp per list.
// off: [blockDim + 1] ints of shared scratch.
template <typename R>
__device__ int gather_sort_lists(const R *ls_base, const u64 *lk_base, const int *cnt,
                                 size_t stride, int n_lists, R cut, int K, int cap, R *ss,
                                 u64 *sk, R *out_s, u64 *out_k, int *s_tot, int *off) {
  __shared__ int ws[32];
  int total = 0;
  if (n_lists <= (int)blockDim.x) {
    const int l = threadIdx.x;
    int lo = 0;
    if (l < n_lists) {
      const R *ls = ls_base + (size_t)l * stride;
      int hi = cnt[l];
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (ls[mid] <= cut) lo = mid + 1; else hi = mid;
      }
    }
    const int before = block_excl_scan(lo, ws, &total);
    off[threadIdx.x] = before;
    if (threadIdx.x == blockDim.x - 1) off[blockDim.x] = total;
    __syncthreads();
    if (total > cap) return -1;
    for (int e = threadIdx.x; e < total; e += blockDim.x) {
      // the list holding placement e: last l with off[l] <= e
      int a = 0, b = n_lists - 1;
      while (a < b) {
        const int mid = (a + b + 1) >> 1;
        if (off[mid] <= e) a = mid; else b = mid - 1;
      }
      const int i = e - off[a];
      ss[e] = ls_base[(size_t)a * stride + i];
      sk[e] = lk_base[(size_t)a * stride + i];
    }
  } else {
    if (threadIdx.x == 0) *s_tot = 0;
    __syncthreads();
    // one warp per list: binary search of the prefix, then copy
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int l = warp; l < n_lists; l += nw) {
      const R *ls = ls_base + (size_t)l * stride;
      const u64 *lk = lk_base + (size_t)l * stride;
      int lo = 0, hi = cnt[l];
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (ls[mid] <= cut) lo = mid + 1; else hi = mid;
      }
      int base = 0;
      if (lane == 0 && lo > 0) base = atomicAdd(s_tot, lo);
      base = __shfl_sync(0xffffffffu, base, 0);
      for (int i = lane; i < lo; i += 32) {
        if (base + i < cap) {
          ss[base + i] = ls[i];
          sk[base + i] = lk[i];
        }
      }
    }
    __syncthreads();
    total = *s_tot;
    if (total > cap) return -1;
  }
  int P = 1;
  while (P < total) P <<= 1;
  for (int i = total + threadIdx.x; i < P; i += blockDim.x) {
    ss[i] = r_inf<R>();
    sk[i] = ~0ull;
  }
  __syncthreads();
  cta_bitonic_sort<R>(ss, sk, P);
  const int nout = total < K ? total : K;
  for (int i = threadIdx.x; i < nout; i += blockDim.x) {
    out_s[i] = ss[i];
    out_k[i] = sk[i];
  }
  __syncthreads();
  return nout;
}

// Streaming fallback: the same prefixes through a CTA list.
template <typename R>
__device__ int stream_lists(const R *ls_base, const u64 *lk_base, const int *cnt, size_t stride,
                            int n_lists, R cut, unsigned char *smem, int K, int S, R *out_s,
                            u64 *out_k) {
  unsigned char *p = smem;
  CtaList<R> L = cta_list_carve<R>(p, K, S);
  cta_list_reset<R>(L, nullptr);
  __syncthreads();
  for (int l = 0; l < n_lists; ++l) {
    const R *ls = ls_base + (size_t)l * stride;
    int lo = 0, hi = cnt[l];
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (ls[mid] <= cut) lo = mid + 1; else hi = mid;
    }
    if (lo > 0) stream_entries<R>(L, ls, lk_base + (size_t)l * stride, lo);
  }
  const int n = *(volatile int *)L.n_list;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    out_s[i] = L.ls[i];
    out_k[i] = L.lk[i];
  }
  __syncthreads();
  return n;
}

// grid (groups, n_probs), 1024 threads.  With one group the CTA of a problem
// gathers every slot list's qualifying prefix, sorts once and writes the
// pool.  Otherwise: the slot lists are sorted and only
// their prefixes at or below the search threshold g can reach the pool.
// Level 1: CTA x sorts the qualifying entries of its share of slots and keeps
// its best K' (a partial list); a full partial's K'-th score is a tighter
// bound g2 (atomicMin).  Level 2: the last CTA of the problem (counter, no
// waiting) gathers the partial prefixes <= g2, sorts them once and keeps K'.
template <typename R>
__global__ void __launch_bounds__(1024, 1)
merge_kernel(const R *in_s, const u64 *in_k, const int *in_cnt, int n_slots,
             int K, int S, const u64 *gthr, R *part_s, u64 *part_k, int *part_cnt, int cap,
             unsigned *counters, R *pool_s, u64 *pool_k, int *pool_cnt) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int s_last, s_tot;
  __shared__ int s_off[1025];
  const int prob = blockIdx.y, g = blockIdx.x, G = gridDim.x;
  unsigned *done = counters + 4 * prob;
  u64 *g2 = (u64 *)(counters + 4 * prob + 2);
  R *ss = (R *)smem;
  u64 *sk = (u64 *)(smem + (size_t)cap * sizeof(R));
  const R gcut = from_ord<R>(gthr[prob]);
  const int a = (int)((long long)n_slots * g / G);
  const int b = (int)((long long)n_slots * (g + 1) / G);
  const size_t pslot = (size_t)prob * G + g;
  R *ps = part_s + pslot * K;
  u64 *pk = part_k + pslot * K;
  const size_t s0 = (size_t)prob * n_slots + a;
  if (G == 1) {   // one CTA per problem: straight into the pool
    R *os = pool_s + (size_t)prob * K;
    u64 *ok = pool_k + (size_t)prob * K;
    int n1 = gather_sort_lists<R>(in_s + s0 * K, in_k + s0 * K, in_cnt + s0, (size_t)K, b - a,
                                  gcut, K, cap, ss, sk, os, ok, &s_tot, s_off);
    if (n1 < 0)
      n1 = stream_lists<R>(in_s + s0 * K, in_k + s0 * K, in_cnt + s0, (size_t)K, b - a, gcut,
                           smem, K, S, os, ok);
    if (threadIdx.x == 0) pool_cnt[prob] = n1;
    return;
  }
  int n = gather_sort_lists<R>(in_s + s0 * K, in_k + s0 * K, in_cnt + s0, (size_t)K, b - a,
                               gcut, K, cap, ss, sk, ps, pk, &s_tot, s_off);
  if (n < 0)
    n = stream_lists<R>(in_s + s0 * K, in_k + s0 * K, in_cnt + s0, (size_t)K, b - a, gcut, smem,
                        K, S, ps, pk);
  if (threadIdx.x == 0) {
    part_cnt[pslot] = n;
    if (n >= K) atomicMin(g2, ord_of(ps[K - 1]));
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = (atomicAdd(done, 1u) == (unsigned)(G - 1));
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  R cut2 = from_ord<R>(*(volatile u64 *)g2);
  if (gcut < cut2) cut2 = gcut;
  const size_t p0 = (size_t)prob * G;
  R *os = pool_s + (size_t)prob * K;
  u64 *ok = pool_k + (size_t)prob * K;
  int n2 = gather_sort_lists<R>(part_s + p0 * K, part_k + p0 * K, part_cnt + p0, (size_t)K, G,
                                cut2, K, cap, ss, sk, os, ok, &s_tot, s_off);
  if (n2 < 0)
    n2 = stream_lists<R>(part_s + p0 * K, part_k + p0 * K, part_cnt + p0, (size_t)K, G, cut2,
                         smem, K, S, os, ok);
  if (threadIdx.x == 0) {
    pool_cnt[prob] = n2;
    *done = 0u;
    *g2 = ord_inf<R>();
  }
}

// ------------------------------------------------------------------ re-fit --
constexpr int REFIT_THREADS = 128;

// sum (or max) of nv values per thread over the CTA; every thread gets the
// results.  red: [REFIT_THREADS / 32][L0_DMAX + 1]
__device__ void block_reduce(double *v, int nv, bool take_max, double (*red)[L0_DMAX + 1]) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int i = 0; i < nv; ++i) {
    double x = v[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double y = __shfl_xor_sync(0xffffffffu, x, o);
      x = take_max ? fmax(x, y) : x + y;
    }
    if (lane == 0) red[w][i] = x;
  }
  __syncthreads();
  for (int i = 0; i < nv; ++i) {
    double x = red[0][i];
    for (int q = 1; q < REFIT_THREADS / 32; ++q) x = take_max ? fmax(x, red[q][i]) : x + red[q][i];
    v[i] = x;
  }
  __syncthreads();
}

// Householder least squares of one task's rows (paper Sec. 2.4: QR by
// Householder reflections, least-squares fit, squared deviation) by one CTA.
// A holds the d centred columns and the centred target as column d, each of
// length n; row i is owned by thread i mod REFIT_THREADS.  Each reflection
// takes one pass over the rows for the norm of its column and the dot
// products with the later columns, and one pass for the update.  Norms are
// plain sums of squares (FP64 holds the squares of any centred value below
// 1e150; a column whose sum overflows is rescaled by its maximum first).
// Returns SSE; *rho = min_j |R_jj| / ||a_j||.
__device__ double norm_scaled(const double *a, long long lo, long long n,
                              double (*red)[L0_DMAX + 1]) {
  double v[1] = {0.0};
  for (long long i = lo + threadIdx.x; i < n; i += REFIT_THREADS) v[0] = fmax(v[0], fabs(a[i]));
  block_reduce(v, 1, true, red);
  const double m1 = v[0];
  if (!(m1 > 0.0)) return 0.0;
  const double im1 = 1.0 / m1;
  v[0] = 0.0;
  for (long long i = lo + threadIdx.x; i < n; i += REFIT_THREADS) { const double q = a[i] * im1; v[0] += q * q; }
  block_reduce(v, 1, false, red);
  return m1 * sqrt(v[0]);
}

// Sum over the CTA of nv per-thread partials, by warp 0 alone: an FP64
// instruction costs the SM the same whatever its active lanes (measured:
// one warp instruction per ~20 cycles), so the cross-thread sums and the
// scalar work that follows run once per CTA, not in every warp.  The sums
// are returned in v[] of warp 0's threads (lane 0 is the one that uses
// them).  part: [REFIT_NV][REFIT_THREADS] shared.
constexpr int REFIT_NV = 2 * L0_DMAX;
static_assert(REFIT_THREADS == 128, "four partials per lane of warp 0");
__device__ void sum_warp0(double *v, int nv, double *part) {
  const int tid = threadIdx.x, lane = tid & 31;
  for (int i = 0; i < nv; ++i) part[i * REFIT_THREADS + tid] = v[i];
  __syncthreads();
  if (tid < 32)
    for (int i = 0; i < nv; ++i) {
      const double *q = part + i * REFIT_THREADS;
      double x = (q[lane] + q[lane + 32]) + (q[lane + 64] + q[lane + 96]);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
      v[i] = x;
    }
}

// sc: shared scalars, [2 * L0_DMAX + 8]: [0] rescale sigma, [1..d) rescale
// the norm of original column c, [5] skip the update, [8..8+nc) the update
// coefficients of the later columns.  Thread 0 returns SSE and *rho.
__device__ double householder_cta(double *A, long long n, int d, double (*red)[L0_DMAX + 1],
                                  double *part, double *sc, double *rho) {
  const int tid = threadIdx.x;
  double v[REFIT_NV], cn[L0_DMAX];
  double r = DBL_MAX;
  for (int j = 0; j < d; ++j) {
    double *aj = A + (long long)j * n;
    const int nc = d - j;                 // columns j+1 .. d (the target is column d)
    const int nn = (j == 0) ? d - 1 : 0;  // first pass: norms of the original columns 1..d-1
    // one pass: ||aj[j..n)||^2, aj[j+1..n) . ac[j+1..n) for the later columns
    // (and, in the first pass, ||ac||^2 of the original feature columns)
    for (int c = 0; c <= nc + nn; ++c) v[c] = 0.0;
    for (long long i = j + tid; i < n; i += REFIT_THREADS) {
      const double ai = aj[i];
      v[nc] = fma(ai, ai, v[nc]);
      if (i > j)
        for (int c = 0; c < nc; ++c) v[c] = fma(ai, A[(long long)(j + 1 + c) * n + i], v[c]);
      for (int c = 0; c < nn; ++c) {
        const double x = A[(long long)(1 + c) * n + i];
        v[nc + 1 + c] = fma(x, x, v[nc + 1 + c]);
      }
    }
    sum_warp0(v, nc + 1 + nn, part);
    if (tid == 0) {
      sc[0] = isfinite(v[nc]) ? 0.0 : 1.0;
      for (int c = 0; c < nn; ++c) sc[1 + c] = isfinite(v[nc + 1 + c]) ? 0.0 : 1.0;
    }
    __syncthreads();
    // sums of squares that overflowed: rescaled by their column maxima (rare;
    // the whole CTA)
    double sigma = 0.0;
    if (sc[0] != 0.0) {
      sigma = norm_scaled(aj, j, n, red);
    } else if (tid == 0) {
      sigma = sqrt(v[nc]);
    }
    for (int c = 0; c < nn; ++c) {
      if (sc[1 + c] != 0.0) {
        const double t = norm_scaled(A + (long long)(1 + c) * n, 0, n, red);
        if (tid == 0) cn[1 + c] = t;
      } else if (tid == 0) {
        cn[1 + c] = sqrt(v[nc + 1 + c]);
      }
    }
    if (tid == 0) {
      if (j == 0) cn[0] = sigma;   // nothing has touched column 0 yet
      if (sigma == 0.0) {
        r = 0.0;
        sc[5] = 1.0;
      } else {
        const double x0 = aj[j];
        const double alpha = (x0 >= 0.0) ? -sigma : sigma;
        const double v0 = x0 - alpha;
        const double beta = 1.0 / (sigma * (sigma + fabs(x0)));
        for (int c = 0; c < nc; ++c) {
          double *ac = A + (long long)(j + 1 + c) * n;
          const double sdot = (v[c] + v0 * ac[j]) * beta;
          sc[8 + c] = sdot;
          ac[j] -= sdot * v0;   // row j of the reflected column (rows > j below)
        }
        r = fmin(r, (cn[j] > 0.0) ? fabs(alpha) / cn[j] : 0.0);
        sc[5] = 0.0;
      }
    }
    __syncthreads();
    if (sc[5] == 0.0)
      for (int c = 0; c < nc; ++c) {
        double *ac = A + (long long)(j + 1 + c) * n;
        const double sdot = sc[8 + c];
        for (long long i = j + 1 + tid; i < n; i += REFIT_THREADS) ac[i] -= sdot * aj[i];
      }
    __syncthreads();
  }
  const double *b = A + (long long)d * n;
  v[0] = 0.0;
  for (long long i = d + tid; i < n; i += REFIT_THREADS) v[0] = fma(b[i], b[i], v[0]);
  sum_warp0(v, 1, part);
  *rho = r;
  return v[0];
}

// grid (K, n_probs), REFIT_THREADS threads: one CTA per candidate.  The
// columns live in dynamic shared memory when they fit (a.smem_rows), else in
// the global scratch.
__global__ void __launch_bounds__(REFIT_THREADS)
refit_kernel(RefitArgs a) {
  extern __shared__ __align__(16) double sA[];
  __shared__ double red[REFIT_THREADS / 32][L0_DMAX + 1];
  __shared__ double s_part[REFIT_NV * REFIT_THREADS];
  __shared__ double s_sc[2 * L0_DMAX + 8];
  __shared__ int s_t[L0_DMAX];
  const int prob = blockIdx.y, cidx = blockIdx.x;
  const ProbDesc pd = a.probs[prob];
  const int cnt = a.pool_cnt[prob];
  if (cidx >= refit_count(pd.k, a.K, cnt, a.refit_all)) return;
  const int d = pd.d;
  if (threadIdx.x == 0) {
    int t[L0_DMAX];
    lex_unrank(a.B, pd.m, d, a.pool_k[(size_t)prob * a.K + cidx], pd.total, t);
    for (int q = 0; q < d; ++q) s_t[q] = t[q];
  }
  __syncthreads();
  double *A = a.smem_rows ? sA
                          : a.scratch + ((size_t)prob * a.K + cidx) * (size_t)(d + 1) * a.nmax;
  const int t_lo = a.shared ? 0 : pd.task;
  const int t_hi = a.shared ? a.T : pd.task + 1;
  double total = 0.0;
  bool elig = true;
  for (int tk = t_lo; tk < t_hi; ++tk) {
    const long long lo = a.offsets[tk], hi = a.offsets[tk + 1], n = hi - lo;
    const double *mu = a.mu + (size_t)tk * (a.m + 1);
    // centred columns into A: eight loads in flight per thread per column
    for (int q = 0; q <= d; ++q) {
      const double *src = (q < d) ? a.X + (long long)s_t[q] * a.n_total + lo : a.y + lo;
      const double mean = (q < d) ? mu[s_t[q] + 1] : mu[0];
      double *dst = A + (long long)q * n;
      for (long long i0 = threadIdx.x; i0 < n; i0 += 8 * REFIT_THREADS) {
        double v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const long long i = i0 + (long long)u * REFIT_THREADS;
          v[u] = (i < n) ? __ldg(src + i) : 0.0;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const long long i = i0 + (long long)u * REFIT_THREADS;
          if (i < n) dst[i] = v[u] - mean;
        }
      }
    }
    __syncthreads();
    double rho;
    total += householder_cta(A, n, d, red, s_part, s_sc, &rho);
    if (!(rho >= a.rho_min)) elig = false;
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    double score = total;
    if (a.shared) score = total / (double)a.offsets[a.T];
    a.refit[(size_t)prob * a.K + cidx] = elig ? score : __longlong_as_double(0x7ff0000000000000ll);
  }
}

// ---------------------------------------------------------- block helpers --
__device__ double block_max(double v, double *red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
  for (int i = 0; i < nw; ++i) s = fmax(s, red[i]);
  return s;
}

// --------------------------------------------------------------- select --
// One CTA per problem: sort the pool by (refit score, key), emit the best k,
// and evaluate the certificate.
template <typename R>
__global__ void __launch_bounds__(256)
select_kernel(SelectArgs<R> a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int prob = blockIdx.x;
  const ProbDesc pd = a.probs[prob];
  const int cnt_pool = a.pool_cnt[prob];
  // only the re-fitted head of the (search-score sorted) pool is ranked
  const int cnt = refit_count(pd.k, a.K, cnt_pool, a.refit_all);
  int P = 1;
  while (P < a.K) P <<= 1;
  double *ss = (double *)smem;
  u64 *sk = (u64 *)(ss + P);
  double *us = (double *)(sk + P);   // the head as read (rank-by-counting input)
  u64 *uk = (u64 *)(us + P);
  const bool by_rank = cnt <= 1024;
  __shared__ double red[32];
  double scale = 1.0;
  if (!a.shared) {
    const double is = a.inv_s[(size_t)pd.task * a.mp1];
    scale = (is > 0.0) ? 1.0 / (is * is) : 0.0;
  }
  double dmax = 0.0;
  double *ws = by_rank ? us : ss;
  u64 *wk = by_rank ? uk : sk;
  for (int i = threadIdx.x; i < P; i += blockDim.x) {
    if (i < cnt) {
      const double rf = a.refit[(size_t)prob * a.K + i];
      // ranking by counting compares order-preserving integer images of the
      // scores (on this part a double comparison runs on the narrow FP64 pipe)
      if (by_rank) ((u64 *)ws)[i] = ord_of(rf);
      else ws[i] = rf;
      wk[i] = a.pool_k[(size_t)prob * a.K + i];
      if (isfinite(rf)) {
        const double gs = (double)a.pool_s[(size_t)prob * a.K + i] * scale;
        dmax = fmax(dmax, fabs(gs - rf));
      }
    } else {
      ss[i] = __longlong_as_double(0x7ff0000000000000ll);
      sk[i] = ~0ull;
    }
  }
  __syncthreads();
  if (by_rank) {
    // keys are unique, so each entry's rank -- the count of entries before
    // it in (score, key) order -- is its place: one pass, one barrier
    const u64 *uo = (const u64 *)us;
    for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
      const u64 o_i = uo[i];
      const u64 k_i = uk[i];
      int r = 0;
      for (int j = 0; j < cnt; ++j) {
        const u64 o_j = uo[j];
        r += (o_j < o_i || (o_j == o_i && uk[j] < k_i)) ? 1 : 0;
      }
      ss[r] = from_ord<double>(o_i);
      sk[r] = k_i;
    }
    __syncthreads();
  } else {
    cta_bitonic_sort<double>(ss, sk, P);
  }
  dmax = block_max(dmax, red);
  int nv_local = 0;
  for (int i = threadIdx.x; i < cnt; i += blockDim.x) nv_local += isfinite(ss[i]) ? 1 : 0;
  __shared__ int s_valid;
  if (threadIdx.x == 0) s_valid = 0;
  __syncthreads();
  if (nv_local) atomicAdd(&s_valid, nv_local);
  __syncthreads();
  const int nvalid = s_valid;
  const int d = pd.d, kq = pd.k;
  const double div = a.rmse_div[prob];
  for (int i = threadIdx.x; i < kq; i += blockDim.x) {
    int *ot = a.out_tuples + pd.out_t_off + (size_t)i * d;
    double *orr = a.out_rmse + pd.out_r_off + i;
    if (i < nvalid) {
      int t[L0_DMAX];
      lex_unrank(a.B, pd.m, d, sk[i], pd.total, t);
      for (int q = 0; q < d; ++q) ot[q] = t[q];
      *orr = sqrt(fmax(ss[i], 0.0) / div);
    } else {
      for (int q = 0; q < d; ++q) ot[q] = -1;
      *orr = __longlong_as_double(0x7ff0000000000000ll);
    }
  }
  if (threadIdx.x == 0) {
    CertOut c;
    c.delta = dmax;
    c.pool_cnt = cnt_pool;
    c.pool_full = (cnt_pool >= a.K) ? 1 : 0;
    c.n_valid = nvalid;
    // Tuples outside the pool were either cut by the search threshold (their
    // Gram score exceeded it, and it only ever decreased to its final value
    // g) or lost to the pool's K'-th entry when the pool is full.  So every
    // outside tuple has a Gram score >= bound = min(g, pool K'-th).
    // Pool entries past the re-fitted head have search scores >= that of the
    // first one left out (the pool is sorted by search score).
    const double g = (double)from_ord<R>(a.gthr[prob]);
    double bound = g;
    if (c.pool_full) bound = fmin(bound, (double)a.pool_s[(size_t)prob * a.K + cnt_pool - 1]);
    if (cnt < cnt_pool) bound = fmin(bound, (double)a.pool_s[(size_t)prob * a.K + cnt]);
    const double inf = __longlong_as_double(0x7ff0000000000000ll);
    c.pool_worst = isinf(bound) ? inf : bound * scale;
    c.kth_refit = (nvalid >= kq) ? ss[kq - 1] : inf;
    // The check assumes that no outside tuple's search score is off by more
    // than safety * delta, delta being the largest error measured on the
    // pool (the tuples next to the excluded ones in score).  That is an
    // empirical premise, not a proof: the excluded tuples were never
    // re-fitted, and an ill-conditioned one (pivot ratio just above the FP64
    // redo cut) can carry a larger error.  Under it, every outside tuple's
    // exact score is at least bound - safety * delta, and the pool holds the
    // exact top k when that clears the k-th re-fitted score; trivially so
    // when nothing was excluded at all.
    if (isinf(bound)) c.certified = 1;
    else c.certified = (c.pool_worst - a.cert_safety * dmax >= c.kth_refit) ? 1 : 0;
    if (a.delta_floor) {
      // Band pass: a tuple the FP32 test never flagged scored above the band
      // cut in FP32, so the previous pass's error bound applies to it; one it
      // flagged was scored in FP64 and is bounded as above (delta measured
      // on this pass's pool).  Both must clear the k-th re-fitted score.
      const double df = a.delta_floor[prob];
      const double band = (double)from_ord<float>(a.band_thr[prob]) * scale;
      if (isfinite(band) && !(band - a.cert_safety * df >= c.kth_refit)) c.certified = 0;
      if (!isfinite(band)) c.certified = 0;
      c.delta = fmax(dmax, df);   // a further band pass keeps the FP32 error bound
    }
    a.cert[prob] = c;
  }
}

// Band pass cut per problem (one thread each): the previous pass re-fitted
// its pool in FP64 and measured delta, the largest search-score error on it.
// Tuples whose FP32 score lies below kth + margin * delta (relative units,
// rounded up to FP32) are the ones the FP32 search cannot rank: the band
// pass scores all of them in FP64.  No finite k-th (too few eligible tuples
// in the pool): no cut, +inf.
__global__ void band_cut_kernel(const CertOut *cert, const ProbDesc *probs, int n_probs,
                                const double *inv_s, int mp1, int shared, double margin,
                                u64 *band_thr, double *delta_floor) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n_probs) return;
  const CertOut c = cert[q];
  double scale = 1.0;   // SSE units per unit of search score
  if (!shared) {
    const double is = inv_s[(size_t)probs[q].task * mp1];
    scale = (is > 0.0) ? 1.0 / (is * is) : 0.0;
  }
  const double cut = (scale > 0.0) ? (c.kth_refit + margin * c.delta) / scale
                                   : __longlong_as_double(0x7ff0000000000000ll);
  const float cf = isfinite(cut) ? __double2float_ru(cut) : __int_as_float(0x7f800000);
  band_thr[q] = ord_of(cf);
  delta_floor[q] = c.delta;
}

__global__ void unrank_kernel(Binom B, int m, int d, u64 total, const u64 *ranks,
                              long long count, int *tuples) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  int t[L0_DMAX];
  lex_unrank_arith(m, d, ranks[i], total, t);
  for (int q = 0; q < d; ++q) tuples[i * d + q] = t[q];
}

__global__ void __launch_bounds__(1024)
merge_shards_kernel(Binom B, int m, int d, u64 total, int k, double n_rows, const u64 *keys,
                    const double *sse, long long n_cand, int P, const double *bounds,
                    const double *deltas, int n_shards, double *ss, u64 *sk, int *out_tuples,
                    double *out_rmse, int *certified) {
  const double inf = __longlong_as_double(0x7ff0000000000000ll);
  for (int i = threadIdx.x; i < P; i += blockDim.x) {
    ss[i] = (i < n_cand) ? sse[i] : inf;
    sk[i] = (i < n_cand) ? keys[i] : ~0ull;
  }
  __syncthreads();
  cta_bitonic_sort<double>(ss, sk, P);
  for (int i = threadIdx.x; i < k; i += blockDim.x) {
    int *ot = out_tuples + (size_t)i * d;
    if (i < P && isfinite(ss[i])) {
      int t[L0_DMAX];
      lex_unrank_arith(m, d, sk[i], total, t);
      for (int q = 0; q < d; ++q) ot[q] = t[q];
      out_rmse[i] = sqrt(fmax(ss[i], 0.0) / n_rows);
    } else {
      for (int q = 0; q < d; ++q) ot[q] = -1;
      out_rmse[i] = inf;
    }
  }
  if (threadIdx.x == 0) {
    // every shard's pool holds all of its tuples whose exact SSE is below
    // its bound - 4 delta; the merged k-th must clear the smallest of these
    double worst = inf;
    for (int q = 0; q < n_shards; ++q) {
      const double b = bounds[q];
      if (!isinf(b)) worst = fmin(worst, b - 4.0 * deltas[q]);
    }
    const double kth = (k <= P) ? ss[k - 1] : inf;
    *certified = (isinf(worst) || worst >= kth) ? 1 : 0;
  }
}

}  // namespace

cudaError_t launch_merge_shards(const Binom &B, int m, int d, u64 total, int k, double n_rows,
                                const u64 *keys, const double *sse, long long n_cand,
                                const double *bounds, const double *deltas, int n_shards,
                                double *scratch_s, u64 *scratch_k, int *out_tuples,
                                double *out_rmse, int *certified, cudaStream_t st) {
  int P = 1;
  while (P < n_cand || P < k) P <<= 1;
  merge_shards_kernel<<<1, 1024, 0, st>>>(B, m, d, total, k, n_rows, keys, sse, n_cand, P, bounds,
                                          deltas, n_shards, scratch_s, scratch_k, out_tuples,
                                          out_rmse, certified);
  return cudaGetLastError();
}

template <typename R>
size_t merge_smem_bytes(int K, int S, int cap) {
  size_t a = (size_t)cap * (sizeof(R) + 8);
  size_t b = cta_list_bytes<R>(K, S);
  return (a > b ? a : b) + 16;
}

template <typename R>
int merge_cap() { return sizeof(R) == 4 ? 16384 : 8192; }

template <typename R>
cudaError_t launch_merge(const R *in_s, const u64 *in_k, const int *in_cnt,
                         int n_slots, int n_probs, int K, int S, int groups, const u64 *gthr,
                         R *part_s, u64 *part_k, int *part_cnt, unsigned *counters,
                         R *pool_s, u64 *pool_k, int *pool_cnt, cudaStream_t st) {
  const int cap = merge_cap<R>();
  const size_t smem = merge_smem_bytes<R>(K, S, cap);
  cudaError_t e = cudaFuncSetAttribute(merge_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  merge_kernel<R><<<dim3(groups, n_probs), 1024, smem, st>>>(
      in_s, in_k, in_cnt, n_slots, K, S, gthr, part_s, part_k, part_cnt, cap, counters, pool_s,
      pool_k, pool_cnt);
  return cudaGetLastError();
}

cudaError_t launch_refit(const RefitArgs &a_in, cudaStream_t st) {
  RefitArgs a = a_in;
  const size_t bytes = (size_t)(a.dmax + 1) * (size_t)a.nmax * 8;
  a.smem_rows = bytes <= 200 * 1024 ? 1 : 0;
  const size_t smem = a.smem_rows ? bytes : 0;
  cudaError_t e = cudaFuncSetAttribute(refit_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)(smem > 0 ? smem : 16));
  if (e != cudaSuccess) return e;
  refit_kernel<<<dim3(a.K, a.n_probs), REFIT_THREADS, smem, st>>>(a);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_select(const SelectArgs<R> &a, cudaStream_t st) {
  int P = 1;
  while (P < a.K) P <<= 1;
  size_t smem = (size_t)P * 32;
  cudaError_t e = cudaFuncSetAttribute(select_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  select_kernel<R><<<a.n_probs, 256, smem, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_band_cut(const CertOut *cert, const ProbDesc *probs, int n_probs,
                            const double *inv_s, int mp1, int shared, double margin,
                            u64 *band_thr, double *delta_floor, cudaStream_t st) {
  band_cut_kernel<<<(n_probs + 127) / 128, 128, 0, st>>>(cert, probs, n_probs, inv_s, mp1,
                                                         shared, margin, band_thr, delta_floor);
  return cudaGetLastError();
}

cudaError_t launch_unrank(const Binom &B, int m, int d, u64 total, const u64 *ranks,
                          long long count, int *tuples, cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  unrank_kernel<<<(unsigned)((count + 255) / 256), 256, 0, st>>>(B, m, d, total, ranks,
                                                                 count, tuples);
  return cudaGetLastError();
}

template cudaError_t launch_merge<double>(const double *, const u64 *, const int *, int, int, int, int, int, const u64 *, double *, u64 *, int *, unsigned *, double *, u64 *, int *, cudaStream_t);
template cudaError_t launch_merge<float>(const float *, const u64 *, const int *, int, int, int, int, int, const u64 *, float *, u64 *, int *, unsigned *, float *, u64 *, int *, cudaStream_t);
template cudaError_t launch_select<double>(const SelectArgs<double> &, cudaStream_t);
template cudaError_t launch_select<float>(const SelectArgs<float> &, cudaStream_t);

}  // namespace l0
