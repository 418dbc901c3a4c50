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

// grid (groups, n_probs).  Phase 1: CTA g folds slots [g*n/G, (g+1)*n/G) of
// its problem into one list.  Phase 2: the last CTA of the problem to finish
// (counter, no waiting) folds the G partial lists into the pool.
template <typename R>
__global__ void __launch_bounds__(L0_THREADS)
merge_kernel(const R *in_s, const u64 *in_k, const int *in_cnt, int n_slots,
             int K, int S, R *part_s, u64 *part_k, int *part_cnt,
             unsigned *done, R *pool_s, u64 *pool_k, int *pool_cnt) {
  extern __shared__ __align__(16) unsigned char smem[];
  unsigned char *p = smem;
  CtaList<R> L = cta_list_carve<R>(p, K, S);
  __shared__ int s_last;
  const int prob = blockIdx.y, g = blockIdx.x, G = gridDim.x;
  cta_list_reset<R>(L, nullptr);
  __syncthreads();
  const int a = (int)((long long)n_slots * g / G);
  const int b = (int)((long long)n_slots * (g + 1) / G);
  for (int sl = a; sl < b; ++sl) {
    const size_t slot = (size_t)prob * n_slots + sl;
    const int n = in_cnt[slot];
    if (n > 0) stream_entries<R>(L, in_s + slot * K, in_k + slot * K, n);
  }
  const size_t ps = (size_t)prob * G + g;
  cta_list_flush<R>(L, part_s + ps * K, part_k + ps * K, part_cnt + ps);
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = (atomicAdd(done + prob, 1u) == (unsigned)(G - 1));
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  cta_list_reset<R>(L, nullptr);
  __syncthreads();
  for (int q = 0; q < G; ++q) {
    const size_t qs = (size_t)prob * G + q;
    const int n = *(volatile const int *)(part_cnt + qs);
    if (n > 0) stream_entries<R>(L, part_s + qs * K, part_k + qs * K, n);
  }
  cta_list_flush<R>(L, pool_s + (size_t)prob * K, pool_k + (size_t)prob * K, pool_cnt + prob);
  if (threadIdx.x == 0) done[prob] = 0u;
}

// ------------------------------------------------------------------ re-fit --
__device__ double block_sum(double v, double *red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
  for (int i = 0; i < nw; ++i) s += red[i];
  return s;
}

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

// scaled two-pass 2-norm of v[lo..n) (strided ownership by thread)
__device__ double block_norm(const double *v, long long lo, long long n, double *red) {
  double mx = 0.0;
  for (long long i = lo + threadIdx.x; i < n; i += blockDim.x) mx = fmax(mx, fabs(v[i]));
  mx = block_max(mx, red);
  if (mx == 0.0) return 0.0;
  double ss = 0.0;
  for (long long i = lo + threadIdx.x; i < n; i += blockDim.x) {
    double r = v[i] / mx;
    ss += r * r;
  }
  ss = block_sum(ss, red);
  return mx * sqrt(ss);
}

// Householder least squares of one task's rows (paper Sec. 2.4: QR by
// Householder reflections, least-squares fit, squared deviation).
// A holds d centred columns and the centred target as column d, each of
// length n, in global scratch.  Returns SSE; *rho = min |R_jj| / ||a_j||.
__device__ double householder_sse(double *A, long long n, int d, double *red,
                                  double *rho) {
  double cn[L0_DMAX];
  for (int j = 0; j < d; ++j) cn[j] = block_norm(A + (long long)j * n, 0, n, red);
  double r = DBL_MAX;
  __shared__ double s_dots[L0_DMAX + 1];
  for (int j = 0; j < d; ++j) {
    double *aj = A + (long long)j * n;
    const double sigma = block_norm(aj, j, n, red);
    __syncthreads();
    if (sigma == 0.0) {
      r = 0.0;
      continue;
    }
    const double x0 = aj[j];
    const double alpha = (x0 >= 0.0) ? -sigma : sigma;
    const double v0 = x0 - alpha;
    const double beta = 1.0 / (sigma * (sigma + fabs(x0)));
    // dots v^T a_c for c = j+1 .. d (the target is column d)
    for (int c = j + 1; c <= d; ++c) {
      const double *ac = A + (long long)c * n;
      double s = 0.0;
      for (long long i = j + 1 + threadIdx.x; i < n; i += blockDim.x) s += aj[i] * ac[i];
      s = block_sum(s, red);
      if (threadIdx.x == 0) s_dots[c] = (s + v0 * ac[j]) * beta;
    }
    __syncthreads();
    for (int c = j + 1; c <= d; ++c) {
      double *ac = A + (long long)c * n;
      const double s = s_dots[c];
      for (long long i = j + 1 + threadIdx.x; i < n; i += blockDim.x) ac[i] -= s * aj[i];
      if (threadIdx.x == 0) ac[j] -= s * v0;
    }
    __syncthreads();
    const double q = (cn[j] > 0.0) ? fabs(alpha) / cn[j] : 0.0;
    r = fmin(r, q);
  }
  const double *b = A + (long long)d * n;
  double ss = 0.0;
  for (long long i = d + threadIdx.x; i < n; i += blockDim.x) ss += b[i] * b[i];
  ss = block_sum(ss, red);
  *rho = r;
  return ss;
}

// grid (K, n_probs): one CTA per candidate
__global__ void __launch_bounds__(L0_THREADS)
refit_kernel(RefitArgs a) {
  __shared__ double red[32];
  __shared__ int s_t[L0_DMAX];
  const int prob = blockIdx.y, cidx = blockIdx.x;
  const ProbDesc pd = a.probs[prob];
  const int cnt = a.pool_cnt[prob];
  if (cidx >= cnt) return;
  const int d = pd.d;
  if (threadIdx.x == 0) {
    int t[L0_DMAX];
    lex_unrank(a.B, pd.m, d, a.pool_k[(size_t)prob * a.K + cidx], pd.total, t);
    for (int q = 0; q < d; ++q) s_t[q] = t[q];
  }
  __syncthreads();
  double *A = a.scratch + ((size_t)prob * a.K + cidx) * (size_t)(d + 1) * a.nmax;
  const int t_lo = a.shared ? 0 : pd.task;
  const int t_hi = a.shared ? a.T : pd.task + 1;
  double total = 0.0;
  bool elig = true;
  for (int t = t_lo; t < t_hi; ++t) {
    const long long lo = a.offsets[t], hi = a.offsets[t + 1], n = hi - lo;
    const double *mu = a.mu + (size_t)t * (a.m + 1);
    for (int q = 0; q <= d; ++q) {
      const double *src = (q < d) ? a.X + (long long)s_t[q] * a.n_total + lo : a.y + lo;
      const double mean = (q < d) ? mu[s_t[q] + 1] : mu[0];
      double *dst = A + (long long)q * n;
      for (long long i = threadIdx.x; i < n; i += blockDim.x) dst[i] = src[i] - mean;
    }
    __syncthreads();
    double rho;
    const double sse = householder_sse(A, n, d, red, &rho);
    total += sse;
    if (!(rho >= a.rho_min)) elig = false;
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    double score = total;
    if (a.shared) score = total / (double)a.offsets[a.T];
    a.refit[(size_t)prob * a.K + cidx] = elig ? score : __longlong_as_double(0x7ff0000000000000ll);
  }
}

// --------------------------------------------------------------- select --
// One CTA per problem: sort the pool by (refit score, key), emit the best k,
// and evaluate the certificate.
template <typename R>
__global__ void __launch_bounds__(L0_THREADS)
select_kernel(SelectArgs<R> a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int prob = blockIdx.x;
  const ProbDesc pd = a.probs[prob];
  const int cnt = a.pool_cnt[prob];
  int P = 1;
  while (P < a.K) P <<= 1;
  double *ss = (double *)smem;
  u64 *sk = (u64 *)(ss + P);
  __shared__ double red[32];
  double scale = 1.0;
  if (!a.shared) {
    const double is = a.inv_s[(size_t)pd.task * a.mp1];
    scale = (is > 0.0) ? 1.0 / (is * is) : 0.0;
  }
  double dmax = 0.0;
  for (int i = threadIdx.x; i < P; i += blockDim.x) {
    if (i < cnt) {
      const double rf = a.refit[(size_t)prob * a.K + i];
      ss[i] = rf;
      sk[i] = a.pool_k[(size_t)prob * a.K + i];
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
  cta_bitonic_sort<double>(ss, sk, P);
  dmax = block_max(dmax, red);
  __shared__ int s_valid;
  if (threadIdx.x == 0) {
    int nv = 0;
    for (int i = 0; i < cnt; ++i) nv += isfinite(ss[i]) ? 1 : 0;
    s_valid = nv;
  }
  __syncthreads();
  const int nvalid = s_valid;
  const int d = pd.d;
  const double div = a.rmse_div[prob];
  for (int i = threadIdx.x; i < a.k; i += blockDim.x) {
    int *ot = a.out_tuples + ((size_t)prob * a.k + i) * d;
    if (i < nvalid) {
      int t[L0_DMAX];
      lex_unrank(a.B, pd.m, d, sk[i], pd.total, t);
      for (int q = 0; q < d; ++q) ot[q] = t[q];
      a.out_rmse[(size_t)prob * a.k + i] = sqrt(fmax(ss[i], 0.0) / div);
    } else {
      for (int q = 0; q < d; ++q) ot[q] = -1;
      a.out_rmse[(size_t)prob * a.k + i] = __longlong_as_double(0x7ff0000000000000ll);
    }
  }
  if (threadIdx.x == 0) {
    CertOut c;
    c.delta = dmax;
    c.pool_cnt = cnt;
    c.pool_full = (cnt >= a.K) ? 1 : 0;
    c.n_valid = nvalid;
    c.pool_worst = (cnt > 0) ? (double)a.pool_s[(size_t)prob * a.K + cnt - 1] * scale : 0.0;
    c.kth_refit = (nvalid >= a.k) ? ss[a.k - 1] : __longlong_as_double(0x7ff0000000000000ll);
    // Every tuple outside the pool has a Gram score >= pool_worst; its exact
    // score is at least pool_worst - safety * delta.  The pool provably holds
    // the exact top k when that bound clears the k-th re-fitted score.
    if (!c.pool_full) c.certified = 1;
    else c.certified = (c.pool_worst - a.cert_safety * dmax >= c.kth_refit) ? 1 : 0;
    a.cert[prob] = c;
  }
}

__global__ void unrank_kernel(Binom B, int m, int d, u64 total, const u64 *ranks,
                              long long count, int *tuples) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  int t[L0_DMAX];
  lex_unrank(B, m, d, ranks[i], total, t);
  for (int q = 0; q < d; ++q) tuples[i * d + q] = t[q];
}

}  // namespace

template <typename R>
cudaError_t launch_merge(const R *in_s, const u64 *in_k, const int *in_cnt,
                         int n_slots, int n_probs, int K, int S, int groups,
                         R *part_s, u64 *part_k, int *part_cnt, unsigned *done,
                         R *pool_s, u64 *pool_k, int *pool_cnt, cudaStream_t st) {
  size_t smem = cta_list_bytes<R>(K, S) + 16;
  cudaError_t e = cudaFuncSetAttribute(merge_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  merge_kernel<R><<<dim3(groups, n_probs), L0_THREADS, smem, st>>>(
      in_s, in_k, in_cnt, n_slots, K, S, part_s, part_k, part_cnt, done, pool_s,
      pool_k, pool_cnt);
  return cudaGetLastError();
}

cudaError_t launch_refit(const RefitArgs &a, cudaStream_t st) {
  refit_kernel<<<dim3(a.K, a.n_probs), L0_THREADS, 0, st>>>(a);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_select(const SelectArgs<R> &a, cudaStream_t st) {
  int P = 1;
  while (P < a.K) P <<= 1;
  size_t smem = (size_t)P * 16;
  cudaError_t e = cudaFuncSetAttribute(select_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  select_kernel<R><<<a.n_probs, L0_THREADS, smem, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_unrank(const Binom &B, int m, int d, u64 total, const u64 *ranks,
                          long long count, int *tuples, cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  unrank_kernel<<<(unsigned)((count + 255) / 256), 256, 0, st>>>(B, m, d, total, ranks,
                                                                 count, tuples);
  return cudaGetLastError();
}

template cudaError_t launch_merge<double>(const double *, const u64 *, const int *, int, int, int, int, int, double *, u64 *, int *, unsigned *, double *, u64 *, int *, cudaStream_t);
template cudaError_t launch_merge<float>(const float *, const u64 *, const int *, int, int, int, int, int, float *, u64 *, int *, unsigned *, float *, u64 *, int *, cudaStream_t);
template cudaError_t launch_select<double>(const SelectArgs<double> &, cudaStream_t);
template cudaError_t launch_select<float>(const SelectArgs<float> &, cudaStream_t);

}  // namespace l0
