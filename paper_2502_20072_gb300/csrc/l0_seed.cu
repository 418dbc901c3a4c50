// l0_seed.cu -- initial search threshold per problem.
//
// Before the tuple search every problem's threshold is set to +inf, then
// tightened to the K'-th best score among all d-tuples formed from the M
// columns with the best single-feature fits (smallest 1 - r_j^2, r from
// Eq. 1).  Those are real tuples, so at least K' tuples score at or below the
// bound and nothing better than the global K'-th can be cut by it; the
// columns most correlated with the target give a bound far tighter than an
// arbitrary sample, so the search starts with few candidates instead of a
// flood.  (The paper's SIS step, Sec. 2.3, ranks features the same way.)
#include "l0_kernels.cuh"

namespace l0 {

namespace {

__device__ __forceinline__ u64 small_binom(int n, int k) {
  if (k < 0 || n < k) return 0;
  u64 r = 1;
  for (int i = 1; i <= k; ++i) r = r * (u64)(n - k + i) / (u64)i;
  return r;
}

template <typename R>
__device__ __forceinline__ R gram_at(const R *G, long long ld, int a, int b) {
  return a <= b ? G[(long long)a * ld + b] : G[(long long)b * ld + a];
}

// one CTA per problem
constexpr int SEED_THREADS = 1024;

template <typename R>
__global__ void __launch_bounds__(SEED_THREADS)
seed_kernel(const R *Gbase, const ProbDesc *probs, int K, int S, int seed, double ratio,
            Binom B, u64 *gthr, unsigned *hist) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int cols[64];
  __shared__ u64 s_total;
  unsigned char *p = smem;
  CtaList<R> L = cta_list_carve<R>(p, K, S);
  const int prob = blockIdx.x;
  const ProbDesc pd = probs[prob];
  if (threadIdx.x == 0) gthr[prob] = ord_inf<R>();
  if (hist)   // the search's score histogram starts empty
    for (int i = threadIdx.x; i < L0_HIST_WORDS; i += blockDim.x)
      hist[(size_t)prob * L0_HIST_WORDS + i] = 0u;
  if (!seed || pd.d < 2) return;
  // smallest M with C(M, d) >= 2 K', at most min(m, 64, K')
  const int Mcap = min(min(pd.m, 64), K);
  int M = Mcap;
  for (int q = pd.d; q <= Mcap; ++q)
    if (small_binom(q, pd.d) >= 2ull * (u64)K) { M = q; break; }
  const R *G = Gbase + pd.g_off;
  const long long ld = pd.ld;
  const int m = pd.m, d = pd.d;
  const R G00 = G[0];
  // 1. the M best single columns
  L.K = M;
  cta_list_reset<R>(L, nullptr);
  __syncthreads();
  for (int base = 0; base < m; base += blockDim.x) {
    const int k = base + threadIdx.x;
    R rel = R(0);
    bool ok = false;
    if (k < m) {
      const R ckk = G[(long long)(k + 1) * (ld + 1)];
      const R ck = G[k + 1];
      ok = ckk > R(0);
      rel = G00 - ck * ck / ckk;
    }
    int redo = 0;
    do {
      if (ok && cta_list_admits<R>(L, rel, (u64)k)) cta_list_push<R>(L, rel, (u64)k);
      __syncthreads();
      if (++redo > L0_MAX_REDO) break;
    } while (cta_list_fold<R>(L, nullptr));
  }
  const int Mr = *(volatile int *)L.n_list;
  if (threadIdx.x == 0) {
    for (int i = 0; i < Mr; ++i) cols[i] = (int)L.lk[i];
    for (int i = 1; i < Mr; ++i) {     // ascending column order
      int v = cols[i], q = i - 1;
      while (q >= 0 && cols[q] > v) { cols[q + 1] = cols[q]; --q; }
      cols[q + 1] = v;
    }
    s_total = small_binom(Mr, d);
  }
  __syncthreads();
  const u64 total = s_total;
  if (total < (u64)K) return;     // too few tuples to bound the K'-th
  // 2. every d-tuple of those columns, exact augmented Cholesky
  L.K = K;
  cta_list_reset<R>(L, nullptr);
  __syncthreads();
  for (u64 base = 0; base < total; base += blockDim.x) {
    const u64 r = base + threadIdx.x;
    R rel = R(0);
    bool ok = false;
    u64 key = 0;
    if (r < total) {
      int a[L0_DMAX];
      {  // colex unrank over the Mr seed columns
        u64 q = r;
        int hi = Mr - 1;
        for (int i = d; i >= 1; --i) {
          int lo = i - 1, h = hi;
          while (lo < h) {
            const int mid = (lo + h + 1) >> 1;
            if (small_binom(mid, i) <= q) lo = mid; else h = mid - 1;
          }
          q -= small_binom(lo, i);
          a[i - 1] = lo;
          hi = lo - 1;
        }
      }
      int t[L0_DMAX];
      for (int i = 0; i < d; ++i) t[i] = cols[a[i]];
      // Cholesky of (t_1 .. t_d, target): pivots of the features checked,
      // the last pivot is rel = SSE / S_yy
      R Lm[L0_DMAX + 1][L0_DMAX + 1];
      ok = true;
      for (int i = 0; i <= d; ++i) {
        const int ia = (i < d) ? t[i] + 1 : 0;
        for (int j = 0; j <= i; ++j) {
          const int ib = (j < d) ? t[j] + 1 : 0;
          R c = gram_at<R>(G, ld, ia, ib);
          const R orig = c;
          for (int q = 0; q < j; ++q) c -= Lm[i][q] * Lm[j][q];
          if (j < i) {
            Lm[i][j] = c / Lm[j][j];
          } else if (i < d) {
            ok = ok && orig > R(0) && c >= (R)ratio * orig;
            Lm[i][i] = sqrt(c > R(0) ? c : R(1));
          } else {
            rel = c;
          }
        }
      }
      key = lex_rank(B, m, d, t, pd.total);
    }
    int redo = 0;
    do {
      if (ok && cta_list_admits<R>(L, rel, key)) cta_list_push<R>(L, rel, key);
      __syncthreads();
      if (++redo > L0_MAX_REDO) break;
    } while (cta_list_fold<R>(L, nullptr));
  }
  if (threadIdx.x == 0 && *(volatile int *)L.n_list >= K)
    atomicMin(gthr + prob, ord_of(L.ls[K - 1]));
}

}  // namespace

template <typename R>
size_t seed_smem_bytes(int K, int S) {
  return cta_list_bytes<R>(K, S) + 16;
}

template <typename R>
cudaError_t launch_seed(const R *G, const ProbDesc *probs_dev, int n_probs, int K, int S,
                        int seed, double ratio, const Binom &B, u64 *gthr, unsigned *hist,
                        cudaStream_t st) {
  const size_t smem = seed_smem_bytes<R>(K, S);
  cudaError_t e =
      cudaFuncSetAttribute(seed_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  seed_kernel<R><<<n_probs, SEED_THREADS, smem, st>>>(G, probs_dev, K, S, seed, ratio, B, gthr,
                                                                hist);
  return cudaGetLastError();
}

template size_t seed_smem_bytes<double>(int, int);
template size_t seed_smem_bytes<float>(int, int);
template cudaError_t launch_seed<double>(const double *, const ProbDesc *, int, int, int, int,
                                         double, const Binom &, u64 *, unsigned *, cudaStream_t);
template cudaError_t launch_seed<float>(const float *, const ProbDesc *, int, int, int, int,
                                        double, const Binom &, u64 *, unsigned *, cudaStream_t);

}  // namespace l0
