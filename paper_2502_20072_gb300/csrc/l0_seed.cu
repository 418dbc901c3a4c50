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

__device__ __forceinline__ unsigned ord32f(float x) {
  const unsigned b = __float_as_uint(x);
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float f32_up(float x) { return x; }
__device__ __forceinline__ float f32_up(double x) { return __double2float_ru(x); }

// smallest key T with #{keys <= T} >= want, i.e. the want-th smallest key
// (keys[0..n) in shared memory; all threads; ~0 when n < want).  Radix
// select from the top byte down: per byte, a 256-bin count of the keys that
// share the bytes chosen so far, then the bin where the running count
// reaches the rank still wanted.  Four passes over the keys.
__device__ unsigned select_key(const unsigned *keys, int n, int want, unsigned *bins,
                               int *s_sel) {
  if (n < want || want < 1) return 0xffffffffu;
  unsigned prefix = 0u, pmask = 0u;
  int rem = want;
  const int lane = threadIdx.x & 31;
  for (int shift = 24; shift >= 0; shift -= 8) {
    for (int i = threadIdx.x; i < 256; i += blockDim.x) bins[i] = 0u;
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      const unsigned k = keys[i];
      if ((k & pmask) == prefix) atomicAdd(bins + ((k >> shift) & 255u), 1u);
    }
    __syncthreads();
    if (threadIdx.x < 32) {
      unsigned c[8], sum = 0u;
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        c[i] = bins[lane * 8 + i];
        sum += c[i];
      }
      unsigned inc = sum;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += t;
      }
      const unsigned bl = __ballot_sync(0xffffffffu, inc >= (unsigned)rem);
      const int lk = __ffs(bl) - 1;   // the counts add up to >= rem, so bl != 0
      if (lane == lk) {
        unsigned before = inc - sum;
        int bin = lane * 8 + 7;
        for (int i = 0; i < 8; ++i) {
          if (before + c[i] >= (unsigned)rem) { bin = lane * 8 + i; break; }
          before += c[i];
        }
        s_sel[0] = bin;
        s_sel[1] = (int)before;
      }
    }
    __syncthreads();
    const int bin = s_sel[0];
    rem -= s_sel[1];
    prefix |= (unsigned)bin << shift;
    pmask |= 255u << shift;
    __syncthreads();
  }
  return prefix;
}

// rel = SSE / S_yy of one tuple t[0..d) (ascending columns) by the augmented
// Cholesky of (t, target) in R; false when a feature pivot falls below
// ratio times its diagonal or two columns share a duplicate class
template <typename R>
__device__ bool tuple_rel(const R *G, long long ld, const int *t, int d, double ratio,
                          const int *cls, R *rel_out) {
  if (cls)
    for (int i = 0; i < d; ++i)
      for (int j = 0; j < i; ++j)
        if (__ldg(cls + t[i]) == __ldg(cls + t[j])) return false;
  R Lm[L0_DMAX + 1][L0_DMAX + 1];
  R rel = R(0);
  bool ok = true;
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
  *rel_out = rel;
  return ok;
}

// best pairs of the seed columns whose completions the d = 3 seed scores
constexpr int SEED_PAIRS = 8;

// The K'-th best score of all d-tuples of the M columns with the best
// single-column fits: two order-statistic searches (no sorting).
template <typename R>
__global__ void __launch_bounds__(SEED_THREADS)
seed_kernel(const R *Gbase, const ProbDesc *probs, int K, int S, int seed, double ratio,
            Binom B, u64 *gthr, unsigned *hist, int max_keys, const int *cls) {
  extern __shared__ __align__(16) unsigned char smem[];
  unsigned *keys = (unsigned *)smem;            // [max(m, tuples)]
  __shared__ int cols[64];
  __shared__ int s_n;
  __shared__ unsigned s_bins[256];
  __shared__ int s_sel[2];
  __shared__ int s_pair[SEED_PAIRS][2];
  __shared__ int s_npair;
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
  const int d = pd.d;
  const int m = min(pd.m, max_keys);   // a prefix of the columns when n_sis is huge
  const R G00 = G[0];
  // 1. the M best single columns: 1 - r_j^2 as ordered keys
  for (int k = threadIdx.x; k < m; k += blockDim.x) {
    const R ckk = G[(long long)(k + 1) * (ld + 1)];
    const R ck = G[k + 1];
    keys[k] = (ckk > R(0)) ? ord32f(f32_up(G00 - ck * ck / ckk)) : 0xffffffffu;
  }
  __syncthreads();
  const unsigned t1 = select_key(keys, m, M, s_bins, s_sel);
  if (threadIdx.x == 0) s_n = 0;
  __syncthreads();
  for (int k = threadIdx.x; k < m; k += blockDim.x)
    if (keys[k] < t1) cols[atomicAdd(&s_n, 1)] = k;   // fewer than M by construction
  __syncthreads();
  for (int k = threadIdx.x; k < m; k += blockDim.x)
    if (keys[k] == t1) {
      const int slot = atomicAdd(&s_n, 1);
      if (slot < M) cols[slot] = k;
    }
  __syncthreads();
  if (threadIdx.x == 0) {
    const int Mr = min(s_n, M);
    s_n = Mr;
    for (int i = 1; i < Mr; ++i) {     // ascending column order
      int v = cols[i], q = i - 1;
      while (q >= 0 && cols[q] > v) { cols[q + 1] = cols[q]; --q; }
      cols[q + 1] = v;
    }
  }
  __syncthreads();
  const int Mr = s_n;
  // 2. d = 3: the best SEED_PAIRS pairs of those columns, whose completions
  // by every other column are the tuples the search's best K' mostly are
  if (threadIdx.x == 0) s_npair = 0;
  const int npairs = Mr * (Mr - 1) / 2;
  const int pb = min(SEED_PAIRS, npairs);
  if (d == 3 && pb > 0 && npairs <= max_keys) {
    for (int r = threadIdx.x; r < npairs; r += blockDim.x) {
      int b = 1;
      while (b * (b + 1) / 2 <= r) ++b;   // colex: pair (a, b) has rank b (b - 1) / 2 + a
      const int t[2] = {cols[r - b * (b - 1) / 2], cols[b]};
      R rel;
      keys[r] = tuple_rel<R>(G, ld, t, 2, ratio, cls, &rel) ? ord32f(f32_up(rel)) : 0xffffffffu;
    }
    __syncthreads();
    const unsigned tp = select_key(keys, npairs, pb, s_bins, s_sel);
    for (int r = threadIdx.x; r < npairs; r += blockDim.x) {
      if (keys[r] <= tp && keys[r] != 0xffffffffu) {
        const int slot = atomicAdd(&s_npair, 1);
        if (slot < pb) {
          int b = 1;
          while (b * (b + 1) / 2 <= r) ++b;
          s_pair[slot][0] = cols[r - b * (b - 1) / 2];
          s_pair[slot][1] = cols[b];
        }
      }
    }
    __syncthreads();
  }
  const int nsp = min(s_npair, pb);
  // 3. every d-tuple of the seed columns (at most the key capacity; a subset
  // of real tuples bounds the K'-th best just as well), exact augmented
  // Cholesky; then (d = 3) each chosen pair with every column outside the
  // seed set -- distinct from those tuples and from each other's
  const u64 total = small_binom(Mr, d);
  const int nt = (int)(total < (u64)max_keys ? total : (u64)max_keys);
  const int per_pair = (nsp > 0) ? min(m, (max_keys - nt) / nsp) : 0;
  const int ntot = nt + nsp * per_pair;
  if (ntot < K) return;     // too few tuples to bound the K'-th
  for (int r = threadIdx.x; r < nt; r += blockDim.x) {
    int a[L0_DMAX];
    {  // colex unrank over the Mr seed columns
      u64 q = (u64)r;
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
    R rel;
    keys[r] = tuple_rel<R>(G, ld, t, d, ratio, cls, &rel) ? ord32f(f32_up(rel)) : 0xffffffffu;
  }
  // each chosen pair's factor with the target, once: l11, l21, l22 of the
  // Cholesky of C[a,b][a,b], z of the target, pP = 1 - |z|^2
  __shared__ R s_pf[SEED_PAIRS][6];
  __shared__ int s_pok[SEED_PAIRS];
  if (threadIdx.x < nsp) {
    const int a = s_pair[threadIdx.x][0], b = s_pair[threadIdx.x][1];
    const R caa = gram_at<R>(G, ld, a + 1, a + 1), cbb = gram_at<R>(G, ld, b + 1, b + 1);
    const R cab = gram_at<R>(G, ld, a + 1, b + 1);
    const R l11 = sqrt(caa > R(0) ? caa : R(1));
    const R l21 = cab / l11;
    const R p2 = cbb - l21 * l21;
    const R l22 = sqrt(p2 > R(0) ? p2 : R(1));
    const R z1 = G[a + 1] / l11;
    const R z2 = (G[b + 1] - l21 * z1) / l22;
    s_pf[threadIdx.x][0] = l11;
    s_pf[threadIdx.x][1] = l21;
    s_pf[threadIdx.x][2] = l22;
    s_pf[threadIdx.x][3] = z1;
    s_pf[threadIdx.x][4] = z2;
    s_pf[threadIdx.x][5] = G00 - z1 * z1 - z2 * z2;
    s_pok[threadIdx.x] = caa > R(0) && p2 >= (R)ratio * cbb;
  }
  __syncthreads();
  for (int x = threadIdx.x; x < nsp * per_pair; x += blockDim.x) {
    const int p = x / per_pair, k = x - p * per_pair;
    bool in_seed = false;
    for (int i = 0; i < Mr; ++i) in_seed = in_seed || cols[i] == k;
    unsigned key = 0xffffffffu;
    const int a = s_pair[p][0], b = s_pair[p][1];
    const bool dup = cls && (__ldg(cls + k) == __ldg(cls + a) || __ldg(cls + k) == __ldg(cls + b));
    if (!in_seed && !dup && s_pok[p]) {
      // the completion k after the pair: pivot and target coordinate, then
      // rel = pP - w^2 / pivot
      const R ckk = gram_at<R>(G, ld, k + 1, k + 1);
      const R g1 = gram_at<R>(G, ld, a + 1, k + 1) / s_pf[p][0];
      const R g2 = (gram_at<R>(G, ld, b + 1, k + 1) - s_pf[p][1] * g1) / s_pf[p][2];
      const R piv = ckk - g1 * g1 - g2 * g2;
      const R w = G[k + 1] - g1 * s_pf[p][3] - g2 * s_pf[p][4];
      if (ckk > R(0) && piv >= (R)ratio * ckk) key = ord32f(f32_up(s_pf[p][5] - w * w / piv));
    }
    keys[nt + x] = key;
  }
  __syncthreads();
  // the K'-th smallest score (rounded up to FP32): K' real tuples lie at or
  // below it, so it bounds the search's K'-th best
  const unsigned t2 = select_key(keys, ntot, K, s_bins, s_sel);
  if (threadIdx.x == 0 && t2 != 0xffffffffu) {
    const unsigned b = (t2 & 0x80000000u) ? (t2 & 0x7fffffffu) : ~t2;
    atomicMin(gthr + prob, ord_of((R)__uint_as_float(b)));
  }
}

}  // namespace

template <typename R>
size_t seed_smem_bytes(int K, int S) {
  (void)S;
  return 0;   // the key array is sized per launch (n_sis, 2 K' + 64 tuples)
}

template <typename R>
cudaError_t launch_seed(const R *G, const ProbDesc *probs_dev, int n_probs, int K, int S,
                        int seed, double ratio, const Binom &B, u64 *gthr, unsigned *hist,
                        int max_keys, cudaStream_t st, const int *cls) {
  if (max_keys > 50000) max_keys = 50000;   // 200 KB of keys
  const size_t smem = (size_t)4 * (size_t)max_keys;
  cudaError_t e =
      cudaFuncSetAttribute(seed_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  seed_kernel<R><<<n_probs, SEED_THREADS, smem, st>>>(G, probs_dev, K, S, seed, ratio, B, gthr,
                                                                hist, max_keys, cls);
  return cudaGetLastError();
}

template size_t seed_smem_bytes<double>(int, int);
template size_t seed_smem_bytes<float>(int, int);
template cudaError_t launch_seed<double>(const double *, const ProbDesc *, int, int, int, int,
                                         double, const Binom &, u64 *, unsigned *, int,
                                         cudaStream_t, const int *);
template cudaError_t launch_seed<float>(const float *, const ProbDesc *, int, int, int, int,
                                        double, const Binom &, u64 *, unsigned *, int,
                                        cudaStream_t, const int *);

}  // namespace l0
