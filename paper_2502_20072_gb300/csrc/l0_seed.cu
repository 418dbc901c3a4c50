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

// rel = SSE / S_yy of one tuple of seed columns by the augmented Cholesky of
// (tuple, target) in R, from the seed block Bs (nb x nb, index 0 the target,
// s + 1 seed column s); a[0..d) are ascending seed positions, cols[] their
// columns.  False when a feature pivot falls below ratio times its diagonal
// or two columns share a duplicate class.
template <typename R>
__device__ bool tuple_rel(const R *Bs, int nb, const int *a, const int *cols, int d, double ratio,
                          const int *cls, R *rel_out) {
  if (cls)
    for (int i = 0; i < d; ++i)
      for (int j = 0; j < i; ++j)
        if (__ldg(cls + cols[a[i]]) == __ldg(cls + cols[a[j]])) return false;
  R Lm[L0_DMAX + 1][L0_DMAX + 1];
  R rel = R(0);
  bool ok = true;
  for (int i = 0; i <= d; ++i) {
    const int ia = (i < d) ? a[i] + 1 : 0;
    for (int j = 0; j <= i; ++j) {
      const int ib = (j < d) ? a[j] + 1 : 0;
      R c = Bs[ia * nb + ib];
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

// largest number of seed columns (the block of their Gram is staged in
// shared memory behind the keys)
constexpr int SEED_MAXM = 64;

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
  __shared__ int cols[SEED_MAXM], cols2[SEED_MAXM];
  __shared__ int s_n;
  __shared__ unsigned s_bins[256];
  __shared__ int s_sel[2];
  __shared__ int s_pair[SEED_PAIRS][2];
  __shared__ int s_npair;
  __shared__ u64 s_C[SEED_MAXM + 1][L0_DMAX + 1];   // C(n, i), n <= SEED_MAXM
  const int prob = blockIdx.x;
  const ProbDesc pd = probs[prob];
  if (threadIdx.x == 0) gthr[prob] = ord_inf<R>();
  if (hist)   // the search's score histogram starts empty
    for (int i = threadIdx.x; i < L0_HIST_WORDS; i += blockDim.x)
      hist[(size_t)prob * L0_HIST_WORDS + i] = 0u;
  if (!seed || pd.d < 2) return;
  // smallest M with C(M, d) >= 2 K', at most min(m, 64, K')
  const int Mcap = min(min(pd.m, SEED_MAXM), K);
  int M = Mcap;
  {
    // C(q, d) >= 2K  <=>  q (q - 1) .. (q - d + 1) >= 2K d!  (no divisions;
    // 64^8 < 2^63)
    u64 fact = 1ull;
    for (int i = 2; i <= pd.d; ++i) fact *= (u64)i;
    const u64 want = 2ull * (u64)K * fact;
    for (int q = pd.d; q <= Mcap; ++q) {
      u64 f = 1ull;
      for (int i = 0; i < pd.d; ++i) f *= (u64)(q - i);
      if (f >= want) { M = q; break; }
    }
  }
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
  // ascending column order: each column's rank is the number of smaller ones
  const int Mr = min(s_n, M);
  if (threadIdx.x < Mr) {
    const int v = cols[threadIdx.x];
    int rk = 0;
    for (int i = 0; i < Mr; ++i) rk += cols[i] < v;
    cols2[rk] = v;
  }
  __syncthreads();
  if (threadIdx.x < Mr) cols[threadIdx.x] = cols2[threadIdx.x];
  if (threadIdx.x == 0) s_npair = 0;   // visible after the barrier below
  if (threadIdx.x <= SEED_MAXM) {      // row n of Pascal's triangle, exact divisions
    const int n = threadIdx.x;
    u64 c = 1ull;
    s_C[n][0] = 1ull;
    for (int i = 1; i <= L0_DMAX; ++i) {
      c = (i <= n) ? c * (u64)(n - i + 1) / (u64)i : 0ull;
      s_C[n][i] = c;
    }
  }
  // the seed columns' augmented block, target first (one trip to L2 for all
  // the tuples of seed columns below)
  const int nb = Mr + 1;
  R *Bs = (R *)(keys + ((max_keys + 3) & ~3));   // 16-byte aligned
  for (int x = threadIdx.x; x < nb * nb; x += blockDim.x) {
    const int ia = x / nb, ib = x - (x / nb) * nb;
    Bs[x] = gram_at<R>(G, ld, ia ? cols2[ia - 1] + 1 : 0, ib ? cols2[ib - 1] + 1 : 0);
  }
  __syncthreads();
  // 2. d = 3: the best SEED_PAIRS pairs of those columns, whose completions
  // by every other column are the tuples the search's best K' mostly are
  const int npairs = Mr * (Mr - 1) / 2;
  const int pb = min(SEED_PAIRS, npairs);
  if (d == 3 && pb > 0 && npairs <= max_keys) {
    for (int r = threadIdx.x; r < npairs; r += blockDim.x) {
      int b = 1;
      while (b * (b + 1) / 2 <= r) ++b;   // colex: pair (a, b) has rank b (b - 1) / 2 + a
      const int t[2] = {r - b * (b - 1) / 2, b};
      R rel;
      keys[r] = tuple_rel<R>(Bs, nb, t, cols, 2, ratio, cls, &rel) ? ord32f(f32_up(rel)) : 0xffffffffu;
    }
    __syncthreads();
    const unsigned tp = select_key(keys, npairs, pb, s_bins, s_sel);
    for (int r = threadIdx.x; r < npairs; r += blockDim.x) {
      if (keys[r] <= tp && keys[r] != 0xffffffffu) {
        const int slot = atomicAdd(&s_npair, 1);
        if (slot < pb) {
          int b = 1;
          while (b * (b + 1) / 2 <= r) ++b;
          s_pair[slot][0] = r - b * (b - 1) / 2;   // seed positions
          s_pair[slot][1] = b;
        }
      }
    }
    __syncthreads();
  }
  const int nsp = d == 3 ? min(s_npair, pb) : 0;
  // 3. every d-tuple of the seed columns (at most the key capacity; a subset
  // of real tuples bounds the K'-th best just as well), exact augmented
  // Cholesky; then (d = 3) each chosen pair with every column outside the
  // seed set -- distinct from those tuples and from each other's
  const u64 total = s_C[Mr][d];
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
          if (s_C[mid][i] <= q) lo = mid; else h = mid - 1;
        }
        q -= s_C[lo][i];
        a[i - 1] = lo;
        hi = lo - 1;
      }
    }
    R rel;
    keys[r] = tuple_rel<R>(Bs, nb, a, cols, d, ratio, cls, &rel) ? ord32f(f32_up(rel)) : 0xffffffffu;
  }
  // each chosen pair's factor with the target, once: 1/l11, l21, 1/l22 of the
  // Cholesky of C[a,b][a,b], z of the target, pP = 1 - |z|^2
  __shared__ R s_pf[SEED_PAIRS][6];
  __shared__ int s_pok[SEED_PAIRS];
  if (threadIdx.x < nsp) {
    const int a = s_pair[threadIdx.x][0] + 1, b = s_pair[threadIdx.x][1] + 1;   // block indices
    const R caa = Bs[a * nb + a], cbb = Bs[b * nb + b], cab = Bs[a * nb + b];
    const R l11 = sqrt(caa > R(0) ? caa : R(1));
    const R l21 = cab / l11;
    const R p2 = cbb - l21 * l21;
    const R l22 = sqrt(p2 > R(0) ? p2 : R(1));
    const R z1 = Bs[a] / l11;
    const R z2 = (Bs[b] - l21 * z1) / l22;
    s_pf[threadIdx.x][0] = R(1) / l11;
    s_pf[threadIdx.x][1] = l21;
    s_pf[threadIdx.x][2] = R(1) / l22;
    s_pf[threadIdx.x][3] = z1;
    s_pf[threadIdx.x][4] = z2;
    s_pf[threadIdx.x][5] = G00 - z1 * z1 - z2 * z2;
    s_pok[threadIdx.x] = caa > R(0) && p2 >= (R)ratio * cbb;
  }
  __syncthreads();
  // completions: a thread per column k, its Gram entries with both columns
  // of every chosen pair loaded before any is used
  int pa[SEED_PAIRS], pb2[SEED_PAIRS];
#pragma unroll
  for (int p = 0; p < SEED_PAIRS; ++p) {
    pa[p] = p < nsp ? cols[s_pair[p][0]] : 0;
    pb2[p] = p < nsp ? cols[s_pair[p][1]] : 0;
  }
  constexpr int PC = sizeof(R) == 8 ? 4 : SEED_PAIRS;   // pairs whose loads go together
  for (int k = threadIdx.x; k < per_pair; k += blockDim.x) {
    const R ckk = G[(long long)(k + 1) * (ld + 1)], ck = G[k + 1];
    const int ck_cls = cls ? __ldg(cls + k) : 0;
#pragma unroll
    for (int p0 = 0; p0 < SEED_PAIRS; p0 += PC) {
      if (p0 >= nsp) break;
      R cak[PC], cbk[PC];
#pragma unroll
      for (int u = 0; u < PC; ++u) {
        const int p = p0 + u;
        cak[u] = p < nsp ? gram_at<R>(G, ld, pa[p] + 1, k + 1) : R(0);
        cbk[u] = p < nsp ? gram_at<R>(G, ld, pb2[p] + 1, k + 1) : R(0);
      }
#pragma unroll
      for (int u = 0; u < PC; ++u) {
        const int p = p0 + u;
        if (p >= nsp) break;
        unsigned key = 0xffffffffu;
        const bool dup = cls && (ck_cls == __ldg(cls + pa[p]) || ck_cls == __ldg(cls + pb2[p]));
        if (!dup && s_pok[p]) {
          // the completion k after the pair: pivot and target coordinate,
          // then rel = pP - w^2 / pivot
          const R g1 = cak[u] * s_pf[p][0];
          const R g2 = (cbk[u] - s_pf[p][1] * g1) * s_pf[p][2];
          const R piv = ckk - g1 * g1 - g2 * g2;
          const R w = ck - g1 * s_pf[p][3] - g2 * s_pf[p][4];
          if (ckk > R(0) && piv >= (R)ratio * ckk) key = ord32f(f32_up(s_pf[p][5] - w * w / piv));
        }
        keys[nt + p * per_pair + k] = key;
      }
    }
  }
  __syncthreads();
  // a completion by a seed column repeats a tuple scored above: dropped
  for (int x = threadIdx.x; x < nsp * Mr; x += blockDim.x) {
    const int p = x / Mr, c = cols[x - p * Mr];
    if (c < per_pair) keys[nt + p * per_pair + c] = 0xffffffffu;
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
  if (max_keys > 47000) max_keys = 47000;   // 188 KB of keys, then the seed block
  const size_t smem = (size_t)4 * (size_t)((max_keys + 3) & ~3) +
                      sizeof(R) * (size_t)(SEED_MAXM + 1) * (size_t)(SEED_MAXM + 1);
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
