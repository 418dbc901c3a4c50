// l0_defer.cu -- FP64 scoring of the tuples the FP32 tuple kernel could not
// trust.
//
// In mixed precision the tuple kernel solves in FP32 from the split-BF16
// Gram.  When a pivot of the FP32 Cholesky falls below
// fp32_fallback_pivot_ratio of its diagonal (near-collinear columns), the
// Schur complement rel = 1 - c^T C^-1 c loses all its digits in FP32.  Such
// tuples are queued as runs (first tuple's lexicographic rank, run length,
// problem); this kernel redoes them in FP64 with the full augmented Cholesky
// from the FP64 Gram (or, for large n_sis, from FP64 dot products of the
// scaled columns), applies the FP64 rank-deficiency cut, and feeds the
// survivors into the same top-K' lists as the FP32 kernel.
#include "l0_kernels.cuh"

namespace l0 {

namespace {

// FP64 Cholesky of (target, prefix), then the Schur complement of each k:
// rel = pP - w^2 / piv.  ent(a, b) returns the FP64 correlation of augmented
// indices a, b (0 the target, j+1 feature j).
struct PrefixFactor {
  double Lm[L0_DMAX][L0_DMAX];
  double z[L0_DMAX];
  double pP;
  bool ok;
};

template <typename Ent>
__device__ void factor_prefix(const Ent &ent, const int *t, int dp, double ratio,
                              PrefixFactor &f) {
  f.pP = ent(0, 0);
  f.ok = true;
  for (int i = 0; i < dp; ++i) {
    for (int j = 0; j <= i; ++j) {
      double c = ent(t[j] + 1, t[i] + 1);
      const double orig = c;
      for (int q = 0; q < j; ++q) c -= f.Lm[i][q] * f.Lm[j][q];
      if (j < i) {
        f.Lm[i][j] = c / f.Lm[j][j];
      } else {
        f.ok = f.ok && orig > 0.0 && c >= ratio * orig;
        f.Lm[i][i] = sqrt(c > 0.0 ? c : 1.0);
      }
    }
    double zi = ent(0, t[i] + 1);
    for (int q = 0; q < i; ++q) zi -= f.Lm[i][q] * f.z[q];
    f.z[i] = zi / f.Lm[i][i];
    f.pP -= f.z[i] * f.z[i];
  }
}

// rel of (prefix, k); false when the pivot of k is below the cut
template <typename Ent>
__device__ bool score_last(const Ent &ent, const int *t, int dp, int k, double ratio,
                           const PrefixFactor &f, double *rel) {
  double g[L0_DMAX];
  double piv = ent(k + 1, k + 1);
  const double ckk = piv;
  double w = ent(0, k + 1);
  for (int i = 0; i < dp; ++i) {
    double gi = ent(t[i] + 1, k + 1);
    for (int q = 0; q < i; ++q) gi -= f.Lm[i][q] * g[q];
    g[i] = gi / f.Lm[i][i];
    piv -= g[i] * g[i];
    w -= g[i] * f.z[i];
  }
  if (!(ckk > 0.0) || !(piv >= ratio * ckk)) return false;
  *rel = f.pP - w * w / piv;
  return true;
}

struct GramEnt {
  const double *G;
  long long ld;
  __device__ double operator()(int a, int b) const {
    return a <= b ? G[(long long)a * ld + b] : G[(long long)b * ld + a];
  }
};

// Gram mode (many queued tuples): one thread per run, entries from the FP64
// Gram.  grid (groups, n_probs); CTA (g, p) takes the runs of problem p with
// index = g (mod groups).
__global__ void __launch_bounds__(L0_THREADS)
defer_gram_kernel(DeferArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int prob = blockIdx.y;
  const ProbDesc pd = a.probs[prob];
  if (!defer_wants_gram(a.n_runs[1], pd.m, pd.d)) return;
  unsigned char *p = smem;
  CtaList<float> L = cta_list_carve<float>(p, a.K, a.S);
  const int d = pd.d;
  const int t_lo = a.shared_T > 0 ? 0 : pd.task;
  const int t_hi = a.shared_T > 0 ? a.shared_T : pd.task + 1;
  cta_list_reset<float>(L, a.gthr + prob);
  __syncthreads();
  const long long nr = (long long)a.n_runs[0];
  const long long nrun = nr < a.cap ? nr : a.cap;
  unsigned long long done_tuples = 0;
  for (long long base = (long long)blockIdx.x * blockDim.x; base < nrun;
       base += (long long)gridDim.x * blockDim.x) {
    const long long r = base + threadIdx.x;
    bool mine = false;
    u64 key0 = 0;
    int len = 0;
    if (r < nrun) {
      const unsigned pl = a.run_len[r];
      mine = (int)(pl >> 8) == prob;
      len = (int)(pl & 0xffu);
      key0 = a.run_key[r];
    }
    int t[L0_DMAX];
    if (mine && len > 0) {
      lex_unrank(a.B, pd.m, d, key0, pd.total, t);   // binomial table, no 64-bit divisions
      done_tuples += (unsigned long long)len;
    }
    int redo = 0;
    do {
      if (mine && len > 0 && a.shared_T == 0) {
        // one task: the run's tuples share every index but the last, so the
        // prefix is factored once
        GramEnt ent{a.G64 + (long long)pd.task * a.g64_stride, a.ld64};
        PrefixFactor f;
        factor_prefix(ent, t, d - 1, a.ratio, f);
        if (f.ok) {
          for (int e = 0; e < len; ++e) {
            double rel;
            if (!score_last(ent, t, d - 1, t[d - 1] + e, a.ratio, f, &rel)) continue;
            const float s = (float)rel;
            const u64 key = key0 + (u64)e;
            if (cta_list_admits<float>(L, s, key)) cta_list_push<float>(L, s, key);
          }
        }
      } else if (mine && len > 0) {
        for (int e = 0; e < len; ++e) {
          // SHARED: pooled over the tasks (ineligible if any task is)
          double score = 0.0;
          bool ok = true;
          for (int tk = t_lo; tk < t_hi && ok; ++tk) {
            GramEnt ent{a.G64 + (long long)tk * a.g64_stride, a.ld64};
            PrefixFactor f;
            factor_prefix(ent, t, d - 1, a.ratio, f);
            double rel;
            ok = f.ok && score_last(ent, t, d - 1, t[d - 1] + e, a.ratio, f, &rel);
            if (ok && a.shared_T > 0) {
              const double is = a.inv_s[(long long)tk * a.mp1];
              score += (is > 0.0 ? 1.0 / (is * is * (double)a.n_total) : 0.0) * rel;
            } else if (ok) {
              score = rel;
            }
          }
          if (!ok) continue;
          const float s = (float)score;
          const u64 key = key0 + (u64)e;
          if (cta_list_admits<float>(L, s, key)) cta_list_push<float>(L, s, key);
        }
      }
      __syncthreads();
      if (++redo > L0_MAX_REDO) break;
    } while (cta_list_fold<float>(L, a.gthr + prob));
  }
  if (done_tuples) atomicAdd(a.n_tuples, done_tuples);
  const size_t slot = (size_t)prob * a.n_slots + a.slot0 + blockIdx.x;
  cta_list_flush<float>(L, a.out_s + slot * a.K, a.out_k + slot * a.K, a.out_cnt + slot);
}

// Gram mode, one task per problem: warps take batches of 32 consecutive
// queued runs from the problem's counter and score the batch's tuples
// together -- a warp-wide scan of the run lengths spreads them over the 32
// lanes -- so single-tuple runs and 128-tuple runs share the work evenly.
// Each run is unranked once by the lane that read it; a tuple's indices come
// from that lane by shuffle, its last index advanced by the tuple's offset in
// the run.  A round ends at a CTA barrier, where the list folds (and, on an
// overflow of its staging area, the round is redone, the same batches).
__global__ void __launch_bounds__(L0_THREADS)
defer_batch_kernel(DeferArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ unsigned long long s_batch[L0_THREADS / 32];
  __shared__ int s_more;
  const unsigned FULL = 0xffffffffu;
  const int prob = blockIdx.y;
  const ProbDesc pd = a.probs[prob];
  if (!defer_wants_gram(a.n_runs[1], pd.m, pd.d)) return;
  unsigned char *p = smem;
  CtaList<float> L = cta_list_carve<float>(p, a.K, a.S);
  const int d = pd.d;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  cta_list_reset<float>(L, a.gthr + prob);
  const long long nr = (long long)a.n_runs[0];
  const long long nrun = nr < a.cap ? nr : a.cap;
  const unsigned long long nbatch = (unsigned long long)((nrun + 31) / 32);
  const GramEnt ent{a.G64 + (long long)pd.task * a.g64_stride, a.ld64};
  unsigned long long done_tuples = 0;
  for (;;) {
    if (lane == 0) s_batch[warp] = atomicAdd(a.batch_ctr + prob, 1u);
    if (threadIdx.x == 0) s_more = 0;
    __syncthreads();
    const unsigned long long b = s_batch[warp];
    if (lane == 0 && b < nbatch) atomicOr(&s_more, 1);
    __syncthreads();
    if (!s_more) break;   // every warp of the CTA is past the last batch (uniform)
    const long long r = (long long)b * 32 + lane;
    int len = 0;
    u64 key0 = 0;
    if (b < nbatch && r < nrun) {
      const unsigned pl = a.run_len[r];
      if ((int)(pl >> 8) == prob) {
        len = (int)(pl & 0xffu);
        key0 = a.run_key[r];
      }
    }
    int t[L0_DMAX];
#pragma unroll
    for (int q = 0; q < L0_DMAX; ++q) t[q] = 0;
    if (len > 0) lex_unrank(a.B, pd.m, d, key0, pd.total, t);
    int inc = len;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int v = __shfl_up_sync(FULL, inc, o);
      if (lane >= o) inc += v;
    }
    const int total = __shfl_sync(FULL, inc, 31);
    if (lane == 0) done_tuples += (unsigned long long)total;
    int redo = 0;
    do {
      for (int base = 0; base < total; base += 32) {   // uniform over the warp
        const int x = base + lane;
        // owner: the lane whose run holds tuple x (the first with inc > x)
        int own = 0;
#pragma unroll
        for (int s = 16; s > 0; s >>= 1) {
          const int v = __shfl_sync(FULL, inc, own + s - 1);
          if (v <= x) own += s;
        }
        own = own > 31 ? 31 : own;
        const int oinc = __shfl_sync(FULL, inc, own), olen = __shfl_sync(FULL, len, own);
        const u64 okey = __shfl_sync(FULL, key0, own);
        int tt[L0_DMAX];
#pragma unroll
        for (int q = 0; q < L0_DMAX; ++q) tt[q] = __shfl_sync(FULL, t[q], own);
        if (x >= total) continue;
        const int e = x - (oinc - olen);
        PrefixFactor f;
        factor_prefix(ent, tt, d - 1, a.ratio, f);
        double rel;
        if (!f.ok || !score_last(ent, tt, d - 1, tt[d - 1] + e, a.ratio, f, &rel)) continue;
        const float s = (float)rel;
        const u64 key = okey + (u64)e;
        if (cta_list_admits<float>(L, s, key)) cta_list_push<float>(L, s, key);
      }
      __syncthreads();
      if (++redo > L0_MAX_REDO) break;
    } while (cta_list_fold<float>(L, a.gthr + prob));
  }
  if (done_tuples) atomicAdd(a.n_tuples, done_tuples);
  const size_t slot = (size_t)prob * a.n_slots + a.slot0 + blockIdx.x;
  cta_list_flush<float>(L, a.out_s + slot * a.K, a.out_k + slot * a.K, a.out_cnt + slot);
}

// Dot mode (few queued tuples): one CTA per run at a time.  The CTA computes
// the FP64 correlations the run needs -- rows (target, prefix) against
// (target, prefix, every k of the run), and each k with itself -- as dot
// products of the scaled FP64 columns (warps over pairs, lanes over
// samples), then thread e scores the run's e-th tuple.
constexpr int DOT_MAXC = L0_DMAX + 128;

struct SmemEnt {
  const double *Gs;       // [L0_DMAX][DOT_MAXC]: row r = base index r
  const double *Gkk;      // [128]
  const int *col_of;      // augmented index -> column in Gs (base + ks)
  int nbase, k0;          // base indices: 0 and t[0..dp-1]+1; ks: k0+1 ..
  const int *base_idx;
  __device__ int base_pos(int a) const {
    for (int i = 0; i < nbase; ++i)
      if (base_idx[i] == a) return i;
    return -1;
  }
  __device__ double operator()(int a, int b) const {
    if (a == b && a > k0) return Gkk[a - k0 - 1];
    int pa = base_pos(a), pb = base_pos(b);
    if (pa < 0) { int tmp = a; a = b; b = tmp; pa = pb; }
    // a is a base index now
    int cb = base_pos(b);
    if (cb < 0) cb = nbase + (b - k0 - 1);
    return Gs[pa * DOT_MAXC + cb];
  }
};

__global__ void __launch_bounds__(L0_THREADS)
defer_dot_kernel(DeferArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double Gs[L0_DMAX * DOT_MAXC];
  __shared__ double Gkk[128];
  __shared__ int s_t[L0_DMAX];
  __shared__ int s_idx[L0_DMAX];
  const int prob = blockIdx.y;
  const ProbDesc pd = a.probs[prob];
  const long long nr = (long long)a.n_runs[0];
  if (nr == 0 || defer_wants_gram(a.n_runs[1], pd.m, pd.d)) return;
  unsigned char *p = smem;
  CtaList<float> L = cta_list_carve<float>(p, a.K, a.S);
  const int d = pd.d, dp = d - 1;
  const int t_lo = a.shared_T > 0 ? 0 : pd.task;
  const int t_hi = a.shared_T > 0 ? a.shared_T : pd.task + 1;
  cta_list_reset<float>(L, a.gthr + prob);
  __syncthreads();
  const long long nrun = nr < a.cap ? nr : a.cap;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  unsigned long long done_tuples = 0;
  for (long long r = blockIdx.x; r < nrun; r += gridDim.x) {
    const unsigned pl = a.run_len[r];
    if ((int)(pl >> 8) != prob) continue;
    const int len = (int)(pl & 0xffu);
    const u64 key0 = a.run_key[r];
    if (threadIdx.x == 0) {
      int t[L0_DMAX];
      lex_unrank(a.B, pd.m, d, key0, pd.total, t);
      for (int i = 0; i < d; ++i) s_t[i] = t[i];
      s_idx[0] = 0;
      for (int i = 0; i < dp; ++i) s_idx[i + 1] = t[i] + 1;
    }
    __syncthreads();
    const int nbase = dp + 1;
    const int kfirst = s_t[d - 1];
    const int ncol = nbase + len;
    const int npairs = nbase * ncol + len;
    const int e = threadIdx.x;
    bool scored = e < len;
    double score = 0.0;
    for (int tk = t_lo; tk < t_hi; ++tk) {
      const long long lo = a.offsets[tk];
      const long long n = a.offsets[tk + 1] - lo;
      // dots: base rows x all columns, plus each k with itself
      for (int q = warp; q < npairs; q += nw) {
        int ra, cb;
        if (q < nbase * ncol) {
          const int rr = q / ncol, cc = q % ncol;
          ra = s_idx[rr];
          cb = (cc < nbase) ? s_idx[cc] : kfirst + (cc - nbase) + 1;
        } else {
          ra = kfirst + (q - nbase * ncol) + 1;
          cb = ra;
        }
        const double *x = a.W64 + (long long)ra * a.n_total + lo;
        const double *z = a.W64 + (long long)cb * a.n_total + lo;
        double s4[4] = {0.0, 0.0, 0.0, 0.0};
        for (long long i0 = lane; i0 < n; i0 += 128) {
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const long long i = i0 + 32 * u;
            if (i < n) s4[u] = fma(x[i], z[i], s4[u]);
          }
        }
        double sacc = (s4[0] + s4[1]) + (s4[2] + s4[3]);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) sacc += __shfl_xor_sync(0xffffffffu, sacc, o);
        if (lane == 0) {
          if (q < nbase * ncol) Gs[(q / ncol) * DOT_MAXC + (q % ncol)] = sacc;
          else Gkk[q - nbase * ncol] = sacc;
        }
      }
      __syncthreads();
      SmemEnt ent{Gs, Gkk, nullptr, nbase, kfirst, s_idx};
      if (scored) {
        PrefixFactor f;
        factor_prefix(ent, s_t, dp, a.ratio, f);
        double rel = 0.0;
        scored = f.ok && score_last(ent, s_t, dp, kfirst + e, a.ratio, f, &rel);
        if (scored) {
          if (a.shared_T > 0) {
            const double is = a.inv_s[(long long)tk * a.mp1];
            score += (is > 0.0 ? 1.0 / (is * is * (double)a.n_total) : 0.0) * rel;
          } else {
            score = rel;
          }
        }
      }
      __syncthreads();
    }
    const double rel = score;
    done_tuples += (threadIdx.x == 0) ? (unsigned long long)len : 0ull;
    int redo = 0;
    do {
      if (scored) {
        const float sc = (float)rel;
        const u64 key = key0 + (u64)e;
        if (cta_list_admits<float>(L, sc, key)) cta_list_push<float>(L, sc, key);
      }
      __syncthreads();
      if (++redo > L0_MAX_REDO) break;
    } while (cta_list_fold<float>(L, a.gthr + prob));
  }
  if (done_tuples) atomicAdd(a.n_tuples, done_tuples);
  const size_t slot = (size_t)prob * a.n_slots + a.slot0 + blockIdx.x;
  cta_list_flush<float>(L, a.out_s + slot * a.K, a.out_k + slot * a.K, a.out_cnt + slot);
}

}  // namespace

cudaError_t launch_defer(const DeferArgs &a, int groups, int n_probs, cudaStream_t st) {
  const size_t smem = cta_list_bytes<float>(a.K, a.S) + 16;
  cudaError_t e = cudaFuncSetAttribute(defer_gram_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(defer_dot_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem);
  if (e != cudaSuccess) return e;
  if (a.G64 && a.shared_T > 0) {
    defer_gram_kernel<<<dim3(groups, n_probs), L0_THREADS, smem, st>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  } else if (a.G64) {
    e = cudaFuncSetAttribute(defer_batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
    if (e != cudaSuccess) return e;
    defer_batch_kernel<<<dim3(groups, n_probs), L0_THREADS, smem, st>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  defer_dot_kernel<<<dim3(groups, n_probs), L0_THREADS, smem, st>>>(a);
  return cudaGetLastError();
}

}  // namespace l0
