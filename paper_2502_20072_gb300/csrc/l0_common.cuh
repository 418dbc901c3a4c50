// l0_common.cuh -- device machinery shared by the l0 kernels.
//
// * Tuple ranking (combinatorial number system).  Tuples are n ascending
//   column indices; the paper counts C(m, n) of them (Sec. 3.1).  The
//   lexicographic rank orders equal scores (smaller tuple first).
// * Order-preserving integer images of FP32/FP64 scores (atomicMin on a
//   global threshold).
// * A CTA-wide bounded top-K' list in shared memory with an unsorted staging
//   area: candidates are appended with one shared atomic; at CTA barriers the
//   staging area is bitonic-sorted and merged into the list (paper Sec. 2.4:
//   "returning the best one", here the best K').
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#define L0_DMAX 8
#define L0_THREADS 256

namespace l0 {

typedef unsigned long long u64;

// ------------------------------------------------------- ordered images --
__device__ __forceinline__ u64 ord_of(double x) {
  u64 b = (u64)__double_as_longlong(x);
  return (b & 0x8000000000000000ull) ? ~b : (b | 0x8000000000000000ull);
}
__device__ __forceinline__ u64 ord_of(float x) {
  unsigned b = __float_as_uint(x);
  unsigned o = (b & 0x80000000u) ? ~b : (b | 0x80000000u);
  return (u64)o;
}
template <typename R> __device__ __forceinline__ R from_ord(u64 o);
template <> __device__ __forceinline__ double from_ord<double>(u64 o) {
  u64 b = (o & 0x8000000000000000ull) ? (o & 0x7fffffffffffffffull) : ~o;
  return __longlong_as_double((long long)b);
}
template <> __device__ __forceinline__ float from_ord<float>(u64 o) {
  unsigned v = (unsigned)o;
  unsigned b = (v & 0x80000000u) ? (v & 0x7fffffffu) : ~v;
  return __uint_as_float(b);
}
// ordered image of +inf (the "no threshold yet" value)
template <typename R> __host__ __device__ __forceinline__ u64 ord_inf();
template <> __host__ __device__ __forceinline__ u64 ord_inf<double>() {
  return 0x7ff0000000000000ull | 0x8000000000000000ull;
}
template <> __host__ __device__ __forceinline__ u64 ord_inf<float>() {
  return (u64)(0x7f800000u | 0x80000000u);
}

template <typename R> __device__ __forceinline__ R r_inf();
template <> __device__ __forceinline__ double r_inf<double>() { return __longlong_as_double(0x7ff0000000000000ll); }
template <> __device__ __forceinline__ float r_inf<float>() { return __int_as_float(0x7f800000); }

// ------------------------------------------------------------ binomials --
// C(x, p) = t[p * stride + x] for 0 <= p <= L0_DMAX, 0 <= x < stride,
// saturated at 2^62 (sizes are validated on the host so saturation never
// reaches a rank that is used).
struct Binom {
  const u64 *t;
  int stride;
};
__device__ __forceinline__ u64 binom(const Binom &B, int p, int x) {
  return (x < 0) ? 0ull : __ldg(B.t + (size_t)p * B.stride + x);
}

// colex rank of a p-combination a[0] < .. < a[p-1]: sum C(a[i], i+1)
// lexicographic rank of a d-tuple t over [0, m): total - 1 - colex(b),
// b[i] = m - 1 - t[d - 1 - i]
__device__ __forceinline__ u64 lex_rank(const Binom &B, int m, int d,
                                        const int *t, u64 total) {
  u64 q = 0;
  for (int i = 0; i < d; ++i) q += binom(B, i + 1, m - 1 - t[d - 1 - i]);
  return total - 1ull - q;
}

// largest x in [lo, hi] with C(x, p) <= q  (C(lo, p) <= q required).
// C(x, p) ~ (x - (p - 1) / 2)^p / p! gives x to within a step or two; the
// table then confirms it (two independent loads, C(x, p) and C(x + 1, p)),
// so a level of an unrank waits for one or two trips to memory instead of
// the log2(hi - lo) of a bisection.
__device__ __forceinline__ int binom_floor(const Binom &B, int p, u64 q, int lo,
                                           int hi) {
  if (lo >= hi) return lo;
  if (p == 1) return q < (u64)hi ? (int)q : hi;   // C(x, 1) = x (q >= lo by the premise)
  // in FP32 (FP64 is a narrow pipe here): q to 2^-24, x to well within a step
  float f = 1.f;
  for (int i = 2; i <= p; ++i) f *= (float)i;
  const float xe = exp2f(__log2f((float)q * f) / (float)p) + 0.5f * (float)(p - 1);
  int x = !(xe >= (float)lo) ? lo : (xe > (float)hi ? hi : (int)xe);
  for (int guard = 0; guard < 64; ++guard) {
    const u64 c0 = binom(B, p, x);
    const u64 c1 = x < hi ? binom(B, p, x + 1) : 0ull;
    if (c0 > q) {            // too far: step down (C(lo, p) <= q ends it)
      --x;
      continue;
    }
    if (x < hi && c1 <= q) { // not far enough
      ++x;
      continue;
    }
    return x;
  }
  while (lo < hi) {          // the estimate was far off: bisection
    const int mid = (lo + hi + 1) >> 1;
    if (binom(B, p, mid) <= q) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ void lex_unrank(const Binom &B, int m, int d, u64 r,
                                           u64 total, int *t) {
  u64 q = total - 1ull - r;
  int hi = m - 1;
  for (int i = d; i >= 1; --i) {
    int b = binom_floor(B, i, q, i - 1, hi);
    q -= binom(B, i, b);
    t[d - i] = m - 1 - b;
    hi = b - 1;
  }
}

// colex unrank of a p-combination (universe unbounded, values < xmax)
__device__ __forceinline__ void colex_unrank(const Binom &B, int p, u64 r,
                                             int xmax, int *a) {
  int hi = xmax - 1;
  for (int i = p; i >= 1; --i) {
    int b = binom_floor(B, i, r, i - 1, hi);
    r -= binom(B, i, b);
    a[i - 1] = b;
    hi = b - 1;
  }
}

// C(x, p) by the multiplicative formula (exact while C(x, p) * x < 2^64)
__host__ __device__ __forceinline__ u64 binom_arith(int x, int p) {
  if (p < 0 || x < p) return 0ull;
  u64 r = 1ull;
  for (int i = 0; i < p; ++i) r = r * (u64)(x - i) / (u64)(i + 1);
  return r;
}

// colex unrank with arithmetic binomials (no table loads)
__device__ __forceinline__ void colex_unrank_arith(int p, u64 r, int xmax, int *a) {
  int hi = xmax - 1;
  for (int i = p; i >= 1; --i) {
    int lo = i - 1, h = hi;
    while (lo < h) {
      const int mid = (lo + h + 1) >> 1;
      if (binom_arith(mid, i) <= r) lo = mid; else h = mid - 1;
    }
    r -= binom_arith(lo, i);
    a[i - 1] = lo;
    hi = lo - 1;
  }
}

// lexicographic unrank with arithmetic binomials: no table loads, so no
// chain of dependent memory reads (the inverse of lex_rank)
__device__ __forceinline__ void lex_unrank_arith(int m, int d, u64 r, u64 total, int *t) {
  u64 q = total - 1ull - r;
  int hi = m - 1;
  for (int i = d; i >= 1; --i) {
    int lo = i - 1, h = hi;
    while (lo < h) {
      const int mid = (lo + h + 1) >> 1;
      if (binom_arith(mid, i) <= q) lo = mid; else h = mid - 1;
    }
    q -= binom_arith(lo, i);
    t[d - i] = m - 1 - lo;
    hi = lo - 1;
  }
}

// next p-combination in colex order
template <int P>
__device__ __forceinline__ void colex_next(int *a) {
#pragma unroll
  for (int i = 0; i < P; ++i) {
    int lim = (i + 1 < P) ? a[i + 1] : 0x7fffffff;
    if (a[i] + 1 < lim) {
      a[i] += 1;
#pragma unroll
      for (int q = 0; q < i; ++q) a[q] = q;
      return;
    }
  }
}

// ------------------------------------------------------- CTA top-K' list --
template <typename R>
__device__ __forceinline__ bool cand_less(R sa, u64 ka, R sb, u64 kb) {
  return (sa < sb) || (sa == sb && ka < kb);
}

// number of entries of sorted (s, k)[0..n) composite-less than (x, y)
template <typename R>
__device__ __forceinline__ int lower_count(const R *s, const u64 *k, int n, R x,
                                           u64 y) {
  int lo = 0, hi = n;
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if (cand_less(s[mid], k[mid], x, y)) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// ascending bitonic sort of n (power of two) entries, all threads of the CTA
template <typename R>
__device__ void cta_bitonic_sort(R *s, u64 *k, int n) {
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int size = 2; size <= n; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int i = tid; i < (n >> 1); i += nt) {
        int lo = 2 * stride * (i / stride) + (i % stride);
        int hi = lo + stride;
        bool asc = ((lo & size) == 0);
        R a = s[lo], b = s[hi];
        u64 ka = k[lo], kb = k[hi];
        bool sw = asc ? cand_less(b, kb, a, ka) : cand_less(a, ka, b, kb);
        if (sw) {
          s[lo] = b; s[hi] = a;
          k[lo] = kb; k[hi] = ka;
        }
      }
      __syncthreads();
    }
  }
}

// --------------------------------------------- global score histogram --
// Per problem, counts of the scores every tuple kernel CTA has staged:
// L0_HIST_FINE bins of 1/16 octave over the FP32 image of a score (rounded
// down), then L0_HIST_COARSE per-octave totals.  Every staged entry is a
// distinct real tuple (each tuple is evaluated once per search), so the
// upper edge of the first bin at which the running count reaches K' bounds
// the K'-th best score from above: it is a valid global cut long before any
// single CTA has K' candidates of its own.
#define L0_HIST_FINE 4096
#define L0_HIST_COARSE 256
#define L0_HIST_WORDS (L0_HIST_FINE + L0_HIST_COARSE)

__device__ __forceinline__ float f32_down(float s) { return s; }
__device__ __forceinline__ float f32_down(double s) { return __double2float_rd(s); }

// fine bin of a score, -1 for NaN
template <typename R>
__device__ __forceinline__ int score_bin(R s) {
  const float f = f32_down(s);
  if (f != f) return -1;
  if (!(f > 0.f)) return 0;
  const unsigned b = __float_as_uint(f) >> 19;
  return b < (unsigned)L0_HIST_FINE ? (int)b : L0_HIST_FINE - 1;
}

template <typename R>
__device__ __forceinline__ void hist_count(unsigned *hist, R s) {
  const int b = score_bin<R>(s);
  if (b < 0) return;
  atomicAdd(hist + b, 1u);
  atomicAdd(hist + L0_HIST_FINE + (b >> 4), 1u);
}

// Called by a whole warp: the ordered image of the smallest bin edge that at
// least K counted scores lie below, or ~0 when fewer than K were counted.
// The counts are read while other CTAs add to them; any snapshot undercounts,
// so the bound it gives is still valid.
template <typename R>
__device__ u64 hist_bound(const unsigned *hist, int K) {
  const int lane = threadIdx.x & 31;
  const unsigned FULL = 0xffffffffu;
  unsigned c[8], s = 0u;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    c[i] = __ldcg(hist + L0_HIST_FINE + lane * 8 + i);
    s += c[i];
  }
  unsigned inc = s;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned t = __shfl_up_sync(FULL, inc, o);
    if (lane >= o) inc += t;
  }
  if (__shfl_sync(FULL, inc, 31) < (unsigned)K) return ~0ull;
  const int lk = __ffs(__ballot_sync(FULL, inc >= (unsigned)K)) - 1;
  int oct = 0;
  unsigned before = 0u;
  if (lane == lk) {
    unsigned acc = inc - s;
    bool found = false;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      if (!found && acc + c[i] >= (unsigned)K) { oct = lane * 8 + i; before = acc; found = true; }
      if (!found) acc += c[i];
    }
  }
  oct = __shfl_sync(FULL, oct, lk);
  before = __shfl_sync(FULL, before, lk);
  unsigned f = (lane < 16) ? __ldcg(hist + oct * 16 + lane) : 0u;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned t = __shfl_up_sync(FULL, f, o);
    if (lane >= o) f += t;
  }
  const unsigned bl = __ballot_sync(FULL, lane < 16 && before + f >= (unsigned)K);
  // the fine counts may lag the coarse ones: then the octave's top edge
  const int b = bl ? oct * 16 + __ffs(bl) - 1 : oct * 16 + 15;
  if (b + 1 >= (int)(0x7f800000u >> 19)) return ~0ull;
  return ord_of((R)__uint_as_float((unsigned)(b + 1) << 19));
}

template <typename R>
struct CtaList {
  R *ls; u64 *lk;   // list [K], sorted ascending
  R *ss; u64 *sk;   // staging [S], unsorted
  R *ts; u64 *tk;   // merge temp [K]
  int K, S;
  int *n_list, *n_stage, *ovf;
  R *thr_s; u64 *thr_k;   // current composite threshold (list K'-th, global cut)
  R *gcut;                // global score cut, tightened between barriers
  int *dirty;             // staged since the histogram bound was last taken
  unsigned *hist;         // the problem's score histogram (tuple kernels only)
};

// bytes of shared memory a CtaList needs (plus 64 B of scalars)
template <typename R>
__host__ __device__ inline size_t cta_list_bytes(int K, int S) {
  return (size_t)(2 * K + S) * (sizeof(R) + sizeof(u64)) + 64;
}

template <typename R>
__device__ inline CtaList<R> cta_list_carve(unsigned char *&p, int K, int S) {
  CtaList<R> L;
  L.K = K; L.S = S;
  L.lk = (u64 *)p; p += (size_t)K * 8;
  L.sk = (u64 *)p; p += (size_t)S * 8;
  L.tk = (u64 *)p; p += (size_t)K * 8;
  L.ls = (R *)p; p += (size_t)K * sizeof(R);
  L.ss = (R *)p; p += (size_t)S * sizeof(R);
  L.ts = (R *)p; p += (size_t)K * sizeof(R);
  // scalars, 8-byte aligned
  p = (unsigned char *)(((uintptr_t)p + 7) & ~(uintptr_t)7);
  L.thr_k = (u64 *)p; p += 8;
  L.thr_s = (R *)p; p += 8;
  L.n_list = (int *)p; p += 4;
  L.n_stage = (int *)p; p += 4;
  L.ovf = (int *)p; p += 4;
  L.dirty = (int *)p; p += 4;
  L.gcut = (R *)p; p += 8;
  L.hist = nullptr;
  return L;
}

template <typename R>
__device__ inline void cta_list_reset(CtaList<R> &L, const u64 *gthr) {
  if (threadIdx.x == 0) {
    *L.n_list = 0;
    *L.n_stage = 0;
    *L.ovf = 0;
    *L.thr_s = gthr ? from_ord<R>(*(volatile const u64 *)gthr) : r_inf<R>();
    *L.thr_k = ~0ull;
    *L.gcut = *L.thr_s;
    *L.dirty = 0;
  }
}

// the score cut in force: a tuple scoring above it cannot be among the best K'
template <typename R>
__device__ __forceinline__ R cta_cut(const CtaList<R> &L) {
  const R a = *(volatile R *)L.thr_s, b = *(volatile R *)L.gcut;
  return b < a ? b : a;
}

// composite test against the current threshold, inclusive: the threshold
// is itself the K'-th key of a real tuple, which a redo must admit again
// (keys are unique, so nothing else can tie it)
template <typename R>
__device__ __forceinline__ bool cta_list_admits(const CtaList<R> &L, R s,
                                                u64 k) {
  R ts = *(volatile R *)L.thr_s;
  if (s < ts) return true;
  if (s > ts) return false;
  return k <= *(volatile u64 *)L.thr_k;
}

// bound on consecutive redos of one step; exceeding it is a bug, reported
// through the error word instead of looping
#define L0_MAX_REDO 4096

// append to the staging area; false (and the overflow flag set) when full
template <typename R>
__device__ __forceinline__ bool cta_list_push(CtaList<R> &L, R s, u64 k) {
  int idx = atomicAdd(L.n_stage, 1);
  if (idx < L.S) {
    L.ss[idx] = s;
    L.sk[idx] = k;
    if (L.hist) {
      hist_count<R>(L.hist, s);
      *(volatile int *)L.dirty = 1;
    }
    return true;
  }
  *(volatile int *)L.ovf = 1;
  return false;
}

// Fold the staging area into the list.  Call with all threads, after a
// barrier that follows the last push.  Returns true when the staging area
// had overflowed: nothing was committed, the threshold was tightened to the
// K'-th key of list U staging, and the caller must redo the step that
// produced the candidates (each redo admits at least S - K' fewer tuples,
// S > K').
template <typename R>
__device__ bool cta_list_fold(CtaList<R> &L, u64 *gthr) {
  const int tid = threadIdx.x, nt = blockDim.x;
  int ns = *(volatile int *)L.n_stage;
  const int ovf = *(volatile int *)L.ovf;
  if (ns == 0) return false;
  if (ns > L.S) ns = L.S;
  int P = 1;
  while (P < ns) P <<= 1;
  for (int i = ns + tid; i < P; i += nt) {
    L.ss[i] = r_inf<R>();
    L.sk[i] = ~0ull;
  }
  __syncthreads();
  cta_bitonic_sort<R>(L.ss, L.sk, P);
  const int nl = *(volatile int *)L.n_list;
  const int nout = min(L.K, nl + ns);
  for (int i = tid; i < nl; i += nt) {
    int pos = i + lower_count<R>(L.ss, L.sk, ns, L.ls[i], L.lk[i]);
    if (pos < L.K) { L.ts[pos] = L.ls[i]; L.tk[pos] = L.lk[i]; }
  }
  for (int i = tid; i < ns; i += nt) {
    int pos = i + lower_count<R>(L.ls, L.lk, nl, L.ss[i], L.sk[i]);
    if (pos < L.K) { L.ts[pos] = L.ss[i]; L.tk[pos] = L.sk[i]; }
  }
  __syncthreads();
  if (!ovf) {
    for (int i = tid; i < nout; i += nt) { L.ls[i] = L.ts[i]; L.lk[i] = L.tk[i]; }
  }
  if (tid == 0) {
    R ts = r_inf<R>();
    u64 tk = ~0ull;
    if (nout >= L.K) { ts = L.ts[L.K - 1]; tk = L.tk[L.K - 1]; }
    if (gthr) {
      if (!ovf && nout >= L.K) atomicMin(gthr, ord_of(ts));
      R g = from_ord<R>(*(volatile u64 *)gthr);
      if (g < ts) { ts = g; tk = ~0ull; }
    }
    // never loosen
    R cs = *L.thr_s;
    u64 ck = *L.thr_k;
    if (cand_less(ts, tk, cs, ck)) { *L.thr_s = ts; *L.thr_k = tk; }
    if (!ovf) *L.n_list = nout;
    *L.n_stage = 0;
    *L.ovf = 0;
  }
  __syncthreads();
  return ovf != 0;
}

// Commit every staged entry (all are real tuples that passed the threshold
// when staged) into the list, whatever the overflow flag says; entries that
// did not fit were not staged and their producers know it.  All threads,
// after a barrier that follows the last push.
template <typename R>
__device__ void cta_list_commit(CtaList<R> &L, u64 *gthr) {
  const int tid = threadIdx.x, nt = blockDim.x;
  int ns = *(volatile int *)L.n_stage;
  if (ns == 0) return;
  if (ns > L.S) ns = L.S;
  int P = 1;
  while (P < ns) P <<= 1;
  for (int i = ns + tid; i < P; i += nt) {
    L.ss[i] = r_inf<R>();
    L.sk[i] = ~0ull;
  }
  __syncthreads();
  cta_bitonic_sort<R>(L.ss, L.sk, P);
  const int nl = *(volatile int *)L.n_list;
  const int nout = min(L.K, nl + ns);
  for (int i = tid; i < nl; i += nt) {
    int pos = i + lower_count<R>(L.ss, L.sk, ns, L.ls[i], L.lk[i]);
    if (pos < L.K) { L.ts[pos] = L.ls[i]; L.tk[pos] = L.lk[i]; }
  }
  for (int i = tid; i < ns; i += nt) {
    int pos = i + lower_count<R>(L.ls, L.lk, nl, L.ss[i], L.sk[i]);
    if (pos < L.K) { L.ts[pos] = L.ss[i]; L.tk[pos] = L.sk[i]; }
  }
  __syncthreads();
  for (int i = tid; i < nout; i += nt) { L.ls[i] = L.ts[i]; L.lk[i] = L.tk[i]; }
  if (tid == 0) {
    R ts = r_inf<R>();
    u64 tk = ~0ull;
    if (nout >= L.K) { ts = L.ts[L.K - 1]; tk = L.tk[L.K - 1]; }
    if (gthr) {
      if (nout >= L.K) atomicMin(gthr, ord_of(ts));
      R g = from_ord<R>(*(volatile u64 *)gthr);
      if (g < ts) { ts = g; tk = ~0ull; }
    }
    R cs = *L.thr_s;
    u64 ck = *L.thr_k;
    if (cand_less(ts, tk, cs, ck)) { *L.thr_s = ts; *L.thr_k = tk; }
    if (ts < *L.gcut) *L.gcut = ts;
    *L.n_list = nout;
    *L.n_stage = 0;
    *L.ovf = 0;
  }
  __syncthreads();
}

// After a step, by warp 0 with no barrier: turn new stagings into a global
// bound through the histogram and pull the global bound (read at the start
// of the step, gprev) into the CTA's cut.  Other warps may read the cut
// meanwhile; both the old and the new value are valid cuts.
template <typename R>
__device__ __forceinline__ void cta_step_sync(CtaList<R> &L, u64 *gthr, u64 gprev) {
  if (threadIdx.x >= 32) return;
  u64 g = gprev;
  int dirty = 0;
  if (threadIdx.x == 0 && L.hist) dirty = atomicExch(L.dirty, 0);
  dirty = __shfl_sync(0xffffffffu, dirty, 0);
  if (dirty) {
    const u64 b = hist_bound<R>(L.hist, L.K);
    if (threadIdx.x == 0 && b < g) {
      atomicMin(gthr, b);
      g = b;
    }
  }
  if (threadIdx.x == 0 && g != ~0ull) {
    const R gs = from_ord<R>(g);
    if (gs < *(volatile R *)L.gcut) *(volatile R *)L.gcut = gs;
  }
}

// tighten the CTA threshold from the global one (thread 0; barrier after)
template <typename R>
__device__ __forceinline__ void cta_list_pull_global(CtaList<R> &L, const u64 *gthr) {
  if (threadIdx.x == 0 && gthr) {
    R g = from_ord<R>(*(volatile const u64 *)gthr);
    if (cand_less(g, ~0ull, *L.thr_s, *L.thr_k)) { *L.thr_s = g; *L.thr_k = ~0ull; }
  }
}

// write the list to global slot storage and reset it
template <typename R>
__device__ inline void cta_list_flush(CtaList<R> &L, R *out_s, u64 *out_k,
                                      int *out_cnt) {
  const int n = *(volatile int *)L.n_list;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    out_s[i] = L.ls[i];
    out_k[i] = L.lk[i];
  }
  if (threadIdx.x == 0) *out_cnt = n;
}

// Relaxed GPU-scope load of a word other CTAs update.  The load is issued
// where it stands and waited for only where its value is first used.
__device__ __forceinline__ u64 ld_relaxed(const u64 *p) {
  u64 v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p));
  return v;
}

// ------------------------------------------------------ packed FP32 pairs --
// two IEEE FP32 operations per instruction (fma.rn.f32x2: each half an fmaf)
__device__ __forceinline__ unsigned long long f2_pack(float a, float b) {
  return (unsigned long long)__float_as_uint(a) | ((unsigned long long)__float_as_uint(b) << 32);
}
__device__ __forceinline__ unsigned long long f2_fma(unsigned long long a, unsigned long long b,
                                                     unsigned long long c) {
  unsigned long long d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__device__ __forceinline__ unsigned long long f2_mul(unsigned long long a, unsigned long long b) {
  unsigned long long d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}

// --------------------------------------------------------- misc helpers --
__device__ __forceinline__ void set_err(int *err, int code) {
  if (err) atomicCAS(err, 0, code);
}

}  // namespace l0
