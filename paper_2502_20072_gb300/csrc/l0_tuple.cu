// l0_tuple.cu -- the persistent tuple kernel (enumeration, per-tuple solve,
// top-K' selection) and the d = 1 kernel.
//
// Score of a tuple (paper Sec. 2.4): the least-squares fit of the tuple's
// features (plus intercept) to the target, scored by its squared deviation.
// With the augmented correlation matrix G of the centred, scaled columns
// (target first), the relative residual of tuple tau is the last pivot of the
// Cholesky factorisation of G restricted to (target, tau):
//     rel(tau) = SSE(tau) / S_yy = 1 - c_tau^T C_tau^{-1} c_tau .
// The paper computes the same quantity by Householder QR of the descriptor
// matrix assembled per descriptor; here one Gram serves all tuples.
//
// Enumeration.  A tuple is (P, j, k): an outer prefix P of d-2 indices (in
// colex order), then j < k.  A CTA owns a 64 x 128 tile of (j, k) pairs, keeps
// the Gram entries C[j][k] of the tile in registers and walks a chunk of
// prefixes P.  For each P the CTA computes, in shared memory,
//   row records   (P, j): g_j = L_P^{-1} C[P][j], 1/l_j, z2_j, pP_j, e_j
//   column records(P, k): g_k = L_P^{-1} C[P][k], p1_k - pthr_k, w1_k
// where L_P is the Cholesky factor of C[P][P] and l_j the pivot of j after P.
// Each tuple then costs (d = 3: one FMA for h, then 5 FP ops)
//     h   = C[j][k] - g_j . g_k          (Schur complement of P)
//     g2  = h / l_j
//     pp  = p1_k - pthr_k - g2^2         (pivot of k after P and j, minus cut)
//     w   = w1_k - g2 z2_j
//     t   = w^2 - e_j pp,   e_j = pP_j - threshold
// t >= 0 flags a tuple that may beat the current threshold (or a singular
// one); flagged tuples are redone exactly (rel = pP_j - w^2 / p) on a slow
// path that feeds the CTA's top-K' list.
#include "l0_kernels.cuh"

namespace l0 {

namespace {

constexpr int UJ = TILE_UJ;
constexpr int UK = TILE_UK;
constexpr int TJ = TILE_TJ;
constexpr int TK = TILE_TK;

template <typename R> struct Eps;
template <> struct Eps<double> { static constexpr double v = 2.220446049250313e-16; };
template <> struct Eps<float> { static constexpr double v = 1.1920928955078125e-07; };

template <typename R, int DPM>
struct RecBuf {
  R *jg;                       // [DPM][TJ]
  R *jinvl, *jz2, *je, *jpP;   // [TJ]
  R *kg;                       // [DPM][TK]
  R *kp1, *kw1, *kpt;          // [TK]
  int *jflag;                  // [TJ]: 0 skip, 1 fast, 2 exact, 3 redo in FP64
  int *pidx;                   // [DPM]
};

template <typename R, int DPM>
__host__ __device__ constexpr size_t rec_bytes() {
  return (size_t)((DPM + 4) * TJ + (DPM + 3) * TK) * sizeof(R) +
         (size_t)(TJ + DPM + 4) * sizeof(int);
}

template <typename R, int DPM>
__device__ RecBuf<R, DPM> rec_carve(unsigned char *p) {
  RecBuf<R, DPM> b;
  R *r = (R *)p;
  b.jg = r; r += DPM * TJ;
  b.jinvl = r; r += TJ;
  b.jz2 = r; r += TJ;
  b.je = r; r += TJ;
  b.jpP = r; r += TJ;
  b.kg = r; r += DPM * TK;
  b.kp1 = r; r += TK;
  b.kw1 = r; r += TK;
  b.kpt = r; r += TK;
  int *q = (int *)r;
  b.jflag = q; q += TJ;
  b.pidx = q;
  return b;
}

__host__ __device__ constexpr size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }

// Context of one work item shared by the step functions.
template <typename R>
struct ItemCtx {
  const R *G;
  long long ld;
  int m, d, j0, k0, prob;
  bool diag;
  u64 total;
  Binom B;
  R ratio;
};

template <typename R, int DP>
__device__ __forceinline__ void defer_run(const TileArgs<R> &A, const ItemCtx<R> &c,
                                          const int *pidx, int j, int kfirst, int count) {
  if (count <= 0) return;
  int t[L0_DMAX];
#pragma unroll
  for (int p = 0; p < DP; ++p) t[p] = pidx[p];
  t[DP] = j;
  t[DP + 1] = kfirst;
  u64 key = lex_rank(c.B, c.m, c.d, t, c.total);
  atomicAdd(A.dfr_n + 1, (u64)count);
  u64 slot = atomicAdd(A.dfr_n, 1ull);
  if ((long long)slot < A.dfr_cap) {
    A.dfr_key[slot] = key;
    A.dfr_len[slot] = ((unsigned)c.prob << 8) | (unsigned)count;
  } else {
    set_err(A.err, 7);   // deferral buffer overflow
  }
}

// ---------------------------------------------------------------- records --
template <typename R, int DP>
__device__ __forceinline__ void compute_records(const ItemCtx<R> &c, const int *pidx,
                                                R cdiag, R cy, R G00, R thr_s,
                                                const RecBuf<R, (DP > 0 ? DP : 1)> &rb) {
  constexpr int DPM = DP > 0 ? DP : 1;
  constexpr bool MIXED = sizeof(R) == 4;
  const int tid = threadIdx.x;
  const bool isj = tid < TJ;
  const bool isk = (tid >= TJ) && (tid < TJ + TK);
  if (tid == 0) {
#pragma unroll
    for (int p = 0; p < DP; ++p) rb.pidx[p] = pidx[p];
  }
  if (!isj && !isk) return;
  const R *G = c.G;
  const long long ld = c.ld;
  // Cholesky of the prefix block C[P][P] and z_P = L_P^{-1} c_P
  R Lp[DPM][DPM];
  R invd[DPM];
  R zP[DPM];
  R pPb = G00;
  bool pok = true;
#pragma unroll
  for (int a = 0; a < DP; ++a) {
    const int ia = pidx[a];
#pragma unroll
    for (int b = 0; b <= a; ++b) {
      R cab = G[(long long)(pidx[b] + 1) * ld + ia + 1];
      const R orig = cab;
#pragma unroll
      for (int q = 0; q < b; ++q) cab -= Lp[a][q] * Lp[b][q];
      if (b < a) {
        Lp[a][b] = cab * invd[b];
      } else {
        pok = pok && (orig > R(0)) && (cab >= (R)c.ratio * orig);
        R piv = cab > R(0) ? cab : R(1);
        R l = sqrt(piv);
        Lp[a][a] = l;
        invd[a] = R(1) / l;
      }
    }
    R za = G[ia + 1];
#pragma unroll
    for (int q = 0; q < a; ++q) za -= Lp[a][q] * zP[q];
    zP[a] = za * invd[a];
    pPb -= zP[a] * zP[a];
  }
  const int idx = isj ? tid : tid - TJ;
  const int col = isj ? c.j0 + idx : c.k0 + idx;
  R g[DPM];
  R piv = cdiag, w1 = cy;
  if (col < c.m) {
#pragma unroll
    for (int p = 0; p < DP; ++p) {
      R gp = G[(long long)(pidx[p] + 1) * ld + col + 1];
#pragma unroll
      for (int q = 0; q < p; ++q) gp -= Lp[p][q] * g[q];
      g[p] = gp * invd[p];
      piv -= g[p] * g[p];
      w1 -= g[p] * zP[p];
    }
  } else {
#pragma unroll
    for (int p = 0; p < DP; ++p) g[p] = R(0);
  }
  const bool elig = (cdiag > R(0)) && (piv >= (R)c.ratio * cdiag);
  if (isj) {
    const int j = col;
    const bool shape = (j < c.m) && (DP == 0 || pidx[DP > 0 ? DP - 1 : 0] < j);
    int flag;
    R invl = R(0), z2 = R(0), pPj = R(0), e = R(0);
    if (!shape) {
      flag = 0;
    } else if (!pok || !elig) {
      flag = MIXED ? 3 : 0;
    } else {
      R l = sqrt(piv);
      invl = R(1) / l;
      z2 = w1 * invl;
      pPj = pPb - z2 * z2;
      R tl = thr_s + (R)(16.0 * Eps<R>::v);
      e = pPj - tl;
      flag = (e > R(0)) ? 1 : 2;
    }
#pragma unroll
    for (int p = 0; p < DPM; ++p) rb.jg[p * TJ + idx] = (p < DP) ? g[p] : R(0);
    rb.jinvl[idx] = invl;
    rb.jz2[idx] = z2;
    rb.je[idx] = e;
    rb.jpP[idx] = pPj;
    rb.jflag[idx] = flag;
  } else {
    R kp1, kw1, kpt;
    if (col >= c.m) {
      kp1 = r_inf<R>();
      kw1 = R(0);
      kpt = R(0);
    } else {
      kpt = (R)c.ratio * cdiag;
      kp1 = elig ? (piv - kpt) : (MIXED ? -r_inf<R>() : r_inf<R>());
      kw1 = w1;
    }
#pragma unroll
    for (int p = 0; p < DPM; ++p) rb.kg[p * TK + idx] = (p < DP) ? g[p] : R(0);
    rb.kp1[idx] = kp1;
    rb.kw1[idx] = kw1;
    rb.kpt[idx] = kpt;
  }
}

// ------------------------------------------------------------------ tuples --
template <typename R, int DPM>
struct KVals {
  R kg[DPM];
  R kp, kw;
};

// Exact re-evaluation of one flagged tuple (rare): singular tuples are
// skipped (FP64) or queued for FP64 (FP32); the rest enter the CTA list when
// their (rel, lexicographic rank) beats the threshold.
template <typename R, int DP>
__device__ __noinline__ void slow_tuple(const TileArgs<R> &A, const ItemCtx<R> &c,
                                        const RecBuf<R, (DP > 0 ? DP : 1)> &rb,
                                        CtaList<R> &L, int jl, int v, R cjk,
                                        KVals<R, (DP > 0 ? DP : 1)> kv) {
  constexpr int DPM = DP > 0 ? DP : 1;
  constexpr bool MIXED = sizeof(R) == 4;
  const int lane = threadIdx.x & 31;
  const int j = c.j0 + jl;
  const int kk = lane + 32 * v;
  const int k = c.k0 + kk;
  if (k >= c.m || k <= j) return;
  const R kp = kv.kp;
  if (kp == r_inf<R>()) return;   // column ineligible after P (FP64) or past m
  if (MIXED && kp == -r_inf<R>()) {
    defer_run<R, DP>(A, c, rb.pidx, j, k, 1);
    return;
  }
  R h = cjk;
#pragma unroll
  for (int p = 0; p < DP; ++p) h = fma(-rb.jg[p * TJ + jl], kv.kg[p], h);
  const R g2 = h * rb.jinvl[jl];
  const R pp = fma(-g2, g2, kp);
  const R w = fma(-g2, rb.jz2[jl], kv.kw);
  if (!(pp >= R(0))) {           // pivot of k below the cut
    if (MIXED) defer_run<R, DP>(A, c, rb.pidx, j, k, 1);
    return;
  }
  const R p = pp + rb.kpt[kk];
  const R rel = rb.jpP[jl] - w * w / p;
  const R ts = *(volatile R *)L.thr_s;
  if (rel > ts) return;
  int t[L0_DMAX];
#pragma unroll
  for (int q = 0; q < DP; ++q) t[q] = rb.pidx[q];
  t[DP] = j;
  t[DP + 1] = k;
  const u64 key = lex_rank(c.B, c.m, c.d, t, c.total);
  if (cta_list_admits<R>(L, rel, key)) cta_list_push<R>(L, rel, key);
  (void)DPM;
}

template <typename R, int DP>
__device__ __forceinline__ void tuple_step(const TileArgs<R> &A, const ItemCtx<R> &c,
                                           const RecBuf<R, (DP > 0 ? DP : 1)> &rb,
                                           const R (&creg)[UJ][UK], CtaList<R> &L) {
  constexpr int DPM = DP > 0 ? DP : 1;
  constexpr bool MIXED = sizeof(R) == 4;
  const int lane = threadIdx.x & 31;
  const int w = threadIdx.x >> 5;
  KVals<R, DPM> kv[UK];
#pragma unroll
  for (int v = 0; v < UK; ++v) {
    const int kk = lane + 32 * v;
    kv[v].kp = rb.kp1[kk];
    kv[v].kw = rb.kw1[kk];
#pragma unroll
    for (int p = 0; p < DPM; ++p) kv[v].kg[p] = rb.kg[p * TK + kk];
  }
  R acc = -r_inf<R>();
  unsigned exact_rows = 0u;
#pragma unroll
  for (int u = 0; u < UJ; ++u) {
    const int jl = w * UJ + u;
    const int flag = rb.jflag[jl];
    if (flag == 1) {
      R jg[DPM];
#pragma unroll
      for (int p = 0; p < DPM; ++p) jg[p] = rb.jg[p * TJ + jl];
      const R invl = rb.jinvl[jl], z2 = rb.jz2[jl], e = rb.je[jl];
#pragma unroll
      for (int v = 0; v < UK; ++v) {
        R h = creg[u][v];
#pragma unroll
        for (int p = 0; p < DP; ++p) h = fma(-jg[p], kv[v].kg[p], h);
        const R g2 = h * invl;
        const R pp = fma(-g2, g2, kv[v].kp);
        const R wv = fma(-g2, z2, kv[v].kw);
        R t = fma(-e, pp, wv * wv);
        if (c.diag && (c.k0 + lane + 32 * v <= c.j0 + jl)) t = -r_inf<R>();
        acc = fmax(acc, t);
      }
    } else if (flag == 2) {
      exact_rows |= 1u << u;
    } else if (flag == 3) {  // the row is singular in FP32: redo it in FP64
      if (MIXED && lane == 0) {
        const int j = c.j0 + jl;
        const int kf = c.k0 > j + 1 ? c.k0 : j + 1;
        const int kl = c.k0 + TK < c.m ? c.k0 + TK : c.m;
        defer_run<R, DP>(A, c, rb.pidx, j, kf, kl - kf);
      }
    }
  }
  if (exact_rows) {
#pragma unroll
    for (int u = 0; u < UJ; ++u) {
      if (!((exact_rows >> u) & 1u)) continue;
      const int jl = w * UJ + u;
#pragma unroll
      for (int v = 0; v < UK; ++v)
        slow_tuple<R, DP>(A, c, rb, L, jl, v, creg[u][v], kv[v]);
    }
  }
  if (acc >= R(0)) {
    // a flagged tuple in this thread's block: recompute the cheap test and
    // re-evaluate only the flagged tuples exactly
#pragma unroll
    for (int u = 0; u < UJ; ++u) {
      const int jl = w * UJ + u;
      if (rb.jflag[jl] != 1) continue;
      R jg[DPM];
#pragma unroll
      for (int p = 0; p < DPM; ++p) jg[p] = rb.jg[p * TJ + jl];
      const R invl = rb.jinvl[jl], z2 = rb.jz2[jl], e = rb.je[jl];
#pragma unroll
      for (int v = 0; v < UK; ++v) {
        R h = creg[u][v];
#pragma unroll
        for (int p = 0; p < DP; ++p) h = fma(-jg[p], kv[v].kg[p], h);
        const R g2 = h * invl;
        const R pp = fma(-g2, g2, kv[v].kp);
        const R wv = fma(-g2, z2, kv[v].kw);
        const R t = fma(-e, pp, wv * wv);
        if (t >= R(0)) slow_tuple<R, DP>(A, c, rb, L, jl, v, creg[u][v], kv[v]);
      }
    }
  }
}

template <typename R, int DP>
__device__ void run_item(const TileArgs<R> &A, const ProbDesc &pd, int prob, int bj, int bk,
                         u64 r0, u64 r1, CtaList<R> &L, unsigned char *recbase,
                         u64 *gthr) {
  constexpr int DPM = DP > 0 ? DP : 1;
  constexpr size_t RB = align16(rec_bytes<R, DPM>());
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  ItemCtx<R> c;
  c.G = A.G + pd.g_off;
  c.ld = pd.ld;
  c.prob = prob;
  c.m = pd.m;
  c.d = pd.d;
  c.j0 = bj * TJ;
  c.k0 = bk * TK;
  c.diag = (c.k0 <= c.j0 + TJ - 1);
  c.total = pd.total;
  c.B = A.B;
  c.ratio = (R)A.ratio;
  const R *G = c.G;
  const long long ld = c.ld;
  R creg[UJ][UK];
#pragma unroll
  for (int u = 0; u < UJ; ++u) {
    const int j = c.j0 + w * UJ + u;
#pragma unroll
    for (int v = 0; v < UK; ++v) {
      const int k = c.k0 + lane + 32 * v;
      creg[u][v] = (j < c.m && k < c.m) ? G[(long long)(j + 1) * ld + k + 1] : R(0);
    }
  }
  // base values of this thread's record column
  R cdiag = R(0), cy = R(0);
  {
    int col = -1;
    if (tid < TJ) col = c.j0 + tid;
    else if (tid < TJ + TK) col = c.k0 + tid - TJ;
    if (col >= 0 && col < c.m) {
      cdiag = G[(long long)(col + 1) * (ld + 1)];
      cy = G[col + 1];
    }
  }
  const R G00 = G[0];
  int pidx[DPM];
  {
    int jend = min(c.j0 + TJ, c.m);
    if (DP > 0) colex_unrank(c.B, DP, r0, jend - 1, pidx);
    else pidx[0] = 0;
  }
  const RecBuf<R, DPM> rb = rec_carve<R, DPM>(recbase);
  for (u64 r = r0; r < r1; ++r) {
    compute_records<R, DP>(c, pidx, cdiag, cy, G00, *(volatile R *)L.thr_s, rb);
    __syncthreads();
    int redo = 0;
    do {
      tuple_step<R, DP>(A, c, rb, creg, L);
      __syncthreads();
      if (++redo > L0_MAX_REDO) {
        set_err(A.err, 8);
        break;
      }
    } while (cta_list_fold<R>(L, gthr));
    if (DP > 0) colex_next<DP>(pidx);
  }
  (void)RB;
}

template <typename R, int DPLO, int DPHI>
__global__ void __launch_bounds__(L0_THREADS)
tile_kernel(TileArgs<R> A) {
  extern __shared__ __align__(16) unsigned char smem[];
  unsigned char *p = smem;
  CtaList<R> L = cta_list_carve<R>(p, A.K, A.S);
  p = (unsigned char *)(((uintptr_t)p + 15) & ~(uintptr_t)15);
  unsigned char *recbase = p;
  __shared__ long long s_item;
  int cur = -1;
  const int tid = threadIdx.x;
  for (;;) {
    if (tid == 0) s_item = (long long)atomicAdd(A.item_counter, 1ull);
    __syncthreads();
    const long long item = s_item;
    int prob = -1;
    for (int q = 0; q < A.n_probs; ++q)
      if (item >= A.probs[q].item_begin && item < A.probs[q].item_end) { prob = q; break; }
    if (prob != cur) {
      if (cur >= 0) {
        const size_t slot = (size_t)cur * A.n_slots + blockIdx.x;
        cta_list_flush<R>(L, A.out_s + slot * A.K, A.out_k + slot * A.K, A.out_cnt + slot);
      }
      __syncthreads();
      cur = prob;
      if (prob >= 0) cta_list_reset<R>(L, A.gthr + prob);
    } else if (prob >= 0) {
      cta_list_pull_global<R>(L, A.gthr + prob);
    }
    __syncthreads();
    if (prob < 0) break;   // past the last item (uniform)
    const ProbDesc pd = A.probs[prob];
    const long long local = item - pd.item_begin;
    const long long *rp = A.row_prefix + pd.prefix_off;
    int lo = 0, hi = pd.n_jt - 1;
    while (lo < hi) {
      int mid = (lo + hi + 1) >> 1;
      if (rp[mid] <= local) lo = mid; else hi = mid - 1;
    }
    const int bj = lo;
    const long long rem = local - rp[bj];
    const int jend = min((bj + 1) * TJ, pd.m);
    const u64 np = binom(A.B, pd.dp, jend - 1);
    const long long nch = (long long)((np + (u64)pd.L - 1) / (u64)pd.L);
    const int bk_min = (bj * TJ + 1) / TK;
    const int bk = bk_min + (int)(rem / nch);
    const u64 r0 = (u64)(rem % nch) * (u64)pd.L;
    const u64 r1 = (r0 + (u64)pd.L < np) ? r0 + (u64)pd.L : np;
    if (bk >= pd.n_kt || r1 <= r0 || r1 - r0 > (u64)pd.L) {   // inconsistent plan
      set_err(A.err, 9);
      break;
    }
    u64 *gthr = A.gthr + prob;
    switch (pd.dp) {
#define L0_CASE(X)                                                           \
  case X:                                                                    \
    if (X >= DPLO && X <= DPHI)                                              \
      run_item<R, (X >= DPLO && X <= DPHI ? X : DPLO)>(A, pd, prob, bj, bk,  \
                                                             r0, r1, L,      \
                                                             recbase, gthr); \
    break;
      L0_CASE(0)
      L0_CASE(1)
      L0_CASE(2)
      L0_CASE(3)
      L0_CASE(4)
      L0_CASE(5)
      L0_CASE(6)
#undef L0_CASE
      default:
        break;
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------------ d = 1 --
template <typename R>
__global__ void __launch_bounds__(L0_THREADS)
singles_kernel(const R *Gbase, const ProbDesc *probs, int K, int S, u64 *gthr,
               R *out_s, u64 *out_k, int *out_cnt, int n_slots) {
  extern __shared__ __align__(16) unsigned char smem[];
  unsigned char *p = smem;
  CtaList<R> L = cta_list_carve<R>(p, K, S);
  const int prob = blockIdx.y;
  const ProbDesc pd = probs[prob];
  const R *G = Gbase + pd.g_off;
  const long long ld = pd.ld;
  cta_list_reset<R>(L, gthr + prob);
  __syncthreads();
  const R G00 = G[0];
  const int nt = blockDim.x;
  for (int base = blockIdx.x * nt; base < pd.m; base += gridDim.x * nt) {
    const int k = base + threadIdx.x;
    R rel = R(0);
    bool ok = false;
    if (k < pd.m) {
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
    } while (cta_list_fold<R>(L, gthr + prob));
  }
  const size_t slot = (size_t)prob * n_slots + blockIdx.x;
  cta_list_flush<R>(L, out_s + slot * K, out_k + slot * K, out_cnt + slot);
}

}  // namespace

template <typename R>
size_t tile_smem_bytes(int K, int S, int dp_hi) {
  size_t rb = 0;
  switch (dp_hi) {
    case 0: case 1: rb = align16(rec_bytes<R, 1>()); break;
    case 2: rb = align16(rec_bytes<R, 2>()); break;
    case 3: rb = align16(rec_bytes<R, 3>()); break;
    case 4: rb = align16(rec_bytes<R, 4>()); break;
    case 5: rb = align16(rec_bytes<R, 5>()); break;
    default: rb = align16(rec_bytes<R, 6>()); break;
  }
  return align16(cta_list_bytes<R>(K, S)) + 16 + rb;
}

template <typename R>
static const void *tile_fn(int dp_lo, int dp_hi) {
#define L0_K(LO, HI) \
  if (dp_lo == LO && dp_hi == HI) return (const void *)tile_kernel<R, LO, HI>;
  L0_K(0, 0) L0_K(1, 1) L0_K(2, 2) L0_K(3, 3) L0_K(4, 4) L0_K(5, 5) L0_K(6, 6)
#undef L0_K
  return nullptr;
}

template <typename R>
cudaError_t tile_occupancy(int dp_lo, int dp_hi, size_t smem, int *blocks_per_sm) {
  const void *fn = tile_fn<R>(dp_lo, dp_hi);
  if (!fn) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, fn, L0_THREADS, smem);
}

template <typename R>
cudaError_t launch_tile(const TileArgs<R> &a, int dp_lo, int dp_hi, int grid,
                        size_t smem, cudaStream_t st) {
  const void *fn = tile_fn<R>(dp_lo, dp_hi);
  if (!fn) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  void *args[] = {(void *)&a};
  return cudaLaunchKernel(fn, dim3(grid), dim3(L0_THREADS), args, smem, st);
}

template <typename R>
cudaError_t launch_singles(const R *G, const ProbDesc *, const ProbDesc *probs_dev,
                           int n_probs, int K, int S, int grid_x, u64 *gthr,
                           R *out_s, u64 *out_k, int *out_cnt, int n_slots,
                           cudaStream_t st) {
  size_t smem = cta_list_bytes<R>(K, S) + 16;
  cudaError_t e = cudaFuncSetAttribute(singles_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  singles_kernel<R><<<dim3(grid_x, n_probs), L0_THREADS, smem, st>>>(
      G, probs_dev, K, S, gthr, out_s, out_k, out_cnt, n_slots);
  return cudaGetLastError();
}

template size_t tile_smem_bytes<double>(int, int, int);
template size_t tile_smem_bytes<float>(int, int, int);
template cudaError_t tile_occupancy<double>(int, int, size_t, int *);
template cudaError_t tile_occupancy<float>(int, int, size_t, int *);
template cudaError_t launch_tile<double>(const TileArgs<double> &, int, int, int, size_t, cudaStream_t);
template cudaError_t launch_tile<float>(const TileArgs<float> &, int, int, int, size_t, cudaStream_t);
template cudaError_t launch_singles<double>(const double *, const ProbDesc *, const ProbDesc *, int, int, int, int, u64 *, double *, u64 *, int *, int, cudaStream_t);
template cudaError_t launch_singles<float>(const float *, const ProbDesc *, const ProbDesc *, int, int, int, int, u64 *, float *, u64 *, int *, int, cudaStream_t);

}  // namespace l0
