// l0_tile.cuh -- building blocks of the persistent tuple kernels: record
// buffers, records, the per-tuple fast test and its exact slow path, the
// step loop of one work item.  Included by l0_tuple.cu (PER_TASK problems)
// and l0_shared.cu (SHARED multi-task scoring).
#pragma once

#include "l0_kernels.cuh"

namespace l0 {
namespace tile {


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

// 1 / sqrt(x) for x > 0.  FP32: the hardware reciprocal square root.  FP64:
// that FP32 estimate refined by three Newton-Raphson steps
// y <- y (3 - x y^2) / 2, each of which squares the relative error, so the
// result carries full FP64 precision at the cost of a few FP64 FMAs (the
// records only need a consistent, accurate 1/l; no IEEE division).
__device__ __forceinline__ float inv_sqrt(float x) { return rsqrtf(x); }
__device__ __forceinline__ double inv_sqrt(double x) {
  double y = (double)rsqrtf((float)x);
#pragma unroll
  for (int i = 0; i < 3; ++i) y = y * fma(-0.5 * x, y * y, 1.5);
  return y;
}

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
  const int *cls;   // duplicate classes (or null)
  unsigned smem_dq; // tile32_kernel: shared address of its scratch (FP64-redo queue)
};

__device__ __forceinline__ bool same_class(const int *cls, int a, int b) {
  return cls && __ldg(cls + a) == __ldg(cls + b);
}

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
// Records are stored pre-negated where that turns every per-tuple operation
// into a plain FMA (bitwise the same values as the textbook signs):
//   row    jg = -g_j,  jinvl = 1 / l_j,  jz2 = z2_j,  je = pP_j - threshold
//   column kg = g_k,   kp1 = pthr_k - p1_k,  kw1 = -w1_k,  kpt = pthr_k
// so that  h = C_jk + jg.kg,  g2 = h jinvl,  -pp = g2^2 + kp1,
//          -w = g2 z2 + kw1,  t = w^2 + je (-pp).
//
// Record roles: in warp w, lanes 0..UJ-1 make the row records of the warp's
// own rows (w*UJ + lane), lanes UJ..UJ+15 the column records w*16 + lane-UJ;
// every warp does the same amount of record work.
constexpr int KREC_PER_WARP = TK / (L0_THREADS / 32);   // 16

__device__ __forceinline__ int record_col(int j0, int k0, bool &isj, bool &isk, int &idx) {
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  isj = lane < UJ;
  isk = !isj && lane < UJ + KREC_PER_WARP;
  if (isj) { idx = w * UJ + lane; return j0 + idx; }
  if (isk) { idx = w * KREC_PER_WARP + lane - UJ; return k0 + idx; }
  idx = -1;
  return -1;
}

// raw Gram values one record needs for prefix P
template <typename R, int DP>
struct RecRaw {
  R cpp[DP > 0 ? DP * (DP + 1) / 2 : 1];   // C[P_b][P_a], b <= a
  R cyp[DP > 0 ? DP : 1];                  // c_{P_a}
  R cpc[DP > 0 ? DP : 1];                  // C[P_p][col]
};

template <typename R, int DP>
__device__ __forceinline__ void load_raw(const ItemCtx<R> &c, const int *pidx, int col,
                                         RecRaw<R, DP> &raw) {
  const R *G = c.G;
  const long long ld = c.ld;
  int q = 0;
#pragma unroll
  for (int a = 0; a < DP; ++a) {
#pragma unroll
    for (int b = 0; b <= a; ++b) raw.cpp[q++] = G[(long long)(pidx[b] + 1) * ld + pidx[a] + 1];
    raw.cyp[a] = G[pidx[a] + 1];
    raw.cpc[a] = (col >= 0 && col < c.m) ? G[(long long)(pidx[a] + 1) * ld + col + 1] : R(0);
  }
}

// Values of one record (row j or column k) for one prefix.
template <typename R, int DPM>
struct RecOut {
  R g[DPM];
  R invl, z2, e, pPj;       // row record
  int flag;
  R kp1, kw1, kpt;          // column record
};

// Arithmetic of a record, free of branches on data (selects instead), then
// stored by rec_store.
template <typename R, int DP>
__device__ __forceinline__ void rec_compute(const ItemCtx<R> &c, const int *pidx,
                                            const RecRaw<R, DP> &raw, int col, R cdiag, R cy,
                                            R G00, R thr_s,
                                            RecOut<R, (DP > 0 ? DP : 1)> &o) {
  constexpr int DPM = DP > 0 ? DP : 1;
  constexpr bool MIXED = sizeof(R) == 4;
  // Cholesky of the prefix block C[P][P] and z_P = L_P^{-1} c_P
  R Lp[DPM][DPM];
  R invd[DPM];
  R zP[DPM];
  R pPb = G00;
  bool pok = true;
  int q = 0;
#pragma unroll
  for (int a = 0; a < DP; ++a) {
#pragma unroll
    for (int b = 0; b <= a; ++b) {
      R cab = raw.cpp[q++];
      const R orig = cab;
#pragma unroll
      for (int t = 0; t < b; ++t) cab -= Lp[a][t] * Lp[b][t];
      if (b < a) {
        Lp[a][b] = cab * invd[b];
      } else {
        pok = pok && (orig > R(0)) && (cab >= (R)c.ratio * orig);
        const R piv = cab > R(0) ? cab : R(1);
        invd[a] = inv_sqrt(piv);
        Lp[a][a] = piv * invd[a];
      }
    }
    R za = raw.cyp[a];
#pragma unroll
    for (int t = 0; t < a; ++t) za -= Lp[a][t] * zP[t];
    zP[a] = za * invd[a];
    pPb -= zP[a] * zP[a];
  }
  R piv = cdiag, w1 = cy;
#pragma unroll
  for (int p = 0; p < DP; ++p) {
    R gp = raw.cpc[p];
#pragma unroll
    for (int t = 0; t < p; ++t) gp -= Lp[p][t] * o.g[t];
    o.g[p] = gp * invd[p];
    piv -= o.g[p] * o.g[p];
    w1 -= o.g[p] * zP[p];
  }
  const bool inm = col < c.m;
#pragma unroll
  for (int p = 0; p < DPM; ++p) o.g[p] = (p < DP && inm) ? o.g[p] : R(0);
  const bool elig = (cdiag > R(0)) && (piv >= (R)c.ratio * cdiag);
  // two columns of one duplicate class: exactly rank deficient, ineligible
  // (never worth an FP64 redo)
  bool dup = false;
  if (c.cls && inm) {
#pragma unroll
    for (int a = 0; a < DP; ++a) {
      dup = dup || same_class(c.cls, pidx[a], col);
#pragma unroll
      for (int b = 0; b < a; ++b) dup = dup || same_class(c.cls, pidx[a], pidx[b]);
    }
  }
  // row record
  const bool shape = inm && (DP == 0 || pidx[DP > 0 ? DP - 1 : 0] < col);
  const R invl = inv_sqrt(piv > R(0) ? piv : R(1));
  const R z2 = w1 * invl;
  const R pPj = pPb - z2 * z2;
  const R e = pPj - (thr_s + (R)(16.0 * Eps<R>::v));
  const bool fast_ok = shape && !dup && pok && elig;
  o.flag = (!shape || dup) ? 0 : (!pok || !elig) ? (MIXED ? 3 : 0) : (e > R(0) ? 1 : 2);
  o.invl = fast_ok ? invl : R(0);
  o.z2 = fast_ok ? z2 : R(0);
  o.pPj = fast_ok ? pPj : R(0);
  o.e = fast_ok ? e : R(0);
  // column record: kp1 = pthr - p1 (negated); past m or ineligible: -inf
  // skips the column (FP64), +inf flags it for the FP64 redo (FP32)
  const R kpt = (R)c.ratio * cdiag;
  o.kpt = inm ? kpt : R(0);
  o.kw1 = inm ? -w1 : R(0);
  o.kp1 = !inm ? -r_inf<R>()
               : dup ? -r_inf<R>() : elig ? (kpt - piv) : (MIXED ? r_inf<R>() : -r_inf<R>());
}

template <typename R, int DPM>
__device__ __forceinline__ void rec_store(const RecOut<R, DPM> &o, bool isj, int idx,
                                          const RecBuf<R, DPM> &rb) {
  if (isj) {
#pragma unroll
    for (int p = 0; p < DPM; ++p) rb.jg[p * TJ + idx] = -o.g[p];
    rb.jinvl[idx] = o.invl;
    rb.jz2[idx] = o.z2;
    rb.je[idx] = o.e;
    rb.jpP[idx] = o.pPj;
    rb.jflag[idx] = o.flag;
  } else {
#pragma unroll
    for (int p = 0; p < DPM; ++p) rb.kg[p * TK + idx] = o.g[p];
    rb.kp1[idx] = o.kp1;
    rb.kw1[idx] = o.kw1;
    rb.kpt[idx] = o.kpt;
  }
}

template <typename R, int DP>
__device__ __forceinline__ void make_record(const ItemCtx<R> &c, const int *pidx,
                                            const RecRaw<R, DP> &raw, bool isj, bool isk,
                                            int idx, int col, R cdiag, R cy, R G00, R thr_s,
                                            const RecBuf<R, (DP > 0 ? DP : 1)> &rb) {
  constexpr int DPM = DP > 0 ? DP : 1;
  if (threadIdx.x == 0) {
#pragma unroll
    for (int p = 0; p < DP; ++p) rb.pidx[p] = pidx[p];
  }
  if (!isj && !isk) return;
  RecOut<R, DPM> o;
  rec_compute<R, DP>(c, pidx, raw, col, cdiag, cy, G00, thr_s, o);
  rec_store<R, DPM>(o, isj, idx, rb);
}

// ------------------------------------------------------------------ tuples --
template <typename R, int DPM>
struct KVals {
  R kg[DPM];
  R kp, kw;   // negated forms (kp1, kw1 of the records)
};

// Exact re-evaluation of one flagged tuple (rare): singular tuples are
// skipped (FP64) or queued for FP64 (FP32); the rest enter the CTA list when
// their (rel, lexicographic rank) beats the threshold.
// returns 1 when the tuple was staged (or needs nothing more), 0 when it must
// be looked at again after the staging area is emptied
template <typename R, int DP>
__device__ __noinline__ int slow_tuple(const TileArgs<R> &A, const ItemCtx<R> &c,
                                        const RecBuf<R, (DP > 0 ? DP : 1)> &rb,
                                        CtaList<R> &L, int jl, int v, R cjk,
                                        KVals<R, (DP > 0 ? DP : 1)> kv) {
  constexpr bool MIXED = sizeof(R) == 4;
  const int lane = threadIdx.x & 31;
  const int j = c.j0 + jl;
  const int kk = lane + 32 * v;
  const int k = c.k0 + kk;
  if (k >= c.m || k <= j) return 1;
  const R kpn = kv.kp;
  if (kpn == -r_inf<R>()) return 1;   // column ineligible after P (FP64) or past m
  if (MIXED && kpn == r_inf<R>()) {
    defer_run<R, DP>(A, c, rb.pidx, j, k, 1);
    return 1;
  }
  R h = cjk;
#pragma unroll
  for (int p = 0; p < DP; ++p) h = fma(rb.jg[p * TJ + jl], kv.kg[p], h);
  const R g2 = h * rb.jinvl[jl];
  const R pp = -fma(g2, g2, kpn);
  const R wn = fma(g2, rb.jz2[jl], kv.kw);
  if (!(pp >= R(0))) {           // pivot of k below the cut
    if (MIXED && !same_class(c.cls, j, k)) defer_run<R, DP>(A, c, rb.pidx, j, k, 1);
    return 1;
  }
  const R p = pp + rb.kpt[kk];
  const R rel = rb.jpP[jl] - wn * wn / p;
  if (rel > cta_cut<R>(L)) return 1;
  if (MIXED && A.band) {   // band pass: scored again in FP64
    defer_run<R, DP>(A, c, rb.pidx, j, k, 1);
    return 1;
  }
  int t[L0_DMAX];
#pragma unroll
  for (int q = 0; q < DP; ++q) t[q] = rb.pidx[q];
  t[DP] = j;
  t[DP + 1] = k;
  const u64 key = lex_rank(c.B, c.m, c.d, t, c.total);
  if (!cta_list_admits<R>(L, rel, key)) return 1;
  return cta_list_push<R>(L, rel, key) ? 1 : 0;
}

// sign bit of t (high word for FP64): 0 when t >= +0 (or NaN with clear sign)
__device__ __forceinline__ unsigned sign_word(float t) { return __float_as_uint(t); }
__device__ __forceinline__ unsigned sign_word(double t) { return (unsigned)__double2hiint(t); }


// Fast test of one row u against this thread's UK columns; returns the AND
// of the tuples' sign words (sign bit clear <=> some tuple flagged).
template <typename R, int DP, bool DIAG>
struct RowTest {
  static __device__ __forceinline__ unsigned run(const R (&cr)[UK],
                                                 const KVals<R, (DP > 0 ? DP : 1)> (&kv)[UK],
                                                 const R *jgn, R invl, R z2, R e,
                                                 unsigned diagmask) {
    unsigned acc = 0xffffffffu;
#pragma unroll
    for (int v = 0; v < UK; ++v) {
      R h = cr[v];
#pragma unroll
      for (int p = 0; p < DP; ++p) h = fma(jgn[p], kv[v].kg[p], h);
      const R g2 = h * invl;
      const R ppn = fma(g2, g2, kv[v].kp);
      const R wn = fma(g2, z2, kv[v].kw);
      const R t = fma(e, ppn, wn * wn);
      unsigned sw = sign_word(t);
      if (DIAG) sw |= ((diagmask >> v) & 1u) << 31;
      acc &= sw;
    }
    return acc;
  }
};

template <int DP, bool DIAG>
struct RowTest<float, DP, DIAG> {
  static __device__ __forceinline__ unsigned run(const float (&cr)[UK],
                                                 const KVals<float, (DP > 0 ? DP : 1)> (&kv)[UK],
                                                 const float *jgn, float invl, float z2, float e,
                                                 unsigned diagmask) {
    const unsigned long long invl2 = f2_pack(invl, invl), z22 = f2_pack(z2, z2),
                             e2 = f2_pack(e, e);
    unsigned acc = 0xffffffffu;
#pragma unroll
    for (int v = 0; v < UK; v += 2) {
      unsigned long long h = f2_pack(cr[v], cr[v + 1]);
#pragma unroll
      for (int p = 0; p < DP; ++p)
        h = f2_fma(f2_pack(jgn[p], jgn[p]), f2_pack(kv[v].kg[p], kv[v + 1].kg[p]), h);
      const unsigned long long g2 = f2_mul(h, invl2);
      const unsigned long long ppn = f2_fma(g2, g2, f2_pack(kv[v].kp, kv[v + 1].kp));
      const unsigned long long wn = f2_fma(g2, z22, f2_pack(kv[v].kw, kv[v + 1].kw));
      const unsigned long long t = f2_fma(e2, ppn, f2_mul(wn, wn));
      unsigned lo = (unsigned)t, hi = (unsigned)(t >> 32);
      if (DIAG) {
        lo |= ((diagmask >> v) & 1u) << 31;
        hi |= ((diagmask >> (v + 1)) & 1u) << 31;
      }
      acc &= lo & hi;
    }
    return acc;
  }
};

// `done` has a bit per (u, v) tuple of this thread already handled in this
// step (staged or redone); a pass after an overflow skips them.
template <typename R, int DP, bool DIAG>
__device__ __forceinline__ void tuple_step(const TileArgs<R> &A, const ItemCtx<R> &c,
                                           const RecBuf<R, (DP > 0 ? DP : 1)> &rb,
                                           const R (&creg)[UJ][UK], CtaList<R> &L,
                                           unsigned &done) {
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
  // flags of the warp's rows first (one pass), then every row's fast test
  // without branches; rows that are not fast rows are masked out
  unsigned fast_rows = 0u, exact_rows = 0u, dfr_rows = 0u;
#pragma unroll
  for (int u = 0; u < UJ; ++u) {
    const int f = rb.jflag[w * UJ + u];
    fast_rows |= (f == 1 ? 1u : 0u) << u;
    exact_rows |= (f == 2 ? 1u : 0u) << u;
    dfr_rows |= (f == 3 ? 1u : 0u) << u;
  }
  unsigned acc = 0xffffffffu;
  if (fast_rows) {
#pragma unroll
    for (int u = 0; u < UJ; ++u) {
      const int jl = w * UJ + u;
      R jg[DPM];
#pragma unroll
      for (int p = 0; p < DPM; ++p) jg[p] = rb.jg[p * TJ + jl];
      unsigned dm = 0u;
      if (DIAG) {
#pragma unroll
        for (int v = 0; v < UK; ++v) dm |= (c.k0 + lane + 32 * v <= c.j0 + jl ? 1u : 0u) << v;
      }
      const unsigned r = RowTest<R, DP, DIAG>::run(creg[u], kv, jg, rb.jinvl[jl], rb.jz2[jl],
                                                   rb.je[jl], dm);
      acc &= ((fast_rows >> u) & 1u) ? r : 0xffffffffu;
    }
  }
  if (MIXED && dfr_rows) {   // rows singular in FP32: redo them in FP64
#pragma unroll
    for (int u = 0; u < UJ; ++u) {
      if (!((dfr_rows >> u) & 1u)) continue;
      const int jl = w * UJ + u;
      if (lane == 0 && !((done >> (u * UK)) & 1u)) {
        const int j = c.j0 + jl;
        const int kf = c.k0 > j + 1 ? c.k0 : j + 1;
        const int kl = c.k0 + TK < c.m ? c.k0 + TK : c.m;
        defer_run<R, DP>(A, c, rb.pidx, j, kf, kl - kf);
      }
      done |= 1u << (u * UK);
    }
  }
  if (exact_rows) {
#pragma unroll
    for (int u = 0; u < UJ; ++u) {
      if (!((exact_rows >> u) & 1u)) continue;
      const int jl = w * UJ + u;
#pragma unroll
      for (int v = 0; v < UK; ++v) {
        const unsigned bit = 1u << (u * UK + v);
        if (!(done & bit) && slow_tuple<R, DP>(A, c, rb, L, jl, v, creg[u][v], kv[v])) done |= bit;
      }
    }
  }
  if (!(acc >> 31)) {
    // a flagged tuple in this thread's block: redo the cheap test per tuple
    // and re-evaluate only the flagged ones exactly
#pragma unroll
    for (int u = 0; u < UJ; ++u) {
      const int jl = w * UJ + u;
      if (!((fast_rows >> u) & 1u)) continue;
      R jg[DPM];
#pragma unroll
      for (int p = 0; p < DPM; ++p) jg[p] = rb.jg[p * TJ + jl];
      const R invl = rb.jinvl[jl], z2 = rb.jz2[jl], e = rb.je[jl];
#pragma unroll
      for (int v = 0; v < UK; ++v) {
        R h = creg[u][v];
#pragma unroll
        for (int p = 0; p < DP; ++p) h = fma(jg[p], kv[v].kg[p], h);
        const R g2 = h * invl;
        const R ppn = fma(g2, g2, kv[v].kp);
        const R wn = fma(g2, z2, kv[v].kw);
        const R t = fma(e, ppn, wn * wn);
        const unsigned bit = 1u << (u * UK + v);
        if (!(sign_word(t) >> 31) && !(done & bit) &&
            slow_tuple<R, DP>(A, c, rb, L, jl, v, creg[u][v], kv[v]))
          done |= bit;
      }
    }
  }
}

// One work item: the CTA's (j, k) tile against prefix colex ranks [r0, r1).
// Records for step r+1 are made before the tuples of step r, into the other
// buffer, so each step needs one barrier; the global loads for the records
// of step r+2 are issued before the tuples of step r, so their latency hides
// behind a full step.
template <typename R, int DP, bool DIAG>
__device__ __forceinline__ void run_steps(const TileArgs<R> &A, const ItemCtx<R> &c,
                                          int *pidx, u64 r0, u64 r1, R cdiag, R cy, R G00,
                                          const RecBuf<R, (DP > 0 ? DP : 1)> (&rbs)[2],
                                          const R (&creg)[UJ][UK], CtaList<R> &L, u64 *gthr) {
  constexpr int DPM = DP > 0 ? DP : 1;
  bool isj, isk;
  int idx;
  const int col = record_col(c.j0, c.k0, isj, isk, idx);
  const bool rec = isj || isk;
  RecRaw<R, DP> raw;
  if (rec) load_raw<R, DP>(c, pidx, col, raw);
  make_record<R, DP>(c, pidx, raw, isj, isk, idx, col, cdiag, cy, G00, cta_cut<R>(L), rbs[0]);
  int pn[DPM];   // prefix of step r + 1
#pragma unroll
  for (int p = 0; p < DPM; ++p) pn[p] = pidx[p];
  if (DP > 0) colex_next<DP>(pn);
  if (rec && r0 + 1 < r1) load_raw<R, DP>(c, pn, col, raw);
  __syncthreads();
  u64 gnext = ~0ull;   // warp 0: the global bound, read a step before it is used
  for (u64 r = r0; r < r1; ++r) {
    const int buf = (int)((r - r0) & 1ull);
    const u64 gprev = gnext;
    if (threadIdx.x < 32) gnext = ld_relaxed(gthr);
    if (r + 1 < r1) {
      make_record<R, DP>(c, pn, raw, isj, isk, idx, col, cdiag, cy, G00, cta_cut<R>(L),
                         rbs[buf ^ 1]);
      if (DP > 0) colex_next<DP>(pn);
      if (rec && r + 2 < r1) load_raw<R, DP>(c, pn, col, raw);
    }
    // Candidates stay staged across steps; the list is folded when the
    // staging area is half full.  A step that overflows it commits what was
    // staged and resumes, skipping the tuples it already handled.
    unsigned done = 0u;
    for (int pass = 0;; ++pass) {
      tuple_step<R, DP, DIAG>(A, c, rbs[buf], creg, L, done);
      __syncthreads();
      const bool ovf = *(volatile int *)L.ovf != 0;
      if (ovf || *(volatile int *)L.n_stage > L.S / 2) cta_list_commit<R>(L, gthr);
      if (!ovf) break;
      if (pass > L0_MAX_REDO) {
        set_err(A.err, 8);
        break;
      }
    }
    cta_step_sync<R>(L, gthr, gprev);
  }
  // staged entries are committed by the caller at the end of the item
}



// Persistent work loop shared by the tuple kernels: fetch a work item with
// one atomic, decode it into (problem, j tile, k tile, prefix range), hand it
// to run(), and write the CTA's list to its slot whenever the problem changes.
// Per item the loop costs one barrier pair and no trip to global memory: the
// next item's number is fetched during the current one, the decode reads the
// row-block table (cached in shared memory) with 32-bit arithmetic, the
// item bodies keep the global cut fresh themselves (a relaxed read a step or
// group ahead), and staged candidates are committed to the CTA list only when
// the staging area fills, by the item bodies, and before the list is
// written out.  `forward`: items go out in row-block order, first row block
// first (see the decode below).
template <typename R, typename RunItem>
__device__ __forceinline__ void persistent_items(const TileArgs<R> &A, RunItem run,
                                                 bool forward = false) {
  extern __shared__ __align__(16) unsigned char smem[];
  unsigned char *p = smem;
  CtaList<R> L = cta_list_carve<R>(p, A.K, A.S);
  p = (unsigned char *)(((uintptr_t)p + 15) & ~(uintptr_t)15);
  unsigned char *recbase = p;
  __shared__ long long s_item;
  __shared__ long long s_rowpre[1024];
  int cur = -1;
  // the problem descriptors, when few, live in shared memory for the loop
  constexpr int PD_SMEM = 16;
  __shared__ ProbDesc s_pd[PD_SMEM];
  const int tid = threadIdx.x;
  const bool rp_smem = A.rowpre_len <= 1024;
  if (rp_smem)
    for (int i = tid; i < A.rowpre_len; i += blockDim.x) s_rowpre[i] = A.row_prefix[i];
  const bool pd_smem = A.n_probs <= PD_SMEM;
  if (pd_smem)
    for (int q = tid; q < A.n_probs; q += blockDim.x) s_pd[q] = A.probs[q];
  const ProbDesc *probs = pd_smem ? s_pd : A.probs;
  // thread 0 takes the next item's number while the CTA runs the current
  // one, so no item waits for the atomic's round trip, and publishes it in
  // s_item before the barrier that ends each item
  if (tid == 0) s_item = (long long)atomicAdd(A.item_counter, 1ull);
  long long nxt = 0;
  __syncthreads();
  for (;;) {
    const long long item = s_item * A.item_stride + A.item_offset;
    if (tid == 0 && item < A.item_limit) nxt = (long long)atomicAdd(A.item_counter, 1ull);
    int prob = -1;
    if (item < A.item_limit)
      for (int q = 0; q < A.n_probs; ++q)
        if (item >= probs[q].item_begin && item < probs[q].item_end) { prob = q; break; }
    if (prob != cur) {
      if (cur >= 0) {
        cta_list_commit<R>(L, A.gthr + cur);   // what is still staged joins the list
        __syncthreads();
        const size_t slot = (size_t)cur * A.n_slots + blockIdx.x;
        cta_list_flush<R>(L, A.out_s + slot * A.K, A.out_k + slot * A.K, A.out_cnt + slot);
      }
      __syncthreads();
      cur = prob;
      if (prob >= 0) cta_list_reset<R>(L, A.gthr + prob);
      L.hist = (prob >= 0 && A.hist) ? A.hist + (size_t)prob * L0_HIST_WORDS : nullptr;
      __syncthreads();
    }
    if (prob < 0) break;   // past the last item (uniform)
    const ProbDesc pd = probs[prob];
    // Items are laid out by row block, the later blocks holding the most
    // prefix steps.  By default they go out last block first, so the
    // persistent CTAs end on the small items and finish together.  With
    // equal chunks (the FP32 d <= 3 kernel) the cost of an item is set by
    // how often its tuples flag instead: a tile holding the strongest
    // columns flags on every group.  Columns come ranked by SIS score, so
    // the first row blocks hold the strongest; `forward` hands those out
    // first, and the tail of the launch is made of ordinary items.
    const long long local = forward ? item - pd.item_begin : pd.item_end - 1 - item;
    const long long *rp =
        (rp_smem ? s_rowpre : A.row_prefix) + (size_t)pd.prefix_off * ROWINFO;
    int lo = 0, hi = pd.n_jt - 1;
    while (lo < hi) {
      int mid = (lo + hi + 1) >> 1;
      if (rp[(size_t)mid * ROWINFO] <= local) lo = mid; else hi = mid - 1;
    }
    const int bj = lo;
    const long long *ri = rp + (size_t)bj * ROWINFO;
    // the row block's items: k tile major, then the tile's nch prefix
    // chunks, which split its prefixes evenly (the first rr hold q + 1, the
    // rest q; none above L), so items of one tile cost the same
    const int rem = (int)(local - ri[0]);   // < k tiles x chunks of one row block
    const int nch = (int)ri[1];
    const int bk = nch > 0 ? rem / nch : 0;
    const u64 ch = (u64)(rem - bk * nch);
    const u64 q = (u64)ri[2], rr = (u64)ri[3];
    const u64 r0 = ch * q + (ch < rr ? ch : rr);
    const u64 r1 = r0 + q + (ch < rr ? 1ull : 0ull);
    if (nch <= 0 || bk >= tile_k_count(bj, pd.m) || r1 <= r0 || r1 - r0 > (u64)pd.L) {   // inconsistent plan
      set_err(A.err, 9);
      break;
    }
    u64 *gthr = A.gthr + prob;
    run(pd, prob, bj, bk, r0, r1, L, recbase, gthr);
    if (tid == 0) s_item = nxt;   // every thread read this item's number before run()
    __syncthreads();
  }
}

}  // namespace tile
}  // namespace l0
