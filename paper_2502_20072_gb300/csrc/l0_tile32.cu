// l0_tile32.cu -- the FP32 tuple kernel for d = 2 and d = 3.
//
// The same search as tile_kernel (l0_tuple.cu; paper Sec. 2.4: every tuple
// fitted by least squares, the best kept), on the same work items, CTA lists,
// global cut, FP64 redo queue and merge, written for the two tuple sizes the
// FP32 form runs most: one prefix index i (d = 3) or none (d = 2).  A CTA owns
// a 64 (j) x 128 (k) tile of the Gram in registers and walks prefixes i < j;
// per prefix ("step") it needs only row i of the Gram:
//
//   row record j    g_j = C_ij / l_i, 1/l_j, z2_j, e_j = pP_j - cut
//   column record k g_k = C_ik / l_i, pthr_k - p1_k, -w1_k
//
// (l_i = sqrt(C_ii), l_j the pivot of j after i, z2_j and pP_j the target
// column of the Cholesky factor after (i, j)).  Each tuple then costs the
// five packed operations of the fast test
//
//   h = C_jk - g_j g_k,  g2 = h / l_j,  -p = g2^2 + (pthr_k - p1_k),
//   -w = g2 z2_j - w1_k,  t = w^2 - e_j p      (flagged when t >= 0),
//
// two tuples per fma.rn.f32x2.  What differs from tile_kernel:
//  * steps go in groups of T32_G prefixes: the records of a whole group are
//    built by all threads together (load-balanced, per-record constants in
//    shared memory), then every thread runs the test of the group's steps
//    against the same register tile, with one barrier and one list check
//    per group instead of per step;
//  * the row segments of G[i+1] a step needs (64 + 128 entries) are copied
//    into shared memory by the TMA unit (cp.async.bulk) through a ring of
//    two groups of stages with mbarrier completion, a group ahead;
//  * records are stored duplicated ((x, x) pairs) so that every operand of
//    the packed test comes from one 64- or 128-bit shared load, with no
//    register moves; each lane holds adjacent column pairs (2 lane, 2 lane+1)
//    so the column records load as pairs too;
//  * the row state (skip, exact, redo in FP64) is folded into e: +inf never
//    flags, a positive NaN always flags (and the exact path reads the
//    state); no flag loads or masks in the test;
//  * the diagonal tile masks k <= j with the sign of (2 lane - j), one
//    integer add per row; every other tile runs the bare test;
//  * the histogram bound that tightens the global cut is read with cp.async
//    a phase per group, never waited for inside a group;
//  * shapes of 256 threads (8 rows per warp, one or two CTAs per SM) and
//    512 threads (4 rows per warp).
// Flagged tuples take the same exact path as tile_kernel (FP32 relative
// score, composite admission with the lexicographic rank, FP64 redo of
// near-singular tuples), so both kernels produce the same candidate lists.
#include "l0_tile.cuh"
#include "l0_tc.cuh"

namespace l0 {

namespace {

using namespace tile;

constexpr int T32_G = 4;           // prefix steps per group (one barrier each)
constexpr int T32_NS = 2 * T32_G;  // stages of the Gram-row ring: two groups
constexpr int T32_JSEG = 68;       // floats of G[i+1][j0 .. j0 + 68)
constexpr int T32_KSEG = 132;      // floats of G[i+1][k0 - 1 .. k0 + 131)
constexpr int T32_SEG = T32_JSEG + T32_KSEG;
constexpr int T32_MAXL = 256;      // prefix steps per item (plan_problems caps L)
constexpr int T32_NREC = TJ + TK;  // records per step

// Shared memory beyond the CTA list, at fixed offsets from one base pointer
// (one register addresses all of it):
//   2 T32_G record buffers (two groups), each
//     row   [TJ] x 32 B: {(-g, -g), (1/l, 1/l)}, {(z2, z2), (e, e)}
//     jpP   [TJ] floats (pP_j, exact path), jflag [TJ] ints (0 skip, 1 fast,
//           2 exact, 3 redo in FP64)
//     kg, kp, kw, kpt [TK] floats
//   the ring [NS][SEG] floats, the item's prefix scalars (1/l_i, z_i, pP_i,
//   class) [MAXL] each, the item's per-record constants (column, C_cc, r_c, class)
//   [TJ + TK] each, the ring's mbarriers [NS], the histogram copies
constexpr int R_ROW = 0;
constexpr int R_JPP = R_ROW + TJ * 32;
constexpr int R_JFLAG = R_JPP + TJ * 4;
constexpr int R_KG = R_JFLAG + TJ * 4;
constexpr int R_KP = R_KG + TK * 4;
constexpr int R_KW = R_KP + TK * 4;
constexpr int R_KPT = R_KW + TK * 4;
constexpr int T32_REC_BYTES = R_KPT + TK * 4;
constexpr int O_STAGE = 2 * T32_G * T32_REC_BYTES;
constexpr int O_PDG = O_STAGE + T32_NS * T32_SEG * 4;
constexpr int O_PRY = O_PDG + T32_MAXL * 4;
constexpr int O_PCLS = O_PRY + T32_MAXL * 4;
constexpr int O_PPB = O_PCLS + T32_MAXL * 4;
constexpr int O_RCOL = O_PPB + T32_MAXL * 4;
constexpr int O_RDG = O_RCOL + T32_NREC * 4;
constexpr int O_RY = O_RDG + T32_NREC * 4;
constexpr int O_RCLS = O_RY + T32_NREC * 4;
constexpr int O_BAR = O_RCLS + T32_NREC * 4;
constexpr int O_HC = O_BAR + T32_NS * 8;              // histogram octave counts [256]
constexpr int O_HF = O_HC + L0_HIST_COARSE * 4;       // one octave's fine counts [16]
constexpr int T32_DQ = 512;                           // FP64-redo runs queued per group
constexpr int O_DQK = O_HF + 64;                      // queued runs: first lex rank [DQ]
constexpr int O_DQL = O_DQK + T32_DQ * 8;             // (problem << 8) | length [DQ]
constexpr int O_DQN = O_DQL + T32_DQ * 4;             // runs, tuples, global base
constexpr int T32_FQ = 2048;                          // flagged tuples queued per group
constexpr int O_FQ = O_DQN + 16;                      // flagged tuples [FQ] (see fq_pack)
constexpr int O_FQS = O_FQ + T32_FQ * 8;              // their state: 1 once handled [FQ]
constexpr int O_FQN = O_FQS + T32_FQ;                 // queued count, overflow flag
constexpr size_t T32_EXTRA_BYTES = (size_t)O_FQN + 16;
static_assert(O_STAGE % 16 == 0 && (T32_JSEG * 4) % 16 == 0 && (T32_SEG * 4) % 16 == 0,
              "TMA destinations must be 16-byte aligned");
static_assert(O_BAR % 8 == 0, "mbarriers are 8-byte aligned");
static_assert(O_HC % 16 == 0 && O_HF % 16 == 0, "cp.async destinations are 16-byte aligned");
static_assert(O_DQK % 8 == 0 && O_FQ % 8 == 0 && O_FQN % 4 == 0, "queue alignment");

// one record buffer
struct Rec32 {
  unsigned char *p;
  __device__ __forceinline__ ulonglong2 *row() const { return (ulonglong2 *)(p + R_ROW); }
  __device__ __forceinline__ float *jpP() const { return (float *)(p + R_JPP); }
  __device__ __forceinline__ int *jflag() const { return (int *)(p + R_JFLAG); }
  __device__ __forceinline__ float *kg() const { return (float *)(p + R_KG); }
  __device__ __forceinline__ float *kp() const { return (float *)(p + R_KP); }
  __device__ __forceinline__ float *kw() const { return (float *)(p + R_KW); }
  __device__ __forceinline__ float *kpt() const { return (float *)(p + R_KPT); }
};

constexpr float T32_MARGIN = (float)(16.0 * 1.1920928955078125e-07);   // 16 ulp of 1

// Shared-memory accesses of the hot path by 32-bit shared addresses
// (ld.shared / st.shared), so they never go through generic addressing.
__device__ __forceinline__ u64 lds64(uint32_t a) {
  u64 v;
  asm volatile("ld.shared.b64 %0, [%1];" : "=l"(v) : "r"(a));
  return v;
}
__device__ __forceinline__ ulonglong2 lds128(uint32_t a) {
  ulonglong2 v;
  asm volatile("ld.shared.v2.b64 {%0, %1}, [%2];" : "=l"(v.x), "=l"(v.y) : "r"(a));
  return v;
}
__device__ __forceinline__ void sts128(uint32_t a, ulonglong2 v) {
  asm volatile("st.shared.v2.b64 [%0], {%1, %2};" ::"r"(a), "l"(v.x), "l"(v.y) : "memory");
}
__device__ __forceinline__ void sts32(uint32_t a, float v) {
  asm volatile("st.shared.f32 [%0], %1;" ::"r"(a), "f"(v) : "memory");
}
__device__ __forceinline__ void sts32i(uint32_t a, int v) {
  asm volatile("st.shared.b32 [%0], %1;" ::"r"(a), "r"(v) : "memory");
}
__device__ __forceinline__ float lds32(uint32_t a) {
  float v;
  asm volatile("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"(a));
  return v;
}
__device__ __forceinline__ int lds32i(uint32_t a) {
  int v;
  asm volatile("ld.shared.b32 %0, [%1];" : "=r"(v) : "r"(a));
  return v;
}

// ------------------------------------------------- histogram bound, pipelined --
// The global cut is tightened from the problem's score histogram (see
// hist_bound in l0_common.cuh) whenever this CTA staged something.  Reading
// the counts takes two dependent trips to L2; tile_kernel's warp 0 waits for
// both inside the step and the next barrier waits for warp 0.  Here warp 0
// copies the counts into shared memory with cp.async (L2 only, so the other
// CTAs' atomics are seen) and uses them a step later, one phase per step:
//   phase 0: if something was staged, start the copy of the octave counts;
//   phase 1: find the octave where the running count reaches K', start the
//            copy of its 16 fine counts;
//   phase 2: the bin where it reaches K' -> its upper edge bounds the K'-th
//            best score -> atomicMin on the global cut.
// Any snapshot undercounts, so a bound from older counts is still valid.
struct HistPipe {
  int phase;
  int oct;
  unsigned before;
};

__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// warp 0, after each step, no barrier; gprev = the global cut read a step ago
__device__ __forceinline__ void step_sync32(CtaList<float> &L, u64 *gthr, u64 gprev,
                                            HistPipe &hp, unsigned char *sb) {
  if (threadIdx.x >= 32) return;
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x;
  unsigned *hc = (unsigned *)(sb + O_HC), *hf = (unsigned *)(sb + O_HF);
  u64 g = gprev;
  if (hp.phase == 2) {
    cp_async_wait_all();
    __syncwarp();
    unsigned f = lane < 16 ? hf[lane] : 0u;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned t = __shfl_up_sync(FULL, f, o);
      if (lane >= o) f += t;
    }
    const unsigned bl = __ballot_sync(FULL, lane < 16 && hp.before + f >= (unsigned)L.K);
    // fine counts may lag the octave's: then the octave's top edge
    const int b = bl ? hp.oct * 16 + __ffs(bl) - 1 : hp.oct * 16 + 15;
    if (b + 1 < (int)(0x7f800000u >> 19)) {
      const u64 bound = ord_of(__uint_as_float((unsigned)(b + 1) << 19));
      if (bound < g) {
        if (lane == 0) atomicMin(gthr, bound);
        g = bound;
      }
    }
    hp.phase = 0;
  } else if (hp.phase == 1) {
    cp_async_wait_all();
    __syncwarp();
    unsigned c[8], s = 0u;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      c[i] = hc[lane * 8 + i];
      s += c[i];
    }
    unsigned inc = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned t = __shfl_up_sync(FULL, inc, o);
      if (lane >= o) inc += t;
    }
    hp.phase = 0;
    if (__shfl_sync(FULL, inc, 31) >= (unsigned)L.K) {
      const int lk = __ffs(__ballot_sync(FULL, inc >= (unsigned)L.K)) - 1;
      int oct = 0;
      unsigned before = 0u;
      if (lane == lk) {
        unsigned acc = inc - s;
        bool found = false;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          if (!found && acc + c[i] >= (unsigned)L.K) { oct = lane * 8 + i; before = acc; found = true; }
          if (!found) acc += c[i];
        }
      }
      hp.oct = __shfl_sync(FULL, oct, lk);
      hp.before = __shfl_sync(FULL, before, lk);
      if (lane < 4) cp_async16(tc::smem_u32(hf + 4 * lane), L.hist + hp.oct * 16 + 4 * lane);
      cp_async_commit();
      hp.phase = 2;
    }
  } else {
    int dirty = 0;
    if (lane == 0 && L.hist) dirty = atomicExch(L.dirty, 0);
    if (__shfl_sync(FULL, dirty, 0)) {
      const unsigned *src = L.hist + L0_HIST_FINE + lane * 8;
      cp_async16(tc::smem_u32(hc + lane * 8), src);
      cp_async16(tc::smem_u32(hc + lane * 8 + 4), src + 4);
      cp_async_commit();
      hp.phase = 1;
    }
  }
  if (lane == 0 && g != ~0ull) {
    const float gs = from_ord<float>(g);
    if (gs < *(volatile float *)L.gcut) *(volatile float *)L.gcut = gs;
  }
}

// state of one work item shared by the record builds
struct Item32 {
  ItemCtx<float> c;   // tile position, problem, binomials (shared with tile_kernel's helpers)
  float G00;          // 1 (the scaled target's own entry)
};

// One record (r < TJ: row record of j0 + r; else column record of
// k0 + r - TJ) of one step.  DP = 1: prefix i with 1/l_i = |pinv| (negative
// when C_ii is not positive), z_i = pz, pP_i = ppb and class pcls (computed
// once per step for all the step's records), the raw entry C_i,col from the
// staged row segment; DP = 0: no prefix.  The arithmetic is tile_kernel's
// rec_compute for these sizes.
template <int DP>
__device__ __forceinline__ void build32(const Item32 &it, unsigned char *sb, int r, int i,
                                        float pinv, float pz, float ppb, int pcls,
                                        const float *seg, const Rec32 &rb, float cut) {
  const ItemCtx<float> &c = it.c;
  const bool isj = r < TJ;
  const uint32_t s0 = tc::smem_u32(sb);
  const int col = lds32i(s0 + O_RCOL + 4u * r);
  const float cdiag = lds32(s0 + O_RDG + 4u * r);
  const float cy = lds32(s0 + O_RY + 4u * r);
  const int ccls = lds32i(s0 + O_RCLS + 4u * r);
  const float ratio = c.ratio;
  float invd = 1.f, zP = 0.f, pPb = it.G00, craw = 0.f;
  bool pok = true;
  if (DP == 1) {
    pok = pinv > 0.f;
    invd = fabsf(pinv);
    zP = pz;
    pPb = ppb;
    // seg: [JSEG] = G[i+1][j0 ..), then [KSEG] = G[i+1][k0 - 1 ..)
    craw = isj ? seg[r + 1] : seg[T32_JSEG + (r - TJ) + 2];
  }
  const bool inm = col < c.m;
  const float g = craw * invd;
  const float piv = cdiag - g * g;
  const float w1 = cy - g * zP;
  const bool elig = (cdiag > 0.f) && (piv >= ratio * cdiag);
  const bool dup = DP == 1 && c.cls != nullptr && inm && pcls == ccls;
  if (isj) {
    const bool shape = inm && (DP == 0 || i < col);
    const float invl = rsqrtf(piv > 0.f ? piv : 1.f);
    const float z2 = w1 * invl;
    const float pPj = pPb - z2 * z2;
    const float e = pPj - (cut + T32_MARGIN);
    const int flag = (!shape || dup) ? 0 : (!pok || !elig) ? 3 : (e > 0.f ? 1 : 2);
    const bool fast = flag == 1 || flag == 2;
    const float gn = fast ? -g : 0.f, il = fast ? invl : 0.f, zz = fast ? z2 : 0.f;
    // +inf never flags a tuple (skipped row); a positive NaN always does (exact
    // and redo rows: the exact path reads the state, whatever the column)
    const float ee = flag == 1 ? e : (flag == 0 ? r_inf<float>() : __uint_as_float(0x7fc00000u));
    ulonglong2 a, b;
    a.x = f2_pack(gn, gn);
    a.y = f2_pack(il, il);
    b.x = f2_pack(zz, zz);
    b.y = f2_pack(ee, ee);
    const uint32_t rs = tc::smem_u32(rb.p);
    sts128(rs + R_ROW + (uint32_t)r * 32u, a);
    sts128(rs + R_ROW + (uint32_t)r * 32u + 16u, b);
    sts32(rs + R_JPP + (uint32_t)r * 4u, fast ? pPj : 0.f);
    sts32i(rs + R_JFLAG + (uint32_t)r * 4u, flag);
  } else {
    const uint32_t kk4 = (uint32_t)(r - TJ) * 4u;
    const float kpt = ratio * cdiag;
    const uint32_t rs = tc::smem_u32(rb.p);
    sts32(rs + R_KG + kk4, inm ? g : 0.f);
    sts32(rs + R_KP + kk4, (!inm || dup) ? -r_inf<float>() : (elig ? kpt - piv : r_inf<float>()));
    sts32(rs + R_KW + kk4, inm ? -w1 : 0.f);
    sts32(rs + R_KPT + kk4, inm ? kpt : 0.f);
  }
}

// Fast test of this thread's UJ rows x 4 columns (columns 2 lane + b + 64 q of
// the tile): the AND of the tuples' sign words (bit 31 clear <=> something
// flagged).  In the diagonal tile (k0 = j0 + 1) column 2 lane + b of half q = 0
// is k <= j exactly when 2 lane + b - jl < 0: that sign is OR-ed in.
template <int UJ, bool DIAG>
__device__ __forceinline__ unsigned fast32(const u64 (&creg)[UJ][2], uint32_t rw, uint32_t rl,
                                           int d0base) {
  // rw = record buffer + row records of this warp's first row; rl = record
  // buffer + this lane's first column pair (kg); the rest are immediates
  u64 kg[2], kp[2], kw[2];
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    kg[q] = lds64(rl + 256u * q);
    kp[q] = lds64(rl + (R_KP - R_KG) + 256u * q);
    kw[q] = lds64(rl + (R_KW - R_KG) + 256u * q);
  }
  unsigned acc = 0xffffffffu;
#pragma unroll
  for (int u = 0; u < UJ; ++u) {
    const ulonglong2 a = lds128(rw + 32u * u);
    const ulonglong2 b = lds128(rw + 32u * u + 16u);
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const u64 h = f2_fma(a.x, kg[q], creg[u][q]);
      const u64 g2 = f2_mul(h, a.y);
      const u64 ppn = f2_fma(g2, g2, kp[q]);
      const u64 wn = f2_fma(g2, b.x, kw[q]);
      const u64 t = f2_fma(b.y, ppn, f2_mul(wn, wn));
      const unsigned lo = (unsigned)t, hi = (unsigned)(t >> 32);
      if (DIAG && q == 0) {
        const int d0 = d0base - u;   // 2 lane - jl: negative where k <= j
        acc &= (lo | (unsigned)d0) & (hi | (unsigned)(d0 + 1));
      } else {
        acc &= lo & hi;
      }
    }
  }
  return acc;
}

// FP64-redo runs of a group are queued in shared memory (a shared atomic
// each) and handed to the global queue by flush32 after the group's barrier,
// with one global atomic per counter per CTA instead of two per run.  A full
// shared queue falls back to the global queue directly.
template <int DP>
__device__ __forceinline__ void defer32(const TileArgs<float> &A, const ItemCtx<float> &c, int i,
                                        int j, int kfirst, int count) {
  if (count <= 0) return;
  unsigned char *sb = (unsigned char *)__cvta_shared_to_generic(c.smem_dq);
  int *dqn = (int *)(sb + O_DQN);
  const int slot = atomicAdd(dqn, 1);
  if (slot < T32_DQ) {
    int t[L0_DMAX];
    if (DP == 1) {
      t[0] = i;
      t[1] = j;
      t[2] = kfirst;
    } else {
      t[0] = j;
      t[1] = kfirst;
    }
    ((u64 *)(sb + O_DQK))[slot] = lex_rank(c.B, c.m, c.d, t, c.total);
    ((unsigned *)(sb + O_DQL))[slot] = ((unsigned)c.prob << 8) | (unsigned)count;
    atomicAdd(dqn + 1, count);
  } else {
    int pidx[1] = {i};
    defer_run<float, DP>(A, c, pidx, j, kfirst, count);
  }
}

// After a group's barrier, when runs were queued (uniform: read after the
// barrier): reserve their slots in the global queue with one atomic, copy,
// and empty the shared queue.  Two barriers: the slots are known to all
// before the copy, and the copy ends before the queue is written again.
__device__ __forceinline__ void flush32(const TileArgs<float> &A, unsigned char *sb, int n_q) {
  int *dqn = (int *)(sb + O_DQN);
  const int n = n_q < T32_DQ ? n_q : T32_DQ;
  if (threadIdx.x == 0) {
    const u64 base = atomicAdd(A.dfr_n, (u64)n);
    atomicAdd(A.dfr_n + 1, (u64)dqn[1]);
    ((u64 *)(dqn + 2))[0] = base;
  }
  __syncthreads();
  const u64 base = ((const u64 *)(dqn + 2))[0];
  if (threadIdx.x == 0) {
    dqn[0] = 0;
    dqn[1] = 0;
  }
  for (int x = threadIdx.x; x < n; x += blockDim.x) {
    const u64 slot = base + (u64)x;
    if ((long long)slot < A.dfr_cap) {
      A.dfr_key[slot] = ((const u64 *)(sb + O_DQK))[x];
      A.dfr_len[slot] = ((const unsigned *)(sb + O_DQL))[x];
    } else {
      set_err(A.err, 7);   // deferral buffer overflow
    }
  }
  __syncthreads();
}

// Exact path of one flagged tuple (tile_kernel's slow_tuple for these
// layouts): 1 when handled, 0 when the staging area was full (look again
// after the commit).
template <int DP>
__device__ __forceinline__ int slow32(const TileArgs<float> &A, const ItemCtx<float> &c,
                                      const Rec32 rb, CtaList<float> &L, int i, int jl, int kk,
                                      float cjk) {
  const int j = c.j0 + jl, k = c.k0 + kk;
  const float kpn = rb.kp()[kk];
  if (kpn == -r_inf<float>()) return 1;   // column past m or a duplicate of the prefix
  if (kpn == r_inf<float>()) {             // column near-singular after the prefix
    defer32<DP>(A, c, i, j, k, 1);
    return 1;
  }
  const float *rf = (const float *)(rb.row() + 2 * jl);   // -g, -g, 1/l, 1/l, z2, z2, e, e
  float h = cjk;
  if (DP == 1) h = __fmaf_rn(rf[0], rb.kg()[kk], h);
  const float g2 = __fmul_rn(h, rf[2]);
  const float pp = -__fmaf_rn(g2, g2, kpn);
  const float wn = __fmaf_rn(g2, rf[4], rb.kw()[kk]);
  if (!(pp >= 0.f)) {                       // pivot of k after (i, j) below the cut
    if (!same_class(c.cls, j, k)) defer32<DP>(A, c, i, j, k, 1);
    return 1;
  }
  const float p = pp + rb.kpt()[kk];
  const float rel = rb.jpP()[jl] - wn * wn / p;
  if (rel > cta_cut<float>(L)) return 1;
  if (A.band) {   // band pass: scored again in FP64
    defer32<DP>(A, c, i, j, k, 1);
    return 1;
  }
  int t[L0_DMAX];
  if (DP == 1) {
    t[0] = i;
    t[1] = j;
    t[2] = k;
  } else {
    t[0] = j;
    t[1] = k;
  }
  const u64 key = lex_rank(c.B, c.m, c.d, t, c.total);
  if (!cta_list_admits<float>(L, rel, key)) return 1;
  return cta_list_push<float>(L, rel, key) ? 1 : 0;
}

// The rare part of a step: some tuple of this thread was flagged.  Every
// tuple is tested again one by one (the same IEEE operations as the packed
// test, so the same decisions), C_jk re-read from the Gram; flagged tuples
// take the exact path, rows in the redo state queue their run once.  `done`
// has a bit per (u, q, b) already handled in this step (staged, queued or
// skipped); a pass after an overflow of the staging area skips them.
template <int DP, int UJ>
__device__ __noinline__ void recheck32(const TileArgs<float> &A, const ItemCtx<float> &c,
                                       const Rec32 rb, CtaList<float> &L, int i,
                                       unsigned *done_p) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  unsigned done = *done_p;
  // this thread's C_jk, all loads issued before any is used
  float cj[UJ * 4];
#pragma unroll
  for (int u = 0; u < UJ; ++u) {
    const int j = c.j0 + w * UJ + u;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int k = c.k0 + 2 * lane + (v & 1) + 64 * (v >> 1);
      cj[4 * u + v] = (j < c.m && k < c.m && k > j) ? c.G[(long long)(j + 1) * c.ld + k + 1] : 0.f;
    }
  }
#pragma unroll 1
  for (int u = 0; u < UJ; ++u) {
    const int jl = w * UJ + u;
    const int j = c.j0 + jl;
    const unsigned rowbits = 0xfu << (4 * u);
    if ((done & rowbits) == rowbits) continue;
    const int flag = rb.jflag()[jl];
    if (flag == 0) {
      done |= rowbits;
      continue;
    }
    if (flag == 3) {   // prefix or row singular in FP32: the row's run goes to the FP64 redo
      if (lane == 0) {
        const int kf = c.k0 > j + 1 ? c.k0 : j + 1;
        const int kl = c.k0 + TK < c.m ? c.k0 + TK : c.m;
        defer32<DP>(A, c, i, j, kf, kl - kf);
      }
      done |= rowbits;
      continue;
    }
    const float *rf = (const float *)(rb.row() + 2 * jl);
    const float jg = rf[0], invl = rf[2], z2 = rf[4], e = rf[6];
#pragma unroll 1
    for (int v = 0; v < 4; ++v) {
      const int q = v >> 1, b = v & 1;
      const unsigned bit = 1u << (4 * u + v);
      if (done & bit) continue;
      const int kk = 2 * lane + b + 64 * q;
      const int k = c.k0 + kk;
      if (k >= c.m || k <= j) {   // past m, or below the diagonal of the first k tile
        done |= bit;
        continue;
      }
      const float cjk = cj[4 * u + v];
      const float h = __fmaf_rn(jg, rb.kg()[kk], cjk);
      const float g2 = __fmul_rn(h, invl);
      const float ppn = __fmaf_rn(g2, g2, rb.kp()[kk]);
      const float wn = __fmaf_rn(g2, z2, rb.kw()[kk]);
      const float t = __fmaf_rn(e, ppn, __fmul_rn(wn, wn));
      if (__float_as_uint(t) >> 31) {   // not flagged
        done |= bit;
        continue;
      }
      if (slow32<DP>(A, c, rb, L, i, jl, kk, cjk)) done |= bit;
    }
  }
  *done_p = done;
}

// ------------------------------------------------------------ flagged tuples --
// A thread whose fast test flagged something appends its flagged tuples
// (step of the group, row, column, C_jk) to a queue in shared memory, inline
// in the hot loop; after the group's barrier the whole CTA takes the exact
// path of the queued tuples, one per thread.  So a tile whose tuples flag on
// every step (one holding two columns of the best descriptor) costs one
// queue append per flag, and no warp of the CTA waits on another's exact
// path.  A full queue sends the group to the per-thread exact path instead.
__device__ __forceinline__ u64 fq_pack(int q, int jl, int kk, float cjk) {
  return ((u64)__float_as_uint(cjk) << 32) | ((u64)q << 16) | ((u64)jl << 8) | (u64)kk;
}

// the thread's flagged tuples of step q of the group (the same IEEE
// operations as the packed test, so the same decisions); false if the queue
// was full
template <int UJ, bool DIAG>
__device__ __forceinline__ bool enqueue32(const u64 (&creg)[UJ][2], uint32_t rbs, int w, int lane,
                                          int q, unsigned char *sb) {
  bool ok = true;
  int *fqn = (int *)(sb + O_FQN);
#pragma unroll
  for (int u = 0; u < UJ; ++u) {
    const int jl = w * UJ + u;
    const uint32_t ra = rbs + R_ROW + (uint32_t)jl * 32u;
    const float jg = lds32(ra), invl = lds32(ra + 8u), z2 = lds32(ra + 16u), e = lds32(ra + 24u);
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int qq = v >> 1, b = v & 1;
      const int kk = 2 * lane + b + 64 * qq;
      if (DIAG && qq == 0 && kk < jl) continue;   // k <= j in the diagonal tile
      const u64 cw = creg[u][qq];
      const float cjk = __uint_as_float(b ? (unsigned)(cw >> 32) : (unsigned)cw);
      const float h = __fmaf_rn(jg, lds32(rbs + R_KG + 4u * kk), cjk);
      const float g2 = __fmul_rn(h, invl);
      const float ppn = __fmaf_rn(g2, g2, lds32(rbs + R_KP + 4u * kk));
      const float wn = __fmaf_rn(g2, z2, lds32(rbs + R_KW + 4u * kk));
      const float t = __fmaf_rn(e, ppn, __fmul_rn(wn, wn));
      if (__float_as_uint(t) >> 31) continue;   // not flagged
      const int slot = atomicAdd(fqn, 1);
      if (slot < T32_FQ) ((u64 *)(sb + O_FQ))[slot] = fq_pack(q, jl, kk, cjk);
      else ok = false;
    }
  }
  return ok;
}

// exact path of one queued tuple: 1 handled, 0 staging area full (again
// after the commit)
template <int DP>
__device__ __forceinline__ int exact32(const TileArgs<float> &A, const ItemCtx<float> &c,
                                       unsigned char *sb, CtaList<float> &L, int g, int i0,
                                       u64 ent) {
  const int q = (int)((ent >> 16) & 0xffu), jl = (int)((ent >> 8) & 0xffu), kk = (int)(ent & 0xffu);
  const float cjk = __uint_as_float((unsigned)(ent >> 32));
  const Rec32 rb{sb + ((g & 1) * T32_G + q) * T32_REC_BYTES};
  const int i = i0 + g * T32_G + q;
  const int j = c.j0 + jl, k = c.k0 + kk;
  if (k >= c.m || k <= j) return 1;
  const int flag = rb.jflag()[jl];
  if (flag == 0) return 1;
  if (flag == 3) {   // prefix or row singular in FP32: the row's run, once (its first column)
    const int kf = c.k0 > j + 1 ? c.k0 : j + 1;
    if (k == kf) {
      const int kl = c.k0 + TK < c.m ? c.k0 + TK : c.m;
      defer32<DP>(A, c, i, j, kf, kl - kf);
    }
    return 1;
  }
  return slow32<DP>(A, c, rb, L, i, jl, kk, cjk);
}

// the whole CTA, after the group's barrier, nq > 0 queued (all threads read
// nq before this call): empty the counters, then rounds of exact paths until
// none is left waiting for room in the staging area
template <int DP>
__device__ __noinline__ void drain32(const TileArgs<float> &A, const ItemCtx<float> &c,
                                     unsigned char *sb, CtaList<float> &L, u64 *gthr, int g,
                                     int i0, int nq) {
  unsigned char *st = sb + O_FQS;
  const u64 *fq = (const u64 *)(sb + O_FQ);
  for (int x = threadIdx.x; x < nq; x += blockDim.x) st[x] = 0;
  __syncthreads();   // every thread has read nq; the counters can be emptied
  if (threadIdx.x == 0) ((int *)(sb + O_FQN))[0] = 0;
  for (int round = 0;; ++round) {
    for (int x = threadIdx.x; x < nq; x += blockDim.x)
      if (!st[x] && exact32<DP>(A, c, sb, L, g, i0, fq[x])) st[x] = 1;
    __syncthreads();
    const bool ovf = *(volatile int *)L.ovf != 0;
    if (ovf || *(volatile int *)L.n_stage > L.S / 2) cta_list_commit<float>(L, gthr);
    if (!ovf) break;
    if (round > L0_MAX_REDO) {
      set_err(A.err, 8);
      break;
    }
  }
}

// TMA copy of the two row segments step s of the item needs (one thread,
// after a fence.proxy.async that orders the block's earlier reads of the
// stage).  Copy lengths are clamped to the problem's Gram so no read leaves
// it; the entries a record reads (columns <= m of row i + 1) lie inside.
__device__ __forceinline__ void issue32(const ItemCtx<float> &c, unsigned char *sb, int i,
                                        unsigned copy_idx) {
  const int slot = (int)(copy_idx % T32_NS);
  const long long end = (long long)(c.m + 1) * c.ld;   // floats of this problem's Gram
  const long long js = (long long)(i + 1) * c.ld + c.j0;
  const long long ks = (long long)(i + 1) * c.ld + (c.k0 - 1);
  const long long jn = min((long long)T32_JSEG, end - js);
  const long long kn = min((long long)T32_KSEG, end - ks);
  const uint32_t bar = tc::smem_u32(sb + O_BAR + 8 * slot);
  const uint32_t dst = tc::smem_u32(sb + O_STAGE + slot * T32_SEG * 4);
  tc::mbar_expect_tx(bar, (uint32_t)((jn + kn) * 4));
  tc::bulk_load(dst, c.G + js, (uint32_t)(jn * 4), bar);
  tc::bulk_load(dst + T32_JSEG * 4, c.G + ks, (uint32_t)(kn * 4), bar);
}

// Records of group g (steps g G .. g G + G - 1 < nsteps) into the group's
// buffers: all threads, records spread round-robin; each waits for the ring
// stage of the step it builds.  `cons` = ring copies consumed before this item.
template <int DP>
__device__ __forceinline__ void build_group32(const TileArgs<float> &A, const Item32 &it,
                                              unsigned char *sb, int g, int nsteps, int i0,
                                              unsigned cons, float cut) {
  const float *pdg = (const float *)(sb + O_PDG), *pry = (const float *)(sb + O_PRY);
  const float *ppb = (const float *)(sb + O_PPB);
  const int *pcls = (const int *)(sb + O_PCLS);
  const int s0 = g * T32_G;
  const int ns = min(T32_G, nsteps - s0);
  for (int x = threadIdx.x; x < ns * T32_NREC; x += blockDim.x) {
    const int q = x / T32_NREC, r = x - q * T32_NREC;
    const int s = s0 + q;
    const unsigned copy = cons + (unsigned)s;
    const float *seg = nullptr;
    if (DP == 1) {
      tc::mbar_wait(tc::smem_u32(sb + O_BAR + 8 * (copy % T32_NS)), (copy / T32_NS) & 1u, A.err);
      seg = (const float *)(sb + O_STAGE) + (copy % T32_NS) * T32_SEG;
    }
    const Rec32 rb{sb + ((g & 1) * T32_G + q) * T32_REC_BYTES};
    build32<DP>(it, sb, r, i0 + s, DP == 1 ? pdg[s] : 0.f, DP == 1 ? pry[s] : 0.f,
                DP == 1 ? ppb[s] : 0.f, DP == 1 ? pcls[s] : -1, seg, rb, cut);
  }
}

// one thread: the ring copies of group g's steps
__device__ __forceinline__ void issue_group32(const ItemCtx<float> &c, unsigned char *sb, int g,
                                              int nsteps, int i0, unsigned cons) {
  if (g * T32_G >= nsteps) return;
  tc::fence_proxy_async_smem();
  for (int s = g * T32_G; s < nsteps && s < (g + 1) * T32_G; ++s)
    issue32(c, sb, i0 + s, cons + (unsigned)s);
}

// One work item: the (j, k) tile against prefixes [r0, r1) (DP = 1) or the
// single prefix-free step (DP = 0).  `cons` counts the ring copies this CTA
// has consumed (the ring slot and mbarrier parity of every copy follow).
// Group g's records are built while group g - 1 is tested; group g + 2's
// rows are copied into the stages group g's used, after the barrier.
template <int DP, int UJ>
__device__ __forceinline__ void run32(const TileArgs<float> &A, const ProbDesc &pd, int prob, int bj, int bk,
                      u64 r0, u64 r1, CtaList<float> &L, unsigned char *sb, u64 *gthr,
                      unsigned &cons) {
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  Item32 it;
  ItemCtx<float> &c = it.c;
  c.G = A.G + pd.g_off;
  c.ld = pd.ld;
  c.prob = prob;
  c.m = pd.m;
  c.d = pd.d;
  c.j0 = bj * TJ;
  c.k0 = tile_k0(bj, bk);
  c.diag = bk == 0;   // only the first k tile of a row block reaches k <= j
  c.total = pd.total;
  c.B = A.B;
  c.ratio = (float)A.ratio;
  c.cls = A.cls;
  c.smem_dq = tc::smem_u32(sb);
  const float *G = c.G;
  const long long ld = c.ld;
  const int nsteps = DP == 1 ? (int)(r1 - r0) : 1;
  const int i0 = DP == 1 ? (int)r0 : 0;   // colex rank of a one-index prefix is the index
  if (nsteps > T32_MAXL || nsteps > (int)blockDim.x) {   // the plan never makes such items
    set_err(A.err, 9);
    return;
  }
  const int ngroups = (nsteps + T32_G - 1) / T32_G;
  const bool issuer = tid == (int)blockDim.x - 32;   // lane 0 of the last warp: the ring copies
  if (DP == 1 && issuer) {
    issue_group32(c, sb, 0, nsteps, i0, cons);
    issue_group32(c, sb, 1, nsteps, i0, cons);
  }
  // Set-up of the item: every load is issued before the first shared store
  // (a store through a generic pointer may not be moved above a later global
  // load), so the item waits for one round trip to L2, not three.  Thread s
  // takes prefix step s (nsteps <= blockDim) and record s (T32_NREC <= blockDim).
  // the tile's Gram entries: rows j0 + w UJ + u, columns k0 + 2 lane + {0, 1} + 64 q
  u64 creg[UJ][2];
#pragma unroll
  for (int u = 0; u < UJ; ++u) {
    const int j = c.j0 + w * UJ + u;
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int k = c.k0 + 2 * lane + 64 * q;
      u64 v = 0ull;
      if (j < c.m && k < c.m) {
        v = __ldg((const unsigned long long *)(G + (long long)(j + 1) * ld + k + 1));
        if (k + 1 >= c.m) v &= 0xffffffffull;   // the pair's second column is past m
      }
      creg[u][q] = v;
    }
  }
  it.G00 = __ldg(G);
  float p_cii = 1.f, p_ry = 0.f;
  int p_cls = -1;
  if (DP == 1 && tid < nsteps) {
    const int i = i0 + tid;
    p_cii = __ldg(G + (long long)(i + 1) * (ld + 1));
    p_ry = __ldg(G + i + 1);
    if (c.cls) p_cls = __ldg(c.cls + i);
  }
  const int rcol = tid < TJ ? c.j0 + tid : c.k0 + tid - TJ;
  float r_dg = 0.f, r_cy = 0.f;
  int r_cc = -2;
  if (tid < T32_NREC && rcol < c.m) {
    r_dg = __ldg(G + (long long)(rcol + 1) * (ld + 1));
    r_cy = __ldg(G + rcol + 1);
    if (c.cls) r_cc = __ldg(c.cls + rcol);
  }
  if (tid == 0) {   // the queues start empty (the previous item emptied them)
    ((int *)(sb + O_DQN))[0] = 0;
    ((int *)(sb + O_DQN))[1] = 0;
    ((int *)(sb + O_FQN))[0] = 0;
    ((int *)(sb + O_FQN))[1] = 0;
  }
  if (DP == 1 && tid < nsteps) {
    // the prefix's own factor, shared by the step's records: 1/l_i (its
    // sign marks C_ii <= 0), z_i = r_i / l_i, pP_i = 1 - z_i^2
    const bool pok = p_cii > 0.f;
    const float invd = rsqrtf(pok ? p_cii : 1.f);
    const float zP = p_ry * invd;
    ((float *)(sb + O_PDG))[tid] = pok ? invd : -invd;
    ((float *)(sb + O_PRY))[tid] = zP;
    ((float *)(sb + O_PPB))[tid] = it.G00 - zP * zP;
    ((int *)(sb + O_PCLS))[tid] = p_cls;
  }
  if (tid < T32_NREC) {
    ((int *)(sb + O_RCOL))[tid] = rcol;
    ((float *)(sb + O_RDG))[tid] = r_dg;
    ((float *)(sb + O_RY))[tid] = r_cy;
    ((int *)(sb + O_RCLS))[tid] = r_cc;
  }
  __syncthreads();   // prefix scalars and record constants visible
  build_group32<DP>(A, it, sb, 0, nsteps, i0, cons, cta_cut<float>(L));
  __syncthreads();
  if (DP == 1 && issuer) issue_group32(c, sb, 2, nsteps, i0, cons);
  u64 gnext = ~0ull;   // warp 0: the global bound, read a group before it is used
  HistPipe hp{0, 0, 0u};
  const uint32_t sbs = tc::smem_u32(sb);
  const int d0b = 2 * lane - w * UJ;   // diagonal tile: 2 lane - jl = d0b - u
  for (int g = 0; g < ngroups; ++g) {
    const u64 gprev = gnext;
    if (tid < 32) gnext = ld_relaxed(gthr);
    if (g + 1 < ngroups) build_group32<DP>(A, it, sb, g + 1, nsteps, i0, cons, cta_cut<float>(L));
    const int ns = min(T32_G, nsteps - g * T32_G);
    unsigned done[T32_G];
#pragma unroll
    for (int q = 0; q < T32_G; ++q) done[q] = 0u;
    const uint32_t gb = sbs + (uint32_t)((g & 1) * (T32_G * T32_REC_BYTES));
    const uint32_t rw = gb + R_ROW + (uint32_t)(w * UJ * 32), rl = gb + R_KG + 8u * lane;
    unsigned acc[T32_G];
    if (ns == T32_G) {   // a full group: the tests straight through, one check
#pragma unroll
      for (int q = 0; q < T32_G; ++q)
        acc[q] = c.diag ? fast32<UJ, true>(creg, rw + q * T32_REC_BYTES, rl + q * T32_REC_BYTES, d0b)
                        : fast32<UJ, false>(creg, rw + q * T32_REC_BYTES, rl + q * T32_REC_BYTES, d0b);
    } else {
#pragma unroll
      for (int q = 0; q < T32_G; ++q)
        acc[q] = q >= ns ? 0xffffffffu
                 : c.diag ? fast32<UJ, true>(creg, rw + q * T32_REC_BYTES, rl + q * T32_REC_BYTES, d0b)
                          : fast32<UJ, false>(creg, rw + q * T32_REC_BYTES, rl + q * T32_REC_BYTES, d0b);
    }
    unsigned all = 0xffffffffu;
#pragma unroll
    for (int q = 0; q < T32_G; ++q) all &= acc[q];
    if (!(all >> 31)) {   // something of this thread flagged: queue it
      bool qok = true;
#pragma unroll
      for (int q = 0; q < T32_G; ++q)
        if (q < ns && !(acc[q] >> 31)) {
          const uint32_t rbs = gb + (uint32_t)(q * T32_REC_BYTES);
          qok = (c.diag ? enqueue32<UJ, true>(creg, rbs, w, lane, q, sb)
                        : enqueue32<UJ, false>(creg, rbs, w, lane, q, sb)) && qok;
        }
      if (!qok) ((volatile int *)(sb + O_FQN))[1] = 1;
    }
    __syncthreads();
    const int nq = *(volatile int *)(sb + O_FQN), qovf = ((volatile int *)(sb + O_FQN))[1];
    if (qovf) {
      // the queue overflowed: the group's flagged tuples take the exact path
      // thread by thread (the queued entries are dropped)
      __syncthreads();
      if (tid == 0) {
        ((int *)(sb + O_FQN))[0] = 0;
        ((int *)(sb + O_FQN))[1] = 0;
      }
      for (int pass = 0;; ++pass) {
        if (!(all >> 31)) {
#pragma unroll
          for (int q = 0; q < T32_G; ++q)
            if (q < ns && !(acc[q] >> 31))
              recheck32<DP, UJ>(A, c, Rec32{sb + ((g & 1) * T32_G + q) * T32_REC_BYTES}, L,
                                i0 + g * T32_G + q, &done[q]);
        }
        __syncthreads();
        const bool ovf = *(volatile int *)L.ovf != 0;
        if (ovf || *(volatile int *)L.n_stage > L.S / 2) cta_list_commit<float>(L, gthr);
        if (!ovf) break;
        if (pass > L0_MAX_REDO) {
          set_err(A.err, 8);
          break;
        }
      }
    } else if (nq > 0) {
      drain32<DP>(A, c, sb, L, gthr, g, i0, nq);
    }
    {
      const int nq = *(volatile int *)(sb + O_DQN);   // read after the barrier: uniform
      if (nq > 0) flush32(A, sb, nq);
    }
    // the stages that held group g + 1's rows are free after the barrier above
    if (DP == 1 && issuer) issue_group32(c, sb, g + 3, nsteps, i0, cons);
    step_sync32(L, gthr, gprev, hp, sb);
  }
  if (tid < 32) cp_async_wait_all();   // no copy into the histogram buffers outlives the item
  if (DP == 1) cons += (unsigned)nsteps;
}

template <int DPLO, int DPHI, int UJ, int MINB>
__global__ void __launch_bounds__(TJ / UJ * 32, MINB)
tile32_kernel(TileArgs<float> A) {
  bool ready = false;   // ring mbarriers initialised (first item)
  unsigned cons = 0u;
  persistent_items<float>(A, [&](const ProbDesc &pd, int prob, int bj, int bk, u64 r0, u64 r1,
                                 CtaList<float> &L, unsigned char *recbase, u64 *gthr) {
    if (!ready) {
      if (threadIdx.x == 0) {
        for (int s = 0; s < T32_NS; ++s) tc::mbar_init(tc::smem_u32(recbase + O_BAR + 8 * s), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
      }
      __syncthreads();
      ready = true;
    }
    if (pd.dp == 0) {
      if (DPLO == 0) run32<0, UJ>(A, pd, prob, bj, bk, r0, r1, L, recbase, gthr, cons);
    } else if (pd.dp == 1) {
      if (DPHI >= 1) run32<1, UJ>(A, pd, prob, bj, bk, r0, r1, L, recbase, gthr, cons);
    }
  }, /*forward=*/true);
}

}  // namespace

// shape 1: 8 rows per warp, 256 threads, one CTA per SM; shape 2: the same
// with two CTAs per SM (at most 128 registers); shape 3: 4 rows per warp,
// 512 threads, one CTA per SM
static const void *tile32_fn(int variant, int dp_lo, int dp_hi) {
#define L0_T32(V, UJ, MB)                                                            \
  if (variant == V) {                                                               \
    if (dp_lo == 0 && dp_hi == 0) return (const void *)tile32_kernel<0, 0, UJ, MB>; \
    if (dp_lo == 1 && dp_hi == 1) return (const void *)tile32_kernel<1, 1, UJ, MB>; \
    if (dp_lo == 0 && dp_hi == 1) return (const void *)tile32_kernel<0, 1, UJ, MB>; \
  }
  L0_T32(1, 8, 1)
  L0_T32(2, 8, 2)
  L0_T32(3, 4, 1)
#undef L0_T32
  return nullptr;
}

int tile32_threads(int variant) { return variant == 3 ? 512 : 256; }

size_t tile32_smem_bytes(int K, int S) {
  return align16(cta_list_bytes<float>(K, S)) + 16 + T32_EXTRA_BYTES;
}

bool tile32_supports(int variant, int dp_lo, int dp_hi) {
  return tile32_fn(variant, dp_lo, dp_hi) != nullptr;
}

cudaError_t tile32_occupancy(int variant, int dp_lo, int dp_hi, size_t smem, int *blocks_per_sm) {
  const void *fn = tile32_fn(variant, dp_lo, dp_hi);
  if (!fn) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, fn, tile32_threads(variant),
                                                       smem);
}

cudaError_t launch_tile32(const TileArgs<float> &a, int variant, int dp_lo, int dp_hi, int grid,
                          size_t smem, cudaStream_t st) {
  const void *fn = tile32_fn(variant, dp_lo, dp_hi);
  if (!fn) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  void *args[] = {(void *)&a};
  return cudaLaunchKernel(fn, dim3(grid), dim3(tile32_threads(variant)), args, smem, st);
}

}  // namespace l0
