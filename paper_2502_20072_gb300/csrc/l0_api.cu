// l0_api.cu -- host orchestrator behind the C ABI of include/sisso_l0.h.
//
// One fit (paper Sec. 2.4, all n-tuples of the m SIS features):
//   1. centre and scale every column and the target per task (FP64)
//   2. augmented Gram per task (FP64 FFMA, or split-BF16 tensor cores)
//   3. persistent tuple kernel -> per-CTA top-K' lists
//   4. grid merge -> one top-K' pool per output list
//   5. FP64 Householder re-fit of the pool from the raw centred columns
//   6. final ranking; certificate (an empirical check, see select_kernel):
//      the outside tuples' search scores must clear the k-th re-fitted score
//      by four times the largest search-score error measured on the pool,
//      otherwise K' is doubled and steps 3-6 rerun.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <functional>
#include <map>
#include <new>
#include <string>
#include <thread>
#include <type_traits>
#include <vector>

#include "../../include/sisso_l0.h"
#include "l0_kernels.cuh"
#include "l0_screen.cuh"

using l0::u64;

namespace {

// Test hook (sisso_l0_debug_fail_allocation): when >= 0, the number of
// device allocations this thread still makes before one reports
// cudaErrorMemoryAllocation without calling cudaMalloc.
thread_local long long g_alloc_fail_countdown = -1;

struct DevBuf {
  void *p = nullptr;
  size_t n = 0;
  cudaError_t ensure(size_t bytes) {
    if (bytes <= n && p) return cudaSuccess;
    if (p) cudaFree(p);
    p = nullptr;
    n = 0;
    if (g_alloc_fail_countdown >= 0 && g_alloc_fail_countdown-- == 0)
      return cudaErrorMemoryAllocation;
    size_t want = std::max<size_t>(bytes, 256);
    cudaError_t e = cudaMalloc(&p, want);
    if (e != cudaSuccess) {
      p = nullptr;
      return e;
    }
    n = want;
    return cudaSuccess;
  }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    n = 0;
  }
  template <typename T> T *as() const { return (T *)p; }
};

struct Status {
  int code = SISSO_L0_OK;
  std::string msg;
};

}  // namespace

struct sisso_l0_handle {
  sisso_l0_options opt;
  cudaStream_t st = nullptr;        // stream the library's work is ordered on
  cudaStream_t user_st = nullptr;   // the caller's stream (options.stream)
  bool own_st = false;              // st created by the handle (graph capture
                                    // cannot use the legacy stream)
  int n_sm = 0;
  std::string last_error;
  sisso_l0_stats stats;
  // workspace
  DevBuf xin, yin, offs, mu, inv_s, w64, gram, binom;
  DevBuf probs, rowpre, ctr, gthr, hist, lists_s, lists_k, lists_cnt;
  DevBuf part_s, part_k, part_cnt, done, pool_s, pool_k, pool_cnt;
  DevBuf scratch, refit, rdiv, cert, out_t, out_r, err;
  DevBuf dfr_key, dfr_len, dfr_n, dfr_cnt;
  DevBuf abf, bbf, kmeta, gram32;
  DevBuf gpart, gctr;                                 // split-K partial Gram tiles, tile counters
  DevBuf prop_in, prop_pairs, prop_bits, prop_ctr, sel_hist, sel_bin, scores, diag;
  DevBuf col_hash, col_cls;
  DevBuf band_thr, band_floor;                        // band pass: cut, previous delta
  DevBuf g64_have;                                    // the fit's FP64 Gram exists (mixed)
  DevBuf dfr_bctr;                                    // FP64 redo: run batches handed out
  DevBuf sis_ex, sis_y;                               // screening: exclusions, targets
  DevBuf gen_ops, gen_c1, gen_c2, gen_valid;          // generated candidates
  DevBuf gen_cf, gen_csafe;                           // their FP32 children (pre-screen)
  DevBuf loop_x, loop_y, loop_xs, loop_res, loop_q, loop_tup, loop_rows;   // dimension loop
  int binom_m = -1;
  int done_init_for = 0;
  cudaEvent_t ev[8] = {nullptr};
  cudaEvent_t ev_user = nullptr;    // orders the handle's stream after the caller's
  cudaEvent_t ev_k[2] = {nullptr, nullptr};   // around the tuple kernel
  float ms_tuple_kernel = 0.f;
  cudaGraphExec_t graph_exec = nullptr;
  std::string graph_key;
  struct Tune { int f, b, v; };                      // items factor, CTAs per SM, kernel shape
  std::map<std::string, int> bps_cache;              // resident tuple-kernel CTAs per SM
  std::string dev_name;                              // device name (tuning keys)
  std::map<std::string, Tune> tune;                   // autotuner choices
  std::string fp64_key;   // inputs whose last mixed-precision fit needed FP64
  // pinned host staging for the small per-call uploads and status reads (so
  // they are asynchronous), handed out from the start at every call; ev_pin
  // follows the last copy that read it
  unsigned char *pin = nullptr;
  size_t pin_n = 0, pin_used = 0;
  cudaEvent_t ev_pin = nullptr;
  // side stream: the duplicate-class kernels run beside the centring and
  // the Gram (they read only X), forked and joined by events
  cudaStream_t st2 = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  bool pin_pending = false;
  // last bytes uploaded to a small device table; an identical upload is skipped
  struct UpCache {
    const void *dev = nullptr;
    std::vector<unsigned char> bytes;
  };
  UpCache up_probs, up_rowpre, up_rdiv, up_offs, up_kmeta;
};

namespace {

const char *kNullHandleMsg = "null handle";

int fail(sisso_l0_t h, int code, const std::string &m) {
  if (h) h->last_error = m;
  return code;
}

int cuda_fail(sisso_l0_t h, cudaError_t e, const char *where) {
  std::string m = std::string(where) + ": " + cudaGetErrorString(e);
  return fail(h, (e == cudaErrorMemoryAllocation) ? SISSO_L0_ENOMEM : SISSO_L0_ECUDA, m);
}

#define L0_CK(call, where)                           \
  do {                                               \
    cudaError_t e_ = (call);                         \
    if (e_ != cudaSuccess) return cuda_fail(h, e_, where); \
  } while (0)

const u64 kSat = 1ull << 62;

u64 binom_host(long long x, int p) {
  if (p < 0 || x < p) return 0;
  if (p == 0) return 1;
  // multiplicative with saturation
  unsigned __int128 r = 1;
  for (int i = 1; i <= p; ++i) {
    r = r * (unsigned __int128)(x - p + i) / (unsigned __int128)i;
    if (r >= kSat) return kSat;
  }
  return (u64)r;
}

bool is_device_ptr(const void *p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Wait for the handle's stream with the host-side deadline.  The first 2 ms
// are polled without sleeping (a fit's tail is a few short kernels, and a
// sleep would add its whole granularity to every call); after that the
// host sleeps 20 us between polls.
int wait_stream(sisso_l0_t h) {
  cudaEvent_t e = h->ev[7];
  L0_CK(cudaEventRecord(e, h->st), "event record");
  const double tmo = h->opt.timeout_seconds;
  auto t0 = std::chrono::steady_clock::now();
  for (;;) {
    cudaError_t q = cudaEventQuery(e);
    if (q == cudaSuccess) break;
    if (q != cudaErrorNotReady) return cuda_fail(h, q, "stream");
    const double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (tmo > 0 && el > tmo)
      return fail(h, SISSO_L0_ETIMEOUT, "stream did not finish within timeout_seconds");
    if (el > 2e-3) std::this_thread::sleep_for(std::chrono::microseconds(20));
    else std::this_thread::yield();
  }
  h->pin_pending = false;   // every copy from the staging buffer has completed
  return SISSO_L0_OK;
}

// Pinned staging: start handing out the buffer from its beginning (after the
// copies that last read it, if the previous call returned before its wait).
int pin_reset(sisso_l0_t h) {
  if (h->pin_pending && h->ev_pin) L0_CK(cudaEventSynchronize(h->ev_pin), "staging event");
  h->pin_pending = false;
  h->pin_used = 0;
  if (!h->pin) {
    const size_t n = 256 * 1024;
    if (cudaHostAlloc((void **)&h->pin, n, cudaHostAllocDefault) != cudaSuccess) {
      (void)cudaGetLastError();
      h->pin = nullptr;   // without it, copies go through pageable memory
      return SISSO_L0_OK;
    }
    h->pin_n = n;
  }
  return SISSO_L0_OK;
}

unsigned char *pin_take(sisso_l0_t h, size_t n) {
  const size_t a = (h->pin_used + 15) & ~(size_t)15;
  if (!h->pin || a + n > h->pin_n) return nullptr;
  h->pin_used = a + n;
  return h->pin + a;
}

// Host -> device copy of a small table, skipped when the device buffer
// already holds exactly these bytes from the previous upload through `c`.
int upload(sisso_l0_t h, void *dev, const void *src, size_t n, sisso_l0_handle::UpCache *c) {
  if (n == 0) return SISSO_L0_OK;
  if (c && c->dev == dev && c->bytes.size() == n && memcmp(c->bytes.data(), src, n) == 0)
    return SISSO_L0_OK;
  unsigned char *stg = pin_take(h, n);
  if (stg) {
    memcpy(stg, src, n);
    L0_CK(cudaMemcpyAsync(dev, stg, n, cudaMemcpyHostToDevice, h->st), "upload");
    L0_CK(cudaEventRecord(h->ev_pin, h->st), "staging event");
    h->pin_pending = true;
  } else {
    L0_CK(cudaMemcpyAsync(dev, src, n, cudaMemcpyHostToDevice, h->st), "upload");
  }
  if (c) {
    c->dev = dev;
    c->bytes.assign((const unsigned char *)src, (const unsigned char *)src + n);
  }
  return SISSO_L0_OK;
}

int ensure_binom(sisso_l0_t h, int m) {
  if (h->binom_m == m) return SISSO_L0_OK;
  const int stride = m + 1;
  std::vector<u64> t((size_t)(L0_DMAX + 1) * stride);
  for (int p = 0; p <= L0_DMAX; ++p)
    for (int x = 0; x <= m; ++x) t[(size_t)p * stride + x] = binom_host(x, p);
  L0_CK(h->binom.ensure(t.size() * 8), "alloc binom");
  L0_CK(cudaMemcpy(h->binom.p, t.data(), t.size() * 8, cudaMemcpyHostToDevice), "copy binom");
  h->binom_m = m;
  return SISSO_L0_OK;
}

struct Req {
  int d, k;
  int32_t *out_t;
  double *out_r;
};

struct FitPlan {
  int T = 0, m = 0, n_out = 0, shared = 0, mixed = 0;
  int dmax = 0, dp_lo = -1, dp_hi = -1;    // tuple sizes; dp range of the d >= 2 requests
  bool has_singles = false, has_tuples = false;
  const double *Xd = nullptr, *yd = nullptr;   // device copies of the inputs
  long long N = 0, nmax = 0, ld = 0, gstride = 0, ldk = 0;
  int gsplit = 1;           // K splits of the tensor-core Gram
  std::vector<long long> off;
  std::vector<Req> req;
  std::vector<l0::ProbDesc> pd;
  std::vector<long long> rowpre;
  int grid = 0;             // tuple-kernel CTAs
  int max_bps = 1;          // largest resident CTAs per SM the kernel allows
  int items_factor = 2;     // work items per tuple-kernel CTA (at least)
  int variant = 0;          // tuple kernel shape (sisso_l0_options::tuple_kernel values)
  int kmax_pool = 2048;     // largest candidate pool of the fit (shared-memory sizing)
  // FP32 band pass (mixed precision): the search reruns with the cut fixed at
  // the previous pass's k-th re-fitted score + kBandMargin * delta and queues
  // every tuple below it for the FP64 redo
  int band = 0;
  long long n_items = 0;
  long long out_t_total = 0, out_r_total = 0;
  bool have_g64 = false;    // FP64 Gram computed (always in FP64 mode)
  unsigned long long fallback_tuples = 0;
  u64 fits_per_pass = 0;    // (task, tuple) fits of one search pass
  // learned forms (d = 3, one task): the search runs over the triples of a
  // pair list (proposal); or the call stops after the Gram (prep_only).
  // after_prep runs once the symmetric Gram and its diagonal exist.
  int proposal = 0, prep_only = 0;
  int shard = 0, n_shards = 1;   // the tuple kernel takes items shard, shard + n_shards, ...
  int exports_pool = 0;          // every pool entry is re-fitted (the caller reads them all)
  long long n_pairs = 0;
  u64 prop_fits = 0;
  std::function<int(sisso_l0_t, FitPlan &)> after_prep;
};

constexpr int kDeferGroups = 148;   // FP64 redo CTAs (and candidate lists) per problem
constexpr double kBandMargin = 8.0;   // band cut = k-th re-fitted score + 8 delta
constexpr long long kDeferCap = 1LL << 24;

int staging_for(int K) {
  int S = 1024;
  while (S < 2 * K) S <<= 1;
  return S;
}

// problem descriptors: one per (request, task) -- or per request in SHARED
// mode -- and their work items (prefix steps per item chosen so that there
// are at least items_factor items per CTA)
void plan_problems(FitPlan &P) {
  const int TJ = l0::TILE_TJ, TK = l0::TILE_TK;
  const int n_jt = (P.m + TJ - 1) / TJ;
  const int n_kt = (P.m + TK - 1) / TK;
  P.pd.clear();
  long long ot = 0, orr = 0;
  for (const Req &r : P.req) {
    for (int t = 0; t < (P.shared ? 1 : P.T); ++t) {
      l0::ProbDesc d{};
      d.g_off = (long long)t * P.gstride;
      d.ld = P.ld;
      d.m = P.m;
      d.d = r.d;
      d.dp = r.d - 2;
      d.task = t;
      d.total = binom_host(P.m, r.d);
      d.k = r.k;
      d.out_t_off = ot;
      d.out_r_off = orr;
      ot += (long long)r.k * r.d;
      orr += r.k;
      P.pd.push_back(d);
    }
  }
  P.out_t_total = ot;
  P.out_r_total = orr;
  auto np_of = [&](int bj, int dp) -> u64 {
    int jend = std::min((bj + 1) * TJ, P.m);
    return binom_host(jend - 1, dp);
  };
  // one prefix-chunk length for all problems
  int Lsel = 1;
  if (P.dp_hi > 0) {
    const int cands[] = {256, 128, 64, 32, 16, 8, 4, 2, 1};
    for (int L : cands) {
      long long items = 0;
      for (const l0::ProbDesc &d : P.pd) {
        if (d.d < 2) continue;
        for (int bj = 0; bj < n_jt; ++bj)
          items += l0::tile_row_items(bj, P.m, d.dp, L, n_kt, np_of(bj, d.dp));
      }
      Lsel = L;
      if (items >= (long long)P.items_factor * std::max(1, P.grid)) break;
    }
  }
  // per row block, l0::ROWINFO words: cumulative items before it, then the
  // chunking of a tile's prefixes (chunks, chunk size, chunks one larger) so
  // the kernels decode an item without 64-bit divisions
  long long item = 0;
  P.rowpre.clear();
  for (l0::ProbDesc &d : P.pd) {
    d.n_jt = n_jt;
    d.n_kt = n_kt;
    d.L = Lsel;
    d.prefix_off = (int)(P.rowpre.size() / l0::ROWINFO);
    d.item_begin = item;
    long long acc = 0;
    for (int bj = 0; bj <= n_jt; ++bj) {
      long long nch = 0, q = 0, rr = 0;
      if (d.d >= 2 && bj < n_jt) {
        const u64 np = np_of(bj, d.dp);
        nch = (long long)((np + (u64)Lsel - 1) / (u64)Lsel);
        if (nch > 0) {
          q = (long long)(np / (u64)nch);
          rr = (long long)(np % (u64)nch);
        }
      }
      P.rowpre.push_back(acc);
      P.rowpre.push_back(nch);
      P.rowpre.push_back(q);
      P.rowpre.push_back(rr);
      if (d.d >= 2 && bj < n_jt) acc += l0::tile_row_items(bj, P.m, d.dp, Lsel, n_kt, np_of(bj, d.dp));
    }
    item += acc;
    d.item_end = item;
  }
  P.n_items = item;
}

// the d <= 3 FP32 kernel runs PER_TASK exhaustive searches over a Gram whose
// rows the TMA unit can copy (16-byte aligned leading dimension and stride)
bool tile32_ok(const FitPlan &P, int v) {
  return v > 0 && P.mixed && !P.shared && !P.proposal && P.dp_lo >= 0 && P.dp_hi <= 1 &&
         P.ld % 4 == 0 && P.gstride % 4 == 0 && l0::tile32_supports(v, P.dp_lo, P.dp_hi);
}

template <typename R>
int tile_bps(sisso_l0_t h, const FitPlan &P, int Kmax, int *bps) {
  // the driver's occupancy answer is fixed per kernel and shared memory:
  // asked once per handle, not on every fit
  char key[96];
  snprintf(key, sizeof(key), "%d|%d|%d|%d|%d|%d|%zu", P.variant, P.dp_lo, P.dp_hi, P.shared,
           Kmax, (int)sizeof(R), sizeof(l0::ProbDesc));
  auto it = h->bps_cache.find(key);
  if (it != h->bps_cache.end()) {
    *bps = it->second;
    return SISSO_L0_OK;
  }
  const int S0 = staging_for(Kmax);
  if (P.variant > 0) {
    L0_CK(l0::tile32_occupancy(P.variant, std::max(P.dp_lo, 0), std::max(P.dp_hi, 0),
                               l0::tile32_smem_bytes(Kmax, S0), bps),
          "occupancy");
  } else {
    const size_t smem = l0::tile_smem_bytes<R>(Kmax, S0, std::max(P.dp_hi, 0));
    if (P.shared) L0_CK(l0::shared_occupancy<R>(std::max(P.dp_hi, 0), smem, bps), "occupancy");
    else L0_CK(l0::tile_occupancy<R>(std::max(P.dp_lo, 0), std::max(P.dp_hi, 0), smem, bps), "occupancy");
  }
  h->bps_cache[key] = *bps;
  return SISSO_L0_OK;
}

// upload the problem table, row prefixes, divisors; size the search buffers
template <typename R>
int setup_search(sisso_l0_t h, FitPlan &P, int K) {
  cudaStream_t st = h->st;
  const int n_probs = (int)P.pd.size();
  L0_CK(h->probs.ensure(P.pd.size() * sizeof(l0::ProbDesc)), "alloc probs");
  int urc = upload(h, h->probs.p, P.pd.data(), P.pd.size() * sizeof(l0::ProbDesc), &h->up_probs);
  if (urc) return urc;
  L0_CK(h->rowpre.ensure(std::max<size_t>(1, P.rowpre.size()) * 8), "alloc rowpre");
  urc = upload(h, h->rowpre.p, P.rowpre.data(), P.rowpre.size() * 8, &h->up_rowpre);
  if (urc) return urc;
  // rmse divisor per problem: n_t (PER_TASK); SHARED scores are already the
  // pooled mean SSE
  std::vector<double> div(P.pd.size());
  for (size_t q = 0; q < P.pd.size(); ++q)
    div[q] = P.shared ? 1.0 : (double)(P.off[P.pd[q].task + 1] - P.off[P.pd[q].task]);
  L0_CK(h->rdiv.ensure(div.size() * 8), "alloc");
  urc = upload(h, h->rdiv.p, div.data(), div.size() * 8, &h->up_rdiv);
  if (urc) return urc;
  L0_CK(h->out_t.ensure((size_t)P.out_t_total * 4), "alloc out");
  L0_CK(h->out_r.ensure((size_t)P.out_r_total * 8), "alloc out");
  L0_CK(h->dfr_n.ensure(24), "alloc");   // queued runs, queued tuples, redone tuples
  if (P.mixed && P.has_tuples) {
    L0_CK(h->dfr_key.ensure((size_t)kDeferCap * 8), "alloc deferral buffer");
    L0_CK(h->dfr_len.ensure((size_t)kDeferCap * 4), "alloc deferral buffer");
    L0_CK(h->dfr_bctr.ensure((size_t)n_probs * 4), "alloc deferral counters");
    if (P.m <= 8192) L0_CK(h->gram.ensure((size_t)P.T * P.gstride * 8), "alloc Gram");
  }
  const int S = staging_for(K);
  const int n_slots = std::max(P.has_singles ? 64 : 0, P.grid) + (P.mixed ? kDeferGroups : 0);
  const size_t nl = (size_t)n_probs * n_slots * K;
  L0_CK(h->lists_s.ensure(nl * sizeof(R)), "alloc lists");
  L0_CK(h->lists_k.ensure(nl * 8), "alloc lists");
  L0_CK(h->lists_cnt.ensure((size_t)n_probs * n_slots * 4), "alloc lists");
  L0_CK(h->gthr.ensure((size_t)n_probs * 8), "alloc gthr");
  L0_CK(h->hist.ensure((size_t)n_probs * L0_HIST_WORDS * 4), "alloc histogram");
  L0_CK(h->ctr.ensure(8), "alloc counter");
  const int groups = std::max(1, std::min(n_slots, 32));
  L0_CK(h->part_s.ensure((size_t)n_probs * groups * K * sizeof(R)), "alloc merge");
  L0_CK(h->part_k.ensure((size_t)n_probs * groups * K * 8), "alloc merge");
  L0_CK(h->part_cnt.ensure((size_t)n_probs * groups * 4), "alloc merge");
  if (h->done.n < (size_t)n_probs * 16 || h->done_init_for != (int)sizeof(R)) {
    // per problem: done counter, pad, ordered +inf bound; the merge leaves
    // them in this state
    L0_CK(h->done.ensure((size_t)n_probs * 16), "alloc merge");
    std::vector<unsigned> c0(4 * (size_t)(h->done.n / 16), 0u);
    for (size_t q = 0; q < h->done.n / 16; ++q) {
      const u64 inf = l0::ord_inf<R>();
      memcpy(&c0[4 * q + 2], &inf, 8);
    }
    L0_CK(cudaMemcpy(h->done.p, c0.data(), c0.size() * 4, cudaMemcpyHostToDevice), "copy");
    h->done_init_for = (int)sizeof(R);
  }
  L0_CK(h->pool_s.ensure((size_t)n_probs * K * sizeof(R)), "alloc pool");
  L0_CK(h->pool_k.ensure((size_t)n_probs * K * 8), "alloc pool");
  L0_CK(h->pool_cnt.ensure((size_t)n_probs * 4), "alloc pool");
  if ((size_t)(P.dmax + 1) * (size_t)P.nmax * 8 > 200 * 1024)
    L0_CK(h->scratch.ensure((size_t)n_probs * K * (P.dmax + 1) * (size_t)P.nmax * 8),
          "alloc refit scratch");
  L0_CK(h->refit.ensure((size_t)n_probs * K * 8), "alloc refit");
  L0_CK(h->cert.ensure((size_t)n_probs * sizeof(l0::CertOut)), "alloc cert");
  return SISSO_L0_OK;
}

// centring (+ split rows) and the Gram: device work only
int prep_pass(sisso_l0_t h, FitPlan &P) {
  cudaStream_t st = h->st;
  const int m = P.m, n_tasks = P.T;
  const long long N = P.N;
  L0_CK(cudaMemsetAsync(h->err.p, 0, 16, st), "memset");
  L0_CK(cudaEventRecord(h->ev[0], st), "event");
  L0_CK(cudaEventRecord(h->ev_fork, st), "event");
  L0_CK(cudaStreamWaitEvent(h->st2, h->ev_fork, 0), "event");
  L0_CK(l0::launch_column_classes(P.Xd, N, m, h->col_hash.as<u64>(), h->col_cls.as<int>(), h->st2),
        "class kernel");
  L0_CK(cudaEventRecord(h->ev_join, h->st2), "event");
  if (!P.mixed) {
    L0_CK(l0::launch_centre(P.Xd, P.yd, N, m, h->offs.as<long long>(), n_tasks, h->mu.as<double>(),
                            h->inv_s.as<double>(), h->w64.as<double>(), h->err.as<int>(), st),
          "centre kernel");
    L0_CK(cudaEventRecord(h->ev[1], st), "event");
    L0_CK(l0::launch_gram64(h->w64.as<double>(), N, m, P.off.data(), n_tasks,
                            h->gram.as<double>(), P.ld, P.gstride, st),
          "gram kernel");
  } else {
    // (the split rows need no clearing: the centring kernel writes every
    // entry of rows 0..m, padding included; TMA fills rows past m with zeros)
    L0_CK(cudaMemsetAsync(h->g64_have.p, 0, 4, st), "memset");   // new data: no FP64 Gram yet
    const int *kbeg = h->kmeta.as<int>();
    L0_CK(l0::launch_centre_split(P.Xd, P.yd, N, m, h->offs.as<long long>(), n_tasks,
                                  h->mu.as<double>(), h->inv_s.as<double>(), h->w64.as<double>(),
                                  h->abf.p, h->bbf.p, P.ldk, kbeg, kbeg + n_tasks,
                                  h->err.as<int>(), st),
          "centre kernel");
    L0_CK(cudaEventRecord(h->ev[1], st), "event");
    if (P.gsplit > 1)
      L0_CK(cudaMemsetAsync(h->gctr.p, 0, (size_t)l0::gram_tc_tiles(m) * n_tasks * 4, st), "memset");
    L0_CK(l0::launch_gram_tc(h->abf.p, h->bbf.p, P.ldk, m, n_tasks, kbeg, kbeg + 2 * n_tasks,
                             h->gram32.as<float>(), P.ld, P.gstride, h->err.as<int>(), st,
                             P.gsplit, h->gpart.as<float>(), h->gctr.as<unsigned>()),
          "tensor-core gram kernel");
  }
  L0_CK(cudaEventRecord(h->ev[6], st), "event");
  L0_CK(cudaStreamWaitEvent(st, h->ev_join, 0), "event");   // the classes, before any reader
  return SISSO_L0_OK;
}

template <typename R>
l0::TileArgs<R> tile_args(sisso_l0_t h, const FitPlan &P, int K, int S, const R *G, int n_slots,
                          long long item_limit) {
  l0::TileArgs<R> a{};
  a.G = G;
  a.probs = h->probs.as<l0::ProbDesc>();
  a.n_probs = (int)P.pd.size();
  a.row_prefix = h->rowpre.as<long long>();
  a.rowpre_len = (int)P.rowpre.size();
  a.B = l0::Binom{h->binom.as<u64>(), P.m + 1};
  a.ratio = P.mixed ? h->opt.fp32_fallback_pivot_ratio : h->opt.rank_deficient_pivot_ratio;
  a.K = K;
  a.S = S;
  a.item_counter = h->ctr.as<u64>();
  a.item_limit = item_limit;
  a.item_stride = P.n_shards;
  a.item_offset = P.shard;
  a.gthr = h->gthr.as<u64>();
  a.hist = h->hist.as<unsigned>();
  a.out_s = h->lists_s.as<R>();
  a.out_k = h->lists_k.as<u64>();
  a.out_cnt = h->lists_cnt.as<int>();
  a.n_slots = n_slots;
  a.dfr_key = h->dfr_key.as<u64>();
  a.dfr_len = h->dfr_len.as<unsigned>();
  a.dfr_n = h->dfr_n.as<u64>();
  a.dfr_cap = P.mixed ? kDeferCap : 0;
  a.err = h->err.as<int>();
  a.shared_T = P.shared ? P.T : 0;
  a.shared_gstride = P.gstride;
  a.inv_s = h->inv_s.as<double>();
  a.mp1 = P.m + 1;
  a.n_total = P.N;
  a.cls = h->col_cls.as<int>();
  a.band = P.band;
  return a;
}

template <typename R>
int launch_tuple_kernel(sisso_l0_t h, const FitPlan &P, const l0::TileArgs<R> &a) {
  if constexpr (std::is_same<R, float>::value) {
    if (P.variant > 0) {
      L0_CK(l0::launch_tile32(a, P.variant, std::max(P.dp_lo, 0), std::max(P.dp_hi, 0), P.grid,
                              l0::tile32_smem_bytes(a.K, a.S), h->st),
            "tile32 kernel");
      return SISSO_L0_OK;
    }
  }
  const size_t smem = l0::tile_smem_bytes<R>(a.K, a.S, std::max(P.dp_hi, 0));
  if (P.shared)
    L0_CK(l0::launch_tile_shared<R>(a, std::max(P.dp_hi, 0), P.grid, smem, h->st), "shared tile kernel");
  else
    L0_CK(l0::launch_tile<R>(a, std::max(P.dp_lo, 0), std::max(P.dp_hi, 0), P.grid, smem, h->st),
          "tile kernel");
  return SISSO_L0_OK;
}

// One search pass (device work only, so that it can be captured in a graph):
// seed, tuple kernel(s), FP64 redo, merge, re-fit, select.
template <typename R>
int search_pass(sisso_l0_t h, FitPlan &P, int K, const R *G) {
  cudaStream_t st = h->st;
  const int n_probs = (int)P.pd.size();
  const int S = staging_for(K);
  l0::Binom B{h->binom.as<u64>(), P.m + 1};
  const int n_slots = std::max(P.has_singles ? 64 : 0, P.grid) + (P.mixed ? kDeferGroups : 0);
  L0_CK(cudaMemsetAsync(h->lists_cnt.p, 0, (size_t)n_probs * n_slots * 4, st), "memset");
  L0_CK(cudaEventRecord(h->ev[2], st), "event");
  if (P.band) {
    // the band's cut from the previous pass's certificate (read before this
    // pass overwrites it)
    L0_CK(h->band_thr.ensure((size_t)n_probs * 8), "alloc band");
    L0_CK(h->band_floor.ensure((size_t)n_probs * 8), "alloc band");
    L0_CK(l0::launch_band_cut(h->cert.as<l0::CertOut>(), h->probs.as<l0::ProbDesc>(), n_probs,
                              h->inv_s.as<double>(), P.m + 1, P.shared, kBandMargin,
                              h->band_thr.as<u64>(), h->band_floor.as<double>(), st),
          "band kernel");
  }
  {
    const double ratio = P.mixed ? h->opt.fp32_fallback_pivot_ratio : h->opt.rank_deficient_pivot_ratio;
    // a proposal search ranks only its reachable triples, and a band pass
    // starts from its own cut: no seed bound
    L0_CK(l0::launch_seed<R>(G, h->probs.as<l0::ProbDesc>(), n_probs, K, S,
                             (P.shared || P.proposal || P.band) ? 0 : 1, ratio, B,
                             h->gthr.as<u64>(), h->hist.as<unsigned>(), l0::seed_keys(P.m, K),
                             st, h->col_cls.as<int>()),
          "seed kernel");
  }
  if (P.band)
    L0_CK(cudaMemcpyAsync(h->gthr.p, h->band_thr.p, (size_t)n_probs * 8, cudaMemcpyDeviceToDevice,
                          st),
          "band cut");
  if (P.has_singles) {
    const int gx = std::max(1, std::min(64, (P.m + L0_THREADS - 1) / L0_THREADS));
    L0_CK(l0::launch_singles<R>(G, P.pd.data(), h->probs.as<l0::ProbDesc>(), n_probs, K, S, gx,
                                h->gthr.as<u64>(), h->lists_s.as<R>(), h->lists_k.as<u64>(),
                                h->lists_cnt.as<int>(), n_slots, st, P.shared ? P.T : 0,
                                P.gstride, h->inv_s.as<double>(), P.m + 1, P.N),
          "singles kernel");
  }
  if (P.has_tuples) {
    L0_CK(cudaMemsetAsync(h->ctr.p, 0, 8, st), "memset");
    if (P.mixed) L0_CK(cudaMemsetAsync(h->dfr_n.p, 0, 24, st), "memset");
    L0_CK(cudaEventRecord(h->ev_k[0], st), "event");
    if (P.proposal) {
      L0_CK(cudaMemsetAsync(h->prop_ctr.p, 0, 16, st), "memset");
      l0::PropArgs<R> pa{};
      pa.G = G;
      pa.ld = P.ld;
      pa.diag = h->diag.as<R>();
      pa.m = P.m;
      pa.cls = h->col_cls.as<int>();
      pa.pairs = h->prop_pairs.as<int>();
      pa.n_pairs = P.n_pairs;
      pa.bits = h->prop_bits.as<unsigned>();
      pa.pair_ctr = h->prop_ctr.as<u64>();
      pa.fits = h->prop_ctr.as<u64>() + 1;
      pa.B = B;
      pa.total = binom_host(P.m, 3);
      pa.ratio = P.mixed ? h->opt.fp32_fallback_pivot_ratio : h->opt.rank_deficient_pivot_ratio;
      pa.mixed = P.mixed;
      pa.K = K;
      pa.S = S;
      pa.gthr = h->gthr.as<u64>();
      pa.hist = h->hist.as<unsigned>();
      pa.out_s = h->lists_s.as<R>();
      pa.out_k = h->lists_k.as<u64>();
      pa.out_cnt = h->lists_cnt.as<int>();
      pa.dfr_key = h->dfr_key.as<u64>();
      pa.dfr_len = h->dfr_len.as<unsigned>();
      pa.dfr_n = h->dfr_n.as<u64>();
      pa.dfr_cap = P.mixed ? kDeferCap : 0;
      pa.err = h->err.as<int>();
      L0_CK(l0::launch_proposal<R>(pa, P.grid, st), "proposal kernel");
    } else {
      l0::TileArgs<R> a = tile_args<R>(h, P, K, S, G, n_slots, P.n_items);
      int rc = launch_tuple_kernel<R>(h, P, a);
      if (rc) return rc;
    }
    L0_CK(cudaEventRecord(h->ev_k[1], st), "event");
    if (P.mixed) {
      // FP64 redo of the near-singular tuples the FP32 kernel queued: the
      // FP64 Gram and the Gram-mode redo run only when many were queued, the
      // dot-product redo only when a few were (decided on the device)
      const bool can_gram = P.m <= 8192;
      if (can_gram) {
        L0_CK(l0::launch_gram64(h->w64.as<double>(), P.N, P.m, P.off.data(), P.T,
                                h->gram.as<double>(), P.ld, P.gstride, st, h->dfr_n.as<u64>(),
                                P.dmax, 0, h->g64_have.as<int>()),
              "gram kernel");
        L0_CK(l0::launch_mark_gram64(h->dfr_n.as<u64>(), P.m, P.dmax, h->g64_have.as<int>(), st),
              "gram mark kernel");
      }
      l0::DeferArgs da{};
      da.G64 = can_gram ? h->gram.as<double>() : nullptr;
      da.ld64 = P.ld;
      da.g64_stride = P.gstride;
      da.W64 = h->w64.as<double>();
      da.n_total = P.N;
      da.offsets = h->offs.as<long long>();
      da.probs = h->probs.as<l0::ProbDesc>();
      da.B = B;
      da.ratio = h->opt.rank_deficient_pivot_ratio;
      da.run_key = h->dfr_key.as<u64>();
      da.run_len = h->dfr_len.as<unsigned>();
      da.n_runs = h->dfr_n.as<u64>();
      da.cap = kDeferCap;
      da.K = K;
      da.S = S;
      da.gthr = (u64 *)h->gthr.p;
      da.out_s = (float *)h->lists_s.p;
      da.out_k = h->lists_k.as<u64>();
      da.out_cnt = h->lists_cnt.as<int>();
      da.n_slots = n_slots;
      da.slot0 = n_slots - kDeferGroups;
      da.n_tuples = h->dfr_n.as<u64>() + 2;
      da.shared_T = P.shared ? P.T : 0;
      da.inv_s = h->inv_s.as<double>();
      da.mp1 = P.m + 1;
      da.batch_ctr = h->dfr_bctr.as<unsigned>();
      L0_CK(cudaMemsetAsync(h->dfr_bctr.p, 0, (size_t)n_probs * 4, st), "memset");
      L0_CK(l0::launch_defer(da, kDeferGroups, n_probs, st), "defer kernel");
    }
  }
  L0_CK(cudaEventRecord(h->ev[3], st), "event");
  // up to 1024 slot lists: one CTA per problem searches them all at once and
  // writes the pool; more: groups and a second level
  const int groups = n_slots <= 1024 ? 1 : std::min(n_slots, 32);
  L0_CK(l0::launch_merge<R>(h->lists_s.as<R>(), h->lists_k.as<u64>(), h->lists_cnt.as<int>(),
                            n_slots, n_probs, K, S, groups, h->gthr.as<u64>(), h->part_s.as<R>(),
                            h->part_k.as<u64>(), h->part_cnt.as<int>(), h->done.as<unsigned>(),
                            h->pool_s.as<R>(), h->pool_k.as<u64>(), h->pool_cnt.as<int>(), st),
        "merge kernel");
  L0_CK(cudaEventRecord(h->ev[4], st), "event");
  l0::RefitArgs ra{};
  ra.X = P.Xd;
  ra.y = P.yd;
  ra.n_total = P.N;
  ra.m = P.m;
  ra.offsets = h->offs.as<long long>();
  ra.mu = h->mu.as<double>();
  ra.T = P.T;
  ra.shared = P.shared;
  ra.probs = h->probs.as<l0::ProbDesc>();
  ra.n_probs = n_probs;
  ra.K = K;
  ra.pool_k = h->pool_k.as<u64>();
  ra.pool_cnt = h->pool_cnt.as<int>();
  ra.B = B;
  ra.rho_min = std::sqrt(h->opt.rank_deficient_pivot_ratio);
  ra.scratch = h->scratch.as<double>();
  ra.nmax = P.nmax;
  ra.dmax = P.dmax;
  ra.smem_rows = 0;
  ra.refit = h->refit.as<double>();
  ra.refit_all = P.exports_pool;   // a shard hands its whole re-fitted pool on
  L0_CK(l0::launch_refit(ra, st), "refit kernel");
  l0::SelectArgs<R> sa{};
  sa.probs = h->probs.as<l0::ProbDesc>();
  sa.n_probs = n_probs;
  sa.K = K;
  sa.pool_s = h->pool_s.as<R>();
  sa.pool_k = h->pool_k.as<u64>();
  sa.pool_cnt = h->pool_cnt.as<int>();
  sa.refit = h->refit.as<double>();
  sa.inv_s = h->inv_s.as<double>();
  sa.mp1 = P.m + 1;
  sa.shared = P.shared;
  sa.rmse_div = h->rdiv.as<double>();
  sa.B = B;
  sa.out_tuples = h->out_t.as<int>();
  sa.out_rmse = h->out_r.as<double>();
  sa.cert = h->cert.as<l0::CertOut>();
  sa.cert_safety = 4.0;
  sa.gthr = h->gthr.as<u64>();
  sa.refit_all = ra.refit_all;
  sa.delta_floor = P.band ? h->band_floor.as<double>() : nullptr;
  sa.band_thr = P.band ? h->band_thr.as<u64>() : nullptr;
  L0_CK(l0::launch_select<R>(sa, st), "select kernel");
  L0_CK(cudaEventRecord(h->ev[5], st), "event");
  return SISSO_L0_OK;
}

// after a pass: error word, certificate, statistics (host sync)
int finish_pass(sisso_l0_t h, FitPlan &P, int *certified, double *delta_max, float *ms_tuple,
                float *ms_merge, float *ms_refit, int *hopeless, int *bandable) {
  cudaStream_t st = h->st;
  const int n_probs = (int)P.pd.size();
  // status of the pass, read into pinned staging (asynchronous) when there
  // is room, else into pageable memory
  const size_t cb = (size_t)n_probs * sizeof(l0::CertOut);
  unsigned char *pst = pin_take(h, cb + 24 + 16 + 8);
  std::vector<unsigned char> pageable;
  if (!pst) {
    pageable.assign(cb + 24 + 16 + 8, 0);
    pst = pageable.data();
  }
  memset(pst, 0, cb + 24 + 16 + 8);
  L0_CK(cudaMemcpyAsync(pst, h->cert.p, cb, cudaMemcpyDeviceToHost, st), "copy cert");
  if (P.mixed && P.has_tuples)
    L0_CK(cudaMemcpyAsync(pst + cb, h->dfr_n.p, 24, cudaMemcpyDeviceToHost, st), "copy");
  if (P.proposal)
    L0_CK(cudaMemcpyAsync(pst + cb + 24, h->prop_ctr.p, 16, cudaMemcpyDeviceToHost, st), "copy");
  L0_CK(cudaMemcpyAsync(pst + cb + 40, h->err.p, 4, cudaMemcpyDeviceToHost, st), "copy err");
  int rc = wait_stream(h);
  if (rc) return rc;
  std::vector<l0::CertOut> cert(n_probs);
  memcpy(cert.data(), pst, cb);
  u64 dfr_stats[3], pfits[2];
  memcpy(dfr_stats, pst + cb, 24);
  memcpy(pfits, pst + cb + 24, 16);
  int host_err = 0;
  memcpy(&host_err, pst + cb + 40, 4);
  if (host_err == 5) return fail(h, SISSO_L0_ENONFINITE, "NaN or Inf in X or y");
  if (host_err == 7)
    return fail(h, SISSO_L0_EUNSUPPORTED,
                "too many near-singular tuples for the FP32 search; use SISSO_L0_FP64");
  if (host_err == 11) return fail(h, SISSO_L0_EINVAL, "pair list holds an index outside [0, n_sis) or i == j");
  if (host_err != 0) return fail(h, SISSO_L0_ECUDA, "device error flag " + std::to_string(host_err));
  P.fallback_tuples += dfr_stats[2];
  P.prop_fits += pfits[1];
  *certified = 1;
  *delta_max = 0;
  *hopeless = 0;
  *bandable = 1;   // a band cut needs a finite k-th re-fitted score everywhere
  for (auto &c : cert) {
    if (!std::isfinite(c.kth_refit) || !std::isfinite(c.delta)) *bandable = 0;
    if (!c.certified) {
      *certified = 0;
      // search-score errors of a quarter of the k-th score itself: a larger
      // pool cannot separate the best tuples
      if (4.0 * c.delta >= c.kth_refit) *hopeless = 1;
    }
    *delta_max = std::max(*delta_max, c.delta);
  }
  // phase timings are statistics only: a failed read (e.g. events recorded
  // inside a replayed graph) leaves them 0 and must not leave a pending error
  float t1 = 0, t2 = 0, t3 = 0;
  if (cudaEventElapsedTime(&t1, h->ev[2], h->ev[3]) != cudaSuccess) t1 = 0;
  if (cudaEventElapsedTime(&t2, h->ev[3], h->ev[4]) != cudaSuccess) t2 = 0;
  if (cudaEventElapsedTime(&t3, h->ev[4], h->ev[5]) != cudaSuccess) t3 = 0;
  if (!P.has_tuples || cudaEventElapsedTime(&h->ms_tuple_kernel, h->ev_k[0], h->ev_k[1]) != cudaSuccess)
    h->ms_tuple_kernel = 0.f;
  (void)cudaGetLastError();
  *ms_tuple += t1;
  *ms_merge += t2;
  *ms_refit += t3;
  return SISSO_L0_OK;
}

// ---------------------------------------------------------------- tuning --
// Like the paper's launch tuning (Sec. 2.4: the first batch is timed under a
// preset list of launch configurations and the best is kept), the first
// search of a shape times the tuple kernel (the whole search up to 1e9
// tuples, else its first quarter of work items; best of two runs) under each
// (kernel shape, resident CTAs per SM, work items per CTA) triple and keeps
// the fastest; choices persist in autotune_cache_path.
// Kernel shapes: the general kernel (8 rows x 4 columns per thread) and, for
// FP32 searches of d = 2 and 3, the kernel of l0_tile32.cu with 8 rows x 4
// columns per thread (one or two CTAs per SM) or 4 x 4 (512 threads).
std::string tune_key(sisso_l0_t h, const FitPlan &P) {
  if (h->dev_name.empty()) {   // one property query per handle, not per fit
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, h->opt.device) == cudaSuccess) h->dev_name = prop.name;
    else h->dev_name = "unknown";
  }
  int mb = 1;
  while (mb < P.m) mb <<= 1;
  char buf[256];
  snprintf(buf, sizeof(buf), "%s|prec=%d|shared=%d|dp=%d-%d|m<=%d|T=%d|shapes=%d", h->dev_name.c_str(),
           P.mixed, P.shared, P.dp_lo, P.dp_hi, mb, P.T, h->opt.tuple_kernel);
  std::string s(buf);
  for (char &c : s)
    if (c == ' ') c = '_';
  return s;
}

void load_tune_cache(sisso_l0_t h) {
  if (!h->opt.autotune_cache_path) return;
  FILE *f = fopen(h->opt.autotune_cache_path, "r");
  if (!f) return;
  // one choice per line: key, items factor, CTAs per SM, kernel shape
  char line[768], key[512];
  while (fgets(line, sizeof(line), f)) {
    int fa = 0, ba = 0, va = 0;
    if (sscanf(line, "%511s %d %d %d", key, &fa, &ba, &va) == 4 && fa >= 1 && ba >= 1 &&
        va >= 0 && va <= 3)
      h->tune[key] = {fa, ba, va};
  }
  fclose(f);
}

void store_tune(sisso_l0_t h, const std::string &key, int f, int b, int v) {
  h->tune[key] = {f, b, v};
  if (!h->opt.autotune_cache_path) return;
  FILE *fp = fopen(h->opt.autotune_cache_path, "a");
  if (!fp) return;
  fprintf(fp, "%s %d %d %d\n", key.c_str(), f, b, v);
  fclose(fp);
}

template <typename R>
int autotune(sisso_l0_t h, FitPlan &P, int K, const R *G) {
  const std::string key = tune_key(h, P);
  auto it = h->tune.find(key);
  const int Kmax = P.kmax_pool;
  auto apply = [&](int v, int b) -> int {
    P.variant = v;
    int bps = 0;
    int rc = tile_bps<R>(h, P, Kmax, &bps);
    if (rc) return rc;
    P.max_bps = std::max(1, bps);
    P.grid = h->n_sm * std::min(b, P.max_bps);
    return SISSO_L0_OK;
  };
  if (it != h->tune.end()) {
    const int v = tile32_ok(P, it->second.v) ? it->second.v : 0;
    P.items_factor = it->second.f;
    return apply(v, it->second.b);
  }
  cudaStream_t st = h->st;
  const int S = staging_for(K);
  const int n_probs = (int)P.pd.size();
  l0::Binom B{h->binom.as<u64>(), P.m + 1};
  float best = 1e30f;
  int best_f = P.items_factor, best_b = 1, best_v = P.variant;
  std::vector<int> shapes;
  if (h->opt.tuple_kernel >= 0) {
    shapes.push_back(tile32_ok(P, h->opt.tuple_kernel) ? h->opt.tuple_kernel : 0);
  } else {
    shapes.push_back(0);
    for (int v = 1; v <= 3; ++v)
      if (tile32_ok(P, v)) shapes.push_back(v);
  }
  const int factors[] = {1, 2, 4, 8, 16};
  double tuples_all = 0.0;
  for (const l0::ProbDesc &d : P.pd) tuples_all += (double)d.total;
  for (int v : shapes) {
    int rc = apply(v, 1);
    if (rc) return rc;
    const int bmax = std::min(P.max_bps, 2);
    for (int b = 1; b <= bmax; ++b) {
      for (int f : factors) {
        P.grid = h->n_sm * b;
        P.items_factor = f;
        plan_problems(P);
        rc = setup_search<R>(h, P, K);
        if (rc) return rc;
        const int n_slots = std::max(P.has_singles ? 64 : 0, P.grid) + (P.mixed ? kDeferGroups : 0);
        // each configuration runs twice and keeps its faster time; a search of
        // up to 1e9 tuples runs whole (a slice favours the shapes that suit
        // its own row blocks), a larger one its first quarter of items
        float ms_cfg = 1e30f;
        for (int rep = 0; rep < 2; ++rep) {
          L0_CK(cudaMemsetAsync(h->lists_cnt.p, 0, (size_t)n_probs * n_slots * 4, st), "memset");
          L0_CK(l0::launch_seed<R>(G, h->probs.as<l0::ProbDesc>(), n_probs, K, S, P.shared ? 0 : 1,
                                   P.mixed ? h->opt.fp32_fallback_pivot_ratio
                                           : h->opt.rank_deficient_pivot_ratio,
                                   B, h->gthr.as<u64>(), h->hist.as<unsigned>(),
                                   l0::seed_keys(P.m, K), st, h->col_cls.as<int>()),
                "seed kernel");
          L0_CK(cudaMemsetAsync(h->ctr.p, 0, 8, st), "memset");
          if (P.mixed) L0_CK(cudaMemsetAsync(h->dfr_n.p, 0, 24, st), "memset");
          const long long limit = tuples_all <= 1e9 ? P.n_items : std::max(1LL, P.n_items / 4);
          l0::TileArgs<R> a = tile_args<R>(h, P, K, S, G, n_slots, limit);
          L0_CK(cudaEventRecord(h->ev[2], st), "event");
          rc = launch_tuple_kernel<R>(h, P, a);
          if (rc) return rc;
          L0_CK(cudaEventRecord(h->ev[3], st), "event");
          rc = wait_stream(h);
          if (rc) return rc;
          float ms = 0;
          cudaEventElapsedTime(&ms, h->ev[2], h->ev[3]);
          ms_cfg = std::min(ms_cfg, ms);
        }
        if (ms_cfg < best) { best = ms_cfg; best_f = f; best_b = b; best_v = v; }
      }
    }
  }
  P.items_factor = best_f;
  int rc = apply(best_v, best_b);
  if (rc) return rc;
  store_tune(h, key, best_f, best_b, best_v);
  return SISSO_L0_OK;
}

// ----------------------------------------------------------------- graphs --
// With use_graph, the device work of prep + one search pass is captured once
// per (shape, input pointers, buffer addresses) and replayed afterwards.
std::string graph_key(sisso_l0_t h, const FitPlan &P, int K) {
  std::string k;
  char buf[128];
  snprintf(buf, sizeof(buf), "%p|%p|m=%d|N=%lld|T=%d|K=%d|g=%d|f=%d|p=%d|s=%d|v=%d|", (const void *)P.Xd,
           (const void *)P.yd, P.m, P.N, P.T, K, P.grid, P.items_factor, P.mixed, P.shared,
           P.variant);
  k += buf;
  for (long long o : P.off) k += std::to_string(o) + ",";
  for (const Req &r : P.req) k += "r" + std::to_string(r.d) + "x" + std::to_string(r.k);
  const DevBuf *bufs[] = {&h->xin, &h->yin, &h->offs, &h->mu, &h->inv_s, &h->w64, &h->gram,
                          &h->binom, &h->probs, &h->rowpre, &h->ctr, &h->gthr, &h->hist, &h->lists_s,
                          &h->lists_k, &h->lists_cnt, &h->part_s, &h->part_k, &h->part_cnt,
                          &h->done, &h->pool_s, &h->pool_k, &h->pool_cnt, &h->scratch, &h->refit,
                          &h->rdiv, &h->cert, &h->out_t, &h->out_r, &h->err, &h->dfr_key,
                          &h->dfr_len, &h->dfr_n, &h->abf, &h->bbf, &h->kmeta, &h->gram32,
                          &h->col_hash, &h->col_cls, &h->g64_have, &h->dfr_bctr, &h->gpart,
                          &h->gctr};
  for (const DevBuf *b : bufs) {
    snprintf(buf, sizeof(buf), "|%p", b->p);
    k += buf;
  }
  return k;
}

template <typename R>
int run_pass(sisso_l0_t h, FitPlan &P, int K, const R *G, bool with_prep, bool *replayed) {
  *replayed = false;
  if (!h->opt.use_graph || P.proposal || P.n_shards > 1 || P.band) {
    int rc = with_prep ? prep_pass(h, P) : SISSO_L0_OK;
    if (rc) return rc;
    return search_pass<R>(h, P, K, G);
  }
  const std::string key = graph_key(h, P, K) + (with_prep ? "|prep" : "");
  if (h->graph_exec && h->graph_key == key) {
    L0_CK(cudaGraphLaunch(h->graph_exec, h->st), "graph launch");
    *replayed = true;
    return SISSO_L0_OK;
  }
  if (h->graph_exec) {
    cudaGraphExecDestroy(h->graph_exec);
    h->graph_exec = nullptr;
  }
  L0_CK(cudaStreamBeginCapture(h->st, cudaStreamCaptureModeThreadLocal), "begin capture");
  int rc = with_prep ? prep_pass(h, P) : SISSO_L0_OK;
  if (!rc) rc = search_pass<R>(h, P, K, G);
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamEndCapture(h->st, &graph);
  if (rc) {
    if (graph) cudaGraphDestroy(graph);
    return rc;
  }
  if (e != cudaSuccess) return cuda_fail(h, e, "end capture");
  e = cudaGraphInstantiate(&h->graph_exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return cuda_fail(h, e, "graph instantiate");
  h->graph_key = key;
  L0_CK(cudaGraphLaunch(h->graph_exec, h->st), "graph launch");
  return SISSO_L0_OK;
}

// the learned forms' additions to a fit (see FitPlan)
struct Special {
  int proposal = 0, prep_only = 0;
  int shard = 0, n_shards = 1;
  int exports_pool = 0;   // the caller reads the whole re-fitted pool (a shard)
  std::function<int(sisso_l0_t, FitPlan &)> after_prep;
};

int fit_requests(sisso_l0_t h, const double *X, const double *y, const int64_t *task_offsets,
                 int32_t n_tasks, int64_t n_sis, const sisso_l0_request *reqs, int32_t n_reqs,
                 const Special *sp = nullptr) {
  if (!X || !y || !task_offsets || !reqs) return fail(h, SISSO_L0_EINVAL, "null pointer argument");
  if (n_tasks < 1) return fail(h, SISSO_L0_EINVAL, "n_tasks must be >= 1");
  if (n_reqs < 1) return fail(h, SISSO_L0_EINVAL, "at least one request");
  if (n_sis < 1) return fail(h, SISSO_L0_EINVAL, "n_sis must be >= 1");
  if (n_sis > (1LL << 30)) return fail(h, SISSO_L0_EUNSUPPORTED, "n_sis too large");
  if (task_offsets[0] != 0) return fail(h, SISSO_L0_EINVAL, "task_offsets[0] must be 0");
  if (h->opt.precision != SISSO_L0_FP64 && h->opt.precision != SISSO_L0_MIXED_BF16X3)
    return fail(h, SISSO_L0_EUNSUPPORTED, "precision not supported");
  FitPlan P;
  P.T = n_tasks;
  P.m = (int)n_sis;
  P.shared = (h->opt.task_mode == SISSO_L0_SHARED) ? 1 : 0;
  P.mixed = (h->opt.precision == SISSO_L0_MIXED_BF16X3) ? 1 : 0;
  P.n_out = P.shared ? 1 : n_tasks;
  if (sp) {
    P.proposal = sp->proposal;
    P.prep_only = sp->prep_only;
    P.shard = sp->shard;
    P.n_shards = sp->n_shards;
    P.exports_pool = sp->exports_pool;
    P.after_prep = sp->after_prep;
  }
  int kmax = 0;
  for (int q = 0; q < n_reqs; ++q) {
    const sisso_l0_request &r = reqs[q];
    if (!r.out_tuples || !r.out_rmse) return fail(h, SISSO_L0_EINVAL, "null output pointer");
    if (r.n_dim < 1 || r.n_dim > SISSO_L0_MAX_DIM)
      return fail(h, SISSO_L0_EINVAL, "n_dim must be in [1, 8]");
    if (n_sis < r.n_dim) return fail(h, SISSO_L0_EINVAL, "n_sis must be >= n_dim");
    if (r.k < 1) return fail(h, SISSO_L0_EINVAL, "k must be >= 1");
    const u64 total = binom_host(n_sis, r.n_dim);
    if (total >= kSat)
      return fail(h, SISSO_L0_EUNSUPPORTED, "C(n_sis, n_dim) does not fit in 62 bits");
    if ((u64)r.k > total) return fail(h, SISSO_L0_EINVAL, "k exceeds C(n_sis, n_dim)");
    if (r.k > 2048) return fail(h, SISSO_L0_EUNSUPPORTED, "k above 2048");
    P.req.push_back(Req{r.n_dim, r.k, r.out_tuples, r.out_rmse});
    P.dmax = std::max(P.dmax, r.n_dim);
    kmax = std::max(kmax, r.k);
    if (r.n_dim == 1) {
      P.has_singles = true;
    } else {
      P.has_tuples = true;
      const int dp = r.n_dim - 2;
      P.dp_lo = P.dp_lo < 0 ? dp : std::min(P.dp_lo, dp);
      P.dp_hi = std::max(P.dp_hi, dp);
    }
    P.fits_per_pass += total * (u64)n_tasks;
  }
  if (P.has_tuples && P.dp_hi - P.dp_lo > 0 &&
      !((P.dp_lo == 0 && P.dp_hi <= 2) || (P.dp_lo == 1 && P.dp_hi == 2)) )
    return fail(h, SISSO_L0_EUNSUPPORTED, "tuple sizes of one call must lie within {2, 3, 4}");
  if (P.shared && P.dp_hi > P.dp_lo)
    return fail(h, SISSO_L0_EUNSUPPORTED, "SHARED mode takes one tuple size >= 2 per call");
  P.off.assign(task_offsets, task_offsets + n_tasks + 1);
  for (int t = 0; t < n_tasks; ++t) {
    const long long nt = P.off[t + 1] - P.off[t];
    if (nt < P.dmax + 2) return fail(h, SISSO_L0_EINVAL, "every task needs at least n_dim + 2 rows");
    P.nmax = std::max(P.nmax, nt);
  }
  P.N = P.off[n_tasks];
  const int m = P.m;
  const long long N = P.N;
  // candidate pool K': at least every k, at most 2048 (shared-memory lists),
  // never more than the number of tuples of the smallest request
  u64 total_min = ~0ull;
  for (const Req &r : P.req) total_min = std::min(total_min, binom_host(m, r.d));
  int Kmax = h->opt.max_candidate_pool > 0 ? std::min(h->opt.max_candidate_pool, 2048) : 2048;
  int K = h->opt.candidate_pool > 0 ? h->opt.candidate_pool : std::min(std::max(4 * kmax, 256), 2048);
  K = std::min(std::max(K, kmax), 2048);
  if ((u64)K > total_min) K = (int)std::max<u64>(total_min, (u64)kmax);
  Kmax = std::max(Kmax, K);
  P.kmax_pool = Kmax;
  cudaStream_t st = h->st;
  {
    const int prc = pin_reset(h);
    if (prc) return prc;
  }
  if (h->own_st) {
    // the caller's earlier work (e.g. producing X) precedes ours
    L0_CK(cudaEventRecord(h->ev_user, h->user_st), "event");
    L0_CK(cudaStreamWaitEvent(st, h->ev_user, 0), "stream wait");
  }
  // inputs on the device
  const double *Xd = X, *yd = y;
  if (!is_device_ptr(X)) {
    L0_CK(h->xin.ensure((size_t)m * N * 8), "alloc X");
    L0_CK(cudaMemcpyAsync(h->xin.p, X, (size_t)m * N * 8, cudaMemcpyHostToDevice, st), "copy X");
    Xd = h->xin.as<double>();
  }
  if (!is_device_ptr(y)) {
    L0_CK(h->yin.ensure((size_t)N * 8), "alloc y");
    L0_CK(cudaMemcpyAsync(h->yin.p, y, (size_t)N * 8, cudaMemcpyHostToDevice, st), "copy y");
    yd = h->yin.as<double>();
  }
  P.Xd = Xd;
  P.yd = yd;
  L0_CK(h->offs.ensure((n_tasks + 1) * 8), "alloc offsets");
  int rc = upload(h, h->offs.p, P.off.data(), (n_tasks + 1) * 8, &h->up_offs);
  if (rc) return rc;
  L0_CK(h->err.ensure(16), "alloc err");
  rc = ensure_binom(h, m);
  if (rc) return rc;
  // buffers of the centring and the Gram
  const int mp1 = m + 1;
  P.ld = ((long long)mp1 + 31) / 32 * 32;
  P.gstride = (long long)mp1 * P.ld;
  L0_CK(h->mu.ensure((size_t)n_tasks * mp1 * 8), "alloc mu");
  L0_CK(h->col_hash.ensure((size_t)m * 8), "alloc column hashes");
  L0_CK(h->col_cls.ensure((size_t)m * 4), "alloc column classes");
  L0_CK(h->inv_s.ensure((size_t)n_tasks * mp1 * 8), "alloc inv_s");
  L0_CK(h->w64.ensure((size_t)mp1 * N * 8), "alloc W");
  if (!P.mixed) {
    L0_CK(h->gram.ensure((size_t)n_tasks * P.gstride * 8), "alloc Gram");
    P.have_g64 = true;
  } else {
    // split-BF16 rows: per task three segments of npad_t = roundup(n_t, 64)
    std::vector<int> meta(3 * n_tasks);
    long long ldk = 0;
    for (int t = 0; t < n_tasks; ++t) {
      const long long nt = P.off[t + 1] - P.off[t];
      const long long np = (nt + 63) / 64 * 64;
      if (ldk + 3 * np > (1LL << 30)) return fail(h, SISSO_L0_EUNSUPPORTED, "too many samples");
      meta[t] = (int)ldk;                           // first K column of the task
      meta[n_tasks + t] = (int)np;                  // padded samples
      meta[2 * n_tasks + t] = (int)(3 * np / 64);   // K blocks
      ldk += 3 * np;
    }
    P.ldk = ldk;
    const size_t abytes = (size_t)mp1 * ldk * 2;
    L0_CK(h->abf.ensure(abytes), "alloc split rows");
    L0_CK(h->bbf.ensure(abytes), "alloc split rows");
    L0_CK(h->kmeta.ensure(meta.size() * 4), "alloc");
    rc = upload(h, h->kmeta.p, meta.data(), meta.size() * 4, &h->up_kmeta);
    if (rc) return rc;
    L0_CK(h->gram32.ensure((size_t)n_tasks * P.gstride * 4), "alloc Gram");
    L0_CK(h->g64_have.ensure(4), "alloc");
    // K splits of the tensor-core Gram: about one CTA per SM in all (one
    // fits an SM), no more than the fewest K blocks of a task, at most 8
    {
      int nk_min = 1 << 30;
      for (int t = 0; t < n_tasks; ++t) nk_min = std::min(nk_min, meta[2 * n_tasks + t]);
      const int tiles = l0::gram_tc_tiles(m) * n_tasks;
      P.gsplit = std::max(1, std::min(std::min(8, nk_min), h->n_sm / std::max(1, tiles)));
      if (P.gsplit > 1) {
        L0_CK(h->gpart.ensure(l0::gram_tc_part_floats(m, n_tasks, P.gsplit) * 4), "alloc Gram split");
        L0_CK(h->gctr.ensure((size_t)tiles * 4), "alloc Gram split");
      }
    }
  }
  // persistent grid of the tuple kernel (or of the proposal search)
  if (P.has_tuples && P.proposal) {
    int bps = 0;
    const int S0 = staging_for(Kmax);
    cudaError_t e = P.mixed ? l0::proposal_occupancy<float>(Kmax, S0, &bps)
                            : l0::proposal_occupancy<double>(Kmax, S0, &bps);
    if (e != cudaSuccess) return cuda_fail(h, e, "proposal occupancy");
    if (bps < 1) return fail(h, SISSO_L0_EUNSUPPORTED, "proposal kernel does not fit on an SM");
    P.max_bps = bps;
    P.grid = h->n_sm * bps;
  } else if (P.has_tuples) {
    int bps = 0;
    // default shape: the d <= 3 FP32 kernel, 512 threads, where it applies
    const int want = h->opt.tuple_kernel < 0 ? 3 : h->opt.tuple_kernel;
    P.variant = tile32_ok(P, want) ? want : 0;
    rc = P.mixed ? tile_bps<float>(h, P, Kmax, &bps) : tile_bps<double>(h, P, Kmax, &bps);
    if (rc) return rc;
    if (bps < 1 && P.variant > 0) {
      P.variant = 0;
      rc = P.mixed ? tile_bps<float>(h, P, Kmax, &bps) : tile_bps<double>(h, P, Kmax, &bps);
      if (rc) return rc;
    }
    if (bps < 1) return fail(h, SISSO_L0_EUNSUPPORTED, "tuple kernel does not fit on an SM");
    P.max_bps = bps;
    P.grid = h->n_sm * bps;
  }
  // untuned: 4 items per CTA for the FP32 d <= 3 kernel (fastest on the
  // d = 3, 1000-column search once the tiles holding the strongest columns
  // go out first), 2 for the general one
  P.items_factor = P.variant > 0 ? 4 : 2;
  plan_problems(P);
  rc = P.mixed ? setup_search<float>(h, P, K) : setup_search<double>(h, P, K);
  if (rc) return rc;
  // autotuning needs the Gram: run the prep once outside any graph
  bool prep_done = false;
  h->stats.tuned_items_factor = 0;
  h->stats.tuned_ctas_per_sm = 0;
  if (P.proposal || P.prep_only) {
    // the learned forms: Gram, its symmetric copy, then the pair list (or
    // the pair data) before any search
    rc = prep_pass(h, P);
    if (rc) return rc;
    prep_done = true;
    if (P.mixed) {
      L0_CK(h->diag.ensure((size_t)m * 4), "alloc diagonal");
      L0_CK(l0::launch_gram_mirror<float>(h->gram32.as<float>(), P.ld, m + 1, h->diag.as<float>(), st),
            "mirror kernel");
    } else {
      L0_CK(h->diag.ensure((size_t)m * 8), "alloc diagonal");
      L0_CK(l0::launch_gram_mirror<double>(h->gram.as<double>(), P.ld, m + 1, h->diag.as<double>(), st),
            "mirror kernel");
    }
    if (P.after_prep) {
      rc = P.after_prep(h, P);
      if (rc) return rc;
    }
    if (P.prep_only) {
      int host_err = 0;
      L0_CK(cudaMemcpyAsync(&host_err, h->err.p, 4, cudaMemcpyDeviceToHost, st), "copy err");
      rc = wait_stream(h);
      if (rc) return rc;
      if (host_err == 5) return fail(h, SISSO_L0_ENONFINITE, "NaN or Inf in X or y");
      if (host_err != 0) return fail(h, SISSO_L0_ECUDA, "device error flag " + std::to_string(host_err));
      return SISSO_L0_OK;
    }
  } else if (h->opt.autotune && P.has_tuples && P.n_shards == 1) {
    rc = prep_pass(h, P);
    if (rc) return rc;
    prep_done = true;
    rc = P.mixed ? autotune<float>(h, P, K, h->gram32.as<float>())
                 : autotune<double>(h, P, K, h->gram.as<double>());
    if (rc) return rc;
    plan_problems(P);
    rc = P.mixed ? setup_search<float>(h, P, K) : setup_search<double>(h, P, K);
    if (rc) return rc;
  }
  int certified = 0, enl = 0;
  double delta = 0;
  float ms_tuple = 0, ms_merge = 0, ms_refit = 0;
  bool replayed = false;
  for (;;) {
    if (enl > 0) {
      rc = P.mixed ? setup_search<float>(h, P, K) : setup_search<double>(h, P, K);
      if (rc) break;
    }
    const bool with_prep = !prep_done;
    rc = P.mixed ? run_pass<float>(h, P, K, h->gram32.as<float>(), with_prep, &replayed)
                 : run_pass<double>(h, P, K, h->gram.as<double>(), with_prep, &replayed);
    if (rc) break;
    prep_done = true;
    int hopeless = 0, bandable = 0;
    rc = finish_pass(h, P, &certified, &delta, &ms_tuple, &ms_merge, &ms_refit, &hopeless,
                     &bandable);
    if (rc) break;
    // An FP32 pass that cannot rank the best tuples (its score errors reach
    // the gaps between them, or the pool stays uncertified at the largest
    // K') is followed by a band pass at the same K': the tuples near the cut
    // are scored in FP64.  A band pass that still fails ends the mixed fit
    // (the caller may redo it in FP64).
    if (!certified && P.mixed && !P.band && h->opt.fp64_rerun_uncertified && !P.proposal &&
        P.n_shards == 1 && !P.exports_pool && P.has_tuples && bandable &&
        (hopeless || K >= Kmax)) {
      P.band = 1;
      continue;
    }
    if (!certified && hopeless && !P.band && P.mixed && h->opt.fp64_rerun_uncertified) break;
    // a shard's pool is certified against the merged result, not its own
    if (certified || K >= Kmax || P.n_shards > 1) break;
    K = std::min(2 * K, Kmax);
    ++enl;
  }
  if (rc) return rc;
  // outputs to the caller
  for (size_t q = 0; q < P.req.size(); ++q) {
    const Req &r = P.req[q];
    const l0::ProbDesc &first = P.pd[q * (P.shared ? 1 : P.T)];
    const size_t nt = (size_t)P.n_out * r.k * r.d, nr = (size_t)P.n_out * r.k;
    L0_CK(cudaMemcpyAsync(r.out_t, h->out_t.as<int>() + first.out_t_off, nt * 4, cudaMemcpyDefault,
                          st), "copy out");
    L0_CK(cudaMemcpyAsync(r.out_r, h->out_r.as<double>() + first.out_r_off, nr * 8,
                          cudaMemcpyDefault, st), "copy out");
  }
  rc = wait_stream(h);
  if (rc) return rc;
  float t_prep = 0, t_gram = 0;
  if (cudaEventElapsedTime(&t_prep, h->ev[0], h->ev[1]) != cudaSuccess) t_prep = 0;
  if (cudaEventElapsedTime(&t_gram, h->ev[1], h->ev[6]) != cudaSuccess) t_gram = 0;
  (void)cudaGetLastError();
  sisso_l0_stats &S = h->stats;
  const int tf = S.tuned_items_factor, tb = S.tuned_ctas_per_sm;
  memset(&S, 0, sizeof(S));
  S.struct_size = sizeof(S);
  S.candidate_pool = K;
  S.pool_enlargements = enl;
  S.certified = certified;
  S.tuple_fits = P.proposal ? P.prop_fits : P.fits_per_pass * (u64)(enl + 1);
  S.proposal_pairs = P.proposal ? P.n_pairs : 0;
  S.max_pool_rel_error = delta;
  S.fp64_fallback_tuples = P.fallback_tuples;
  // centring + Gram, then per pass: seed, singles?, tuple, redo (mixed: gated
  // FP64 Gram + two redo kernels), merge, re-fit, select
  const long long per_pass = 5 + (P.has_singles ? 1 : 0) + (P.mixed && P.has_tuples ? 3 : 0) -
                             (P.has_tuples ? 0 : 1);
  S.kernel_launches = 2 + (P.mixed ? 2 : 1 + n_tasks) + per_pass * (enl + 1);
  S.graph_replayed = replayed ? 1 : 0;
  S.tuned_items_factor = h->opt.autotune ? P.items_factor : tf;
  S.tuned_ctas_per_sm = h->opt.autotune ? P.grid / std::max(1, h->n_sm) : tb;
  S.ms_prep = t_prep;
  S.ms_gram = t_gram;
  S.ms_tuple = ms_tuple;
  S.ms_merge = ms_merge;
  S.ms_refit = ms_refit;
  S.ms_total = t_prep + t_gram + ms_tuple + ms_merge + ms_refit;
  S.ms_tuple_kernel = h->ms_tuple_kernel;
  S.tuple_kernel = P.variant;
  S.band_pass = P.band;
  return SISSO_L0_OK;
}

// A mixed-precision fit whose pool stays uncertified at the largest K' is
// one where the FP32 score errors reach the gaps between the best scores;
// FP64 is what stability needs there, so the fit is redone in FP64.
// identity of a call's inputs and requests (pointers, shapes, requests)
std::string inputs_key(const double *X, const double *y, const int64_t *off, int32_t n_tasks,
                       int64_t n_sis, const sisso_l0_request *reqs, int32_t n_reqs) {
  std::string k;
  char buf[96];
  snprintf(buf, sizeof(buf), "%p|%p|%lld|", (const void *)X, (const void *)y, (long long)n_sis);
  k += buf;
  for (int t = 0; t <= n_tasks; ++t) k += std::to_string((long long)off[t]) + ",";
  for (int q = 0; q < n_reqs; ++q) k += "r" + std::to_string(reqs[q].n_dim) + "x" + std::to_string(reqs[q].k);
  return k;
}

int fit_checked(sisso_l0_t h, const double *X, const double *y, const int64_t *task_offsets,
                int32_t n_tasks, int64_t n_sis, const sisso_l0_request *reqs, int32_t n_reqs) {
  const bool mixed = h->opt.precision == SISSO_L0_MIXED_BF16X3;
  std::string key;
  if (mixed && h->opt.fp64_rerun_uncertified && X && y && task_offsets && reqs && n_tasks > 0)
    key = inputs_key(X, y, task_offsets, n_tasks, n_sis, reqs, n_reqs);
  if (!key.empty() && key == h->fp64_key) {
    // the same inputs needed FP64 last time: go there directly
    h->opt.precision = SISSO_L0_FP64;
    int rc = fit_requests(h, X, y, task_offsets, n_tasks, n_sis, reqs, n_reqs);
    h->opt.precision = SISSO_L0_MIXED_BF16X3;
    h->stats.fp64_rerun = 2;
    return rc;
  }
  int rc = fit_requests(h, X, y, task_offsets, n_tasks, n_sis, reqs, n_reqs);
  if (rc || !mixed || h->stats.certified || !h->opt.fp64_rerun_uncertified) return rc;
  const double ms_first = h->stats.ms_total;
  h->opt.precision = SISSO_L0_FP64;
  rc = fit_requests(h, X, y, task_offsets, n_tasks, n_sis, reqs, n_reqs);
  h->opt.precision = SISSO_L0_MIXED_BF16X3;
  h->stats.fp64_rerun = 1;
  h->stats.ms_total += ms_first;
  if (!rc) h->fp64_key = key;
  return rc;
}

}  // namespace

extern "C" {

int sisso_l0_default_options(sisso_l0_options *opt) {
  if (!opt) return SISSO_L0_EINVAL;
  memset(opt, 0, sizeof(*opt));
  opt->struct_size = sizeof(*opt);
  opt->device = 0;
  opt->stream = nullptr;
  opt->precision = SISSO_L0_FP64;
  opt->task_mode = SISSO_L0_PER_TASK;
  opt->candidate_pool = 0;
  opt->max_candidate_pool = 2048;
  opt->fp32_fallback_pivot_ratio = 1e-6;
  opt->rank_deficient_pivot_ratio = 1e-12;
  opt->autotune = 0;
  opt->use_graph = 0;
  opt->autotune_cache_path = nullptr;
  opt->timeout_seconds = 0.0;
  opt->fp64_rerun_uncertified = 1;
  opt->tuple_kernel = -1;
  return SISSO_L0_OK;
}

int sisso_l0_create(sisso_l0_t *out, const sisso_l0_options *opt) {
  if (!out) return SISSO_L0_EINVAL;
  *out = nullptr;
  sisso_l0_options o;
  sisso_l0_default_options(&o);
  if (opt) {
    if (opt->struct_size != (int32_t)sizeof(sisso_l0_options)) return SISSO_L0_EINVAL;
    o = *opt;
  }
  if (o.precision < 0 || o.precision > 2 || o.task_mode < 0 || o.task_mode > 1) return SISSO_L0_EINVAL;
  if (o.tuple_kernel < -1 || o.tuple_kernel > 3) return SISSO_L0_EINVAL;
  if (!(o.rank_deficient_pivot_ratio >= 0) || !(o.fp32_fallback_pivot_ratio >= 0)) return SISSO_L0_EINVAL;
  sisso_l0_handle *h = new (std::nothrow) sisso_l0_handle();
  if (!h) return SISSO_L0_ENOMEM;
  h->opt = o;
  h->st = (cudaStream_t)o.stream;
  h->user_st = h->st;
  cudaError_t e = cudaSetDevice(o.device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&h->n_sm, cudaDevAttrMultiProcessorCount, o.device);
  for (int i = 0; i < 8 && e == cudaSuccess; ++i) e = cudaEventCreate(&h->ev[i]);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_user, cudaEventDisableTiming);
  for (int i = 0; i < 2 && e == cudaSuccess; ++i) e = cudaEventCreate(&h->ev_k[i]);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_pin, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->st2, cudaStreamNonBlocking);
  if (e == cudaSuccess && o.use_graph && h->st == nullptr) {
    e = cudaStreamCreateWithFlags(&h->st, cudaStreamNonBlocking);
    h->own_st = (e == cudaSuccess);
  }
  if (e != cudaSuccess) {
    delete h;
    return (e == cudaErrorMemoryAllocation) ? SISSO_L0_ENOMEM : SISSO_L0_ECUDA;
  }
  load_tune_cache(h);
  *out = h;
  return SISSO_L0_OK;
}

int sisso_l0_fit(sisso_l0_t h, const double *X, const double *y, const int64_t *task_offsets,
                 int32_t n_tasks, int64_t n_sis, int32_t n_dim, int32_t k, int32_t *out_tuples,
                 double *out_rmse) {
  if (!h) return SISSO_L0_EINVAL;
  try {
    cudaError_t e = cudaSetDevice(h->opt.device);
    if (e != cudaSuccess) return cuda_fail(h, e, "set device");
    sisso_l0_request r{n_dim, k, out_tuples, out_rmse};
    return fit_checked(h, X, y, task_offsets, n_tasks, n_sis, &r, 1);
  } catch (const std::bad_alloc &) {
    return fail(h, SISSO_L0_ENOMEM, "host allocation failed");
  } catch (...) {
    return fail(h, SISSO_L0_ECUDA, "unexpected host exception");
  }
}

int sisso_l0_fit_multi(sisso_l0_t h, const double *X, const double *y,
                       const int64_t *task_offsets, int32_t n_tasks, int64_t n_sis,
                       const sisso_l0_request *reqs, int32_t n_reqs) {
  if (!h) return SISSO_L0_EINVAL;
  try {
    cudaError_t e = cudaSetDevice(h->opt.device);
    if (e != cudaSuccess) return cuda_fail(h, e, "set device");
    return fit_checked(h, X, y, task_offsets, n_tasks, n_sis, reqs, n_reqs);
  } catch (const std::bad_alloc &) {
    return fail(h, SISSO_L0_ENOMEM, "host allocation failed");
  } catch (...) {
    return fail(h, SISSO_L0_ECUDA, "unexpected host exception");
  }
}

int sisso_l0_set_timeout(sisso_l0_t h, double timeout_seconds) {
  if (!h || timeout_seconds != timeout_seconds) return SISSO_L0_EINVAL;
  h->opt.timeout_seconds = timeout_seconds;
  return SISSO_L0_OK;
}

int sisso_l0_debug_fail_allocation(int64_t after) {
  g_alloc_fail_countdown = after < 0 ? -1 : (long long)after;
  return SISSO_L0_OK;
}

int sisso_l0_get_stats(sisso_l0_t h, sisso_l0_stats *out) {
  if (!h || !out) return SISSO_L0_EINVAL;
  *out = h->stats;
  return SISSO_L0_OK;
}

const char *sisso_l0_last_error(sisso_l0_t h) {
  if (!h) return kNullHandleMsg;
  return h->last_error.c_str();
}

void sisso_l0_destroy(sisso_l0_t h) {
  if (!h) return;
  cudaSetDevice(h->opt.device);
  if (h->st) cudaStreamSynchronize(h->st);
  else cudaDeviceSynchronize();
  if (h->own_st && h->user_st) cudaStreamSynchronize(h->user_st);
  DevBuf *bufs[] = {&h->xin, &h->yin, &h->offs, &h->mu, &h->inv_s, &h->w64, &h->gram, &h->binom,
                    &h->probs, &h->rowpre, &h->ctr, &h->gthr, &h->hist, &h->lists_s, &h->lists_k,
                    &h->lists_cnt, &h->part_s, &h->part_k, &h->part_cnt, &h->done, &h->pool_s,
                    &h->pool_k, &h->pool_cnt, &h->scratch, &h->refit, &h->rdiv,
                    &h->cert, &h->out_t, &h->out_r, &h->err, &h->dfr_key, &h->dfr_len, &h->dfr_n,
                    &h->dfr_cnt, &h->abf, &h->bbf, &h->kmeta, &h->gram32, &h->prop_in,
                    &h->prop_pairs, &h->prop_bits, &h->prop_ctr, &h->sel_hist, &h->sel_bin,
                    &h->scores, &h->diag, &h->col_hash, &h->col_cls, &h->sis_ex, &h->sis_y,
                    &h->gen_ops, &h->gen_c1, &h->gen_c2, &h->gen_valid, &h->gen_cf, &h->gen_csafe,
                    &h->loop_x, &h->loop_y,
                    &h->loop_xs, &h->loop_res, &h->loop_q, &h->loop_tup, &h->loop_rows,
                    &h->band_thr, &h->band_floor, &h->g64_have, &h->dfr_bctr, &h->gpart,
                    &h->gctr};
  for (DevBuf *b : bufs) b->release();
  if (h->pin) cudaFreeHost(h->pin);
  if (h->ev_pin) cudaEventDestroy(h->ev_pin);
  for (int i = 0; i < 8; ++i)
    if (h->ev[i]) cudaEventDestroy(h->ev[i]);
  if (h->graph_exec) cudaGraphExecDestroy(h->graph_exec);
  if (h->ev_user) cudaEventDestroy(h->ev_user);
  for (int i = 0; i < 2; ++i)
    if (h->ev_k[i]) cudaEventDestroy(h->ev_k[i]);
  if (h->own_st) cudaStreamDestroy(h->st);
  if (h->ev_fork) cudaEventDestroy(h->ev_fork);
  if (h->ev_join) cudaEventDestroy(h->ev_join);
  if (h->st2) cudaStreamDestroy(h->st2);
  delete h;
}

uint64_t sisso_l0_count_tuples(int64_t m, int32_t n) {
  if (m < 0 || n < 0) return 0;
  unsigned __int128 r = 1;
  for (int i = 1; i <= n; ++i) {
    if (m - n + i <= 0) return 0;
    r = r * (unsigned __int128)(m - n + i) / (unsigned __int128)i;
    if (r >> 63) return 0;
  }
  return (uint64_t)r;
}

int sisso_l0_debug_unrank(sisso_l0_t h, int64_t m, int32_t n, const uint64_t *ranks,
                          int64_t count, int32_t *tuples_out) {
  if (!h || !ranks || !tuples_out || m < 1 || n < 1 || n > SISSO_L0_MAX_DIM || n > m || count < 0)
    return fail(h, SISSO_L0_EINVAL, "bad arguments");
  const u64 total = binom_host(m, n);
  if (total >= kSat) return fail(h, SISSO_L0_EUNSUPPORTED, "C(m, n) too large");
  for (int64_t i = 0; i < count; ++i)
    if (ranks[i] >= total) return fail(h, SISSO_L0_EINVAL, "rank out of range");
  L0_CK(cudaSetDevice(h->opt.device), "set device");
  int rc = ensure_binom(h, (int)m);
  if (rc) return rc;
  DevBuf r, t;
  L0_CK(r.ensure((size_t)count * 8 + 8), "alloc");
  L0_CK(t.ensure((size_t)count * n * 4 + 4), "alloc");
  L0_CK(cudaMemcpyAsync(r.p, ranks, (size_t)count * 8, cudaMemcpyHostToDevice, h->st), "copy");
  l0::Binom B{h->binom.as<u64>(), (int)m + 1};
  L0_CK(l0::launch_unrank(B, (int)m, n, total, r.as<u64>(), count, t.as<int>(), h->st), "unrank kernel");
  L0_CK(cudaMemcpyAsync(tuples_out, t.p, (size_t)count * n * 4, cudaMemcpyDeviceToHost, h->st), "copy");
  rc = wait_stream(h);
  r.release();
  t.release();
  return rc;
}

int sisso_l0_debug_gram(sisso_l0_t h, const double *X, const double *y, const int64_t *task_offsets,
                        int32_t n_tasks, int64_t n_sis, int32_t task, double *out) {
  if (!h || !X || !y || !task_offsets || !out || n_tasks < 1 || n_sis < 1 || task < 0 || task >= n_tasks)
    return fail(h, SISSO_L0_EINVAL, "bad arguments");
  if (task_offsets[0] != 0) return fail(h, SISSO_L0_EINVAL, "task_offsets[0] must be 0");
  for (int t = 0; t < n_tasks; ++t)
    if (task_offsets[t + 1] - task_offsets[t] < 2) return fail(h, SISSO_L0_EINVAL, "task too small");
  L0_CK(cudaSetDevice(h->opt.device), "set device");
  cudaStream_t st = h->st;
  const int m = (int)n_sis;
  const long long N = task_offsets[n_tasks];
  DevBuf xd, yd, od, mu, is, w, g, err;
  L0_CK(xd.ensure((size_t)m * N * 8), "alloc");
  L0_CK(yd.ensure((size_t)N * 8), "alloc");
  L0_CK(od.ensure((size_t)(n_tasks + 1) * 8), "alloc");
  L0_CK(cudaMemcpyAsync(xd.p, X, (size_t)m * N * 8, cudaMemcpyDefault, st), "copy");
  L0_CK(cudaMemcpyAsync(yd.p, y, (size_t)N * 8, cudaMemcpyDefault, st), "copy");
  L0_CK(cudaMemcpyAsync(od.p, task_offsets, (size_t)(n_tasks + 1) * 8, cudaMemcpyHostToDevice, st), "copy");
  const int mp1 = m + 1;
  L0_CK(mu.ensure((size_t)n_tasks * mp1 * 8), "alloc");
  L0_CK(is.ensure((size_t)n_tasks * mp1 * 8), "alloc");
  L0_CK(w.ensure((size_t)mp1 * N * 8), "alloc");
  L0_CK(err.ensure(16), "alloc");
  L0_CK(cudaMemsetAsync(err.p, 0, 16, st), "memset");
  L0_CK(l0::launch_centre(xd.as<double>(), yd.as<double>(), N, m, od.as<long long>(), n_tasks,
                          mu.as<double>(), is.as<double>(), w.as<double>(), err.as<int>(), st),
        "centre kernel");
  const long long ld = ((long long)mp1 + 31) / 32 * 32;
  const long long gs = (long long)mp1 * ld;
  L0_CK(g.ensure((size_t)n_tasks * gs * 8), "alloc");
  L0_CK(cudaMemsetAsync(g.p, 0, (size_t)n_tasks * gs * 8, st), "memset");
  std::vector<long long> off(task_offsets, task_offsets + n_tasks + 1);
  L0_CK(l0::launch_gram64(w.as<double>(), N, m, off.data(), n_tasks, g.as<double>(), ld, gs, st), "gram kernel");
  L0_CK(cudaMemcpy2DAsync(out, (size_t)mp1 * 8, g.as<double>() + (size_t)task * gs, (size_t)ld * 8,
                          (size_t)mp1 * 8, (size_t)mp1, cudaMemcpyDeviceToHost, st),
        "copy");
  int rc = wait_stream(h);
  DevBuf *bufs[] = {&xd, &yd, &od, &mu, &is, &w, &g, &err};
  for (DevBuf *b : bufs) b->release();
  return rc;
}

}  // extern "C"

// ====================================================== learned proposals ==
// The pair scorer (a 6-256-256-1 network, kernels in l0_mlp.cu) and the
// pair-restricted d = 3 search (l0_pairs.cu).

struct sisso_l0_scorer {
  int device = 0;
  int n_sm = 0;
  cudaStream_t st = nullptr;
  DevBuf params, m1, m2, w2b, w2tb, partial, grad, loss, err;
  int t = 0;   // Adam steps taken
  std::string last_error;
};

namespace {

int sfail(sisso_l0_scorer_t s, int code, const std::string &m) {
  if (s) s->last_error = m;
  return code;
}
int scuda(sisso_l0_scorer_t s, cudaError_t e, const char *where) {
  return sfail(s, (e == cudaErrorMemoryAllocation) ? SISSO_L0_ENOMEM : SISSO_L0_ECUDA,
               std::string(where) + ": " + cudaGetErrorString(e));
}
#define SC_CK(call, where)                                \
  do {                                                    \
    cudaError_t e_ = (call);                              \
    if (e_ != cudaSuccess) return scuda(s, e_, where);    \
  } while (0)

// BF16 copies of W2 / W2^T from the master weights (no step)
int scorer_refresh(sisso_l0_scorer_t s) {
  SC_CK(l0::launch_mlp_adam(s->params.as<float>(), s->m1.as<float>(), s->m2.as<float>(),
                            s->partial.as<float>(), 0, 0.f, 1, 0, nullptr, nullptr, s->w2b.p,
                            s->w2tb.p, s->st),
        "adam kernel");
  return SISSO_L0_OK;
}

int scorer_sync(sisso_l0_scorer_t s) {
  int herr = 0;
  SC_CK(cudaMemcpyAsync(&herr, s->err.p, 4, cudaMemcpyDeviceToHost, s->st), "copy");
  SC_CK(cudaStreamSynchronize(s->st), "scorer stream");
  if (herr != 0) return sfail(s, SISSO_L0_ECUDA, "device error flag " + std::to_string(herr));
  return SISSO_L0_OK;
}

// splitmix64 (Steele, Lea and Flood, 2014): the weights' initial draw
u64 splitmix64(u64 &x) {
  u64 z = (x += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

int train_rows(sisso_l0_scorer_t s, const float *feats, const float *labels, long long row0,
               long long n, float lr, int do_step, float *loss_dev) {
  const int grid = (int)((n + 127) / 128);
  SC_CK(s->partial.ensure((size_t)grid * l0::MLP_PSTRIDE * 4), "alloc partial gradients");
  l0::MlpArgs a{};
  a.params = s->params.as<float>();
  a.feats = feats;
  a.label = labels;
  a.row0 = row0;
  a.n_rows = n;
  a.partial = s->partial.as<float>();
  a.inv_B = 1.0 / (double)n;
  a.err = s->err.as<int>();
  SC_CK(l0::launch_mlp(l0::MLP_TRAIN, a, s->w2b.p, s->w2tb.p, grid, s->st), "mlp kernel");
  if (do_step) ++s->t;
  SC_CK(l0::launch_mlp_adam(s->params.as<float>(), s->m1.as<float>(), s->m2.as<float>(),
                            s->partial.as<float>(), grid, lr, std::max(1, s->t), do_step,
                            s->grad.as<float>(), loss_dev, s->w2b.p, s->w2tb.p, s->st),
        "adam kernel");
  return SISSO_L0_OK;
}

// single-task inputs for the learned forms
int check_single(sisso_l0_t h, const double *X, const double *y, int64_t n_total, int64_t n_sis,
                 int need_m) {
  if (!X || !y) return fail(h, SISSO_L0_EINVAL, "null pointer argument");
  if (n_sis < need_m) return fail(h, SISSO_L0_EINVAL, "n_sis too small");
  if (n_total < 5) return fail(h, SISSO_L0_EINVAL, "n_total must be >= 5 (d + 2)");
  if (n_sis > 65535) return fail(h, SISSO_L0_EUNSUPPORTED, "n_sis above 65535 for pair ranks");
  return SISSO_L0_OK;
}

template <typename F>
int guarded(sisso_l0_t h, F f) {
  if (!h) return SISSO_L0_EINVAL;
  try {
    cudaError_t e = cudaSetDevice(h->opt.device);
    if (e != cudaSuccess) return cuda_fail(h, e, "set device");
    return f();
  } catch (const std::bad_alloc &) {
    return fail(h, SISSO_L0_ENOMEM, "host allocation failed");
  } catch (...) {
    return fail(h, SISSO_L0_ECUDA, "unexpected host exception");
  }
}

}  // namespace

extern "C" {

int sisso_l0_scorer_create(sisso_l0_scorer_t *out, int32_t device, uint64_t seed) {
  if (!out) return SISSO_L0_EINVAL;
  *out = nullptr;
  sisso_l0_scorer *s = new (std::nothrow) sisso_l0_scorer();
  if (!s) return SISSO_L0_ENOMEM;
  s->device = device;
  cudaError_t e = cudaSetDevice(device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&s->n_sm, cudaDevAttrMultiProcessorCount, device);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->st, cudaStreamNonBlocking);
  const size_t pb = (size_t)l0::MLP_N_PARAMS * 4;
  if (e == cudaSuccess) e = s->params.ensure(pb);
  if (e == cudaSuccess) e = s->m1.ensure(pb);
  if (e == cudaSuccess) e = s->m2.ensure(pb);
  if (e == cudaSuccess) e = s->grad.ensure(pb);
  if (e == cudaSuccess) e = s->w2b.ensure((size_t)l0::MLP_NH * l0::MLP_NH * 2);
  if (e == cudaSuccess) e = s->w2tb.ensure((size_t)l0::MLP_NH * l0::MLP_NH * 2);
  if (e == cudaSuccess) e = s->partial.ensure((size_t)l0::MLP_PSTRIDE * 4);
  if (e == cudaSuccess) e = s->loss.ensure(4096 * 4);
  if (e == cudaSuccess) e = s->err.ensure(16);
  if (e != cudaSuccess) {
    sisso_l0_scorer_destroy(s);
    return (e == cudaErrorMemoryAllocation) ? SISSO_L0_ENOMEM : SISSO_L0_ECUDA;
  }
  // He-uniform weights (bound sqrt(6 / fan_in)), zero biases
  std::vector<float> w(l0::MLP_N_PARAMS, 0.f);
  u64 st = seed;
  auto uni = [&](double bound) {
    const double u = (double)(splitmix64(st) >> 11) * (1.0 / 9007199254740992.0);
    return (float)((2.0 * u - 1.0) * bound);
  };
  for (int q = 0; q < l0::MLP_NH * l0::MLP_NIN; ++q) w[l0::MLP_OFF_W1 + q] = uni(std::sqrt(6.0 / l0::MLP_NIN));
  for (int q = 0; q < l0::MLP_NH * l0::MLP_NH; ++q) w[l0::MLP_OFF_W2 + q] = uni(std::sqrt(6.0 / l0::MLP_NH));
  for (int q = 0; q < l0::MLP_NH; ++q) w[l0::MLP_OFF_W3 + q] = uni(std::sqrt(6.0 / l0::MLP_NH));
  int rc = sisso_l0_scorer_set_params(s, w.data(), l0::MLP_N_PARAMS);
  if (rc) {
    sisso_l0_scorer_destroy(s);
    return rc;
  }
  *out = s;
  return SISSO_L0_OK;
}

void sisso_l0_scorer_destroy(sisso_l0_scorer_t s) {
  if (!s) return;
  cudaSetDevice(s->device);
  if (s->st) cudaStreamSynchronize(s->st);
  DevBuf *bufs[] = {&s->params, &s->m1, &s->m2, &s->w2b, &s->w2tb, &s->partial, &s->grad,
                    &s->loss, &s->err};
  for (DevBuf *b : bufs) b->release();
  if (s->st) cudaStreamDestroy(s->st);
  delete s;
}

const char *sisso_l0_scorer_last_error(sisso_l0_scorer_t s) {
  return s ? s->last_error.c_str() : kNullHandleMsg;
}

int sisso_l0_scorer_set_params(sisso_l0_scorer_t s, const float *params, int64_t n) {
  if (!s || !params) return SISSO_L0_EINVAL;
  if (n != l0::MLP_N_PARAMS) return sfail(s, SISSO_L0_EINVAL, "parameter count");
  SC_CK(cudaSetDevice(s->device), "set device");
  SC_CK(cudaMemcpyAsync(s->params.p, params, (size_t)n * 4, cudaMemcpyDefault, s->st), "copy");
  SC_CK(cudaMemsetAsync(s->m1.p, 0, (size_t)n * 4, s->st), "memset");
  SC_CK(cudaMemsetAsync(s->m2.p, 0, (size_t)n * 4, s->st), "memset");
  SC_CK(cudaMemsetAsync(s->err.p, 0, 16, s->st), "memset");
  s->t = 0;
  int rc = scorer_refresh(s);
  if (rc) return rc;
  return scorer_sync(s);
}

int sisso_l0_scorer_get_params(sisso_l0_scorer_t s, float *params, int64_t n) {
  if (!s || !params) return SISSO_L0_EINVAL;
  if (n != l0::MLP_N_PARAMS) return sfail(s, SISSO_L0_EINVAL, "parameter count");
  SC_CK(cudaSetDevice(s->device), "set device");
  SC_CK(cudaMemcpyAsync(params, s->params.p, (size_t)n * 4, cudaMemcpyDefault, s->st), "copy");
  return scorer_sync(s);
}

int sisso_l0_scorer_loss_grad(sisso_l0_scorer_t s, const float *feats, const float *labels,
                              int64_t n_rows, float *loss, float *grad) {
  if (!s || !feats || !labels || n_rows < 1) return SISSO_L0_EINVAL;
  if (!is_device_ptr(feats) || !is_device_ptr(labels))
    return sfail(s, SISSO_L0_EINVAL, "features and labels must be device pointers");
  SC_CK(cudaSetDevice(s->device), "set device");
  SC_CK(cudaMemsetAsync(s->err.p, 0, 16, s->st), "memset");
  int rc = train_rows(s, feats, labels, 0, n_rows, 0.f, 0, s->loss.as<float>());
  if (rc) return rc;
  if (loss) SC_CK(cudaMemcpyAsync(loss, s->loss.p, 4, cudaMemcpyDefault, s->st), "copy");
  if (grad)
    SC_CK(cudaMemcpyAsync(grad, s->grad.p, (size_t)l0::MLP_N_PARAMS * 4, cudaMemcpyDefault, s->st),
          "copy");
  return scorer_sync(s);
}

int sisso_l0_scorer_train(sisso_l0_scorer_t s, const float *feats, const float *labels,
                          int64_t n_rows, int32_t batch_rows, int32_t steps, float lr,
                          float *losses) {
  if (!s || !feats || !labels || n_rows < 1 || batch_rows < 1 || steps < 0 || !(lr >= 0.f))
    return SISSO_L0_EINVAL;
  if (!is_device_ptr(feats) || !is_device_ptr(labels))
    return sfail(s, SISSO_L0_EINVAL, "features and labels must be device pointers");
  SC_CK(cudaSetDevice(s->device), "set device");
  SC_CK(cudaMemsetAsync(s->err.p, 0, 16, s->st), "memset");
  SC_CK(s->loss.ensure((size_t)std::max(1, steps) * 4), "alloc");
  long long row0 = 0;
  for (int q = 0; q < steps; ++q) {
    if (row0 >= n_rows) row0 = 0;
    const long long n = std::min<long long>(batch_rows, n_rows - row0);
    int rc = train_rows(s, feats, labels, row0, n, lr, 1, s->loss.as<float>() + q);
    if (rc) return rc;
    row0 += n;
  }
  if (losses && steps > 0)
    SC_CK(cudaMemcpyAsync(losses, s->loss.p, (size_t)steps * 4, cudaMemcpyDefault, s->st), "copy");
  return scorer_sync(s);
}

int sisso_l0_scorer_predict(sisso_l0_scorer_t s, const float *feats, int64_t n_rows, float *out) {
  if (!s || !feats || !out || n_rows < 1) return SISSO_L0_EINVAL;
  if (!is_device_ptr(feats) || !is_device_ptr(out))
    return sfail(s, SISSO_L0_EINVAL, "features and output must be device pointers");
  SC_CK(cudaSetDevice(s->device), "set device");
  SC_CK(cudaMemsetAsync(s->err.p, 0, 16, s->st), "memset");
  l0::MlpArgs a{};
  a.params = s->params.as<float>();
  a.feats = feats;
  a.n_rows = n_rows;
  a.out = out;
  a.err = s->err.as<int>();
  const int grid = (int)std::min<long long>((n_rows + 127) / 128, s->n_sm);
  SC_CK(l0::launch_mlp(l0::MLP_INFER_FEATS, a, s->w2b.p, s->w2tb.p, grid, s->st), "mlp kernel");
  return scorer_sync(s);
}

int sisso_l0_pair_data(sisso_l0_t h, const double *X, const double *y, int64_t n_total,
                       int64_t n_sis, float *feats, float *labels, int32_t standardize) {
  return guarded(h, [&]() -> int {
    int rc = check_single(h, X, y, n_total, n_sis, 3);
    if (rc) return rc;
    if (!feats) return fail(h, SISSO_L0_EINVAL, "null output pointer");
    if (h->opt.precision != SISSO_L0_MIXED_BF16X3)
      return fail(h, SISSO_L0_EUNSUPPORTED, "pair data come from the FP32 (mixed-precision) Gram");
    if (!is_device_ptr(feats) || (labels && !is_device_ptr(labels)))
      return fail(h, SISSO_L0_EINVAL, "outputs must be device pointers");
    const int64_t off[2] = {0, n_total};
    int32_t dt[2];
    double dr;
    sisso_l0_request r{2, 1, dt, &dr};
    Special sp;
    sp.prep_only = 1;
    sp.after_prep = [&](sisso_l0_t hh, FitPlan &P) -> int {
      sisso_l0_t h = hh;
      const long long np = (long long)P.m * (P.m - 1) / 2;
      L0_CK(l0::launch_pair_features(h->gram32.as<float>(), P.ld, 0, np, feats, h->st),
            "pair features kernel");
      if (labels)
        L0_CK(l0::launch_pair_best(h->gram32.as<float>(), P.ld, h->diag.as<float>(), P.m, np,
                                   h->opt.fp32_fallback_pivot_ratio, 1e-12f, labels, h->st),
              "pair label kernel");
      if (labels && standardize) {
        L0_CK(h->sel_bin.ensure(16), "alloc");
        L0_CK(l0::launch_label_standardize(labels, np, h->sel_bin.as<double>(), h->st),
              "label kernel");
      }
      return SISSO_L0_OK;
    };
    return fit_requests(h, X, y, off, 1, n_sis, &r, 1, &sp);
  });
}

int sisso_l0_fit_pairs(sisso_l0_t h, const double *X, const double *y, int64_t n_total,
                       int64_t n_sis, const int32_t *pairs, int64_t n_pairs, int32_t k,
                       int32_t *out_tuples, double *out_rmse) {
  return guarded(h, [&]() -> int {
    int rc = check_single(h, X, y, n_total, n_sis, 3);
    if (rc) return rc;
    if (!pairs || n_pairs < 1) return fail(h, SISSO_L0_EINVAL, "empty pair list");
    if (h->opt.task_mode != SISSO_L0_PER_TASK)
      return fail(h, SISSO_L0_EUNSUPPORTED, "pair-restricted search is single-task");
    const int64_t off[2] = {0, n_total};
    sisso_l0_request r{3, k, out_tuples, out_rmse};
    Special sp;
    sp.proposal = 1;
    sp.after_prep = [&](sisso_l0_t hh, FitPlan &P) -> int {
      sisso_l0_t h = hh;
      const long long np = (long long)P.m * (P.m - 1) / 2;
      L0_CK(h->prop_pairs.ensure((size_t)n_pairs * 8), "alloc pairs");
      L0_CK(h->prop_bits.ensure((size_t)((np + 31) / 32) * 4), "alloc pair bitmap");
      L0_CK(h->prop_ctr.ensure(32), "alloc");
      const int *src = pairs;
      if (!is_device_ptr(pairs)) {
        L0_CK(h->prop_in.ensure((size_t)n_pairs * 8), "alloc pairs");
        L0_CK(cudaMemcpyAsync(h->prop_in.p, pairs, (size_t)n_pairs * 8, cudaMemcpyHostToDevice,
                              h->st), "copy pairs");
        src = h->prop_in.as<int>();
      }
      L0_CK(l0::launch_pairs_from_list(src, n_pairs, P.m, h->prop_pairs.as<int>(),
                                       h->prop_bits.as<unsigned>(), h->err.as<int>(), h->st),
            "pair list kernel");
      P.n_pairs = n_pairs;
      return SISSO_L0_OK;
    };
    return fit_requests(h, X, y, off, 1, n_sis, &r, 1, &sp);
  });
}

int sisso_l0_fit_learned(sisso_l0_t h, sisso_l0_scorer_t s, const double *X, const double *y,
                         int64_t n_total, int64_t n_sis, int32_t k, double fraction,
                         int32_t *out_tuples, double *out_rmse) {
  return guarded(h, [&]() -> int {
    int rc = check_single(h, X, y, n_total, n_sis, 3);
    if (rc) return rc;
    if (!s) return fail(h, SISSO_L0_EINVAL, "null scorer");
    if (s->device != h->opt.device) return fail(h, SISSO_L0_EINVAL, "scorer on another device");
    if (!(fraction > 0.0) || fraction > 1.0) return fail(h, SISSO_L0_EINVAL, "fraction in (0, 1]");
    if (h->opt.precision != SISSO_L0_MIXED_BF16X3)
      return fail(h, SISSO_L0_EUNSUPPORTED, "the scorer reads the FP32 (mixed-precision) Gram");
    if (h->opt.task_mode != SISSO_L0_PER_TASK)
      return fail(h, SISSO_L0_EUNSUPPORTED, "learned search is single-task");
    L0_CK(cudaStreamSynchronize(s->st), "scorer stream");
    const int64_t off[2] = {0, n_total};
    sisso_l0_request r{3, k, out_tuples, out_rmse};
    Special sp;
    sp.proposal = 1;
    sp.after_prep = [&](sisso_l0_t hh, FitPlan &P) -> int {
      sisso_l0_t h = hh;
      cudaStream_t st = h->st;
      const long long np = (long long)P.m * (P.m - 1) / 2;
      L0_CK(h->scores.ensure((size_t)np * 4), "alloc scores");
      L0_CK(h->prop_pairs.ensure((size_t)np * 8), "alloc pairs");
      L0_CK(h->prop_bits.ensure((size_t)((np + 31) / 32) * 4), "alloc pair bitmap");
      L0_CK(h->prop_ctr.ensure(32), "alloc");
      L0_CK(h->sel_hist.ensure((size_t)4 << 20), "alloc");
      L0_CK(h->sel_bin.ensure(16), "alloc");
      l0::MlpArgs a{};
      a.params = s->params.as<float>();
      a.row0 = 0;
      a.n_rows = np;
      a.G = h->gram32.as<float>();
      a.ld = P.ld;
      a.out = h->scores.as<float>();
      a.err = h->err.as<int>();
      const int grid = (int)std::min<long long>((np + 127) / 128, h->n_sm);
      L0_CK(l0::launch_mlp(l0::MLP_INFER_GRAM, a, s->w2b.p, s->w2tb.p, grid, st), "mlp kernel");
      const long long want = std::max<long long>(1, (long long)std::ceil(fraction * (double)np));
      L0_CK(l0::launch_select_pairs(h->scores.as<float>(), np, want, h->sel_hist.as<unsigned>(),
                                    h->sel_bin.as<unsigned>(), h->prop_pairs.as<int>(),
                                    h->prop_ctr.as<unsigned long long>() + 2,
                                    h->prop_bits.as<unsigned>(), st),
            "pair selection");
      u64 cnt = 0;
      L0_CK(cudaMemcpyAsync(&cnt, h->prop_ctr.as<u64>() + 2, 8, cudaMemcpyDeviceToHost, st), "copy");
      int rc2 = wait_stream(h);
      if (rc2) return rc2;
      P.n_pairs = (long long)cnt;
      return SISSO_L0_OK;
    };
    return fit_requests(h, X, y, off, 1, n_sis, &r, 1, &sp);
  });
}

}  // extern "C"

// ============================================================== sharding ==
// One search split over shards (one per GPU): shard s of n takes every n-th
// work item (a prefix chunk of one (j, k) tile), so each shard searches a
// disjoint slice of the tuples; its FP64 re-fitted candidate pool is the only
// thing exchanged, and the merge ranks the union (cf. the paper's final
// gather of the selected models, Sec. 3.2.1).
extern "C" {

int sisso_l0_fit_shard(sisso_l0_t h, const double *X, const double *y, int64_t n_total,
                       int64_t n_sis, int32_t n_dim, int32_t k, int32_t shard, int32_t n_shards,
                       uint64_t *out_keys, double *out_sse, int32_t *out_count,
                       double *out_bound, double *out_delta) {
  return guarded(h, [&]() -> int {
    if (!X || !y || !out_keys || !out_sse || !out_count || !out_bound || !out_delta)
      return fail(h, SISSO_L0_EINVAL, "null pointer argument");
    if (n_shards < 1 || shard < 0 || shard >= n_shards)
      return fail(h, SISSO_L0_EINVAL, "shard must be in [0, n_shards)");
    if (n_dim < 2) return fail(h, SISSO_L0_EINVAL, "sharded searches take n_dim >= 2");
    if (h->opt.task_mode != SISSO_L0_PER_TASK)
      return fail(h, SISSO_L0_EUNSUPPORTED, "sharded searches are single-task");
    const int64_t off[2] = {0, n_total};
    std::vector<int32_t> tt((size_t)std::max(1, k) * std::max(1, n_dim));
    std::vector<double> tr((size_t)std::max(1, k));
    sisso_l0_request r{n_dim, k, tt.data(), tr.data()};
    Special sp;
    sp.shard = shard;
    sp.n_shards = n_shards;
    sp.exports_pool = 1;
    int rc = fit_requests(h, X, y, off, 1, n_sis, &r, 1, &sp);
    if (rc) return rc;
    const int K = h->stats.candidate_pool;
    int cnt = 0;
    l0::CertOut c;
    L0_CK(cudaMemcpyAsync(&cnt, h->pool_cnt.p, 4, cudaMemcpyDeviceToHost, h->st), "copy");
    L0_CK(cudaMemcpyAsync(&c, h->cert.p, sizeof(c), cudaMemcpyDeviceToHost, h->st), "copy");
    L0_CK(cudaMemcpyAsync(out_keys, h->pool_k.p, (size_t)K * 8, cudaMemcpyDefault, h->st), "copy");
    L0_CK(cudaMemcpyAsync(out_sse, h->refit.p, (size_t)K * 8, cudaMemcpyDefault, h->st), "copy");
    rc = wait_stream(h);
    if (rc) return rc;
    *out_count = cnt;
    *out_bound = c.pool_worst;
    *out_delta = c.delta;
    return SISSO_L0_OK;
  });
}

int sisso_l0_merge_shards(sisso_l0_t h, int64_t n_sis, int32_t n_dim, int32_t k, int64_t n_total,
                          const uint64_t *keys, const double *sse, int64_t n_cand,
                          const double *bounds, const double *deltas, int32_t n_shards,
                          int32_t *out_tuples, double *out_rmse, int32_t *certified) {
  return guarded(h, [&]() -> int {
    if (!keys || !sse || !bounds || !deltas || !out_tuples || !out_rmse || !certified)
      return fail(h, SISSO_L0_EINVAL, "null pointer argument");
    if (n_dim < 1 || n_dim > SISSO_L0_MAX_DIM || k < 1 || n_cand < 0 || n_shards < 1 ||
        n_total < 1 || n_sis < n_dim)
      return fail(h, SISSO_L0_EINVAL, "bad arguments");
    if (n_cand > (1LL << 20)) return fail(h, SISSO_L0_EUNSUPPORTED, "more than 2^20 candidates");
    const u64 total = binom_host(n_sis, n_dim);
    if (total >= kSat) return fail(h, SISSO_L0_EUNSUPPORTED, "C(n_sis, n_dim) too large");
    cudaStream_t st = h->st;
    int rc = ensure_binom(h, (int)n_sis);
    if (rc) return rc;
    long long P = 1;
    while (P < n_cand || P < k) P <<= 1;
    const size_t in_bytes = (size_t)std::max<int64_t>(n_cand, 1) * 16 + (size_t)n_shards * 16;
    L0_CK(h->prop_in.ensure(in_bytes), "alloc");
    L0_CK(h->scores.ensure((size_t)P * 16), "alloc");
    L0_CK(h->out_t.ensure((size_t)k * n_dim * 4), "alloc");
    L0_CK(h->out_r.ensure((size_t)k * 8 + 16), "alloc");
    unsigned char *in = (unsigned char *)h->prop_in.p;
    u64 *dk = (u64 *)in;
    double *ds = (double *)(in + (size_t)std::max<int64_t>(n_cand, 1) * 8);
    double *db = ds + std::max<int64_t>(n_cand, 1);
    double *dd = db + n_shards;
    if (n_cand > 0) {
      L0_CK(cudaMemcpyAsync(dk, keys, (size_t)n_cand * 8, cudaMemcpyDefault, st), "copy");
      L0_CK(cudaMemcpyAsync(ds, sse, (size_t)n_cand * 8, cudaMemcpyDefault, st), "copy");
    }
    L0_CK(cudaMemcpyAsync(db, bounds, (size_t)n_shards * 8, cudaMemcpyDefault, st), "copy");
    L0_CK(cudaMemcpyAsync(dd, deltas, (size_t)n_shards * 8, cudaMemcpyDefault, st), "copy");
    double *ss = h->scores.as<double>();
    u64 *sk = (u64 *)(ss + P);
    int *dcert = (int *)(h->out_r.as<double>() + k);
    l0::Binom B{h->binom.as<u64>(), (int)n_sis + 1};
    L0_CK(l0::launch_merge_shards(B, (int)n_sis, n_dim, total, k, (double)n_total, dk, ds, n_cand,
                                  db, dd, n_shards, ss, sk, h->out_t.as<int>(),
                                  h->out_r.as<double>(), dcert, st),
          "merge kernel");
    L0_CK(cudaMemcpyAsync(out_tuples, h->out_t.p, (size_t)k * n_dim * 4, cudaMemcpyDefault, st),
          "copy");
    L0_CK(cudaMemcpyAsync(out_rmse, h->out_r.p, (size_t)k * 8, cudaMemcpyDefault, st), "copy");
    L0_CK(cudaMemcpyAsync(certified, dcert, 4, cudaMemcpyDefault, st), "copy");
    return wait_stream(h);
  });
}

}  // extern "C"

// ============================================================ screening ==
namespace {

// Screening against R targets [R][n_total] (host or device), never selecting
// the n_ex features in ex (host or device int32).
int sis_impl(sisso_l0_t h, const double *X, const double *Y, int R, int64_t n_total,
             int64_t n_feat, int32_t m, const int32_t *ex, int64_t n_ex, int32_t *out_idx,
             double *out_r) {
  if (!X || !Y || !out_idx || !out_r || (n_ex > 0 && !ex))
    return fail(h, SISSO_L0_EINVAL, "null pointer argument");
  if (R < 1 || R > l0::SIS_MAX_TARGETS)
    return fail(h, SISSO_L0_EINVAL, "n_targets outside [1, 16]");
  if (n_total < 2 || n_feat < 1 || m < 1 || n_ex < 0 || m > n_feat - n_ex)
    return fail(h, SISSO_L0_EINVAL, "need n_total >= 2 and 1 <= m <= n_feat - n_exclude");
  if (m > 65536 || n_feat >= (1ll << 32))
    return fail(h, SISSO_L0_EUNSUPPORTED, "m above 65536 or n_feat above 2^32");
  cudaStream_t st = h->st;
  const double *Xd = X, *Yd = Y;
  if (!is_device_ptr(X)) {
    const size_t xb = (size_t)n_feat * (size_t)n_total * 8;
    L0_CK(h->xin.ensure(xb), "alloc X");
    L0_CK(cudaMemcpyAsync(h->xin.p, X, xb, cudaMemcpyHostToDevice, st), "copy X");
    Xd = h->xin.as<double>();
  }
  if (!is_device_ptr(Y)) {
    L0_CK(h->sis_y.ensure((size_t)R * n_total * 8), "alloc targets");
    L0_CK(cudaMemcpyAsync(h->sis_y.p, Y, (size_t)R * n_total * 8, cudaMemcpyHostToDevice, st),
          "copy targets");
    Yd = h->sis_y.as<double>();
  }
  const int *exd = nullptr;
  if (n_ex > 0) {
    // distinct, in range (the device marks each listed feature)
    std::vector<int32_t> hx((size_t)n_ex);
    if (is_device_ptr(ex)) {
      L0_CK(cudaMemcpyAsync(hx.data(), ex, (size_t)n_ex * 4, cudaMemcpyDeviceToHost, st), "copy");
      L0_CK(cudaStreamSynchronize(st), "sync");
    } else {
      std::copy(ex, ex + n_ex, hx.begin());
    }
    std::sort(hx.begin(), hx.end());
    for (size_t i = 0; i < hx.size(); ++i)
      if (hx[i] < 0 || hx[i] >= n_feat || (i && hx[i] == hx[i - 1]))
        return fail(h, SISSO_L0_EINVAL, "exclusions must be distinct indices in [0, n_feat)");
    L0_CK(h->sis_ex.ensure((size_t)n_ex * 4), "alloc exclusions");
    L0_CK(cudaMemcpyAsync(h->sis_ex.p, hx.data(), (size_t)n_ex * 4, cudaMemcpyHostToDevice, st),
          "copy exclusions");
    L0_CK(cudaStreamSynchronize(st), "sync");   // hx leaves scope
    exd = h->sis_ex.as<int>();
  }
  L0_CK(h->scores.ensure(l0::sis_scratch_bytes(n_feat, m, n_total, R)), "alloc screening scratch");
  L0_CK(h->out_t.ensure((size_t)m * 4), "alloc");
  L0_CK(h->out_r.ensure((size_t)m * 8), "alloc");
  L0_CK(h->err.ensure(16), "alloc");
  L0_CK(cudaMemsetAsync(h->err.p, 0, 16, st), "memset");
  const bool pre = h->opt.precision == SISSO_L0_MIXED_BF16X3;
  L0_CK(cudaEventRecord(h->ev[0], st), "event");
  L0_CK(l0::launch_sis(Xd, Yd, R, n_total, n_feat, m, exd, n_ex, pre ? 1 : 0, h->scores.p,
                       h->out_t.as<int>(), h->out_r.as<double>(), h->err.as<int>(), st,
                       h->ev_k[0], h->ev_k[1]),
        "screening kernels");
  L0_CK(cudaEventRecord(h->ev[1], st), "event");
  L0_CK(cudaMemcpyAsync(out_idx, h->out_t.p, (size_t)m * 4, cudaMemcpyDefault, st), "copy");
  L0_CK(cudaMemcpyAsync(out_r, h->out_r.p, (size_t)m * 8, cudaMemcpyDefault, st), "copy");
  int herr = 0;
  unsigned long long rescored = 0;
  L0_CK(cudaMemcpyAsync(&herr, h->err.p, 4, cudaMemcpyDeviceToHost, st), "copy");
  L0_CK(cudaMemcpyAsync(&rescored, (char *)h->scores.p + 40, 8, cudaMemcpyDeviceToHost, st),
        "copy");
  int rc = wait_stream(h);
  if (rc) return rc;
  sisso_l0_stats &S = h->stats;
  S = sisso_l0_stats{};
  S.struct_size = (int32_t)sizeof(sisso_l0_stats);
  S.certified = 1;
  S.fp64_fallback_tuples = pre ? rescored : (uint64_t)n_feat;
  S.kernel_launches = (pre ? 19 + R : 13) + (n_ex > 0 ? 1 : 0);
  float ms = 0.f;
  if (cudaEventElapsedTime(&ms, h->ev[0], h->ev[1]) != cudaSuccess) {
    cudaGetLastError();
    ms = 0.f;
  }
  S.ms_total = ms;
  if (cudaEventElapsedTime(&ms, h->ev_k[0], h->ev_k[1]) != cudaSuccess) {
    cudaGetLastError();
    ms = 0.f;
  }
  S.ms_tuple_kernel = ms;
  if (herr == 5) return fail(h, SISSO_L0_ENONFINITE, "NaN or Inf in X or the targets");
  if (herr == 12) return fail(h, SISSO_L0_EUNSUPPORTED, "more than 2^22 features tie at the cut");
  if (herr) return fail(h, SISSO_L0_ECUDA, "device error flag " + std::to_string(herr));
  return SISSO_L0_OK;
}

}  // namespace

extern "C" int sisso_l0_sis(sisso_l0_t h, const double *X, const double *y, int64_t n_total,
                            int64_t n_feat, int32_t m, int32_t *out_idx, double *out_r) {
  return guarded(h, [&]() -> int {
    return sis_impl(h, X, y, 1, n_total, n_feat, m, nullptr, 0, out_idx, out_r);
  });
}

extern "C" int sisso_l0_sis_multi(sisso_l0_t h, const double *X, const double *Y,
                                  int32_t n_targets, int64_t n_total, int64_t n_feat, int32_t m,
                                  const int32_t *exclude, int64_t n_exclude, int32_t *out_idx,
                                  double *out_r) {
  return guarded(h, [&]() -> int {
    return sis_impl(h, X, Y, n_targets, n_total, n_feat, m, exclude, n_exclude, out_idx, out_r);
  });
}

extern "C" int sisso_l0_sis_generated(sisso_l0_t h, const double *C, int64_t n_child,
                                      int64_t n_total, const int32_t *ops, const int32_t *c1,
                                      const int32_t *c2, int64_t n_cand, const double *y,
                                      int32_t m, double l_bound, double u_bound,
                                      int32_t *out_idx, double *out_r, uint8_t *out_valid) {
  return guarded(h, [&]() -> int {
    if (!C || !ops || !c1 || !c2 || !y || !out_idx || !out_r)
      return fail(h, SISSO_L0_EINVAL, "null pointer argument");
    if (n_total < 2 || n_child < 1 || n_cand < 1 || m < 1 || m > n_cand)
      return fail(h, SISSO_L0_EINVAL, "need n_total >= 2, n_child >= 1, 1 <= m <= n_cand");
    if (!(l_bound >= 0.0) || !(u_bound >= l_bound))
      return fail(h, SISSO_L0_EINVAL, "need 0 <= l_bound <= u_bound");
    if (m > 65536 || n_cand >= (1ll << 32))
      return fail(h, SISSO_L0_EUNSUPPORTED, "m above 65536 or n_cand above 2^32");
    cudaStream_t st = h->st;
    const double *Cd = C, *yd = y;
    if (!is_device_ptr(C)) {
      const size_t cb = (size_t)n_child * (size_t)n_total * 8;
      L0_CK(h->xin.ensure(cb), "alloc children");
      L0_CK(cudaMemcpyAsync(h->xin.p, C, cb, cudaMemcpyHostToDevice, st), "copy children");
      Cd = h->xin.as<double>();
    }
    if (!is_device_ptr(y)) {
      L0_CK(h->sis_y.ensure((size_t)n_total * 8), "alloc y");
      L0_CK(cudaMemcpyAsync(h->sis_y.p, y, (size_t)n_total * 8, cudaMemcpyHostToDevice, st),
            "copy y");
      yd = h->sis_y.as<double>();
    }
    auto dev_ints = [&](const int32_t *a, DevBuf &b) -> const int * {
      if (is_device_ptr(a)) return (const int *)a;
      if (b.ensure((size_t)n_cand * 4) != cudaSuccess) return nullptr;
      if (cudaMemcpyAsync(b.p, a, (size_t)n_cand * 4, cudaMemcpyHostToDevice, st) != cudaSuccess)
        return nullptr;
      return b.as<int>();
    };
    l0::SisGen g;
    g.n_child = n_child;
    g.ops = dev_ints(ops, h->gen_ops);
    g.c1 = dev_ints(c1, h->gen_c1);
    g.c2 = dev_ints(c2, h->gen_c2);
    if (!g.ops || !g.c1 || !g.c2) return fail(h, SISSO_L0_ENOMEM, "candidate lists");
    g.lb = l_bound;
    g.ub = u_bound;
    g.valid = nullptr;
    if (out_valid) {
      if (is_device_ptr(out_valid)) {
        g.valid = out_valid;
      } else {
        L0_CK(h->gen_valid.ensure((size_t)n_cand), "alloc");
        g.valid = (unsigned char *)h->gen_valid.p;
      }
    }
    // a mixed-precision handle screens in FP32 first when no per-candidate
    // validity is asked for (validity needs every candidate in FP64)
    const int pre = (h->opt.precision != SISSO_L0_FP64 && !out_valid) ? 1 : 0;
    if (pre) {
      L0_CK(h->gen_cf.ensure((size_t)n_child * (size_t)n_total * 4), "alloc FP32 children");
      L0_CK(h->gen_csafe.ensure((size_t)n_child), "alloc");
      g.cf = h->gen_cf.as<float>();
      g.csafe = (unsigned char *)h->gen_csafe.p;
    }
    L0_CK(h->scores.ensure(l0::sis_scratch_bytes(n_cand, m, n_total, 1)), "alloc screening scratch");
    L0_CK(h->out_t.ensure((size_t)m * 4), "alloc");
    L0_CK(h->out_r.ensure((size_t)m * 8), "alloc");
    L0_CK(h->err.ensure(16), "alloc");
    L0_CK(cudaMemsetAsync(h->err.p, 0, 16, st), "memset");
    L0_CK(cudaEventRecord(h->ev[0], st), "event");
    L0_CK(l0::launch_sis(Cd, yd, 1, n_total, n_cand, m, nullptr, 0, pre, h->scores.p,
                         h->out_t.as<int>(), h->out_r.as<double>(), h->err.as<int>(), st,
                         h->ev_k[0], h->ev_k[1], &g),
          "generated screening kernels");
    L0_CK(cudaEventRecord(h->ev[1], st), "event");
    L0_CK(cudaMemcpyAsync(out_idx, h->out_t.p, (size_t)m * 4, cudaMemcpyDefault, st), "copy");
    L0_CK(cudaMemcpyAsync(out_r, h->out_r.p, (size_t)m * 8, cudaMemcpyDefault, st), "copy");
    if (out_valid && (void *)g.valid != (void *)out_valid)
      L0_CK(cudaMemcpyAsync(out_valid, g.valid, (size_t)n_cand, cudaMemcpyDeviceToHost, st),
            "copy validity");
    int herr = 0;
    L0_CK(cudaMemcpyAsync(&herr, h->err.p, 4, cudaMemcpyDeviceToHost, st), "copy");
    int rc = wait_stream(h);
    if (rc) return rc;
    sisso_l0_stats &S = h->stats;
    S = sisso_l0_stats{};
    S.struct_size = (int32_t)sizeof(sisso_l0_stats);
    S.certified = 1;
    S.fp64_fallback_tuples = pre ? 0 : (uint64_t)n_cand;
    S.kernel_launches = pre ? 19 : 13;
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, h->ev[0], h->ev[1]) != cudaSuccess) {
      cudaGetLastError();
      ms = 0.f;
    }
    S.ms_total = ms;
    if (cudaEventElapsedTime(&ms, h->ev_k[0], h->ev_k[1]) != cudaSuccess) {
      cudaGetLastError();
      ms = 0.f;
    }
    S.ms_tuple_kernel = ms;
    if (herr == 14) return fail(h, SISSO_L0_EINVAL, "operator code or child index out of range");
    if (herr == 5) return fail(h, SISSO_L0_ENONFINITE, "NaN or Inf in y");
    if (herr == 12) return fail(h, SISSO_L0_EUNSUPPORTED, "more than 2^22 candidates tie at the cut");
    if (herr) return fail(h, SISSO_L0_ECUDA, "device error flag " + std::to_string(herr));
    return SISSO_L0_OK;
  });
}

extern "C" int sisso_l0_residuals(sisso_l0_t h, const double *X, const double *y,
                                  int64_t n_total, int64_t n_feat, const int32_t *tuples,
                                  int32_t n_dim, int32_t n_models, double *out) {
  return guarded(h, [&]() -> int {
    if (!X || !y || !tuples || !out) return fail(h, SISSO_L0_EINVAL, "null pointer argument");
    if (n_total < 2 || n_feat < 1 || n_dim < 1 || n_dim > 8 || n_models < 1)
      return fail(h, SISSO_L0_EINVAL, "need n_total >= 2, 1 <= n_dim <= 8, n_models >= 1");
    cudaStream_t st = h->st;
    std::vector<int32_t> ht((size_t)n_models * n_dim);
    if (is_device_ptr(tuples)) {
      L0_CK(cudaMemcpyAsync(ht.data(), tuples, ht.size() * 4, cudaMemcpyDeviceToHost, st), "copy");
      L0_CK(cudaStreamSynchronize(st), "sync");
    } else {
      std::copy(tuples, tuples + ht.size(), ht.begin());
    }
    for (int32_t v : ht)
      if (v < 0 || v >= n_feat) return fail(h, SISSO_L0_EINVAL, "tuple index outside [0, n_feat)");
    const double *Xd = X, *yd = y;
    if (!is_device_ptr(X)) {
      const size_t xb = (size_t)n_feat * (size_t)n_total * 8;
      L0_CK(h->xin.ensure(xb), "alloc X");
      L0_CK(cudaMemcpyAsync(h->xin.p, X, xb, cudaMemcpyHostToDevice, st), "copy X");
      Xd = h->xin.as<double>();
    }
    if (!is_device_ptr(y)) {
      L0_CK(h->yin.ensure((size_t)n_total * 8), "alloc y");
      L0_CK(cudaMemcpyAsync(h->yin.p, y, (size_t)n_total * 8, cudaMemcpyHostToDevice, st), "copy y");
      yd = h->yin.as<double>();
    }
    L0_CK(h->loop_tup.ensure(ht.size() * 4), "alloc");
    L0_CK(cudaMemcpyAsync(h->loop_tup.p, ht.data(), ht.size() * 4, cudaMemcpyHostToDevice, st),
          "copy tuples");
    L0_CK(h->loop_q.ensure((size_t)n_models * n_dim * n_total * 8), "alloc");
    double *od = out;
    if (!is_device_ptr(out)) {
      L0_CK(h->loop_res.ensure((size_t)n_models * n_total * 8), "alloc");
      od = h->loop_res.as<double>();
    }
    L0_CK(l0::launch_residuals(Xd, yd, n_total, h->loop_tup.as<int>(), n_dim, n_models,
                               h->loop_q.as<double>(), od, st),
          "residual kernel");
    if (od != out)
      L0_CK(cudaMemcpyAsync(out, od, (size_t)n_models * n_total * 8, cudaMemcpyDeviceToHost, st),
            "copy residuals");
    return wait_stream(h);
  });
}

extern "C" int sisso_l0_dimension_loop(sisso_l0_t h, const double *X, const double *y,
                                       int64_t n_total, int64_t n_feat, int32_t m, int32_t n_dim_max,
                                       int32_t k, int32_t n_res, int32_t *out_S,
                                       int32_t *out_tuples, double *out_rmse) {
  return guarded(h, [&]() -> int {
    if (!X || !y || !out_S || !out_tuples || !out_rmse)
      return fail(h, SISSO_L0_EINVAL, "null pointer argument");
    if (is_device_ptr(out_S) || is_device_ptr(out_tuples) || is_device_ptr(out_rmse))
      return fail(h, SISSO_L0_EINVAL, "the loop's outputs are host arrays");
    if (n_dim_max < 1 || n_dim_max > 6 || m < 1 || k < 1 || n_res < 1 ||
        n_res > l0::SIS_MAX_TARGETS || (int64_t)m * n_dim_max > n_feat)
      return fail(h, SISSO_L0_EINVAL,
                  "need 1 <= n_dim_max <= 6, m, k >= 1, 1 <= n_res <= 16, m n_dim_max <= n_feat");
    if (n_total < n_dim_max + 2) return fail(h, SISSO_L0_EINVAL, "too few samples");
    cudaStream_t st = h->st;
    // X and y resident on the device for the whole loop
    const double *Xd = X, *yd = y;
    if (!is_device_ptr(X)) {
      const size_t xb = (size_t)n_feat * (size_t)n_total * 8;
      L0_CK(h->loop_x.ensure(xb), "alloc X");
      L0_CK(cudaMemcpyAsync(h->loop_x.p, X, xb, cudaMemcpyHostToDevice, st), "copy X");
      Xd = h->loop_x.as<double>();
    }
    if (!is_device_ptr(y)) {
      L0_CK(h->loop_y.ensure((size_t)n_total * 8), "alloc y");
      L0_CK(cudaMemcpyAsync(h->loop_y.p, y, (size_t)n_total * 8, cudaMemcpyHostToDevice, st),
            "copy y");
      yd = h->loop_y.as<double>();
    }
    const int D = n_dim_max;
    for (size_t i = 0; i < (size_t)D * k * D; ++i) out_tuples[i] = -1;
    for (size_t i = 0; i < (size_t)D * k; ++i) out_rmse[i] = INFINITY;
    std::vector<int32_t> S;
    std::vector<int32_t> prev;      // best models of the previous dimension, [n_prev][n - 1]
    int n_prev = 0;
    int64_t launches = 0;           // library kernels of the whole loop
    const int64_t offs[2] = {0, n_total};
    for (int n = 1; n <= D; ++n) {
      // screening: against y, then against the residuals of the best models
      std::vector<int32_t> idx(m);
      std::vector<double> rr(m);
      int rc;
      if (n == 1) {
        rc = sis_impl(h, Xd, yd, 1, n_total, n_feat, m, nullptr, 0, idx.data(), rr.data());
      } else {
        const int R = std::min(n_prev, (int)n_res);
        if (R < 1) return fail(h, SISSO_L0_EINVAL, "no eligible model to take residuals from");
        L0_CK(h->loop_tup.ensure((size_t)R * (n - 1) * 4), "alloc");
        L0_CK(cudaMemcpyAsync(h->loop_tup.p, prev.data(), (size_t)R * (n - 1) * 4,
                              cudaMemcpyHostToDevice, st),
              "copy models");
        L0_CK(h->loop_q.ensure((size_t)R * (n - 1) * n_total * 8), "alloc");
        L0_CK(h->loop_res.ensure((size_t)R * n_total * 8), "alloc");
        L0_CK(l0::launch_residuals(Xd, yd, n_total, h->loop_tup.as<int>(), n - 1, R,
                                   h->loop_q.as<double>(), h->loop_res.as<double>(), st),
              "residual kernel");
        rc = sis_impl(h, Xd, h->loop_res.as<double>(), R, n_total, n_feat, m, S.data(),
                      (int64_t)S.size(), idx.data(), rr.data());
        launches += 1;              // residual kernel
      }
      if (rc) return rc;
      launches += h->stats.kernel_launches + 1;    // screening, gather
      S.insert(S.end(), idx.begin(), idx.end());
      // the l0 search over every n-tuple of S
      L0_CK(h->loop_rows.ensure(S.size() * 4), "alloc");
      L0_CK(cudaMemcpyAsync(h->loop_rows.p, S.data(), S.size() * 4, cudaMemcpyHostToDevice, st),
            "copy S");
      L0_CK(h->loop_xs.ensure(S.size() * (size_t)n_total * 8), "alloc");
      L0_CK(l0::launch_gather_rows(Xd, n_total, h->loop_rows.as<int>(), (int)S.size(),
                                   h->loop_xs.as<double>(), st),
            "gather S");
      std::vector<int32_t> tl((size_t)k * n);
      std::vector<double> rm(k);
      sisso_l0_request req{n, k, tl.data(), rm.data()};
      rc = fit_checked(h, h->loop_xs.as<double>(), yd, offs, 1, (int64_t)S.size(), &req, 1);
      if (rc) return rc;
      launches += h->stats.kernel_launches;
      prev.clear();
      n_prev = 0;
      for (int q = 0; q < k; ++q) {
        if (tl[(size_t)q * n] < 0) break;
        std::vector<int32_t> g(n);
        for (int a = 0; a < n; ++a) g[a] = S[tl[(size_t)q * n + a]];
        std::sort(g.begin(), g.end());
        for (int a = 0; a < n; ++a) out_tuples[((size_t)(n - 1) * k + q) * D + a] = g[a];
        out_rmse[(size_t)(n - 1) * k + q] = rm[q];
        if (n_prev < n_res) {
          prev.insert(prev.end(), g.begin(), g.end());
          ++n_prev;
        }
      }
    }
    std::copy(S.begin(), S.end(), out_S);
    h->stats.kernel_launches = launches;   // the last fit's stats, launches of the whole loop
    return SISSO_L0_OK;
  });
}
