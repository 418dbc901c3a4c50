// l0_api.cu -- host orchestrator behind the C ABI of include/sisso_l0.h.
//
// One fit (paper Sec. 2.4, all n-tuples of the m SIS features):
//   1. centre and scale every column and the target per task (FP64)
//   2. augmented Gram per task (FP64 FFMA, or split-BF16 tensor cores)
//   3. persistent tuple kernel -> per-CTA top-K' lists
//   4. grid merge -> one top-K' pool per output list
//   5. FP64 Householder re-fit of the pool from the raw centred columns
//   6. final ranking; certificate: the pool must provably contain the exact
//      top k, otherwise K' is doubled and steps 3-6 rerun.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "../../include/sisso_l0.h"
#include "l0_kernels.cuh"

using l0::u64;

namespace {

struct DevBuf {
  void *p = nullptr;
  size_t n = 0;
  cudaError_t ensure(size_t bytes) {
    if (bytes <= n && p) return cudaSuccess;
    if (p) cudaFree(p);
    p = nullptr;
    n = 0;
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
  cudaStream_t st = nullptr;
  int n_sm = 0;
  std::string last_error;
  sisso_l0_stats stats;
  // workspace
  DevBuf xin, yin, offs, mu, inv_s, w64, gram, binom;
  DevBuf probs, rowpre, ctr, gthr, lists_s, lists_k, lists_cnt;
  DevBuf part_s, part_k, part_cnt, done, pool_s, pool_k, pool_cnt;
  DevBuf scratch, refit, rdiv, cert, out_t, out_r, err;
  DevBuf dfr_key, dfr_len, dfr_n, dfr_cnt;
  DevBuf abf, bbf, kmeta, gram32;
  int binom_m = -1;
  cudaEvent_t ev[8] = {nullptr};
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

int wait_stream(sisso_l0_t h) {
  cudaEvent_t e = h->ev[7];
  L0_CK(cudaEventRecord(e, h->st), "event record");
  const double tmo = h->opt.timeout_seconds;
  auto t0 = std::chrono::steady_clock::now();
  for (;;) {
    cudaError_t q = cudaEventQuery(e);
    if (q == cudaSuccess) break;
    if (q != cudaErrorNotReady) return cuda_fail(h, q, "stream");
    if (tmo > 0) {
      double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
      if (el > tmo) return fail(h, SISSO_L0_ETIMEOUT, "stream did not finish within timeout_seconds");
    }
    std::this_thread::sleep_for(std::chrono::microseconds(20));
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

struct FitPlan {
  int T, m, d, k, n_out, shared, mixed;
  const double *Xd = nullptr, *yd = nullptr;   // device copies of the inputs
  long long N, nmax;
  long long ld;
  std::vector<long long> off;
  std::vector<l0::ProbDesc> pd;
  std::vector<long long> rowpre;
  int grid = 0;
  int n_slots = 0;
  long long gstride = 0;
  bool have_g64 = false;       // FP64 Gram computed (always in FP64 mode)
  unsigned long long fallback_tuples = 0;
};

constexpr int kDeferGroups = 64;
constexpr long long kDeferCap = 1LL << 24;

// choose prefix steps per work item and fill problem descriptors
void plan_items(FitPlan &P, const std::vector<u64> &binom_row, int grid_target) {
  const int TJ = l0::TILE_TJ, TK = l0::TILE_TK;
  const int n_jt = (P.m + TJ - 1) / TJ;
  const int n_kt = (P.m + TK - 1) / TK;
  const int dp = P.d - 2;
  auto np_of = [&](int bj) -> u64 {
    int jend = std::min((bj + 1) * TJ, P.m);
    return binom_host(jend - 1, dp);
  };
  int Lsel = 1;
  if (dp > 0) {
    const int cands[] = {256, 128, 64, 32, 16, 8, 4, 2, 1};
    for (int L : cands) {
      long long items = 0;
      for (int bj = 0; bj < n_jt; ++bj) items += l0::tile_row_items(bj, P.m, dp, L, n_kt, np_of(bj));
      Lsel = L;
      if (items * (long long)P.pd.size() >= 2LL * grid_target) break;
    }
  }
  (void)binom_row;
  long long item = 0;
  P.rowpre.clear();
  for (size_t q = 0; q < P.pd.size(); ++q) {
    l0::ProbDesc &d = P.pd[q];
    d.n_jt = n_jt;
    d.n_kt = n_kt;
    d.L = Lsel;
    d.prefix_off = (int)P.rowpre.size();
    d.item_begin = item;
    long long acc = 0;
    for (int bj = 0; bj < n_jt; ++bj) {
      P.rowpre.push_back(acc);
      acc += l0::tile_row_items(bj, P.m, dp, Lsel, n_kt, np_of(bj));
    }
    P.rowpre.push_back(acc);
    item += acc;
    d.item_end = item;
  }
}

template <typename R>
int run_search(sisso_l0_t h, FitPlan &P, int K, int S, const R *G, int *certified,
               double *delta_max, float *ms_tuple, float *ms_merge, float *ms_refit) {
  cudaStream_t st = h->st;
  const int n_probs = (int)P.pd.size();
  const int d = P.d;
  l0::Binom B{h->binom.as<u64>(), P.m + 1};
  // slots
  int n_slots;
  if (d == 1) {
    n_slots = std::max(1, std::min(64, (P.m + L0_THREADS - 1) / L0_THREADS));
  } else {
    n_slots = P.grid + (P.mixed ? kDeferGroups : 0);
  }
  const size_t nl = (size_t)n_probs * n_slots * K;
  L0_CK(h->lists_s.ensure(nl * sizeof(R)), "alloc lists");
  L0_CK(h->lists_k.ensure(nl * 8), "alloc lists");
  L0_CK(h->lists_cnt.ensure((size_t)n_probs * n_slots * 4), "alloc lists");
  L0_CK(cudaMemsetAsync(h->lists_cnt.p, 0, (size_t)n_probs * n_slots * 4, st), "memset");
  L0_CK(h->gthr.ensure((size_t)n_probs * 8), "alloc gthr");
  L0_CK(cudaEventRecord(h->ev[2], st), "event");
  {
    // threshold: +inf, then the K'-th best d-tuple of the M best columns
    int M = 0;
    if (d >= 2 && !P.shared) {
      const int Mcap = std::min(std::min(P.m, 64), K);
      M = Mcap;
      for (int q = d; q <= Mcap; ++q)
        if (binom_host(q, d) >= 2ull * (u64)K) { M = q; break; }
    }
    const double ratio = P.mixed ? h->opt.fp32_fallback_pivot_ratio : h->opt.rank_deficient_pivot_ratio;
    L0_CK(l0::launch_seed<R>(G, h->probs.as<l0::ProbDesc>(), n_probs, K, S, M, ratio, B,
                             h->gthr.as<u64>(), st),
          "seed kernel");
  }
  if (d == 1) {
    L0_CK(l0::launch_singles<R>(G, P.pd.data(), h->probs.as<l0::ProbDesc>(), n_probs, K, S,
                                n_slots, h->gthr.as<u64>(), h->lists_s.as<R>(),
                                h->lists_k.as<u64>(), h->lists_cnt.as<int>(), n_slots, st,
                                P.shared ? P.T : 0, P.gstride, h->inv_s.as<double>(), P.m + 1, P.N),
          "singles kernel");
  } else {
    L0_CK(h->ctr.ensure(8), "alloc counter");
    L0_CK(cudaMemsetAsync(h->ctr.p, 0, 8, st), "memset");
    l0::TileArgs<R> a;
    a.G = G;
    a.probs = h->probs.as<l0::ProbDesc>();
    a.n_probs = n_probs;
    a.row_prefix = h->rowpre.as<long long>();
    a.rowpre_len = (int)P.rowpre.size();
    a.B = B;
    a.ratio = P.mixed ? h->opt.fp32_fallback_pivot_ratio : h->opt.rank_deficient_pivot_ratio;
    a.K = K;
    a.S = S;
    a.item_counter = h->ctr.as<u64>();
    a.gthr = h->gthr.as<u64>();
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
    if (P.mixed) L0_CK(cudaMemsetAsync(h->dfr_n.p, 0, 24, st), "memset");
    const size_t smem = l0::tile_smem_bytes<R>(K, S, d - 2);
    if (P.shared)
      L0_CK(l0::launch_tile_shared<R>(a, d - 2, P.grid, smem, st), "shared tile kernel");
    else
      L0_CK(l0::launch_tile<R>(a, d - 2, d - 2, P.grid, smem, st), "tile kernel");
    if (P.mixed) {
      // FP64 redo of the near-singular tuples the FP32 kernel queued: the
      // FP64 Gram and the Gram-mode redo run only when many were queued, the
      // dot-product redo only when a few were (decided on the device)
      const bool can_gram = P.m <= 8192;
      if (can_gram) {
        L0_CK(h->gram.ensure((size_t)P.T * P.gstride * 8), "alloc Gram");
        L0_CK(l0::launch_gram64(h->w64.as<double>(), P.N, P.m, P.off.data(), P.T,
                                h->gram.as<double>(), P.ld, P.gstride, st, h->dfr_n.as<u64>(), d),
              "gram kernel");
      }
      l0::DeferArgs da;
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
      da.slot0 = P.grid;
      da.n_tuples = h->dfr_n.as<u64>() + 2;
      da.shared_T = P.shared ? P.T : 0;
      da.inv_s = h->inv_s.as<double>();
      da.mp1 = P.m + 1;
      L0_CK(l0::launch_defer(da, kDeferGroups, n_probs, st), "defer kernel");
    }
  }
  L0_CK(cudaEventRecord(h->ev[3], st), "event");
  // merge
  const int groups = std::max(1, std::min(n_slots, 32));
  L0_CK(h->part_s.ensure((size_t)n_probs * groups * K * sizeof(R)), "alloc merge");
  L0_CK(h->part_k.ensure((size_t)n_probs * groups * K * 8), "alloc merge");
  L0_CK(h->part_cnt.ensure((size_t)n_probs * groups * 4), "alloc merge");
  L0_CK(h->done.ensure((size_t)n_probs * 16), "alloc merge");
  {
    // per problem: done counter, pad, ordered +inf bound
    std::vector<unsigned> c0(4 * (size_t)n_probs, 0u);
    for (int q = 0; q < n_probs; ++q) {
      const u64 inf = l0::ord_inf<R>();
      memcpy(&c0[4 * q + 2], &inf, 8);
    }
    L0_CK(cudaMemcpyAsync(h->done.p, c0.data(), c0.size() * 4, cudaMemcpyHostToDevice, st), "copy");
  }
  L0_CK(h->pool_s.ensure((size_t)n_probs * K * sizeof(R)), "alloc pool");
  L0_CK(h->pool_k.ensure((size_t)n_probs * K * 8), "alloc pool");
  L0_CK(h->pool_cnt.ensure((size_t)n_probs * 4), "alloc pool");
  L0_CK(l0::launch_merge<R>(h->lists_s.as<R>(), h->lists_k.as<u64>(), h->lists_cnt.as<int>(),
                            n_slots, n_probs, K, S, groups, h->gthr.as<u64>(), h->part_s.as<R>(),
                            h->part_k.as<u64>(), h->part_cnt.as<int>(), h->done.as<unsigned>(),
                            h->pool_s.as<R>(), h->pool_k.as<u64>(), h->pool_cnt.as<int>(), st),
        "merge kernel");
  L0_CK(cudaEventRecord(h->ev[4], st), "event");
  // re-fit
  const int n_rows_max = (int)P.nmax;
  if ((size_t)(d + 1) * (size_t)n_rows_max * 8 > 200 * 1024)
    L0_CK(h->scratch.ensure((size_t)n_probs * K * (d + 1) * (size_t)n_rows_max * 8), "alloc refit scratch");
  L0_CK(h->refit.ensure((size_t)n_probs * K * 8), "alloc refit");
  l0::RefitArgs ra;
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
  ra.nmax = n_rows_max;
  ra.dmax = d;
  ra.smem_rows = 0;
  ra.refit = h->refit.as<double>();
  L0_CK(l0::launch_refit(ra, st), "refit kernel");
  // select
  L0_CK(h->cert.ensure((size_t)n_probs * sizeof(l0::CertOut)), "alloc cert");
  l0::SelectArgs<R> sa;
  sa.probs = h->probs.as<l0::ProbDesc>();
  sa.n_probs = n_probs;
  sa.K = K;
  sa.k = P.k;
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
  L0_CK(l0::launch_select<R>(sa, st), "select kernel");
  L0_CK(cudaEventRecord(h->ev[5], st), "event");
  std::vector<l0::CertOut> cert(n_probs);
  L0_CK(cudaMemcpyAsync(cert.data(), h->cert.p, n_probs * sizeof(l0::CertOut), cudaMemcpyDeviceToHost, st), "copy cert");
  u64 dfr_stats[3] = {0, 0, 0};
  if (P.mixed && d >= 2)
    L0_CK(cudaMemcpyAsync(dfr_stats, h->dfr_n.p, 24, cudaMemcpyDeviceToHost, st), "copy");
  int rc = wait_stream(h);
  if (rc) return rc;
  int hostErr = 0;
  L0_CK(cudaMemcpy(&hostErr, h->err.p, 4, cudaMemcpyDeviceToHost), "copy err");
  if (hostErr == 5) return fail(h, SISSO_L0_ENONFINITE, "NaN or Inf in X or y");
  if (hostErr == 7)
    return fail(h, SISSO_L0_EUNSUPPORTED,
                "too many near-singular tuples for the FP32 search; use SISSO_L0_FP64");
  if (hostErr != 0) return fail(h, SISSO_L0_ECUDA, "device error flag " + std::to_string(hostErr));
  P.fallback_tuples += dfr_stats[2];
  *certified = 1;
  *delta_max = 0;
  for (auto &c : cert) {
    if (!c.certified) *certified = 0;
    *delta_max = std::max(*delta_max, c.delta);
  }
  float t1 = 0, t2 = 0, t3 = 0;
  cudaEventElapsedTime(&t1, h->ev[2], h->ev[3]);
  cudaEventElapsedTime(&t2, h->ev[3], h->ev[4]);
  cudaEventElapsedTime(&t3, h->ev[4], h->ev[5]);
  *ms_tuple += t1;
  *ms_merge += t2;
  *ms_refit += t3;
  return SISSO_L0_OK;
}

int fit_impl(sisso_l0_t h, const double *X, const double *y, const int64_t *task_offsets,
             int32_t n_tasks, int64_t n_sis, int32_t n_dim, int32_t k, int32_t *out_tuples,
             double *out_rmse) {
  if (!X || !y || !task_offsets || !out_tuples || !out_rmse)
    return fail(h, SISSO_L0_EINVAL, "null pointer argument");
  if (n_tasks < 1) return fail(h, SISSO_L0_EINVAL, "n_tasks must be >= 1");
  if (n_dim < 1 || n_dim > SISSO_L0_MAX_DIM) return fail(h, SISSO_L0_EINVAL, "n_dim must be in [1, 8]");
  if (n_sis < n_dim) return fail(h, SISSO_L0_EINVAL, "n_sis must be >= n_dim");
  if (n_sis > (1LL << 30)) return fail(h, SISSO_L0_EUNSUPPORTED, "n_sis too large");
  if (k < 1) return fail(h, SISSO_L0_EINVAL, "k must be >= 1");
  if (task_offsets[0] != 0) return fail(h, SISSO_L0_EINVAL, "task_offsets[0] must be 0");
  FitPlan P;
  P.T = n_tasks;
  P.m = (int)n_sis;
  P.d = n_dim;
  P.k = k;
  P.shared = (h->opt.task_mode == SISSO_L0_SHARED) ? 1 : 0;
  P.mixed = (h->opt.precision == SISSO_L0_MIXED_BF16X3) ? 1 : 0;
  if (h->opt.precision != SISSO_L0_FP64 && h->opt.precision != SISSO_L0_MIXED_BF16X3)
    return fail(h, SISSO_L0_EUNSUPPORTED, "precision not supported");
  P.off.assign(task_offsets, task_offsets + n_tasks + 1);
  P.nmax = 0;
  for (int t = 0; t < n_tasks; ++t) {
    long long nt = P.off[t + 1] - P.off[t];
    if (nt < n_dim + 2) return fail(h, SISSO_L0_EINVAL, "every task needs at least n_dim + 2 rows");
    P.nmax = std::max(P.nmax, nt);
  }
  P.N = P.off[n_tasks];
  const u64 total = binom_host(n_sis, n_dim);
  if (total >= kSat) return fail(h, SISSO_L0_EUNSUPPORTED, "C(n_sis, n_dim) does not fit in 62 bits");
  if ((u64)k > total) return fail(h, SISSO_L0_EINVAL, "k exceeds C(n_sis, n_dim)");
  P.n_out = P.shared ? 1 : n_tasks;
  // candidate pool K': at least k, at most 2048 (shared-memory lists), never
  // more than the number of tuples
  if (k > 2048) return fail(h, SISSO_L0_EUNSUPPORTED, "k above 2048");
  int Kmax = h->opt.max_candidate_pool > 0 ? std::min(h->opt.max_candidate_pool, 2048) : 2048;
  int K = h->opt.candidate_pool > 0 ? h->opt.candidate_pool : std::min(std::max(4 * k, 256), 2048);
  K = std::min(std::max(K, k), 2048);
  if ((u64)K > total) K = (int)total;
  Kmax = std::max(Kmax, K);
  if ((u64)Kmax > total) Kmax = (int)std::max<u64>(total, (u64)K);
  cudaStream_t st = h->st;
  const int m = P.m;
  const long long N = P.N;
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
  L0_CK(cudaMemcpyAsync(h->offs.p, P.off.data(), (n_tasks + 1) * 8, cudaMemcpyHostToDevice, st), "copy offsets");
  L0_CK(h->err.ensure(16), "alloc err");
  L0_CK(cudaMemsetAsync(h->err.p, 0, 16, st), "memset");
  int rc = ensure_binom(h, m);
  if (rc) return rc;
  L0_CK(cudaEventRecord(h->ev[0], st), "event");
  // 1-2. centre and scale (FP64), then the augmented Gram per task
  const int mp1 = m + 1;
  P.ld = ((long long)mp1 + 31) / 32 * 32;
  P.gstride = (long long)mp1 * P.ld;
  const long long gstride = P.gstride;
  L0_CK(h->mu.ensure((size_t)n_tasks * mp1 * 8), "alloc mu");
  L0_CK(h->inv_s.ensure((size_t)n_tasks * mp1 * 8), "alloc inv_s");
  L0_CK(h->w64.ensure((size_t)mp1 * N * 8), "alloc W");
  if (!P.mixed) {
    L0_CK(l0::launch_centre(Xd, yd, N, m, h->offs.as<long long>(), n_tasks, h->mu.as<double>(),
                            h->inv_s.as<double>(), h->w64.as<double>(), h->err.as<int>(), st),
          "centre kernel");
    L0_CK(cudaEventRecord(h->ev[1], st), "event");
    L0_CK(h->gram.ensure((size_t)n_tasks * gstride * 8), "alloc Gram");
    L0_CK(l0::launch_gram64(h->w64.as<double>(), N, m, P.off.data(), n_tasks,
                            h->gram.as<double>(), P.ld, gstride, st),
          "gram kernel");
    P.have_g64 = true;
  } else {
    // split-BF16 rows: per task three segments of npad_t = roundup(n_t, 64)
    std::vector<int> meta(3 * n_tasks);
    long long ldk = 0;
    for (int t = 0; t < n_tasks; ++t) {
      const long long nt = P.off[t + 1] - P.off[t];
      const long long np = (nt + 63) / 64 * 64;
      if (ldk + 3 * np > (1LL << 30)) return fail(h, SISSO_L0_EUNSUPPORTED, "too many samples");
      meta[t] = (int)ldk;                      // kbeg
      meta[n_tasks + t] = (int)np;             // npad
      meta[2 * n_tasks + t] = (int)(3 * np / 64);   // K blocks
      ldk += 3 * np;
    }
    const size_t abytes = (size_t)mp1 * ldk * 2;
    L0_CK(h->abf.ensure(abytes), "alloc split rows");
    L0_CK(h->bbf.ensure(abytes), "alloc split rows");
    L0_CK(h->kmeta.ensure(meta.size() * 4), "alloc");
    L0_CK(cudaMemcpyAsync(h->kmeta.p, meta.data(), meta.size() * 4, cudaMemcpyHostToDevice, st), "copy");
    L0_CK(cudaMemsetAsync(h->abf.p, 0, abytes, st), "memset");
    L0_CK(cudaMemsetAsync(h->bbf.p, 0, abytes, st), "memset");
    const int *kbeg = h->kmeta.as<int>();
    L0_CK(l0::launch_centre_split(Xd, yd, N, m, h->offs.as<long long>(), n_tasks,
                                  h->mu.as<double>(), h->inv_s.as<double>(), h->w64.as<double>(),
                                  h->abf.p, h->bbf.p, ldk, kbeg, kbeg + n_tasks, h->err.as<int>(),
                                  st),
          "centre kernel");
    L0_CK(cudaEventRecord(h->ev[1], st), "event");
    L0_CK(h->gram32.ensure((size_t)n_tasks * gstride * 4), "alloc Gram");
    L0_CK(l0::launch_gram_tc(h->abf.p, h->bbf.p, ldk, m, n_tasks, kbeg, kbeg + 2 * n_tasks,
                             h->gram32.as<float>(), P.ld, gstride, h->err.as<int>(), st),
          "tensor-core gram kernel");
  }
  L0_CK(cudaEventRecord(h->ev[6], st), "event");
  // problems
  // problems: one per task (PER_TASK), or one spanning all tasks (SHARED)
  P.pd.clear();
  for (int t = 0; t < (P.shared ? 1 : n_tasks); ++t) {
    l0::ProbDesc d{};
    d.g_off = (long long)t * gstride;
    d.ld = P.ld;
    d.m = m;
    d.d = n_dim;
    d.dp = n_dim - 2;
    d.task = t;
    d.total = total;
    P.pd.push_back(d);
  }
  // grid size: persistent CTAs
  const int dp = std::max(0, n_dim - 2);
  if (n_dim >= 2) {
    int S0 = 1024;
    while (S0 < 2 * Kmax) S0 <<= 1;
    int bps = 0;
    if (P.mixed) {
      const size_t smem = l0::tile_smem_bytes<float>(Kmax, S0, dp);
      if (P.shared) L0_CK(l0::shared_occupancy<float>(dp, smem, &bps), "occupancy");
      else L0_CK(l0::tile_occupancy<float>(dp, dp, smem, &bps), "occupancy");
    } else {
      const size_t smem = l0::tile_smem_bytes<double>(Kmax, S0, dp);
      if (P.shared) L0_CK(l0::shared_occupancy<double>(dp, smem, &bps), "occupancy");
      else L0_CK(l0::tile_occupancy<double>(dp, dp, smem, &bps), "occupancy");
    }
    if (bps < 1) return fail(h, SISSO_L0_EUNSUPPORTED, "tuple kernel does not fit on an SM");
    P.grid = h->n_sm * bps;
  }
  plan_items(P, {}, std::max(1, P.grid));
  L0_CK(h->probs.ensure(P.pd.size() * sizeof(l0::ProbDesc)), "alloc probs");
  L0_CK(cudaMemcpyAsync(h->probs.p, P.pd.data(), P.pd.size() * sizeof(l0::ProbDesc), cudaMemcpyHostToDevice, st), "copy probs");
  L0_CK(h->rowpre.ensure(std::max<size_t>(1, P.rowpre.size()) * 8), "alloc rowpre");
  if (!P.rowpre.empty())
    L0_CK(cudaMemcpyAsync(h->rowpre.p, P.rowpre.data(), P.rowpre.size() * 8, cudaMemcpyHostToDevice, st), "copy rowpre");
  // rmse divisor per problem: n_t (PER_TASK); SHARED scores are already the
  // pooled mean SSE
  {
    std::vector<double> div(P.pd.size());
    for (size_t q = 0; q < P.pd.size(); ++q)
      div[q] = P.shared ? 1.0 : (double)(P.off[P.pd[q].task + 1] - P.off[P.pd[q].task]);
    L0_CK(h->rdiv.ensure(div.size() * 8), "alloc");
    L0_CK(cudaMemcpyAsync(h->rdiv.p, div.data(), div.size() * 8, cudaMemcpyHostToDevice, st), "copy");
  }
  L0_CK(h->out_t.ensure((size_t)P.n_out * k * n_dim * 4), "alloc out");
  L0_CK(h->out_r.ensure((size_t)P.n_out * k * 8), "alloc out");
  L0_CK(h->dfr_n.ensure(24), "alloc");   // queued runs, queued tuples, redone tuples
  if (P.mixed && n_dim >= 2) {
    L0_CK(h->dfr_key.ensure((size_t)kDeferCap * 8), "alloc deferral buffer");
    L0_CK(h->dfr_len.ensure((size_t)kDeferCap * 4), "alloc deferral buffer");
  }
  int certified = 0, enl = 0;
  double delta = 0;
  float ms_tuple = 0, ms_merge = 0, ms_refit = 0;
  for (;;) {
    int S = 1024;
    while (S < 2 * K) S <<= 1;
    if (P.mixed)
      rc = run_search<float>(h, P, K, S, h->gram32.as<float>(), &certified, &delta, &ms_tuple,
                             &ms_merge, &ms_refit);
    else
      rc = run_search<double>(h, P, K, S, h->gram.as<double>(), &certified, &delta, &ms_tuple,
                              &ms_merge, &ms_refit);
    if (rc) break;
    if (certified || K >= Kmax) break;
    K = std::min(2 * K, Kmax);
    ++enl;
  }
  if (rc) return rc;
  // outputs to the caller
  L0_CK(cudaMemcpyAsync(out_tuples, h->out_t.p, (size_t)P.n_out * k * n_dim * 4, cudaMemcpyDefault, st), "copy out");
  L0_CK(cudaMemcpyAsync(out_rmse, h->out_r.p, (size_t)P.n_out * k * 8, cudaMemcpyDefault, st), "copy out");
  rc = wait_stream(h);
  if (rc) return rc;
  float t_prep = 0, t_gram = 0;
  cudaEventElapsedTime(&t_prep, h->ev[0], h->ev[1]);
  cudaEventElapsedTime(&t_gram, h->ev[1], h->ev[6]);
  sisso_l0_stats &S = h->stats;
  memset(&S, 0, sizeof(S));
  S.struct_size = sizeof(S);
  S.candidate_pool = K;
  S.pool_enlargements = enl;
  S.certified = certified;
  S.tuple_fits = total * (u64)n_tasks * (u64)(enl + 1);
  S.max_pool_rel_error = delta;
  S.fp64_fallback_tuples = P.fallback_tuples;
  // centre + Gram, then per search pass: seed, tuple, merge, refit, select
  S.kernel_launches = (P.mixed ? 2 : 1 + n_tasks) + 5LL * (enl + 1);
  S.ms_prep = t_prep;
  S.ms_gram = t_gram;
  S.ms_tuple = ms_tuple;
  S.ms_merge = ms_merge;
  S.ms_refit = ms_refit;
  S.ms_total = t_prep + t_gram + ms_tuple + ms_merge + ms_refit;
  return SISSO_L0_OK;
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
  opt->autotune_cache_path = nullptr;
  opt->timeout_seconds = 0.0;
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
  if (!(o.rank_deficient_pivot_ratio >= 0) || !(o.fp32_fallback_pivot_ratio >= 0)) return SISSO_L0_EINVAL;
  sisso_l0_handle *h = new (std::nothrow) sisso_l0_handle();
  if (!h) return SISSO_L0_ENOMEM;
  h->opt = o;
  h->st = (cudaStream_t)o.stream;
  cudaError_t e = cudaSetDevice(o.device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&h->n_sm, cudaDevAttrMultiProcessorCount, o.device);
  for (int i = 0; i < 8 && e == cudaSuccess; ++i) e = cudaEventCreate(&h->ev[i]);
  if (e != cudaSuccess) {
    delete h;
    return (e == cudaErrorMemoryAllocation) ? SISSO_L0_ENOMEM : SISSO_L0_ECUDA;
  }
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
    return fit_impl(h, X, y, task_offsets, n_tasks, n_sis, n_dim, k, out_tuples, out_rmse);
  } catch (const std::bad_alloc &) {
    return fail(h, SISSO_L0_ENOMEM, "host allocation failed");
  } catch (...) {
    return fail(h, SISSO_L0_ECUDA, "unexpected host exception");
  }
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
  DevBuf *bufs[] = {&h->xin, &h->yin, &h->offs, &h->mu, &h->inv_s, &h->w64, &h->gram, &h->binom,
                    &h->probs, &h->rowpre, &h->ctr, &h->gthr, &h->lists_s, &h->lists_k,
                    &h->lists_cnt, &h->part_s, &h->part_k, &h->part_cnt, &h->done, &h->pool_s,
                    &h->pool_k, &h->pool_cnt, &h->scratch, &h->refit, &h->rdiv,
                    &h->cert, &h->out_t, &h->out_r, &h->err, &h->dfr_key, &h->dfr_len, &h->dfr_n,
                    &h->dfr_cnt, &h->abf, &h->bbf, &h->kmeta, &h->gram32};
  for (DevBuf *b : bufs) b->release();
  for (int i = 0; i < 8; ++i)
    if (h->ev[i]) cudaEventDestroy(h->ev[i]);
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
