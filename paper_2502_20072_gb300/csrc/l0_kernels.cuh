// l0_kernels.cuh -- launch interfaces between the host orchestrator
// (l0_api.cu) and the kernels (l0_prep.cu, l0_tuple.cu, l0_select.cu).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "l0_common.cuh"

namespace l0 {

// tile shape of the tuple kernel: 8 warps, each warp UJ rows j, each lane UK
// columns k (k = k0 + lane + 32 v)
constexpr int TILE_WARPS = 8;
constexpr int TILE_UJ = 8;
constexpr int TILE_UK = 4;
constexpr int TILE_TJ = TILE_WARPS * TILE_UJ;   // 64 rows
constexpr int TILE_TK = 32 * TILE_UK;           // 128 columns

// One scoring problem: a task (PER_TASK) and a tuple size d >= 2.
struct ProbDesc {
  long long g_off;        // element offset of the problem's Gram in the Gram buffer
  long long ld;           // leading dimension of that Gram
  int m, d, dp, task;     // dp = d - 2 (size of the outer prefix)
  int n_jt, n_kt, L, prefix_off;   // j/k tile counts, prefix steps per item, row-prefix offset
  long long item_begin, item_end;  // global work-item range
  u64 total;              // C(m, d)
  int k, pad;             // requested list length
  long long out_t_off;    // offset of this problem's tuples in the output staging
  long long out_r_off;    // offset of this problem's errors in the output staging
};

template <typename R>
struct TileArgs {
  const R *G;
  const ProbDesc *probs;
  int n_probs;
  const long long *row_prefix;     // per problem and row block bj <= n_jt, ROWINFO words:
                                   // items before bj, then bj's tiles' prefix chunks:
                                   // count, size q, number of size q + 1
  int rowpre_len;                  // total entries of row_prefix
  Binom B;
  double ratio;                    // pivot ratio: ineligible (FP64) / redo in FP64 (FP32)
  int K, S;                        // list capacity, staging capacity
  u64 *item_counter;
  long long item_limit;            // items at or past this index are not processed
  long long item_stride, item_offset;   // the counter's value c stands for item
                                        // c * stride + offset (a shard's items)
  u64 *gthr;                       // [n_probs] ordered score bits
  unsigned *hist;                  // [n_probs][L0_HIST_WORDS] staged-score counts
  R *out_s; u64 *out_k; int *out_cnt;   // [n_probs][n_slots][K], [n_probs][n_slots]
  int n_slots;
  // FP32 only: runs of tuples redone in FP64: lexicographic rank of the first
  // tuple, (problem << 8) | run length (<= 128); dfr_n[0] runs, dfr_n[1] tuples
  u64 *dfr_key; unsigned *dfr_len; u64 *dfr_n; long long dfr_cap;
  int *err;
  // FP32 band pass: every tuple scoring below the (fixed) cut is queued for
  // the FP64 redo instead of entering the FP32 lists
  int band;
  const int *cls;                  // [m] duplicate class of each column (smallest index
                                   // of the columns equal to it), or null
  // SHARED mode (shared_T > 0): Grams of tasks 0..T-1 at G + t * shared_gstride;
  // task weights S_yy,t / N from inv_s[t * mp1] and n_total
  int shared_T;
  long long shared_gstride;
  const double *inv_s;
  int mp1;
  long long n_total;
};

// k tiles of j-tile row bj: they start right after the row block's first
// column, k0 = j0 + 1 + bk * TILE_TK, so only the first one crosses the
// diagonal (a quarter of its slots have k <= j)
__host__ __device__ inline int tile_k_count(int bj, int m) {
  const int first = bj * TILE_TJ + 1;
  return first < m ? (m - first + TILE_TK - 1) / TILE_TK : 0;
}
__host__ __device__ inline int tile_k0(int bj, int bk) { return bj * TILE_TJ + 1 + bk * TILE_TK; }

constexpr int ROWINFO = 4;   // words per row block in TileArgs::row_prefix

// work items of one j-tile row: (#k tiles) x (#prefix chunks)
__host__ __device__ inline long long tile_row_items(int bj, int m, int dp, int L,
                                                    int n_kt, u64 nprefix) {
  (void)dp;
  (void)n_kt;
  const long long nk = tile_k_count(bj, m);
  if (nk <= 0) return 0;
  long long nch = (long long)((nprefix + (u64)L - 1) / (u64)L);
  return nk * nch;
}

// The FP32 search queues near-singular tuples for an FP64 redo.  Building the
// full FP64 Gram for that pays off only when many tuples were queued (and
// n_sis is moderate); otherwise the redo computes the few FP64 entries it
// needs as dot products.  Host and device evaluate the same rule on the
// queued-tuple counter.
__host__ __device__ inline bool defer_wants_gram(u64 n_tuples, int m, int d) {
  if (m > 8192) return false;
  return (double)n_tuples * (double)((d + 1) * (d + 2) / 2) * 8.0 >
         (double)(m + 1) * (double)(m + 1);
}

// The FP32 tuple kernel for d = 2 and 3 (l0_tile32.cu), PER_TASK exhaustive
// searches on the same work items as tile_kernel.  Shapes: 1 = 256 threads,
// one CTA per SM; 2 = 256 threads, two CTAs per SM; 3 = 512 threads (four
// rows per warp).  The Gram's leading dimension and per-task stride must be
// multiples of 4 floats (its rows are copied by the TMA unit).
bool tile32_supports(int variant, int dp_lo, int dp_hi);
size_t tile32_smem_bytes(int K, int S);
int tile32_threads(int variant);
cudaError_t tile32_occupancy(int variant, int dp_lo, int dp_hi, size_t smem, int *blocks_per_sm);
cudaError_t launch_tile32(const TileArgs<float> &a, int variant, int dp_lo, int dp_hi, int grid,
                          size_t smem, cudaStream_t st);

// kernels (host launch wrappers)
// duplicate classes of the columns: cls[j] = the smallest i with column i
// equal to column j over all rows (relative difference <= 1e-12); a tuple
// holding two columns of one class is exactly rank deficient
cudaError_t launch_column_classes(const double *X, long long n_total, int m, u64 *hash, int *cls,
                                  cudaStream_t st);

cudaError_t launch_centre(const double *X, const double *y, long long n_total,
                          int m, const long long *offsets_dev, int T,
                          double *mu, double *inv_s, double *W64, int *err,
                          cudaStream_t st);
// gate (optional): run only when defer_wants_gram(gate[1], m, gate_d)
cudaError_t launch_gram64(const double *W64, long long n_total, int m,
                          const long long *offsets_host, int T, double *G,
                          long long ld, long long g_stride, cudaStream_t st,
                          const u64 *gate = nullptr, int gate_d = 0,
                          int upper_only = 0, const int *skip = nullptr);
// after a gated FP64 Gram: *have = 1 when the gate let it run (a later pass of
// the same fit can skip it through launch_gram64's skip flag)
cudaError_t launch_mark_gram64(const u64 *gate, int m, int gate_d, int *have, cudaStream_t st);

template <typename R>
cudaError_t launch_tile(const TileArgs<R> &a, int dp_lo, int dp_hi, int grid,
                        size_t smem, cudaStream_t st);
template <typename R>
size_t tile_smem_bytes(int K, int S, int dp_hi);
template <typename R>
cudaError_t tile_occupancy(int dp_lo, int dp_hi, size_t smem, int *blocks_per_sm);

// SHARED mode tuple kernel (one problem spanning all tasks)
template <typename R>
cudaError_t launch_tile_shared(const TileArgs<R> &a, int dp, int grid, size_t smem,
                               cudaStream_t st);
template <typename R>
cudaError_t shared_occupancy(int dp, size_t smem, int *blocks_per_sm);

template <typename R>
cudaError_t launch_singles(const R *G, const ProbDesc *probs_host_view,
                           const ProbDesc *probs_dev, int n_probs, int K, int S,
                           int grid_x, u64 *gthr, R *out_s, u64 *out_k,
                           int *out_cnt, int n_slots, cudaStream_t st,
                           int shared_T, long long gstride, const double *inv_s,
                           int mp1, long long n_total);

// merge all slot lists of every problem into one top-K' pool per problem.
// part_*: [n_probs][groups][K] partial lists; counters: [n_probs][4]
// (done counter, pad, ordered bound of the partials) -- initialise with
// merge_counters_init and they are left initialised.
template <typename R>
cudaError_t launch_merge(const R *in_s, const u64 *in_k, const int *in_cnt,
                         int n_slots, int n_probs, int K, int S, int groups, const u64 *gthr,
                         R *part_s, u64 *part_k, int *part_cnt, unsigned *counters,
                         R *pool_s, u64 *pool_k, int *pool_cnt, cudaStream_t st);

struct RefitArgs {
  const double *X, *y;
  long long n_total;
  int m;
  const long long *offsets;   // device [T+1]
  const double *mu;           // [T][m+1], index 0 = target
  int T, shared;              // SHARED: all tasks, else the problem's task
  const ProbDesc *probs;
  int n_probs, K;
  const u64 *pool_k; const int *pool_cnt;
  Binom B;
  double rho_min;
  double *scratch; long long nmax;   // [n_probs*K][(d+1)][nmax] (when not in shared memory)
  int dmax;                   // largest d over the problems
  int smem_rows;              // set by launch_refit: columns in shared memory
  double *refit;              // [n_probs][K] score (SSE or pooled mean SSE), +inf if ineligible
  int refit_all;              // 0: only the first refit_count(k, K, cnt) pool entries
};
// Pool entries re-fitted in FP64: the pool is sorted by search score, and the
// first max(2k, K'/2) of it are re-fitted (all of it when the caller needs
// every entry's exact score); the rest are bounded by the certificate
// through the first search score left out.
__host__ __device__ inline int refit_count(int k, int K, int cnt, int all) {
  const int r = all ? cnt : (2 * k > K / 2 ? 2 * k : K / 2);
  return r < cnt ? r : cnt;
}
cudaError_t launch_refit(const RefitArgs &a, cudaStream_t st);

struct CertOut {
  double delta;        // max |gram SSE - refit SSE| over the pool
  double pool_worst;   // bound (SSE units) under which the pool holds every tuple
  double kth_refit;    // k-th best refit score (SSE units)
  int pool_cnt, pool_full, n_valid, certified;
};

template <typename R>
struct SelectArgs {
  const ProbDesc *probs;       // per problem: k, d, output offsets
  int n_probs, K;
  const R *pool_s; const u64 *pool_k; const int *pool_cnt;
  const double *refit;
  const double *inv_s;         // [T][m+1]: 1 / ||centred column||, index 0 the target
  int mp1, shared;             // PER_TASK: a pool score times S_yy,t is an SSE
  const double *rmse_div;      // [n_probs] n_t (PER_TASK) or 1 (SHARED: pooled mean)
  Binom B;
  int *out_tuples; double *out_rmse;   // staging; problem q at its out_*_off
  CertOut *cert;
  double cert_safety;
  const u64 *gthr;             // [n_probs] final search threshold (ordered bits of R)
  int refit_all;               // as RefitArgs::refit_all
  const double *delta_floor;   // [n_probs] band pass: the previous pass's search-score
                               // error (null: not a band pass)
  const u64 *band_thr;         // [n_probs] band pass: the fixed FP32 cut it started from
};
// Band pass set-up: from the previous pass's certificate of each problem, the
// cut (k-th re-fitted score + margin * delta, as ordered bits of the FP32
// relative score) into band_thr and delta into delta_floor.
cudaError_t launch_band_cut(const CertOut *cert, const ProbDesc *probs, int n_probs,
                            const double *inv_s, int mp1, int shared, double margin,
                            u64 *band_thr, double *delta_floor, cudaStream_t st);
template <typename R>
cudaError_t launch_select(const SelectArgs<R> &a, cudaStream_t st);

// mixed precision: centring + split-BF16 rows, tensor-core Gram
cudaError_t launch_centre_split(const double *X, const double *y, long long n_total, int m,
                                const long long *offsets_dev, int T, double *mu, double *inv_s,
                                double *W64, void *A, void *B, long long ldk,
                                const int *kbeg_dev, const int *npad_dev, int *err,
                                cudaStream_t st);
size_t gram_tc_smem_bytes();
// upper-triangular 128 x 128 tiles of an (m + 1)-square Gram
int gram_tc_tiles(int m);
// scratch floats for nsplit-way K splits of T tasks' tiles (0 when nsplit = 1)
size_t gram_tc_part_floats(int m, int T, int nsplit);
// nsplit >= 1 ways of splitting every task's K blocks (at most the fewest K
// blocks of a task); nsplit > 1 needs part (gram_tc_part_floats) and
// tile_ctr (gram_tc_tiles(m) * T counters, zero; left zero)
cudaError_t launch_gram_tc(const void *A, const void *B, long long ldk, int m, int T,
                           const int *kbeg_dev, const int *nkb_dev, float *G, long long ld,
                           long long g_stride, int *err, cudaStream_t st, int nsplit = 1,
                           float *part = nullptr, unsigned *tile_ctr = nullptr);

// FP64 redo of the runs the FP32 tuple kernel queued
struct DeferArgs {
  const double *G64;           // FP64 Gram per task (null: dot products of W64)
  long long ld64, g64_stride;
  const double *W64;           // scaled columns [(m+1)][n_total]
  long long n_total;
  const long long *offsets;    // device [T+1]
  const ProbDesc *probs;
  Binom B;
  double ratio;                // FP64 rank-deficiency pivot ratio
  const u64 *run_key; const unsigned *run_len;
  const u64 *n_runs;           // [0] queued runs, [1] queued tuples
  long long cap;
  int K, S;
  u64 *gthr;
  float *out_s; u64 *out_k; int *out_cnt;
  int n_slots, slot0;          // lists go to slots slot0 + blockIdx.x
  u64 *n_tuples;               // tuples redone (statistics)
  // SHARED mode (shared_T > 0): pooled score sum_t S_yy,t rel_t / N
  int shared_T;
  const double *inv_s;
  int mp1;
  unsigned *batch_ctr;         // [n_probs] run batches handed out (zeroed before the launch)
};
// both launched; exactly one does work (see defer_wants_gram)
cudaError_t launch_defer(const DeferArgs &a, int groups, int n_probs, cudaStream_t st);

// initial search threshold per problem: +inf, then the K'-th best score of
// all d-tuples of the M best single columns (a valid bound: real tuples)
// seed == 0: only the +inf initialisation; max_keys >= max(n_sis, 2 K' + 64)
// (d = 3 also scores the completions of the best pairs of those columns while
// the keys fit: seed_keys() sizes room for them); cls: duplicate classes or null
template <typename R>
cudaError_t launch_seed(const R *G, const ProbDesc *probs_dev, int n_probs, int K, int S,
                        int seed, double ratio, const Binom &B, u64 *gthr, unsigned *hist,
                        int max_keys, cudaStream_t st, const int *cls);
inline int seed_keys(int m, int K) {
  const long long v = (long long)m * 9 + 2LL * K + 2112;
  return (int)(v < 50000 ? v : 50000);
}
template <typename R>
size_t seed_smem_bytes(int K, int S);

// ------------------------------------------------ learned pair scorer --
// 6-256-256-1 ReLU network; flat FP32 parameter vector
// [W1 (256 x 6) | b1 | W2 (256 x 256, row = output unit) | b2 | w3 | b3]
constexpr int MLP_NIN = 6, MLP_NH = 256;
constexpr int MLP_OFF_W1 = 0;
constexpr int MLP_OFF_B1 = MLP_OFF_W1 + MLP_NH * MLP_NIN;
constexpr int MLP_OFF_W2 = MLP_OFF_B1 + MLP_NH;
constexpr int MLP_OFF_B2 = MLP_OFF_W2 + MLP_NH * MLP_NH;
constexpr int MLP_OFF_W3 = MLP_OFF_B2 + MLP_NH;
constexpr int MLP_OFF_B3 = MLP_OFF_W3 + MLP_NH;
constexpr int MLP_N_PARAMS = MLP_OFF_B3 + 1;
constexpr int MLP_PSTRIDE = (MLP_N_PARAMS + 1 + 3) / 4 * 4;   // partial gradients + loss
constexpr int MLP_FEAT_LD = 8;                                 // floats per feature row
enum { MLP_INFER_FEATS = 0, MLP_INFER_GRAM = 1, MLP_TRAIN = 2 };

struct MlpArgs {
  const float *params;          // FP32 master parameters
  const float *feats;           // [rows][MLP_FEAT_LD] (INFER_FEATS, TRAIN)
  const float *label;           // [rows] (TRAIN)
  long long row0, n_rows;       // rows [row0, row0 + n_rows); pair ranks in INFER_GRAM
  const float *G;               // FP32 augmented Gram (INFER_GRAM)
  long long ld;
  float *out;                   // [n_rows] network outputs (INFER_*)
  float *partial;               // [grid][MLP_PSTRIDE] partial gradients (TRAIN)
  double inv_B;                 // 1 / rows of the training step
  int *err;
};
size_t mlp_smem_bytes(int mode);
cudaError_t launch_mlp(int mode, const MlpArgs &a, const void *W2b, const void *W2Tb, int grid,
                       cudaStream_t st);
cudaError_t launch_mlp_adam(float *params, float *m1, float *m2, const float *partial,
                            int n_parts, float lr, int t, int do_step, float *grad_out,
                            float *loss_out, void *W2b, void *W2Tb, cudaStream_t st);

// Features of the pair i < j from the augmented correlation Gram (target at
// index 0, upper triangle): r_i, r_j (Pearson r, Eq. 1), C_ij, the
// correlations rho_j.i, rho_i.j of each column with the residual of the
// one-feature fit on the other, and log(1 - R^2) / 8 of the two-feature fit
// (the log residual fraction: R^2 itself sits too close to 1 for a BF16
// input where it matters most).
__device__ __forceinline__ void pair_feature_vec(const float *G, long long ld, int i, int j,
                                                 float *x) {
  const float g00 = G[0];
  const float gii = G[(long long)(i + 1) * ld + i + 1], gjj = G[(long long)(j + 1) * ld + j + 1];
  const float gij = G[(long long)(i + 1) * ld + j + 1];
  const float ri = G[i + 1] * rsqrtf(fmaxf(g00 * gii, 1e-30f));
  const float rj = G[j + 1] * rsqrtf(fmaxf(g00 * gjj, 1e-30f));
  const float c = gij * rsqrtf(fmaxf(gii * gjj, 1e-30f));
  const float ei = fmaxf(1.f - ri * ri, 1e-12f), ej = fmaxf(1.f - rj * rj, 1e-12f);
  const float dc = 1.f - c * c;
  x[0] = ri;
  x[1] = rj;
  x[2] = c;
  x[3] = (rj - c * ri) * rsqrtf(ei);
  x[4] = (ri - c * rj) * rsqrtf(ej);
  const float r2 = dc > 1e-6f ? fminf(fmaxf((ri * ri + rj * rj - 2.f * ri * rj * c) / dc, 0.f), 1.f)
                             : fmaxf(ri * ri, rj * rj);
  x[5] = 0.125f * logf(fmaxf(1.f - r2, 1e-12f));
}

// symmetric copy of an upper-triangular Gram (lower triangle filled) and
// its diagonal in a contiguous array
template <typename T>
cudaError_t launch_gram_mirror(T *G, long long ld, int mp1, T *diag, cudaStream_t st);
// features [n][MLP_FEAT_LD] of the pairs with colex ranks [p0, p0 + n)
cudaError_t launch_pair_features(const float *G, long long ld, long long p0, long long n,
                                 float *feats, cudaStream_t st);
// per pair: log(clamp(min over k of SSE(i, j, k) / S_yy, floor, 1)) over the
// eligible completions, from the mirrored FP32 Gram
cudaError_t launch_pair_best(const float *G, long long ld, const float *diag, int m,
                             long long n_pairs, double ratio, float floor_, float *label,
                             cudaStream_t st);
// labels -> (labels - mean) / std over the n labels (acc: 2 doubles scratch)
cudaError_t launch_label_standardize(float *lab, long long n, double *acc, cudaStream_t st);
// top pairs by network score: all pairs whose score falls in the lowest
// histogram bins holding at least `want` pairs; writes their (i, j) and a
// bitmap over colex pair ranks; counter[0] = pairs written
cudaError_t launch_select_pairs(const float *score, long long n_pairs, long long want,
                                unsigned *hist, unsigned *bin_out, int *pairs,
                                unsigned long long *counter, unsigned *bits, cudaStream_t st);
// bitmap and canonical copy of an explicit pair list
cudaError_t launch_pairs_from_list(const int *in, long long n, int m, int *pairs, unsigned *bits,
                                   int *err, cudaStream_t st);

template <typename R>
struct PropArgs {
  const R *G; long long ld; const R *diag; int m;
  const int *cls;
  const int *pairs; long long n_pairs; const unsigned *bits;
  u64 *pair_ctr; u64 *fits;
  Binom B; u64 total;
  double ratio; int mixed;
  int K, S;
  u64 *gthr; unsigned *hist;
  R *out_s; u64 *out_k; int *out_cnt;
  u64 *dfr_key; unsigned *dfr_len; u64 *dfr_n; long long dfr_cap;
  int *err;
};
template <typename R>
size_t proposal_smem_bytes(int K, int S);
template <typename R>
cudaError_t proposal_occupancy(int K, int S, int *blocks_per_sm);
template <typename R>
cudaError_t launch_proposal(const PropArgs<R> &a, int grid, cudaStream_t st);

// final ranking of candidates gathered from shards (one CTA): sort by (SSE,
// lexicographic rank), unrank the first k, RMSE = sqrt(SSE / n); certified
// when min over shards of (bound - 4 delta) clears the k-th SSE.  scratch
// holds 2 P entries (P = n_cand rounded up to a power of two).
cudaError_t launch_merge_shards(const Binom &B, int m, int d, u64 total, int k, double n_rows,
                                const u64 *keys, const double *sse, long long n_cand,
                                const double *bounds, const double *deltas, int n_shards,
                                double *scratch_s, u64 *scratch_k, int *out_tuples,
                                double *out_rmse, int *certified, cudaStream_t st);

cudaError_t launch_unrank(const Binom &B, int m, int d, u64 total,
                          const u64 *ranks, long long count, int *tuples,
                          cudaStream_t st);

}  // namespace l0
