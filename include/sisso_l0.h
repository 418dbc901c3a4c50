/*
 * sisso_l0.h -- C ABI of the GB300 (sm_103a) l0-regularization library.
 *
 * The operation (paper Sec. 2.4): given the m features selected by SIS and a
 * target, score every n-tuple of features by the least-squares fit of the
 * features to the target and return the best tuples.  The score is the mean
 * squared deviation of the fit; here the fit has an intercept and the
 * reported error is the RMSE, sqrt(SSE / n_t).  Multi-task data (Sec. 3.1,
 * "same descriptor, different coefficients per task") is given as row ranges
 * of the same columns.
 *
 * Conventions shared by every entry point:
 *   - All functions return SISSO_L0_OK (0) or one of the error codes below;
 *     no C++ exception crosses this boundary.  After an error,
 *     sisso_l0_last_error() describes it.
 *   - X is FP64, feature-major: X[j * n_total + i] is feature j of sample i,
 *     so each column is contiguous; rows are grouped by task.  X and y may
 *     live in device memory or in host memory (the pointer kind is queried);
 *     host inputs are copied into library-owned device memory per call.
 *   - Outputs may be device or host pointers likewise.
 *   - The caller owns X, y, task_offsets and the outputs; the library never
 *     frees them and keeps no pointer to them after the call returns.
 *   - Work is ordered on the stream given at create time; fit returns after
 *     the results are complete (bounded by options.timeout_seconds).
 *   - One handle must not be used by two threads at the same time.
 */
#ifndef SISSO_L0_H
#define SISSO_L0_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SISSO_L0_OK 0
#define SISSO_L0_EINVAL 1       /* bad argument: sizes, offsets, null pointers */
#define SISSO_L0_ENOMEM 2       /* device or host allocation failed */
#define SISSO_L0_ECUDA 3        /* a CUDA call failed */
#define SISSO_L0_ETIMEOUT 4     /* the stream did not finish within timeout_seconds */
#define SISSO_L0_ENONFINITE 5   /* NaN or Inf in X or y */
#define SISSO_L0_EUNSUPPORTED 6 /* valid request this build does not handle */

#define SISSO_L0_MAX_DIM 8      /* the paper's descriptors have fewer than 10 features (Sec. 2.4) */

typedef enum {
  SISSO_L0_FP64 = 0,          /* FP64 Gram (FFMA64), FP64 solves, FP64 re-fit */
  SISSO_L0_MIXED_BF16X3 = 1,  /* split-BF16 (3-term) tensor-core Gram, FP32 solves, FP64 re-fit */
  SISSO_L0_MIXED_TF32 = 2     /* reserved */
} sisso_l0_precision;

typedef enum {
  SISSO_L0_PER_TASK = 0,      /* rank each task on its own: n_out = n_tasks lists */
  SISSO_L0_SHARED = 1         /* rank by pooled mean SSE sum_t SSE_t / N: n_out = 1 list */
} sisso_l0_task_mode;

typedef struct sisso_l0_handle *sisso_l0_t;

typedef struct {
  int32_t struct_size;               /* sizeof(sisso_l0_options) */
  int32_t device;                    /* CUDA device ordinal */
  void *stream;                      /* cudaStream_t owned by the caller; NULL = legacy stream */
  int32_t precision;                 /* sisso_l0_precision */
  int32_t task_mode;                 /* sisso_l0_task_mode */
  int32_t candidate_pool;            /* K': candidates re-fitted in FP64 (0 = auto, max(4k, 256)) */
  int32_t max_candidate_pool;        /* ceiling for K' when the certificate doubles it (0 = 2048) */
  double fp32_fallback_pivot_ratio;  /* FP32 pivot ratio below which a tuple is redone in FP64 (1e-6) */
  double rank_deficient_pivot_ratio; /* FP64 Gram pivot ratio below which a tuple is ineligible (1e-12) */
  int32_t autotune;                  /* 1: time preset launch configurations on the first
                                        search of a shape and keep the fastest (0 off) */
  int32_t use_graph;                 /* 1: capture the device work of a search pass in a
                                        CUDA graph on the first call of a shape, replay after */
  const char *autotune_cache_path;   /* file that persists autotuner choices (NULL: none) */
  double timeout_seconds;            /* host-side deadline for stream completion (<= 0: none) */
  int32_t fp64_rerun_uncertified;    /* MIXED: when the candidate pool cannot be certified at
                                        max_candidate_pool (FP32 score errors as large as the
                                        gaps between the best scores), first rerun the FP32
                                        search as a band pass (every tuple below the k-th
                                        re-fitted score + 8 delta scored in FP64), then, if
                                        that is still uncertified, redo the fit in FP64 (1,
                                        default); or return the uncertified result (0) */
  int32_t tuple_kernel;              /* shape of the tuple search kernel: -1 (default) picks
                                        one (the autotuner times them when autotune is on);
                                        0 the general kernel (any d, FP32 or FP64); 1, 2, 3
                                        the FP32 kernel for d = 2 and 3 (PER_TASK, exhaustive)
                                        with 256 threads and one CTA per SM, 256 threads and
                                        two CTAs per SM, 512 threads and one CTA per SM.  A
                                        shape that cannot run a fit falls back to 0 */
} sisso_l0_options;

typedef struct {
  int32_t struct_size;               /* sizeof(sisso_l0_stats) */
  int32_t candidate_pool;            /* K' used by the last fit */
  int32_t pool_enlargements;         /* times K' was doubled by the certificate */
  int32_t certified;                 /* 1 when every output list passed the certificate: the
                                        smallest search score left outside the candidate
                                        pool exceeds the k-th FP64 re-fitted score by at
                                        least 4x the largest search-score error measured on
                                        the pool (an empirical check: the outside tuples
                                        are not re-fitted) */
  uint64_t tuple_fits;               /* (task, tuple) fits evaluated */
  uint64_t fp64_fallback_tuples;     /* tuples recomputed in FP64 (mixed precision) */
  int64_t n_eligible_min;            /* smallest count of filled output slots over lists */
  double max_pool_rel_error;         /* max |SSE_gram - SSE_refit| over the pools, SSE units */
  int64_t kernel_launches;           /* library kernels launched by the last fit */
  int32_t graph_replayed;            /* 1 when the last search pass replayed a CUDA graph */
  int32_t tuned_items_factor;        /* autotuner choice: work items per CTA (at least);
                                        0 when the autotuner did not run (the untuned
                                        default is 4 for the FP32 d <= 3 kernel, else 2) */
  int32_t tuned_ctas_per_sm;         /* autotuner choice: resident CTAs per SM */
  int32_t fp64_rerun;                /* 1: the last fit was redone in FP64 after an
                                        uncertified mixed pass (see options); 2: it ran in
                                        FP64 directly because the same inputs (pointers,
                                        shapes, requests) needed FP64 on the previous call */
  /* phase times (ms, CUDA events on the handle's stream); 0 when unavailable */
  double ms_prep, ms_gram, ms_tuple, ms_merge, ms_refit, ms_total;
  double ms_tuple_kernel;            /* the tuple kernel alone (last search pass) */
  int64_t proposal_pairs;            /* pairs the pair-restricted search started from */
  int32_t tuple_kernel;              /* tuple kernel shape the last fit ran (tuple_kernel
                                        option values 0..3) */
  int32_t band_pass;                 /* MIXED: 1 when the first FP32 pass could not rank the
                                        best tuples and a band pass scored every tuple
                                        below its k-th re-fitted score + 8 delta in FP64 */
} sisso_l0_stats;

/* Fill *opt with defaults (FP64, PER_TASK, device 0, legacy stream). */
int sisso_l0_default_options(sisso_l0_options *opt);

/* Create a handle on opt->device.  *out receives the handle. */
int sisso_l0_create(sisso_l0_t *out, const sisso_l0_options *opt);

/*
 * Exhaustive l0 search (paper Sec. 2.4: score every n-tuple, return the best).
 *   X            FP64 [n_sis][n_total], feature-major (see above)
 *   y            FP64 [n_total]
 *   task_offsets host int64 [n_tasks + 1]; offsets[0] = 0, offsets[n_tasks] =
 *                n_total, every task has at least n_dim + 2 rows
 *   n_dim        tuple size, 1 .. SISSO_L0_MAX_DIM
 *   k            tuples per output list, 1 .. C(n_sis, n_dim)
 *   out_tuples   int32 [n_out][k][n_dim], ascending 0-based column indices
 *   out_rmse     FP64 [n_out][k]: sqrt(SSE_t / n_t) (PER_TASK) or
 *                sqrt(sum_t SSE_t / N) (SHARED), from an FP64 Householder
 *                re-fit on the raw centred columns
 * Lists are ordered by error, ties by the lexicographically smaller tuple.
 * Tuples whose FP64 pivot ratio is below rank_deficient_pivot_ratio are not
 * eligible; unfilled slots hold index -1 and rmse +inf.
 * Errors: EINVAL, ENOMEM, ECUDA, ETIMEOUT, ENONFINITE, EUNSUPPORTED
 * (C(n_sis, n_dim) >= 2^62 or k above 2048; the candidate pool is capped
 * at 2048).
 */
int sisso_l0_fit(sisso_l0_t h, const double *X, const double *y,
                 const int64_t *task_offsets, int32_t n_tasks, int64_t n_sis,
                 int32_t n_dim, int32_t k, int32_t *out_tuples,
                 double *out_rmse);

/* One output request of sisso_l0_fit_multi. */
typedef struct {
  int32_t n_dim;           /* tuple size, 1 .. SISSO_L0_MAX_DIM */
  int32_t k;               /* tuples per output list, 1 .. min(2048, C(n_sis, n_dim)) */
  int32_t *out_tuples;     /* [n_out][k][n_dim], device or host */
  double *out_rmse;        /* [n_out][k], device or host */
} sisso_l0_request;

/*
 * Several searches over the same data in one pass.  SISSO grows the
 * descriptor dimension over the same selected features (paper Sec. 2,
 * Fig. 1b); here every request (tuple size n_dim, list length k) of every
 * task is one problem, all problems share the centring and the Gram, and
 * their tuple spaces run in one persistent launch (tuple sizes in one call
 * must lie within a span of three, e.g. {2, 3, 4}; n_dim = 1 requests may be
 * mixed in).  Arguments X, y, task_offsets, n_tasks, n_sis as for
 * sisso_l0_fit; each request's outputs as out_tuples / out_rmse there.
 * Errors: as sisso_l0_fit; EUNSUPPORTED for tuple sizes spread wider.
 */
int sisso_l0_fit_multi(sisso_l0_t h, const double *X, const double *y,
                       const int64_t *task_offsets, int32_t n_tasks, int64_t n_sis,
                       const sisso_l0_request *reqs, int32_t n_reqs);

/* Statistics of the last fit on this handle. */
int sisso_l0_get_stats(sisso_l0_t h, sisso_l0_stats *out);

/* Replace the handle's host-side deadline (options.timeout_seconds; <= 0:
 * none) for later calls.  A call that hits the deadline returns
 * SISSO_L0_ETIMEOUT with its device work still queued on the stream; the
 * handle stays usable (the next call is ordered after that work).  (No
 * counterpart in the paper: a service-side guard.)  Errors: EINVAL (null
 * handle or NaN). */
int sisso_l0_set_timeout(sisso_l0_t h, double timeout_seconds);

/* Test hook: after `after` more device allocations made by the calling
 * thread inside the library, the next one reports out-of-memory (the call
 * returns SISSO_L0_ENOMEM) without calling cudaMalloc; after < 0 turns the
 * hook off.  The failing buffer is left empty, so a later call allocates it
 * again.  (No counterpart in the paper: it exercises the ENOMEM path without
 * exhausting a shared GPU.)  Always returns SISSO_L0_OK. */
int sisso_l0_debug_fail_allocation(int64_t after);

/* Description of the last error on this handle (valid until the next call
 * on the handle); a static string when h is NULL. */
const char *sisso_l0_last_error(sisso_l0_t h);

/* Synchronise the handle's stream and free everything it owns.  NULL-safe. */
void sisso_l0_destroy(sisso_l0_t h);

/*
 * Number of n-tuples of m features, C(m, n) (paper Sec. 3.1 counts its l0
 * models this way).  Returns 0 when it does not fit in 63 bits.  Host-only.
 */
uint64_t sisso_l0_count_tuples(int64_t m, int32_t n);

/*
 * Diagnostic: lexicographic rank <-> tuple, as the device code computes it
 * (tuples of n ascending indices out of m, rank 0 = (0, 1, .., n-1)).
 * Runs on the handle's device; ranks/tuples are host arrays of count
 * entries.  Used by the tests to check the enumeration against an
 * independent enumerator.
 */
int sisso_l0_debug_unrank(sisso_l0_t h, int64_t m, int32_t n,
                          const uint64_t *ranks, int64_t count,
                          int32_t *tuples_out);

/*
 * Diagnostic: the per-task augmented correlation matrix the tuple kernel
 * reads, for task `task`: out[(m+1) x (m+1)] FP64 host array, index 0 the
 * target, index j+1 feature j; entries (a, b) with a <= b are filled.
 */
int sisso_l0_debug_gram(sisso_l0_t h, const double *X, const double *y,
                        const int64_t *task_offsets, int32_t n_tasks,
                        int64_t n_sis, int32_t task, double *out);

/*
 * Augmented correlation matrix of one task without allocating memory.
 * (The paper has no counterpart: this serves callers that cannot allocate
 * device memory while they run -- a service whose device memory is reserved
 * up front for its own allocator, or a latency-bound loop that cannot take
 * the device-wide synchronisation of cudaMalloc/cudaFree.)
 *   X         device FP64 [n_sis][n_samples], feature-major, one task
 *   y         device FP64 [n_samples]
 *   out_gram  device FP64, row-major with leading dimension ld_out >= n_sis+1;
 *             entries (a, b), a <= b < n_sis+1, receive what
 *             sisso_l0_debug_gram returns for the same data (index 0 the
 *             target, j+1 feature j); every other entry (a > b, and the
 *             columns past n_sis) is left untouched
 *   stream    cudaStream_t (NULL = legacy stream); the call returns after
 *             the stream has finished its work
 * Scratch lives in a fixed 16 MiB array inside the library (held by every
 * GPU that loads the library until the process exits), so
 * (n_sis+1) * n_samples + 2 (n_sis+1) + 3 must not exceed 2^21 doubles;
 * larger inputs (including sizes whose product would overflow 64 bits)
 * return SISSO_L0_EUNSUPPORTED before any work is queued.  The first call on a device
 * looks up the array's device address for that device (the current device).
 * All calls share the array: calls that overlap on the GPU race and must be
 * serialised by the caller.  Calls no cudaMalloc, cudaFree or other
 * allocating routine.  Errors: EINVAL, EUNSUPPORTED, ENONFINITE, ECUDA.
 */
int sisso_l0_gram_noalloc(const double *X, const double *y, int64_t n_samples,
                          int64_t n_sis, double *out_gram, int64_t ld_out,
                          void *stream);

/* ------------------------------------------------ learned proposals ----
 * The paper's l0 step scores every n-tuple exhaustively (Sec. 2.4).  The
 * learned form of the d = 3 search ranks the (d-1)-subsets -- pairs of
 * features -- with a small network trained on the exhaustive search's own
 * results, and fits exactly only the triples reachable from the best pairs;
 * the exhaustive search stays the reference and measures the network's
 * recall.  Pairs are ranked in colex order: rank(i, j) = j (j - 1) / 2 + i,
 * i < j.
 *
 * Network: 6 -> 256 -> 256 -> 1, ReLU, inputs per pair (i, j) (from the
 * task's correlation matrix): r_i, r_j (Pearson r, Eq. 1), C_ij = corr(f_i,
 * f_j), rho_j.i = corr(f_j, residual of y after the fit on f_i), rho_i.j, and
 * log(1 - R2_ij) / 8 of the two-feature fit.  Target: log(min over k of
 * SSE(i, j, k) / S_yy), clamped to [log 1e-12, 0] (0 when no completion is
 * eligible).
 * BF16 operands (features, W1, W2, w3, h1, h2 and the back-propagated dh2),
 * FP32 sums and FP32 master weights; squared-error loss, Adam (beta1 0.9,
 * beta2 0.999, eps 1e-8).  Parameters, flat FP32, SISSO_L0_SCORER_PARAMS
 * floats: W1 [256][6] | b1 [256] | W2 [256][256] (row = output unit) |
 * b2 [256] | w3 [256] | b3.
 */
#define SISSO_L0_SCORER_PARAMS 67841
#define SISSO_L0_PAIR_FEATURES_LD 8   /* floats per feature row (6 used) */

typedef struct sisso_l0_scorer *sisso_l0_scorer_t;

/* New scorer on `device`: He-uniform weights drawn from splitmix64(seed),
 * zero biases.  The scorer owns its device memory and stream.  Errors:
 * EINVAL, ENOMEM, ECUDA. */
int sisso_l0_scorer_create(sisso_l0_scorer_t *out, int32_t device, uint64_t seed);
void sisso_l0_scorer_destroy(sisso_l0_scorer_t s);   /* NULL-safe, syncs first */
const char *sisso_l0_scorer_last_error(sisso_l0_scorer_t s);

/* Copy the flat parameter vector in (host or device; resets Adam) or out.
 * n must be SISSO_L0_SCORER_PARAMS. */
int sisso_l0_scorer_set_params(sisso_l0_scorer_t s, const float *params, int64_t n);
int sisso_l0_scorer_get_params(sisso_l0_scorer_t s, float *params, int64_t n);

/* Mean squared error of the network over n_rows rows and its gradient, no
 * update.  feats: device [n_rows][8], labels: device [n_rows]; loss (1 float)
 * and grad (SISSO_L0_SCORER_PARAMS floats) may be host or device, or NULL. */
int sisso_l0_scorer_loss_grad(sisso_l0_scorer_t s, const float *feats, const float *labels,
                              int64_t n_rows, float *loss, float *grad);

/* `steps` Adam steps with learning rate lr on consecutive windows of
 * batch_rows rows (wrapping around the data); losses (steps floats, host or
 * device, or NULL) receive each step's loss before its update. */
int sisso_l0_scorer_train(sisso_l0_scorer_t s, const float *feats, const float *labels,
                          int64_t n_rows, int32_t batch_rows, int32_t steps, float lr,
                          float *losses);

/* Network outputs (predicted log best completion) of n_rows feature rows;
 * feats and out are device pointers. */
int sisso_l0_scorer_predict(sisso_l0_scorer_t s, const float *feats, int64_t n_rows, float *out);

/* Training data of one task (single task, mixed precision handle): the
 * features of every pair in colex order into feats (device,
 * [C(n_sis, 2)][8]) and, when labels is not NULL, every pair's target
 * (device, [C(n_sis, 2)]), both from the FP32 tensor-core Gram.  With
 * standardize != 0 the labels are z-scored over the task's pairs (only a
 * pair's rank within its task matters to the search).  X, y as in
 * sisso_l0_fit with one task of n_total rows. */
int sisso_l0_pair_data(sisso_l0_t h, const double *X, const double *y, int64_t n_total,
                       int64_t n_sis, float *feats, float *labels, int32_t standardize);

/* Exact d = 3 search over the triples {i, j, k} reachable from a pair list
 * (host or device, int32 [n_pairs][2], any order within a pair, repeats
 * allowed), each triple fitted once, then the FP64 re-fit and ranking of
 * sisso_l0_fit; outputs as sisso_l0_fit with n_dim = 3, one task.  An index
 * outside [0, n_sis) or i == j gives EINVAL. */
int sisso_l0_fit_pairs(sisso_l0_t h, const double *X, const double *y, int64_t n_total,
                       int64_t n_sis, const int32_t *pairs, int64_t n_pairs, int32_t k,
                       int32_t *out_tuples, double *out_rmse);

/* Learned d = 3 search: the scorer ranks every pair (inference fused with
 * the features, on the tensor cores), the pairs in the lowest score bins
 * holding at least ceil(fraction * C(n_sis, 2)) pairs are kept, and the
 * search of sisso_l0_fit_pairs runs over them.  Mixed-precision, single-task
 * handle; get_stats reports proposal_pairs and the triples fitted. */
int sisso_l0_fit_learned(sisso_l0_t h, sisso_l0_scorer_t s, const double *X, const double *y,
                         int64_t n_total, int64_t n_sis, int32_t k, double fraction,
                         int32_t *out_tuples, double *out_rmse);

/* ---------------------------------------------------------- sharding ----
 * One search split over n_shards workers (one GPU each).  The tuples are
 * independent (the paper spreads descriptors over devices and gathers the
 * selected models at the end, Sec. 3.2.1): shard s searches every n-th work
 * item (a chunk of prefixes of one tile of the tuple space), so the shards'
 * tuple sets are disjoint and cover all C(n_sis, n_dim) tuples.  Each shard
 * returns its FP64 re-fitted candidate pool; the pools are the only data
 * exchanged (an all-gather of at most SISSO_L0_MAX_POOL candidates per
 * shard), and sisso_l0_merge_shards ranks their union. */
#define SISSO_L0_MAX_POOL 2048

/* One shard of a single-task search (n_dim >= 2).  Outputs (host or device):
 * out_keys / out_sse [SISSO_L0_MAX_POOL], the first *out_count valid: the
 * lexicographic ranks and exact SSEs (FP64 re-fit; +inf when rank
 * deficient) of the shard's candidates; *out_bound: every tuple of the shard
 * outside them has an SSE of at least out_bound - 4 * out_delta. */
int sisso_l0_fit_shard(sisso_l0_t h, const double *X, const double *y, int64_t n_total,
                       int64_t n_sis, int32_t n_dim, int32_t k, int32_t shard, int32_t n_shards,
                       uint64_t *out_keys, double *out_sse, int32_t *out_count,
                       double *out_bound, double *out_delta);

/* Rank the union of the shards' candidates (host or device arrays, n_cand
 * entries, any order): the k best by (SSE, lexicographic rank) as tuples and
 * RMSE = sqrt(SSE / n_total), -1 / +inf padded; *certified = 1 when every
 * shard's bound - 4 delta clears the k-th SSE (the union then holds the exact
 * top k of the whole search). */
int sisso_l0_merge_shards(sisso_l0_t h, int64_t n_sis, int32_t n_dim, int32_t k, int64_t n_total,
                          const uint64_t *keys, const double *sse, int64_t n_cand,
                          const double *bounds, const double *deltas, int32_t n_shards,
                          int32_t *out_tuples, double *out_rmse, int32_t *certified);

/* SIS screening, the step before l0 (paper Sec. 2.3): the Pearson r (Eq. 1)
 * of every candidate feature with y and the m features of largest |r|
 * (ties: the smaller index), in that order.  X: FP64 feature-major
 * [n_feat][n_total] (host or device), y: [n_total]; outputs out_idx int32
 * [m] and out_r (the signed r) [m], host or device.  One pass over X.  An
 * FP64 handle computes every r in FP64.  A mixed-precision handle gives the
 * same output with a pre-screen: each sample truncated to FP32 by integer
 * operations, FP32 sums, and a rigorous interval around each |r|; only the
 * features whose interval reaches the m-th largest lower bound are re-scored
 * by the FP64 routine (no FP64 operation per sample elsewhere).  get_stats
 * then reports fp64_fallback_tuples = features scored in FP64, ms_total,
 * ms_tuple_kernel = the scan kernel alone (pre-screen or FP64 score) and
 * kernel_launches.  Errors: EINVAL (n_total < 2, m outside
 * [1, n_feat]), EUNSUPPORTED (m > 65536, n_feat >= 2^32, or more than 2^22
 * features tied at the selection cut), ENONFINITE, ENOMEM, ECUDA. */
int sisso_l0_sis(sisso_l0_t h, const double *X, const double *y, int64_t n_total,
                 int64_t n_feat, int32_t m, int32_t *out_idx, double *out_r);

/* SIS against several targets (paper Sec. 2: from the second dimension on,
 * the projection score is taken against the residuals of the previous
 * models; Sec. 3 uses ten residuals per SIS iteration).  A feature's score
 * is max_t |r(x, Y[t])| (Eq. 1); out_r holds the signed r of the first
 * target reaching it.  The n_exclude features listed in `exclude` (distinct
 * indices, host or device int32) are never selected.  Y: FP64
 * [n_targets][n_total], host or device, 1 <= n_targets <= 16; the rest as in
 * sisso_l0_sis.  The pre-screen (mixed handle) makes one pass over X per
 * target and takes the largest bounds; the FP64 re-score reads each
 * candidate once for all targets.  Errors: EINVAL (also m > n_feat -
 * n_exclude, repeated or out-of-range exclusions), as sisso_l0_sis. */
int sisso_l0_sis_multi(sisso_l0_t h, const double *X, const double *Y, int32_t n_targets,
                       int64_t n_total, int64_t n_feat, int32_t m, const int32_t *exclude,
                       int64_t n_exclude, int32_t *out_idx, double *out_r);

/* Operators of on-the-fly feature generation (paper Sec. 3's set). */
enum {
  SISSO_L0_OP_ADD = 0, SISSO_L0_OP_SUB = 1, SISSO_L0_OP_MUL = 2, SISSO_L0_OP_DIV = 3,
  SISSO_L0_OP_ABS_DIFF = 4, SISSO_L0_OP_LOG = 5, SISSO_L0_OP_EXP = 6, SISSO_L0_OP_NEG_EXP = 7,
  SISSO_L0_OP_ABS = 8, SISSO_L0_OP_SQRT = 9, SISSO_L0_OP_CBRT = 10, SISSO_L0_OP_SQ = 11,
  SISSO_L0_OP_CUBE = 12, SISSO_L0_OP_INV = 13
};

/* SIS over generated features that are never stored (paper Sec. 2: the
 * operators applied to child features, their values evaluated and checked
 * on the GPU; the last rung evaluated inside SIS, Sec. 2.3, Sec. 3).
 * Candidate t is ops[t](C[c1[t]], C[c2[t]]) -- codes 0-4 binary, 5-13
 * unary on c1[t] (c2[t] ignored) -- evaluated in FP64.  On a handle of
 * precision MIXED_BF16X3 and with out_valid NULL, every candidate is first
 * evaluated in FP32 with a rigorous interval around its |r| (per-sample
 * bounds on the FP32 values from the operators' rounding and CUDA's
 * documented accuracy of logf / expf / cbrtf) and only the candidates whose
 * interval reaches the m-th largest lower bound of a certainly valid one are
 * evaluated in FP64: the result is the FP64 evaluation's.  A candidate is valid
 * when every value is finite, max |value| lies in [l_bound, u_bound], the
 * values are not all equal and not equal sample by sample to a child; the m
 * valid candidates of largest |r| with y (Eq. 1) are returned, ties to the
 * smaller candidate index, -1 (and r = 0) past the valid count.
 *   C     FP64 [n_child][n_total] child values (host or device)
 *   ops, c1, c2  int32 [n_cand] (host or device)
 *   y     FP64 [n_total]
 *   out_idx int32 [m], out_r FP64 [m] (host or device)
 *   out_valid uint8 [n_cand] (optional, host or device): 1 valid, 0 not
 * Errors: EINVAL (also an operator code or child index out of range,
 * detected on the device), ENONFINITE (y), EUNSUPPORTED (m > 65536,
 * n_cand >= 2^32), ENOMEM, ECUDA. */
int sisso_l0_sis_generated(sisso_l0_t h, const double *C, int64_t n_child, int64_t n_total,
                           const int32_t *ops, const int32_t *c1, const int32_t *c2,
                           int64_t n_cand, const double *y, int32_t m, double l_bound,
                           double u_bound, int32_t *out_idx, double *out_r,
                           uint8_t *out_valid);

/* Residuals y - (b_0 + sum_a b_a x_{t_a}) of the least-squares fits with
 * intercept (Sec. 2.4) of n_models models of n_dim features each.
 * tuples: int32 [n_models][n_dim] feature indices into X (host or device);
 * X as in sisso_l0_sis; out: FP64 [n_models][n_total], host or device.  FP64
 * Gram-Schmidt with a second orthogonalisation pass; a column dependent on
 * the earlier ones (norm below 1e-12 of its centred norm after projection)
 * is dropped, which leaves the residual of the minimum-norm fit.  Errors:
 * EINVAL (1 <= n_dim <= 8, indices in range), ENOMEM, ECUDA. */
int sisso_l0_residuals(sisso_l0_t h, const double *X, const double *y, int64_t n_total,
                       int64_t n_feat, const int32_t *tuples, int32_t n_dim, int32_t n_models,
                       double *out);

/* The dimension loop of descriptor identification (Sec. 2, Fig. 1b): for
 * n = 1 .. n_dim_max, screen m new features (n = 1: against y; n > 1:
 * against the residuals of the min(n_res, eligible) best (n-1)-dimensional
 * models, never re-selecting a feature), append them to the subspace S, and
 * run the exhaustive l0 search of every n-tuple of S (single task, the
 * handle's precision).  Outputs (host arrays): out_S int32 [n_dim_max * m],
 * the features in selection order; out_tuples int32
 * [n_dim_max][k][n_dim_max], row n-1 holding the k best n-tuples as
 * ascending global feature indices (entries past n and unfilled slots -1);
 * out_rmse FP64 [n_dim_max][k] (+inf where unfilled).  X, y host or device
 * (host inputs are copied to the device once).  Errors: EINVAL
 * (1 <= n_dim_max <= 6, 1 <= n_res <= 16, m n_dim_max <= n_feat,
 * n_total >= n_dim_max + 2), and those of sisso_l0_sis_multi and
 * sisso_l0_fit.  get_stats then reports the last l0 search, except
 * kernel_launches, which counts the whole loop. */
int sisso_l0_dimension_loop(sisso_l0_t h, const double *X, const double *y, int64_t n_total,
                            int64_t n_feat, int32_t m, int32_t n_dim_max, int32_t k,
                            int32_t n_res, int32_t *out_S, int32_t *out_tuples,
                            double *out_rmse);

/* Measured rates of the units the l0 kernels are bound by, on `device`
 * (microbenchmarks, CUDA events, a few tens of milliseconds; no paper
 * counterpart): out[0] FP32 FMA TFLOP/s, out[1] FP64 FMA TFLOP/s, out[2]
 * MUFU rsqrt Gop/s, out[3] shared-memory load GB/s, out[4] L2 load GB/s.
 * Allocates 33 MB of scratch for the call.  Errors: EINVAL, ENOMEM, ECUDA. */
int sisso_l0_measure_peaks(int32_t device, double *out);

#ifdef __cplusplus
}
#endif

#endif /* SISSO_L0_H */
