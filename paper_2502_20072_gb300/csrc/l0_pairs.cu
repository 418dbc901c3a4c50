// l0_pairs.cu -- pair-level kernels of the learned d = 3 search.
//
// The exhaustive l0 step fits every triple (paper Sec. 2.4).  The learned form
// fits only the triples reachable from the best-ranked pairs:
//   * gram_mirror: the FP32 Gram made symmetric (row reads for any k) and its
//     diagonal made contiguous;
//   * pair_features: the network inputs of every pair;
//   * pair_best: the training label of a pair, its best completion
//     min_k SSE(i, j, k) / S_yy (one warp per pair, lanes over k);
//   * select_pairs: the pairs with the lowest network scores (a histogram of
//     the scores' ordered bits, a one-block scan for the cut bin, a compaction
//     that also sets a bitmap over pair ranks);
//   * proposal_kernel: the exact FP32 search over the triples {i, j, k} of
//     the selected pairs, each triple fitted once -- from the first selected
//     pair of its three in colex order -- with the CTA top-K' lists, the
//     global score-histogram cut and the FP64 redo queue of the exhaustive
//     search, so that merge, FP64 re-fit and selection are shared with it.
#include <algorithm>

#include "l0_kernels.cuh"

namespace l0 {

namespace {

// ------------------------------------------------------------- mirror --
template <typename T>
__global__ void __launch_bounds__(256)
gram_mirror_kernel(T *G, long long ld, int mp1, T *diag) {
  __shared__ T tile[32][33];
  const int bx = blockIdx.x, by = blockIdx.y;   // source tile (row block by, col block bx), by <= bx
  if (by > bx) return;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  for (int r = ty; r < 32; r += 8) {
    const int row = by * 32 + r, col = bx * 32 + tx;
    if (row < mp1 && col < mp1) tile[r][tx] = G[(long long)row * ld + col];
  }
  __syncthreads();
  for (int r = ty; r < 32; r += 8) {
    const int row = bx * 32 + r, col = by * 32 + tx;   // destination (lower triangle)
    if (row < mp1 && col < mp1 && row > col) G[(long long)row * ld + col] = tile[tx][r];
  }
  if (by == bx && ty == 0) {
    const int c = bx * 32 + tx;
    if (c >= 1 && c < mp1) diag[c - 1] = tile[tx][tx];
  }
}

// ----------------------------------------------------------- features --
__device__ __forceinline__ void pair_of_rank(long long p, int &i, int &j) {
  long long jj = (long long)((1.0 + sqrt(1.0 + 8.0 * (double)p)) * 0.5);
  while (jj * (jj - 1) / 2 > p) --jj;
  while ((jj + 1) * jj / 2 <= p) ++jj;
  j = (int)jj;
  i = (int)(p - jj * (jj - 1) / 2);
}

__global__ void __launch_bounds__(256)
pair_features_kernel(const float *G, long long ld, long long p0, long long n, float *feats) {
  const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n) return;
  int i, j;
  pair_of_rank(p0 + q, i, j);
  float x[MLP_NIN];
  pair_feature_vec(G, ld, i, j, x);
  float4 *dst = reinterpret_cast<float4 *>(feats + q * MLP_FEAT_LD);
  dst[0] = make_float4(x[0], x[1], x[2], x[3]);
  dst[1] = make_float4(x[4], x[5], 0.f, 0.f);
}

// -------------------------------------------------- best completion --
// Augmented Cholesky of the pair (i, j) and the target, then per third
// column k the last pivot SSE / S_yy = pP - w^2 / p_k (Schur complement).
__global__ void __launch_bounds__(256)
pair_best_kernel(const float *G, long long ld, const float *diag, int m, long long n_pairs,
                 float ratio, float floor_, float *label) {
  const long long q = (long long)blockIdx.x * 8 + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (q >= n_pairs) return;
  int i, j;
  pair_of_rank(q, i, j);
  const float *Gi = G + (long long)(i + 1) * ld + 1, *Gj = G + (long long)(j + 1) * ld + 1;
  const float *cy = G + 1;
  const float g00 = G[0], gii = diag[i], gjj = diag[j], gij = Gi[j];
  const float l11 = sqrtf(fmaxf(gii, 1e-30f)), il11 = 1.f / l11;
  const float l21 = gij * il11, d2 = gjj - l21 * l21;
  const bool pair_ok = gii > 0.f && gjj > 0.f && d2 >= ratio * gjj;
  const float il22 = 1.f / sqrtf(fmaxf(d2, 1e-30f));
  const float z1 = cy[i] * il11, z2 = (cy[j] - l21 * z1) * il22;
  const float pP = g00 - z1 * z1 - z2 * z2;
  float best = 1.f;
  if (pair_ok) {
    for (int k = lane; k < m; k += 32) {
      if (k == i || k == j) continue;
      const float gkk = diag[k];
      const float g1 = Gi[k] * il11, g2 = (Gj[k] - l21 * g1) * il22;
      const float pk = gkk - g1 * g1 - g2 * g2;
      if (!(gkk > 0.f) || !(pk >= ratio * gkk)) continue;
      const float w = cy[k] - g1 * z1 - g2 * z2;
      best = fminf(best, pP - w * w / pk);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) best = fminf(best, __shfl_xor_sync(0xffffffffu, best, o));
  if (lane == 0) label[q] = logf(fminf(fmaxf(best, floor_), 1.f));
}

// z-score of one task's labels (mean and standard deviation in FP64): the
// training target is the instance-relative rank of a pair's completion
__global__ void __launch_bounds__(256)
label_moments_kernel(const float *lab, long long n, double *acc) {
  double s = 0.0, q = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const double v = lab[i];
    s += v;
    q += v * v;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    s += __shfl_xor_sync(0xffffffffu, s, o);
    q += __shfl_xor_sync(0xffffffffu, q, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(acc, s);
    atomicAdd(acc + 1, q);
  }
}

__global__ void __launch_bounds__(256)
label_normalize_kernel(float *lab, long long n, const double *acc) {
  const double mean = acc[0] / (double)n;
  const double var = acc[1] / (double)n - mean * mean;
  const float inv = (float)(1.0 / sqrt(var > 1e-12 ? var : 1e-12));
  const float mu = (float)mean;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    lab[i] = (lab[i] - mu) * inv;
}

// ---------------------------------------------------------- selection --
constexpr int SEL_SHIFT = 12;                  // 2^20 bins of the ordered score bits
constexpr int SEL_BINS = 1 << (32 - SEL_SHIFT);

__device__ __forceinline__ unsigned ord32(float x) {
  const unsigned b = __float_as_uint(x);
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

__global__ void __launch_bounds__(256)
score_hist_kernel(const float *score, long long n, unsigned *hist) {
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n;
       q += (long long)gridDim.x * blockDim.x) {
    const float s = score[q];
    if (s == s) atomicAdd(hist + (ord32(s) >> SEL_SHIFT), 1u);
  }
}

// one block of 1024: the smallest bin b with count(bins <= b) >= want
__global__ void __launch_bounds__(1024)
cut_bin_kernel(const unsigned *hist, long long want, unsigned *bin_out) {
  __shared__ unsigned long long part[1024];
  __shared__ unsigned s_bin;
  const int tid = threadIdx.x;
  constexpr int PER = SEL_BINS / 1024;
  unsigned long long s = 0;
  for (int b = 0; b < PER; ++b) s += hist[tid * PER + b];
  part[tid] = s;
  if (tid == 0) s_bin = SEL_BINS - 1;
  __syncthreads();
  for (int o = 1; o < 1024; o <<= 1) {   // inclusive scan
    unsigned long long v = (tid >= o) ? part[tid - o] : 0ull;
    __syncthreads();
    part[tid] += v;
    __syncthreads();
  }
  const unsigned long long before = tid ? part[tid - 1] : 0ull;
  if (before < (unsigned long long)want && part[tid] >= (unsigned long long)want) {
    unsigned long long acc = before;
    for (int b = 0; b < PER; ++b) {
      acc += hist[tid * PER + b];
      if (acc >= (unsigned long long)want) { s_bin = tid * PER + b; break; }
    }
  }
  __syncthreads();
  if (tid == 0) *bin_out = s_bin;
}

__global__ void __launch_bounds__(256)
compact_pairs_kernel(const float *score, long long n, const unsigned *bin, int *pairs,
                     unsigned long long *counter, unsigned *bits) {
  const unsigned cut = *bin;
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n;
       q += (long long)gridDim.x * blockDim.x) {
    const float s = score[q];
    if (!(s == s) || (ord32(s) >> SEL_SHIFT) > cut) continue;
    int i, j;
    pair_of_rank(q, i, j);
    const unsigned long long slot = atomicAdd(counter, 1ull);
    pairs[2 * slot] = i;
    pairs[2 * slot + 1] = j;
    atomicOr(bits + (q >> 5), 1u << (q & 31));
  }
}

__global__ void __launch_bounds__(256)
pairs_from_list_kernel(const int *in, long long n, int m, int *pairs, unsigned *bits, int *err) {
  const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n) return;
  int a = in[2 * q], b = in[2 * q + 1];
  if (a > b) { const int t = a; a = b; b = t; }
  if (a < 0 || b >= m || a == b) {
    set_err(err, 11);
    a = 0;
    b = 1;
  }
  const long long r = (long long)b * (b - 1) / 2 + a;
  const unsigned old = atomicOr(bits + (r >> 5), 1u << (r & 31));
  if (old & (1u << (r & 31))) a = b = -1;   // repeated pair: fitted through its other copy
  pairs[2 * q] = a;
  pairs[2 * q + 1] = b;
}

// ------------------------------------------------------ proposal search --
__device__ __forceinline__ bool selected(const unsigned *bits, int x, int y) {   // x < y
  const long long r = (long long)y * (y - 1) / 2 + x;
  return (__ldg(bits + (r >> 5)) >> (r & 31)) & 1u;
}

template <typename R>
__device__ __forceinline__ void defer_one(const PropArgs<R> &A, u64 key) {
  atomicAdd(A.dfr_n + 1, 1ull);
  const u64 slot = atomicAdd(A.dfr_n, 1ull);
  if ((long long)slot < A.dfr_cap) {
    A.dfr_key[slot] = key;
    A.dfr_len[slot] = 1u;   // problem 0, one tuple
  } else {
    set_err(A.err, 7);
  }
}

constexpr int PROP_THREADS = 256;
constexpr int PROP_U = 8;   // third columns per lane per round

template <typename R>
__global__ void __launch_bounds__(PROP_THREADS, 2)
proposal_kernel(PropArgs<R> A) {
  extern __shared__ __align__(16) unsigned char smem[];
  unsigned char *p = smem;
  CtaList<R> L = cta_list_carve<R>(p, A.K, A.S);
  __shared__ long long s_base;
  const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
  constexpr bool MIXED = sizeof(R) == 4;
  cta_list_reset<R>(L, A.gthr);
  L.hist = A.hist;
  __syncthreads();
  u64 fits = 0;
  u64 gnext = ~0ull;
  for (;;) {
    if (tid == 0) s_base = (long long)atomicAdd(A.pair_ctr, (u64)(PROP_THREADS / 32));
    __syncthreads();
    const long long base = s_base;
    __syncthreads();
    if (base >= A.n_pairs) break;   // uniform
    const long long q = base + w;
    int pi = 0, pj = 1;
    bool has = q < A.n_pairs;
    if (has) {
      pi = A.pairs[2 * q];
      pj = A.pairs[2 * q + 1];
      if (pi < 0) { has = false; pi = 0; pj = 1; }
    }
    const R *Gi = A.G + (long long)(pi + 1) * A.ld + 1, *Gj = A.G + (long long)(pj + 1) * A.ld + 1;
    const R *cy = A.G + 1;
    const R g00 = A.G[0], gii = A.diag[pi], gjj = A.diag[pj], gij = Gi[pj];
    const R l11 = sqrt(gii > R(0) ? gii : R(1)), il11 = R(1) / l11;
    const R l21 = gij * il11, d2 = gjj - l21 * l21;
    const bool pair_ok = gii > R(0) && gjj > R(0) && d2 >= (R)A.ratio * gjj;
    // a pair of one duplicate class: all its triples are rank deficient
    const bool pair_dup = A.cls && A.cls[pi] == A.cls[pj];
    const R il22 = R(1) / sqrt(d2 > R(0) ? d2 : R(1));
    const R z1 = cy[pi] * il11, z2 = (cy[pj] - l21 * z1) * il22;
    const R pP = g00 - z1 * z1 - z2 * z2;
    for (int k0 = 0; k0 < A.m; k0 += 32 * PROP_U) {
      const u64 gprev = gnext;
      if (tid < 32) gnext = ld_relaxed(A.gthr);
      unsigned done = 0u;
      // all loads of the round first (no branches between them), so that the
      // lane has its 8 columns' Gram entries and bitmap words in flight at once
      R ld_gi[PROP_U], ld_gj[PROP_U], ld_gk[PROP_U], ld_cy[PROP_U];
      unsigned ld_w1[PROP_U], ld_w2[PROP_U];
      int ld_cl[PROP_U];
#pragma unroll
      for (int u = 0; u < PROP_U; ++u) {
        const int k = k0 + u * 32 + lane;
        const int kc = k < A.m ? k : A.m - 1;
        ld_gi[u] = Gi[kc];
        ld_gj[u] = Gj[kc];
        ld_gk[u] = A.diag[kc];
        ld_cy[u] = cy[kc];
        ld_cl[u] = A.cls ? __ldg(A.cls + kc) : kc;
        // bitmap words: (k, pi) and (k, pj) when k < pi; (pi, k) when pi < k < pj
        const int a1 = kc < pi ? kc : pi, b1 = kc < pi ? pi : (kc > pi ? kc : pi + 1);
        const long long r1 = (long long)b1 * (b1 - 1) / 2 + a1;
        const long long r2 = (long long)pj * (pj - 1) / 2 + (kc < pj ? kc : 0);
        ld_w1[u] = __ldg(A.bits + (r1 >> 5)) >> (r1 & 31);
        ld_w2[u] = __ldg(A.bits + (r2 >> 5)) >> (r2 & 31);
      }
      const int cpi = A.cls ? __ldg(A.cls + pi) : pi, cpj = A.cls ? __ldg(A.cls + pj) : pj;
      for (int pass = 0;; ++pass) {
        const R cut = cta_cut<R>(L);
#pragma unroll
        for (int u = 0; u < PROP_U; ++u) {
          const int k = k0 + u * 32 + lane;
          const unsigned bit = 1u << u;
          if (!has || k >= A.m || k == pi || k == pj || (done & bit)) continue;
          int t[3];
          bool eval;
          if (k < pi) {
            eval = !(ld_w1[u] & 1u) && !(ld_w2[u] & 1u);
            t[0] = k; t[1] = pi; t[2] = pj;
          } else if (k < pj) {
            eval = !(ld_w1[u] & 1u);
            t[0] = pi; t[1] = k; t[2] = pj;
          } else {
            eval = true;
            t[0] = pi; t[1] = pj; t[2] = k;
          }
          if (!eval) { done |= bit; continue; }
          if (pass == 0) ++fits;
          if (pair_dup || ld_cl[u] == cpi || ld_cl[u] == cpj) {
            done |= bit;   // two columns of one duplicate class: ineligible
            continue;
          }
          const R gkk = ld_gk[u];
          const R g1 = ld_gi[u] * il11, g2 = (ld_gj[u] - l21 * g1) * il22;
          const R pk = gkk - g1 * g1 - g2 * g2;
          if (!pair_ok || !(gkk > R(0)) || !(pk >= (R)A.ratio * gkk)) {
            // near-singular in FP32: exact FP64 redo; in FP64: ineligible
            if (MIXED) defer_one<R>(A, lex_rank(A.B, A.m, 3, t, A.total));
            done |= bit;
            continue;
          }
          const R wv = ld_cy[u] - g1 * z1 - g2 * z2;
          const R rel = pP - wv * wv / pk;
          if (rel > cut) { done |= bit; continue; }
          const u64 key = lex_rank(A.B, A.m, 3, t, A.total);
          if (!cta_list_admits<R>(L, rel, key) || cta_list_push<R>(L, rel, key)) done |= bit;
        }
        __syncthreads();
        const bool ovf = *(volatile int *)L.ovf != 0;
        if (ovf || *(volatile int *)L.n_stage > L.S / 2) cta_list_commit<R>(L, A.gthr);
        if (!ovf) break;
        if (pass > L0_MAX_REDO) {
          set_err(A.err, 8);
          break;
        }
      }
      cta_step_sync<R>(L, A.gthr, gprev);
    }
  }
  __syncthreads();
  cta_list_commit<R>(L, A.gthr);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) fits += __shfl_xor_sync(0xffffffffu, fits, o);
  if (lane == 0 && fits) atomicAdd(A.fits, fits);
  cta_list_flush<R>(L, A.out_s + (size_t)blockIdx.x * A.K, A.out_k + (size_t)blockIdx.x * A.K,
                    A.out_cnt + blockIdx.x);
}

}  // namespace

template <typename T>
cudaError_t launch_gram_mirror(T *G, long long ld, int mp1, T *diag, cudaStream_t st) {
  const int nb = (mp1 + 31) / 32;
  gram_mirror_kernel<T><<<dim3(nb, nb), 256, 0, st>>>(G, ld, mp1, diag);
  return cudaGetLastError();
}
template cudaError_t launch_gram_mirror<float>(float *, long long, int, float *, cudaStream_t);
template cudaError_t launch_gram_mirror<double>(double *, long long, int, double *, cudaStream_t);

cudaError_t launch_pair_features(const float *G, long long ld, long long p0, long long n,
                                 float *feats, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  pair_features_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(G, ld, p0, n, feats);
  return cudaGetLastError();
}

cudaError_t launch_pair_best(const float *G, long long ld, const float *diag, int m,
                             long long n_pairs, double ratio, float floor_, float *label,
                             cudaStream_t st) {
  if (n_pairs <= 0) return cudaSuccess;
  pair_best_kernel<<<(unsigned)((n_pairs + 7) / 8), 256, 0, st>>>(G, ld, diag, m, n_pairs,
                                                                  (float)ratio, floor_, label);
  return cudaGetLastError();
}

cudaError_t launch_label_standardize(float *lab, long long n, double *acc, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(acc, 0, 16, st);
  if (e != cudaSuccess) return e;
  const unsigned g = (unsigned)std::min<long long>((n + 255) / 256, 152 * 8);
  label_moments_kernel<<<g, 256, 0, st>>>(lab, n, acc);
  label_normalize_kernel<<<g, 256, 0, st>>>(lab, n, acc);
  return cudaGetLastError();
}

cudaError_t launch_select_pairs(const float *score, long long n_pairs, long long want,
                                unsigned *hist, unsigned *bin_out, int *pairs,
                                unsigned long long *counter, unsigned *bits, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(hist, 0, (size_t)SEL_BINS * 4, st);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(counter, 0, 8, st);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(bits, 0, (size_t)((n_pairs + 31) / 32) * 4, st);
  if (e != cudaSuccess) return e;
  const unsigned g = (unsigned)std::min<long long>((n_pairs + 255) / 256, 152 * 16);
  score_hist_kernel<<<g, 256, 0, st>>>(score, n_pairs, hist);
  cut_bin_kernel<<<1, 1024, 0, st>>>(hist, want, bin_out);
  compact_pairs_kernel<<<g, 256, 0, st>>>(score, n_pairs, bin_out, pairs, counter, bits);
  return cudaGetLastError();
}

cudaError_t launch_pairs_from_list(const int *in, long long n, int m, int *pairs, unsigned *bits,
                                   int *err, cudaStream_t st) {
  const long long np = (long long)m * (m - 1) / 2;
  cudaError_t e = cudaMemsetAsync(bits, 0, (size_t)((np + 31) / 32) * 4, st);
  if (e != cudaSuccess || n <= 0) return e;
  pairs_from_list_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(in, n, m, pairs, bits, err);
  return cudaGetLastError();
}

template <typename R>
size_t proposal_smem_bytes(int K, int S) {
  return cta_list_bytes<R>(K, S) + 16;
}

template <typename R>
cudaError_t proposal_occupancy(int K, int S, int *blocks_per_sm) {
  const size_t smem = proposal_smem_bytes<R>(K, S);
  cudaError_t e = cudaFuncSetAttribute(proposal_kernel<R>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, proposal_kernel<R>,
                                                       PROP_THREADS, smem);
}

template <typename R>
cudaError_t launch_proposal(const PropArgs<R> &a, int grid, cudaStream_t st) {
  const size_t smem = proposal_smem_bytes<R>(a.K, a.S);
  cudaError_t e = cudaFuncSetAttribute(proposal_kernel<R>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  proposal_kernel<R><<<grid, PROP_THREADS, smem, st>>>(a);
  return cudaGetLastError();
}

template size_t proposal_smem_bytes<float>(int, int);
template size_t proposal_smem_bytes<double>(int, int);
template cudaError_t proposal_occupancy<float>(int, int, int *);
template cudaError_t proposal_occupancy<double>(int, int, int *);
template cudaError_t launch_proposal<float>(const PropArgs<float> &, int, cudaStream_t);
template cudaError_t launch_proposal<double>(const PropArgs<double> &, int, cudaStream_t);

}  // namespace l0
