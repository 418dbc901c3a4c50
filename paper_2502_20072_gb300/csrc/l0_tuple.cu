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
#include "l0_tile.cuh"


namespace l0 {

namespace {

using namespace tile;

template <typename R, int DP>
__device__ void run_item(const TileArgs<R> &A, const ProbDesc &pd, int prob, int bj, int bk,
                         u64 r0, u64 r1, CtaList<R> &L, unsigned char *recbase,
                         u64 *gthr) {
  constexpr int DPM = DP > 0 ? DP : 1;
  constexpr size_t RB = align16(rec_bytes<R, DPM>());
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  ItemCtx<R> c;
  c.G = A.G + pd.g_off;
  c.ld = pd.ld;
  c.prob = prob;
  c.m = pd.m;
  c.d = pd.d;
  c.j0 = bj * TJ;
  c.k0 = tile_k0(bj, bk);
  c.diag = (c.k0 <= c.j0 + TJ - 1);
  c.total = pd.total;
  c.B = A.B;
  c.ratio = (R)A.ratio;
  c.cls = A.cls;
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
    bool isj, isk;
    int idx;
    const int col = record_col(c.j0, c.k0, isj, isk, idx);
    if (col >= 0 && col < c.m) {
      cdiag = G[(long long)(col + 1) * (ld + 1)];
      cy = G[col + 1];
    }
  }
  const R G00 = G[0];
  int pidx[DPM];
  {
    int jend = min(c.j0 + TJ, c.m);
    if (DP > 0) colex_unrank_arith(DP, r0, jend - 1, pidx);
    else pidx[0] = 0;
  }
  const RecBuf<R, DPM> rbs[2] = {rec_carve<R, DPM>(recbase), rec_carve<R, DPM>(recbase + RB)};
  if (c.diag)
    run_steps<R, DP, true>(A, c, pidx, r0, r1, cdiag, cy, G00, rbs, creg, L, gthr);
  else
    run_steps<R, DP, false>(A, c, pidx, r0, r1, cdiag, cy, G00, rbs, creg, L, gthr);
}

template <typename R, int DPLO, int DPHI>
__global__ void __launch_bounds__(L0_THREADS, 1)
tile_kernel(TileArgs<R> A) {
  persistent_items<R>(A, [&](const ProbDesc &pd, int prob, int bj, int bk, u64 r0, u64 r1,
                             CtaList<R> &L, unsigned char *recbase, u64 *gthr) {
    switch (pd.dp) {
#define L0_CASE(X)                                                                     \
  case X:                                                                              \
    if (X >= DPLO && X <= DPHI)                                                        \
      run_item<R, (X >= DPLO && X <= DPHI ? X : DPLO)>(A, pd, prob, bj, bk, r0, r1, L, \
                                                       recbase, gthr);                 \
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
  });
}

// ------------------------------------------------------------------ d = 1 --
// SHARED (shared_T > 0): score = sum_t S_yy,t rel_t / N over the tasks.
template <typename R>
__global__ void __launch_bounds__(L0_THREADS)
singles_kernel(const R *Gbase, const ProbDesc *probs, int K, int S, u64 *gthr,
               R *out_s, u64 *out_k, int *out_cnt, int n_slots, int shared_T,
               long long gstride, const double *inv_s, int mp1, long long n_total) {
  extern __shared__ __align__(16) unsigned char smem[];
  unsigned char *p = smem;
  CtaList<R> L = cta_list_carve<R>(p, K, S);
  const int prob = blockIdx.y;
  const ProbDesc pd = probs[prob];
  if (pd.d != 1) return;          // other problems run in the tuple kernel
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
    if (k < pd.m && shared_T == 0) {
      const R ckk = G[(long long)(k + 1) * (ld + 1)];
      const R ck = G[k + 1];
      ok = ckk > R(0);
      rel = G00 - ck * ck / ckk;
    } else if (k < pd.m) {
      ok = true;
      for (int t = 0; t < shared_T; ++t) {
        const R *Gt = Gbase + (long long)t * gstride;
        const R ckk = Gt[(long long)(k + 1) * (ld + 1)];
        const R ck = Gt[k + 1];
        ok = ok && ckk > R(0);
        const double is = inv_s[(long long)t * mp1];
        const R wt = (R)((is > 0.0) ? 1.0 / (is * is * (double)n_total) : 0.0);
        if (ckk > R(0)) rel += wt * (Gt[0] - ck * ck / ckk);
      }
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
  return align16(cta_list_bytes<R>(K, S)) + 16 + 2 * rb;
}

template <typename R>
static const void *tile_fn(int dp_lo, int dp_hi) {
#define L0_K(LO, HI) \
  if (dp_lo == LO && dp_hi == HI) return (const void *)tile_kernel<R, LO, HI>;
  L0_K(0, 0) L0_K(1, 1) L0_K(2, 2) L0_K(3, 3) L0_K(4, 4) L0_K(5, 5) L0_K(6, 6)
  L0_K(0, 1) L0_K(1, 2) L0_K(0, 2)
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
                           cudaStream_t st, int shared_T, long long gstride,
                           const double *inv_s, int mp1, long long n_total) {
  size_t smem = cta_list_bytes<R>(K, S) + 16;
  cudaError_t e = cudaFuncSetAttribute(singles_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  singles_kernel<R><<<dim3(grid_x, n_probs), L0_THREADS, smem, st>>>(
      G, probs_dev, K, S, gthr, out_s, out_k, out_cnt, n_slots, shared_T, gstride, inv_s, mp1,
      n_total);
  return cudaGetLastError();
}

template size_t tile_smem_bytes<double>(int, int, int);
template size_t tile_smem_bytes<float>(int, int, int);
template cudaError_t tile_occupancy<double>(int, int, size_t, int *);
template cudaError_t tile_occupancy<float>(int, int, size_t, int *);
template cudaError_t launch_tile<double>(const TileArgs<double> &, int, int, int, size_t, cudaStream_t);
template cudaError_t launch_tile<float>(const TileArgs<float> &, int, int, int, size_t, cudaStream_t);
template cudaError_t launch_singles<double>(const double *, const ProbDesc *, const ProbDesc *, int, int, int, int, u64 *, double *, u64 *, int *, int, cudaStream_t, int, long long, const double *, int, long long);
template cudaError_t launch_singles<float>(const float *, const ProbDesc *, const ProbDesc *, int, int, int, int, u64 *, float *, u64 *, int *, int, cudaStream_t, int, long long, const double *, int, long long);

}  // namespace l0
