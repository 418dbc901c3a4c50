// l0_shared.cu -- multi-task l0 search with one shared descriptor.
//
// Multi-task SISSO (paper Sec. 3.1) fits the same descriptor to every task
// with task-specific coefficients.  In SHARED mode a tuple is ranked by the
// pooled mean squared deviation sum_t SSE_t / N over the tasks; it is not
// eligible when it is rank deficient in any task.
//
// The work decomposition is the PER_TASK one (tiles of (j, k) pairs against
// chunks of outer prefixes P).  Within a step the CTA walks the tasks: for
// task t it loads its Gram tile, builds the task's records, and every thread
// adds S_yy,t * rel_t / N for its 32 tuples; after the last task the pooled
// scores are compared with the threshold and the survivors staged.  Tuples
// that are near-singular in FP32 in some task are queued for the FP64 redo,
// which pools over the tasks the same way.
#include "l0_tile.cuh"

namespace l0 {

namespace {

using namespace tile;

template <typename R, int DP>
__device__ void run_item_shared(const TileArgs<R> &A, const ProbDesc &pd, int prob, int bj,
                                int bk, u64 r0, u64 r1, CtaList<R> &L, unsigned char *recbase,
                                u64 *gthr) {
  constexpr int DPM = DP > 0 ? DP : 1;
  constexpr bool MIXED = sizeof(R) == 4;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  ItemCtx<R> c;
  c.G = A.G;
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
  int pidx[DPM];
  {
    const int jend = min(c.j0 + TJ, c.m);
    if (DP > 0) colex_unrank_arith(DP, r0, jend - 1, pidx);
    else pidx[0] = 0;
  }
  const RecBuf<R, DPM> rb = rec_carve<R, DPM>(recbase);
  bool isj, isk;
  int idx;
  const int col = record_col(c.j0, c.k0, isj, isk, idx);
  const int T = A.shared_T;
  u64 gnext = ~0ull;   // warp 0: the global bound, read a step before it is used
  for (u64 r = r0; r < r1; ++r) {
    const u64 gprev = gnext;
    if (threadIdx.x < 32) gnext = ld_relaxed(gthr);
    R score[UJ][UK];
#pragma unroll
    for (int u = 0; u < UJ; ++u)
#pragma unroll
      for (int v = 0; v < UK; ++v) score[u][v] = R(0);
    unsigned bad = 0u, dfr = 0u;   // per (u, v): ineligible / FP64 redo
    for (int t = 0; t < T; ++t) {
      ItemCtx<R> ct = c;
      ct.G = A.G + (long long)t * A.shared_gstride;
      const double is = A.inv_s[(long long)t * A.mp1];
      const R wt = (R)((is > 0.0) ? 1.0 / (is * is * (double)A.n_total) : 0.0);
      R cr[UJ][UK];
#pragma unroll
      for (int u = 0; u < UJ; ++u) {
        const int j = c.j0 + w * UJ + u;
#pragma unroll
        for (int v = 0; v < UK; ++v) {
          const int k = c.k0 + lane + 32 * v;
          cr[u][v] = (j < c.m && k < c.m) ? ct.G[(long long)(j + 1) * c.ld + k + 1] : R(0);
        }
      }
      R cdiag = R(0), cy = R(0);
      if (col >= 0 && col < c.m) {
        cdiag = ct.G[(long long)(col + 1) * (c.ld + 1)];
        cy = ct.G[col + 1];
      }
      RecRaw<R, DP> raw;
      if (isj || isk) load_raw<R, DP>(ct, pidx, col, raw);
      make_record<R, DP>(ct, pidx, raw, isj, isk, idx, col, cdiag, cy, ct.G[0], R(0), rb);
      __syncthreads();
#pragma unroll
      for (int u = 0; u < UJ; ++u) {
        const int jl = w * UJ + u;
        const int flag = rb.jflag[jl];
        const unsigned rowbits = ((1u << UK) - 1u) << (u * UK);
        if (flag == 0) { bad |= rowbits; continue; }       // ineligible or out of shape
        if (flag == 3) { dfr |= rowbits; continue; }       // singular in FP32
        R jg[DPM];
#pragma unroll
        for (int p = 0; p < DPM; ++p) jg[p] = rb.jg[p * TJ + jl];
        const R invl = rb.jinvl[jl], z2 = rb.jz2[jl], pP = rb.jpP[jl];
#pragma unroll
        for (int v = 0; v < UK; ++v) {
          const int kk = lane + 32 * v;
          const unsigned bit = 1u << (u * UK + v);
          const R kpn = rb.kp1[kk];
          if (kpn == -r_inf<R>()) { bad |= bit; continue; }
          if (MIXED && kpn == r_inf<R>()) { dfr |= bit; continue; }
          R h = cr[u][v];
#pragma unroll
          for (int p = 0; p < DP; ++p) h = fma(jg[p], rb.kg[p * TK + kk], h);
          const R g2 = h * invl;
          const R pp = -fma(g2, g2, kpn);
          const R wn = fma(g2, z2, rb.kw1[kk]);
          if (!(pp >= R(0))) {
            if (MIXED && !same_class(c.cls, c.j0 + jl, c.k0 + kk)) dfr |= bit; else bad |= bit;
            continue;
          }
          score[u][v] += wt * (pP - wn * wn / (pp + rb.kpt[kk]));
        }
      }
      __syncthreads();
    }
    // stage the pooled scores that beat the threshold
    unsigned done = 0u;
    for (int pass = 0;; ++pass) {
      const R ts = cta_cut<R>(L);
#pragma unroll
      for (int u = 0; u < UJ; ++u) {
        const int j = c.j0 + w * UJ + u;
        const bool row_ok = j < c.m && (DP == 0 || pidx[DP > 0 ? DP - 1 : 0] < j);
#pragma unroll
        for (int v = 0; v < UK; ++v) {
          const unsigned bit = 1u << (u * UK + v);
          const int k = c.k0 + lane + 32 * v;
          if (!row_ok || k >= c.m || k <= j || (done & bit)) continue;
          if (dfr & bit) {
            if (MIXED) defer_run<R, DP>(A, c, pidx, j, k, 1);
            done |= bit;
            continue;
          }
          if ((bad & bit) || score[u][v] > ts) { done |= bit; continue; }
          int tt[L0_DMAX];
#pragma unroll
          for (int q = 0; q < DP; ++q) tt[q] = pidx[q];
          tt[DP] = j;
          tt[DP + 1] = k;
          const u64 key = lex_rank(c.B, c.m, c.d, tt, c.total);
          if (!cta_list_admits<R>(L, score[u][v], key) || cta_list_push<R>(L, score[u][v], key))
            done |= bit;
        }
      }
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
    if (DP > 0) colex_next<DP>(pidx);
  }
}

template <typename R, int DP>
__global__ void __launch_bounds__(L0_THREADS)
shared_tile_kernel(TileArgs<R> A) {
  persistent_items<R>(A, [&](const ProbDesc &pd, int prob, int bj, int bk, u64 r0, u64 r1,
                             CtaList<R> &L, unsigned char *recbase, u64 *gthr) {
    run_item_shared<R, DP>(A, pd, prob, bj, bk, r0, r1, L, recbase, gthr);
  });
}

template <typename R>
const void *shared_fn(int dp) {
  switch (dp) {
    case 0: return (const void *)shared_tile_kernel<R, 0>;
    case 1: return (const void *)shared_tile_kernel<R, 1>;
    case 2: return (const void *)shared_tile_kernel<R, 2>;
    case 3: return (const void *)shared_tile_kernel<R, 3>;
    case 4: return (const void *)shared_tile_kernel<R, 4>;
    case 5: return (const void *)shared_tile_kernel<R, 5>;
    case 6: return (const void *)shared_tile_kernel<R, 6>;
    default: return nullptr;
  }
}

}  // namespace

template <typename R>
cudaError_t shared_occupancy(int dp, size_t smem, int *blocks_per_sm) {
  const void *fn = shared_fn<R>(dp);
  if (!fn) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, fn, L0_THREADS, smem);
}

template <typename R>
cudaError_t launch_tile_shared(const TileArgs<R> &a, int dp, int grid, size_t smem,
                               cudaStream_t st) {
  const void *fn = shared_fn<R>(dp);
  if (!fn) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  void *args[] = {(void *)&a};
  return cudaLaunchKernel(fn, dim3(grid), dim3(L0_THREADS), args, smem, st);
}

template cudaError_t shared_occupancy<double>(int, size_t, int *);
template cudaError_t shared_occupancy<float>(int, size_t, int *);
template cudaError_t launch_tile_shared<double>(const TileArgs<double> &, int, int, size_t, cudaStream_t);
template cudaError_t launch_tile_shared<float>(const TileArgs<float> &, int, int, size_t, cudaStream_t);

}  // namespace l0
