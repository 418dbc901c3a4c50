// l0_gram_tc.cu -- split-BF16 Gram on the 5th-generation tensor cores.
//
// The tuple search needs the augmented correlation matrix of every task,
// G = W^T W with W the centred, scaled columns (target first).  In FP32 this
// is a dense contraction, so it runs as a BF16 GEMM with FP32 accumulation
// in tensor memory.  Each scaled value z is split as z = hi + lo + r with
// hi = bf16(z), lo = bf16(z - hi) (|r| <~ 2^-17 |z|), and
//     z_a z_b ~= hi_a hi_b + hi_a lo_b + lo_a hi_b          (3 terms)
// which is one GEMM over a K axis three times longer: row a of A is
// [hi_a | hi_a | lo_a], row b of B is [hi_b | lo_b | hi_b] (per task, each
// segment padded to a multiple of 64 samples with zeros).
//
// Kernel: one CTA per upper-triangular 128 x 128 output tile, task and
// K split.  With few tiles (the 1000-column Gram has 36) one CTA per tile
// would leave most SMs idle while each streams 1.5 MB of A and B rows, so
// the K blocks are split nsplit ways: each CTA writes its partial tile to a
// scratch buffer and the last CTA of a tile (a counter, no waiting) adds the
// nsplit partials in split order -- the same sum every run -- into G.
// Thread 0 streams 64-wide K blocks of A and B into a 4-stage shared-memory
// ring with TMA (128-byte swizzle); thread 32 issues tcgen05.mma
// (M = N = 128, K = 16, BF16 -> FP32 in TMEM) and frees each stage through
// tcgen05.commit; all four warps then read the accumulator with tcgen05.ld
// and store the tile.  Every wait is bounded (2 s on the global timer);
// on expiry the kernel records an error, waits (bounded) for its own copies
// and MMAs, frees its tensor memory and returns.
#include <cuda.h>
#include <cuda_bf16.h>

#include "l0_kernels.cuh"
#include "l0_tc.cuh"

namespace l0 {

namespace {

using namespace tc;

constexpr int BM = 128, BN = 128, BK = 64, STAGES = 4;
constexpr int THREADS = 128;
constexpr uint32_t TILE_A_BYTES = BM * BK * 2;     // 16 KB
constexpr uint32_t TILE_B_BYTES = BN * BK * 2;     // 16 KB
constexpr uint32_t STAGE_BYTES = TILE_A_BYTES + TILE_B_BYTES;
constexpr uint32_t TMEM_COLS = 128;
// grid (upper-triangular tile pairs, tasks), 128 threads
__global__ void __launch_bounds__(THREADS, 1)
gram_tc_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
               float *__restrict__ G, long long ld, long long g_stride, int mp1,
               const int *__restrict__ kbeg, const int *__restrict__ nkb, int nb, int *err,
               int nsplit, float *__restrict__ part, unsigned *__restrict__ tile_ctr) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char *smem =
      (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  __shared__ __align__(8) unsigned long long full_bar[STAGES];
  __shared__ __align__(8) unsigned long long empty_bar[STAGES];
  __shared__ __align__(8) unsigned long long done_bar;
  __shared__ uint32_t s_tmem;
  __shared__ int s_last;

  const int ks = (int)blockIdx.x % nsplit;
  const int tile = (int)blockIdx.x / nsplit;
  int idx = tile;
  int bi = 0;
  while (idx >= nb - bi) { idx -= nb - bi; ++bi; }
  const int bj = bi + idx;
  const int task = blockIdx.y;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  if (tid == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(smem_u32(&full_bar[s]), 1);
      mbar_init(smem_u32(&empty_bar[s]), 1);
    }
    mbar_init(smem_u32(&done_bar), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&s_tmem)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = s_tmem;
  const int nk_all = nkb[task];
  // this CTA's K blocks: [kb_lo, kb_hi) of the task's nk_all (nsplit <= nk_all)
  const int kb_lo = (int)((long long)nk_all * ks / nsplit);
  const int nk = (int)((long long)nk_all * (ks + 1) / nsplit) - kb_lo;
  const int k0 = kbeg[task] + kb_lo * BK;
  const uint32_t sbase = smem_u32(smem);

  if (tid == 0) {
    // producer: TMA loads of K blocks into the ring
    for (int kb = 0; kb < nk; ++kb) {
      const int s = kb % STAGES;
      if (kb >= STAGES) {
        if (!mbar_wait(smem_u32(&empty_bar[s]), ((kb / STAGES) - 1) & 1, err)) {
          break;
        }
      }
      const uint32_t fb = smem_u32(&full_bar[s]);
      mbar_expect_tx(fb, STAGE_BYTES);
      const uint32_t a_dst = sbase + s * STAGE_BYTES;
      tma_load_2d(a_dst, &mapA, fb, k0 + kb * BK, bi * BM);
      tma_load_2d(a_dst + TILE_A_BYTES, &mapB, fb, k0 + kb * BK, bj * BN);
    }
  } else if (tid == 32) {
    // MMA issuer
    const uint32_t idesc = idesc_bf16(BM, BN);
    for (int kb = 0; kb < nk; ++kb) {
      const int s = kb % STAGES;
      if (!mbar_wait(smem_u32(&full_bar[s]), (kb / STAGES) & 1, err)) {
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t a_s = sbase + s * STAGE_BYTES;
      const uint32_t b_s = a_s + TILE_A_BYTES;
#pragma unroll
      for (int kk = 0; kk < BK / 16; ++kk) {
        umma_bf16(tmem, sw128_desc(a_s + kk * 32), sw128_desc(b_s + kk * 32), idesc,
                  (kb | kk) != 0 ? 1u : 0u);
      }
      umma_commit(smem_u32(&empty_bar[s]));
    }
    umma_commit(smem_u32(&done_bar));
  }
  __syncwarp();
  // everyone: wait for the accumulator (the commit also fires when nothing
  // was issued, so this wait ends after a failure too)
  // warp-uniform: the tcgen05.ld below is .sync.aligned
  const bool done = __all_sync(0xffffffffu, mbar_wait(smem_u32(&done_bar), 0, err));
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const int row = bi * BM + warp * 32 + lane;
  float *grow = G + (long long)task * g_stride + (long long)row * ld;
  const uint32_t tbase = tmem + ((uint32_t)(warp * 32) << 16);
  const long long tile_g = (long long)task * gridDim.x / nsplit + tile;   // tile over all tasks
  if (nsplit == 1) {
    if (done && nk > 0) {
#pragma unroll 1
      for (int c0 = 0; c0 < BN; c0 += 16) {
        float v[16];
        tmem_ld16(tbase + (uint32_t)c0, v);
        if (row < mp1) {
#pragma unroll
          for (int i = 0; i < 16; ++i) {
            const int col = bj * BN + c0 + i;
            if (col < mp1) grow[col] = v[i];
          }
        }
      }
    }
  } else {
    // partial tile: [tile_g][ks][128 rows][128 columns], this thread's row
    float *prow = part + ((tile_g * nsplit + ks) * BM + warp * 32 + lane) * (long long)BN;
    if (done && nk > 0) {
#pragma unroll 1
      for (int c0 = 0; c0 < BN; c0 += 16) {
        float v[16];
        tmem_ld16(tbase + (uint32_t)c0, v);
#pragma unroll
        for (int i = 0; i < 16; i += 4)
          *(float4 *)(prow + c0 + i) = make_float4(v[i], v[i + 1], v[i + 2], v[i + 3]);
      }
    }
    __threadfence();
    __syncthreads();
    if (tid == 0) s_last = atomicAdd(tile_ctr + tile_g, 1u) == (unsigned)(nsplit - 1);
    __syncthreads();
    if (s_last) {
      __threadfence();
      // the tile's 128 x 128 floats as 4096 float4s, thread t taking float4s
      // t + 128 u (a warp covers one tile row per u: coalesced reads of the
      // partials and writes of G); eight float4s' loads of all splits in
      // flight before any is summed
      const float *p0 = part + tile_g * nsplit * (long long)(BM * BN);
#pragma unroll 1
      for (int u0 = 0; u0 < (BM * BN / 4) / THREADS; u0 += 8) {
        float4 acc[8];
#pragma unroll
        for (int u = 0; u < 8; ++u)
          acc[u] = __ldcg((const float4 *)p0 + tid + THREADS * (u0 + u));
        for (int q = 1; q < nsplit; ++q) {
          float4 v[8];
#pragma unroll
          for (int u = 0; u < 8; ++u)
            v[u] = __ldcg((const float4 *)(p0 + (long long)q * BM * BN) + tid + THREADS * (u0 + u));
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            acc[u].x += v[u].x;
            acc[u].y += v[u].y;
            acc[u].z += v[u].z;
            acc[u].w += v[u].w;
          }
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int f = tid + THREADS * (u0 + u);   // float4 index in the tile
          const int r = bi * BM + (f * 4) / BN, c0 = bj * BN + (f * 4) % BN;
          if (r < mp1) {
            float *gr = G + (long long)task * g_stride + (long long)r * ld;
            const float a4[4] = {acc[u].x, acc[u].y, acc[u].z, acc[u].w};
#pragma unroll
            for (int i = 0; i < 4; ++i)
              if (c0 + i < mp1) gr[c0 + i] = a4[i];
          }
        }
      }
      if (tid == 0) tile_ctr[tile_g] = 0u;   // ready for the next launch
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(TMEM_COLS)
                 : "memory");
  }
}

// ------------------------------------------------- centring + BF16 split --
// One warp per (column c in [0, m], task t), c == 0 the target.  Same
// two-pass FP64 mean / norm as the FP64 path (eight loads in flight per lane),
// then the split rows:
//   A[c][kbeg_t + s*np_t + i] = (hi, hi, lo)[s],  B[c][...] = (hi, lo, hi)[s]
// and zeros in each segment's padding [n_t, np_t).  The scaled value z is
// formed in FP64 (it is also the FP64 copy W) and split from its FP32
// rounding: hi = bf16(z), lo = bf16(z - hi) carry ~16 of its 24 bits, and
// FP32 keeps the split off GB300's narrow FP64 pipe.
__global__ void __launch_bounds__(256)
centre_split_kernel(const double *__restrict__ X, const double *__restrict__ y,
                    long long n_total, int m, const long long *__restrict__ offsets,
                    double *__restrict__ mu, double *__restrict__ inv_s,
                    double *__restrict__ W, __nv_bfloat16 *__restrict__ A,
                    __nv_bfloat16 *__restrict__ B, long long ldk,
                    const int *__restrict__ kbeg, const int *__restrict__ npad, int *err) {
  const int lane = threadIdx.x & 31;
  const int c = blockIdx.x * 8 + (threadIdx.x >> 5);
  const int t = blockIdx.y;
  if (c > m) return;
  const long long lo = offsets[t], hi = offsets[t + 1];
  const long long n = hi - lo;
  const double *src = (c == 0) ? (y + lo) : (X + (long long)(c - 1) * n_total + lo);
  double s8[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  bool finite = true;
  for (long long i0 = lane; i0 < n; i0 += 256) {
    double v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const long long i = i0 + 32 * u;
      v[u] = (i < n) ? src[i] : 0.0;
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      finite &= isfinite(v[u]);
      s8[u] += v[u];
    }
  }
  double s = ((s8[0] + s8[1]) + (s8[2] + s8[3])) + ((s8[4] + s8[5]) + (s8[6] + s8[7]));
  if (__any_sync(0xffffffffu, !finite) && lane == 0) set_err(err, 5);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  const double mean = s / (double)n;
  double q8[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  for (long long i0 = lane; i0 < n; i0 += 256) {
    double v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const long long i = i0 + 32 * u;
      v[u] = (i < n) ? src[i] - mean : 0.0;
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) q8[u] = fma(v[u], v[u], q8[u]);
  }
  double ss = ((q8[0] + q8[1]) + (q8[2] + q8[3])) + ((q8[4] + q8[5]) + (q8[6] + q8[7]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
  const double nrm = sqrt(ss);
  const double is = (nrm > 0.0) ? 1.0 / nrm : 0.0;
  if (lane == 0) {
    mu[(long long)t * (m + 1) + c] = mean;
    inv_s[(long long)t * (m + 1) + c] = is;
  }
  const long long kb = kbeg[t];
  const long long np = npad[t];
  __nv_bfloat16 *Ar = A + (long long)c * ldk + kb;
  __nv_bfloat16 *Br = B + (long long)c * ldk + kb;
#pragma unroll 4
  for (long long i = lane; i < n; i += 32) {
    const double z = (src[i] - mean) * is;
    if (W) W[(long long)c * n_total + lo + i] = z;
    const float zf = __double2float_rn(z);
    const __nv_bfloat16 h = __float2bfloat16_rn(zf);
    const __nv_bfloat16 l = __float2bfloat16_rn(zf - __bfloat162float(h));
    Ar[i] = h;
    Ar[np + i] = h;
    Ar[2 * np + i] = l;
    Br[i] = h;
    Br[np + i] = l;
    Br[2 * np + i] = h;
  }
  const __nv_bfloat16 zero = __float2bfloat16_rn(0.f);
  for (long long i = n + lane; i < np; i += 32) {
#pragma unroll
    for (int sg = 0; sg < 3; ++sg) {
      Ar[sg * np + i] = zero;
      Br[sg * np + i] = zero;
    }
  }
}

bool make_map(CUtensorMap *map, const void *base, long long rows, long long ldk) {
  return tma_map_bf16_2d(map, base, rows, ldk, ldk, BK, BM);
}

}  // namespace

cudaError_t launch_centre_split(const double *X, const double *y, long long n_total, int m,
                                const long long *offsets_dev, int T, double *mu, double *inv_s,
                                double *W64, void *A, void *B, long long ldk,
                                const int *kbeg_dev, const int *npad_dev, int *err,
                                cudaStream_t st) {
  dim3 grid((m + 1 + 7) / 8, T);
  centre_split_kernel<<<grid, 256, 0, st>>>(X, y, n_total, m, offsets_dev, mu, inv_s, W64,
                                            (__nv_bfloat16 *)A, (__nv_bfloat16 *)B, ldk,
                                            kbeg_dev, npad_dev, err);
  return cudaGetLastError();
}

size_t gram_tc_smem_bytes() { return (size_t)STAGES * STAGE_BYTES + 1024; }

int gram_tc_tiles(int m) {
  const int nb = (m + 1 + BM - 1) / BM;
  return nb * (nb + 1) / 2;
}
size_t gram_tc_part_floats(int m, int T, int nsplit) {
  return nsplit > 1 ? (size_t)gram_tc_tiles(m) * T * nsplit * BM * BN : 0;
}

cudaError_t launch_gram_tc(const void *A, const void *B, long long ldk, int m, int T,
                           const int *kbeg_dev, const int *nkb_dev, float *G, long long ld,
                           long long g_stride, int *err, cudaStream_t st, int nsplit,
                           float *part, unsigned *tile_ctr) {
  const int mp1 = m + 1;
  CUtensorMap ma, mb;
  if (!make_map(&ma, A, mp1, ldk) || !make_map(&mb, B, mp1, ldk)) return cudaErrorInvalidValue;
  const int nb = (mp1 + BM - 1) / BM;
  const int ntiles = nb * (nb + 1) / 2;
  const size_t smem = gram_tc_smem_bytes();
  cudaError_t e = cudaFuncSetAttribute(gram_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  if (nsplit < 1 || (nsplit > 1 && (part == nullptr || tile_ctr == nullptr)))
    return cudaErrorInvalidValue;
  gram_tc_kernel<<<dim3(ntiles * nsplit, T), THREADS, smem, st>>>(
      ma, mb, G, ld, g_stride, mp1, kbeg_dev, nkb_dev, nb, err, nsplit, part, tile_ctr);
  return cudaGetLastError();
}

}  // namespace l0
