// l0_mlp.cu -- the learned pair scorer: a 6-256-256-1 ReLU network with
// BF16 operands, FP32 accumulation and FP32 master weights.
//
// The paper's l0 step scores every tuple (Sec. 2.4).  The learned form ranks
// the pairs of a d = 3 search by this network and fits exactly only the
// triples reachable from the best pairs; the network is trained on the
// exhaustive search's own results.
//
// Rounding points (the oracle uses the same): features, W1, W2, w3, the
// hidden activations h1, h2 and the back-propagated dh2 are BF16; sums are
// FP32.
//
// mlp_kernel<MODE>: 128 threads, one row (a pair, or a training sample) per
// thread, 128 rows per tile, one CTA per SM (about 200 KB of shared memory).
//   layer 1 (K = 6) on the FP32 pipe: h1 = bf16(relu(W1 x + b1)) is written
//     straight into shared memory in the 128-byte-swizzled K-major layout of
//     a UMMA operand;
//   layer 2 on the tensor cores: pre2 = h1 W2^T (M = 128 rows, N = 256,
//     K = 256) by tcgen05.mma with W2 streamed by TMA through a 2-stage ring
//     and the accumulator in tensor memory (256 columns);
//   layer 3 in the epilogue: out = bf16(relu(pre2 + b2)) . w3 + b3.
// Training (MODE_TRAIN, one tile per CTA per step) continues in the same CTA:
//   dh2 = bf16(g w3 [pre2 > 0]), g = 2 (out - t) / B, written as a K-major
//     operand (for dH1) and transposed (for dW2);
//   dW2 = dh2^T h1 on the tensor cores (two M = 128 halves, K = the tile's
//     128 rows, 512 TMEM columns), written to the CTA's partial gradient;
//   dH1 = dh2 W2 on the tensor cores (W2^T streamed by TMA);
//   dW1, db1, db2, dw3, db3 by warp reductions over the rows.
// mlp_adam_kernel sums the partials and takes one Adam step, refreshing the
// BF16 copies of W2 and W2^T the tensor cores read.
//
// Every mbarrier wait is bounded (2 s); on expiry the kernel records an
// error, stops issuing, frees its tensor memory and returns.
#include <cuda_bf16.h>

#include "l0_kernels.cuh"
#include "l0_tc.cuh"

namespace l0 {

namespace {

using namespace tc;

constexpr int THREADS = 128;
constexpr int ROWS = 128;
constexpr int NH = MLP_NH, NIN = MLP_NIN;
constexpr uint32_t A_BYTES = ROWS * NH * 2;      // 64 KB: 128 rows x 256 K
constexpr uint32_t KB_A = ROWS * 64 * 2;         // one 64-wide K block of A: 16 KB
constexpr uint32_t W_STAGE = NH * 64 * 2;        // one K block of W2: 256 rows, 32 KB
constexpr uint32_t T_KB = NH * 64 * 2;           // one K block of a transposed tile: 32 KB
constexpr uint32_t TMEM_COLS = 512;

__device__ __forceinline__ float bf16r(float x) {
  return __bfloat162float(__float2bfloat16_rn(x));
}

__device__ __forceinline__ uint32_t pack_bf16x2(float a, float b) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<const uint32_t *>(&v);
}

__device__ __forceinline__ void st_shared_v4(uint32_t addr, uint32_t a, uint32_t b, uint32_t c,
                                             uint32_t d) {
  asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(a), "r"(b), "r"(c),
               "r"(d)
               : "memory");
}
__device__ __forceinline__ void st_shared_b16(uint32_t addr, float v) {
  const __nv_bfloat16 h = __float2bfloat16_rn(v);
  const unsigned short u = *reinterpret_cast<const unsigned short *>(&h);
  asm volatile("st.shared.b16 [%0], %1;" ::"r"(addr), "h"(u) : "memory");
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// the UMMA pipeline state of one CTA: ring loads and MMA completions are
// counted across the kernel's phases so that barrier parities stay in step
struct Pipe {
  uint32_t full[2], empty[2], done;
  uint32_t loads;       // K blocks loaded through the ring so far
  uint32_t done_waits;  // completions of `done` waited for so far
};

// M = 128 rows of A (K-major, resident, 4 K blocks of 64) times a 256-row
// B streamed by TMA (K-major, 4 K blocks): D (256 TMEM columns at d_col).
// Thread 0 loads, thread 32 issues; returns false (error set) on a timeout.
__device__ bool mma_a_resident_b_streamed(Pipe &p, uint32_t a_base, uint32_t ring,
                                          const CUtensorMap *mapB, uint32_t tmem, uint32_t d_col,
                                          int *err) {
  const int tid = threadIdx.x;
  bool ok = true;
  if (tid == 0) {
    for (int kb = 0; kb < 4; ++kb) {
      const uint32_t it = p.loads + kb;
      const uint32_t s = it & 1u;
      if (it >= 2 && !mbar_wait(p.empty[s], ((it >> 1) - 1) & 1u, err)) { ok = false; break; }
      mbar_expect_tx(p.full[s], W_STAGE);
      tma_load_2d(ring + s * W_STAGE, mapB, p.full[s], kb * 64, 0);
    }
  } else if (tid == 32) {
    const uint32_t idesc = idesc_bf16(128, 256);
    for (int kb = 0; kb < 4; ++kb) {
      const uint32_t it = p.loads + kb;
      const uint32_t s = it & 1u;
      if (!mbar_wait(p.full[s], (it >> 1) & 1u, err)) { ok = false; break; }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
      for (int kk = 0; kk < 4; ++kk)
        umma_bf16(tmem + d_col, sw128_desc(a_base + kb * KB_A + kk * 32),
                  sw128_desc(ring + s * W_STAGE + kk * 32), idesc, (kb | kk) != 0 ? 1u : 0u);
      umma_commit(p.empty[s]);
    }
    umma_commit(p.done);
  }
  p.loads += 4;
  return ok;
}

// all threads: wait for the last commit on `done`; warp-uniform result
__device__ bool wait_done(Pipe &p, int *err) {
  const bool ok = __all_sync(0xffffffffu, mbar_wait(p.done, p.done_waits & 1u, err));
  p.done_waits += 1;
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  return ok;
}

// colex unrank of a pair rank: p = j (j - 1) / 2 + i, i < j
__device__ __forceinline__ void pair_of(long long p, int &i, int &j) {
  long long jj = (long long)((1.0 + sqrt(1.0 + 8.0 * (double)p)) * 0.5);
  while (jj * (jj - 1) / 2 > p) --jj;
  while ((jj + 1) * jj / 2 <= p) ++jj;
  j = (int)jj;
  i = (int)(p - jj * (jj - 1) / 2);
}

template <int MODE>
__global__ void __launch_bounds__(THREADS, 1)
mlp_kernel(const __grid_constant__ CUtensorMap mapW2, const __grid_constant__ CUtensorMap mapW2T,
           MlpArgs a) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char *smem = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  __shared__ float sW1[NH * NIN], sb1[NH], sb2[NH], sw3[NH];
  __shared__ float gW1[NH * NIN], gb1[NH], gb2[NH], gw3[NH], gsc[2];   // partial gradients
  __shared__ __align__(8) unsigned long long bars[5];
  __shared__ uint32_t s_tmem;
  constexpr bool TRAIN = MODE == MLP_TRAIN;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t R1 = smem_u32(smem), R2 = R1 + A_BYTES, R3 = R2 + A_BYTES;
  Pipe p;
  p.full[0] = smem_u32(&bars[0]);
  p.full[1] = smem_u32(&bars[1]);
  p.empty[0] = smem_u32(&bars[2]);
  p.empty[1] = smem_u32(&bars[3]);
  p.done = smem_u32(&bars[4]);
  p.loads = 0;
  p.done_waits = 0;
  if (tid == 0) {
    for (int q = 0; q < 5; ++q) mbar_init(smem_u32(&bars[q]), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  for (int q = tid; q < NH * NIN; q += THREADS) {
    sW1[q] = bf16r(a.params[MLP_OFF_W1 + q]);
    if (TRAIN) gW1[q] = 0.f;
  }
  for (int q = tid; q < NH; q += THREADS) {
    sb1[q] = a.params[MLP_OFF_B1 + q];
    sb2[q] = a.params[MLP_OFF_B2 + q];
    sw3[q] = bf16r(a.params[MLP_OFF_W3 + q]);
    if (TRAIN) { gb1[q] = 0.f; gb2[q] = 0.f; gw3[q] = 0.f; }
  }
  if (tid < 2) gsc[tid] = 0.f;
  const float b3 = a.params[MLP_OFF_B3];
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
  const uint32_t tlane = (uint32_t)(warp * 32) << 16;
  const long long n_tiles = (a.n_rows + ROWS - 1) / ROWS;
  bool alive = true;

  for (long long tile = blockIdx.x; tile < n_tiles && alive; tile += gridDim.x) {
    const long long r = tile * ROWS + tid;
    const bool valid = r < a.n_rows;
    // ---- features
    float x[NIN];
#pragma unroll
    for (int f = 0; f < NIN; ++f) x[f] = 0.f;
    if (valid) {
      if (MODE == MLP_INFER_GRAM) {
        int i, j;
        pair_of(a.row0 + r, i, j);
        pair_feature_vec(a.G, a.ld, i, j, x);
      } else {
        const float *fr = a.feats + (size_t)(a.row0 + r) * MLP_FEAT_LD;
#pragma unroll
        for (int f = 0; f < NIN; ++f) x[f] = fr[f];
      }
    }
#pragma unroll
    for (int f = 0; f < NIN; ++f) x[f] = bf16r(x[f]);
    // ---- layer 1 -> h1 (A operand, and transposed for dW2)
    for (int o0 = 0; o0 < NH; o0 += 8) {
      float h[8];
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const int o = o0 + e;
        float s = sb1[o];
#pragma unroll
        for (int f = 0; f < NIN; ++f) s = fmaf(sW1[o * NIN + f], x[f], s);
        h[e] = valid ? fmaxf(s, 0.f) : 0.f;
      }
      st_shared_v4(R1 + (o0 >> 6) * KB_A + sw128_offset(tid, o0 & 63), pack_bf16x2(h[0], h[1]),
                   pack_bf16x2(h[2], h[3]), pack_bf16x2(h[4], h[5]), pack_bf16x2(h[6], h[7]));
      if (TRAIN) {
#pragma unroll
        for (int e = 0; e < 8; ++e)
          st_shared_b16(R3 + (tid >> 6) * T_KB + sw128_offset(o0 + e, tid & 63), h[e]);
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // ---- layer 2 on the tensor cores: TMEM[0, 256) = h1 W2^T
    mma_a_resident_b_streamed(p, R1, R2, &mapW2, tmem, 0, a.err);
    __syncwarp();
    if (!wait_done(p, a.err)) { alive = false; break; }
    // ---- layer 3
    float out = b3;
    for (int c0 = 0; c0 < NH; c0 += 16) {
      float v[16];
      tmem_ld16(tmem + tlane + (uint32_t)c0, v);
#pragma unroll
      for (int e = 0; e < 16; ++e) out = fmaf(bf16r(fmaxf(v[e] + sb2[c0 + e], 0.f)), sw3[c0 + e], out);
    }
    if (!TRAIN) {
      if (valid) a.out[r] = out;
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncthreads();
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      continue;
    }
    // ---- training: loss gradient and dh2
    const float diff = valid ? out - a.label[a.row0 + r] : 0.f;
    const float g = (float)(2.0 * a.inv_B) * diff;
    {
      const float l = warp_sum(diff * diff);
      const float sg = warp_sum(g);
      if (lane == 0) {
        atomicAdd(&gsc[0], l * (float)a.inv_B);
        atomicAdd(&gsc[1], sg);
      }
    }
    for (int c0 = 0; c0 < NH; c0 += 16) {
      float v[16];
      tmem_ld16(tmem + tlane + (uint32_t)c0, v);
      float d[16];
#pragma unroll
      for (int e = 0; e < 16; ++e) {
        const int c = c0 + e;
        const float pre = v[e] + sb2[c];
        const float h2 = bf16r(fmaxf(pre, 0.f));
        d[e] = bf16r(pre > 0.f ? g * sw3[c] : 0.f);
        const float s_w3 = warp_sum(g * h2);
        const float s_b2 = warp_sum(d[e]);
        if (lane == 0) {
          atomicAdd(&gw3[c], s_w3);
          atomicAdd(&gb2[c], s_b2);
        }
        // dh2 transposed (rows = output unit c, K = the tile row) for dW2
        st_shared_b16(R1 + (tid >> 6) * T_KB + sw128_offset(c, tid & 63), d[e]);
      }
      // dh2 as a K-major operand (rows = tile rows, K = output unit) for dH1
#pragma unroll
      for (int e0 = 0; e0 < 16; e0 += 8)
        st_shared_v4(R2 + ((c0 + e0) >> 6) * KB_A + sw128_offset(tid, (c0 + e0) & 63),
                     pack_bf16x2(d[e0], d[e0 + 1]), pack_bf16x2(d[e0 + 2], d[e0 + 3]),
                     pack_bf16x2(d[e0 + 4], d[e0 + 5]), pack_bf16x2(d[e0 + 6], d[e0 + 7]));
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // ---- dW2[o][i] = sum_r dh2[r][o] h1[r][i]: A = dh2^T (R1), B = h1^T (R3)
    if (tid == 32) {
      const uint32_t idesc = idesc_bf16(128, 256);
#pragma unroll
      for (int hm = 0; hm < 2; ++hm)
#pragma unroll
        for (int kb = 0; kb < 2; ++kb)
#pragma unroll
          for (int kk = 0; kk < 4; ++kk)
            umma_bf16(tmem + hm * 256, sw128_desc(R1 + kb * T_KB + hm * (T_KB / 2) + kk * 32),
                      sw128_desc(R3 + kb * T_KB + kk * 32), idesc, (kb | kk) != 0 ? 1u : 0u);
      umma_commit(p.done);
    }
    __syncwarp();
    if (!wait_done(p, a.err)) { alive = false; break; }
    {
      float *gp = a.partial + (size_t)blockIdx.x * MLP_PSTRIDE + MLP_OFF_W2;
#pragma unroll 1
      for (int hm = 0; hm < 2; ++hm) {
        const int o = hm * 128 + warp * 32 + lane;
        for (int c0 = 0; c0 < NH; c0 += 16) {
          float v[16];
          tmem_ld16(tmem + tlane + (uint32_t)(hm * 256 + c0), v);
          float4 *dst = reinterpret_cast<float4 *>(gp + (size_t)o * NH + c0);
#pragma unroll
          for (int e = 0; e < 16; e += 4) dst[e / 4] = make_float4(v[e], v[e + 1], v[e + 2], v[e + 3]);
        }
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // ---- dH1 = dh2 W2: A = dh2 (R2), B = W2^T streamed through R1
    mma_a_resident_b_streamed(p, R2, R1, &mapW2T, tmem, 0, a.err);
    __syncwarp();
    if (!wait_done(p, a.err)) { alive = false; break; }
    for (int c0 = 0; c0 < NH; c0 += 16) {
      float v[16];
      tmem_ld16(tmem + tlane + (uint32_t)c0, v);
#pragma unroll
      for (int e = 0; e < 16; ++e) {
        const int o = c0 + e;
        float s = sb1[o];
#pragma unroll
        for (int f = 0; f < NIN; ++f) s = fmaf(sW1[o * NIN + f], x[f], s);
        const float dp = (valid && s > 0.f) ? v[e] : 0.f;
        const float sb = warp_sum(dp);
        float sw[NIN];
#pragma unroll
        for (int f = 0; f < NIN; ++f) sw[f] = warp_sum(dp * x[f]);
        if (lane == 0) {
          atomicAdd(&gb1[o], sb);
#pragma unroll
          for (int f = 0; f < NIN; ++f) atomicAdd(&gW1[o * NIN + f], sw[f]);
        }
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  }
  if (TRAIN) {
    __syncthreads();
    float *gp = a.partial + (size_t)blockIdx.x * MLP_PSTRIDE;
    for (int q = tid; q < NH * NIN; q += THREADS) gp[MLP_OFF_W1 + q] = gW1[q];
    for (int q = tid; q < NH; q += THREADS) {
      gp[MLP_OFF_B1 + q] = gb1[q];
      gp[MLP_OFF_B2 + q] = gb2[q];
      gp[MLP_OFF_W3 + q] = gw3[q];
    }
    if (tid == 0) {
      gp[MLP_OFF_B3] = gsc[1];
      gp[MLP_N_PARAMS] = gsc[0];
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(TMEM_COLS)
                 : "memory");
}

// Sum of the per-CTA partial gradients (and loss), optionally one Adam step
// (t counts from 1), and the BF16 copies of W2 and W2^T.
__global__ void __launch_bounds__(256)
mlp_adam_kernel(float *params, float *m1, float *m2, const float *partial, int n_parts,
                float lr, float beta1, float beta2, float eps, int t, int do_step, float *grad_out,
                float *loss_out, __nv_bfloat16 *W2b, __nv_bfloat16 *W2Tb) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q > MLP_N_PARAMS) return;
  float g = 0.f;
  for (int c = 0; c < n_parts; ++c) g += partial[(size_t)c * MLP_PSTRIDE + q];
  if (q == MLP_N_PARAMS) {   // the loss slot
    if (loss_out) *loss_out = g;
    return;
  }
  if (grad_out) grad_out[q] = g;
  float w = params[q];
  if (do_step) {
    const float a1 = beta1 * m1[q] + (1.f - beta1) * g;
    const float a2 = beta2 * m2[q] + (1.f - beta2) * g * g;
    m1[q] = a1;
    m2[q] = a2;
    const float mh = a1 / (1.f - powf(beta1, (float)t));
    const float vh = a2 / (1.f - powf(beta2, (float)t));
    w = w - lr * mh / (sqrtf(vh) + eps);
    params[q] = w;
  }
  if (q >= MLP_OFF_W2 && q < MLP_OFF_W2 + NH * NH) {
    const int o = (q - MLP_OFF_W2) / NH, i = (q - MLP_OFF_W2) % NH;
    const __nv_bfloat16 b = __float2bfloat16_rn(w);
    W2b[o * NH + i] = b;
    W2Tb[i * NH + o] = b;
  }
}

}  // namespace

size_t mlp_smem_bytes(int mode) {
  return (size_t)(mode == MLP_TRAIN ? 3 : 2) * A_BYTES + 1024;
}

cudaError_t launch_mlp(int mode, const MlpArgs &a, const void *W2b, const void *W2Tb, int grid,
                       cudaStream_t st) {
  CUtensorMap m2, m2t;
  if (!tma_map_bf16_2d(&m2, W2b, NH, NH, NH, 64, NH) ||
      !tma_map_bf16_2d(&m2t, W2Tb, NH, NH, NH, 64, NH))
    return cudaErrorInvalidValue;
  const size_t smem = mlp_smem_bytes(mode);
  const void *fn = mode == MLP_TRAIN ? (const void *)mlp_kernel<MLP_TRAIN>
                   : mode == MLP_INFER_GRAM ? (const void *)mlp_kernel<MLP_INFER_GRAM>
                                            : (const void *)mlp_kernel<MLP_INFER_FEATS>;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  MlpArgs aa = a;
  void *args[] = {(void *)&m2, (void *)&m2t, (void *)&aa};
  return cudaLaunchKernel(fn, dim3(grid), dim3(THREADS), args, smem, st);
}

cudaError_t launch_mlp_adam(float *params, float *m1, float *m2, const float *partial,
                            int n_parts, float lr, int t, int do_step, float *grad_out,
                            float *loss_out, void *W2b, void *W2Tb, cudaStream_t st) {
  const int n = MLP_N_PARAMS + 1;
  mlp_adam_kernel<<<(n + 255) / 256, 256, 0, st>>>(params, m1, m2, partial, n_parts, lr, 0.9f,
                                                   0.999f, 1e-8f, t, do_step, grad_out, loss_out,
                                                   (__nv_bfloat16 *)W2b, (__nv_bfloat16 *)W2Tb);
  return cudaGetLastError();
}

}  // namespace l0
