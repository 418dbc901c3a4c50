// l0_sis.cu -- sure independence screening: the step before l0.
//
// SIS (paper Sec. 2.3) ranks candidate features by the magnitude of their
// Pearson correlation with the target (Eq. 1) and keeps the best m, which
// the l0 search then combines.  The scan reads every feature once, so it is
// bound by HBM bandwidth:
//   sis_target_kernel: mean of y, S_yy and the residual sum of y - mean (one
//     block, two passes in FP64);
//   sis_score_kernel: one warp per feature, one pass over its samples with
//     the data shifted by its first value (the shifted-data sums of Chan,
//     Golub and LeVeque): S1 = sum (x - c), S2 = sum (x - c)^2,
//     S3 = sum (x - c)(y - mean_y); then S_xx = S2 - S1^2 / n and
//     S_xy = S3 - S1 sum(y - mean_y) / n, r = S_xy / sqrt(S_xx S_yy);
//   selection of the m largest |r| (ties: smaller index): two 16-bit
//     histogram levels over the ordered FP64 bits of -|r| give a cut that
//     keeps at least m candidates, which are compacted and sorted exactly by
//     (-|r|, index) in one block.
#include <algorithm>

#include "l0_kernels.cuh"

namespace l0 {

namespace {

__global__ void __launch_bounds__(1024)
sis_target_kernel(const double *y, long long n, double *out) {
  __shared__ double red[32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  auto block_sum = [&](double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if (lane == 0) red[w] = v;
    __syncthreads();
    double s = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
    return s;
  };
  double s = 0.0;
  for (long long i = threadIdx.x; i < n; i += blockDim.x) s += y[i];
  const double mean = block_sum(s) / (double)n;
  double q = 0.0, t = 0.0;
  for (long long i = threadIdx.x; i < n; i += blockDim.x) {
    const double d = y[i] - mean;
    q = fma(d, d, q);
    t += d;
  }
  const double syy = block_sum(q);
  const double sy0 = block_sum(t);
  if (threadIdx.x == 0) {
    out[0] = mean;
    out[1] = syy;
    out[2] = sy0;
  }
}

__global__ void __launch_bounds__(256)
sis_score_kernel(const double *__restrict__ X, long long n, long long n_feat,
                 const double *__restrict__ y, const double *__restrict__ tgt,
                 double *__restrict__ r_out, int *err) {
  const int lane = threadIdx.x & 31;
  const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
  const double my = tgt[0], syy = tgt[1], sy0 = tgt[2];
  for (long long f = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); f < n_feat;
       f += warps) {
    const double *x = X + f * n;
    const double c = __ldg(x);
    double S1 = 0.0, S2 = 0.0, S3 = 0.0;
    bool finite = true;
    // 16 loads per lane in flight per chunk of 512 samples
    constexpr int U = 16;
    for (long long i0 = lane; i0 < n; i0 += 32 * U) {
      double v[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const long long i = i0 + 32 * u;
        v[u] = (i < n) ? __ldcs(x + i) : c;
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const long long i = i0 + 32 * u;
        finite &= isfinite(v[u]);
        const double d = v[u] - c;            // 0 past the end
        S1 += d;
        S2 = fma(d, d, S2);
        S3 = fma(d, (i < n) ? __ldg(y + i) - my : 0.0, S3);
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      S1 += __shfl_xor_sync(0xffffffffu, S1, o);
      S2 += __shfl_xor_sync(0xffffffffu, S2, o);
      S3 += __shfl_xor_sync(0xffffffffu, S3, o);
    }
    if (__any_sync(0xffffffffu, !finite) && lane == 0) set_err(err, 5);
    if (lane == 0) {
      const double sxx = S2 - S1 * S1 / (double)n;
      const double sxy = S3 - S1 * sy0 / (double)n;
      r_out[f] = (sxx > 0.0 && syy > 0.0) ? sxy / sqrt(sxx * syy) : 0.0;
    }
  }
}

// The same sums with the products in FP32: each sample costs one FP64
// subtraction (x - c) and one conversion; the centred value, the centred
// target and their products are FP32, summed in FP32 over 16 samples per
// lane and then in FP64.  GB300's FP64 pipe (~1 TFLOP/s) cannot keep up
// with HBM at five FP64 operations per sample; at one it nearly can.
// r carries ~1e-6 relative error (FP32 rounding of x - c).
__global__ void __launch_bounds__(256)
sis_score32_kernel(const double *__restrict__ X, long long n, long long n_feat,
                   const float *__restrict__ yc, const double *__restrict__ tgt,
                   double *__restrict__ r_out, int *err) {
  const int lane = threadIdx.x & 31;
  const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
  const double syy = tgt[1], sy0 = tgt[2];
  for (long long f = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); f < n_feat;
       f += warps) {
    const double *x = X + f * n;
    const double c = __ldg(x);
    double S1 = 0.0, S2 = 0.0, S3 = 0.0;
    bool finite = true;
    constexpr int U = 16;
    for (long long i0 = lane; i0 < n; i0 += 32 * U) {
      double v[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const long long i = i0 + 32 * u;
        v[u] = (i < n) ? __ldcs(x + i) : c;
      }
      float a1 = 0.f, a2 = 0.f, a3 = 0.f;
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const long long i = i0 + 32 * u;
        finite &= isfinite(v[u]);
        const float d = (float)(v[u] - c);
        a1 += d;
        a2 = fmaf(d, d, a2);
        a3 = fmaf(d, (i < n) ? __ldg(yc + i) : 0.f, a3);
      }
      S1 += (double)a1;
      S2 += (double)a2;
      S3 += (double)a3;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      S1 += __shfl_xor_sync(0xffffffffu, S1, o);
      S2 += __shfl_xor_sync(0xffffffffu, S2, o);
      S3 += __shfl_xor_sync(0xffffffffu, S3, o);
    }
    if (__any_sync(0xffffffffu, !finite) && lane == 0) set_err(err, 5);
    if (lane == 0) {
      const double sxx = S2 - S1 * S1 / (double)n;
      const double sxy = S3 - S1 * sy0 / (double)n;
      r_out[f] = (sxx > 0.0 && syy > 0.0) ? sxy / sqrt(sxx * syy) : 0.0;
    }
  }
}

// centred target in FP32 (the FP64 sum of its rounded values goes to sy0)
__global__ void __launch_bounds__(1024)
sis_target32_kernel(const double *y, long long n, double *tgt, float *yc) {
  __shared__ double red[32];
  const double mean = tgt[0];
  double t = 0.0;
  for (long long i = threadIdx.x; i < n; i += blockDim.x) {
    const float v = (float)(y[i] - mean);
    yc[i] = v;
    t += (double)v;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = t;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
    tgt[2] = s;
  }
}

// ordered image of -|r| (ascending = best first)
__device__ __forceinline__ u64 sis_key(double r) { return ord_of(-fabs(r)); }

__global__ void __launch_bounds__(256)
sis_hist_kernel(const double *r, long long n_feat, int level, const unsigned *cut1,
                unsigned *hist) {
  const unsigned c1 = level ? *cut1 : 0u;
  for (long long f = (long long)blockIdx.x * blockDim.x + threadIdx.x; f < n_feat;
       f += (long long)gridDim.x * blockDim.x) {
    const u64 k = sis_key(r[f]);
    const unsigned b1 = (unsigned)(k >> 48);
    if (level == 0) atomicAdd(hist + b1, 1u);
    else if (b1 == c1) atomicAdd(hist + ((unsigned)(k >> 32) & 0xffffu), 1u);
  }
}

// one block of 1024: the smallest bin b with before + count(bins <= b) >= want
__global__ void __launch_bounds__(1024)
sis_cut_kernel(const unsigned *hist, long long want, unsigned long long *below, unsigned *cut) {
  __shared__ unsigned long long part[1024];
  __shared__ unsigned s_bin;
  __shared__ unsigned long long s_before;
  const int tid = threadIdx.x;
  constexpr int PER = 65536 / 1024;
  const unsigned long long base = below ? *below : 0ull;
  unsigned long long s = 0;
  for (int b = 0; b < PER; ++b) s += hist[tid * PER + b];
  part[tid] = s;
  if (tid == 0) { s_bin = 0xffffu; s_before = base; }
  __syncthreads();
  for (int o = 1; o < 1024; o <<= 1) {
    const unsigned long long v = (tid >= o) ? part[tid - o] : 0ull;
    __syncthreads();
    part[tid] += v;
    __syncthreads();
  }
  const unsigned long long before = base + (tid ? part[tid - 1] : 0ull);
  if (before < (unsigned long long)want && base + part[tid] >= (unsigned long long)want) {
    unsigned long long acc = before;
    for (int b = 0; b < PER; ++b) {
      if (acc + hist[tid * PER + b] >= (unsigned long long)want) {
        s_bin = tid * PER + b;
        s_before = acc;
        break;
      }
      acc += hist[tid * PER + b];
    }
  }
  __syncthreads();
  if (tid == 0) {
    *cut = s_bin;
    if (below) *below = s_before;   // features in the bins before the cut bin
  }
}

__global__ void __launch_bounds__(256)
sis_compact_kernel(const double *r, long long n_feat, const unsigned *cut1, const unsigned *cut2,
                   u64 *keys, unsigned *idx, unsigned long long *count, long long cap) {
  const unsigned c1 = *cut1, c2 = *cut2;
  for (long long f = (long long)blockIdx.x * blockDim.x + threadIdx.x; f < n_feat;
       f += (long long)gridDim.x * blockDim.x) {
    const u64 k = sis_key(r[f]);
    const unsigned b1 = (unsigned)(k >> 48), b2 = (unsigned)(k >> 32) & 0xffffu;
    if (b1 < c1 || (b1 == c1 && b2 <= c2)) {
      const unsigned long long s = atomicAdd(count, 1ull);
      if ((long long)s < cap) {
        keys[s] = k;
        idx[s] = (unsigned)f;
      }
    }
  }
}

__device__ __forceinline__ bool sis_less(u64 ka, unsigned ia, u64 kb, unsigned ib) {
  return ka < kb || (ka == kb && ia < ib);
}

// one block: sort the candidates by (key, index), emit the first m
__global__ void __launch_bounds__(1024)
sis_sort_kernel(u64 *keys, unsigned *idx, const unsigned long long *count, long long cap,
                int m, const double *r, int *out_idx, double *out_r, int *err) {
  long long n = (long long)*count;
  if (n > cap) {
    if (threadIdx.x == 0) set_err(err, 12);
    n = cap;
  }
  long long P = 1;
  while (P < n) P <<= 1;
  for (long long i = n + threadIdx.x; i < P; i += blockDim.x) {
    keys[i] = ~0ull;
    idx[i] = 0xffffffffu;
  }
  __syncthreads();
  for (long long size = 2; size <= P; size <<= 1) {
    for (long long stride = size >> 1; stride > 0; stride >>= 1) {
      for (long long i = threadIdx.x; i < (P >> 1); i += blockDim.x) {
        const long long lo = 2 * stride * (i / stride) + (i % stride);
        const long long hi = lo + stride;
        const bool asc = ((lo & size) == 0);
        const u64 ka = keys[lo], kb = keys[hi];
        const unsigned ia = idx[lo], ib = idx[hi];
        const bool sw = asc ? sis_less(kb, ib, ka, ia) : sis_less(ka, ia, kb, ib);
        if (sw) {
          keys[lo] = kb; keys[hi] = ka;
          idx[lo] = ib; idx[hi] = ia;
        }
      }
      __syncthreads();
    }
  }
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    if (i < n) {
      out_idx[i] = (int)idx[i];
      out_r[i] = r[idx[i]];
    } else {
      out_idx[i] = -1;
      out_r[i] = 0.0;
    }
  }
}

}  // namespace

}  // namespace l0

// ------------------------------------------------------------- launcher --
namespace l0 {

size_t sis_scratch_bytes(long long n_feat, int m, long long n) {
  const long long cap = std::min<long long>(n_feat, 1ll << 22);
  return (size_t)n_feat * 8 + 64 + 65536 * 4 + 64 + (size_t)cap * 16 * 2 + (size_t)cap * 8 * 2 +
         (size_t)m * 16 + (size_t)n * 4 + 2048;
}

// scratch: sis_scratch_bytes; out_idx / out_r device [m]; err: device int
cudaError_t launch_sis(const double *X, const double *y, long long n, long long n_feat, int m,
                       int fp32_products, void *scratch, int *out_idx, double *out_r, int *err,
                       cudaStream_t st) {
  const long long cap = std::min<long long>(n_feat, 1ll << 22);
  char *p = (char *)scratch;
  auto take = [&](size_t bytes) {
    char *q = p;
    p += (bytes + 255) / 256 * 256;
    return q;
  };
  double *r = (double *)take((size_t)n_feat * 8);
  double *tgt = (double *)take(64);
  unsigned *hist = (unsigned *)take(65536 * 4);
  char *small = take(64);
  unsigned *cuts = (unsigned *)small;                                   // cut1, cut2
  unsigned long long *cnt = (unsigned long long *)(small + 16);         // below, count
  u64 *keys = (u64 *)take((size_t)cap * 16);
  unsigned *idx = (unsigned *)take((size_t)cap * 8);
  float *yc = (float *)take((size_t)n * 4);
  const unsigned g = (unsigned)std::min<long long>((n_feat + 255) / 256, 152 * 16);
  const unsigned gw = (unsigned)std::min<long long>((n_feat + 7) / 8, 152 * 32);
  cudaError_t e = cudaMemsetAsync(small, 0, 64, st);
  if (e != cudaSuccess) return e;
  sis_target_kernel<<<1, 1024, 0, st>>>(y, n, tgt);
  if (fp32_products) {
    sis_target32_kernel<<<1, 1024, 0, st>>>(y, n, tgt, yc);
    sis_score32_kernel<<<gw, 256, 0, st>>>(X, n, n_feat, yc, tgt, r, err);
  } else {
    sis_score_kernel<<<gw, 256, 0, st>>>(X, n, n_feat, y, tgt, r, err);
  }
  e = cudaMemsetAsync(hist, 0, 65536 * 4, st);
  if (e != cudaSuccess) return e;
  sis_hist_kernel<<<g, 256, 0, st>>>(r, n_feat, 0, cuts, hist);
  sis_cut_kernel<<<1, 1024, 0, st>>>(hist, m, cnt, cuts);
  e = cudaMemsetAsync(hist, 0, 65536 * 4, st);
  if (e != cudaSuccess) return e;
  sis_hist_kernel<<<g, 256, 0, st>>>(r, n_feat, 1, cuts, hist);
  sis_cut_kernel<<<1, 1024, 0, st>>>(hist, m, cnt, cuts + 1);
  sis_compact_kernel<<<g, 256, 0, st>>>(r, n_feat, cuts, cuts + 1, keys, idx, cnt + 1, cap);
  sis_sort_kernel<<<1, 1024, 0, st>>>(keys, idx, cnt + 1, cap, m, r, out_idx, out_r, err);
  return cudaGetLastError();
}

}  // namespace l0
