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
#include "l0_screen.cuh"
#include "l0_tc.cuh"

namespace l0 {

namespace {

__global__ void __launch_bounds__(1024)
sis_target_kernel(const double *y, long long n, double *out, double *yd, int *err) {
  y += (long long)blockIdx.x * n;            // one block per target
  yd += (long long)blockIdx.x * n;
  out += 8 * blockIdx.x;
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
    yd[i] = d;
    q = fma(d, d, q);
    t += d;
  }
  const double syy = block_sum(q);
  const double sy0 = block_sum(t);
  if (threadIdx.x == 0) {
    out[0] = mean;
    out[1] = syy;
    out[2] = sy0;
    if (!isfinite(syy)) set_err(err, 5);
  }
}

// Pearson r of one feature by one warp, in FP64 (all lanes take part; the
// value is valid in every lane): shifted-data sums over 16 samples per lane
// in flight; yd = y - mean(y) (computed once, the same rounding as inline).
// `finite` is cleared when a sample is NaN or Inf (exponent field all ones,
// tested on the high word so that the FP64 pipe only does the four sums).
__device__ __forceinline__ double sis_r64_warp(const double *__restrict__ x, long long n,
                                               const double *__restrict__ yd, double syy,
                                               double sy0, int lane, bool &finite) {
  const double c = __ldg(x);
  double S1 = 0.0, S2 = 0.0, S3 = 0.0;
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
      finite &= ((unsigned)__double2hiint(v[u]) & 0x7ff00000u) != 0x7ff00000u;
      const double d = v[u] - c;            // 0 past the end
      S1 += d;
      S2 = fma(d, d, S2);
      S3 = fma(d, (i < n) ? __ldg(yd + i) : 0.0, S3);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    S1 += __shfl_xor_sync(0xffffffffu, S1, o);
    S2 += __shfl_xor_sync(0xffffffffu, S2, o);
    S3 += __shfl_xor_sync(0xffffffffu, S3, o);
  }
  const double sxx = S2 - S1 * S1 / (double)n;
  const double sxy = S3 - S1 * sy0 / (double)n;
  return (sxx > 0.0 && syy > 0.0) ? sxy / sqrt(sxx * syy) : 0.0;
}

// The same for R targets at once (R <= SIS_MAX_TARGETS): the row is read
// once and S3 accumulated against every target's centred values yd[t][.];
// returns the signed r of the first target with the largest |r| (the
// projection score against several residuals).
__device__ __forceinline__ double sis_r64_multi_warp(const double *__restrict__ x, long long n,
                                                     const double *__restrict__ yd,
                                                     const double *__restrict__ tgt, int R,
                                                     int lane, bool &finite) {
  const double c = __ldg(x);
  double S1 = 0.0, S2 = 0.0, S3[SIS_MAX_TARGETS];
#pragma unroll
  for (int t = 0; t < SIS_MAX_TARGETS; ++t) S3[t] = 0.0;
  constexpr int U = 8;
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
      finite &= ((unsigned)__double2hiint(v[u]) & 0x7ff00000u) != 0x7ff00000u;
      const double d = v[u] - c;
      S1 += d;
      S2 = fma(d, d, S2);
      if (i < n) {
#pragma unroll
        for (int t = 0; t < SIS_MAX_TARGETS; ++t)
          if (t < R) S3[t] = fma(d, __ldg(yd + (long long)t * n + i), S3[t]);
      }
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    S1 += __shfl_xor_sync(0xffffffffu, S1, o);
    S2 += __shfl_xor_sync(0xffffffffu, S2, o);
#pragma unroll
    for (int t = 0; t < SIS_MAX_TARGETS; ++t)
      if (t < R) S3[t] += __shfl_xor_sync(0xffffffffu, S3[t], o);
  }
  const double sxx = S2 - S1 * S1 / (double)n;
  double best = 0.0, babs = -1.0;
#pragma unroll
  for (int t = 0; t < SIS_MAX_TARGETS; ++t)
    if (t < R) {
      const double syy = tgt[8 * t + 1], sy0 = tgt[8 * t + 2];
      const double sxy = S3[t] - S1 * sy0 / (double)n;
      const double rt = (sxx > 0.0 && syy > 0.0) ? sxy / sqrt(sxx * syy) : 0.0;
      if (fabs(rt) > babs) {
        babs = fabs(rt);
        best = rt;
      }
    }
  return best;
}

__global__ void __launch_bounds__(256)
sis_score_kernel(const double *__restrict__ X, long long n, long long n_feat,
                 const double *__restrict__ yd, const double *__restrict__ tgt, int R,
                 double *__restrict__ r_out, int *err) {
  const int lane = threadIdx.x & 31;
  const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
  const double syy = tgt[1], sy0 = tgt[2];
  for (long long f = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); f < n_feat;
       f += warps) {
    bool finite = true;
    const double r = R == 1 ? sis_r64_warp(X + f * n, n, yd, syy, sy0, lane, finite)
                            : sis_r64_multi_warp(X + f * n, n, yd, tgt, R, lane, finite);
    if (__any_sync(0xffffffffu, !finite) && lane == 0) set_err(err, 5);
    if (lane == 0) r_out[f] = r;
  }
}

// ---------------------------------------------------------- pre-screen --
// GB300's FP64 pipe retires ~1.7 FMA per clock per SM, so a scan with even
// one FP64 operation per sample falls far behind HBM.  The pre-screen does
// none: each sample is truncated to FP32 with integer operations, the sums
// run in FP32, and every feature gets an interval [lo, hi] that holds its
// exact |r|.  Only features whose interval reaches the m-th largest lower
// bound are re-scored by sis_r64_warp; the others cannot be selected.  The
// selection that follows is therefore the one the FP64 scan makes.
constexpr double SIS_U = 5.9604644775390625e-8;   // 2^-24, FP32 unit roundoff

// x with its 29 low mantissa bits cleared, as a float (exact), by integer
// operations: the exponent is re-biased by adding 128 to its low 8 bits
// (1023 - 127 = 896 = 128 mod 256).  Exact to |f - x| <= 2^-23 |x| for
// 2^-60 <= |x| < 2^61; |x| < 2^-60 (zero and subnormals included) gives 0,
// off by less than 2^-60.  mx keeps the largest |x| bit pattern (high word):
// SIS_MX_BAD or above (|x| >= 2^61, Inf, NaN) sends the feature to FP64.
constexpr unsigned SIS_MX_LO = 963u << 20;    // 2^-60
constexpr unsigned SIS_MX_BAD = 1084u << 20;  // 2^61
__device__ __forceinline__ float sis_trunc32(double v, unsigned &mx) {
  const unsigned hi = (unsigned)__double2hiint(v), lo = (unsigned)__double2loint(v);
  const unsigned a = hi & 0x7fffffffu;
  mx = max(mx, a);
  const unsigned t = __funnelshift_l(lo, hi, 3);          // (hi << 3) | (lo >> 29)
  const unsigned f = ((t + 0x40000000u) & 0x7fffffffu) | (hi & 0x80000000u);
  return a < SIS_MX_LO ? 0.f : __uint_as_float(f);
}

// Centred target in FP32, scaled by a power of two 2^-k with 2^-k sqrt(S_yy/n)
// in [0.5, 1): yc[i] = fl32((y_i - mean) 2^-k).  tgt[3] = S_yy 4^-k (exact),
// tgt[4] = sum yc^2, tgt[5] = sum yc (both FP64 over the rounded values).
__global__ void __launch_bounds__(1024)
sis_target32_kernel(const double *y, long long n, double *tgt, float *yc) {
  __shared__ double red[2][32];
  y += (long long)blockIdx.x * n;            // one block per target
  yc += (long long)blockIdx.x * n;
  tgt += 8 * blockIdx.x;
  const double mean = tgt[0], syy = tgt[1];
  int k = 0;
  if (syy > 0.0 && isfinite(syy)) frexp(sqrt(syy / (double)n), &k);
  double t = 0.0, q = 0.0;
  for (long long i = threadIdx.x; i < n; i += blockDim.x) {
    const float v = (float)ldexp(y[i] - mean, -k);
    yc[i] = v;
    t += (double)v;
    q = fma((double)v, (double)v, q);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    t += __shfl_xor_sync(0xffffffffu, t, o);
    q += __shfl_xor_sync(0xffffffffu, q, o);
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = t;
    red[1][threadIdx.x >> 5] = q;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double st = 0.0, sq = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) {
      st += red[0][i];
      sq += red[1][i];
    }
    tgt[3] = ldexp(syy, -2 * k);
    tgt[4] = sq;
    tgt[5] = st;
  }
}

// [lo, hi] around |r| from the FP32 sums S1, S2, S3 of a feature whose
// first sample is c (error model below)
__device__ __forceinline__ void sis_bounds(double S1, double S2, double S3, double c, bool bad,
                                           const double *tgt, long long n, double &lo,
                                           double &hi) {
  // |d_i - (x_i - c)| <= 2^-22 (|x_i| + |c|) + 2^-59 (two flushes below 2^-60)
  const double syy_s = tgt[3], syc2 = tgt[4], sy0 = tgt[5];
  const double nn = (double)n;
  const double g = 80.0 * SIS_U + nn * 2.220446049250313e-16;
  const double sxx = S2 - S1 * S1 / nn;
  const double sxy = S3 - S1 * sy0 / nn;
  const double sxx_lo = sxx - 3.0 * g * S2;
  const double E = (2.384185791015625e-7 * (sqrt(fmax(S2, 0.0) * (1.0 + g)) + 2.0 * sqrt(nn) * fabs(c)) +
                    1.7347234759768071e-18 * sqrt(nn)) *
                   (1.0 + 4.8e-7);
  lo = 0.0;
  hi = INFINITY;
  if (!bad && isfinite(S1) && isfinite(S2) && isfinite(S3) && syy_s > 0.0 && sxx_lo > 0.0 &&
      9.0 * E * E < sxx_lo && 30.0 * g * S2 < sxx_lo) {
    const double a = fabs(sxy / sqrt(sxx * syy_s));
    const double nx = sqrt(sxx_lo);
    const double eps =
        1.01 * (1.05 * E / (nx - E) + SIS_U + 2.0 * g * sqrt(S2 * syc2 / (sxx_lo * syy_s)) +
                a * 1.65 * g * S2 / sxx_lo) +
        1e-10;
    lo = fmax(a - eps, 0.0);
    hi = a + eps;
  }
}

// One warp per group of 32 features; writes lo_out[f] = max(|r~| - eps, 0)
// and hi_out[f] = |r~| + eps, eps bounding |r~ - r| for the exact r (and
// for the FP64 scan's r, which lies within n 2^-52 of it in the same terms).
// The warp streams the features of its group one after the other, leaving
// feature t's sums in lane t; the FP64 epilogue then runs once for all 32
// (a masked FP64 instruction costs the pipe as much as a full one).
//
// Error model, with d_i = fl32(t(x_i) - t(c)), t the truncation above and c
// the first sample: |d_i - (x_i - c)| <= (2^-22 (|d_i| + 2|c|) + 2^-59) / (1 - 2^-22),
// so the error vector e has
// ||e|| <= E = (2^-22 (sqrt(S2) + 2 sqrt(n)|c|) + 2^-59 sqrt(n)) (1 + 2^-21).
// The angle between the centred sample vector and its computed image is
// at most asin(||e|| / ||a||) <= 1.05 E / (||a~|| - E) while 3E < ||a~||.
// The FP32 partial sums (<= 64 terms per lane, then a 5-level tree) carry
// at most g sum|terms| with g = 80 u; by Cauchy-Schwarz this moves S_xx by
// <= 3 g S2 and S_xy by <= 2 g sqrt(S2 sum yc^2).  Rounding yc moves r by <= u.
__global__ void __launch_bounds__(256, 4)
sis_prescreen_kernel(const double *__restrict__ X, long long n, long long n_feat,
                     const float *__restrict__ yc, const double *__restrict__ tgt, int accum,
                     double *__restrict__ lo_out, double *__restrict__ hi_out) {
  const int lane = threadIdx.x & 31;
  const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
  constexpr int U = 16;
  constexpr long long CHUNK = 32 * U;
  for (long long g0 = ((long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * 32;
       g0 < n_feat; g0 += warps * 32) {
    const int G = (int)min(32ll, n_feat - g0);
    // lane t: sums of feature g0 + t (earlier chunks in FP64, the last in FP32)
    double D1 = 0.0, D2 = 0.0, D3 = 0.0, cm = 0.0;
    float F1 = 0.f, F2 = 0.f, F3 = 0.f;
    bool badm = false;
    for (int t = 0; t < G; ++t) {
      const double *x = X + (g0 + t) * n;
      const double c = __ldg(x);
      unsigned mx = 0;
      const float fc = sis_trunc32(c, mx);
      float a1 = 0.f, a2 = 0.f, a3 = 0.f;
      int pending = 0;
      for (long long b0 = 0; b0 < n; b0 += CHUNK) {    // same trip count in every lane
        double v[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const long long i = b0 + lane + 32 * u;
          v[u] = (i < n) ? __ldcs(x + i) : c;
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const long long i = b0 + lane + 32 * u;
          const float d = sis_trunc32(v[u], mx) - fc;      // 0 past the end
          a1 += d;
          a2 = fmaf(d, d, a2);
          a3 = fmaf(d, (i < n) ? __ldg(yc + i) : 0.f, a3);
        }
        const bool last = b0 + CHUNK >= n;
        if (++pending == 4 || last) {                      // <= 64 terms per lane
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) {
            a1 += __shfl_xor_sync(0xffffffffu, a1, o);
            a2 += __shfl_xor_sync(0xffffffffu, a2, o);
            a3 += __shfl_xor_sync(0xffffffffu, a3, o);
          }
          if (lane == t) {
            if (last) {
              F1 = a1;
              F2 = a2;
              F3 = a3;
            } else {                                      // n > 2048 only
              D1 += (double)a1;
              D2 += (double)a2;
              D3 += (double)a3;
            }
          }
          a1 = a2 = a3 = 0.f;
          pending = 0;
        }
      }
      const bool bad = __any_sync(0xffffffffu, mx >= SIS_MX_BAD);
      if (lane == t) {
        cm = c;
        badm = bad;
      }
    }
    if (lane < G) {
      double lo, hi;
      sis_bounds(D1 + (double)F1, D2 + (double)F2, D3 + (double)F3, cm, badm, tgt, n, lo, hi);
      if (accum) {                        // several targets: the largest bounds
        lo = fmax(lo, lo_out[g0 + lane]);
        hi = fmax(hi, hi_out[g0 + lane]);
      }
      lo_out[g0 + lane] = lo;
      hi_out[g0 + lane] = hi;
    }
  }
}

// The same pre-screen with the rows staged in shared memory by the TMA
// unit: each warp owns a ring of PB_STAGES buffers; lane 0 keeps
// PB_STAGES - 1 bulk copies (one segment of up to PB_SEG samples each) in
// flight while the warp reduces the oldest.  Feature-major rows are
// contiguous, so a segment is one copy; its start is rounded down to 16
// bytes (off = 1 when it falls on an odd sample) and its length up.  A copy
// that would end past the last sample of X stops one sample short and that
// sample is read directly.  Requires X 16-byte aligned.  With n <= 2 PB_SEG
// (YREG) every lane keeps the centred target of its sample positions in
// registers: the same positions recur in every row.
constexpr int PB_WARPS = 16, PB_STAGES = 3, PB_SEG = 512, PB_K = PB_SEG / 32;
constexpr int PB_STAGE_BYTES = PB_SEG * 8 + 16;
constexpr size_t PB_SMEM = (size_t)PB_WARPS * PB_STAGES * PB_STAGE_BYTES + PB_WARPS * PB_STAGES * 8;

// A warp's jobs in order: group kg (features (warp + kg warps) 32 + t),
// feature t of the group, segment s of the feature; advanced one job at a
// time (no divisions in the loop).
struct PbCursor {
  long long kg = 0;
  int t = 0, s = 0;
  __device__ __forceinline__ void advance(int nseg) {
    if (++s == nseg) {
      s = 0;
      if (++t == 32) {
        t = 0;
        ++kg;
      }
    }
  }
};

struct PbJob {
  long long f, e0;      // feature, first sample (flat index into X)
  int s, len, off;      // segment, samples, offset in the stage (0 or 1)
  bool tail;            // last sample read from global
  bool valid;
};

__device__ __forceinline__ PbJob pb_job(const PbCursor &cur, long long warp, long long warps,
                                        long long n, long long n_feat) {
  PbJob j;
  j.s = cur.s;
  j.f = (warp + cur.kg * warps) * 32 + cur.t;
  j.valid = j.f < n_feat;
  j.len = (int)min((long long)PB_SEG, n - (long long)j.s * PB_SEG);
  j.e0 = j.f * n + (long long)j.s * PB_SEG;
  j.off = (int)(j.e0 & 1);
  j.tail = ((j.off + j.len) & 1) && (j.e0 + j.len == n_feat * n);
  return j;
}

__device__ __forceinline__ void pb_issue(const PbJob &j, const double *X, uint32_t stage,
                                         uint32_t bar) {
  const uint32_t bytes = (uint32_t)(((j.off + j.len - (j.tail ? 1 : 0)) * 8 + 15) & ~15);
  tc::fence_proxy_async_smem();
  tc::mbar_expect_tx(bar, bytes);      // bytes = 0 (a lone tail sample): a plain arrive
  if (bytes) tc::bulk_load(stage, X + (j.e0 - j.off), bytes, bar);
}

template <bool YREG>
__global__ void __launch_bounds__(PB_WARPS * 32, 1)
sis_prescreen_bulk_kernel(const double *__restrict__ X, long long n, long long n_feat,
                          const float *__restrict__ yc, const double *__restrict__ tgt, int accum,
                          double *__restrict__ lo_out, double *__restrict__ hi_out, int *err) {
  extern __shared__ __align__(128) unsigned char smem[];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const long long warp = (long long)blockIdx.x * PB_WARPS + w;
  const long long warps = (long long)gridDim.x * PB_WARPS;
  unsigned char *ring = smem + (size_t)w * PB_STAGES * PB_STAGE_BYTES;
  const uint32_t bar0 =
      tc::smem_u32(smem + (size_t)PB_WARPS * PB_STAGES * PB_STAGE_BYTES) + w * PB_STAGES * 8;
  const uint32_t ring0 = tc::smem_u32(ring);
  const int nseg = (int)((n + PB_SEG - 1) / PB_SEG);
  if (lane == 0) {
    for (int b = 0; b < PB_STAGES; ++b) tc::mbar_init(bar0 + 8 * b, 1);
    tc::fence_proxy_async_smem();
  }
  __syncwarp();
  // producer cursor: PB_STAGES jobs ahead of the consumer once the ring is full
  PbCursor pc;
  for (int q = 0; q < PB_STAGES; ++q) {
    const PbJob j = pb_job(pc, warp, warps, n, n_feat);
    if (lane == 0 && j.valid) pb_issue(j, X, ring0 + q * PB_STAGE_BYTES, bar0 + 8 * q);
    pc.advance(nseg);
  }
  float yr0[PB_K], yr1[PB_K];
#pragma unroll
  for (int k = 0; k < PB_K; ++k) {
    const long long i = lane + 32 * k;
    yr0[k] = (YREG && i < n) ? yc[i] : 0.f;
    yr1[k] = (YREG && i + PB_SEG < n) ? yc[i + PB_SEG] : 0.f;
  }
  double D1 = 0.0, D2 = 0.0, D3 = 0.0, cm = 0.0;   // lane t: feature t of the group
  float F1 = 0.f, F2 = 0.f, F3 = 0.f;
  bool badm = false;
  float a1 = 0.f, a2 = 0.f, a3 = 0.f, b1 = 0.f, b2 = 0.f, b3 = 0.f;
  double c = 0.0;
  float fc = 0.f;
  unsigned mx = 0;
  PbCursor cc;
  int st = 0;
  uint32_t phase = 0;
  int inflight = 0;      // copies issued and not yet waited on (for the drain)
  for (;;) {
    const PbJob j = pb_job(cc, warp, warps, n, n_feat);
    if (!j.valid) break;
    if (!__all_sync(0xffffffffu, tc::mbar_wait(bar0 + 8 * st, phase, err))) {
      inflight = PB_STAGES - 1;     // the later copies may still be in flight
      break;
    }
    const double *sv = (const double *)(ring + (size_t)st * PB_STAGE_BYTES) + j.off;
    const int t = cc.t;
    if (j.s == 0) {
      c = sv[0];
      mx = 0;
      fc = sis_trunc32(c, mx);
    }
    const long long ib = (long long)j.s * PB_SEG;
    // one segment; yv: this lane's centred target values (YREG), by constant index
    auto segment = [&](const float (&yv)[PB_K]) {
      if (j.len == PB_SEG) {
#pragma unroll
        for (int k = 0; k < PB_K; k += 2) {
          const float d0 = sis_trunc32(sv[lane + 32 * k], mx) - fc;
          const float d1 = sis_trunc32(sv[lane + 32 * (k + 1)], mx) - fc;
          const float y0 = YREG ? yv[k] : __ldg(yc + ib + lane + 32 * k);
          const float y1 = YREG ? yv[k + 1] : __ldg(yc + ib + lane + 32 * (k + 1));
          a1 += d0;
          a2 = fmaf(d0, d0, a2);
          a3 = fmaf(d0, y0, a3);
          b1 += d1;
          b2 = fmaf(d1, d1, b2);
          b3 = fmaf(d1, y1, b3);
        }
      } else {
#pragma unroll
        for (int k = 0; k < PB_K; ++k) {
          const int i = lane + 32 * k;
          if (i < j.len) {
            const float d = sis_trunc32(sv[i], mx) - fc;
            const float y0 = YREG ? yv[k] : __ldg(yc + ib + i);
            a1 += d;
            a2 = fmaf(d, d, a2);
            a3 = fmaf(d, y0, a3);
          }
        }
      }
    };
    if (j.tail) {
      // the last sample of X came through a global load: stage it in place
      // (the stage holds PB_SEG + 2 samples, so the slot exists)
      __syncwarp();
      if (lane == 0) ((double *)sv)[j.len - 1] = __ldg(X + j.e0 + j.len - 1);
      __syncwarp();
    }
    if (j.s == 0)
      segment(yr0);
    else
      segment(yr1);
    const bool last = j.s == nseg - 1;
    if (last || (j.s & 3) == 3) {                   // <= 64 terms per lane
      a1 += b1;
      a2 += b2;
      a3 += b3;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        a1 += __shfl_xor_sync(0xffffffffu, a1, o);
        a2 += __shfl_xor_sync(0xffffffffu, a2, o);
        a3 += __shfl_xor_sync(0xffffffffu, a3, o);
      }
      if (lane == t) {
        if (last) {
          F1 = a1;
          F2 = a2;
          F3 = a3;
        } else {                                    // n > 4 PB_SEG only
          D1 += (double)a1;
          D2 += (double)a2;
          D3 += (double)a3;
        }
      }
      a1 = a2 = a3 = b1 = b2 = b3 = 0.f;
    }
    if (last) {
      const bool bad = __any_sync(0xffffffffu, mx >= SIS_MX_BAD);
      if (lane == t) {
        cm = c;
        badm = bad;
      }
    }
    // the stage is free once every lane has read it: refill it
    __syncwarp();
    {
      const PbJob jn = pb_job(pc, warp, warps, n, n_feat);
      if (lane == 0 && jn.valid) pb_issue(jn, X, ring0 + st * PB_STAGE_BYTES, bar0 + 8 * st);
      pc.advance(nseg);
    }
    const long long g0 = j.f - t;
    if (last && (t == 31 || j.f == n_feat - 1)) {   // group done: bounds of its features
      if (g0 + lane < n_feat) {
        double lo, hi;
        sis_bounds(D1 + (double)F1, D2 + (double)F2, D3 + (double)F3, cm, badm, tgt, n, lo, hi);
        if (accum) {                      // several targets: the largest bounds
          lo = fmax(lo, lo_out[g0 + lane]);
          hi = fmax(hi, hi_out[g0 + lane]);
        }
        lo_out[g0 + lane] = lo;
        hi_out[g0 + lane] = hi;
      }
      D1 = D2 = D3 = 0.0;
      F1 = F2 = F3 = 0.f;
      badm = false;
    }
    cc.advance(nseg);
    if (++st == PB_STAGES) {
      st = 0;
      phase ^= 1u;
    }
  }
  // drain after an expired wait: give the copies still in flight their time
  for (int r = 0; r < inflight; ++r) {
    cc.advance(nseg);
    if (++st == PB_STAGES) {
      st = 0;
      phase ^= 1u;
    }
    if (!pb_job(cc, warp, warps, n, n_feat).valid) break;
    if (!__all_sync(0xffffffffu, tc::mbar_wait(bar0 + 8 * st, phase, err))) break;
  }
}

// Several targets in one pass over X (the residual screening of the
// dimension loop): the FP32 centred values of all R targets sit in shared
// memory as target pairs ([R/2][n] float2, n <= PM_NMAX; an odd R padded
// with a zero target), each lane accumulates S3 for every target two at a
// time with fma.rn.f32x2 (each half the same fmaf as one at a time: the
// sums, and so the bounds, are unchanged, for half the instructions), and
// the epilogue takes, per feature, the largest lower and upper bounds over
// the targets -- an interval around max_t |r_t|.  Same staging, error model
// and cursors as sis_prescreen_bulk_kernel; 12 warps so that the targets fit
// beside the rings.
constexpr int PM_WARPS = 12;
constexpr int PM_NMAX = 2 * PB_SEG;
constexpr int PM_PAIRS = (SIS_MAX_TARGETS + 1) / 2;
constexpr size_t PM_RING_BYTES = (size_t)PM_WARPS * PB_STAGES * PB_STAGE_BYTES;
constexpr size_t pm_smem(int R, long long n) {
  return PM_RING_BYTES + (size_t)PM_WARPS * PB_STAGES * 8 + (size_t)((R + 1) / 2) * n * 8;
}

__global__ void __launch_bounds__(PM_WARPS * 32, 1)
sis_prescreen_multi_kernel(const double *__restrict__ X, long long n, long long n_feat,
                           const float *__restrict__ yc, const double *__restrict__ tgt, int R,
                           double *__restrict__ lo_out, double *__restrict__ hi_out, int *err) {
  extern __shared__ __align__(128) unsigned char smem[];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const long long warp = (long long)blockIdx.x * PM_WARPS + w;
  const long long warps = (long long)gridDim.x * PM_WARPS;
  unsigned char *ring = smem + (size_t)w * PB_STAGES * PB_STAGE_BYTES;
  const uint32_t bar0 = tc::smem_u32(smem + PM_RING_BYTES) + w * PB_STAGES * 8;
  float *ys = (float *)(smem + PM_RING_BYTES + (size_t)PM_WARPS * PB_STAGES * 8);
  const int RP = (R + 1) / 2;   // target pairs
  const uint32_t ring0 = tc::smem_u32(ring);
  const int nseg = (int)((n + PB_SEG - 1) / PB_SEG);    // 1 or 2
  if (lane == 0) {
    for (int b = 0; b < PB_STAGES; ++b) tc::mbar_init(bar0 + 8 * b, 1);
    tc::fence_proxy_async_smem();
  }
  __syncwarp();
  PbCursor pc;
  for (int q = 0; q < PB_STAGES; ++q) {
    const PbJob j = pb_job(pc, warp, warps, n, n_feat);
    if (lane == 0 && j.valid) pb_issue(j, X, ring0 + q * PB_STAGE_BYTES, bar0 + 8 * q);
    pc.advance(nseg);
  }
  // ys[(p n + i) 2 + h] = target 2p + h at sample i (0 past R)
  for (long long x = threadIdx.x; x < (long long)RP * n * 2; x += blockDim.x) {
    const long long pi = x >> 1;
    const int u = (int)(pi / n) * 2 + (int)(x & 1);
    const long long i = pi - (pi / n) * n;
    ys[x] = u < R ? yc[(long long)u * n + i] : 0.f;
  }
  __syncthreads();
  float F1 = 0.f, F2 = 0.f, F3[SIS_MAX_TARGETS];      // lane t: feature t of the group
  double cm = 0.0;
  bool badm = false;
  float a1 = 0.f, a2 = 0.f;
  unsigned long long a3p[PM_PAIRS];   // S3 of targets 2p, 2p + 1
#pragma unroll
  for (int t = 0; t < SIS_MAX_TARGETS; ++t) F3[t] = 0.f;
#pragma unroll
  for (int q = 0; q < PM_PAIRS; ++q) a3p[q] = 0ull;
  double c = 0.0;
  float fc = 0.f;
  unsigned mx = 0;
  PbCursor cc;
  int st = 0;
  uint32_t phase = 0;
  int inflight = 0;
  for (;;) {
    const PbJob j = pb_job(cc, warp, warps, n, n_feat);
    if (!j.valid) break;
    if (!__all_sync(0xffffffffu, tc::mbar_wait(bar0 + 8 * st, phase, err))) {
      inflight = PB_STAGES - 1;
      break;
    }
    const double *sv = (const double *)(ring + (size_t)st * PB_STAGE_BYTES) + j.off;
    const int t = cc.t;
    if (j.s == 0) {
      c = sv[0];
      mx = 0;
      fc = sis_trunc32(c, mx);
    }
    if (j.tail) {
      __syncwarp();
      if (lane == 0) ((double *)sv)[j.len - 1] = __ldg(X + j.e0 + j.len - 1);
      __syncwarp();
    }
    const unsigned long long *yb2 = (const unsigned long long *)ys + (long long)j.s * PB_SEG;
#pragma unroll 4
    for (int k = 0; k < PB_K; ++k) {
      const int i = lane + 32 * k;
      if (i < j.len) {
        const float d = sis_trunc32(sv[i], mx) - fc;
        a1 += d;
        a2 = fmaf(d, d, a2);
        const unsigned long long d2 = f2_pack(d, d);
#pragma unroll
        for (int q = 0; q < PM_PAIRS; ++q)
          if (q < RP) a3p[q] = f2_fma(d2, yb2[(long long)q * n + i], a3p[q]);
      }
    }
    const bool last = j.s == nseg - 1;
    if (last) {                                     // <= 32 terms per lane
      float a3[SIS_MAX_TARGETS];
#pragma unroll
      for (int q = 0; q < PM_PAIRS; ++q) {
        a3[2 * q] = __uint_as_float((unsigned)a3p[q]);
        if (2 * q + 1 < SIS_MAX_TARGETS) a3[2 * q + 1] = __uint_as_float((unsigned)(a3p[q] >> 32));
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        a1 += __shfl_xor_sync(0xffffffffu, a1, o);
        a2 += __shfl_xor_sync(0xffffffffu, a2, o);
#pragma unroll
        for (int u = 0; u < SIS_MAX_TARGETS; ++u)
          if (u < R) a3[u] += __shfl_xor_sync(0xffffffffu, a3[u], o);
      }
      const bool bad = __any_sync(0xffffffffu, mx >= SIS_MX_BAD);
      if (lane == t) {
        F1 = a1;
        F2 = a2;
#pragma unroll
        for (int u = 0; u < SIS_MAX_TARGETS; ++u) F3[u] = a3[u];
        cm = c;
        badm = bad;
      }
      a1 = a2 = 0.f;
#pragma unroll
      for (int q = 0; q < PM_PAIRS; ++q) a3p[q] = 0ull;
    }
    __syncwarp();
    {
      const PbJob jn = pb_job(pc, warp, warps, n, n_feat);
      if (lane == 0 && jn.valid) pb_issue(jn, X, ring0 + st * PB_STAGE_BYTES, bar0 + 8 * st);
      pc.advance(nseg);
    }
    const long long g0 = j.f - t;
    if (last && (t == 31 || j.f == n_feat - 1)) {
      if (g0 + lane < n_feat) {
        double lo = 0.0, hi = 0.0;
#pragma unroll
        for (int u = 0; u < SIS_MAX_TARGETS; ++u)
          if (u < R) {
            double l1, h1;
            sis_bounds((double)F1, (double)F2, (double)F3[u], cm, badm, tgt + 8 * u, n, l1, h1);
            lo = fmax(lo, l1);
            hi = fmax(hi, h1);
          }
        lo_out[g0 + lane] = lo;
        hi_out[g0 + lane] = hi;
      }
      badm = false;
    }
    cc.advance(nseg);
    if (++st == PB_STAGES) {
      st = 0;
      phase ^= 1u;
    }
  }
  for (int r = 0; r < inflight; ++r) {
    cc.advance(nseg);
    if (++st == PB_STAGES) {
      st = 0;
      phase ^= 1u;
    }
    if (!pb_job(cc, warp, warps, n, n_feat).valid) break;
    if (!__all_sync(0xffffffffu, tc::mbar_wait(bar0 + 8 * st, phase, err))) break;
  }
}

// --------------------------------------------------- generated features --
// On-the-fly feature values (paper Sec. 2: operators applied to child
// features; the last rung is evaluated inside SIS, Sec. 2.3 and Sec. 3).
// Candidate t is ops[t](C[c1[t]], C[c2[t]]) (unary operators read c1 only),
// evaluated in FP64 sample by sample and screened in the same pass: one warp
// per candidate, shifted-data sums as in sis_r64_warp.  Value rules: every
// value finite, the largest |value| in [lb, ub], not constant, not equal
// sample by sample to a child.  An invalid candidate's r is NaN (its key
// sorts after every score, so the selection never takes it).
__device__ __forceinline__ double gen_apply(int op, double a, double b) {
  switch (op) {
    case 0: return a + b;
    case 1: return a - b;
    case 2: return a * b;
    case 3: return a / b;
    case 4: return fabs(a - b);
    case 5: return log(a);
    case 6: return exp(a);
    case 7: return exp(-a);
    case 8: return fabs(a);
    case 9: return sqrt(a);
    case 10: return cbrt(a);
    case 11: return a * a;
    case 12: return a * a * a;
    default: return 1.0 / a;
  }
}

// FP64 r of candidate t by one warp (lane 0 returns it; NaN when the
// candidate breaks a value rule); *ok (all lanes) tells whether it is valid.
// A malformed candidate is reported (err 14) and never read.
__device__ double gen_r64_warp(const double *__restrict__ C, long long n, long long n_child,
                               const int *__restrict__ ops, const int *__restrict__ c1,
                               const int *__restrict__ c2, long long t,
                               const double *__restrict__ yd, double syy, double sy0, double lb,
                               double ub, int lane, bool *ok_out, int *err) {
  const int op = ops[t];
  const bool binary = op <= 4;
  if (op < 0 || op > 13 || c1[t] < 0 || c1[t] >= n_child ||
      (binary && (c2[t] < 0 || c2[t] >= n_child))) {
    if (lane == 0) set_err(err, 14);
    *ok_out = false;
    return __longlong_as_double(0x7ff8000000000000ll);
  }
  const double *xa = C + (long long)c1[t] * n;
  const double *xb = C + (long long)(binary ? c2[t] : c1[t]) * n;
  const double v0 = gen_apply(op, __ldg(xa), __ldg(xb));
  double S1 = 0.0, S2 = 0.0, S3 = 0.0, mx = 0.0;
  bool finite = true, same = true, eqa = true, eqb = binary;
  for (long long i = lane; i < n; i += 32) {
    const double a = __ldg(xa + i), b = __ldg(xb + i);
    const double v = gen_apply(op, a, b);
    finite &= ((unsigned)__double2hiint(v) & 0x7ff00000u) != 0x7ff00000u;
    mx = fmax(mx, fabs(v));
    same &= v == v0;
    eqa &= v == a;
    eqb &= v == b;
    const double d = v - v0;
    S1 += d;
    S2 = fma(d, d, S2);
    S3 = fma(d, __ldg(yd + i), S3);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    S1 += __shfl_xor_sync(0xffffffffu, S1, o);
    S2 += __shfl_xor_sync(0xffffffffu, S2, o);
    S3 += __shfl_xor_sync(0xffffffffu, S3, o);
    mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  }
  const bool ok = __all_sync(0xffffffffu, finite) && !__all_sync(0xffffffffu, same) &&
                  !__all_sync(0xffffffffu, eqa) && !(binary && __all_sync(0xffffffffu, eqb)) &&
                  mx <= ub && mx >= lb;
  *ok_out = ok;
  const double sxx = S2 - S1 * S1 / (double)n;
  const double sxy = S3 - S1 * sy0 / (double)n;
  double r = (sxx > 0.0 && syy > 0.0) ? sxy / sqrt(sxx * syy) : 0.0;
  if (!ok) r = __longlong_as_double(0x7ff8000000000000ll);
  return r;
}

__global__ void __launch_bounds__(256)
gen_score_kernel(const double *__restrict__ C, long long n, long long n_child,
                 const int *__restrict__ ops, const int *__restrict__ c1,
                 const int *__restrict__ c2, long long n_cand, const double *__restrict__ yd,
                 const double *__restrict__ tgt, double lb, double ub,
                 double *__restrict__ r_out, unsigned char *__restrict__ valid_out, int *err) {
  const int lane = threadIdx.x & 31;
  const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
  const double syy = tgt[1], sy0 = tgt[2];
  for (long long t = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); t < n_cand;
       t += warps) {
    bool ok = false;
    const double r = gen_r64_warp(C, n, n_child, ops, c1, c2, t, yd, syy, sy0, lb, ub, lane, &ok,
                                  err);
    if (lane == 0) {
      r_out[t] = r;
      if (valid_out) valid_out[t] = ok ? 1 : 0;
    }
  }
}

// FP64 r of the listed candidates (the pre-screen's survivors), one warp each
__global__ void __launch_bounds__(256)
gen_rescore_kernel(const double *__restrict__ C, long long n, long long n_child,
                   const int *__restrict__ ops, const int *__restrict__ c1,
                   const int *__restrict__ c2, const unsigned *list,
                   const unsigned long long *count, const double *__restrict__ yd,
                   const double *__restrict__ tgt, double lb, double ub,
                   double *__restrict__ r_out, int *err) {
  const int lane = threadIdx.x & 31;
  const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
  const long long nc = (long long)*count;
  const double syy = tgt[1], sy0 = tgt[2];
  for (long long q = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); q < nc;
       q += warps) {
    const long long t = list[q];
    bool ok = false;
    const double r = gen_r64_warp(C, n, n_child, ops, c1, c2, t, yd, syy, sy0, lb, ub, lane, &ok,
                                  err);
    if (lane == 0) r_out[t] = r;
  }
}

// ------------------------------------- generated features: FP32 pre-screen --
// The FP64 evaluation above keeps GB300's FP64 pipe busy (~10 FP64
// instructions per sample).  The pre-screen evaluates every candidate in FP32
// from an FP32 copy of the children, carries for each sample a bound beta on
// |value32 - value| (the operator's rounding, CUDA's documented accuracy of
// logf / expf / cbrtf -- 1, 2 and 1 ulp; sqrtf and division are IEEE --, and
// the inputs' own rounding), and turns the FP32 Pearson sums into an interval
// [lo, hi] around the exact |r| with the error model of sis_bounds, E being
// the norm of the per-sample bounds of the shifted values.  The value rules
// are decided only when the bounds settle them: "certainly invalid" (a
// non-finite FP32 value, or max |value| outside [lb, ub] by more than its
// bound) gives hi = NaN; "certainly valid" (finite, inside the bounds with
// room, some sample distinct from the first and from each child by more than
// the bounds) keeps lo; anything unsettled gets lo = 0 and, when the bounds
// do not hold (children or values outside [1e-30, 1e30]), hi = +inf.  The
// m-th largest lo is then a score at least m valid candidates reach, and
// only candidates whose hi reaches it are evaluated in FP64.

__device__ __forceinline__ float gen_apply32(int op, float a, float b) {
  switch (op) {
    case 0: return a + b;
    case 1: return a - b;
    case 2: return a * b;
    case 3: return a / b;
    case 4: return fabsf(a - b);
    case 5: return logf(a);
    case 6: return expf(a);
    case 7: return expf(-a);
    case 8: return fabsf(a);
    case 9: return sqrtf(a);
    case 10: return cbrtf(a);
    case 11: return a * a;
    case 12: return a * a * a;
    default: return 1.f / a;
  }
}

// bound on |v - op(a_exact, b_exact)| for v = gen_apply32(op, a, b), where a
// and b are the round-to-nearest FP32 images of the exact children (relative
// error <= u each) and v is finite
__device__ __forceinline__ float gen_beta32(int op, float a, float b, float v) {
  constexpr float u = 5.9604644775390625e-8f;   // 2^-24
  const float av = fabsf(v);
  float rel, abs0 = 0.f;
  switch (op) {
    case 0: case 1: case 4: abs0 = u * (fabsf(a) + fabsf(b) + av); rel = 0.f; break;
    case 2: case 3: case 11: rel = 4.f * u; break;
    case 5: abs0 = 1.01f * u; rel = 2.01f * u; break;   // input: log(1 + d) ~ d; logf 1 ulp
    case 6: case 7: rel = 1.01f * u * fabsf(a) + 4.01f * u; break;   // exp(a + e) = exp(a)(1 + e); expf 2 ulp
    case 8: rel = 1.01f * u; break;
    case 9: rel = 1.6f * u; break;    // sqrt(a(1 + d)) = sqrt(a)(1 + d/2); sqrtf correctly rounded
    case 10: rel = 2.5f * u; break;   // input d/3; cbrtf 1 ulp
    case 12: rel = 6.f * u; break;
    default: rel = 3.f * u; break;    // 1/a: input + one rounding
  }
  return (abs0 + rel * av) * 1.001f + 1e-37f;
}

// children in FP32 (round to nearest) and, per child, whether every value is
// 0 or within [1e-30, 1e30] (the FP32 error model's range); one warp each
__global__ void __launch_bounds__(256)
gen_child32_kernel(const double *__restrict__ C, long long n, long long n_child,
                   float *__restrict__ Cf, unsigned char *__restrict__ safe) {
  const int lane = threadIdx.x & 31;
  const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
  for (long long c = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); c < n_child;
       c += warps) {
    bool ok = true;
    for (long long i = lane; i < n; i += 32) {
      const double x = __ldg(C + c * n + i);
      const double ax = fabs(x);
      ok &= (x == 0.0) || (ax >= 1e-30 && ax <= 1e30);
      Cf[c * n + i] = __double2float_rn(x);
    }
    ok = __all_sync(0xffffffffu, ok);
    if (lane == 0) safe[c] = ok ? 1 : 0;
  }
}

// [lo, hi] around |r| from FP32 sums of shifted values whose error vector has
// norm <= E (see sis_bounds; the partial sums hold ceil(n / 32) terms a lane)
__device__ __forceinline__ void gen_bounds(double S1, double S2, double S3, double E,
                                           const double *tgt, long long n, double &lo,
                                           double &hi) {
  const double syy_s = tgt[3], syc2 = tgt[4], sy0 = tgt[5];
  const double nn = (double)n;
  const double terms = (double)((n + 31) / 32) + 16.0;
  const double g = fmax(80.0, 1.1 * terms) * SIS_U + nn * 2.220446049250313e-16;
  const double sxx = S2 - S1 * S1 / nn;
  const double sxy = S3 - S1 * sy0 / nn;
  const double sxx_lo = sxx - 3.0 * g * S2;
  lo = 0.0;
  hi = INFINITY;
  if (isfinite(S1) && isfinite(S2) && isfinite(S3) && isfinite(E) && syy_s > 0.0 &&
      sxx_lo > 0.0 && 9.0 * E * E < sxx_lo && 30.0 * g * S2 < sxx_lo) {
    const double a = fabs(sxy / sqrt(sxx * syy_s));
    const double nx = sqrt(sxx_lo);
    const double eps =
        1.01 * (1.05 * E / (nx - E) + SIS_U + 2.0 * g * sqrt(S2 * syc2 / (sxx_lo * syy_s)) +
                a * 1.65 * g * S2 / sxx_lo) +
        1e-10;
    lo = fmax(a - eps, 0.0);
    hi = a + eps;
  }
}

// One warp per group of 32 candidates: the warp evaluates them one after
// the other (lanes over samples) and leaves candidate t's sums and flags in
// lane t; the FP64 epilogue (interval, rules) then runs once for all 32 -- an
// FP64 instruction costs the SM the same whatever its active lanes.
__global__ void __launch_bounds__(256)
gen_prescreen_kernel(const float *__restrict__ Cf, const unsigned char *__restrict__ safe,
                     long long n, long long n_child, const int *__restrict__ ops,
                     const int *__restrict__ c1, const int *__restrict__ c2, long long n_cand,
                     const float *__restrict__ yc, const double *__restrict__ tgt, double lb,
                     double ub, double *__restrict__ lo_out, double *__restrict__ hi_out) {
  constexpr float u = 5.9604644775390625e-8f;
  const int lane = threadIdx.x & 31;
  const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
  for (long long g0 = ((long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * 32;
       g0 < n_cand; g0 += warps * 32) {
    const int G = (int)min(32ll, n_cand - g0);
    // lane t: candidate g0 + t
    float S1 = 0.f, S2 = 0.f, S3 = 0.f, E2 = 0.f, MXH = 0.f, MXL = 0.f;
    unsigned F = 0u;   // bits: 1 malformed, 2 finite, 4 vsafe, 8 dif0, 16 difa, 32 difb,
                       // 64 binary, 128 children safe
    for (int t = 0; t < G; ++t) {
      const long long c = g0 + t;
      const int op = ops[c];
      const bool binary = op <= 4;
      if (op < 0 || op > 13 || c1[c] < 0 || c1[c] >= n_child ||
          (binary && (c2[c] < 0 || c2[c] >= n_child))) {
        if (lane == t) F = 1u;   // malformed: the FP64 re-score reports it
        continue;
      }
      const long long ca = c1[c], cb = binary ? c2[c] : ca;
      const float *xa = Cf + ca * n, *xb = Cf + cb * n;
      const float a0 = __ldg(xa), b0 = __ldg(xb);
      const float v0 = gen_apply32(op, a0, b0);
      const float be0 = isfinite(v0) ? gen_beta32(op, a0, b0, v0) : 0.f;
      float s1 = 0.f, s2 = 0.f, s3 = 0.f, e2 = 0.f, mxhi = 0.f, mxlo = 0.f;
      bool finite = true, vsafe = true, dif0 = false, difa = false, difb = false;
      for (long long i = lane; i < n; i += 32) {
        const float a = __ldg(xa + i), b = __ldg(xb + i);
        const float v = gen_apply32(op, a, b);
        const float av = fabsf(v);
        const bool fin = isfinite(v);
        finite &= fin;
        vsafe &= (v == 0.f) || (av >= 1e-30f && av <= 1e30f);
        const float be = fin ? gen_beta32(op, a, b, v) : 0.f;
        mxhi = fmaxf(mxhi, av + be);
        mxlo = fmaxf(mxlo, av - be);
        // distinct beyond the bounds (1e-6 covers the FP32 rounding of these tests)
        dif0 |= fabsf(v - v0) > 1.001f * (be + be0) + 1e-6f * (av + fabsf(v0));
        difa |= fabsf(v - a) > 1.001f * (be + u * fabsf(a)) + 1e-6f * (av + fabsf(a));
        difb |= binary && fabsf(v - b) > 1.001f * (be + u * fabsf(b)) + 1e-6f * (av + fabsf(b));
        const float d = v - v0;
        s1 += d;
        s2 = fmaf(d, d, s2);
        s3 = fmaf(d, __ldg(yc + i), s3);
        const float ed = be + be0 + u * fabsf(d);
        e2 = fmaf(ed, ed, e2);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        s1 += __shfl_xor_sync(0xffffffffu, s1, o);
        s2 += __shfl_xor_sync(0xffffffffu, s2, o);
        s3 += __shfl_xor_sync(0xffffffffu, s3, o);
        e2 += __shfl_xor_sync(0xffffffffu, e2, o);
        mxhi = fmaxf(mxhi, __shfl_xor_sync(0xffffffffu, mxhi, o));
        mxlo = fmaxf(mxlo, __shfl_xor_sync(0xffffffffu, mxlo, o));
      }
      const unsigned f = (__all_sync(0xffffffffu, finite) ? 2u : 0u) |
                         (__all_sync(0xffffffffu, vsafe) ? 4u : 0u) |
                         (__any_sync(0xffffffffu, dif0) ? 8u : 0u) |
                         (__any_sync(0xffffffffu, difa) ? 16u : 0u) |
                         (__any_sync(0xffffffffu, difb) ? 32u : 0u) | (binary ? 64u : 0u) |
                         ((safe[ca] && safe[cb]) ? 128u : 0u);
      if (lane == t) {
        S1 = s1;
        S2 = s2;
        S3 = s3;
        E2 = e2;
        MXH = mxhi;
        MXL = mxlo;
        F = f;
      }
    }
    if (lane < G) {
      double lo = 0.0, hi = INFINITY;
      if (!(F & 1u)) {
        const bool children_safe = F & 128u, finite = F & 2u, vsafe = F & 4u;
        const bool bounded = children_safe && vsafe && finite;
        // certainly invalid: decided by FP32 values whatever their error (the
        // 1e-6 margins cover the FP32 rounding of |v| +- beta)
        const bool invalid =
            children_safe && ub <= 1e30 &&
            (!finite || (double)MXL > ub * (1.0 + 1e-6) ||
             (finite && vsafe && (double)MXH < lb * (1.0 - 1e-6)));
        const bool valid = bounded && (double)MXH <= ub * (1.0 - 1e-6) &&
                           (double)MXL >= lb * (1.0 + 1e-6) && (F & 8u) && (F & 16u) &&
                           (!(F & 64u) || (F & 32u));
        if (invalid) {
          lo = hi = __longlong_as_double(0x7ff8000000000000ll);
        } else if (bounded) {
          // the FP32 sum of squared bounds, inflated for its own rounding
          const double E = sqrt((double)E2 * (1.0 + 64.0 * (double)u * (double)((n + 31) / 32 + 8))) *
                               1.0001 + 1e-30;
          gen_bounds((double)S1, (double)S2, (double)S3, E, tgt, n, lo, hi);
          if (!valid) lo = 0.0;
        }
      }
      lo_out[g0 + lane] = lo;
      hi_out[g0 + lane] = hi;
    }
  }
}

// ordered image of -|r| (ascending = best first)
__device__ __forceinline__ u64 sis_key(double r) { return r != r ? ~0ull : ord_of(-fabs(r)); }

// Level-0 histogram privatised per block: 65536 16-bit counters packed two
// to a word in shared memory (a block takes at most 65535 features), then
// one global atomic per non-empty bin and block.
constexpr int H0_THREADS = 1024;
constexpr long long H0_MAX_PER_BLOCK = 65535;
__global__ void __launch_bounds__(H0_THREADS)
sis_hist0_kernel(const double *r, long long n_feat, long long per, unsigned *hist) {
  extern __shared__ unsigned sh[];          // 32768 words
  for (int i = threadIdx.x; i < 32768; i += H0_THREADS) sh[i] = 0u;
  __syncthreads();
  const long long f0 = (long long)blockIdx.x * per;
  const long long f1 = min(n_feat, f0 + per);
  for (long long f = f0 + threadIdx.x; f < f0 + (per + 31) / 32 * 32; f += H0_THREADS) {
    unsigned bin = 0xffffffffu;
    if (f < f1) bin = (unsigned)(sis_key(r[f]) >> 48);
    const unsigned peers = __match_any_sync(0xffffffffu, bin);
    if (bin != 0xffffffffu && (threadIdx.x & 31) == __ffs(peers) - 1)
      atomicAdd(sh + (bin >> 1), (unsigned)__popc(peers) << (16 * (bin & 1)));
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 32768; i += H0_THREADS) {
    const unsigned v = sh[i];
    if (v & 0xffffu) atomicAdd(hist + 2 * i, v & 0xffffu);
    if (v >> 16) atomicAdd(hist + 2 * i + 1, v >> 16);
  }
}

// level 0: bins of the top 16 bits of the key; level 1: the next 16 bits
// within the level-0 bin *cut1.  Lanes that hit the same bin add once.
__global__ void __launch_bounds__(256)
sis_hist_kernel(const double *r, long long n_feat, int level, const unsigned *cut1,
                unsigned *hist) {
  const unsigned c1 = level ? *cut1 : 0u;
  const long long stride = (long long)gridDim.x * blockDim.x;
  const long long end = (n_feat + 31) / 32 * 32;         // whole warps stay in the loop
  for (long long f = (long long)blockIdx.x * blockDim.x + threadIdx.x; f < end; f += stride) {
    unsigned bin = 0xffffffffu;
    if (f < n_feat) {
      const u64 k = sis_key(r[f]);
      const unsigned b1 = (unsigned)(k >> 48);
      if (level == 0) bin = b1;
      else if (b1 == c1) bin = (unsigned)(k >> 32) & 0xffffu;
    }
    const unsigned peers = __match_any_sync(0xffffffffu, bin);
    if (bin != 0xffffffffu && (threadIdx.x & 31) == __ffs(peers) - 1)
      atomicAdd(hist + bin, (unsigned)__popc(peers));
  }
}

// one block of 1024: the smallest bin b with before + count(bins <= b) >= want.
// Each thread holds 64 bins in registers (16 vector loads issued together);
// a warp-shuffle scan gives every thread the count before its bins.
__global__ void __launch_bounds__(1024)
sis_cut_kernel(const unsigned *hist, long long want, unsigned long long *below, unsigned *cut) {
  __shared__ unsigned long long wsum[32];
  __shared__ unsigned s_bin;
  __shared__ unsigned long long s_before;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const unsigned long long base = below ? *below : 0ull;
  const uint4 *h4 = (const uint4 *)hist + tid * 16;
  uint4 v[16];
#pragma unroll
  for (int k = 0; k < 16; ++k) v[k] = h4[k];
  unsigned long long s = 0;
#pragma unroll
  for (int k = 0; k < 16; ++k) s += (unsigned long long)v[k].x + v[k].y + v[k].z + v[k].w;
  if (tid == 0) {
    s_bin = 0xffffu;
    s_before = base;
  }
  unsigned long long inc = s;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned long long t = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += t;
  }
  if (lane == 31) wsum[w] = inc;
  __syncthreads();
  if (w == 0) {
    unsigned long long t = wsum[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long u = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += u;
    }
    wsum[lane] = t;
  }
  __syncthreads();
  inc += w ? wsum[w - 1] : 0ull;
  const unsigned long long before = base + inc - s;
  const unsigned long long W = (unsigned long long)want;
  if (before < W && base + inc >= W) {
    unsigned long long acc = before;
    bool found = false;
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      const unsigned c4[4] = {v[k].x, v[k].y, v[k].z, v[k].w};
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        if (!found && acc + c4[q] >= W) {
          found = true;
          s_bin = tid * 64 + 4 * k + q;
          s_before = acc;
        }
        if (!found) acc += c4[q];
      }
    }
  }
  __syncthreads();
  if (tid == 0) {
    *cut = s_bin;
    if (below) *below = s_before;   // features in the bins before the cut bin
  }
}

// append (key, index) of every feature at or before the cut bin; one
// atomic per warp
__global__ void __launch_bounds__(256)
sis_compact_kernel(const double *r, long long n_feat, const unsigned *cut1, const unsigned *cut2,
                   u64 *keys, unsigned *idx, unsigned long long *count, long long cap,
                   unsigned long long *krange) {
  const unsigned c1 = *cut1, c2 = *cut2;
  const int lane = threadIdx.x & 31;
  const long long stride = (long long)gridDim.x * blockDim.x;
  const long long end = (n_feat + 31) / 32 * 32;
  for (long long f = (long long)blockIdx.x * blockDim.x + threadIdx.x; f < end; f += stride) {
    bool take = false;
    u64 k = 0;
    if (f < n_feat) {
      k = sis_key(r[f]);
      const unsigned b1 = (unsigned)(k >> 48), b2 = (unsigned)(k >> 32) & 0xffffu;
      take = (b1 < c1 || (b1 == c1 && b2 <= c2)) && k != ~0ull;   // never a NaN (excluded, invalid)
    }
    const unsigned ball = __ballot_sync(0xffffffffu, take);
    if (!ball) continue;
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(count, (unsigned long long)__popc(ball));
    base = __shfl_sync(0xffffffffu, base, 0);
    // key range of the taken: krange[0] = max ~key, krange[1] = max key
    unsigned long long kn = take ? ~k : 0ull, kx = take ? k : 0ull;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      kn = max(kn, __shfl_xor_sync(0xffffffffu, kn, o));
      kx = max(kx, __shfl_xor_sync(0xffffffffu, kx, o));
    }
    if (lane == 0) {
      atomicMax(krange, kn);
      atomicMax(krange + 1, kx);
    }
    if (take) {
      const unsigned long long s = base + __popc(ball & ((1u << lane) - 1u));
      if ((long long)s < cap) {
        keys[s] = k;
        idx[s] = (unsigned)f;
      }
    }
  }
}

// Pre-screen candidates: a feature whose upper bound hi reaches the cut bin
// of the lower bounds (key prefix <= (cut1, cut2)) is listed for the FP64
// re-score; any other feature has |r| below the m-th largest |r| and its
// entry of r becomes 0.
__global__ void __launch_bounds__(256)
sis_candidates_kernel(const double *hi, long long n_feat, const unsigned *cut1,
                      const unsigned *cut2, double *r, unsigned *list,
                      unsigned long long *count) {
  const unsigned long long P = ((unsigned long long)*cut1 << 16) | *cut2;
  const int lane = threadIdx.x & 31;
  const long long stride = (long long)gridDim.x * blockDim.x;
  const long long end = (n_feat + 31) / 32 * 32;
  for (long long f = (long long)blockIdx.x * blockDim.x + threadIdx.x; f < end; f += stride) {
    bool take = false;
    if (f < n_feat) {
      const double h = hi[f];
      take = (sis_key(h) >> 32) <= P;
      if (!take) r[f] = (h != h) ? h : 0.0;      // excluded stay NaN
    }
    const unsigned ball = __ballot_sync(0xffffffffu, take);
    if (!ball) continue;
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(count, (unsigned long long)__popc(ball));
    base = __shfl_sync(0xffffffffu, base, 0);
    if (take) list[base + __popc(ball & ((1u << lane) - 1u))] = (unsigned)f;
  }
}

// FP64 r of the listed candidates, one warp each
__global__ void __launch_bounds__(256)
sis_rescore_kernel(const double *__restrict__ X, long long n, const unsigned *list,
                   const unsigned long long *count, const double *__restrict__ yd,
                   const double *__restrict__ tgt, int R, double *__restrict__ r_out, int *err) {
  const int lane = threadIdx.x & 31;
  const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
  const long long nc = (long long)*count;
  const double syy = tgt[1], sy0 = tgt[2];
  for (long long t = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); t < nc;
       t += warps) {
    const long long f = list[t];
    bool finite = true;
    const double r = R == 1 ? sis_r64_warp(X + f * n, n, yd, syy, sy0, lane, finite)
                            : sis_r64_multi_warp(X + f * n, n, yd, tgt, R, lane, finite);
    if (__any_sync(0xffffffffu, !finite) && lane == 0) set_err(err, 5);
    if (lane == 0) r_out[f] = r;
  }
}

// Excluded features (already selected): NaN in the given arrays, whose key
// sorts after every score, so that no cut, candidate list or compaction
// takes them.
__global__ void __launch_bounds__(256)
sis_exclude_kernel(const int *ex, long long n_ex, double *a, double *b) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n_ex;
       i += (long long)gridDim.x * blockDim.x) {
    const long long j = ex[i];
    a[j] = __longlong_as_double(0x7ff8000000000000ll);
    if (b) b[j] = __longlong_as_double(0x7ff8000000000000ll);
  }
}

__device__ __forceinline__ bool sis_less(u64 ka, unsigned ia, u64 kb, unsigned ib) {
  return ka < kb || (ka == kb && ia < ib);
}

// Exact order of up to SIS_RANK_MAX compacted candidates.  The key range
// [kmin, kmax] is cut into SIS_NB buckets by the leading bits of key - kmin
// (monotone in the key); a pair's rank is the count of the buckets before
// its own plus the pairs of its bucket that precede it by (key, index).
// All pairs differ in the index, so the ranks are a permutation.
constexpr long long SIS_RANK_MAX = 65536;
constexpr int SIS_NB = 4096;

__device__ __forceinline__ unsigned sis_bucket(u64 k, const unsigned long long *krange) {
  const u64 kmin = ~krange[0], span = krange[1] - kmin;
  const int shift = max(0, 64 - __clzll((long long)span) - 12);   // span >> shift < 4096
  return (unsigned)((k - kmin) >> shift);
}

__global__ void __launch_bounds__(256)
sis_bucket_kernel(const u64 *keys, const unsigned long long *count, long long cap,
                  const unsigned long long *krange, unsigned *bidx, unsigned *bcount) {
  const long long c = min((long long)*count, cap);
  if (c > SIS_RANK_MAX) return;                 // sis_sort_kernel orders these
  const long long end = (c + 31) / 32 * 32;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < end;
       i += (long long)gridDim.x * blockDim.x) {
    unsigned b = 0xffffffffu;
    if (i < c) {
      b = sis_bucket(keys[i], krange);
      bidx[i] = b;
    }
    const unsigned peers = __match_any_sync(0xffffffffu, b);
    if (b != 0xffffffffu && (threadIdx.x & 31) == __ffs(peers) - 1)
      atomicAdd(bcount + b, (unsigned)__popc(peers));
  }
}

// one block of 1024: exclusive scan of the SIS_NB bucket counts
__global__ void __launch_bounds__(1024)
sis_bucket_scan_kernel(const unsigned *bcount, unsigned *bstart) {
  __shared__ unsigned wsum[32];
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const uint4 v = ((const uint4 *)bcount)[tid];
  const unsigned s = v.x + v.y + v.z + v.w;
  unsigned inc = s;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned t = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += t;
  }
  if (lane == 31) wsum[w] = inc;
  __syncthreads();
  if (w == 0) {
    unsigned t = wsum[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned u = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += u;
    }
    wsum[lane] = t;
  }
  __syncthreads();
  const unsigned ex = inc - s + (w ? wsum[w - 1] : 0u);
  ((uint4 *)bstart)[tid] = make_uint4(ex, ex + v.x, ex + v.x + v.y, ex + v.x + v.y + v.z);
}

__global__ void __launch_bounds__(256)
sis_bucket_place_kernel(const unsigned long long *count, long long cap, const unsigned *bidx,
                        const unsigned *bstart, unsigned *bfill, unsigned *order) {
  const long long c = min((long long)*count, cap);
  if (c > SIS_RANK_MAX) return;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < c;
       i += (long long)gridDim.x * blockDim.x) {
    const unsigned b = bidx[i];
    order[bstart[b] + atomicAdd(bfill + b, 1u)] = (unsigned)i;
  }
}

__global__ void __launch_bounds__(256)
sis_rank_kernel(const u64 *keys, const unsigned *idx, const unsigned long long *count,
                long long cap, const unsigned *bidx, const unsigned *bstart,
                const unsigned *bcount, const unsigned *order, unsigned *rank) {
  const long long c = min((long long)*count, cap);
  if (c > SIS_RANK_MAX) return;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < c;
       i += (long long)gridDim.x * blockDim.x) {
    const u64 ki = keys[i];
    const unsigned ii = idx[i], b = bidx[i];
    const unsigned s0 = bstart[b], nb = bcount[b];
    unsigned cnt = s0;
    for (unsigned t = s0; t < s0 + nb; ++t) {
      const unsigned jx = order[t];
      const u64 kj = keys[jx];
      cnt += (kj < ki || (kj == ki && idx[jx] < ii)) ? 1u : 0u;
    }
    rank[i] = cnt;
  }
}

__global__ void __launch_bounds__(256)
sis_scatter_kernel(const unsigned *idx, const unsigned *rank, const unsigned long long *count,
                   long long cap, int m, const double *r, int *out_idx, double *out_r) {
  const long long c = min((long long)*count, cap);
  if (c > SIS_RANK_MAX) return;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < max(c, (long long)m);
       i += (long long)gridDim.x * blockDim.x) {
    if (i < c) {
      const unsigned q = rank[i];
      if (q < (unsigned)m) {
        out_idx[q] = (int)idx[i];
        out_r[q] = r[idx[i]];
      }
    } else {
      out_idx[i] = -1;
      out_r[i] = 0.0;
    }
  }
}

// Above SIS_RANK_MAX candidates (many features tied near the cut): one
// block sorts them by (key, index) and emits the first m.
__global__ void __launch_bounds__(1024)
sis_sort_kernel(u64 *keys, unsigned *idx, const unsigned long long *count, long long cap,
                int m, const double *r, int *out_idx, double *out_r, int *err) {
  long long n = (long long)*count;
  if (n > cap) {
    if (threadIdx.x == 0) set_err(err, 12);
    n = cap;
  }
  if (n <= SIS_RANK_MAX) return;
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

size_t sis_scratch_bytes(long long n_feat, int m, long long n, int R) {
  const long long cap = std::min<long long>(n_feat, 1ll << 22);
  const long long rcap = std::min<long long>(cap, SIS_RANK_MAX);
  (void)m;
  return 256 * 2 + (size_t)n_feat * (8 + 8 + 4) + 256 + 65536 * 4 + (size_t)cap * (16 + 8) +
         (size_t)rcap * 12 + (size_t)SIS_NB * 12 + (size_t)n * 12 * R + 64 * (size_t)R + 22 * 256;
}

// y: R targets [R][n] (R <= SIS_RMAX); ex: n_ex distinct feature indices
// never selected (device; may be null when n_ex = 0).
// scratch: sis_scratch_bytes, its first 64 bytes the counters (bytes
// [40, 48): features re-scored in FP64 by the pre-screen path);
// out_idx / out_r device [m]; err: device int; scan0 / scan1 (optional):
// events recorded around the scan kernel (pre-screen or FP64 score); gen
// (optional): the candidates are generated features of the children X
// (n_feat = candidates, R = 1)
cudaError_t launch_sis(const double *X, const double *y, int R, long long n, long long n_feat,
                       int m, const int *ex, long long n_ex, int prescreen, void *scratch,
                       int *out_idx, double *out_r, int *err, cudaStream_t st, cudaEvent_t scan0,
                       cudaEvent_t scan1, const SisGen *gen) {
  const long long cap = std::min<long long>(n_feat, 1ll << 22);
  const long long rcap = std::min<long long>(cap, SIS_RANK_MAX);
  char *p = (char *)scratch;
  auto take = [&](size_t bytes) {
    char *q = p;
    p += (bytes + 255) / 256 * 256;
    return q;
  };
  char *small = take(64);
  unsigned *cuts = (unsigned *)small;                                 // selection cut1, cut2
  unsigned *pcuts = cuts + 2;                                         // pre-screen cut1, cut2
  unsigned long long *cnt = (unsigned long long *)(small + 16);       // below, count
  unsigned long long *pcnt = cnt + 2;                                 // below, candidates
  unsigned long long *krange = (unsigned long long *)take(64);        // max ~key, max key
  double *r = (double *)take((size_t)n_feat * 8);
  double *hi = (double *)take((size_t)n_feat * 8);
  unsigned *list = (unsigned *)take((size_t)n_feat * 4);
  double *tgt = (double *)take((size_t)64 * R);          // [R][8]
  unsigned *hist = (unsigned *)take(65536 * 4);
  u64 *keys = (u64 *)take((size_t)cap * 16);
  unsigned *idx = (unsigned *)take((size_t)cap * 8);
  unsigned *rank = (unsigned *)take((size_t)rcap * 4);
  unsigned *bidx = (unsigned *)take((size_t)rcap * 4);
  unsigned *order = (unsigned *)take((size_t)rcap * 4);
  unsigned *bcount = (unsigned *)take((size_t)SIS_NB * 4 * 2);   // counts, fill cursors
  unsigned *bfill = bcount + SIS_NB;
  unsigned *bstart = (unsigned *)take((size_t)SIS_NB * 4);
  float *yc = (float *)take((size_t)n * 4 * R);          // [R][n]
  double *yd = (double *)take((size_t)n * 8 * R);        // [R][n]
  const unsigned g = (unsigned)std::min<long long>((n_feat + 255) / 256, 152 * 16);
  const unsigned gw = (unsigned)std::min<long long>((n_feat + 7) / 8, 152 * 32);
  cudaError_t e = cudaMemsetAsync(small, 0, 64, st);
  if (e != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(krange, 0, 16, st)) != cudaSuccess) return e;
  int dev = 0, n_sm = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
    return e;
  if ((e = cudaFuncSetAttribute(sis_hist0_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                32768 * 4)) != cudaSuccess)
    return e;
  const long long h0_per =
      std::min<long long>(H0_MAX_PER_BLOCK, std::max<long long>(1024, (n_feat + n_sm - 1) / n_sm));
  // the m-th smallest key of r: two 16-bit levels
  auto cut_of = [&](const double *v, unsigned *c2, unsigned long long *below) -> cudaError_t {
    cudaError_t e2 = cudaMemsetAsync(hist, 0, 65536 * 4, st);
    if (e2 != cudaSuccess) return e2;
    sis_hist0_kernel<<<(unsigned)((n_feat + h0_per - 1) / h0_per), H0_THREADS, 32768 * 4, st>>>(
        v, n_feat, h0_per, hist);
    sis_cut_kernel<<<1, 1024, 0, st>>>(hist, m, below, c2);
    e2 = cudaMemsetAsync(hist, 0, 65536 * 4, st);
    if (e2 != cudaSuccess) return e2;
    sis_hist_kernel<<<g, 256, 0, st>>>(v, n_feat, 1, c2, hist);
    sis_cut_kernel<<<1, 1024, 0, st>>>(hist, m, below, c2 + 1);
    return cudaSuccess;
  };
  const unsigned gx = (unsigned)std::min<long long>((n_ex + 255) / 256, 1024);
  sis_target_kernel<<<R, 1024, 0, st>>>(y, n, tgt, yd, err);
  if (gen && prescreen && gen->cf && gen->csafe && !gen->valid) {
    // generated candidates, FP32 pre-screen, FP64 re-score of the survivors
    sis_target32_kernel<<<1, 1024, 0, st>>>(y, n, tgt, yc);
    const unsigned gc = (unsigned)std::min<long long>((gen->n_child + 7) / 8, 152 * 32);
    gen_child32_kernel<<<gc, 256, 0, st>>>(X, n, gen->n_child, gen->cf, gen->csafe);
    if (scan0 && (e = cudaEventRecord(scan0, st)) != cudaSuccess) return e;
    gen_prescreen_kernel<<<gw, 256, 0, st>>>(gen->cf, gen->csafe, n, gen->n_child, gen->ops,
                                             gen->c1, gen->c2, n_feat, yc, tgt, gen->lb, gen->ub,
                                             r, hi);
    if (scan1 && (e = cudaEventRecord(scan1, st)) != cudaSuccess) return e;
    if ((e = cut_of(r, pcuts, pcnt)) != cudaSuccess) return e;
    sis_candidates_kernel<<<g, 256, 0, st>>>(hi, n_feat, pcuts, pcuts + 1, r, list, pcnt + 1);
    gen_rescore_kernel<<<gw, 256, 0, st>>>(X, n, gen->n_child, gen->ops, gen->c1, gen->c2, list,
                                           pcnt + 1, yd, tgt, gen->lb, gen->ub, r, err);
  } else if (gen) {                    // generated candidates, FP64 (R = 1)
    if (scan0 && (e = cudaEventRecord(scan0, st)) != cudaSuccess) return e;
    gen_score_kernel<<<gw, 256, 0, st>>>(X, n, gen->n_child, gen->ops, gen->c1, gen->c2, n_feat,
                                         yd, tgt, gen->lb, gen->ub, r, gen->valid, err);
    if (scan1 && (e = cudaEventRecord(scan1, st)) != cudaSuccess) return e;
  } else if (prescreen) {
    sis_target32_kernel<<<R, 1024, 0, st>>>(y, n, tgt, yc);
    if (scan0 && (e = cudaEventRecord(scan0, st)) != cudaSuccess) return e;
    // one wave of resident blocks: every warp takes groups of 32 features
    int per_sm = 0;
    if (((uintptr_t)X & 15) == 0) {
      const bool yreg = n <= 2 * PB_SEG;
      const void *fn = yreg ? (const void *)sis_prescreen_bulk_kernel<true>
                            : (const void *)sis_prescreen_bulk_kernel<false>;
      if ((e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)PB_SMEM)) != cudaSuccess)
        return e;
      const long long groups = (n_feat + 31) / 32;
      const unsigned grid = (unsigned)std::min<long long>((groups + PB_WARPS - 1) / PB_WARPS, n_sm);
      if (R > 1 && n <= PM_NMAX && pm_smem(R, n) <= 227 * 1024) {   // one pass for all targets
        const size_t sm = pm_smem(R, n);
        if ((e = cudaFuncSetAttribute(sis_prescreen_multi_kernel,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm)) !=
            cudaSuccess)
          return e;
        const unsigned gm =
            (unsigned)std::min<long long>((groups + PM_WARPS - 1) / PM_WARPS, n_sm);
        sis_prescreen_multi_kernel<<<gm, PM_WARPS * 32, sm, st>>>(X, n, n_feat, yc, tgt, R, r, hi,
                                                                  err);
      } else
      for (int t = 0; t < R; ++t) {      // one pass over X per target
        if (yreg)
          sis_prescreen_bulk_kernel<true><<<grid, PB_WARPS * 32, PB_SMEM, st>>>(
              X, n, n_feat, yc + (size_t)t * n, tgt + 8 * t, t > 0, r, hi, err);
        else
          sis_prescreen_bulk_kernel<false><<<grid, PB_WARPS * 32, PB_SMEM, st>>>(
              X, n, n_feat, yc + (size_t)t * n, tgt + 8 * t, t > 0, r, hi, err);
      }
    } else {
      if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sis_prescreen_kernel, 256,
                                                             0)) != cudaSuccess)
        return e;
      const long long waves = (long long)n_sm * std::max(per_sm, 1);
      for (int t = 0; t < R; ++t)
        sis_prescreen_kernel<<<(unsigned)std::min<long long>((n_feat + 255) / 256, waves), 256, 0,
                               st>>>(X, n, n_feat, yc + (size_t)t * n, tgt + 8 * t, t > 0, r, hi);
    }
    if (scan1 && (e = cudaEventRecord(scan1, st)) != cudaSuccess) return e;
    if (n_ex) sis_exclude_kernel<<<gx, 256, 0, st>>>(ex, n_ex, r, hi);
    if ((e = cut_of(r, pcuts, pcnt)) != cudaSuccess) return e;
    sis_candidates_kernel<<<g, 256, 0, st>>>(hi, n_feat, pcuts, pcuts + 1, r, list, pcnt + 1);
    sis_rescore_kernel<<<gw, 256, 0, st>>>(X, n, list, pcnt + 1, yd, tgt, R, r, err);
  } else {
    if (scan0 && (e = cudaEventRecord(scan0, st)) != cudaSuccess) return e;
    sis_score_kernel<<<gw, 256, 0, st>>>(X, n, n_feat, yd, tgt, R, r, err);
    if (scan1 && (e = cudaEventRecord(scan1, st)) != cudaSuccess) return e;
    if (n_ex) sis_exclude_kernel<<<gx, 256, 0, st>>>(ex, n_ex, r, nullptr);
  }
  if ((e = cut_of(r, cuts, cnt)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(bcount, 0, (size_t)SIS_NB * 8, st)) != cudaSuccess) return e;
  sis_compact_kernel<<<g, 256, 0, st>>>(r, n_feat, cuts, cuts + 1, keys, idx, cnt + 1, cap,
                                        krange);
  const unsigned gr = (unsigned)((rcap + 255) / 256);
  sis_bucket_kernel<<<gr, 256, 0, st>>>(keys, cnt + 1, cap, krange, bidx, bcount);
  sis_bucket_scan_kernel<<<1, 1024, 0, st>>>(bcount, bstart);
  sis_bucket_place_kernel<<<gr, 256, 0, st>>>(cnt + 1, cap, bidx, bstart, bfill, order);
  sis_rank_kernel<<<gr, 256, 0, st>>>(keys, idx, cnt + 1, cap, bidx, bstart, bcount, order, rank);
  sis_scatter_kernel<<<(unsigned)std::min<long long>((std::max<long long>(rcap, m) + 255) / 256,
                                                     152 * 8),
                       256, 0, st>>>(idx, rank, cnt + 1, cap, m, r, out_idx, out_r);
  sis_sort_kernel<<<1, 1024, 0, st>>>(keys, idx, cnt + 1, cap, m, r, out_idx, out_r, err);
  return cudaGetLastError();
}

}  // namespace l0
