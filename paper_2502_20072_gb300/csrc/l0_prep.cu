// l0_prep.cu -- per-task centring/scaling (FP64) and the FP64 Gram.
//
// Centring every column and the target by its task mean removes the
// intercept of the least-squares fit exactly; dividing by the centred norm
// turns the Gram of the columns into a correlation matrix (unit diagonal),
// which is what the tuple kernel factorises.  With the scaled target placed
// first, the augmented Gram is
//     G[0][0] = 1,  G[0][j+1] = r_j (Pearson r of feature j, Eq. 1),
//     G[i+1][j+1] = corr(f_i, f_j),
// so the l0 score of a tuple (paper Sec. 2.4) is a Schur complement of G.
#include "l0_kernels.cuh"

namespace l0 {

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// One warp per (column c in [0, m], task t); c == 0 is the target.
__global__ void __launch_bounds__(256)
centre_kernel(const double *__restrict__ X, const double *__restrict__ y,
              long long n_total, int m, const long long *__restrict__ offsets,
              double *__restrict__ mu, double *__restrict__ inv_s,
              double *__restrict__ W, int *err) {
  const int lane = threadIdx.x & 31;
  const int c = blockIdx.x * 8 + (threadIdx.x >> 5);
  const int t = blockIdx.y;
  if (c > m) return;
  const long long lo = offsets[t], hi = offsets[t + 1];
  const long long n = hi - lo;
  const double *src = (c == 0) ? (y + lo) : (X + (long long)(c - 1) * n_total + lo);
  double s = 0.0;
  bool finite = true;
  for (long long i = lane; i < n; i += 32) {
    double v = src[i];
    finite &= isfinite(v);
    s += v;
  }
  if (__any_sync(0xffffffffu, !finite)) {
    if (lane == 0) set_err(err, 5);
  }
  s = warp_sum(s);
  const double mean = s / (double)n;
  double ss = 0.0;
  for (long long i = lane; i < n; i += 32) {
    double v = src[i] - mean;
    ss += v * v;
  }
  ss = warp_sum(ss);
  const double nrm = sqrt(ss);
  const double is = (nrm > 0.0) ? 1.0 / nrm : 0.0;
  if (lane == 0) {
    mu[(long long)t * (m + 1) + c] = mean;
    inv_s[(long long)t * (m + 1) + c] = is;
  }
  if (W) {
    double *dst = W + (long long)c * n_total + lo;
    for (long long i = lane; i < n; i += 32) dst[i] = (src[i] - mean) * is;
  }
}

// ---------------------------------------------------- duplicate classes --
// Column hash: XOR over rows of a mix of the row index and the value rounded
// to 36 mantissa bits (values that differ in the last bits hash alike).
__device__ __forceinline__ u64 mix64(u64 z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__global__ void __launch_bounds__(256)
column_hash_kernel(const double *__restrict__ X, long long n_total, int m, u64 *hash) {
  const int lane = threadIdx.x & 31;
  const int c = blockIdx.x * 8 + (threadIdx.x >> 5);
  if (c >= m) return;
  const double *src = X + (long long)c * n_total;
  u64 h = 0;
  for (long long i0 = lane; i0 < n_total; i0 += 256) {   // eight loads in flight
    long long raw[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const long long i = i0 + 32 * u;
      raw[u] = i < n_total ? __double_as_longlong(__ldg(src + i)) : 0ll;
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const long long i = i0 + 32 * u;
      if (i < n_total) {
        const u64 b = ((u64)raw[u] + 0x8000ull) & ~0xFFFFull;
        h ^= mix64(b ^ ((u64)i * 0x9E3779B97F4A7C15ull));
      }
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) h ^= __shfl_xor_sync(0xffffffffu, h, o);
  if (lane == 0) hash[c] = h;
}

// one warp per column j: lanes scan the hashes of the columns before it, 256
// at a time (eight loads in flight per lane); each hash match is verified by
// the whole warp (coalesced rows)
__global__ void __launch_bounds__(256)
column_class_kernel(const double *__restrict__ X, long long n_total, int m, const u64 *hash,
                    int *cls) {
  const int lane = threadIdx.x & 31;
  const int j = blockIdx.x * 8 + (threadIdx.x >> 5);
  if (j >= m) return;
  const u64 hj = hash[j];
  const double *xj = X + (long long)j * n_total;
  int c = j;
  for (int i00 = 0; i00 < j && c == j; i00 += 256) {
    unsigned eq = 0u;   // bit u: the hash of column i00 + 32 u + lane matches
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int i = i00 + 32 * u + lane;
      if (i < j && __ldg(hash + i) == hj) eq |= 1u << u;
    }
    for (int u = 0; u < 8 && c == j; ++u) {
      const int i0 = i00 + 32 * u;
      unsigned hit = __ballot_sync(0xffffffffu, (eq >> u) & 1u);
      while (hit && c == j) {
        const int q = i0 + __ffs(hit) - 1;
        hit &= hit - 1;
        const double *xi = X + (long long)q * n_total;
        bool same = true;
        for (long long r = lane; r < n_total; r += 32) {
          const double a = xi[r], b = xj[r];
          same = same && fabs(a - b) <= 1e-12 * fmax(fabs(a), fabs(b));
        }
        if (__all_sync(0xffffffffu, same)) c = q;
      }
    }
  }
  if (lane == 0) cls[j] = c;
}

cudaError_t launch_column_classes(const double *X, long long n_total, int m, u64 *hash, int *cls,
                                  cudaStream_t st) {
  column_hash_kernel<<<(m + 7) / 8, 256, 0, st>>>(X, n_total, m, hash);
  column_class_kernel<<<(m + 7) / 8, 256, 0, st>>>(X, n_total, m, hash, cls);
  return cudaGetLastError();
}

cudaError_t launch_centre(const double *X, const double *y, long long n_total,
                          int m, const long long *offsets_dev, int T,
                          double *mu, double *inv_s, double *W64, int *err,
                          cudaStream_t st) {
  dim3 grid((m + 1 + 7) / 8, T);
  centre_kernel<<<grid, 256, 0, st>>>(X, y, n_total, m, offsets_dev, mu, inv_s,
                                      W64, err);
  return cudaGetLastError();
}

// FP64 Gram of the scaled columns of one task: G = W_t^T W_t over the task's
// rows, upper-triangular 64x64 tiles only (FFMA64, 4x4 outputs per thread).
// A diagonal tile stores its full 64x64 block (the entries below the diagonal
// are the mirrored values) unless upper_only is set, in which case only
// entries (r, c) with r <= c are stored.
__global__ void __launch_bounds__(256)
gram64_kernel(const double *__restrict__ W, long long n_total, int mp1,
              long long lo, long long hi, double *__restrict__ G, long long ld,
              int nb, const u64 *gate, int gate_d, int upper_only, const int *skip) {
  if (skip && *skip) return;   // computed by an earlier pass of this fit
  if (gate && !defer_wants_gram(gate[1], mp1 - 1, gate_d)) return;
  // decode the upper-triangular tile index (bi <= bj)
  int idx = blockIdx.x;
  int bi = 0;
  while (idx >= nb - bi) { idx -= nb - bi; ++bi; }
  const int bj = bi + idx;
  __shared__ double As[16][65];
  __shared__ double Bs[16][65];
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  double acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
  const int lr = tid >> 2;            // row within the tile for loads
  const int lk = (tid & 3) * 4;       // first k of this thread's 4 loads
  const int ra = bi * 64 + lr, rb = bj * 64 + lr;
  for (long long k0 = lo; k0 < hi; k0 += 16) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      long long kk = k0 + lk + q;
      double a = 0.0, b = 0.0;
      if (kk < hi) {
        if (ra < mp1) a = W[(long long)ra * n_total + kk];
        if (rb < mp1) b = W[(long long)rb * n_total + kk];
      }
      As[lk + q][lr] = a;
      Bs[lk + q][lr] = b;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      double a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int r = bi * 64 + ty + 16 * i;
    if (r >= mp1) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int c = bj * 64 + tx + 16 * j;
      if (c < mp1 && (!upper_only || c >= r)) G[(long long)r * ld + c] = acc[i][j];
    }
  }
}

cudaError_t launch_gram64(const double *W64, long long n_total, int m,
                          const long long *offsets_host, int T, double *G,
                          long long ld, long long g_stride, cudaStream_t st,
                          const u64 *gate, int gate_d, int upper_only, const int *skip) {
  const int mp1 = m + 1;
  const int nb = (mp1 + 63) / 64;
  const int ntiles = nb * (nb + 1) / 2;
  for (int t = 0; t < T; ++t) {
    gram64_kernel<<<ntiles, 256, 0, st>>>(W64, n_total, mp1, offsets_host[t],
                                          offsets_host[t + 1],
                                          G + (long long)t * g_stride, ld, nb, gate, gate_d,
                                          upper_only, skip);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

__global__ void mark_gram64_kernel(const u64 *gate, int m, int gate_d, int *have) {
  if (defer_wants_gram(gate[1], m, gate_d)) *have = 1;
}

cudaError_t launch_mark_gram64(const u64 *gate, int m, int gate_d, int *have, cudaStream_t st) {
  mark_gram64_kernel<<<1, 1, 0, st>>>(gate, m, gate_d, have);
  return cudaGetLastError();
}

}  // namespace l0
