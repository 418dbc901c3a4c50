// l0_loop.cu -- device pieces of the dimension loop (paper Sec. 2, Fig. 1b):
// the residuals of the best models of one dimension, which the next SIS
// screens against, and the gather of the selected subspace's rows.
//
// residual_kernel: one block per model (d global feature indices).  The
// least-squares fit with intercept (Sec. 2.4) leaves the residual
// (I - P) (y - mean y), P the projector onto the span of the model's centred
// columns.  The block orthonormalises the centred columns by Gram-Schmidt
// with a second orthogonalisation pass (each pass removes the components
// along the earlier vectors), drops a column whose norm falls below 1e-12 of
// its centred norm (dependent: the minimum-norm least-squares fit leaves the
// same residual), then removes the components of the centred y, again in
// two passes.  All in FP64.
#include "../../include/sisso_l0.h"
#include "l0_kernels.cuh"
#include "l0_screen.cuh"

namespace l0 {

namespace {

constexpr int RS_THREADS = 256;

__device__ double rs_block_sum(double v, double *red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double s = 0.0;
  for (int i = 0; i < RS_THREADS / 32; ++i) s += red[i];
  return s;
}

__global__ void __launch_bounds__(RS_THREADS)
residual_kernel(const double *__restrict__ X, const double *__restrict__ y, long long n,
                const int *__restrict__ tuples, int d, double *__restrict__ Q,
                double *__restrict__ out) {
  __shared__ double red[RS_THREADS / 32];
  const int model = blockIdx.x;
  const int *tup = tuples + (long long)model * d;
  double *q0 = Q + (long long)model * d * n;
  double *w = out + (long long)model * n;
  const double nn = (double)n;
  bool keep[8];
  // centred y
  double s = 0.0;
  for (long long i = threadIdx.x; i < n; i += RS_THREADS) s += y[i];
  const double my = rs_block_sum(s, red) / nn;
  for (long long i = threadIdx.x; i < n; i += RS_THREADS) w[i] = y[i] - my;
  // orthonormal basis of the centred columns
  for (int a = 0; a < d; ++a) {
    const double *x = X + (long long)tup[a] * n;
    double *qa = q0 + (long long)a * n;
    s = 0.0;
    for (long long i = threadIdx.x; i < n; i += RS_THREADS) s += x[i];
    const double mx = rs_block_sum(s, red) / nn;
    double ss = 0.0;
    for (long long i = threadIdx.x; i < n; i += RS_THREADS) {
      const double v = x[i] - mx;
      qa[i] = v;
      ss = fma(v, v, ss);
    }
    const double nu = sqrt(rs_block_sum(ss, red));
    for (int pass = 0; pass < 2; ++pass)
      for (int b = 0; b < a; ++b) {
        if (!keep[b]) continue;
        const double *qb = q0 + (long long)b * n;
        double c = 0.0;
        for (long long i = threadIdx.x; i < n; i += RS_THREADS) c = fma(qb[i], qa[i], c);
        c = rs_block_sum(c, red);
        for (long long i = threadIdx.x; i < n; i += RS_THREADS) qa[i] = fma(-c, qb[i], qa[i]);
      }
    ss = 0.0;
    for (long long i = threadIdx.x; i < n; i += RS_THREADS) ss = fma(qa[i], qa[i], ss);
    const double nq = sqrt(rs_block_sum(ss, red));
    keep[a] = nq > 1e-12 * nu && nq > 0.0;
    const double inv = keep[a] ? 1.0 / nq : 0.0;
    for (long long i = threadIdx.x; i < n; i += RS_THREADS) qa[i] *= inv;
  }
  // residual: remove the components of the centred y along the basis
  for (int pass = 0; pass < 2; ++pass)
    for (int b = 0; b < d; ++b) {
      if (!keep[b]) continue;
      const double *qb = q0 + (long long)b * n;
      double c = 0.0;
      for (long long i = threadIdx.x; i < n; i += RS_THREADS) c = fma(qb[i], w[i], c);
      c = rs_block_sum(c, red);
      for (long long i = threadIdx.x; i < n; i += RS_THREADS) w[i] = fma(-c, qb[i], w[i]);
    }
}

// out[r][.] = X[rows[r]][.]
__global__ void __launch_bounds__(256)
gather_rows_kernel(const double *__restrict__ X, long long n, const int *__restrict__ rows,
                   int n_rows, double *__restrict__ out) {
  const long long total = (long long)n_rows * n;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long r = e / n, i = e - r * n;
    out[e] = X[(long long)rows[r] * n + i];
  }
}

}  // namespace

// tuples: [R][d] global feature indices (device), d <= 8; Q: scratch [R][d][n];
// out: [R][n] residuals (device)
cudaError_t launch_residuals(const double *X, const double *y, long long n, const int *tuples,
                             int d, int R, double *Q, double *out, cudaStream_t st) {
  if (d < 1 || d > 8 || R < 1) return cudaErrorInvalidValue;
  residual_kernel<<<R, RS_THREADS, 0, st>>>(X, y, n, tuples, d, Q, out);
  return cudaGetLastError();
}

cudaError_t launch_gather_rows(const double *X, long long n, const int *rows, int n_rows,
                               double *out, cudaStream_t st) {
  const long long total = (long long)n_rows * n;
  const unsigned g = (unsigned)std::min<long long>((total + 255) / 256, 152 * 16);
  gather_rows_kernel<<<g, 256, 0, st>>>(X, n, rows, n_rows, out);
  return cudaGetLastError();
}

}  // namespace l0
