// l0_noalloc.cu -- a Gram entry point that allocates no memory.
//
// Some callers cannot allocate device memory at the moment they need the
// correlation matrix: a service that reserves its whole device-memory budget
// at start-up and hands it to its own allocator has no room for a
// cudaMalloc on the request path, and a latency-bound loop cannot afford
// the device-wide synchronisation that cudaMalloc/cudaFree imply.  For them
// sisso_l0_gram_noalloc() runs the same centring and FP64 Gram kernels as the
// rest of the library, but keeps its scratch (the centred, scaled columns,
// the column means and inverse norms, the task offsets and an error word) in
// one fixed array compiled into the library instead of allocating it.
//
// Costs and rules of that array:
//   * it holds L0_NOALLOC_SCRATCH_DOUBLES doubles (16 MiB); every GPU on
//     which the library's kernels are loaded keeps it until the process exits;
//   * every call shares it and finds the previous call's contents there, so
//     each call re-initialises what must start from a known value (the
//     offsets and the error word) before using it;
//   * two calls whose work overlaps on the GPU (different streams, or
//     different host threads) race on it: serialise them.
#include <mutex>

#include "../../include/sisso_l0.h"
#include "l0_kernels.cuh"

#define L0_NOALLOC_SCRATCH_DOUBLES (2u * 1024u * 1024u)   // 16 MiB
#define L0_NOALLOC_MAX_DEVICES 64

namespace {

static __device__ __align__(256) double g_noalloc_scratch[L0_NOALLOC_SCRATCH_DOUBLES];

// device address of g_noalloc_scratch per device, looked up once per device
std::mutex g_noalloc_mu;
double *g_noalloc_ptr[L0_NOALLOC_MAX_DEVICES] = {nullptr};

__global__ void noalloc_init_kernel(long long *offsets, long long n_total, int *err) {
  offsets[0] = 0;
  offsets[1] = n_total;
  *err = 0;
}

}  // namespace

extern "C" int sisso_l0_gram_noalloc(const double *X, const double *y, int64_t n_samples,
                                     int64_t n_sis, double *out_gram, int64_t ld_out,
                                     void *stream) {
  if (!X || !y || !out_gram || n_samples < 2 || n_sis < 1 || ld_out < n_sis + 1)
    return SISSO_L0_EINVAL;
  // scratch layout (in doubles): W [(m+1) * n] | mu [m+1] | inv_s [m+1] |
  // offsets (2 x int64) | error word; it fits when (m+1)(n+2) + 3 <= the
  // array's size.  Both factors are bounded before they are multiplied, so
  // no size can wrap the product.
  const uint64_t cap = L0_NOALLOC_SCRATCH_DOUBLES - 3ull;
  if ((uint64_t)n_sis >= cap || (uint64_t)n_samples >= cap) return SISSO_L0_EUNSUPPORTED;
  const int64_t mp1 = n_sis + 1;
  if ((uint64_t)n_samples + 2ull > cap / (uint64_t)mp1) return SISSO_L0_EUNSUPPORTED;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= L0_NOALLOC_MAX_DEVICES)
    return SISSO_L0_ECUDA;
  double *base = nullptr;
  {
    // set-up on the first call per device: the host-side name of the array is
    // only a stand-in, the kernels need its device address
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
      void *p = nullptr;
      if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
        cudaGetLastError();
        return SISSO_L0_ECUDA;
      }
      g_noalloc_ptr[dev] = (double *)p;
    }
    base = g_noalloc_ptr[dev];
  }
  cudaStream_t st = (cudaStream_t)stream;
  double *W = base;
  double *mu = W + (size_t)mp1 * (size_t)n_samples;
  double *inv_s = mu + mp1;
  long long *offs = (long long *)(inv_s + mp1);
  int *err = (int *)(offs + 2);
  noalloc_init_kernel<<<1, 1, 0, st>>>(offs, (long long)n_samples, err);
  if (cudaGetLastError() != cudaSuccess) return SISSO_L0_ECUDA;
  if (l0::launch_centre(X, y, (long long)n_samples, (int)n_sis, offs, 1, mu, inv_s, W, err, st) !=
      cudaSuccess)
    return SISSO_L0_ECUDA;
  const long long off_host[2] = {0, (long long)n_samples};
  if (l0::launch_gram64(W, (long long)n_samples, (int)n_sis, off_host, 1, out_gram,
                        (long long)ld_out, 0, st, nullptr, 0, /*upper_only=*/1) != cudaSuccess)
    return SISSO_L0_ECUDA;
  int herr = 0;
  if (cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return SISSO_L0_ECUDA;
  return herr == 5 ? SISSO_L0_ENONFINITE : (herr ? SISSO_L0_ECUDA : SISSO_L0_OK);
}
