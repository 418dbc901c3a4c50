// l0_peaks.cu -- microbenchmarks of the units the l0 kernels are bound by.
//
// The tuple search is bound by the FP32 pipe (mixed precision) or the FP64
// pipe (plain FP64 path), its records by the multi-function unit and shared
// memory, and its Gram reads by L2.  These kernels measure each rate on the
// device at hand so that roofline fractions divide by measured peaks:
//   ffma32 / dfma: independent FMA chains (2 flop each) on every lane;
//   rsqrt: MUFU reciprocal square roots;
//   smem: 16-byte shared-memory loads, conflict-free;
//   l2: 16-byte global loads over a buffer far smaller than L2, reread.
// Each is timed with CUDA events after a warm-up launch.
#include "../../include/sisso_l0.h"
#include "l0_kernels.cuh"

namespace l0 {

namespace {

constexpr int PK_THREADS = 256;
constexpr int PK_ITERS = 4096;

template <typename T>
__global__ void __launch_bounds__(PK_THREADS)
fma_peak_kernel(T seed, T *sink) {
  T a[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) a[i] = seed + (T)(threadIdx.x + i);
  const T b = (T)0.999999, c = (T)1e-7;
#pragma unroll 4
  for (int it = 0; it < PK_ITERS; ++it) {
#pragma unroll
    for (int i = 0; i < 8; ++i) a[i] = fma(a[i], b, c);
  }
  T s = 0;
#pragma unroll
  for (int i = 0; i < 8; ++i) s += a[i];
  if (s == (T)-12345.0) sink[blockIdx.x] = s;   // never true; keeps the chains
}

__global__ void __launch_bounds__(PK_THREADS)
rsqrt_peak_kernel(float seed, float *sink) {
  float a[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) a[i] = seed + (float)(threadIdx.x + i + 1);
#pragma unroll 4
  for (int it = 0; it < PK_ITERS; ++it) {
#pragma unroll
    for (int i = 0; i < 8; ++i) a[i] = rsqrtf(a[i]) + 1.0f;
  }
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < 8; ++i) s += a[i];
  if (s == -12345.0f) sink[blockIdx.x] = s;
}

__global__ void __launch_bounds__(PK_THREADS)
smem_peak_kernel(float *sink) {
  __shared__ float4 buf[PK_THREADS * 4];
  for (int i = threadIdx.x; i < PK_THREADS * 4; i += PK_THREADS)
    buf[i] = make_float4((float)i, 1.f, 2.f, 3.f);
  __syncthreads();
  float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll 8
  for (int it = 0; it < PK_ITERS; ++it) {
    const float4 v = buf[(threadIdx.x + it * 32) & (PK_THREADS * 4 - 1)];
    acc.x += v.x; acc.y += v.y; acc.z += v.z; acc.w += v.w;
  }
  if (acc.x + acc.y + acc.z + acc.w == -12345.0f) sink[blockIdx.x] = acc.x;
}

__global__ void __launch_bounds__(PK_THREADS)
l2_peak_kernel(const float4 *__restrict__ buf, long long n4, int reps, float *sink) {
  float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (int r = 0; r < reps; ++r)
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += stride) {
      const float4 v = __ldcg(buf + i);
      acc.x += v.x; acc.y += v.y; acc.z += v.z; acc.w += v.w;
    }
  if (acc.x + acc.y + acc.z + acc.w == -12345.0f) sink[blockIdx.x] = acc.x;
}

template <typename F>
cudaError_t time_ms(F launch, float *ms) {
  cudaEvent_t a, b;
  cudaError_t e = cudaEventCreate(&a);
  if (e != cudaSuccess) return e;
  e = cudaEventCreate(&b);
  if (e != cudaSuccess) return e;
  launch();                       // warm-up
  e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaEventRecord(a);
  launch();
  if (e == cudaSuccess) e = cudaEventRecord(b);
  if (e == cudaSuccess) e = cudaEventSynchronize(b);
  if (e == cudaSuccess) e = cudaEventElapsedTime(ms, a, b);
  if (e == cudaSuccess) e = cudaGetLastError();
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return e;
}

}  // namespace

}  // namespace l0

extern "C" int sisso_l0_measure_peaks(int32_t device, double *out) {
  using namespace l0;
  if (!out) return SISSO_L0_EINVAL;
  if (cudaSetDevice(device) != cudaSuccess) return SISSO_L0_ECUDA;
  int n_sm = 0;
  if (cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, device) != cudaSuccess)
    return SISSO_L0_ECUDA;
  float *sink = nullptr;
  float4 *buf = nullptr;
  const long long l2_bytes = 32ll << 20;   // 32 MB, resident in L2
  if (cudaMalloc(&sink, 1 << 20) != cudaSuccess) return SISSO_L0_ENOMEM;
  if (cudaMalloc(&buf, l2_bytes) != cudaSuccess) {
    cudaFree(sink);
    return SISSO_L0_ENOMEM;
  }
  cudaMemset(buf, 0, l2_bytes);
  const int grid = n_sm * 8;
  const double thr = (double)grid * PK_THREADS;
  float ms = 0.f;
  int rc = SISSO_L0_OK;
  // FP32 FMA
  if (time_ms([&] { fma_peak_kernel<float><<<grid, PK_THREADS>>>(1.f, sink); }, &ms) != cudaSuccess)
    rc = SISSO_L0_ECUDA;
  out[0] = rc ? 0.0 : thr * PK_ITERS * 8 * 2 / (ms * 1e-3) / 1e12;
  // FP64 FMA (a smaller grid: the FP64 pipe is narrow)
  const int grid64 = n_sm * 2;
  if (!rc && time_ms([&] { fma_peak_kernel<double><<<grid64, PK_THREADS>>>(1.0, (double *)sink); },
                     &ms) != cudaSuccess)
    rc = SISSO_L0_ECUDA;
  out[1] = rc ? 0.0 : (double)grid64 * PK_THREADS * PK_ITERS * 8 * 2 / (ms * 1e-3) / 1e12;
  // MUFU rsqrt
  if (!rc && time_ms([&] { rsqrt_peak_kernel<<<grid, PK_THREADS>>>(1.f, sink); }, &ms) != cudaSuccess)
    rc = SISSO_L0_ECUDA;
  out[2] = rc ? 0.0 : thr * PK_ITERS * 8 / (ms * 1e-3) / 1e9;
  // shared memory
  if (!rc && time_ms([&] { smem_peak_kernel<<<grid, PK_THREADS>>>(sink); }, &ms) != cudaSuccess)
    rc = SISSO_L0_ECUDA;
  out[3] = rc ? 0.0 : thr * PK_ITERS * 16 / (ms * 1e-3) / 1e9;
  // L2
  const int reps = 32;
  if (!rc && time_ms([&] { l2_peak_kernel<<<grid, PK_THREADS>>>(buf, l2_bytes / 16, reps, sink); },
                     &ms) != cudaSuccess)
    rc = SISSO_L0_ECUDA;
  out[4] = rc ? 0.0 : (double)l2_bytes * reps / (ms * 1e-3) / 1e9;
  cudaFree(buf);
  cudaFree(sink);
  return rc;
}
