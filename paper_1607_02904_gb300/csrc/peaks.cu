// Arithmetic-pipe peaks of the current device, measured by loop kernels: the
// denominators of the force kernels' rooflines (FP32 FMA for the mixed path,
// FP64 FMA for the FP64 path, the special-function unit for the
// transcendentals). The paper has no counterpart; it reports run times only.
//
// Each kernel runs independent dependency chains per thread (enough of them,
// over enough warps, to hide the pipe latency) for a fixed number of
// iterations; the time comes from CUDA events around the launch. The chains'
// results are stored so that the compiler keeps the work.
#include <cstdio>

#include "internal.cuh"

namespace tgb {
namespace {

constexpr int PK_BLOCK = 256;
constexpr int PK_CHAINS = 8;    // independent chains per thread
constexpr int PK_UNROLL = 16;   // chain steps per loop iteration

__global__ void __launch_bounds__(PK_BLOCK) k_peak_ffma(float b, float c, int iters, float* out) {
  float a[PK_CHAINS];
#pragma unroll
  for (int q = 0; q < PK_CHAINS; ++q) a[q] = (float)(threadIdx.x + q) * 1e-3f;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < PK_UNROLL; ++u)
#pragma unroll
      for (int q = 0; q < PK_CHAINS; ++q) a[q] = fmaf(a[q], b, c);
  }
  float s = 0.0f;
#pragma unroll
  for (int q = 0; q < PK_CHAINS; ++q) s += a[q];
  out[blockIdx.x * PK_BLOCK + threadIdx.x] = s;
}

__global__ void __launch_bounds__(PK_BLOCK) k_peak_dfma(double b, double c, int iters,
                                                       double* out) {
  double a[PK_CHAINS];
#pragma unroll
  for (int q = 0; q < PK_CHAINS; ++q) a[q] = (double)(threadIdx.x + q) * 1e-3;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < PK_UNROLL; ++u)
#pragma unroll
      for (int q = 0; q < PK_CHAINS; ++q) a[q] = fma(a[q], b, c);
  }
  double s = 0.0;
#pragma unroll
  for (int q = 0; q < PK_CHAINS; ++q) s += a[q];
  out[blockIdx.x * PK_BLOCK + threadIdx.x] = s;
}

// OP 0: rsqrt.approx (y -> 1/sqrt(y), converges to 1); OP 1: ex2.approx of
// -y (stays in (0, 1]); OP 2: lg2.approx of y + 2 (the add is an FP32 op on
// another pipe, issued beside the MUFU op).
template <int OP>
__global__ void __launch_bounds__(PK_BLOCK) k_peak_mufu(int iters, float* out) {
  float a[PK_CHAINS];
#pragma unroll
  for (int q = 0; q < PK_CHAINS; ++q) a[q] = 1.5f + (float)(threadIdx.x + q) * 1e-3f;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < PK_UNROLL; ++u)
#pragma unroll
      for (int q = 0; q < PK_CHAINS; ++q) {
        if (OP == 0)
          asm volatile("rsqrt.approx.ftz.f32 %0, %0;" : "+f"(a[q]));
        else if (OP == 1)
          asm volatile("{.reg .f32 t; neg.f32 t, %0; ex2.approx.ftz.f32 %0, t;}" : "+f"(a[q]));
        else
          asm volatile("{.reg .f32 t; add.f32 t, %0, 0f40000000; lg2.approx.ftz.f32 %0, t;}"
                       : "+f"(a[q]));
      }
  }
  float s = 0.0f;
#pragma unroll
  for (int q = 0; q < PK_CHAINS; ++q) s += a[q];
  out[blockIdx.x * PK_BLOCK + threadIdx.x] = s;
}

// Median of `reps` event-timed launches of fn (after one untimed launch), ms.
template <class F>
float time_launch(F fn, cudaStream_t s, cudaEvent_t e0, cudaEvent_t e1, int reps) {
  fn();
  float best[9];
  for (int r = 0; r < reps; ++r) {
    cudaEventRecord(e0, s);
    fn();
    cudaEventRecord(e1, s);
    cudaEventSynchronize(e1);
    cudaEventElapsedTime(&best[r], e0, e1);
  }
  for (int i = 1; i < reps; ++i)
    for (int j = i; j > 0 && best[j] < best[j - 1]; --j) {
      float t = best[j];
      best[j] = best[j - 1];
      best[j - 1] = t;
    }
  return best[reps / 2];
}

}  // namespace
}  // namespace tgb

extern "C" int tersoff_pipe_peaks(double* out, void* stream) {
  using namespace tgb;
  if (!out) return TERSOFF_E_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  int dev = 0, n_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      n_sm <= 0) {
    cudaGetLastError();
    return TERSOFF_E_CUDA;
  }
  // four blocks of 256 per SM: 32 warps, 8 chains each
  const int grid = 4 * n_sm;
  const size_t threads = (size_t)grid * PK_BLOCK;
  void* buf = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaMalloc(&buf, threads * sizeof(double)) != cudaSuccess ||
      cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    cudaGetLastError();
    if (buf) cudaFree(buf);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    return TERSOFF_E_CUDA;
  }
  const int reps = 5;
  // work per launch: threads x chains x unroll x iters operations
  const double per_iter = (double)threads * PK_CHAINS * PK_UNROLL;
  const int it32 = 2048, it64 = 64, itmu = 256;
  float* f = (float*)buf;
  double* d = (double*)buf;
  const float ms32 = time_launch(
      [&] { k_peak_ffma<<<grid, PK_BLOCK, 0, s>>>(0.999999f, 1e-7f, it32, f); }, s, e0, e1, reps);
  const float ms64 = time_launch(
      [&] { k_peak_dfma<<<grid, PK_BLOCK, 0, s>>>(0.999999, 1e-7, it64, d); }, s, e0, e1, reps);
  const float msr = time_launch([&] { k_peak_mufu<0><<<grid, PK_BLOCK, 0, s>>>(itmu, f); }, s, e0,
                                e1, reps);
  const float mse = time_launch([&] { k_peak_mufu<1><<<grid, PK_BLOCK, 0, s>>>(itmu, f); }, s, e0,
                                e1, reps);
  const float msl = time_launch([&] { k_peak_mufu<2><<<grid, PK_BLOCK, 0, s>>>(itmu, f); }, s, e0,
                                e1, reps);
  const cudaError_t err = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(buf);
  if (err != cudaSuccess) return TERSOFF_E_CUDA;
  out[0] = 2.0 * per_iter * it32 / (ms32 * 1e-3) / 1e12;  // FP32 TFLOP/s (FMA = 2)
  out[1] = 2.0 * per_iter * it64 / (ms64 * 1e-3) / 1e12;  // FP64 TFLOP/s
  out[2] = per_iter * itmu / (msr * 1e-3) / 1e12;         // rsqrt, 1e12 ops/s
  out[3] = per_iter * itmu / (mse * 1e-3) / 1e12;         // ex2
  out[4] = per_iter * itmu / (msl * 1e-3) / 1e12;         // lg2
  out[5] = (double)n_sm;
  return TERSOFF_OK;
}
