// Calibration: the device's FP32 fused multiply-add throughput, measured.
//
// The update kernel is bound by FP32 arithmetic, so its roofline denominator is
// the rate at which this device retires FFMA instructions at the clocks it runs
// at.  The kernel below keeps every FP32 lane busy: each thread advances eight
// independent FFMA chains (enough to cover the pipeline latency), 16 warps per
// scheduler, and the host times repeated launches with CUDA events.
#include <cuda_runtime.h>

#include <algorithm>

#include "internal.h"

namespace fpm {

constexpr int kCalibChains = 8;

static __global__ void __launch_bounds__(256) ffma_chains_kernel(float *out, int iters, float a, float b) {
  float x[kCalibChains];
#pragma unroll
  for (int k = 0; k < kCalibChains; ++k) x[k] = (float)(threadIdx.x + k) * 1e-7f;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kCalibChains; ++k) x[k] = __fmaf_rn(x[k], a, b);
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < kCalibChains; ++k) s += x[k];
  if (s == 1234.5f) out[threadIdx.x] = s;   // keeps the chains alive; never true for a = b = 0.5
}

}  // namespace fpm

using fpm::fail;

extern "C" int fpm_fp32_peak(double *tflops, void *stream) {
  fpm::clear_error();
  if (!tflops) return fail(FPM_EINVAL, "fpm_fp32_peak: null argument");
  *tflops = 0.0;
  int dev = 0, sms = 0;
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  float *out = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (e == cudaSuccess) e = cudaMalloc((void **)&out, 256 * sizeof(float));
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  const int threads = 256, blocks = sms * 8, iters = 1 << 15;
  double best = 0.0;
  for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {      // first launch warms up
    e = cudaEventRecord(e0, st);
    if (e == cudaSuccess) fpm::ffma_chains_kernel<<<blocks, threads, 0, st>>>(out, iters, 0.5f, 0.5f);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess && rep > 0 && ms > 0.f) {
      const double flops = 2.0 * fpm::kCalibChains * (double)iters * threads * blocks;
      best = std::max(best, flops / (ms * 1e-3) / 1e12);
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (out) cudaFree(out);
  if (e != cudaSuccess) return fail(FPM_ECUDA, "fpm_fp32_peak: %s", cudaGetErrorString(e));
  *tflops = best;
  return FPM_OK;
}
