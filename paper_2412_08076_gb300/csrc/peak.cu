// FMA throughput microbenchmark: the arithmetic ceilings of the temporally blocked sweep
// (which is bound by its FP32 pipe, not HBM) and of the FP64 refinement, measured on
// the device rather than taken from unit counts. Every thread runs eight independent
// multiply-add chains a <- a * q + c (q just below 1, so the values settle near
// c / (1 - q) and never overflow or go subnormal); the chains' sum is stored so that
// nothing is dead code.
#include "common.cuh"

namespace richm {

constexpr int kPeakChains = 8;
constexpr int kPeakBlock = 256;
constexpr int kPeakBlocksPerSM = 8;

__global__ void __launch_bounds__(kPeakBlock) fma_f32_kernel(float* out, int iters) {
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  float a[kPeakChains];
#pragma unroll
  for (int j = 0; j < kPeakChains; ++j) a[j] = 1e-3f * (float)(j + (tid & 7));
  const float q = 0.9999999f, c = 1e-7f;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < kPeakChains; ++j) a[j] = __fmaf_rn(a[j], q, c);
  }
  float s = 0.f;
#pragma unroll
  for (int j = 0; j < kPeakChains; ++j) s += a[j];
  out[tid] = s;
}

__global__ void __launch_bounds__(kPeakBlock) fma_f32x2_kernel(float* out, int iters) {
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  float2 a[kPeakChains];
#pragma unroll
  for (int j = 0; j < kPeakChains; ++j) a[j] = make_float2(1e-3f * (float)(j + (tid & 7)), 2e-3f * (float)j);
  const float2 q = make_float2(0.9999999f, 0.9999999f), c = make_float2(1e-7f, 1e-7f);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < kPeakChains; ++j) a[j] = __ffma2_rn(a[j], q, c);
  }
  float s = 0.f;
#pragma unroll
  for (int j = 0; j < kPeakChains; ++j) s += a[j].x + a[j].y;
  out[tid] = s;
}

__global__ void __launch_bounds__(kPeakBlock) fma_f64_kernel(float* out, int iters) {
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  double a[kPeakChains];
#pragma unroll
  for (int j = 0; j < kPeakChains; ++j) a[j] = 1e-3 * (double)(j + (tid & 7));
  const double q = 0.9999999, c = 1e-7;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < kPeakChains; ++j) a[j] = __fma_rn(a[j], q, c);
  }
  double s = 0.0;
#pragma unroll
  for (int j = 0; j < kPeakChains; ++j) s += a[j];
  out[tid] = (float)s;
}

}  // namespace richm

using namespace richm;

extern "C" {

richm_status richm_fma_peak(int kind, double* tflops) {
  clear_error();
  RICHM_ARG(tflops != nullptr, "null output");
  RICHM_ARG(kind >= 0 && kind <= 2, "kind must be 0 (FP32), 1 (packed FP32 pairs) or 2 (FP64)");
  int dev = 0, sms = 0;
  RICHM_CUDA_TRY(cudaGetDevice(&dev));
  RICHM_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int blocks = sms * kPeakBlocksPerSM;
  const long long threads = (long long)blocks * kPeakBlock;
  const int iters = kind == 2 ? 256 : 4096;
  float* out = nullptr;
  RICHM_CUDA_TRY(cudaMalloc(&out, sizeof(float) * threads));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  auto launch = [&]() {
    if (kind == 0) fma_f32_kernel<<<blocks, kPeakBlock>>>(out, iters);
    else if (kind == 1) fma_f32x2_kernel<<<blocks, kPeakBlock>>>(out, iters);
    else fma_f64_kernel<<<blocks, kPeakBlock>>>(out, iters);
  };
  constexpr int kReps = 5;
  float ms = 0.f;
  if (e == cudaSuccess) {
    launch();  // warm-up
    e = cudaEventRecord(e0);
    for (int r = 0; r < kReps && e == cudaSuccess; ++r) launch();
    if (e == cudaSuccess) e = cudaEventRecord(e1);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(out);
  if (e != cudaSuccess) return set_error(RICHM_ERR_CUDA, "FMA microbenchmark failed: %s", cudaGetErrorString(e));
  const double fma_per_thread = (double)iters * kPeakChains * (kind == 1 ? 2.0 : 1.0);
  const double flops = 2.0 * fma_per_thread * (double)threads * kReps;
  *tflops = ms > 0.f ? flops / ((double)ms * 1e-3) / 1e12 : 0.0;
  return RICHM_OK;
}

}  // extern "C"
