// Bit-for-bit self-test of the integer-field FP32 <-> FP64 conversions
// (f32_to_f64_exact, f64_to_f32_rn) against the hardware conversions.
#include "common.cuh"

namespace richm {

__device__ __forceinline__ unsigned long long mix64_dev(unsigned long long z) {
  // SplitMix64 finaliser (Steele, Lea, Flood 2014): only spreads the low test words.
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
  return z ^ (z >> 31);
}

__device__ __forceinline__ void count_mismatch(bool bad, unsigned long long* counter) {
  const unsigned mask = __ballot_sync(0xffffffffu, bad);
  if ((threadIdx.x & 31) == 0 && mask) atomicAdd(counter, (unsigned long long)__popc(mask));
}

// Every binary32 bit pattern, widened both ways.
__global__ void widen_check_kernel(unsigned long long* bad) {
  const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
  for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < (1ULL << 32);
       i += stride) {
    const float f = __uint_as_float((unsigned)i);
    const bool diff = __double_as_longlong(f32_to_f64_exact(f)) != __double_as_longlong((double)f);
    count_mismatch(diff, bad);
  }
}

// Every binary64 high word (sign, exponent, top 20 fraction bits) with low words at
// and around the rounding boundary of the 29 dropped bits, and one spread low word.
__global__ void narrow_check_kernel(unsigned long long* bad) {
  const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
  for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < (1ULL << 32);
       i += stride) {
    const unsigned hi = (unsigned)i;
    const unsigned lows[8] = {0u,          0x0fffffffu, 0x10000000u, 0x10000001u,
                              0x1fffffffu, 0x20000000u, 0x30000000u, (unsigned)mix64_dev(i)};
    bool diff = false;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const double d = __hiloint2double((int)hi, (int)lows[k]);
      diff |= __float_as_uint(f64_to_f32_rn(d)) != __float_as_uint((float)d);
    }
    count_mismatch(diff, bad);
  }
}

}  // namespace richm

using namespace richm;

extern "C" {

richm_status richm_selftest_conversions(long long* mismatches) {
  clear_error();
  RICHM_ARG(mismatches != nullptr, "null output");
  unsigned long long* d = nullptr;
  RICHM_CUDA_TRY(cudaMalloc(&d, 2 * sizeof(unsigned long long)));
  int dev = 0, sms = 0;
  cudaError_t e = cudaMemset(d, 0, 2 * sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) {
    // grid-stride loops: eight blocks per multiprocessor
    widen_check_kernel<<<sms * 8, 256>>>(d);
    narrow_check_kernel<<<sms * 8, 256>>>(d + 1);
    e = cudaGetLastError();
  }
  unsigned long long h[2] = {0, 0};
  if (e == cudaSuccess) e = cudaMemcpy(h, d, sizeof(h), cudaMemcpyDeviceToHost);
  cudaFree(d);
  if (e != cudaSuccess) return set_error(RICHM_ERR_CUDA, "conversion self-test failed: %s", cudaGetErrorString(e));
  mismatches[0] = (long long)h[0];
  mismatches[1] = (long long)h[1];
  return RICHM_OK;
}

}  // extern "C"
