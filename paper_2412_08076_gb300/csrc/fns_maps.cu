// Parameter maps of the Richardson(m)-FNS neural iteration (Sec. 3.1, eq. 20):
// the Meta-Lambda and Meta-T networks' outputs turned into the symbol S and the
// transition field t that richm_fourier_correction_t applies, and their reverse modes.
//
// Symbol: Lambda approximates the inverses of A's eigenvalues. Here it is the regularised
// inverse of a periodic 9-point symbol whose coefficients are the instance's own Q1
// stencil scaled by the network: p_m = q_m exp(o_m) (m < 5), delta = q_5 exp(o_5),
//   sigma(k) = p0 + 2 p1 cos t2 + 2 p2 cos t1 + 2 p3 cos(t1 + t2) + 2 p4 cos(t1 - t2),
//   S(k) = sigma / (sigma^2 + delta^2),   t = 2 pi k / n,
// so that the network starts (o = 0) at the periodic inverse of the instance's stencil.
//
// Transition: a band kernel of half-width 1, Hermitian-symmetric so that its field is
// real: tau[9] = (tau_0, then (re, im) of the offsets (0,1), (1,0), (1,1), (1,-1)), and
//   t(i, j) = tau_0 + 2 sum_d (re_d cos(2 pi d.x / n) - im_d sin(2 pi d.x / n)),
// d.x = d_row i + d_col j.
//
// The reverse modes sum over the n^2 frequencies or grid points in FP64 per block and
// then over the blocks in a fixed order (deterministic).
#include <cmath>

#include "common.cuh"

namespace richm {

struct SymQ {
  float q[6];
};

constexpr int kMapThreads = 256;

__device__ __forceinline__ void symbol_at(int k1, int k2, int n, const SymQ& Q, const float* __restrict__ o,
                                          float* p, float* basis, float& sigma, float& delta) {
#pragma unroll
  for (int m = 0; m < 5; ++m) p[m] = Q.q[m] * expf(o[m]);
  delta = Q.q[5] * expf(o[5]);
  const float f = 2.f / (float)n;
  const float c1 = cospif(f * k1), c2 = cospif(f * k2);
  const float cp = cospif(f * ((k1 + k2) % n)), cm = cospif(f * ((k1 - k2 + n) % n));
  basis[0] = 1.f;
  basis[1] = 2.f * c2;
  basis[2] = 2.f * c1;
  basis[3] = 2.f * cp;
  basis[4] = 2.f * cm;
  sigma = 0.f;
#pragma unroll
  for (int m = 0; m < 5; ++m) sigma = fmaf(p[m], basis[m], sigma);
}

__global__ void __launch_bounds__(kMapThreads) symbol_map_kernel(int n, SymQ Q, const float* __restrict__ o,
                                                                 float2* __restrict__ S) {
  const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= (long long)n * n) return;
  float p[5], basis[5], sigma, delta;
  symbol_at((int)(k / n), (int)(k % n), n, Q, o, p, basis, sigma, delta);
  S[k] = make_float2(sigma / fmaf(sigma, sigma, delta * delta), 0.f);
}

// Block-wide sum of NV FP64 values per thread into partials[block][NV].
template <int NV>
__device__ __forceinline__ void block_sum(double* v, double* __restrict__ partials) {
  __shared__ double sh[kMapThreads / 32][NV];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < NV; ++i) {
    const double s = warp_sum(v[i]);
    if (lane == 0) sh[warp][i] = s;
  }
  __syncthreads();
  if (threadIdx.x < NV) {
    double s = 0.0;
    for (int w = 0; w < kMapThreads / 32; ++w) s += sh[w][threadIdx.x];
    partials[(long long)blockIdx.x * NV + threadIdx.x] = s;
  }
}

template <int NV>
__global__ void partials_sum_kernel(const double* __restrict__ partials, int nblocks, float* __restrict__ out) {
  const int i = threadIdx.x;
  if (i >= NV) return;
  double s = 0.0;
  for (int b = 0; b < nblocks; ++b) s += partials[(long long)b * NV + i];
  out[i] = (float)s;
}

// do_m = sum_k Re(dS(k)) dS/dsigma basis_m p_m (m < 5), do_5 = sum_k Re(dS(k)) dS/ddelta delta
__global__ void __launch_bounds__(kMapThreads) symbol_map_vjp_kernel(int n, SymQ Q, const float* __restrict__ o,
                                                                     const float2* __restrict__ dS,
                                                                     double* __restrict__ partials) {
  const long long nn = (long long)n * n;
  const long long per = (nn + gridDim.x - 1) / gridDim.x;
  const long long k0 = (long long)blockIdx.x * per, k1 = min(k0 + per, nn);
  double v[6] = {0, 0, 0, 0, 0, 0};
  for (long long k = k0 + threadIdx.x; k < k1; k += blockDim.x) {
    float p[5], basis[5], sigma, delta;
    symbol_at((int)(k / n), (int)(k % n), n, Q, o, p, basis, sigma, delta);
    const double s = sigma, d = delta, den = s * s + d * d;
    const double dsig = (d * d - s * s) / (den * den), ddel = -2.0 * s * d / (den * den);
    const double g = dS[k].x;
#pragma unroll
    for (int m = 0; m < 5; ++m) v[m] += g * dsig * basis[m] * p[m];
    v[5] += g * ddel * d;
  }
  block_sum<6>(v, partials);
}

__device__ __forceinline__ void transition_basis(int i, int j, int n, float* bs) {
  const float f = 2.f / (float)n;
  const int a[4] = {j % n, i % n, (i + j) % n, ((i - j) % n + n) % n};
  bs[0] = 1.f;
#pragma unroll
  for (int d = 0; d < 4; ++d) {
    float sn, cs;
    sincospif(f * a[d], &sn, &cs);
    bs[1 + 2 * d] = 2.f * cs;
    bs[2 + 2 * d] = -2.f * sn;
  }
}

__global__ void __launch_bounds__(kMapThreads) transition_map_kernel(int n, const float* __restrict__ tau,
                                                                     float* __restrict__ t) {
  const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= (long long)n * n) return;
  float bs[9];
  transition_basis((int)(k / n), (int)(k % n), n, bs);
  float v = 0.f;
#pragma unroll
  for (int q = 0; q < 9; ++q) v = fmaf(tau[q], bs[q], v);
  t[k] = v;
}

__global__ void __launch_bounds__(kMapThreads) transition_map_vjp_kernel(int n, const float* __restrict__ dt,
                                                                         double* __restrict__ partials) {
  const long long nn = (long long)n * n;
  const long long per = (nn + gridDim.x - 1) / gridDim.x;
  const long long k0 = (long long)blockIdx.x * per, k1 = min(k0 + per, nn);
  double v[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  for (long long k = k0 + threadIdx.x; k < k1; k += blockDim.x) {
    float bs[9];
    transition_basis((int)(k / n), (int)(k % n), n, bs);
    const double g = dt[k];
#pragma unroll
    for (int q = 0; q < 9; ++q) v[q] += g * bs[q];
  }
  block_sum<9>(v, partials);
}

constexpr int kMapBlocks = 304;  // reverse-mode blocks (a fixed count: the summation order does not depend on the GPU)

}  // namespace richm

using namespace richm;

extern "C" {

richm_status richm_fns_map_workspace(size_t* bytes) {
  clear_error();
  RICHM_ARG(bytes != nullptr, "null output");
  *bytes = sizeof(double) * kMapBlocks * 9;
  return RICHM_OK;
}

richm_status richm_symbol_from_stencil(int n, const double* q, const float* o, void* symbol, void* stream) {
  clear_error();
  RICHM_ARG(n >= 1 && q && o && symbol, "null argument or n < 1");
  SymQ Q;
  for (int m = 0; m < 6; ++m) Q.q[m] = (float)q[m];
  const long long nn = (long long)n * n;
  symbol_map_kernel<<<(unsigned)((nn + kMapThreads - 1) / kMapThreads), kMapThreads, 0, (cudaStream_t)stream>>>(
      n, Q, o, (float2*)symbol);
  RICHM_LAUNCH_CHECK("symbol map");
  return RICHM_OK;
}

richm_status richm_symbol_from_stencil_vjp(int n, const double* q, const float* o, const void* dsymbol, float* d_o,
                                           void* work, size_t work_bytes, void* stream) {
  clear_error();
  RICHM_ARG(n >= 1 && q && o && dsymbol && d_o && work, "null argument or n < 1");
  if (work_bytes < sizeof(double) * kMapBlocks * 9)
    return set_error(RICHM_ERR_NOMEM, "workspace %zu < %zu bytes", work_bytes, sizeof(double) * kMapBlocks * 9);
  SymQ Q;
  for (int m = 0; m < 6; ++m) Q.q[m] = (float)q[m];
  cudaStream_t s = (cudaStream_t)stream;
  symbol_map_vjp_kernel<<<kMapBlocks, kMapThreads, 0, s>>>(n, Q, o, (const float2*)dsymbol, (double*)work);
  RICHM_LAUNCH_CHECK("symbol map reverse");
  partials_sum_kernel<6><<<1, 32, 0, s>>>((const double*)work, kMapBlocks, d_o);
  RICHM_LAUNCH_CHECK("symbol map reduction");
  return RICHM_OK;
}

richm_status richm_transition_from_band(int n, const float* tau, float* transition, void* stream) {
  clear_error();
  RICHM_ARG(n >= 1 && tau && transition, "null argument or n < 1");
  const long long nn = (long long)n * n;
  transition_map_kernel<<<(unsigned)((nn + kMapThreads - 1) / kMapThreads), kMapThreads, 0,
                          (cudaStream_t)stream>>>(n, tau, transition);
  RICHM_LAUNCH_CHECK("transition map");
  return RICHM_OK;
}

richm_status richm_transition_from_band_vjp(int n, const float* dtransition, float* dtau, void* work,
                                            size_t work_bytes, void* stream) {
  clear_error();
  RICHM_ARG(n >= 1 && dtransition && dtau && work, "null argument or n < 1");
  if (work_bytes < sizeof(double) * kMapBlocks * 9)
    return set_error(RICHM_ERR_NOMEM, "workspace %zu < %zu bytes", work_bytes, sizeof(double) * kMapBlocks * 9);
  cudaStream_t s = (cudaStream_t)stream;
  transition_map_vjp_kernel<<<kMapBlocks, kMapThreads, 0, s>>>(n, dtransition, (double*)work);
  RICHM_LAUNCH_CHECK("transition map reverse");
  partials_sum_kernel<9><<<1, 32, 0, s>>>((const double*)work, kMapBlocks, dtau);
  RICHM_LAUNCH_CHECK("transition map reduction");
  return RICHM_OK;
}

}  // extern "C"
