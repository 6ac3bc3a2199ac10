// Order of the steps inside one period of Richardson(m) and its momentum forms.
//
// Eqs. 8-9 fix the set of the m weights of a period, not the order in which its
// steps run. In exact arithmetic the order of the Richardson(m) steps does not change
// the period's result (the factors (I - w_i A) commute), but in FP32 the rounding
// made at step s is carried by the product of the later factors, which with the long
// Chebyshev steps (w_i lambda up to ~30) can grow by orders of magnitude inside a
// period. A Leja ordering of the nodes z_i = 1/w_i (the roots of the period's residual
// polynomial) keeps the partial products small (Reichel, BIT 30 (1990) 332-346): first
// the node of largest |z|, then repeatedly the node that maximises the product of its
// distances to the nodes already taken; ties go to the smaller index.
//
// The product is formed in FP64 in the order the nodes were taken, on the host and on
// the device alike, so both give the same permutation for the same weights.
#include <cmath>

#include "common.cuh"

namespace richm {

// perm[s] = index of the step that runs at position s of the period.
__host__ __device__ static void leja_perm(const double* z, int m, int* perm) {
  unsigned long long taken = 0ull;  // m <= 64
  int first = 0;
  for (int i = 1; i < m; ++i)
    if (fabs(z[i]) > fabs(z[first])) first = i;
  perm[0] = first;
  taken |= 1ull << first;
  for (int s = 1; s < m; ++s) {
    int best = -1;
    double best_score = 0.0;
    for (int i = 0; i < m; ++i) {
      if (taken & (1ull << i)) continue;
      double p = 1.0;
      for (int j = 0; j < s; ++j) p *= fabs(z[i] - z[perm[j]]);
      if (best < 0 || p > best_score) {
        best = i;
        best_score = p;
      }
    }
    perm[s] = best;
    taken |= 1ull << best;
  }
}

template <typename R>
__global__ void leja_permute_kernel(int batch, int m, const R* __restrict__ w, const R* __restrict__ a,
                                    const R* __restrict__ at, R* __restrict__ w_out, R* __restrict__ a_out,
                                    R* __restrict__ at_out) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= batch) return;
  double z[64];
  int perm[64];
  for (int i = 0; i < m; ++i) z[i] = 1.0 / (double)w[(long long)b * m + i];
  leja_perm(z, m, perm);
  const long long o = (long long)b * m;
  for (int s = 0; s < m; ++s) {
    w_out[o + s] = w[o + perm[s]];
    if (a_out) a_out[o + s] = a[o + perm[s]];
    if (at_out) at_out[o + s] = at[o + perm[s]];
  }
}

}  // namespace richm

using namespace richm;

extern "C" {

richm_status richm_leja_order(const double* w, int m, int* perm) {
  clear_error();
  RICHM_ARG(w != nullptr && perm != nullptr, "null argument");
  RICHM_ARG(m >= 1 && m <= 64, "m = %d out of range [1, 64]", m);
  double z[64];
  for (int i = 0; i < m; ++i) {
    RICHM_ARG(std::isfinite(w[i]) && w[i] != 0.0, "weight %d is zero or not finite", i);
    z[i] = 1.0 / w[i];
  }
  leja_perm(z, m, perm);
  return RICHM_OK;
}

richm_status richm_leja_permute(const richm_operator* op, richm_dtype dtype, const void* w, const void* alpha,
                                const void* alpha_t, int m, void* w_out, void* alpha_out, void* alpha_t_out,
                                void* stream) {
  clear_error();
  RICHM_ARG(op != nullptr, "null operator");
  RICHM_ARG(m >= 1 && m <= 64, "m = %d out of range [1, 64]", m);
  RICHM_ARG(w != nullptr && w_out != nullptr, "null weights");
  RICHM_ARG((alpha == nullptr) == (alpha_out == nullptr), "alpha and alpha_out must both be given or both NULL");
  RICHM_ARG((alpha_t == nullptr) == (alpha_t_out == nullptr),
            "alpha_t and alpha_t_out must both be given or both NULL");
  RICHM_ARG(w != w_out && (alpha == nullptr || alpha != alpha_out) && (alpha_t == nullptr || alpha_t != alpha_t_out),
            "the permutation is not done in place");
  const bool dbl = dtype == RICHM_F64 || dtype == RICHM_C128;
  RICHM_ARG(dbl || dtype == RICHM_F32 || dtype == RICHM_C64 || dtype == RICHM_BF16, "unknown dtype %d", (int)dtype);
  const int batch = op->batch;
  const int thr = 64;
  const int blocks = (batch + thr - 1) / thr;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (dbl)
    leja_permute_kernel<double><<<blocks, thr, 0, s>>>(batch, m, (const double*)w, (const double*)alpha,
                                                       (const double*)alpha_t, (double*)w_out, (double*)alpha_out,
                                                       (double*)alpha_t_out);
  else
    leja_permute_kernel<float><<<blocks, thr, 0, s>>>(batch, m, (const float*)w, (const float*)alpha,
                                                      (const float*)alpha_t, (float*)w_out, (float*)alpha_out,
                                                      (float*)alpha_t_out);
  RICHM_LAUNCH_CHECK("Leja permutation");
  return RICHM_OK;
}

}  // extern "C"
