// Meta(theta; mu) network of Sec. 2.3 (an MLP 2 -> 64 -> 64 -> m+1, ReLU, FP32),
// its backward pass and the Adam update used to train it (Algorithm 1).
//
// The network is tiny (5457 parameters for m = 16), so one 64-thread block handles
// one instance; per-instance parameter gradients are written to a workspace and
// summed over the batch by a second kernel in a fixed order (deterministic).
#include <cmath>

#include "common.cuh"

namespace richm {

constexpr int kHid = 64;

__host__ __device__ inline int meta_count(int m) { return kHid * 2 + kHid + kHid * kHid + kHid + (m + 1) * kHid + (m + 1); }

struct MetaPtrs {
  const float *W1, *b1, *W2, *b2, *W3, *b3;
};
__device__ inline MetaPtrs meta_ptrs(const float* P, int m) {
  MetaPtrs p;
  p.W1 = P;
  p.b1 = p.W1 + kHid * 2;
  p.W2 = p.b1 + kHid;
  p.b2 = p.W2 + kHid * kHid;
  p.W3 = p.b2 + kHid;
  p.b3 = p.W3 + (m + 1) * kHid;
  return p;
}

__global__ void __launch_bounds__(kHid) meta_forward_kernel(const float* __restrict__ P, const float* __restrict__ X,
                                                            const float* __restrict__ G, int m, float* w_out,
                                                            float* a_out, float* acts) {
  const int b = blockIdx.x, j = threadIdx.x;
  __shared__ float h1[kHid], h2[kHid], o[kHid];
  const MetaPtrs p = meta_ptrs(P, m);
  const float x0 = X[2 * b], x1 = X[2 * b + 1];
  const float z1 = fmaf(p.W1[2 * j], x0, fmaf(p.W1[2 * j + 1], x1, p.b1[j]));
  h1[j] = fmaxf(z1, 0.f);
  __syncthreads();
  float z2 = p.b2[j];
  for (int k = 0; k < kHid; ++k) z2 = fmaf(p.W2[kHid * j + k], h1[k], z2);
  h2[j] = fmaxf(z2, 0.f);
  __syncthreads();
  if (j <= m) {
    float oj = p.b3[j];
    for (int k = 0; k < kHid; ++k) oj = fmaf(p.W3[kHid * j + k], h2[k], oj);
    o[j] = oj;
  }
  __syncthreads();
  const int na = 2 * kHid + m + 1;
  if (acts) {
    acts[(long long)b * na + j] = z1;
    acts[(long long)b * na + kHid + j] = z2;
    if (j <= m) acts[(long long)b * na + 2 * kHid + j] = o[j];
  }
  const float alpha = 1.f / (1.f + expf(-o[m]));
  if (j < m) {
    w_out[(long long)b * m + j] = expf(o[j]) / G[b];
    a_out[(long long)b * m + j] = alpha;
  }
}

__global__ void __launch_bounds__(kHid) meta_backward_kernel(const float* __restrict__ P, const float* __restrict__ X,
                                                             const float* __restrict__ G, const float* __restrict__ acts,
                                                             int m, const float* __restrict__ g_w,
                                                             const float* __restrict__ g_a, float* __restrict__ gP) {
  const int b = blockIdx.x, j = threadIdx.x;
  __shared__ float h1[kHid], h2[kHid], go[kHid], gz2[kHid];
  const MetaPtrs p = meta_ptrs(P, m);
  const int na = 2 * kHid + m + 1;
  const float* A = acts + (long long)b * na;
  const float z1 = A[j], z2 = A[kHid + j];
  h1[j] = fmaxf(z1, 0.f);
  h2[j] = fmaxf(z2, 0.f);
  if (j < m) {
    const float wj = expf(A[2 * kHid + j]) / G[b];
    go[j] = g_w[(long long)b * m + j] * wj;  // dw/do = w
  } else if (j == m) {
    float ga = 0.f;
    for (int i = 0; i < m; ++i) ga += g_a[(long long)b * m + i];
    const float s = 1.f / (1.f + expf(-A[2 * kHid + m]));
    go[m] = ga * s * (1.f - s);
  }
  __syncthreads();
  const int cnt = meta_count(m);
  float* g = gP + (long long)b * cnt;
  float* gW1 = g;
  float* gb1 = gW1 + kHid * 2;
  float* gW2 = gb1 + kHid;
  float* gb2 = gW2 + kHid * kHid;
  float* gW3 = gb2 + kHid;
  float* gb3 = gW3 + (m + 1) * kHid;
  // layer 3
  for (int r = 0; r <= m; ++r) gW3[kHid * r + j] = go[r] * h2[j];
  if (j <= m) gb3[j] = go[j];
  float gh2 = 0.f;
  for (int r = 0; r <= m; ++r) gh2 = fmaf(p.W3[kHid * r + j], go[r], gh2);
  const float gz2j = z2 > 0.f ? gh2 : 0.f;
  gz2[j] = gz2j;
  __syncthreads();
  // layer 2
  for (int c = 0; c < kHid; ++c) gW2[kHid * j + c] = gz2j * h1[c];
  gb2[j] = gz2j;
  float gh1 = 0.f;
  for (int r = 0; r < kHid; ++r) gh1 = fmaf(p.W2[kHid * r + j], gz2[r], gh1);
  const float gz1 = z1 > 0.f ? gh1 : 0.f;
  gW1[2 * j] = gz1 * X[2 * b];
  gW1[2 * j + 1] = gz1 * X[2 * b + 1];
  gb1[j] = gz1;
}

__global__ void batch_sum_kernel(const float* __restrict__ gP, int B, int cnt, float* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= cnt) return;
  float s = 0.f;
  for (int b = 0; b < B; ++b) s += gP[(long long)b * cnt + i];
  out[i] = s;
}

__global__ void adam_kernel(float* p, const float* g, float* m1, float* m2, int count, float lr, float b1, float b2,
                            float eps, float c1, float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  const float gi = g[i];
  const float a = b1 * m1[i] + (1.f - b1) * gi;
  const float v = b2 * m2[i] + (1.f - b2) * gi * gi;
  m1[i] = a;
  m2[i] = v;
  const float mh = a / c1, vh = v / c2;
  p[i] -= lr * mh / (sqrtf(vh) + eps);
}

}  // namespace richm

using namespace richm;

extern "C" {

richm_status richm_meta_param_count(int m, int* count) {
  clear_error();
  RICHM_ARG(count != nullptr, "null output");
  RICHM_ARG(m >= 1 && m <= kHid - 1, "m = %d out of range [1, 63]", m);
  *count = meta_count(m);
  return RICHM_OK;
}

richm_status richm_meta_forward(const float* params, const float* inputs, const float* G, int B, int m,
                                float* w_out, float* alpha_out, float* acts, void* stream) {
  clear_error();
  RICHM_ARG(params && inputs && G && w_out && alpha_out, "null argument");
  RICHM_ARG(B >= 1, "B < 1");
  RICHM_ARG(m >= 1 && m <= kHid - 1, "m = %d out of range [1, 63]", m);
  meta_forward_kernel<<<B, kHid, 0, (cudaStream_t)stream>>>(params, inputs, G, m, w_out, alpha_out, acts);
  RICHM_LAUNCH_CHECK("meta forward");
  return RICHM_OK;
}

richm_status richm_meta_backward(const float* params, const float* inputs, const float* G, const float* acts,
                                 int B, int m, const float* g_w, const float* g_alpha, float* g_params, void* work,
                                 size_t work_bytes, void* stream) {
  clear_error();
  RICHM_ARG(params && inputs && G && acts && g_w && g_alpha && g_params && work, "null argument");
  RICHM_ARG(B >= 1, "B < 1");
  RICHM_ARG(m >= 1 && m <= kHid - 1, "m = %d out of range [1, 63]", m);
  const int cnt = meta_count(m);
  const size_t need = sizeof(float) * (size_t)B * cnt;
  if (work_bytes < need) return set_error(RICHM_ERR_NOMEM, "workspace %zu < %zu bytes", work_bytes, need);
  cudaStream_t s = (cudaStream_t)stream;
  meta_backward_kernel<<<B, kHid, 0, s>>>(params, inputs, G, acts, m, g_w, g_alpha, (float*)work);
  RICHM_LAUNCH_CHECK("meta backward");
  batch_sum_kernel<<<(cnt + 255) / 256, 256, 0, s>>>((const float*)work, B, cnt, g_params);
  RICHM_LAUNCH_CHECK("meta gradient sum");
  return RICHM_OK;
}

richm_status richm_adam_step(float* params, const float* grads, float* m1, float* m2, int count, int t, float lr,
                             float beta1, float beta2, float eps, void* stream) {
  clear_error();
  RICHM_ARG(params && grads && m1 && m2, "null argument");
  RICHM_ARG(count >= 1 && t >= 1, "count and t must be >= 1");
  const float c1 = 1.f - powf(beta1, (float)t);
  const float c2 = 1.f - powf(beta2, (float)t);
  adam_kernel<<<(count + 255) / 256, 256, 0, (cudaStream_t)stream>>>(params, grads, m1, m2, count, lr, beta1, beta2,
                                                                     eps, c1, c2);
  RICHM_LAUNCH_CHECK("adam");
  return RICHM_OK;
}

}  // extern "C"
