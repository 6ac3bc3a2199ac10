// Meta(theta; mu) network of Sec. 2.3 (an MLP 2 -> 64 -> 64 -> nout, ReLU, FP32),
// its backward pass and the Adam update used to train it (Algorithm 1).
//
// The output head says which Table 1 method the outputs parametrise: m weights
// w_i = exp(o_i) / G, then one shared momentum (NAG), none (Richardson), m per-step
// momenta a_i = sigmoid(o_{m+i}) (MOM with at = 0, NAG with at = a), or 2m (NAGex:
// a_i and at_i = sigmoid(o_{2m+i})).
//
// The network is tiny (5457 parameters for m = 16 and one momentum), so one 64-thread
// block handles one instance (one thread per hidden unit and per output); per-instance
// parameter gradients are written to a workspace and summed over the batch by a
// second kernel in a fixed order (deterministic).
#include <cmath>

#include "common.cuh"

namespace richm {

constexpr int kHid = 64;

__host__ __device__ inline int head_outputs(int head, int m) {
  switch (head) {
    case RICHM_HEAD_NAG_SHARED: return m + 1;
    case RICHM_HEAD_RICHARDSON: return m;
    case RICHM_HEAD_MOM:
    case RICHM_HEAD_NAG: return 2 * m;
    case RICHM_HEAD_NAGEX: return 3 * m;
    case RICHM_HEAD_RAW: return m;
    default: return -1;
  }
}

__host__ __device__ inline int meta_count(int nout) { return kHid * 2 + kHid + kHid * kHid + kHid + nout * kHid + nout; }

__device__ inline float sigmoidf(float x) { return 1.f / (1.f + expf(-x)); }

struct MetaPtrs {
  const float *W1, *b1, *W2, *b2, *W3, *b3;
};
__device__ inline MetaPtrs meta_ptrs(const float* P, int nout) {
  MetaPtrs p;
  p.W1 = P;
  p.b1 = p.W1 + kHid * 2;
  p.W2 = p.b1 + kHid;
  p.b2 = p.W2 + kHid * kHid;
  p.W3 = p.b2 + kHid;
  p.b3 = p.W3 + nout * kHid;
  return p;
}

__global__ void __launch_bounds__(kHid) meta_forward_kernel(const float* __restrict__ P, const float* __restrict__ X,
                                                            const float* __restrict__ G, int m, int head,
                                                            float* w_out, float* a_out, float* at_out, float* acts) {
  const int b = blockIdx.x, j = threadIdx.x;
  __shared__ float h1[kHid], h2[kHid], o[kHid];
  const int nout = head_outputs(head, m);
  const MetaPtrs p = meta_ptrs(P, nout);
  const float x0 = X[2 * b], x1 = X[2 * b + 1];
  const float z1 = fmaf(p.W1[2 * j], x0, fmaf(p.W1[2 * j + 1], x1, p.b1[j]));
  h1[j] = fmaxf(z1, 0.f);
  __syncthreads();
  float z2 = p.b2[j];
  for (int k = 0; k < kHid; ++k) z2 = fmaf(p.W2[kHid * j + k], h1[k], z2);
  h2[j] = fmaxf(z2, 0.f);
  __syncthreads();
  if (j < nout) {
    float oj = p.b3[j];
    for (int k = 0; k < kHid; ++k) oj = fmaf(p.W3[kHid * j + k], h2[k], oj);
    o[j] = oj;
  }
  __syncthreads();
  const int na = 2 * kHid + nout;
  if (acts) {
    acts[(long long)b * na + j] = z1;
    acts[(long long)b * na + kHid + j] = z2;
    if (j < nout) acts[(long long)b * na + 2 * kHid + j] = o[j];
  }
  if (j < m && head == RICHM_HEAD_RAW) {
    w_out[(long long)b * m + j] = o[j];
  } else if (j < m) {
    const long long i = (long long)b * m + j;
    w_out[i] = expf(o[j]) / G[b];
    switch (head) {
      case RICHM_HEAD_NAG_SHARED: a_out[i] = sigmoidf(o[m]); break;
      case RICHM_HEAD_RICHARDSON: break;
      case RICHM_HEAD_MOM:
        a_out[i] = sigmoidf(o[m + j]);
        if (at_out) at_out[i] = 0.f;
        break;
      case RICHM_HEAD_NAG: a_out[i] = sigmoidf(o[m + j]); break;
      default:
        a_out[i] = sigmoidf(o[m + j]);
        at_out[i] = sigmoidf(o[2 * m + j]);
    }
  }
}

__global__ void __launch_bounds__(kHid) meta_backward_kernel(const float* __restrict__ P, const float* __restrict__ X,
                                                             const float* __restrict__ G, const float* __restrict__ acts,
                                                             int m, int head, const float* __restrict__ g_w,
                                                             const float* __restrict__ g_a,
                                                             const float* __restrict__ g_at, float* __restrict__ gP) {
  const int b = blockIdx.x, j = threadIdx.x;
  __shared__ float h1[kHid], h2[kHid], go[kHid], gz2[kHid];
  const int nout = head_outputs(head, m);
  const MetaPtrs p = meta_ptrs(P, nout);
  const int na = 2 * kHid + nout;
  const float* A = acts + (long long)b * na;
  const float z1 = A[j], z2 = A[kHid + j];
  h1[j] = fmaxf(z1, 0.f);
  h2[j] = fmaxf(z2, 0.f);
  const long long row = (long long)b * m;
  if (j < m && head == RICHM_HEAD_RAW) {
    go[j] = g_w[row + j];
  } else if (j < m) {
    const float wj = expf(A[2 * kHid + j]) / G[b];
    go[j] = g_w[row + j] * wj;  // dw/do = w
  } else if (j < nout) {
    // momentum outputs: d sigmoid / do = s (1 - s)
    const float s = sigmoidf(A[2 * kHid + j]);
    float g;
    if (head == RICHM_HEAD_NAG_SHARED) {
      g = 0.f;
      for (int i = 0; i < m; ++i) g += g_a[row + i];
    } else if (j < 2 * m) {
      g = g_a[row + j - m];
    } else {
      g = g_at[row + j - 2 * m];
    }
    go[j] = g * s * (1.f - s);
  }
  __syncthreads();
  const int cnt = meta_count(nout);
  float* g = gP + (long long)b * cnt;
  float* gW1 = g;
  float* gb1 = gW1 + kHid * 2;
  float* gW2 = gb1 + kHid;
  float* gb2 = gW2 + kHid * kHid;
  float* gW3 = gb2 + kHid;
  float* gb3 = gW3 + nout * kHid;
  // layer 3
  for (int r = 0; r < nout; ++r) gW3[kHid * r + j] = go[r] * h2[j];
  if (j < nout) gb3[j] = go[j];
  float gh2 = 0.f;
  for (int r = 0; r < nout; ++r) gh2 = fmaf(p.W3[kHid * r + j], go[r], gh2);
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

static richm_status check_head(int m, int head) {
  RICHM_ARG(head >= RICHM_HEAD_NAG_SHARED && head <= RICHM_HEAD_RAW, "unknown meta head %d", head);
  const int nout = head_outputs(head, m);
  RICHM_ARG(m >= 1 && nout <= kHid, "m = %d out of range for head %d (at most %d outputs)", m, head, kHid);
  return RICHM_OK;
}

richm_status richm_meta_param_count(int m, int head, int* count) {
  clear_error();
  RICHM_ARG(count != nullptr, "null output");
  RICHM_TRY(check_head(m, head));
  *count = meta_count(head_outputs(head, m));
  return RICHM_OK;
}

richm_status richm_meta_forward(const float* params, const float* inputs, const float* G, int B, int m, int head,
                                float* w_out, float* alpha_out, float* alpha_t_out, float* acts, void* stream) {
  clear_error();
  RICHM_TRY(check_head(m, head));
  RICHM_ARG(params && inputs && G && w_out, "null argument");
  RICHM_ARG(head == RICHM_HEAD_RICHARDSON || head == RICHM_HEAD_RAW || alpha_out, "null alpha_out");
  RICHM_ARG(head != RICHM_HEAD_NAGEX || alpha_t_out, "null alpha_t_out (NAGex head)");
  RICHM_ARG(B >= 1, "B < 1");
  meta_forward_kernel<<<B, kHid, 0, (cudaStream_t)stream>>>(params, inputs, G, m, head, w_out, alpha_out,
                                                             alpha_t_out, acts);
  RICHM_LAUNCH_CHECK("meta forward");
  return RICHM_OK;
}

richm_status richm_meta_backward(const float* params, const float* inputs, const float* G, const float* acts,
                                 int B, int m, int head, const float* g_w, const float* g_alpha,
                                 const float* g_alpha_t, float* g_params, void* work, size_t work_bytes,
                                 void* stream) {
  clear_error();
  RICHM_TRY(check_head(m, head));
  RICHM_ARG(params && inputs && G && acts && g_w && g_params && work, "null argument");
  RICHM_ARG(head == RICHM_HEAD_RICHARDSON || head == RICHM_HEAD_RAW || g_alpha, "null g_alpha");
  RICHM_ARG(head != RICHM_HEAD_NAGEX || g_alpha_t, "null g_alpha_t (NAGex head)");
  RICHM_ARG(B >= 1, "B < 1");
  const int cnt = meta_count(head_outputs(head, m));
  const size_t need = sizeof(float) * (size_t)B * cnt;
  if (work_bytes < need) return set_error(RICHM_ERR_NOMEM, "workspace %zu < %zu bytes", work_bytes, need);
  cudaStream_t s = (cudaStream_t)stream;
  meta_backward_kernel<<<B, kHid, 0, s>>>(params, inputs, G, acts, m, head, g_w, g_alpha, g_alpha_t, (float*)work);
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
