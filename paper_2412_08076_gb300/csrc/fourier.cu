// Fourier-domain correction of the FNS iteration (eqs. 19-20 with T = I):
//   x += Re( IFFT2( S .* FFT2(b - A x) ) )
// The residual is real, so its spectrum R is Hermitian (R(-k) = conj(R(k))), and the
// real part of IFFT2(S .* R) is the inverse transform of the Hermitian part of S .* R,
// which is R(k) (S(k) + conj(S(-k))) / 2. The correction is therefore computed with a
// real-to-complex forward transform, the symmetrised symbol on the half spectrum and a
// complex-to-real inverse: half the transform work of the complex form, same result.
// The residual (FP32 state, FP32 arithmetic like the sweeps it corrects) and the update
// of x are single passes; the transforms are batched cuFFT calls (a library FFT).
#include <cufft.h>

#include <cmath>

#include "common.cuh"

namespace richm {

struct FftState {
  cufftHandle fwd = 0, inv = 0;
  int n = 0;
  int batch = 0;
  size_t work = 0;
};

static size_t a256(size_t v) { return (v + 255) / 256 * 256; }

void fourier_release(richm_operator* op) {
  if (!op || !op->fft_state) return;
  auto* st = reinterpret_cast<FftState*>(op->fft_state);
  if (st->fwd) cufftDestroy(st->fwd);
  if (st->inv) cufftDestroy(st->inv);
  delete st;
  op->fft_state = nullptr;
}

static richm_status ensure_plan(richm_operator* op, FftState** out) {
  const int n = op->h_inst[0].n;
  for (int b = 0; b < op->batch; ++b)
    if (op->h_inst[b].kind != RICHM_ANISO_Q1 || op->h_inst[b].n != n)
      return set_error(RICHM_ERR_UNSUPPORTED, "the Fourier correction needs Q1 instances of one size");
  if (!op->fft_state) {
    auto* st = new FftState();
    int dims[2] = {n, n};
    const int nh = n / 2 + 1;
    size_t wf = 0, wi = 0;
    cufftResult r = cufftCreate(&st->fwd);
    if (r == CUFFT_SUCCESS) r = cufftCreate(&st->inv);
    if (r == CUFFT_SUCCESS) r = cufftSetAutoAllocation(st->fwd, 0);
    if (r == CUFFT_SUCCESS) r = cufftSetAutoAllocation(st->inv, 0);
    if (r == CUFFT_SUCCESS)
      r = cufftMakePlanMany(st->fwd, 2, dims, nullptr, 1, n * n, nullptr, 1, n * nh, CUFFT_R2C, op->batch, &wf);
    if (r == CUFFT_SUCCESS)
      r = cufftMakePlanMany(st->inv, 2, dims, nullptr, 1, n * nh, nullptr, 1, n * n, CUFFT_C2R, op->batch, &wi);
    if (r != CUFFT_SUCCESS) {
      if (st->fwd) cufftDestroy(st->fwd);
      if (st->inv) cufftDestroy(st->inv);
      delete st;
      return set_error(RICHM_ERR_CUDA, "cuFFT plan creation failed (%d)", (int)r);
    }
    st->n = n;
    st->batch = op->batch;
    st->work = wf > wi ? wf : wi;
    op->fft_state = st;
  }
  *out = reinterpret_cast<FftState*>(op->fft_state);
  return RICHM_OK;
}

// res[b][i][j] = (b - A x)(i, j) (dense n x n per instance, FP32).
__global__ void fourier_resid_kernel(const Inst* insts, int n, const float* __restrict__ x,
                                     const float* __restrict__ rhs, float* __restrict__ res) {
  const int b = blockIdx.z;
  const int i = blockIdx.y;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const Inst& I = insts[b];
  const long long o = I.off + (long long)(i + 1) * I.pitch + j;
  const long long p = I.pitch;
  // rows 0 and n + 1 and the columns from n on are zero padding (pitch > n); column -1
  // is not read (for the first row of the first instance it would lie before the buffer)
  const bool west = j > 0;
  const float xc = x[o], xw = west ? x[o - 1] : 0.f, xe = x[o + 1];
  const float xn = x[o - p], xs = x[o + p];
  const float xnw = west ? x[o - p - 1] : 0.f, xne = x[o - p + 1];
  const float xsw = west ? x[o + p - 1] : 0.f, xse = x[o + p + 1];
  const float ax = (float)I.c * xc + (float)I.ax * (xw + xe) + (float)I.ay * (xn + xs) +
                   (float)I.d1 * (xse + xnw) + (float)I.d2 * (xne + xsw);
  res[((long long)b * n + i) * n + j] = rhs[o] - ax;
}

// half[b][k1][k2] *= (S(k1, k2) + conj(S(-k1, -k2))) / (2 n^2), k2 = 0 .. n/2 (symbol
// [n][n] shared by the batch; indices mod n).
__global__ void fourier_symbol_kernel(float2* __restrict__ half, const float2* __restrict__ S, int n, int batch,
                                      float scale) {
  const int nh = n / 2 + 1;
  const long long per = (long long)n * nh;
  const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= per * batch) return;
  const int q = (int)(k % per);
  const int k1 = q / nh, k2 = q % nh;
  const int m1 = k1 == 0 ? 0 : n - k1, m2 = k2 == 0 ? 0 : n - k2;
  const float2 s = S[(long long)k1 * n + k2];
  const float2 t = S[(long long)m1 * n + m2];
  const float sr = 0.5f * scale * (s.x + t.x), si = 0.5f * scale * (s.y - t.y);
  const float2 v = half[k];
  half[k] = make_float2(sr * v.x - si * v.y, sr * v.y + si * v.x);
}

// x += res on the interior.
__global__ void fourier_update_kernel(const Inst* insts, int n, float* __restrict__ x,
                                      const float* __restrict__ res) {
  const int b = blockIdx.z;
  const int i = blockIdx.y;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const Inst& I = insts[b];
  const long long o = I.off + (long long)(i + 1) * I.pitch + j;
  x[o] += res[((long long)b * n + i) * n + j];
}

}  // namespace richm

using namespace richm;

extern "C" {

richm_status richm_fourier_workspace(const richm_operator* op, size_t* bytes) {
  clear_error();
  RICHM_ARG(op && bytes, "null argument");
  FftState* st = nullptr;
  RICHM_TRY(ensure_plan(const_cast<richm_operator*>(op), &st));
  const size_t nn = (size_t)st->n * st->n, nh = (size_t)st->n * (st->n / 2 + 1);
  *bytes = a256(sizeof(float) * nn * st->batch) + a256(sizeof(float2) * nh * st->batch) + a256(st->work);
  return RICHM_OK;
}

richm_status richm_fourier_correction(richm_operator* op, richm_dtype dtype, void* x, const void* b,
                                      const void* symbol, void* work, size_t work_bytes, void* stream) {
  clear_error();
  RICHM_ARG(op != nullptr, "null operator");
  RICHM_ARG(dtype == RICHM_F32, "the Fourier correction takes RICHM_F32 state");
  RICHM_ARG(x && b && symbol && work, "null argument");
  FftState* st = nullptr;
  RICHM_TRY(ensure_plan(op, &st));
  const int n = st->n;
  const size_t nn = (size_t)n * n, nh = (size_t)n * (n / 2 + 1);
  const size_t res_bytes = a256(sizeof(float) * nn * st->batch);
  const size_t half_bytes = a256(sizeof(float2) * nh * st->batch);
  if (work_bytes < res_bytes + half_bytes + a256(st->work))
    return set_error(RICHM_ERR_NOMEM, "workspace %zu < %zu bytes", work_bytes,
                     res_bytes + half_bytes + a256(st->work));
  cudaStream_t s = (cudaStream_t)stream;
  float* res = reinterpret_cast<float*>(work);
  float2* half = reinterpret_cast<float2*>(reinterpret_cast<char*>(work) + res_bytes);
  void* fwork = reinterpret_cast<char*>(work) + res_bytes + half_bytes;
  for (cufftHandle h : {st->fwd, st->inv}) {
    if (cufftSetStream(h, s) != CUFFT_SUCCESS) return set_error(RICHM_ERR_CUDA, "cufftSetStream failed");
    if (cufftSetWorkArea(h, fwork) != CUFFT_SUCCESS) return set_error(RICHM_ERR_CUDA, "cufftSetWorkArea failed");
  }
  dim3 grid((n + 127) / 128, n, op->batch);
  fourier_resid_kernel<<<grid, 128, 0, s>>>(op->d_inst, n, (const float*)x, (const float*)b, res);
  RICHM_LAUNCH_CHECK("fourier residual");
  if (cufftExecR2C(st->fwd, res, (cufftComplex*)half) != CUFFT_SUCCESS)
    return set_error(RICHM_ERR_CUDA, "forward FFT failed");
  const long long tot = (long long)nh * op->batch;
  fourier_symbol_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(half, (const float2*)symbol, n, op->batch,
                                                                        (float)(1.0 / (double)nn));
  RICHM_LAUNCH_CHECK("fourier symbol");
  if (cufftExecC2R(st->inv, (cufftComplex*)half, res) != CUFFT_SUCCESS)
    return set_error(RICHM_ERR_CUDA, "inverse FFT failed");
  fourier_update_kernel<<<grid, 128, 0, s>>>(op->d_inst, n, (float*)x, res);
  RICHM_LAUNCH_CHECK("fourier update");
  return RICHM_OK;
}

}  // extern "C"
