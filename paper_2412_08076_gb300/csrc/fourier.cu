// Fourier-domain correction of the FNS iteration (eqs. 19-20 with T = I):
//   x += Re( IFFT2( S .* FFT2(b - A x) ) )
// The residual is formed directly into the complex64 spectrum buffer, the 2-D
// transforms are batched cuFFT C2C calls (a library FFT), and the symbol multiply
// (with the 1/n^2 of the inverse) and the update of x are single fused passes.
#include <cufft.h>

#include <cmath>

#include "common.cuh"

namespace richm {

struct FftState {
  cufftHandle plan = 0;
  int n = 0;
  int batch = 0;
  size_t work = 0;
};

static size_t a256(size_t v) { return (v + 255) / 256 * 256; }

void fourier_release(richm_operator* op) {
  if (!op || !op->fft_state) return;
  auto* st = reinterpret_cast<FftState*>(op->fft_state);
  if (st->plan) cufftDestroy(st->plan);
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
    size_t ws = 0;
    cufftResult r = cufftCreate(&st->plan);
    if (r == CUFFT_SUCCESS) r = cufftSetAutoAllocation(st->plan, 0);
    if (r == CUFFT_SUCCESS)
      r = cufftMakePlanMany(st->plan, 2, dims, nullptr, 1, n * n, nullptr, 1, n * n, CUFFT_C2C, op->batch, &ws);
    if (r != CUFFT_SUCCESS) {
      if (st->plan) cufftDestroy(st->plan);
      delete st;
      return set_error(RICHM_ERR_CUDA, "cuFFT plan creation failed (%d)", (int)r);
    }
    st->n = n;
    st->batch = op->batch;
    st->work = ws;
    op->fft_state = st;
  }
  *out = reinterpret_cast<FftState*>(op->fft_state);
  return RICHM_OK;
}

// spec[b][i][j] = (b - A x)(i, j) + 0i, residual formed in FP64.
__global__ void fourier_resid_kernel(const Inst* insts, int n, const float* __restrict__ x,
                                     const float* __restrict__ rhs, float2* __restrict__ spec) {
  const int b = blockIdx.z;
  const int i = blockIdx.y;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const Inst& I = insts[b];
  const long long o = I.off + (long long)(i + 1) * I.pitch + j;
  const long long p = I.pitch;
  auto X = [&](long long q, int col) -> double { return (col < 0 || col >= n) ? 0.0 : (double)x[q]; };
  const double xc = X(o, j), xw = X(o - 1, j - 1), xe = X(o + 1, j + 1);
  const double xn = X(o - p, j), xs = X(o + p, j);  // rows i-1 and i+1 (halo rows are zero)
  const double xnw = X(o - p - 1, j - 1), xne = X(o - p + 1, j + 1);
  const double xsw = X(o + p - 1, j - 1), xse = X(o + p + 1, j + 1);
  const double ax = I.c * xc + I.ax * (xw + xe) + I.ay * (xn + xs) + I.d1 * (xse + xnw) + I.d2 * (xne + xsw);
  const double r = (double)rhs[o] - ax;
  spec[((long long)b * n + i) * n + j] = make_float2((float)r, 0.f);
}

// spec *= S / n^2 (symbol shared by the batch).
__global__ void fourier_symbol_kernel(float2* __restrict__ spec, const float2* __restrict__ S, long long nn,
                                      int batch, float scale) {
  const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nn * batch) return;
  const float2 s = S[k % nn];
  const float2 v = spec[k];
  spec[k] = make_float2(scale * (s.x * v.x - s.y * v.y), scale * (s.x * v.y + s.y * v.x));
}

// x += Re(spec) on the interior.
__global__ void fourier_update_kernel(const Inst* insts, int n, float* __restrict__ x,
                                      const float2* __restrict__ spec) {
  const int b = blockIdx.z;
  const int i = blockIdx.y;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const Inst& I = insts[b];
  const long long o = I.off + (long long)(i + 1) * I.pitch + j;
  x[o] += spec[((long long)b * n + i) * n + j].x;
}

}  // namespace richm

using namespace richm;

extern "C" {

richm_status richm_fourier_workspace(const richm_operator* op, size_t* bytes) {
  clear_error();
  RICHM_ARG(op && bytes, "null argument");
  FftState* st = nullptr;
  RICHM_TRY(ensure_plan(const_cast<richm_operator*>(op), &st));
  *bytes = a256(sizeof(float2) * (size_t)st->n * st->n * st->batch) + a256(st->work);
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
  const size_t spec_bytes = a256(sizeof(float2) * (size_t)st->n * st->n * st->batch);
  if (work_bytes < spec_bytes + a256(st->work))
    return set_error(RICHM_ERR_NOMEM, "workspace %zu < %zu bytes", work_bytes, spec_bytes + a256(st->work));
  cudaStream_t s = (cudaStream_t)stream;
  float2* spec = reinterpret_cast<float2*>(work);
  void* fwork = reinterpret_cast<char*>(work) + spec_bytes;
  if (cufftSetStream(st->plan, s) != CUFFT_SUCCESS) return set_error(RICHM_ERR_CUDA, "cufftSetStream failed");
  if (cufftSetWorkArea(st->plan, fwork) != CUFFT_SUCCESS) return set_error(RICHM_ERR_CUDA, "cufftSetWorkArea failed");
  const int n = st->n;
  dim3 grid((n + 127) / 128, n, op->batch);
  fourier_resid_kernel<<<grid, 128, 0, s>>>(op->d_inst, n, (const float*)x, (const float*)b, spec);
  RICHM_LAUNCH_CHECK("fourier residual");
  if (cufftExecC2C(st->plan, (cufftComplex*)spec, (cufftComplex*)spec, CUFFT_FORWARD) != CUFFT_SUCCESS)
    return set_error(RICHM_ERR_CUDA, "forward FFT failed");
  const long long nn = (long long)n * n;
  const long long tot = nn * op->batch;
  fourier_symbol_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(spec, (const float2*)symbol, nn, op->batch,
                                                                        (float)(1.0 / (double)nn));
  RICHM_LAUNCH_CHECK("fourier symbol");
  if (cufftExecC2C(st->plan, (cufftComplex*)spec, (cufftComplex*)spec, CUFFT_INVERSE) != CUFFT_SUCCESS)
    return set_error(RICHM_ERR_CUDA, "inverse FFT failed");
  fourier_update_kernel<<<grid, 128, 0, s>>>(op->d_inst, n, (float*)x, spec);
  RICHM_LAUNCH_CHECK("fourier update");
  return RICHM_OK;
}

}  // extern "C"
