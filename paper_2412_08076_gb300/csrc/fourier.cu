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
  // neighbours outside the grid are zero (Dirichlet) and are not read: the halo rows of
  // a buffer written by the checkpointed forward keep whatever the caller's buffer held,
  // and column -1 of the first row would lie before the buffer
  const bool west = j > 0, east = j < n - 1, north = i > 0, south = i < n - 1;
  const float xc = x[o], xw = west ? x[o - 1] : 0.f, xe = east ? x[o + 1] : 0.f;
  const float xn = north ? x[o - p] : 0.f, xs = south ? x[o + p] : 0.f;
  const float xnw = (west && north) ? x[o - p - 1] : 0.f, xne = (east && north) ? x[o - p + 1] : 0.f;
  const float xsw = (west && south) ? x[o + p - 1] : 0.f, xse = (east && south) ? x[o + p + 1] : 0.f;
  const float ax = (float)I.c * xc + (float)I.ax * (xw + xe) + (float)I.ay * (xn + xs) +
                   (float)I.d1 * (xse + xnw) + (float)I.d2 * (xne + xsw);
  res[((long long)b * n + i) * n + j] = rhs[o] - ax;
}

// half[b][k1][k2] *= (S(k1, k2) + conj(S(-k1, -k2))) / (2 n^2), k2 = 0 .. n/2 (symbol
// [n][n] shared by the batch; indices mod n); with sign_im = -1 the conjugate of that
// factor (the transpose of the correction, for the reverse mode).
__global__ void fourier_symbol_kernel(float2* __restrict__ half, const float2* __restrict__ S, int n, int batch,
                                      float scale, float sign_im) {
  const int nh = n / 2 + 1;
  const long long per = (long long)n * nh;
  const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= per * batch) return;
  const int q = (int)(k % per);
  const int k1 = q / nh, k2 = q % nh;
  const int m1 = k1 == 0 ? 0 : n - k1, m2 = k2 == 0 ? 0 : n - k2;
  const float2 s = S[(long long)k1 * n + k2];
  const float2 t = S[(long long)m1 * n + m2];
  const float sr = 0.5f * scale * (s.x + t.x), si = sign_im * 0.5f * scale * (s.y - t.y);
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

// ---------------------------------------------------------------- reverse mode
// For u' = u + Re(IFFT2(S .* FFT2(b - A u))) and g = dL/du' (real), with R and G the
// spectra of the residual and of g:
//   dL/dRe S(k) + i dL/dIm S(k) = conj(R(k)) G(k) / n^2   (summed over the batch),
//   dL/du = g - A Re(IFFT2(conj(S) .* G))                  (A symmetric).
// Both spectra are real-to-complex transforms; the symbol gradient's columns beyond n/2
// follow from conj(R(-k)) G(-k) = conj(conj(R(k)) G(k)).

// dense[b][i][j] = g(i, j) (the interior of a padded buffer).
__global__ void fourier_gather_kernel(const Inst* insts, int n, const float* __restrict__ g,
                                      float* __restrict__ dense) {
  const int b = blockIdx.z;
  const int i = blockIdx.y;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const Inst& I = insts[b];
  dense[((long long)b * n + i) * n + j] = g[I.off + (long long)(i + 1) * I.pitch + j];
}

// dS[k1][k2] = scale * sum_b conj(R_b(k)) G_b(k) over the full n x n spectrum.
__global__ void fourier_symbol_grad_kernel(const float2* __restrict__ R, const float2* __restrict__ G, int n,
                                           int batch, float scale, float2* __restrict__ dS) {
  const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= (long long)n * n) return;
  const int nh = n / 2 + 1;
  const int k1 = (int)(k / n), k2 = (int)(k % n);
  const bool mirror = k2 >= nh;
  const int q1 = mirror ? (n - k1) % n : k1, q2 = mirror ? n - k2 : k2;
  const long long per = (long long)n * nh, q = (long long)q1 * nh + q2;
  float re = 0.f, im = 0.f;
  for (int b = 0; b < batch; ++b) {
    const float2 r = R[b * per + q], gg = G[b * per + q];
    re += r.x * gg.x + r.y * gg.y;
    im += r.x * gg.y - r.y * gg.x;
  }
  dS[k] = make_float2(scale * re, (mirror ? -scale : scale) * im);
}

// gout = g - A h on the interior (h dense, zero outside the grid); gout may alias g.
__global__ void fourier_adjoint_kernel(const Inst* insts, int n, const float* g, const float* __restrict__ h,
                                       float* gout) {
  const int b = blockIdx.z;
  const int i = blockIdx.y;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const Inst& I = insts[b];
  const float* hb = h + (long long)b * n * n;
  auto hv = [&](int ii, int jj) { return (ii >= 0 && ii < n && jj >= 0 && jj < n) ? hb[ii * n + jj] : 0.f; };
  const float ax = (float)I.c * hv(i, j) + (float)I.ax * (hv(i, j - 1) + hv(i, j + 1)) +
                   (float)I.ay * (hv(i - 1, j) + hv(i + 1, j)) + (float)I.d1 * (hv(i + 1, j + 1) + hv(i - 1, j - 1)) +
                   (float)I.d2 * (hv(i - 1, j + 1) + hv(i + 1, j - 1));
  const long long o = I.off + (long long)(i + 1) * I.pitch + j;
  gout[o] = g[o] - ax;
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

richm_status richm_fourier_vjp_workspace(const richm_operator* op, size_t* bytes) {
  clear_error();
  RICHM_ARG(op && bytes, "null argument");
  FftState* st = nullptr;
  RICHM_TRY(ensure_plan(const_cast<richm_operator*>(op), &st));
  const size_t nn = (size_t)st->n * st->n, nh = (size_t)st->n * (st->n / 2 + 1);
  *bytes = 2 * a256(sizeof(float) * nn * st->batch) + 2 * a256(sizeof(float2) * nh * st->batch) + a256(st->work);
  return RICHM_OK;
}

richm_status richm_fourier_correction_vjp(richm_operator* op, richm_dtype dtype, const void* x, const void* b,
                                          const void* g, const void* symbol, void* dsymbol, void* g_x, void* work,
                                          size_t work_bytes, void* stream) {
  clear_error();
  RICHM_ARG(op != nullptr, "null operator");
  RICHM_ARG(dtype == RICHM_F32, "the Fourier correction takes RICHM_F32 state");
  RICHM_ARG(g && symbol && work, "null argument");
  RICHM_ARG(!dsymbol || (x && b), "the symbol gradient needs x and b");
  FftState* st = nullptr;
  RICHM_TRY(ensure_plan(op, &st));
  const int n = st->n;
  const size_t nn = (size_t)n * n, nh = (size_t)n * (n / 2 + 1);
  const size_t dense_bytes = a256(sizeof(float) * nn * st->batch);
  const size_t half_bytes = a256(sizeof(float2) * nh * st->batch);
  const size_t need = 2 * dense_bytes + 2 * half_bytes + a256(st->work);
  if (work_bytes < need) return set_error(RICHM_ERR_NOMEM, "workspace %zu < %zu bytes", work_bytes, need);
  cudaStream_t s = (cudaStream_t)stream;
  char* wp = reinterpret_cast<char*>(work);
  float* dres = reinterpret_cast<float*>(wp);
  float* dg = reinterpret_cast<float*>(wp + dense_bytes);
  float2* hres = reinterpret_cast<float2*>(wp + 2 * dense_bytes);
  float2* hg = reinterpret_cast<float2*>(wp + 2 * dense_bytes + half_bytes);
  void* fwork = wp + 2 * dense_bytes + 2 * half_bytes;
  for (cufftHandle h : {st->fwd, st->inv}) {
    if (cufftSetStream(h, s) != CUFFT_SUCCESS) return set_error(RICHM_ERR_CUDA, "cufftSetStream failed");
    if (cufftSetWorkArea(h, fwork) != CUFFT_SUCCESS) return set_error(RICHM_ERR_CUDA, "cufftSetWorkArea failed");
  }
  const dim3 grid((n + 127) / 128, n, op->batch);
  const float inv_nn = (float)(1.0 / (double)nn);
  fourier_gather_kernel<<<grid, 128, 0, s>>>(op->d_inst, n, (const float*)g, dg);
  RICHM_LAUNCH_CHECK("fourier gather");
  if (cufftExecR2C(st->fwd, dg, (cufftComplex*)hg) != CUFFT_SUCCESS)
    return set_error(RICHM_ERR_CUDA, "forward FFT failed");
  if (dsymbol) {
    fourier_resid_kernel<<<grid, 128, 0, s>>>(op->d_inst, n, (const float*)x, (const float*)b, dres);
    RICHM_LAUNCH_CHECK("fourier residual");
    if (cufftExecR2C(st->fwd, dres, (cufftComplex*)hres) != CUFFT_SUCCESS)
      return set_error(RICHM_ERR_CUDA, "forward FFT failed");
    fourier_symbol_grad_kernel<<<(unsigned)((nn + 255) / 256), 256, 0, s>>>(hres, hg, n, op->batch, inv_nn,
                                                                             (float2*)dsymbol);
    RICHM_LAUNCH_CHECK("fourier symbol gradient");
  }
  if (g_x) {
    const long long tot = (long long)nh * op->batch;
    fourier_symbol_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(hg, (const float2*)symbol, n, op->batch,
                                                                          inv_nn, -1.f);
    RICHM_LAUNCH_CHECK("fourier symbol");
    if (cufftExecC2R(st->inv, (cufftComplex*)hg, dg) != CUFFT_SUCCESS)
      return set_error(RICHM_ERR_CUDA, "inverse FFT failed");
    fourier_adjoint_kernel<<<grid, 128, 0, s>>>(op->d_inst, n, (const float*)g, dg, (float*)g_x);
    RICHM_LAUNCH_CHECK("fourier adjoint");
  }
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
                                                                        (float)(1.0 / (double)nn), 1.f);
  RICHM_LAUNCH_CHECK("fourier symbol");
  if (cufftExecC2R(st->inv, (cufftComplex*)half, res) != CUFFT_SUCCESS)
    return set_error(RICHM_ERR_CUDA, "inverse FFT failed");
  fourier_update_kernel<<<grid, 128, 0, s>>>(op->d_inst, n, (float*)x, res);
  RICHM_LAUNCH_CHECK("fourier update");
  return RICHM_OK;
}

}  // extern "C"
