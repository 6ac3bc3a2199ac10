// Fourier-domain correction of the FNS iteration (eqs. 19-20):
//   x += t .* Re( IFFT2( S .* FFT2(t .* (b - A x)) ) ),
// the correction H (b - A x), H = F T S T^H F^{-1}, for a banded transition T applied as
// the real field t on the grid (a band kernel convolving the spectrum is a pointwise
// product in space; t = 1 is T = I).
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

// res[b][i][j] = t(i, j) (b - A x)(i, j) (dense n x n per instance, FP32); t: the
// transition field [n][n] shared by the batch, or NULL for t = 1.
__global__ void fourier_resid_kernel(const Inst* insts, int n, const float* __restrict__ x,
                                     const float* __restrict__ rhs, float* __restrict__ res,
                                     const float* __restrict__ t = nullptr) {
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
  const float r = rhs[o] - ax;
  res[((long long)b * n + i) * n + j] = t ? t[(long long)i * n + j] * r : r;
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

// x += t res on the interior (t NULL: t = 1).
__global__ void fourier_update_kernel(const Inst* insts, int n, float* __restrict__ x,
                                      const float* __restrict__ res, const float* __restrict__ t = nullptr) {
  const int b = blockIdx.z;
  const int i = blockIdx.y;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const Inst& I = insts[b];
  const long long o = I.off + (long long)(i + 1) * I.pitch + j;
  const float c = res[((long long)b * n + i) * n + j];
  x[o] += t ? t[(long long)i * n + j] * c : c;
}

// ---------------------------------------------------------------- reverse mode
// For u' = u + Re(IFFT2(S .* FFT2(b - A u))) and g = dL/du' (real), with R and G the
// spectra of the residual and of g:
//   dL/dRe S(k) + i dL/dIm S(k) = conj(R(k)) G(k) / n^2   (summed over the batch),
//   dL/du = g - A Re(IFFT2(conj(S) .* G))                  (A symmetric).
// Both spectra are real-to-complex transforms; the symbol gradient's columns beyond n/2
// follow from conj(R(-k)) G(-k) = conj(conj(R(k)) G(k)).

// dense[b][i][j] = t(i, j) g(i, j) (the interior of a padded buffer; t NULL: t = 1).
__global__ void fourier_gather_kernel(const Inst* insts, int n, const float* __restrict__ g,
                                      float* __restrict__ dense, const float* __restrict__ t = nullptr) {
  const int b = blockIdx.z;
  const int i = blockIdx.y;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const Inst& I = insts[b];
  const float v = g[I.off + (long long)(i + 1) * I.pitch + j];
  dense[((long long)b * n + i) * n + j] = t ? t[(long long)i * n + j] * v : v;
}

// dt[i][j] = sum over the batch of g p + r h at (i, j), with r = b - A x recomputed,
// p = Re(IFFT2(S Q)) and h = Re(IFFT2(conj(S) G^)) dense (the transition's gradient;
// the batch is summed in a fixed order).
__global__ void fourier_transition_grad_kernel(const Inst* insts, int n, int batch, const float* __restrict__ x,
                                               const float* __restrict__ rhs, const float* __restrict__ g,
                                               const float* __restrict__ p, const float* __restrict__ h,
                                               float* __restrict__ dt) {
  const int i = blockIdx.y;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  float acc = 0.f;
  for (int b = 0; b < batch; ++b) {
    const Inst& I = insts[b];
    const long long o = I.off + (long long)(i + 1) * I.pitch + j;
    const long long pp = I.pitch;
    const bool west = j > 0, east = j < n - 1, north = i > 0, south = i < n - 1;
    const float xc = x[o], xw = west ? x[o - 1] : 0.f, xe = east ? x[o + 1] : 0.f;
    const float xn = north ? x[o - pp] : 0.f, xs = south ? x[o + pp] : 0.f;
    const float xnw = (west && north) ? x[o - pp - 1] : 0.f, xne = (east && north) ? x[o - pp + 1] : 0.f;
    const float xsw = (west && south) ? x[o + pp - 1] : 0.f, xse = (east && south) ? x[o + pp + 1] : 0.f;
    const float ax = (float)I.c * xc + (float)I.ax * (xw + xe) + (float)I.ay * (xn + xs) +
                     (float)I.d1 * (xse + xnw) + (float)I.d2 * (xne + xsw);
    const long long d = ((long long)b * n + i) * n + j;
    acc += g[o] * p[d] + (rhs[o] - ax) * h[d];
  }
  dt[(long long)i * n + j] = acc;
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

// gout = g - A (t h) on the interior (h dense, zero outside the grid; t NULL: t = 1);
// gout may alias g.
__global__ void fourier_adjoint_kernel(const Inst* insts, int n, const float* g, const float* __restrict__ h,
                                       float* gout, const float* __restrict__ t = nullptr) {
  const int b = blockIdx.z;
  const int i = blockIdx.y;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const Inst& I = insts[b];
  const float* hb = h + (long long)b * n * n;
  auto hv = [&](int ii, int jj) {
    return (ii >= 0 && ii < n && jj >= 0 && jj < n) ? (t ? t[ii * n + jj] : 1.f) * hb[ii * n + jj] : 0.f;
  };
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

richm_status richm_fourier_t_vjp_workspace(const richm_operator* op, size_t* bytes) {
  clear_error();
  RICHM_ARG(op && bytes, "null argument");
  FftState* st = nullptr;
  RICHM_TRY(ensure_plan(const_cast<richm_operator*>(op), &st));
  const size_t nn = (size_t)st->n * st->n, nh = (size_t)st->n * (st->n / 2 + 1);
  *bytes = 3 * a256(sizeof(float) * nn * st->batch) + 3 * a256(sizeof(float2) * nh * st->batch) + a256(st->work);
  return RICHM_OK;
}

static richm_status bind_work(FftState* st, void* fwork, cudaStream_t s) {
  for (cufftHandle h : {st->fwd, st->inv}) {
    if (cufftSetStream(h, s) != CUFFT_SUCCESS) return set_error(RICHM_ERR_CUDA, "cufftSetStream failed");
    if (cufftSetWorkArea(h, fwork) != CUFFT_SUCCESS) return set_error(RICHM_ERR_CUDA, "cufftSetWorkArea failed");
  }
  return RICHM_OK;
}

// Reverse mode with an optional transition field t (NULL: t = 1) and its gradient dt.
static richm_status fourier_vjp_impl(richm_operator* op, const float* x, const float* b, const float* g,
                                     const float2* symbol, const float* t, float2* dsymbol, float* dt, float* g_x,
                                     void* work, size_t work_bytes, cudaStream_t s, bool three) {
  FftState* st = nullptr;
  RICHM_TRY(ensure_plan(op, &st));
  const int n = st->n;
  const size_t nn = (size_t)n * n, nh = (size_t)n * (n / 2 + 1);
  const size_t dense_bytes = a256(sizeof(float) * nn * st->batch);
  const size_t half_bytes = a256(sizeof(float2) * nh * st->batch);
  const int nb = three ? 3 : 2;
  const size_t need = nb * dense_bytes + nb * half_bytes + a256(st->work);
  if (work_bytes < need) return set_error(RICHM_ERR_NOMEM, "workspace %zu < %zu bytes", work_bytes, need);
  char* wp = reinterpret_cast<char*>(work);
  float* dres = reinterpret_cast<float*>(wp);
  float* dg = reinterpret_cast<float*>(wp + dense_bytes);
  float* dp = three ? reinterpret_cast<float*>(wp + 2 * dense_bytes) : nullptr;
  float2* hres = reinterpret_cast<float2*>(wp + nb * dense_bytes);
  float2* hg = reinterpret_cast<float2*>(wp + nb * dense_bytes + half_bytes);
  float2* hq2 = three ? reinterpret_cast<float2*>(wp + nb * dense_bytes + 2 * half_bytes) : nullptr;
  RICHM_TRY(bind_work(st, wp + nb * dense_bytes + nb * half_bytes, s));
  const dim3 grid((n + 127) / 128, n, op->batch);
  const float inv_nn = (float)(1.0 / (double)nn);
  const long long tot = (long long)nh * op->batch;
  fourier_gather_kernel<<<grid, 128, 0, s>>>(op->d_inst, n, g, dg, t);
  RICHM_LAUNCH_CHECK("fourier gather");
  if (cufftExecR2C(st->fwd, dg, (cufftComplex*)hg) != CUFFT_SUCCESS)
    return set_error(RICHM_ERR_CUDA, "forward FFT failed");
  if (dsymbol || dt) {
    fourier_resid_kernel<<<grid, 128, 0, s>>>(op->d_inst, n, x, b, dres, t);
    RICHM_LAUNCH_CHECK("fourier residual");
    if (cufftExecR2C(st->fwd, dres, (cufftComplex*)hres) != CUFFT_SUCCESS)
      return set_error(RICHM_ERR_CUDA, "forward FFT failed");
  }
  if (dsymbol) {
    fourier_symbol_grad_kernel<<<(unsigned)((nn + 255) / 256), 256, 0, s>>>(hres, hg, n, op->batch, inv_nn, dsymbol);
    RICHM_LAUNCH_CHECK("fourier symbol gradient");
  }
  if (dt) {
    // p = Re(IFFT2(S Q)), the correction before its product with t
    RICHM_CUDA_TRY(cudaMemcpyAsync(hq2, hres, sizeof(float2) * nh * op->batch, cudaMemcpyDeviceToDevice, s));
    fourier_symbol_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(hq2, symbol, n, op->batch, inv_nn, 1.f);
    RICHM_LAUNCH_CHECK("fourier symbol");
    if (cufftExecC2R(st->inv, (cufftComplex*)hq2, dp) != CUFFT_SUCCESS)
      return set_error(RICHM_ERR_CUDA, "inverse FFT failed");
  }
  if (g_x || dt) {
    // h = Re(IFFT2(conj(S) G^)), the transpose of the correction's inner map applied to t g
    fourier_symbol_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(hg, symbol, n, op->batch, inv_nn, -1.f);
    RICHM_LAUNCH_CHECK("fourier symbol");
    if (cufftExecC2R(st->inv, (cufftComplex*)hg, dg) != CUFFT_SUCCESS)
      return set_error(RICHM_ERR_CUDA, "inverse FFT failed");
  }
  if (dt) {
    fourier_transition_grad_kernel<<<dim3((n + 127) / 128, n), 128, 0, s>>>(op->d_inst, n, op->batch, x, b, g, dp,
                                                                             dg, dt);
    RICHM_LAUNCH_CHECK("fourier transition gradient");
  }
  if (g_x) {
    fourier_adjoint_kernel<<<grid, 128, 0, s>>>(op->d_inst, n, g, dg, g_x, t);
    RICHM_LAUNCH_CHECK("fourier adjoint");
  }
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
  return fourier_vjp_impl(op, (const float*)x, (const float*)b, (const float*)g, (const float2*)symbol, nullptr,
                          (float2*)dsymbol, nullptr, (float*)g_x, work, work_bytes, (cudaStream_t)stream, false);
}

richm_status richm_fourier_correction_t_vjp(richm_operator* op, richm_dtype dtype, const void* x, const void* b,
                                            const void* g, const void* symbol, const void* transition,
                                            void* dsymbol, void* dtransition, void* g_x, void* work,
                                            size_t work_bytes, void* stream) {
  clear_error();
  RICHM_ARG(op != nullptr, "null operator");
  RICHM_ARG(dtype == RICHM_F32, "the Fourier correction takes RICHM_F32 state");
  RICHM_ARG(g && symbol && work, "null argument");
  RICHM_ARG(!(dsymbol || dtransition) || (x && b), "the parameter gradients need x and b");
  RICHM_ARG(!dtransition || transition, "the transition gradient needs the transition");
  return fourier_vjp_impl(op, (const float*)x, (const float*)b, (const float*)g, (const float2*)symbol,
                          (const float*)transition, (float2*)dsymbol, (float*)dtransition, (float*)g_x, work,
                          work_bytes, (cudaStream_t)stream, true);
}

static richm_status fourier_correction_impl(richm_operator* op, float* x, const float* b, const float2* symbol,
                                            const float* t, void* work, size_t work_bytes, cudaStream_t s) {
  FftState* st = nullptr;
  RICHM_TRY(ensure_plan(op, &st));
  const int n = st->n;
  const size_t nn = (size_t)n * n, nh = (size_t)n * (n / 2 + 1);
  const size_t res_bytes = a256(sizeof(float) * nn * st->batch);
  const size_t half_bytes = a256(sizeof(float2) * nh * st->batch);
  if (work_bytes < res_bytes + half_bytes + a256(st->work))
    return set_error(RICHM_ERR_NOMEM, "workspace %zu < %zu bytes", work_bytes,
                     res_bytes + half_bytes + a256(st->work));
  float* res = reinterpret_cast<float*>(work);
  float2* half = reinterpret_cast<float2*>(reinterpret_cast<char*>(work) + res_bytes);
  RICHM_TRY(bind_work(st, reinterpret_cast<char*>(work) + res_bytes + half_bytes, s));
  dim3 grid((n + 127) / 128, n, op->batch);
  fourier_resid_kernel<<<grid, 128, 0, s>>>(op->d_inst, n, x, b, res, t);
  RICHM_LAUNCH_CHECK("fourier residual");
  if (cufftExecR2C(st->fwd, res, (cufftComplex*)half) != CUFFT_SUCCESS)
    return set_error(RICHM_ERR_CUDA, "forward FFT failed");
  const long long tot = (long long)nh * op->batch;
  fourier_symbol_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(half, symbol, n, op->batch,
                                                                        (float)(1.0 / (double)nn), 1.f);
  RICHM_LAUNCH_CHECK("fourier symbol");
  if (cufftExecC2R(st->inv, (cufftComplex*)half, res) != CUFFT_SUCCESS)
    return set_error(RICHM_ERR_CUDA, "inverse FFT failed");
  fourier_update_kernel<<<grid, 128, 0, s>>>(op->d_inst, n, x, res, t);
  RICHM_LAUNCH_CHECK("fourier update");
  return RICHM_OK;
}

richm_status richm_fourier_correction(richm_operator* op, richm_dtype dtype, void* x, const void* b,
                                      const void* symbol, void* work, size_t work_bytes, void* stream) {
  clear_error();
  RICHM_ARG(op != nullptr, "null operator");
  RICHM_ARG(dtype == RICHM_F32, "the Fourier correction takes RICHM_F32 state");
  RICHM_ARG(x && b && symbol && work, "null argument");
  return fourier_correction_impl(op, (float*)x, (const float*)b, (const float2*)symbol, nullptr, work, work_bytes,
                                 (cudaStream_t)stream);
}

richm_status richm_fourier_correction_t(richm_operator* op, richm_dtype dtype, void* x, const void* b,
                                        const void* symbol, const void* transition, void* work, size_t work_bytes,
                                        void* stream) {
  clear_error();
  RICHM_ARG(op != nullptr, "null operator");
  RICHM_ARG(dtype == RICHM_F32, "the Fourier correction takes RICHM_F32 state");
  RICHM_ARG(x && b && symbol && work, "null argument");
  return fourier_correction_impl(op, (float*)x, (const float*)b, (const float2*)symbol, (const float*)transition,
                                 work, work_bytes, (cudaStream_t)stream);
}

}  // extern "C"
