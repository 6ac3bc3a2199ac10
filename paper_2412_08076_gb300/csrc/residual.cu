// Residual r = b - A x and its norms (eq. 15, stopping test of Sec. 2.4), and the
// log-residual training loss with its gradient (Algorithm 1's L2 loss in log form).
//
// The residual is formed in FP64 whatever the storage type, and the squared norms
// are summed in FP64: first per warp tile (written to a partials array), then per
// instance by one warp in a fixed order, so results are bitwise reproducible.
#include <cmath>
#include <type_traits>

#include "common.cuh"
#include "kernels.cuh"

namespace richm {

template <typename E> struct WideOf { using type = double; };
template <> struct WideOf<cplx<float>> { using type = cplx<double>; };
template <> struct WideOf<cplx<double>> { using type = cplx<double>; };

template <typename ED, typename E> __device__ inline ED widen(E v) { return (ED)v; }
template <> __device__ inline double widen<double, float>(float v) { return f32_to_f64_exact(v); }
template <> __device__ inline cplx<double> widen<cplx<double>, cplx<float>>(cplx<float> v) {
  return {f32_to_f64_exact(v.re), f32_to_f64_exact(v.im)};
}
template <> __device__ inline cplx<double> widen<cplx<double>, cplx<double>>(cplx<double> v) { return v; }
template <typename E, typename ED> __device__ inline E narrow(ED v) { return (E)v; }
template <> __device__ inline float narrow<float, double>(double v) { return f64_to_f32_rn(v); }
template <> __device__ inline cplx<float> narrow<cplx<float>, cplx<double>>(cplx<double> v) {
  return {f64_to_f32_rn(v.re), f64_to_f32_rn(v.im)};
}
template <> __device__ inline cplx<double> narrow<cplx<double>, cplx<double>>(cplx<double> v) { return v; }

// MODE 0: residual (+ optional r_out) and partial sums (|r|^2, |b|^2).
// MODE 1: out = scale_b * (A^H x) (the loss gradient; A^H = A for the real Q1 stencil,
//         conj(A) for the complex symmetric Helmholtz stencil), no partials.
// MODE 3: out = A x, no partials (the Krylov solver's products).
// MODE 2: the solver's refinement residual (real FP64 x and b): b folded into the
//         stencil's multiply-adds and partial sums (|r|^2, 0), since |b| is known.
template <typename E, int MODE, typename RO>
__global__ void __launch_bounds__(kWarpsPerBlock * 32)
    resid_kernel(const Inst* insts, const Tile* tiles, int ntiles, const E* __restrict__ x,
                 const E* __restrict__ b, RO* __restrict__ r_out, double2* __restrict__ partials,
                 const double* __restrict__ scale, const int* __restrict__ active) {
  using ED = typename WideOf<E>::type;
  constexpr int VW = VecWidth<E>::value;
  constexpr bool CPLX = IsCplx<E>::value;
  const int lane = threadIdx.x & 31;
  const int wt = blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
  if (wt >= ntiles) return;
  const Tile t = tiles[wt];
  if (active && active[t.inst] == 0) return;
  const Inst& I = insts[t.inst];
  const int n = I.n, pitch = I.pitch;
  const int c0 = t.tx * 32 * VW + lane * VW;
  const bool live = c0 < pitch;
  const int r0 = t.ty * kRows + 1;
  const int r1 = min(r0 + kRows - 1, n);
  const E* xb = x + I.off;
  const E* bb = (MODE == 0 || MODE == 2) ? b + I.off : nullptr;
  RO* ob = r_out ? r_out + I.off : nullptr;
  const double sc = (MODE == 1) ? scale[t.inst] : 1.0;

  auto load = [&](int pr, RowT<ED, VW>& Y) {
    const bool in = (pr >= 1) && (pr <= n);
    VecN<E, VW> X{};
    const long long ro = (long long)pr * pitch;
    if (in && live) X = ldv<E, VW>(xb + ro + c0);
#pragma unroll
    for (int e = 0; e < VW; ++e) Y.y[e] = widen<ED, E>(X.v[e]);
    ED le{}, re{};
    if (in) {
      if (lane == 0 && c0 > 0) le = widen<ED, E>(xb[ro + c0 - 1]);
      if (lane == 31 && c0 + VW < pitch) re = widen<ED, E>(xb[ro + c0 + VW]);
    }
    row_neighbours<ED, VW>(Y, lane, le, re);
  };

  double sr = 0.0, sb = 0.0;
  RowT<ED, VW> U, C, D;
  load(r0 - 1, U);
  load(r0, C);
  for (int r = r0; r <= r1; ++r) {
    load(r + 1, D);
    ED Ax[VW];
    if constexpr (CPLX) {
      const double sg = MODE == 1 ? -1.0 : 1.0;  // conj(A) for the loss gradient
      apply_fd5<ED, VW, double>(U, C, D, r - 1, c0, n, I.c, I.ax, I.abc_re, sg * I.abc_im, sg * I.sp_im, I.sp_iw, Ax);
    } else {
      apply_q1<ED, VW, double>(U, C, D, I.c, I.ax, I.ay, I.d1, I.d2, Ax);
    }
    VecN<RO, VW> O;
    if constexpr (MODE == 2) {
      static_assert(!CPLX, "the refinement residual is real");
      VecN<E, VW> Bv{};
      if (live) Bv = ldv<E, VW>(bb + (long long)r * pitch + c0);
      double rv[VW];
      resid_q1<VW>(U, C, D, Bv.v, I.c, I.ax, I.ay, I.d1, I.d2, rv);
#pragma unroll
      for (int e = 0; e < VW; ++e) {
        const bool ok = (c0 + e) < n;
        if (ok) sr = fma(rv[e], rv[e], sr);
        O.v[e] = ok ? narrow<RO, ED>(rv[e]) : RO{};
      }
    } else if (MODE == 0) {
      VecN<E, VW> Bv{};
      if (live) Bv = ldv<E, VW>(bb + (long long)r * pitch + c0);
#pragma unroll
      for (int e = 0; e < VW; ++e) {
        const bool ok = (c0 + e) < n;
        ED bv = widen<ED, E>(Bv.v[e]);
        ED rv = bv - Ax[e];
        if (ok) {
          sr += abs2_d(rv);
          sb += abs2_d(bv);
        }
        O.v[e] = ok ? narrow<RO, ED>(rv) : RO{};
      }
    } else {
#pragma unroll
      for (int e = 0; e < VW; ++e) {
        const bool ok = (c0 + e) < n;
        O.v[e] = ok ? narrow<RO, ED>(sc * Ax[e]) : RO{};
      }
    }
    if (ob && live) stv<RO, VW>(ob + (long long)r * pitch + c0, O);
    U = C;
    C = D;
  }
  if (MODE == 0 || MODE == 2) {
    sr = warp_sum(sr);
    sb = warp_sum(sb);
    if (lane == 0) partials[wt] = make_double2(sr, sb);
  }
}

__global__ void norm_reduce_kernel(const double2* __restrict__ partials, const int* __restrict__ inst_begin,
                                   int batch, double* rnorm, double* bnorm, double* rel) {
  const int lane = threadIdx.x & 31;
  const int bi = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (bi >= batch) return;
  double sr = 0.0, sb = 0.0;
  for (int t = inst_begin[bi] + lane; t < inst_begin[bi + 1]; t += 32) {
    double2 p = partials[t];
    sr += p.x;
    sb += p.y;
  }
  sr = warp_sum(sr);
  sb = warp_sum(sb);
  if (lane == 0) {
    const double rn = sqrt(sr), bn = sqrt(sb);
    if (rnorm) rnorm[bi] = rn;
    if (bnorm) bnorm[bi] = bn;
    if (rel) rel[bi] = bn > 0.0 ? rn / bn : rn;
  }
}

// loss = (1/B) sum_b ln(rnorm_b / bnorm_b); scale_b = -1 / (B rnorm_b^2).
__global__ void loss_kernel(const double* __restrict__ rnorm, const double* __restrict__ bnorm, int batch,
                            double* loss, double* scale) {
  const int lane = threadIdx.x;
  double s = 0.0;
  for (int b = lane; b < batch; b += 32) {
    s += log(rnorm[b] / bnorm[b]);
    if (scale) scale[b] = -1.0 / ((double)batch * rnorm[b] * rnorm[b]);
  }
  s = warp_sum(s);
  if (lane == 0) *loss = s / (double)batch;
}

template <typename E>
richm_status residual_tiles(richm_operator* op, int* ntiles) {
  const TileMap* tm = nullptr;
  RICHM_TRY(get_tiles(op, 32 * VecWidth<E>::value, kRows, &tm));
  *ntiles = tm->ntiles;
  return RICHM_OK;
}

template <typename E, typename RO>
richm_status launch_residual_to(richm_operator* op, const E* x, const E* b, RO* r_out, double2* partials,
                                const int* active, cudaStream_t s, bool refinement) {
  const TileMap* tm = nullptr;
  RICHM_TRY(get_tiles(op, 32 * VecWidth<E>::value, kRows, &tm));
  const int blocks = (tm->ntiles + kWarpsPerBlock - 1) / kWarpsPerBlock;
  if constexpr (std::is_same<E, double>::value) {
    if (refinement) {
      resid_kernel<E, 2, RO><<<blocks, kWarpsPerBlock * 32, 0, s>>>(op->d_inst, tm->d_tiles, tm->ntiles, x, b,
                                                                    r_out, partials, nullptr, active);
      RICHM_LAUNCH_CHECK("refinement residual");
      return RICHM_OK;
    }
  }
  resid_kernel<E, 0, RO><<<blocks, kWarpsPerBlock * 32, 0, s>>>(op->d_inst, tm->d_tiles, tm->ntiles, x, b, r_out,
                                                                partials, nullptr, active);
  RICHM_LAUNCH_CHECK("residual");
  return RICHM_OK;
}

template <typename E>
richm_status launch_residual(richm_operator* op, const E* x, const E* b, E* r_out, double2* partials,
                             cudaStream_t s) {
  return launch_residual_to<E, E>(op, x, b, r_out, partials, nullptr, s, false);
}

template richm_status launch_residual_to<double, float>(richm_operator*, const double*, const double*, float*,
                                                        double2*, const int*, cudaStream_t, bool);
template richm_status launch_residual_to<double, double>(richm_operator*, const double*, const double*, double*,
                                                         double2*, const int*, cudaStream_t, bool);
template richm_status launch_residual_to<cplx<double>, cplx<float>>(richm_operator*, const cplx<double>*,
                                                                    const cplx<double>*, cplx<float>*, double2*,
                                                                    const int*, cudaStream_t, bool);

template <typename E>
static richm_status launch_scaled_apply(richm_operator* op, const E* x, E* out, const double* scale,
                                        cudaStream_t s) {
  const TileMap* tm = nullptr;
  RICHM_TRY(get_tiles(op, 32 * VecWidth<E>::value, kRows, &tm));
  const int blocks = (tm->ntiles + kWarpsPerBlock - 1) / kWarpsPerBlock;
  resid_kernel<E, 1, E><<<blocks, kWarpsPerBlock * 32, 0, s>>>(op->d_inst, tm->d_tiles, tm->ntiles, x, nullptr,
                                                               out, nullptr, scale, nullptr);
  RICHM_LAUNCH_CHECK("scaled stencil");
  return RICHM_OK;
}

template <typename E, typename RO>
richm_status launch_apply_to(richm_operator* op, const E* x, RO* out, cudaStream_t s) {
  const TileMap* tm = nullptr;
  RICHM_TRY(get_tiles(op, 32 * VecWidth<E>::value, kRows, &tm));
  const int blocks = (tm->ntiles + kWarpsPerBlock - 1) / kWarpsPerBlock;
  resid_kernel<E, 3, RO><<<blocks, kWarpsPerBlock * 32, 0, s>>>(op->d_inst, tm->d_tiles, tm->ntiles, x, nullptr,
                                                                out, nullptr, nullptr, nullptr);
  RICHM_LAUNCH_CHECK("stencil product");
  return RICHM_OK;
}
template richm_status launch_apply_to<cplx<float>, cplx<double>>(richm_operator*, const cplx<float>*, cplx<double>*,
                                                                 cudaStream_t);
template richm_status launch_apply_to<cplx<double>, cplx<double>>(richm_operator*, const cplx<double>*,
                                                                  cplx<double>*, cudaStream_t);

richm_status launch_norm_reduce(richm_operator* op, int residual_vw, const double2* partials, double* rnorm,
                                double* bnorm, double* rel, cudaStream_t s) {
  const TileMap* tm = nullptr;
  RICHM_TRY(get_tiles(op, 32 * residual_vw, kRows, &tm));
  const int wpb = 8;
  norm_reduce_kernel<<<(op->batch + wpb - 1) / wpb, wpb * 32, 0, s>>>(partials, tm->d_inst_begin, op->batch, rnorm,
                                                                      bnorm, rel);
  RICHM_LAUNCH_CHECK("norm reduce");
  return RICHM_OK;
}

#define RICHM_INST_RESID(E)                                                                            \
  template richm_status launch_residual<E>(richm_operator*, const E*, const E*, E*, double2*, cudaStream_t); \
  template richm_status residual_tiles<E>(richm_operator*, int*);
RICHM_INST_RESID(float)
RICHM_INST_RESID(double)
RICHM_INST_RESID(cplx<float>)
RICHM_INST_RESID(cplx<double>)

static size_t align256(size_t v) { return (v + 255) / 256 * 256; }

template <typename E>
static richm_status residual_norm_t(richm_operator* op, const E* x, const E* b, double* rnorm, double* bnorm,
                                    double* rel, E* r_out, void* work, size_t work_bytes, cudaStream_t s) {
  int nt = 0;
  RICHM_TRY(residual_tiles<E>(op, &nt));
  if (work_bytes < sizeof(double2) * (size_t)nt)
    return set_error(RICHM_ERR_NOMEM, "workspace %zu < %zu bytes", work_bytes, sizeof(double2) * (size_t)nt);
  double2* partials = reinterpret_cast<double2*>(work);
  RICHM_TRY(launch_residual<E>(op, x, b, r_out, partials, s));
  return launch_norm_reduce(op, VecWidth<E>::value, partials, rnorm, bnorm, rel, s);
}

// Loss workspace: r buffer (dtype), partials, rnorm, bnorm, scale.
template <typename E>
static richm_status loss_t(richm_operator* op, const E* x, const E* b, double* loss, E* g, void* work,
                           size_t work_bytes, cudaStream_t s) {
  int nt = 0;
  RICHM_TRY(residual_tiles<E>(op, &nt));
  char* p = reinterpret_cast<char*>(work);
  E* r = reinterpret_cast<E*>(p);
  p += align256(op->elems * sizeof(E));
  double2* partials = reinterpret_cast<double2*>(p);
  p += align256(sizeof(double2) * nt);
  double* rn = reinterpret_cast<double*>(p);
  p += align256(sizeof(double) * op->batch);
  double* bn = reinterpret_cast<double*>(p);
  p += align256(sizeof(double) * op->batch);
  double* scale = reinterpret_cast<double*>(p);
  p += align256(sizeof(double) * op->batch);
  if ((size_t)(p - reinterpret_cast<char*>(work)) > work_bytes)
    return set_error(RICHM_ERR_NOMEM, "workspace too small for the loss");
  RICHM_TRY(launch_residual<E>(op, x, b, r, partials, s));
  RICHM_TRY(launch_norm_reduce(op, VecWidth<E>::value, partials, rn, bn, nullptr, s));
  loss_kernel<<<1, 32, 0, s>>>(rn, bn, op->batch, loss, scale);
  RICHM_LAUNCH_CHECK("loss");
  if (g) RICHM_TRY(launch_scaled_apply<E>(op, r, g, scale, s));
  return RICHM_OK;
}

size_t loss_workspace_bytes(richm_operator* op, size_t elem_size, int ntiles) {
  return align256(op->elems * elem_size) + align256(sizeof(double2) * ntiles) + 3 * align256(sizeof(double) * op->batch);
}

}  // namespace richm

using namespace richm;

extern "C" {

richm_status richm_residual_workspace(const richm_operator* op, size_t* bytes) {
  clear_error();
  RICHM_ARG(op && bytes, "null argument");
  // the widest tile count is that of the narrowest vector (complex128: 32 columns)
  int nt = 0;
  RICHM_TRY(residual_tiles<cplx<double>>(const_cast<richm_operator*>(op), &nt));
  *bytes = sizeof(double2) * (size_t)nt;
  return RICHM_OK;
}

richm_status richm_residual_norm(richm_operator* op, richm_dtype dtype, const void* x, const void* b,
                                 double* rnorm, double* bnorm, double* rel, void* r_out, void* work,
                                 size_t work_bytes, void* stream) {
  clear_error();
  RICHM_ARG(op != nullptr, "null operator");
  RICHM_TRY(check_dtype_for_op(op, dtype));
  RICHM_ARG(x && b, "null x or b");
  RICHM_ARG(work != nullptr, "null workspace");
  cudaStream_t s = (cudaStream_t)stream;
  switch (dtype) {
    case RICHM_F32:
      return residual_norm_t<float>(op, (const float*)x, (const float*)b, rnorm, bnorm, rel, (float*)r_out, work,
                                    work_bytes, s);
    case RICHM_F64:
      return residual_norm_t<double>(op, (const double*)x, (const double*)b, rnorm, bnorm, rel, (double*)r_out,
                                     work, work_bytes, s);
    case RICHM_C64:
      return residual_norm_t<cplx<float>>(op, (const cplx<float>*)x, (const cplx<float>*)b, rnorm, bnorm, rel,
                                          (cplx<float>*)r_out, work, work_bytes, s);
    case RICHM_C128:
      return residual_norm_t<cplx<double>>(op, (const cplx<double>*)x, (const cplx<double>*)b, rnorm, bnorm, rel,
                                           (cplx<double>*)r_out, work, work_bytes, s);
  }
  return set_error(RICHM_ERR_ARG, "invalid dtype");
}

richm_status richm_loss_log_residual(richm_operator* op, richm_dtype dtype, const void* x, const void* b,
                                     double* loss, void* g, void* work, size_t work_bytes, void* stream) {
  clear_error();
  RICHM_ARG(op != nullptr, "null operator");
  RICHM_TRY(check_dtype_for_op(op, dtype));
  RICHM_ARG(x && b && loss && work, "null argument");
  cudaStream_t s = (cudaStream_t)stream;
  switch (dtype) {
    case RICHM_F32:
      return loss_t<float>(op, (const float*)x, (const float*)b, loss, (float*)g, work, work_bytes, s);
    case RICHM_F64:
      return loss_t<double>(op, (const double*)x, (const double*)b, loss, (double*)g, work, work_bytes, s);
    case RICHM_C64:
      return loss_t<cplx<float>>(op, (const cplx<float>*)x, (const cplx<float>*)b, loss, (cplx<float>*)g, work,
                                 work_bytes, s);
    case RICHM_C128:
      return loss_t<cplx<double>>(op, (const cplx<double>*)x, (const cplx<double>*)b, loss, (cplx<double>*)g, work,
                                  work_bytes, s);
  }
  return set_error(RICHM_ERR_ARG, "invalid dtype");
}

}  // extern "C"
