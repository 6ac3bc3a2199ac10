// Residual norms without any device allocation (richm_residual_norm_static).
//
// Some callers cannot allocate device memory at the point where they need a
// residual: code running inside a memory pool they do not own, an allocator
// callback, or a process whose allocations are reserved up front by another
// framework. richm_residual_norm needs a caller-provided workspace for its per-tile
// partial sums; this variant keeps that scratch in file-scope device arrays instead,
// so the caller passes only inputs and outputs. The arrays live in every GPU that
// loads this library until the process exits: 1 MiB of FP64 partial sums (at most
// kMaxTiles warp tiles of 16 rows x one 16-byte vector per lane, i.e. about 134 M FP32,
// 67 M FP64 or complex64 and 33 M complex128 unknowns, less the padding of each row to
// the 32-element pitch) and 256 KiB of per-instance tile offsets (at most
// kMaxInstances instances). The entry point computes the same quantities, with the
// same kernels' arithmetic and summation order, as richm_residual_norm.
#include "common.cuh"
#include "kernels.cuh"

namespace richm {

constexpr int kMaxTiles = 65536;      // warp tiles (16 rows x 32 lanes x one 16-byte vector)
constexpr int kMaxInstances = 65536;  // instances per operator

static __device__ __align__(256) double2 g_static_partials[kMaxTiles];
static __device__ __align__(256) int g_static_tile_begin[kMaxInstances + 1];

// Device addresses of the static arrays on the current device, looked up on every call
// (a host-side query, cheap once the module is loaded): an address kept across calls
// would go stale if the context were destroyed and made again (cudaDeviceReset), and a
// kernel given a stale address would fault.
static richm_status static_scratch(double2** partials, int** begin) {
  void* p = nullptr;
  void* q = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_static_partials);
  if (e == cudaSuccess) e = cudaGetSymbolAddress(&q, g_static_tile_begin);
  if (e != cudaSuccess)
    return set_error(RICHM_ERR_CUDA, "cudaGetSymbolAddress of the static scratch failed: %s", cudaGetErrorString(e));
  *partials = reinterpret_cast<double2*>(p);
  *begin = reinterpret_cast<int*>(q);
  return RICHM_OK;
}

constexpr int kPrefixThreads = 1024;

__device__ __forceinline__ int inst_tiles(const Inst& I, int tw) {
  return ((I.pitch + tw - 1) / tw) * ((I.n + kRows - 1) / kRows);
}

// begin[b] = first warp tile of instance b for tiles of `tw` columns x kRows rows, and
// begin[batch] = the total: one block of kPrefixThreads threads, each summing a run of
// consecutive instances, then a block-wide exclusive scan of the run sums (the total
// fits an int: the host checks it against kMaxTiles before the launch).
__global__ void __launch_bounds__(kPrefixThreads) tile_prefix_kernel(const Inst* insts, int batch, int tw,
                                                                     int* begin) {
  __shared__ int warp_excl[kPrefixThreads / 32];
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int per = (batch + kPrefixThreads - 1) / kPrefixThreads;
  const int lo = min(t * per, batch), hi = min(lo + per, batch);
  int own = 0;
  for (int b = lo; b < hi; ++b) own += inst_tiles(insts[b], tw);
  int inc = own;  // inclusive scan within the warp
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int u = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += u;
  }
  if (lane == 31) warp_excl[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    const int tot = warp_excl[lane];  // kPrefixThreads / 32 == 32 warp totals
    int wi = tot;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int u = __shfl_up_sync(0xffffffffu, wi, o);
      if (lane >= o) wi += u;
    }
    warp_excl[lane] = wi - tot;
  }
  __syncthreads();
  int acc = warp_excl[warp] + inc - own;
  for (int b = lo; b < hi; ++b) {
    begin[b] = acc;
    acc += inst_tiles(insts[b], tw);
  }
  if (t == kPrefixThreads - 1) begin[batch] = acc;  // the last run ends at the batch's end
}

template <typename E> struct WideT { using type = double; };
template <> struct WideT<cplx<float>> { using type = cplx<double>; };
template <> struct WideT<cplx<double>> { using type = cplx<double>; };

template <typename ED, typename E> __device__ inline ED to_wide(E v) { return (ED)v; }
template <> __device__ inline cplx<double> to_wide<cplx<double>, cplx<float>>(cplx<float> v) {
  return {(double)v.re, (double)v.im};
}
template <> __device__ inline cplx<double> to_wide<cplx<double>, cplx<double>>(cplx<double> v) { return v; }
template <typename E, typename ED> __device__ inline E to_narrow(ED v) { return (E)v; }
template <> __device__ inline cplx<float> to_narrow<cplx<float>, cplx<double>>(cplx<double> v) {
  return {(float)v.re, (float)v.im};
}
template <> __device__ inline cplx<double> to_narrow<cplx<double>, cplx<double>>(cplx<double> v) { return v; }

// r = b - A x in FP64 over one warp tile found from the tile offsets; writes the
// tile's (sum |r|^2, sum |b|^2).
template <typename E>
__global__ void __launch_bounds__(kWarpsPerBlock * 32)
    resid_static_kernel(const Inst* insts, int batch, const int* __restrict__ begin, int ntiles,
                        const E* __restrict__ x, const E* __restrict__ b, E* __restrict__ r_out,
                        double2* __restrict__ partials) {
  using ED = typename WideT<E>::type;
  constexpr int VW = VecWidth<E>::value;
  constexpr bool CPLX = IsCplx<E>::value;
  const int lane = threadIdx.x & 31;
  const int wt = blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
  if (wt >= ntiles) return;
  int lo = 0, hi = batch - 1;  // instance with begin[inst] <= wt < begin[inst + 1]
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (begin[mid] <= wt) lo = mid;
    else hi = mid - 1;
  }
  const int inst = lo;
  const Inst& I = insts[inst];
  const int n = I.n, pitch = I.pitch;
  const int txn = (pitch + 32 * VW - 1) / (32 * VW);
  const int local = wt - begin[inst];
  const int ty = local / txn, tx = local % txn;
  const int c0 = tx * 32 * VW + lane * VW;
  const bool live = c0 < pitch;
  const int r0 = ty * kRows + 1;
  const int r1 = min(r0 + kRows - 1, n);
  const E* xb = x + I.off;
  const E* bb = b + I.off;
  E* ob = r_out ? r_out + I.off : nullptr;

  auto load = [&](int pr, RowT<ED, VW>& Y) {
    const bool in = (pr >= 1) && (pr <= n);
    VecN<E, VW> X{};
    const long long ro = (long long)pr * pitch;
    if (in && live) X = ldv<E, VW>(xb + ro + c0);
#pragma unroll
    for (int e = 0; e < VW; ++e) Y.y[e] = to_wide<ED, E>(X.v[e]);
    ED le{}, re{};
    if (in) {
      if (lane == 0 && c0 > 0) le = to_wide<ED, E>(xb[ro + c0 - 1]);
      if (lane == 31 && c0 + VW < pitch) re = to_wide<ED, E>(xb[ro + c0 + VW]);
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
      apply_fd5<ED, VW, double>(U, C, D, r - 1, c0, n, I.c, I.ax, I.abc_re, I.abc_im, I.sp_im, I.sp_iw, Ax);
    } else {
      apply_q1<ED, VW, double>(U, C, D, I.c, I.ax, I.ay, I.d1, I.d2, Ax);
    }
    VecN<E, VW> Bv{};
    if (live) Bv = ldv<E, VW>(bb + (long long)r * pitch + c0);
    VecN<E, VW> O;
#pragma unroll
    for (int e = 0; e < VW; ++e) {
      const bool ok = (c0 + e) < n;
      const ED bv = to_wide<ED, E>(Bv.v[e]);
      const ED rv = bv - Ax[e];
      if (ok) {
        sr += abs2_d(rv);
        sb += abs2_d(bv);
      }
      O.v[e] = ok ? to_narrow<E, ED>(rv) : E{};
    }
    if (ob && live) stv<E, VW>(ob + (long long)r * pitch + c0, O);
    U = C;
    C = D;
  }
  sr = warp_sum(sr);
  sb = warp_sum(sb);
  if (lane == 0) partials[wt] = make_double2(sr, sb);
}

__global__ void norm_static_kernel(const double2* __restrict__ partials, const int* __restrict__ begin, int batch,
                                   double* rnorm, double* bnorm, double* rel) {
  const int lane = threadIdx.x & 31;
  const int bi = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (bi >= batch) return;
  double sr = 0.0, sb = 0.0;
  for (int t = begin[bi] + lane; t < begin[bi + 1]; t += 32) {
    const double2 p = partials[t];
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

template <typename E>
static richm_status residual_static_t(richm_operator* op, const E* x, const E* b, double* rnorm, double* bnorm,
                                      double* rel, E* r_out, cudaStream_t s) {
  constexpr int VW = VecWidth<E>::value;
  const int tw = 32 * VW;
  long long nt = 0;
  for (int i = 0; i < op->batch; ++i) {
    const Inst& I = op->h_inst[i];
    nt += (long long)((I.pitch + tw - 1) / tw) * ((I.n + kRows - 1) / kRows);
  }
  if (nt > kMaxTiles)
    return set_error(RICHM_ERR_NOMEM,
                     "richm_residual_norm_static: the batch needs %lld warp tiles; the static scratch holds %d "
                     "(use richm_residual_norm with a workspace)",
                     nt, kMaxTiles);
  double2* partials = nullptr;
  int* begin = nullptr;
  RICHM_TRY(static_scratch(&partials, &begin));
  tile_prefix_kernel<<<1, kPrefixThreads, 0, s>>>(op->d_inst, op->batch, tw, begin);
  RICHM_LAUNCH_CHECK("tile prefix");
  const int blocks = (int)((nt + kWarpsPerBlock - 1) / kWarpsPerBlock);
  resid_static_kernel<E><<<blocks, kWarpsPerBlock * 32, 0, s>>>(op->d_inst, op->batch, begin, (int)nt, x, b, r_out,
                                                                partials);
  RICHM_LAUNCH_CHECK("static-scratch residual");
  const int wpb = 8;
  norm_static_kernel<<<(op->batch + wpb - 1) / wpb, wpb * 32, 0, s>>>(partials, begin, op->batch, rnorm, bnorm, rel);
  RICHM_LAUNCH_CHECK("static-scratch norm");
  return RICHM_OK;
}

}  // namespace richm

using namespace richm;

extern "C" {

richm_status richm_residual_norm_static(richm_operator* op, richm_dtype dtype, const void* x, const void* b,
                                        double* rnorm, double* bnorm, double* rel, void* r_out, void* stream) {
  clear_error();
  RICHM_ARG(op != nullptr, "null operator");
  RICHM_TRY(check_dtype_for_op(op, dtype));
  RICHM_ARG(x && b, "null x or b");
  if (op->batch > kMaxInstances)
    return set_error(RICHM_ERR_NOMEM, "richm_residual_norm_static: %d instances exceed the static limit of %d",
                     op->batch, kMaxInstances);
  cudaStream_t s = (cudaStream_t)stream;
  switch (dtype) {
    case RICHM_F32:
      return residual_static_t<float>(op, (const float*)x, (const float*)b, rnorm, bnorm, rel, (float*)r_out, s);
    case RICHM_F64:
      return residual_static_t<double>(op, (const double*)x, (const double*)b, rnorm, bnorm, rel, (double*)r_out, s);
    case RICHM_C64:
      return residual_static_t<cplx<float>>(op, (const cplx<float>*)x, (const cplx<float>*)b, rnorm, bnorm, rel,
                                            (cplx<float>*)r_out, s);
    case RICHM_C128:
      return residual_static_t<cplx<double>>(op, (const cplx<double>*)x, (const cplx<double>*)b, rnorm, bnorm, rel,
                                             (cplx<double>*)r_out, s);
  }
  return set_error(RICHM_ERR_ARG, "invalid dtype");
}

}  // extern "C"
