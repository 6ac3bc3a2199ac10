// Internal definitions shared by the library's translation units.
//
// Grid layout (see include/richm.h): instance b is a block of (n_b + 2) rows of
// `pitch_b` elements at element offset off_b; interior unknown (i, j) is element
// off_b + (i + 1) * pitch_b + j. Rows 0 and n_b + 1 and columns n_b .. pitch_b - 1
// are zero. Every kernel in this library streams an instance row by row: one warp
// owns a "warp tile" of 32 lanes x VW elements (one 16-byte vector per lane) and R
// consecutive rows, and keeps a three-row window in registers so that each input
// row is loaded once per tile.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdarg>
#include <cstdint>
#include <map>
#include <string>
#include <vector>

#include "richm.h"

namespace richm {

constexpr int kRows = 16;          // rows streamed by one warp tile of the one-sweep, residual and adjoint kernels
constexpr int kWarpsPerBlock = 8;  // warp tiles per thread block of those kernels
constexpr int kFuseRows = 256;     // default output rows of a fused-sweep warp tile

// --------------------------------------------------------------- errors

richm_status set_error(richm_status s, const char* fmt, ...);
void clear_error();

#define RICHM_CUDA_TRY(call)                                                                      \
  do {                                                                                            \
    cudaError_t e_ = (call);                                                                      \
    if (e_ != cudaSuccess)                                                                        \
      return ::richm::set_error(RICHM_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

#define RICHM_LAUNCH_CHECK(what)                                                                   \
  do {                                                                                             \
    cudaError_t e_ = cudaGetLastError();                                                           \
    if (e_ != cudaSuccess)                                                                         \
      return ::richm::set_error(RICHM_ERR_CUDA, "launch of %s failed: %s", what, cudaGetErrorString(e_)); \
  } while (0)

#define RICHM_ARG(cond, ...)                                         \
  do {                                                               \
    if (!(cond)) return ::richm::set_error(RICHM_ERR_ARG, __VA_ARGS__); \
  } while (0)

#define RICHM_TRY(expr)                  \
  do {                                   \
    richm_status s_ = (expr);            \
    if (s_ != RICHM_OK) return s_;       \
  } while (0)

// --------------------------------------------------------------- descriptors

// Device descriptor of one instance (128 bytes).
struct Inst {
  long long off;  // element offset of padded row 0
  int n;          // interior size
  int pitch;      // row pitch in elements
  int kind;       // richm_problem
  int pad0;
  double c;       // centre coefficient
  double ax;      // x-neighbour (Helmholtz: the 4 neighbours)
  double ay;      // y-neighbour
  double d1;      // corners (+1,+1) and (-1,-1)
  double d2;      // corners (+1,-1) and (-1,+1)
  double abc_re;  // Helmholtz: added to the diagonal per missing neighbour
  double abc_im;
  double dinv;    // Q1: 1 / centre
  double G;       // Gershgorin bound
  long long dense_off;  // element offset of the instance in a dense concatenation (n*n each)
  double sp_im;   // sponge layer (eq. 21): imaginary diagonal term on the boundary (0: none)
  double sp_iw;   // 1 / (layer width in grid spacings)
  double pad1;
};
static_assert(sizeof(Inst) == 128, "Inst layout");

// One warp tile: instance, row block, column block.
struct Tile {
  int inst;
  int ty;
  int tx;
  int pad;
};

// A tile list for one (tile width, rows) geometry, with per-instance ranges.
struct TileMap {
  int tw = 0, rows = 0;
  int ntiles = 0;
  Tile* d_tiles = nullptr;
  int* d_inst_begin = nullptr;  // [batch + 1] tile index ranges per instance
  std::vector<int> h_inst_begin;
};

}  // namespace richm

struct richm_operator {
  int device = 0;
  int sms = 152;  // multiprocessors of the device (queried at creation)
  int batch = 0;
  std::vector<richm_pde> pdes;
  std::vector<richm::Inst> h_inst;
  richm::Inst* d_inst = nullptr;
  size_t elems = 0;
  int max_n = 0;
  std::map<long long, richm::TileMap> tiles;
  int best_fuse = 4;    // sweeps per pass used when a call asks for fuse = 0 (set by richm_autotune)
  int best_rows = 256;  // rows of a fused-sweep warp tile (set by richm_autotune)
  // cuFFT state for richm_fourier_correction (created on first use)
  void* fft_state = nullptr;
  // The session richm_solve / richm_solve_host keep for the next call with the same
  // options, weights, workspace and tuned settings: its stream, events, pinned words and
  // captured cycle graphs are reused instead of being set up again for every solve.
  richm_solver* oneshot = nullptr;
  richm_solve_opts oneshot_opts{};
  const void* oneshot_ptrs[4] = {nullptr, nullptr, nullptr, nullptr};  // w, alpha, alpha_t, work
  size_t oneshot_bytes = 0;
  int oneshot_tuned[2] = {0, 0};  // best_fuse, best_rows when it was created
};

namespace richm {

// Column tiling of the TL-sweep fused kernel for an instance of n columns: `full`
// warp-wide tiles of `width` columns (128 real, 64 complex) at stride width - 2 TL,
// and, when the rest fits, one tail tile of width / 2 columns at the same stride
// (`half` = 1). Tail tiles of two row bands of an instance share one warp (16 lanes
// each).
inline void fused_columns(int n, int TL, int* full, int* half, int width = 128) {
  const int stride = width - 2 * TL;
  const int t = 1 + (n > width ? (n - width + stride - 1) / stride : 0);
  if (t > 1 && n <= (t - 1) * stride + width / 2) {
    *full = t - 1;
    *half = 1;
  } else {
    *full = t;
    *half = 0;
  }
}

// Warps of the fused kernel for an instance of n columns and `bands` row bands.
inline long long fused_warps(int n, int TL, int bands) {
  int full = 0, half = 0;
  fused_columns(n, TL, &full, &half);
  return (long long)full * bands + (half ? (bands + 1) / 2 : 0);
}

// Tile list for tiles of `tw` elements x `rows` rows (cached in the operator);
// tw = -TL gives the overlapping 128-column tiles of the TL-sweep fused kernel
// (tw = -100 - TL: the 64-column tiles of the complex fused kernel)
// (Tile.pad = 0: a full tile; pad > 0: a pair of tail tiles at column block tx, row
// band ty in lanes 0-15 and row band pad - 2 in lanes 16-31, none if pad == 1).
richm_status get_tiles(richm_operator* op, int tw, int rows, const TileMap** out);

inline size_t dtype_size(richm_dtype t) {
  switch (t) {
    case RICHM_F64: return 8;
    case RICHM_F32: return 4;
    case RICHM_C64: return 8;
    case RICHM_C128: return 16;
    case RICHM_BF16: return 2;
  }
  return 0;
}
inline bool dtype_valid(int t) { return t >= RICHM_F64 && t <= RICHM_BF16; }
inline bool dtype_complex(richm_dtype t) { return t == RICHM_C64 || t == RICHM_C128; }

// True if every instance of the operator is of a problem kind that uses `t`.
richm_status check_dtype_for_op(const richm_operator* op, richm_dtype t);

// --------------------------------------------------------------- element types

template <typename T>
struct cplx {
  T re, im;
};

template <typename T> struct RealOf { using type = T; };
template <typename T> struct RealOf<cplx<T>> { using type = T; };
template <typename T> struct IsCplx { static constexpr bool value = false; };
template <typename T> struct IsCplx<cplx<T>> { static constexpr bool value = true; };

template <typename T> __host__ __device__ inline cplx<T> operator+(cplx<T> a, cplx<T> b) { return {a.re + b.re, a.im + b.im}; }
template <typename T> __host__ __device__ inline cplx<T> operator-(cplx<T> a, cplx<T> b) { return {a.re - b.re, a.im - b.im}; }
template <typename T> __host__ __device__ inline cplx<T> operator*(T s, cplx<T> a) { return {s * a.re, s * a.im}; }
template <typename T> __host__ __device__ inline cplx<T> cmul(cplx<T> a, cplx<T> b) {
  return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
template <typename T> __host__ __device__ inline cplx<T> cdiv(cplx<T> a, cplx<T> b) {
  T d = b.re * b.re + b.im * b.im;
  return {(a.re * b.re + a.im * b.im) / d, (a.im * b.re - a.re * b.im) / d};
}
__host__ __device__ inline float cmul(float a, float b) { return a * b; }
__host__ __device__ inline double cmul(double a, double b) { return a * b; }

template <typename E> __device__ inline E zero_e() { return E{}; }
template <> __device__ inline float zero_e<float>() { return 0.f; }
template <> __device__ inline double zero_e<double>() { return 0.0; }

// binary32 <-> binary64 conversions by moving the IEEE 754 fields with integer
// operations. GB300 runs FP64 instructions, conversions to and from FP64 included, at
// a small fraction of its FP32 rate; these keep the FP64 pipe free for arithmetic.
// Normal numbers (and zero for the widening) take the integer path, every other input
// (subnormal, infinite, NaN, and narrowing results outside the binary32 normal range)
// the hardware conversion, so both give the hardware's bits for every input.
//
// Widening is exact: exponent bias 127 -> 1023, the 23 fraction bits become the top
// of the 52.
__device__ __forceinline__ double f32_to_f64_exact(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned ex = (u >> 23) & 0xffu;
  if (ex - 1u < 254u) {
    const unsigned hi = (u & 0x80000000u) | ((ex + 896u) << 20) | ((u >> 3) & 0xfffffu);
    return __hiloint2double((int)hi, (int)(u << 29));
  }
  if ((u << 1) == 0u) return __hiloint2double((int)(u & 0x80000000u), 0);
  return (double)f;
}

// Narrowing rounds to nearest, ties to even: keep the top 23 of the 52 fraction
// bits and add one unit when the 29 dropped bits exceed half a unit, or equal it and
// the kept fraction is odd (a carry out of the fraction steps the exponent, which
// also rounds FLT_MAX + half an ulp up to infinity as IEEE 754 does).
__device__ __forceinline__ float f64_to_f32_rn(double d) {
  const unsigned hi = (unsigned)__double2hiint(d), lo = (unsigned)__double2loint(d);
  const unsigned ex = (hi >> 20) & 0x7ffu;
  if (ex - 897u < 254u) {  // binary32 exponent ex - 896 in [1, 254]
    unsigned bits = (hi & 0x80000000u) | ((ex - 896u) << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29);
    const unsigned rest = lo & 0x1fffffffu;
    bits += (rest > 0x10000000u || (rest == 0x10000000u && (bits & 1u))) ? 1u : 0u;
    return __uint_as_float(bits);
  }
  return (float)d;
}

template <typename E> __device__ inline double abs2_d(E v) { return (double)v * (double)v; }
template <> __device__ inline double abs2_d<cplx<float>>(cplx<float> v) { return (double)v.re * v.re + (double)v.im * v.im; }
template <> __device__ inline double abs2_d<cplx<double>>(cplx<double> v) { return v.re * v.re + v.im * v.im; }

// Elements per 16-byte vector.
template <typename E> struct VecWidth { static constexpr int value = 16 / sizeof(E); };

template <typename E> __device__ inline E shfl_up_e(E v, int d) { return __shfl_up_sync(0xffffffffu, v, d); }
template <typename E> __device__ inline E shfl_down_e(E v, int d) { return __shfl_down_sync(0xffffffffu, v, d); }
template <> __device__ inline cplx<float> shfl_up_e(cplx<float> v, int d) {
  return {__shfl_up_sync(0xffffffffu, v.re, d), __shfl_up_sync(0xffffffffu, v.im, d)};
}
template <> __device__ inline cplx<float> shfl_down_e(cplx<float> v, int d) {
  return {__shfl_down_sync(0xffffffffu, v.re, d), __shfl_down_sync(0xffffffffu, v.im, d)};
}
template <> __device__ inline cplx<double> shfl_up_e(cplx<double> v, int d) {
  return {__shfl_up_sync(0xffffffffu, v.re, d), __shfl_up_sync(0xffffffffu, v.im, d)};
}
template <> __device__ inline cplx<double> shfl_down_e(cplx<double> v, int d) {
  return {__shfl_down_sync(0xffffffffu, v.re, d), __shfl_down_sync(0xffffffffu, v.im, d)};
}

__device__ inline double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// A row of stencil inputs for one lane: its VW consecutive values and the two
// neighbours to the left and right of them.
template <typename E, int VW>
struct RowT {
  E y[VW];
  E yl, yr;
};

// Fill the neighbour values of a row from adjacent lanes; the warp's edge lanes
// take `left_edge` / `right_edge` (computed by the caller from a scalar load).
template <typename E, int VW>
__device__ inline void row_neighbours(RowT<E, VW>& r, int lane, E left_edge, E right_edge) {
  E l = shfl_up_e(r.y[VW - 1], 1);
  E rr = shfl_down_e(r.y[0], 1);
  r.yl = (lane == 0) ? left_edge : l;
  r.yr = (lane == 31) ? right_edge : rr;
}

// A y of the 9-point Q1 stencil at the VW points of the centre row (real E).
// U = row i-1 (y - h), C = row i, D = row i+1 (y + h); d1 couples (+1,+1)/(-1,-1),
// d2 couples (+1,-1)/(-1,+1) in (dx, dy).
template <typename E, int VW, typename S>
__device__ inline void apply_q1(const RowT<E, VW>& U, const RowT<E, VW>& C, const RowT<E, VW>& D, S c, S ax,
                                S ay, S d1, S d2, E* out) {
#pragma unroll
  for (int e = 0; e < VW; ++e) {
    E cw = (e == 0) ? C.yl : C.y[e - 1];
    E ce = (e == VW - 1) ? C.yr : C.y[e + 1];
    E uw = (e == 0) ? U.yl : U.y[e - 1];
    E ue = (e == VW - 1) ? U.yr : U.y[e + 1];
    E dw = (e == 0) ? D.yl : D.y[e - 1];
    E de = (e == VW - 1) ? D.yr : D.y[e + 1];
    out[e] = c * C.y[e] + ax * (cw + ce) + ay * (U.y[e] + D.y[e]) + d1 * (de + uw) + d2 * (ue + dw);
  }
}

// b - A y of the 9-point Q1 stencil (FP64) at the VW points of the centre row, with
// b taken into the first fused multiply-add: four sums and five multiply-adds.
template <int VW>
__device__ inline void resid_q1(const RowT<double, VW>& U, const RowT<double, VW>& C, const RowT<double, VW>& D,
                                const double* b, double c, double ax, double ay, double d1, double d2, double* out) {
#pragma unroll
  for (int e = 0; e < VW; ++e) {
    const double cw = (e == 0) ? C.yl : C.y[e - 1];
    const double ce = (e == VW - 1) ? C.yr : C.y[e + 1];
    const double uw = (e == 0) ? U.yl : U.y[e - 1];
    const double ue = (e == VW - 1) ? U.yr : U.y[e + 1];
    const double dw = (e == 0) ? D.yl : D.y[e - 1];
    const double de = (e == VW - 1) ? D.yr : D.y[e + 1];
    double t = fma(-c, C.y[e], b[e]);
    t = fma(-ax, cw + ce, t);
    t = fma(-ay, U.y[e] + D.y[e], t);
    t = fma(-d1, de + uw, t);
    out[e] = fma(-d2, ue + dw, t);
  }
}

// A y of the 5-point Helmholtz stencil (complex E) at the VW points of the centre
// row; i = interior row index, c0 = first column. The diagonal gains `abc` per
// neighbour that lies outside the domain (absorbing boundary, ghost eliminated) and,
// in a sponge layer (eq. 21), i sp_im max(0, 1 - d sp_iw) at distance d (in grid
// spacings) from the boundary.
template <typename S>
__device__ __forceinline__ S sponge_im(int i, int col, int n, S sp_im, S sp_iw) {
  const int d = min(min(i + 1, n - i), min(col + 1, n - col));
  return sp_im * max((S)0, (S)1 - (S)d * sp_iw);
}
template <typename E, int VW, typename S>
__device__ inline void apply_fd5(const RowT<E, VW>& U, const RowT<E, VW>& C, const RowT<E, VW>& D, int i, int c0,
                                 int n, S c, S off, S abc_re, S abc_im, S sp_im, S sp_iw, E* out) {
  int rmiss = (i == 0) + (i == n - 1);
#pragma unroll
  for (int e = 0; e < VW; ++e) {
    int col = c0 + e;
    int miss = rmiss + (col == 0) + (col == n - 1);
    E cw = (e == 0) ? C.yl : C.y[e - 1];
    E ce = (e == VW - 1) ? C.yr : C.y[e + 1];
    E sum = (cw + ce) + (U.y[e] + D.y[e]);
    E diag = {c + (S)miss * abc_re, (S)miss * abc_im + sponge_im<S>(i, col, n, sp_im, sp_iw)};
    out[e] = cmul(diag, C.y[e]) + off * sum;
  }
}

// Generic vector load/store of N consecutive T (N * sizeof(T) in {4, 8, 16} bytes).
template <typename T, int N>
struct alignas(N * sizeof(T)) VecN {
  T v[N];
};
template <typename T, int N>
__device__ inline VecN<T, N> ldv(const T* p) {
  VecN<T, N> r;
  if constexpr (sizeof(VecN<T, N>) == 16) {
    uint4 u = __ldg(reinterpret_cast<const uint4*>(p));
    *reinterpret_cast<uint4*>(&r) = u;
  } else if constexpr (sizeof(VecN<T, N>) == 8) {
    uint2 u = __ldg(reinterpret_cast<const uint2*>(p));
    *reinterpret_cast<uint2*>(&r) = u;
  } else {
    static_assert(sizeof(VecN<T, N>) == 4, "vector size");
    unsigned u = __ldg(reinterpret_cast<const unsigned*>(p));
    *reinterpret_cast<unsigned*>(&r) = u;
  }
  return r;
}
template <typename T, int N>
__device__ inline void stv(T* p, const VecN<T, N>& r) {
  if constexpr (sizeof(VecN<T, N>) == 32) {  // e.g. two complex128 values
    reinterpret_cast<uint4*>(p)[0] = reinterpret_cast<const uint4*>(&r)[0];
    reinterpret_cast<uint4*>(p)[1] = reinterpret_cast<const uint4*>(&r)[1];
  } else if constexpr (sizeof(VecN<T, N>) == 16) {
    *reinterpret_cast<uint4*>(p) = *reinterpret_cast<const uint4*>(&r);
  } else if constexpr (sizeof(VecN<T, N>) == 8) {
    *reinterpret_cast<uint2*>(p) = *reinterpret_cast<const uint2*>(&r);
  } else {
    static_assert(sizeof(VecN<T, N>) == 4, "vector size");
    *reinterpret_cast<unsigned*>(p) = *reinterpret_cast<const unsigned*>(&r);
  }
}

// Releases the cuFFT state of an operator (defined with the Fourier correction).
void fourier_release(richm_operator* op);

// Destroys the session richm_solve keeps between calls (defined with the solver).
void solver_release_oneshot(richm_operator* op);

}  // namespace richm
