// Batched solve to tolerance with FP64 iterative refinement (the evaluation loop of
// Sec. 2.3: iterate until a tolerance or a maximum number of iterations).
//
// State per instance: x (FP64, the caller's buffer), the inner correction pair
// (e_k, e_{k-1}) in the inner type, and the inner right-hand side rhs. One
// refinement cycle is
//   S sweeps of the Table 1 iteration on A e = rhs
//   update  x += e_k;  e_{k-1} <- e_{k-1} - e_k;  e_k <- 0  (FP64 add)
//   rhs = b - A x in FP64 (written in the inner type) and its squared norm
//   per-instance convergence test; converged instances leave the active set
// The update keeps the inner velocity e_k - e_{k-1} and the weight index, so the
// split is the same affine iteration as sweeping x directly.
//
// With fused sweeps (FP32 or bfloat16 state) the update costs no pass of its own:
// the refinement kernel forms x + e_k on the fly, writes it to the other of two
// FP64 buffers (the caller's x and one in the workspace, alternating by cycle) and
// takes its residual; the stored pair (e_k, e_{k-1}) is left as it is and the next
// cycle's first fused pass reads it as (0, e_{k-1} - e_k). richm_solver_finish copies
// the solution of every instance whose last cycle wrote the workspace buffer back to
// x. Otherwise (one sweep per launch, or FP64 state) a pointwise kernel applies the
// update in place before the residual.
//
// A cycle's launches depend only on the fused tile height and on the parity of the
// cycle index; each such cycle is captured once as a CUDA graph (as instances
// converge, shorter tiles keep the remaining work spread over the GPU).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <numeric>
#include <type_traits>

#include "common.cuh"
#include "kernels.cuh"

// Readbacks of the active count in flight in richm_solve's loop: the host acts on the
// count of the cycle kSolveReadDepth - 1 cycles before the newest one queued, so that a
// late host thread (a preempted wait on a shared machine) finds cycles still queued.
static constexpr int kSolveReadDepth = 4;

struct richm_solver {
  richm_operator* op = nullptr;
  richm_solve_opts o{};
  const void* w = nullptr;
  const void* a = nullptr;
  const void* at = nullptr;
  // workspace carve-up
  void* E[4] = {nullptr, nullptr, nullptr, nullptr};
  void* rhs = nullptr;
  double2* partials = nullptr;
  double* bnorm = nullptr;
  double* rel = nullptr;
  long long* sweeps = nullptr;
  int* status = nullptr;
  int* active = nullptr;
  int* count = nullptr;
  double* x2 = nullptr;  // second FP64 solution buffer (fused cycles)
  int* xloc = nullptr;   // [batch]: 1 where an instance's newest x is in x2
  // bound by richm_solver_start
  const double* b = nullptr;
  double* x = nullptr;
  // execution
  cudaStream_t s = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  std::map<int, cudaGraphExec_t> execs;  // captured cycles by fused tile height and cycle parity
  int graph_cycles = 1;      // cycles captured in one graph replay
  long long cycles_run = 0;  // cycles since start
  int* h_count = nullptr;    // pinned: [0] active count, [1 .. batch] per-instance active flags
  int* h_stage = nullptr;    // pinned: kSolveReadDepth more such records for readbacks in flight
  cudaEvent_t ev_read[kSolveReadDepth] = {};
  int rows_now = 256;        // fused tile height used by the next cycles
  int rows_max = 256;        // the operator's tuned tile height
  bool started = false;
};

namespace richm {

static size_t a256(size_t v) { return (v + 255) / 256 * 256; }

// Inner right-hand-side type: FP64 for FP64 inner sweeps, FP32 otherwise (also for
// bfloat16 state, whose arithmetic is FP32).
template <typename T> struct RhsOf { using type = float; };
template <> struct RhsOf<double> { using type = double; };

__device__ __forceinline__ double to_d(float v) { return f32_to_f64_exact(v); }
__device__ __forceinline__ double to_d(double v) { return v; }
__device__ __forceinline__ double to_d(__nv_bfloat16 v) { return f32_to_f64_exact(__bfloat162float(v)); }
__device__ __forceinline__ float to_f(float v) { return v; }
__device__ __forceinline__ double to_f(double v) { return v; }
__device__ __forceinline__ float to_f(__nv_bfloat16 v) { return __bfloat162float(v); }
template <typename T> __device__ __forceinline__ T from_f(float v) { return (T)v; }
template <> __device__ __forceinline__ __nv_bfloat16 from_f<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }
template <typename T> __device__ __forceinline__ T diff_e(T p, T e) { return p - e; }
template <> __device__ __forceinline__ __nv_bfloat16 diff_e<__nv_bfloat16>(__nv_bfloat16 p, __nv_bfloat16 e) {
  return __float2bfloat16_rn(__bfloat162float(p) - __bfloat162float(e));
}

// x += e_k; ep_out = ep - e_k; e_out = 0 (pointwise; e_out/ep_out may alias inputs).
template <typename T>
__global__ void __launch_bounds__(kWarpsPerBlock * 32)
    refine_update_kernel(const Inst* insts, const Tile* tiles, int ntiles, double* x, const T* e, const T* ep,
                         T* e_out, T* ep_out, const int* __restrict__ active) {
  const int lane = threadIdx.x & 31;
  const int wt = blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
  if (wt >= ntiles) return;
  const Tile t = tiles[wt];
  if (active && active[t.inst] == 0) return;
  const Inst& I = insts[t.inst];
  const int c0 = t.tx * 64 + lane * 2;  // two doubles per lane
  if (c0 >= I.pitch) return;
  const int r0 = t.ty * kRows + 1;
  const int r1 = min(r0 + kRows - 1, I.n);
  for (int r = r0; r <= r1; ++r) {
    const long long o = I.off + (long long)r * I.pitch + c0;
    double2 xv = *reinterpret_cast<const double2*>(x + o);
    VecN<T, 2> ev = *reinterpret_cast<const VecN<T, 2>*>(e + o);
    xv.x += to_d(ev.v[0]);
    xv.y += to_d(ev.v[1]);
    if (ep) {
      VecN<T, 2> pv = *reinterpret_cast<const VecN<T, 2>*>(ep + o);
      VecN<T, 2> np;
      np.v[0] = diff_e(pv.v[0], ev.v[0]);
      np.v[1] = diff_e(pv.v[1], ev.v[1]);
      *reinterpret_cast<VecN<T, 2>*>(ep_out + o) = np;
    }
    VecN<T, 2> nz;
    nz.v[0] = from_f<T>(0.f);
    nz.v[1] = from_f<T>(0.f);
    *reinterpret_cast<double2*>(x + o) = xv;
    *reinterpret_cast<VecN<T, 2>*>(e_out + o) = nz;
  }
}

// (s_hi, s_lo) += (hi + lo)^2 with the square of hi exact as a pair (FMA remainder),
// the cross term 2 hi lo added to the remainder, lo^2 dropped (below 2^-46 of the
// square), and the sum kept as an unevaluated pair (two-sum).
__device__ __forceinline__ void sq_acc(float hi, float lo, float& s_hi, float& s_lo) {
  const float p = hi * hi;
  const float q = fmaf(2.f * hi, lo, fmaf(hi, hi, -p));
  const float s = s_hi + p;
  const float bp = s - s_hi;
  const float err = (s_hi - (s - bp)) + (p - bp);
  s_hi = s;
  s_lo += err + q;
}

// Exponent bound: the smallest E with |v| < 2^E for a finite nonzero v (infinite and
// NaN inputs give a bound above every range used here), -4096 for zero and subnormals.
__device__ __forceinline__ int ebound_f64(double v) {
  const unsigned ex = ((unsigned)__double2hiint(v) >> 20) & 0x7ffu;
  return ex == 0u ? -4096 : (int)ex - 1022;
}

// trunc(v 2^s) as a 64-bit integer, from the fields of v (subnormal v gives 0); the
// caller guarantees |v| 2^s < 2^63.
__device__ __forceinline__ long long fixed_from_f64(double v, int s) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(v);
  const int ex = (int)((u >> 52) & 0x7ffull);
  if (ex == 0) return 0;
  const unsigned long long m = (u & 0xfffffffffffffull) | 0x10000000000000ull;
  const int sh = ex - 1075 + s;  // |v| 2^s = m 2^sh
  const unsigned long long q = sh >= 0 ? (m << sh) : (sh > -64 ? (m >> -sh) : 0ull);
  return (u >> 63) ? -(long long)q : (long long)q;
}

// acc (|acc| < 2^62) as hi + lo with hi = RN(acc) in binary32 and lo the remainder to
// within 2^-45 of |hi|, from integer operations: |acc| normalised by its leading zeros,
// the top 24 bits rounded to nearest (ties to even; a carry steps the exponent), the
// next 23 bits of the signed remainder made exact in binary32 through the 2^23 bias.
__device__ __forceinline__ void fixed_to_pair(long long acc, float& hi, float& lo) {
  const unsigned long long ua = acc < 0 ? 0ull - (unsigned long long)acc : (unsigned long long)acc;
  if (ua == 0ull) {
    hi = lo = 0.f;
    return;
  }
  const int lz = __clzll((long long)ua);  // >= 2
  const unsigned long long m = ua << lz;  // leading one at bit 63
  const unsigned top = (unsigned)(m >> 40);
  const unsigned long long rest = m & 0xffffffffffull;
  const unsigned up = (rest > 0x8000000000ull || (rest == 0x8000000000ull && (top & 1u))) ? 1u : 0u;
  const unsigned sign = acc < 0 ? 0x80000000u : 0u;
  hi = __uint_as_float((((unsigned)(63 - lz + 127) << 23) + (top - 0x800000u) + up) | sign);
  const int r23 = (int)(((long long)rest - (long long)((unsigned long long)up << 40)) >> 17);  // |r23| <= 2^22
  const float fr = __uint_as_float(0x4b000000u | (unsigned)(r23 + 0x400000)) - 12582912.f;  // 2^23 + 2^22
  const float l = fr * __uint_as_float((unsigned)(17 - lz + 127) << 23);                     // 2^(17 - lz)
  lo = sign ? -l : l;
}

// Refinement after a fused cycle: for the tile's rows, x_out = x_in + e (FP64; e is
// the cycle's final correction, read here and left in place), rhs = b - A (x_in + e)
// rounded to FP32, and the tile's partial sum (|r|^2, 0). GB300 runs FP64 arithmetic
// at about 1/70 of its FP32 rate (charged per active lane), which bound the FP64 form
// of this kernel, so the residual is formed in 64-bit fixed point on the integer
// pipes instead: one power-of-two scale per tile from the exponents of x, e, b and
// the stencil, the neighbour pairs summed exactly, the top 64 bits of each
// coefficient product, b at the same unit. That stays within a few units of 2^-57 of the tile's largest product,
// below the FP64 evaluation's rounding of the same sum; tiles whose scale falls outside
// the range the conversions allow (all-zero, extreme or non-finite values) take the
// FP64 form. On the fixed-point path |r|^2 is summed on the FP32 pipe: each residual
// as its binary32 rounding and remainder at the tile's scale, each square exact as a
// pair, the lane's sum a two-sum pair (relative error ~2^-43 over a tile's 32 terms),
// only the lanes' sums widened to FP64 and scaled back.
// (three blocks per SM: the one-row prefetch below costs a few spilled registers,
// which measured faster than two blocks per SM without spills)
template <typename T>
__global__ void __launch_bounds__(kWarpsPerBlock * 32, 3)
    refine_fused_kernel(const Inst* insts, const Tile* tiles, int ntiles, const double* __restrict__ x_in,
                        const T* __restrict__ e, const double* __restrict__ b, float* __restrict__ rhs,
                        double* __restrict__ x_out, double2* __restrict__ partials, const int* __restrict__ active,
                        int fp64_residual) {
  const int lane = threadIdx.x & 31;
  const int wt = blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
  if (wt >= ntiles) return;
  const Tile t = tiles[wt];
  if (active[t.inst] == 0) return;
  const Inst& I = insts[t.inst];
  const int n = I.n, pitch = I.pitch;
  const int c0 = t.tx * 64 + lane * 2;  // two doubles per lane
  const bool live = c0 < pitch;
  const int r0 = t.ty * kRows + 1;
  const int r1 = min(r0 + kRows - 1, n);
  const double* xb = x_in + I.off;
  const T* eb = e + I.off;
  const bool has_l = lane == 0 && c0 > 0, has_r = lane == 31 && c0 + 2 < pitch;
  const int hc = lane == 0 ? c0 - 1 : c0 + 2;

  // The tile's scale: bounds of |x|, |e| over its rows with the halo and of |b| over its
  // output rows, and of the stencil's coefficients.
  // (maxima of the magnitudes' bit patterns: their exponent fields order them)
  unsigned mx = 0u, me = 0u, mb = 0u;
  auto mag64 = [](double v) { return (unsigned)__double2hiint(v) & 0x7fffffffu; };
  auto mag_e = [](T v) { return __float_as_uint(to_f(v)) & 0x7fffffffu; };
  const int pre_hi = fp64_residual ? 0 : min(r1 + 1, n);  // no prepass for the FP64 form
#pragma unroll 6
  for (int pr = max(r0 - 1, 1); pr <= pre_hi; ++pr) {
    const long long ro = (long long)pr * pitch;
    if (live) {
      const double2 xv = *reinterpret_cast<const double2*>(xb + ro + c0);
      const VecN<T, 2> ev = *reinterpret_cast<const VecN<T, 2>*>(eb + ro + c0);
      mx = max(mx, max(mag64(xv.x), mag64(xv.y)));
      me = max(me, max(mag_e(ev.v[0]), mag_e(ev.v[1])));
      if (pr >= r0 && pr <= r1) {
        const double2 bv = *reinterpret_cast<const double2*>(b + I.off + ro + c0);
        mb = max(mb, max(mag64(bv.x), mag64(bv.y)));
      }
    }
    if (has_l || has_r) {
      mx = max(mx, mag64(xb[ro + hc]));
      me = max(me, mag_e(eb[ro + hc]));
    }
  }
  mx = __reduce_max_sync(0xffffffffu, mx);
  me = __reduce_max_sync(0xffffffffu, me);
  mb = __reduce_max_sync(0xffffffffu, mb);
  const int ey = max(mx >> 20 ? (int)(mx >> 20) - 1022 : -4096, me >> 23 ? (int)(me >> 23) - 126 : -4096);
  const int ebb = mb >> 20 ? (int)(mb >> 20) - 1022 : -4096;
  const int ea = max(max(ebound_f64(I.c), ebound_f64(I.ax)),
                     max(ebound_f64(I.ay), max(ebound_f64(I.d1), ebound_f64(I.d2))));
  // |x + e| <= 2^(ey + 1) (the FP64 sum may round up to it); |b| < 2^(ea + eyp + 4)
  const int eyp = max(ey + 1, ebb - ea - 4);
  const int k = ea + eyp - 57;  // the residual's unit is 2^k
  const bool fixed = !fp64_residual && k >= -120 && k <= 60;

  // the right-hand side and x + e of an output row
  auto emit = [&](int r, float r0v, float r1v, double x0, double x1) {
    if (live) {
      const long long o = I.off + (long long)r * pitch + c0;
      *reinterpret_cast<float2*>(rhs + o) = make_float2(c0 < n ? r0v : 0.f, c0 + 1 < n ? r1v : 0.f);
      *reinterpret_cast<double2*>(x_out + o) = make_double2(x0, x1);
    }
  };
  // x + e of a row (FP64) and of the edge lanes' outer neighbours
  auto row_sum = [&](int pr, double* y, double& h) {
    const bool in = (pr >= 1) && (pr <= n);
    const long long ro = (long long)pr * pitch;
    double2 xv = make_double2(0.0, 0.0);
    VecN<T, 2> ev;
    ev.v[0] = ev.v[1] = from_f<T>(0.f);
    if (in && live) {
      xv = *reinterpret_cast<const double2*>(xb + ro + c0);
      ev = *reinterpret_cast<const VecN<T, 2>*>(eb + ro + c0);
    }
    y[0] = xv.x + to_d(ev.v[0]);
    y[1] = xv.y + to_d(ev.v[1]);
    h = 0.0;
    if (in && has_l) h = xb[ro + hc] + to_d(eb[ro + hc]);
    if (in && has_r) h = xb[ro + hc] + to_d(eb[ro + hc]);
  };

  double sr;  // the lane's |r|^2
  if (fixed) {
    // r = b - A (x + e) in 64-bit fixed point: x + e at unit 2^(eyp - 59) (|Y| <= 2^59),
    // the coefficients at 2^(ea - 62) (|A| < 2^62), neighbour pairs summed exactly, each
    // product's top 64 bits (unit 2^k), b at 2^k; |acc| < 2^62. The error per point is
    // a few units of 2^k, below the FP64 evaluation's rounding of the same sum. |r|^2
    // is summed as (acc 2^-40)^2 (every square a normal binary32) and scaled back.
    const long long Ac = fixed_from_f64(I.c, 62 - ea), Aax = fixed_from_f64(I.ax, 62 - ea),
                    Aay = fixed_from_f64(I.ay, 62 - ea), Ad1 = fixed_from_f64(I.d1, 62 - ea),
                    Ad2 = fixed_from_f64(I.d2, 62 - ea);
    const int sy = 59 - eyp, sb = 57 - ea - eyp;
    const float scale = __uint_as_float((unsigned)(k + 127) << 23);  // 2^k
    const float down = 0x1p-40f;
    // a row's raw inputs, fetched one row step before they are used
    struct Raw {
      double2 x;
      VecN<T, 2> e;
      double hx;
      T he;
    };
    auto fetch = [&](int pr, Raw& w) {
      const bool in = (pr >= 1) && (pr <= n);
      const long long ro = (long long)pr * pitch;
      w.x = make_double2(0.0, 0.0);
      w.e.v[0] = w.e.v[1] = from_f<T>(0.f);
      w.hx = 0.0;
      w.he = from_f<T>(0.f);
      if (in && live) {
        w.x = *reinterpret_cast<const double2*>(xb + ro + c0);
        w.e = *reinterpret_cast<const VecN<T, 2>*>(eb + ro + c0);
      }
      if (in && (has_l || has_r)) {
        w.hx = xb[ro + hc];
        w.he = eb[ro + hc];
      }
    };
    auto fetch_b = [&](int r) {
      double2 bv = make_double2(0.0, 0.0);
      if (live && r <= r1) bv = *reinterpret_cast<const double2*>(b + I.off + (long long)r * pitch + c0);
      return bv;
    };
    // x + e (FP64) of a fetched row and its fixed-point form with the edge neighbours
    auto convert = [&](const Raw& w, RowT<long long, 2>& Y, double* xn) {
      xn[0] = w.x.x + to_d(w.e.v[0]);
      xn[1] = w.x.y + to_d(w.e.v[1]);
      const double h = w.hx + to_d(w.he);
      Y.y[0] = fixed_from_f64(xn[0], sy);
      Y.y[1] = fixed_from_f64(xn[1], sy);
      const long long hf = fixed_from_f64(h, sy);
      row_neighbours<long long, 2>(Y, lane, hf, hf);
    };
    float s_hi = 0.f, s_lo = 0.f;  // the lane's sum of (acc 2^-40)^2 as an unevaluated pair
    RowT<long long, 2> U, C, D;
    double xu[2], xc[2], xd[2];
    Raw w;
    fetch(r0 - 1, w);
    convert(w, U, xu);
    fetch(r0, w);
    convert(w, C, xc);
    fetch(r0 + 1, w);
    double2 bv = fetch_b(r0);
    for (int r = r0; r <= r1; ++r) {
      const Raw cur = w;
      const double2 bcur = bv;
      if (r < r1) {
        fetch(r + 2, w);
        bv = fetch_b(r + 1);
      }
      convert(cur, D, xd);
      const double bb[2] = {bcur.x, bcur.y};
      float out[2];
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const long long cw = q == 0 ? C.yl : C.y[0], ce = q == 1 ? C.yr : C.y[1];
        const long long uw = q == 0 ? U.yl : U.y[0], ue = q == 1 ? U.yr : U.y[1];
        const long long dw = q == 0 ? D.yl : D.y[0], de = q == 1 ? D.yr : D.y[1];
        long long acc = fixed_from_f64(bb[q], sb);
        acc -= __mul64hi(Ac, C.y[q]);
        acc -= __mul64hi(Aax, cw + ce);
        acc -= __mul64hi(Aay, U.y[q] + D.y[q]);
        acc -= __mul64hi(Ad1, de + uw);
        acc -= __mul64hi(Ad2, ue + dw);
        float hf, lf;
        fixed_to_pair(acc, hf, lf);
        out[q] = hf * scale;
        if (c0 + q < n) sq_acc(hf * down, lf * down, s_hi, s_lo);
      }
      emit(r, out[0], out[1], xc[0], xc[1]);
      U = C;
      C = D;
      xc[0] = xd[0];
      xc[1] = xd[1];
    }
    // (s_hi + s_lo) 2^(2k + 80) in FP64, the power of two exact
    sr = (f32_to_f64_exact(s_hi) + f32_to_f64_exact(s_lo)) * __hiloint2double((2 * k + 80 + 1023) << 20, 0);
  } else {
    // outside that range (all-zero tiles, extreme or non-finite values): FP64 arithmetic
    auto load = [&](int pr, RowT<double, 2>& Y) {
      double h;
      row_sum(pr, Y.y, h);
      row_neighbours<double, 2>(Y, lane, h, h);
    };
    sr = 0.0;
    RowT<double, 2> U, C, D;
    load(r0 - 1, U);
    load(r0, C);
    for (int r = r0; r <= r1; ++r) {
      load(r + 1, D);
      double2 bv = make_double2(0.0, 0.0);
      if (live) bv = *reinterpret_cast<const double2*>(b + I.off + (long long)r * pitch + c0);
      const double bb[2] = {bv.x, bv.y};
      double rv[2];
      resid_q1<2>(U, C, D, bb, I.c, I.ax, I.ay, I.d1, I.d2, rv);
      if (c0 < n) sr = fma(rv[0], rv[0], sr);
      if (c0 + 1 < n) sr = fma(rv[1], rv[1], sr);
      emit(r, f64_to_f32_rn(rv[0]), f64_to_f32_rn(rv[1]), C.y[0], C.y[1]);
      U = C;
      C = D;
    }
  }
  sr = warp_sum(sr);
  if (lane == 0) partials[wt] = make_double2(sr, 0.0);
}

// x <- x2 for the instances whose newest solution is in x2 (xloc[b] == 1).
__global__ void __launch_bounds__(kWarpsPerBlock * 32)
    solution_gather_kernel(const Inst* insts, const Tile* tiles, int ntiles, const double* __restrict__ x2,
                           double* __restrict__ x, const int* __restrict__ xloc) {
  const int lane = threadIdx.x & 31;
  const int wt = blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
  if (wt >= ntiles) return;
  const Tile t = tiles[wt];
  if (xloc[t.inst] == 0) return;
  const Inst& I = insts[t.inst];
  const int c0 = t.tx * 64 + lane * 2;
  if (c0 >= I.pitch) return;
  const int r0 = t.ty * kRows + 1;
  const int r1 = min(r0 + kRows - 1, I.n);
  for (int r = r0; r <= r1; ++r) {
    const long long o = I.off + (long long)r * I.pitch + c0;
    *reinterpret_cast<double2*>(x + o) = *reinterpret_cast<const double2*>(x2 + o);
  }
}

__global__ void clear_ints_kernel(int* v, int count) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < count) v[i] = 0;
}

// Per-instance convergence bookkeeping after a refinement residual; xpar >= 0 records
// where the cycle wrote the solution of the instances that took part (1: x2).
__global__ void solve_reduce_kernel(const double2* __restrict__ partials, const int* __restrict__ inst_begin,
                                    int batch, int init, int add_sweeps, double tol, long long max_sweeps,
                                    double* bnorm, double* rel, long long* sweeps, int* status, int* active,
                                    int* count, int xpar, int* xloc) {
  const int lane = threadIdx.x & 31;
  const int bi = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (bi >= batch) return;
  if (active[bi] == 0) return;
  if (lane == 0 && xpar >= 0) xloc[bi] = xpar;
  double sr = 0.0, sb = 0.0;
  for (int t = inst_begin[bi] + lane; t < inst_begin[bi + 1]; t += 32) {
    double2 p = partials[t];
    sr += p.x;
    sb += p.y;
  }
  sr = warp_sum(sr);
  sb = warp_sum(sb);
  if (lane != 0) return;
  if (init) bnorm[bi] = sqrt(sb);
  const double bn = bnorm[bi];
  const double rn = sqrt(sr);
  const double rr = bn > 0.0 ? rn / bn : rn;
  rel[bi] = rr;
  const long long sw = sweeps[bi] + add_sweeps;
  sweeps[bi] = sw;
  if (!(rr <= 1e30)) {
    status[bi] = RICHM_ERR_DIVERGED;
    active[bi] = 0;
  } else if (rr <= tol) {
    status[bi] = RICHM_OK;
    active[bi] = 0;
  } else if (sw >= max_sweeps) {
    status[bi] = RICHM_ERR_NOT_CONVERGED;
    active[bi] = 0;
  } else {
    atomicAdd(count, 1);
  }
}

// x0 = 0: the initial residual is b itself; rhs = b (inner type) and the tile's
// partial sums (|b|^2, |b|^2), without the FP64 stencil.
template <typename T>
__global__ void __launch_bounds__(kWarpsPerBlock * 32)
    zero_start_kernel(const Inst* insts, const Tile* tiles, int ntiles, const double* __restrict__ b,
                      T* __restrict__ rhs, double2* __restrict__ partials) {
  const int lane = threadIdx.x & 31;
  const int wt = blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
  if (wt >= ntiles) return;
  const Tile t = tiles[wt];
  const Inst& I = insts[t.inst];
  const int c0 = t.tx * 64 + lane * 2;  // two doubles per lane (FP64 residual geometry)
  const bool live = c0 < I.pitch;
  const int r0 = t.ty * kRows + 1;
  const int r1 = min(r0 + kRows - 1, I.n);
  double sb = 0.0;
  for (int r = r0; r <= r1 && live; ++r) {
    const long long o = I.off + (long long)r * I.pitch + c0;
    const double2 bv = *reinterpret_cast<const double2*>(b + o);
    VecN<T, 2> out;
    out.v[0] = (T)bv.x;
    out.v[1] = (T)bv.y;
    *reinterpret_cast<VecN<T, 2>*>(rhs + o) = out;
    sb += bv.x * bv.x;  // same order as the residual kernel's sum; padding columns are zero
    sb += bv.y * bv.y;
  }
  sb = warp_sum(sb);
  if (lane == 0) partials[wt] = make_double2(sb, sb);
}

__global__ void solve_init_kernel(int batch, long long* sweeps, int* status, int* active, int* xloc) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < batch) {
    sweeps[i] = 0;
    status[i] = RICHM_ERR_NOT_CONVERGED;
    active[i] = 1;
    xloc[i] = 0;
  }
}

// Fused cycles keep the solution in two FP64 buffers, alternating by cycle.
static bool fused_cycles(const richm_solver* S) {
  return S->o.fuse > 1 && (S->o.inner == RICHM_F32 || S->o.inner == RICHM_BF16);
}

// Refinement closing cycle number `cycle` (ignored for init), whose final pair is
// (E[cur], E[prv]).
template <typename T>
static richm_status refine_t(richm_solver* S, bool init, int cur = 0, int prv = 1, bool x0_zero = false,
                             long long cycle = 0) {
  using R = typename RhsOf<T>::type;
  richm_operator* op = S->op;
  const TileMap* tm = nullptr;
  RICHM_TRY(get_tiles(op, 64, kRows, &tm));  // residual / update geometry of FP64
  const int blocks = (tm->ntiles + kWarpsPerBlock - 1) / kWarpsPerBlock;
  int xpar = -1;
  if (init && x0_zero) {
    zero_start_kernel<R><<<blocks, kWarpsPerBlock * 32, 0, S->s>>>(op->d_inst, tm->d_tiles, tm->ntiles, S->b,
                                                                   (R*)S->rhs, S->partials);
    RICHM_LAUNCH_CHECK("zero start");
  }
  if constexpr (!std::is_same<T, double>::value) {
    if (!init && fused_cycles(S)) {
      xpar = (int)((cycle + 1) & 1);
      double* xin = (cycle & 1) ? S->x2 : S->x;
      double* xout = xpar ? S->x2 : S->x;
      refine_fused_kernel<T><<<blocks, kWarpsPerBlock * 32, 0, S->s>>>(op->d_inst, tm->d_tiles, tm->ntiles, xin,
                                                                        (const T*)S->E[cur], S->b, (float*)S->rhs,
                                                                        xout, S->partials, S->active,
                                                                        S->o.fp64_residual);
      RICHM_LAUNCH_CHECK("fused refinement");
    }
  }
  if (xpar < 0) {
    if (!init) {
      // pointwise, so the new pair may overwrite the buffers it reads
      refine_update_kernel<T><<<blocks, kWarpsPerBlock * 32, 0, S->s>>>(
          op->d_inst, tm->d_tiles, tm->ntiles, S->x, (const T*)S->E[cur], (const T*)S->E[prv], (T*)S->E[0],
          (T*)S->E[1], S->active);
      RICHM_LAUNCH_CHECK("refine update");
    }
    if (!(init && x0_zero))
      RICHM_TRY((launch_residual_to<double, R>(op, S->x, S->b, (R*)S->rhs, S->partials, S->active, S->s, !init)));
  }
  RICHM_CUDA_TRY(cudaMemsetAsync(S->count, 0, sizeof(int), S->s));
  const int wpb = 8;
  solve_reduce_kernel<<<(op->batch + wpb - 1) / wpb, wpb * 32, 0, S->s>>>(
      S->partials, tm->d_inst_begin, op->batch, init ? 1 : 0, init ? 0 : S->o.refine_every, S->o.tol,
      S->o.max_sweeps, S->bnorm, S->rel, S->sweeps, S->status, S->active, S->count, xpar, S->xloc);
  RICHM_LAUNCH_CHECK("solve reduce");
  return RICHM_OK;
}

// One refinement cycle starting at global sweep index k0.
// One refinement cycle (number `cycle`) starting at global sweep index k0.
template <typename T>
static richm_status cycle_t(richm_solver* S, long long k0, long long cycle) {
  const int Sw = S->o.refine_every;
  int cur = 0, prv = 1;
  if constexpr (!std::is_same<T, double>::value) {
    if (fused_cycles(S)) {
      // temporally blocked passes alternate between the pairs (E0, E1) and (E2, E3);
      // a cycle starts on the pair the previous one ended on, which its first pass
      // absorbs (see the file comment)
      const int TL = S->o.fuse;
      const long long passes = Sw / TL;
      if ((cycle * passes) & 1) cur = 2, prv = 3;
      for (int k = 0; k < Sw; k += TL) {
        const int oc = cur == 0 ? 2 : 0, op_ = cur == 0 ? 3 : 1;
        const bool absorb = k == 0;
        if constexpr (std::is_same<T, __nv_bfloat16>::value) {
          RICHM_TRY(launch_sweep_fused_bf16(S->op, TL, (const T*)S->E[cur], (const T*)S->E[prv],
                                            (const float*)S->rhs, (T*)S->E[oc], (T*)S->E[op_], (const float*)S->w,
                                            (const float*)S->a, (const float*)S->at, S->o.m,
                                            (int)((k0 + k) % S->o.m), S->o.precond, S->active, S->s, S->rows_now,
                                            absorb));
        } else {
          RICHM_TRY(launch_sweep_fused(S->op, TL, (const float*)S->E[cur], (const float*)S->E[prv],
                                       (const float*)S->rhs, (float*)S->E[oc], (float*)S->E[op_],
                                       (const float*)S->w, (const float*)S->a, (const float*)S->at, S->o.m,
                                       (int)((k0 + k) % S->o.m), S->o.precond, S->active, S->s, S->rows_now,
                                       absorb));
        }
        cur = oc;
        prv = op_;
      }
      return refine_t<T>(S, false, cur, prv, false, cycle);
    }
  }
  if constexpr (std::is_same<T, __nv_bfloat16>::value) {
    return set_error(RICHM_ERR_UNSUPPORTED, "bfloat16 inner state needs fused sweeps");
  } else {
  int fre = 2;
  for (int k = 0; k < Sw; ++k) {
    const int kidx = (int)((k0 + k) % S->o.m);
    if (S->o.precond == 2) {  // SSOR: the fourth state buffer holds the triangular solves' intermediate
      RICHM_TRY(launch_ssor_sweep<T>(S->op, (const T*)S->E[cur], S->a ? (const T*)S->E[prv] : nullptr,
                                     (const T*)S->rhs, (T*)S->E[3], (T*)S->E[fre], nullptr, (const T*)S->w,
                                     (const T*)S->a, (const T*)S->at, S->o.m, kidx, S->o.relax, S->active, S->s));
    } else {
      RICHM_TRY(launch_sweep<T>(S->op, (const T*)S->E[cur], (const T*)S->E[prv], (const T*)S->rhs,
                                (T*)S->E[fre], (const T*)S->w, (const T*)S->a, (const T*)S->at, S->o.m, kidx,
                                S->o.precond, S->active, S->s));
    }
    const int nf = prv;
    prv = cur;
    cur = fre;
    fre = nf;
  }
  return refine_t<T>(S, false, cur, prv);
  }
}

// Fused tile height (the tuned height halved down to 16 rows) for the instances
// still iterating, from a wave model of the
// fused pass: its tiles form blocks (4 one-warp tiles at 4 sweeps per pass, 2 two-warp
// tiles at 8), which run in waves of (SM count) x K resident blocks (K = 4 and 3, set by
// the registers); a wave takes rows + 2 TL row steps, and a row step takes 1 + 0.65 (k - 1) times its
// single-block time when k blocks share an SM (fitted to GB300 timings of both pass
// lengths over 1..77 instances of 511^2 and the 256-instance mix, where it picks
// within 1 % of the best height on average). Short tiles spread few instances over
// the GPU at the price of more pipeline fill; tall tiles waste nothing on fill but
// can leave most SMs idle or start a nearly empty extra wave.
static double fused_pass_cost(const richm_solver* S, int rows) {
  const richm_operator* op = S->op;
  const int TL = S->o.fuse;
  const int K = TL == 8 ? 3 : 4;           // resident blocks per SM
  const int per_block = TL == 8 ? 2 : 4;  // tiles per block
  long long warps = 0;
  int nmax = 0;
  for (int b = 0; b < op->batch; ++b) {
    if (!S->h_count[1 + b]) continue;
    const int n = op->h_inst[b].n;
    warps += fused_warps(n, TL, (n + rows - 1) / rows);
    nmax = std::max(nmax, n);
  }
  const long long blocks = (warps + per_block - 1) / per_block;
  const long long sms = op->sms;
  const long long wave = sms * K;
  const long long full = blocks / wave, rem = blocks % wave;
  const double per_wave = 1.0 + 0.65 * (K - 1);
  double cost = (double)full * per_wave;
  if (rem > 0) cost += 1.0 + 0.65 * (double)((rem + sms - 1) / sms - 1);
  const int steps = (std::min(rows, nmax) + 2 * TL + 3) / 3 * 3;
  return cost * steps;
}

static int choose_rows(const richm_solver* S) {
  int best = S->rows_max;
  double best_cost = -1.0;
  for (int rows = S->rows_max; rows >= 16; rows /= 2) {
    const double c = fused_pass_cost(S, rows);
    if (best_cost < 0.0 || c < best_cost) {
      best_cost = c;
      best = rows;
    }
  }
  return best;
}

static richm_status run_cycles(richm_solver* S, int cycles) {
  for (int c = 0; c < cycles; ++c) {
    const long long cyc = S->cycles_run + c;
    const long long k0 = cyc * (long long)S->o.refine_every;
    if (S->o.inner == RICHM_F32) RICHM_TRY(cycle_t<float>(S, k0, cyc));
    else if (S->o.inner == RICHM_BF16) RICHM_TRY(cycle_t<__nv_bfloat16>(S, k0, cyc));
    else RICHM_TRY(cycle_t<double>(S, k0, cyc));
  }
  return RICHM_OK;
}

}  // namespace richm

using namespace richm;

static richm_status launch_cycles(richm_solver* S, int cycles);
static richm_status enqueue_readback(richm_solver* S, int* rec);
static richm_status run_to_completion(richm_solver* S, long long max_cycles, cudaStream_t stream);

extern "C" {

static richm_status check_solve_opts(const richm_operator* op, const richm_solve_opts* o) {
  RICHM_ARG(op != nullptr && o != nullptr, "null operator or options");
  RICHM_ARG(o->m >= 1 && o->m <= 64, "m = %d out of range [1, 64]", o->m);
  RICHM_ARG(o->refine_every >= 1, "refine_every must be >= 1");
  RICHM_ARG(o->max_sweeps >= 0, "max_sweeps < 0");
  RICHM_ARG(o->tol >= 0.0, "tol < 0");
  RICHM_ARG(o->inner == RICHM_F32 || o->inner == RICHM_F64 || o->inner == RICHM_BF16,
            "inner dtype must be RICHM_F32, RICHM_F64 or RICHM_BF16");
  RICHM_ARG(o->precond == 0 || o->precond == 1 || o->precond == 2, "precond must be 0, 1 or 2");
  RICHM_ARG(o->fp64_residual == 0 || o->fp64_residual == 1, "fp64_residual must be 0 or 1");
  if (o->precond == 2) {
    RICHM_ARG(o->relax > 0.0 && o->relax < 2.0, "SSOR relaxation factor %g outside (0, 2)", o->relax);
    RICHM_ARG(o->fuse == 0 || o->fuse == 1, "SSOR sweeps run one per launch (fuse 0 or 1)");
    if (o->inner != RICHM_F32 && o->inner != RICHM_F64)
      return set_error(RICHM_ERR_UNSUPPORTED, "SSOR preconditioning takes an FP32 or FP64 inner state");
  }
  RICHM_ARG(o->fuse == 0 || o->fuse == 1 || o->fuse == 4 || o->fuse == 8, "fuse must be 0, 1, 4 or 8");
  RICHM_ARG(o->fuse <= 1 || (o->inner != RICHM_F64 && o->refine_every % o->fuse == 0),
            "fused sweeps need an FP32 or bfloat16 inner state and refine_every divisible by fuse");
  if (o->inner == RICHM_BF16) {
    const int f = o->fuse ? o->fuse : op->best_fuse;
    if ((f != 4 && f != 8) || o->refine_every % f != 0)
      return set_error(RICHM_ERR_UNSUPPORTED, "bfloat16 inner state needs fused sweeps (4 or 8 per pass) dividing "
                                              "refine_every");
  }
  for (int b = 0; b < op->batch; ++b)
    if (op->h_inst[b].kind != RICHM_ANISO_Q1)
      return set_error(RICHM_ERR_UNSUPPORTED, "richm_solve handles Q1 instances (instance %d is not)", b);
  return RICHM_OK;
}

richm_status richm_solve_workspace(const richm_operator* op, const richm_solve_opts* o, size_t* bytes) {
  clear_error();
  RICHM_TRY(check_solve_opts(op, o));
  RICHM_ARG(bytes != nullptr, "null output");
  const size_t es = o->inner == RICHM_F64 ? 8 : (o->inner == RICHM_F32 ? 4 : 2);  // inner state
  const size_t rs = o->inner == RICHM_F64 ? 8 : 4;                                  // inner rhs
  int nt = 0;
  RICHM_TRY(residual_tiles<double>(const_cast<richm_operator*>(op), &nt));
  size_t B = (size_t)op->batch;
  const size_t x2 = o->inner == RICHM_F64 ? 0 : a256(op->elems * sizeof(double));  // fused cycles' second x
  *bytes = 4 * a256(op->elems * es) + a256(op->elems * rs) + a256(sizeof(double2) * nt) + 2 * a256(sizeof(double) * B) +
           a256(sizeof(long long) * B) + 3 * a256(sizeof(int) * B) + a256(sizeof(int)) + x2;
  return RICHM_OK;
}

richm_status richm_solver_create(richm_operator* op, const richm_solve_opts* o, const void* w, const void* alpha,
                                 const void* alpha_t, void* work, size_t work_bytes, richm_solver** out) {
  clear_error();
  RICHM_ARG(out != nullptr, "null output handle");
  *out = nullptr;
  RICHM_TRY(check_solve_opts(op, o));
  RICHM_ARG(w != nullptr, "null weights");
  RICHM_ARG(alpha != nullptr || alpha_t == nullptr, "alpha_t given without alpha");
  size_t need = 0;
  RICHM_TRY(richm_solve_workspace(op, o, &need));
  RICHM_ARG(work != nullptr, "null workspace");
  if (work_bytes < need) return set_error(RICHM_ERR_NOMEM, "workspace %zu < %zu bytes", work_bytes, need);
  auto* S = new (std::nothrow) richm_solver();
  if (!S) return set_error(RICHM_ERR_NOMEM, "host allocation failed");
  S->op = op;
  S->o = *o;
  if (S->o.fuse == 0) {
    S->o.fuse = (o->inner != RICHM_F64 && o->precond != 2 && o->refine_every % op->best_fuse == 0) ? op->best_fuse
                                                                                                    : 1;
  }
  S->w = w;
  S->a = alpha;
  S->at = alpha_t;
  const size_t es = o->inner == RICHM_F64 ? 8 : (o->inner == RICHM_F32 ? 4 : 2);
  const size_t rs = o->inner == RICHM_F64 ? 8 : 4;
  int nt = 0;
  residual_tiles<double>(op, &nt);
  char* p = reinterpret_cast<char*>(work);
  for (int i = 0; i < 4; ++i) {
    S->E[i] = p;
    p += a256(op->elems * es);
  }
  S->rhs = p;
  p += a256(op->elems * rs);
  S->partials = reinterpret_cast<double2*>(p);
  p += a256(sizeof(double2) * nt);
  const size_t B = (size_t)op->batch;
  S->bnorm = reinterpret_cast<double*>(p);
  p += a256(sizeof(double) * B);
  S->rel = reinterpret_cast<double*>(p);
  p += a256(sizeof(double) * B);
  S->sweeps = reinterpret_cast<long long*>(p);
  p += a256(sizeof(long long) * B);
  S->status = reinterpret_cast<int*>(p);
  p += a256(sizeof(int) * B);
  S->active = reinterpret_cast<int*>(p);
  p += a256(sizeof(int) * B);
  S->xloc = reinterpret_cast<int*>(p);
  p += a256(sizeof(int) * B);
  S->count = reinterpret_cast<int*>(p);
  p += a256(sizeof(int));
  if (o->inner != RICHM_F64) S->x2 = reinterpret_cast<double*>(p);
  // the weight phase repeats every m / gcd(S, m) cycles: one graph replay covers them
  S->graph_cycles = o->m / std::gcd(o->m, o->refine_every);
  cudaError_t e = cudaStreamCreateWithFlags(&S->s, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&S->ev_in, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&S->ev_out, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaHostAlloc((void**)&S->h_count, sizeof(int) * (op->batch + 1), cudaHostAllocDefault);
  if (e == cudaSuccess)
    e = cudaHostAlloc((void**)&S->h_stage, sizeof(int) * kSolveReadDepth * (op->batch + 1), cudaHostAllocDefault);
  for (int i = 0; i < kSolveReadDepth && e == cudaSuccess; ++i)
    e = cudaEventCreateWithFlags(&S->ev_read[i], cudaEventDisableTiming);
  if (e != cudaSuccess) {
    richm_solver_destroy(S);
    return set_error(RICHM_ERR_CUDA, "solver setup failed: %s", cudaGetErrorString(e));
  }
  // warm the tile maps before any capture (they allocate on first use)
  const TileMap* tm = nullptr;
  richm_status st = get_tiles(op, 64, kRows, &tm);
  if (st == RICHM_OK) st = get_tiles(op, o->inner == RICHM_F64 ? 64 : 128, kRows, &tm);
  S->rows_max = S->rows_now = op->best_rows;
  if (S->o.fuse > 1)
    for (int rows = S->rows_max; rows >= 16 && st == RICHM_OK; rows /= 2) st = get_tiles(op, -S->o.fuse, rows, &tm);
  if (st != RICHM_OK) {
    richm_solver_destroy(S);
    return st;
  }
  *out = S;
  return RICHM_OK;
}

void richm_solver_destroy(richm_solver* S) {
  if (!S) return;
  for (auto& kv : S->execs) cudaGraphExecDestroy(kv.second);
  if (S->s) cudaStreamDestroy(S->s);
  if (S->ev_in) cudaEventDestroy(S->ev_in);
  if (S->ev_out) cudaEventDestroy(S->ev_out);
  if (S->h_count) cudaFreeHost(S->h_count);
  if (S->h_stage) cudaFreeHost(S->h_stage);
  for (cudaEvent_t ev : S->ev_read)
    if (ev) cudaEventDestroy(ev);
  delete S;
}

static richm_status solver_start_impl(richm_solver* S, const double* b, double* x, bool x0_zero, void* stream) {
  clear_error();
  RICHM_ARG(S != nullptr && b != nullptr && x != nullptr, "null argument");
  richm_operator* op = S->op;
  if (S->b != b || S->x != x) {
    for (auto& kv : S->execs) cudaGraphExecDestroy(kv.second);
    S->execs.clear();
  }
  S->b = b;
  S->x = x;
  S->cycles_run = 0;
  S->rows_now = S->rows_max;
  if (S->o.fuse > 1) {
    for (int b = 0; b < op->batch; ++b) S->h_count[1 + b] = 1;
    S->rows_now = choose_rows(S);
  }
  RICHM_CUDA_TRY(cudaEventRecord(S->ev_in, (cudaStream_t)stream));
  RICHM_CUDA_TRY(cudaStreamWaitEvent(S->s, S->ev_in, 0));
  const size_t es = S->o.inner == RICHM_F64 ? 8 : (S->o.inner == RICHM_F32 ? 4 : 2);
  RICHM_CUDA_TRY(cudaMemsetAsync(S->E[0], 0, op->elems * es, S->s));
  RICHM_CUDA_TRY(cudaMemsetAsync(S->E[1], 0, op->elems * es, S->s));
  RICHM_CUDA_TRY(cudaMemsetAsync(S->E[2], 0, op->elems * es, S->s));
  RICHM_CUDA_TRY(cudaMemsetAsync(S->E[3], 0, op->elems * es, S->s));
  solve_init_kernel<<<(op->batch + 255) / 256, 256, 0, S->s>>>(op->batch, S->sweeps, S->status, S->active,
                                                                  S->xloc);
  RICHM_LAUNCH_CHECK("solve init");
  if (fused_cycles(S)) RICHM_CUDA_TRY(cudaMemsetAsync(S->x2, 0, op->elems * sizeof(double), S->s));
  if (x0_zero) RICHM_CUDA_TRY(cudaMemsetAsync(x, 0, op->elems * sizeof(double), S->s));
  if (S->o.inner == RICHM_F32) RICHM_TRY(refine_t<float>(S, true, 0, 1, x0_zero));
  else if (S->o.inner == RICHM_BF16) RICHM_TRY(refine_t<__nv_bfloat16>(S, true, 0, 1, x0_zero));
  else RICHM_TRY(refine_t<double>(S, true, 0, 1, x0_zero));
  RICHM_CUDA_TRY(cudaEventRecord(S->ev_out, S->s));
  RICHM_CUDA_TRY(cudaStreamWaitEvent((cudaStream_t)stream, S->ev_out, 0));
  S->started = true;
  return RICHM_OK;
}

richm_status richm_solver_start(richm_solver* S, const double* b, double* x, void* stream) {
  return solver_start_impl(S, b, x, false, stream);
}

richm_status richm_solver_start_zero(richm_solver* S, const double* b, double* x, void* stream) {
  return solver_start_impl(S, b, x, true, stream);
}

richm_status richm_solver_step(richm_solver* S, int cycles, int* active_out, void* stream) {
  clear_error();
  RICHM_ARG(S != nullptr, "null solver");
  RICHM_ARG(S->started, "richm_solver_start has not been called");
  RICHM_ARG(cycles >= 0, "cycles < 0");
  RICHM_CUDA_TRY(cudaEventRecord(S->ev_in, (cudaStream_t)stream));
  RICHM_CUDA_TRY(cudaStreamWaitEvent(S->s, S->ev_in, 0));
  RICHM_TRY(launch_cycles(S, cycles));
  if (active_out) {
    RICHM_TRY(enqueue_readback(S, S->h_count));
    RICHM_CUDA_TRY(cudaStreamSynchronize(S->s));
    *active_out = *S->h_count;
    if (S->o.fuse > 1 && *active_out > 0) S->rows_now = choose_rows(S);
  }
  RICHM_CUDA_TRY(cudaEventRecord(S->ev_out, S->s));
  RICHM_CUDA_TRY(cudaStreamWaitEvent((cudaStream_t)stream, S->ev_out, 0));
  return RICHM_OK;
}

}  // extern "C"

// Queue `cycles` refinement cycles on the solver's stream (graph replays where whole
// weight periods fit, plain launches for the rest).
static richm_status launch_cycles(richm_solver* S, int cycles) {
  const int G = S->graph_cycles;
  int done = 0;
  if (S->o.use_graph) {
    // replays cover whole weight periods; a remainder runs as plain launches. The
    // graph of a replay depends on the tile height and on the parity of its first cycle.
    while (cycles - done >= G && S->cycles_run % G == 0) {
      const int key = S->rows_now * 2 + (int)(S->cycles_run & 1);
      auto it = S->execs.find(key);
      if (it == S->execs.end()) {
        cudaGraph_t g = nullptr;
        RICHM_CUDA_TRY(cudaStreamBeginCapture(S->s, cudaStreamCaptureModeThreadLocal));
        richm_status st = run_cycles(S, G);
        cudaError_t e = cudaStreamEndCapture(S->s, &g);
        if (st != RICHM_OK) {
          if (g) cudaGraphDestroy(g);
          return st;
        }
        if (e != cudaSuccess) return set_error(RICHM_ERR_CUDA, "graph capture failed: %s", cudaGetErrorString(e));
        cudaGraphExec_t ex = nullptr;
        e = cudaGraphInstantiate(&ex, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess)
          return set_error(RICHM_ERR_CUDA, "graph instantiation failed: %s", cudaGetErrorString(e));
        it = S->execs.emplace(key, ex).first;
      }
      RICHM_CUDA_TRY(cudaGraphLaunch(it->second, S->s));
      S->cycles_run += G;
      done += G;
    }
  }
  if (done < cycles) {
    RICHM_TRY(run_cycles(S, cycles - done));
    S->cycles_run += cycles - done;
  }
  return RICHM_OK;
}

// Copy the active count (and, with fused passes, the per-instance flags) into a
// pinned host record, ordered after the work queued on the solver's stream.
static richm_status enqueue_readback(richm_solver* S, int* rec) {
  RICHM_CUDA_TRY(cudaMemcpyAsync(rec, S->count, sizeof(int), cudaMemcpyDeviceToHost, S->s));
  if (S->o.fuse > 1)
    RICHM_CUDA_TRY(cudaMemcpyAsync(rec + 1, S->active, sizeof(int) * S->op->batch, cudaMemcpyDeviceToHost, S->s));
  return RICHM_OK;
}

// The loop of richm_solve: cycles until no instance is active or max_cycles ran. The
// readback of a cycle's active count is not waited for until kSolveReadDepth - 1 more
// cycles are queued behind it, so the GPU does not idle on the host round trip or on a
// late host thread; the tile height and the stopping decision use that older count (up
// to kSolveReadDepth - 1 cycles may run with every instance already converged; their
// kernels skip inactive instances).
static richm_status run_to_completion(richm_solver* S, long long max_cycles, cudaStream_t stream) {
  RICHM_CUDA_TRY(cudaEventRecord(S->ev_in, stream));
  RICHM_CUDA_TRY(cudaStreamWaitEvent(S->s, S->ev_in, 0));
  RICHM_TRY(enqueue_readback(S, S->h_count));  // after solver start
  RICHM_CUDA_TRY(cudaStreamSynchronize(S->s));
  int active = *S->h_count;
  if (S->o.fuse > 1 && active > 0) S->rows_now = choose_rows(S);
  const size_t rec = (size_t)S->op->batch + 1;
  long long c = 0, issued = 0, consumed = 0;  // cycles queued; readbacks queued and read
  while (active > 0 && c < max_cycles) {
    RICHM_TRY(launch_cycles(S, S->graph_cycles));
    c += S->graph_cycles;
    const int slot = (int)(issued % kSolveReadDepth);
    RICHM_TRY(enqueue_readback(S, S->h_stage + slot * rec));
    RICHM_CUDA_TRY(cudaEventRecord(S->ev_read[slot], S->s));
    ++issued;
    if (issued - consumed == kSolveReadDepth) {  // every slot in flight: read the oldest
      const int old = (int)(consumed % kSolveReadDepth);
      RICHM_CUDA_TRY(cudaEventSynchronize(S->ev_read[old]));
      memcpy(S->h_count, S->h_stage + old * rec, sizeof(int) * rec);
      ++consumed;
      active = *S->h_count;
      if (S->o.fuse > 1 && active > 0) S->rows_now = choose_rows(S);
    }
  }
  RICHM_CUDA_TRY(cudaStreamSynchronize(S->s));
  RICHM_CUDA_TRY(cudaEventRecord(S->ev_out, S->s));
  RICHM_CUDA_TRY(cudaStreamWaitEvent(stream, S->ev_out, 0));
  return RICHM_OK;
}

extern "C" {

richm_status richm_solver_finish(richm_solver* S, richm_solve_info* info, void* stream) {
  clear_error();
  RICHM_ARG(S != nullptr && info != nullptr, "null argument");
  const int B = S->op->batch;
  std::vector<long long> sw(B);
  std::vector<double> rel(B);
  std::vector<int> st(B);
  RICHM_CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
  if (S->started && fused_cycles(S)) {
    // solutions last written to the workspace buffer go back to x
    const TileMap* tm = nullptr;
    RICHM_TRY(get_tiles(S->op, 64, kRows, &tm));
    const int blocks = (tm->ntiles + kWarpsPerBlock - 1) / kWarpsPerBlock;
    solution_gather_kernel<<<blocks, kWarpsPerBlock * 32, 0, S->s>>>(S->op->d_inst, tm->d_tiles, tm->ntiles, S->x2,
                                                                      S->x, S->xloc);
    RICHM_LAUNCH_CHECK("solution gather");
    clear_ints_kernel<<<(B + 255) / 256, 256, 0, S->s>>>(S->xloc, B);
    RICHM_LAUNCH_CHECK("clear");
  }
  RICHM_CUDA_TRY(cudaMemcpyAsync(sw.data(), S->sweeps, sizeof(long long) * B, cudaMemcpyDeviceToHost, S->s));
  RICHM_CUDA_TRY(cudaMemcpyAsync(rel.data(), S->rel, sizeof(double) * B, cudaMemcpyDeviceToHost, S->s));
  RICHM_CUDA_TRY(cudaMemcpyAsync(st.data(), S->status, sizeof(int) * B, cudaMemcpyDeviceToHost, S->s));
  RICHM_CUDA_TRY(cudaStreamSynchronize(S->s));
  richm_status worst = RICHM_OK;
  for (int b = 0; b < B; ++b) {
    info[b].sweeps = sw[b];
    info[b].rel_res = rel[b];
    info[b].status = st[b];
    if (st[b] == RICHM_ERR_DIVERGED) worst = RICHM_ERR_DIVERGED;
    else if (st[b] != RICHM_OK && worst == RICHM_OK) worst = RICHM_ERR_NOT_CONVERGED;
  }
  return worst;
}

richm_status richm_refine(richm_operator* op, double* x, const double* b, void* e, void* e_prev, int inner,
                          void* rhs_out, double* rel, void* work, size_t work_bytes, void* stream) {
  clear_error();
  RICHM_ARG(op != nullptr, "null operator");
  RICHM_TRY(check_dtype_for_op(op, RICHM_F64));
  RICHM_ARG(x && b && rhs_out && work, "null argument");
  RICHM_ARG(inner == RICHM_F32 || inner == RICHM_F64, "inner dtype must be RICHM_F32 or RICHM_F64");
  int nt = 0;
  RICHM_TRY(residual_tiles<double>(op, &nt));
  if (work_bytes < sizeof(double2) * (size_t)nt)
    return set_error(RICHM_ERR_NOMEM, "workspace %zu < %zu bytes", work_bytes, sizeof(double2) * (size_t)nt);
  cudaStream_t s = (cudaStream_t)stream;
  const TileMap* tm = nullptr;
  RICHM_TRY(get_tiles(op, 64, kRows, &tm));
  const int blocks = (tm->ntiles + kWarpsPerBlock - 1) / kWarpsPerBlock;
  double2* partials = reinterpret_cast<double2*>(work);
  if (inner == RICHM_F32) {
    if (e) {
      refine_update_kernel<float><<<blocks, kWarpsPerBlock * 32, 0, s>>>(
          op->d_inst, tm->d_tiles, tm->ntiles, x, (const float*)e, (const float*)e_prev, (float*)e, (float*)e_prev,
          nullptr);
      RICHM_LAUNCH_CHECK("refine update");
    }
    RICHM_TRY((launch_residual_to<double, float>(op, x, b, (float*)rhs_out, partials, nullptr, s, rel == nullptr)));
  } else {
    if (e) {
      refine_update_kernel<double><<<blocks, kWarpsPerBlock * 32, 0, s>>>(
          op->d_inst, tm->d_tiles, tm->ntiles, x, (const double*)e, (const double*)e_prev, (double*)e,
          (double*)e_prev, nullptr);
      RICHM_LAUNCH_CHECK("refine update");
    }
    RICHM_TRY((launch_residual_to<double, double>(op, x, b, (double*)rhs_out, partials, nullptr, s,
                                                  rel == nullptr)));
  }
  // without rel the residual skips |b|^2 (the refinement form) and no norm is formed
  if (!rel) return RICHM_OK;
  return launch_norm_reduce(op, 2, partials, nullptr, nullptr, rel, s);
}

richm_status richm_solve_host_workspace(const richm_operator* op, const richm_solve_opts* o, size_t* bytes) {
  clear_error();
  size_t sw = 0;
  RICHM_TRY(richm_solve_workspace(op, o, &sw));
  RICHM_ARG(bytes != nullptr, "null output");
  size_t dense = 0;
  for (int b = 0; b < op->batch; ++b) dense += (size_t)op->h_inst[b].n * op->h_inst[b].n;
  *bytes = sw + 2 * a256(op->elems * sizeof(double)) + a256(dense * sizeof(double));
  return RICHM_OK;
}

}  // extern "C"

namespace richm {

void solver_release_oneshot(richm_operator* op) {
  richm_solver_destroy(op->oneshot);
  op->oneshot = nullptr;
}

// The session of a one-call solve: the operator's kept session when the options, the
// weight and workspace pointers and the tuned fused settings are those it was created
// with, else a new one (replacing it). A session is only pointers and launch plans, so
// reuse changes no arithmetic; its graphs are captured again when b or x move.
static bool same_solve_opts(const richm_solve_opts& a, const richm_solve_opts& b) {
  return a.m == b.m && a.tol == b.tol && a.max_sweeps == b.max_sweeps && a.refine_every == b.refine_every &&
         a.inner == b.inner && a.precond == b.precond && a.fuse == b.fuse && a.use_graph == b.use_graph &&
         a.relax == b.relax && a.fp64_residual == b.fp64_residual;
}

static richm_status oneshot_solver(richm_operator* op, const richm_solve_opts* o, const void* w, const void* alpha,
                                   const void* alpha_t, void* work, size_t work_bytes, richm_solver** out) {
  const void* ptrs[4] = {w, alpha, alpha_t, work};
  const int tuned[2] = {op->best_fuse, op->best_rows};
  if (op->oneshot && same_solve_opts(op->oneshot_opts, *o) && memcmp(op->oneshot_ptrs, ptrs, sizeof(ptrs)) == 0 &&
      op->oneshot_bytes == work_bytes && memcmp(op->oneshot_tuned, tuned, sizeof(tuned)) == 0) {
    *out = op->oneshot;
    return RICHM_OK;
  }
  solver_release_oneshot(op);
  RICHM_TRY(richm_solver_create(op, o, w, alpha, alpha_t, work, work_bytes, out));
  op->oneshot = *out;
  op->oneshot_opts = *o;
  memcpy(op->oneshot_ptrs, ptrs, sizeof(ptrs));
  op->oneshot_bytes = work_bytes;
  memcpy(op->oneshot_tuned, tuned, sizeof(tuned));
  return RICHM_OK;
}

// Ends a one-call solve: a session that met a CUDA or argument error is not kept.
static void oneshot_done(richm_operator* op, richm_status st) {
  if (st != RICHM_OK && st != RICHM_ERR_NOT_CONVERGED && st != RICHM_ERR_DIVERGED) solver_release_oneshot(op);
}

}  // namespace richm

extern "C" {

richm_status richm_solve_host(richm_operator* op, const double* b_host, double* x_host, const void* w,
                              const void* alpha, const void* alpha_t, const richm_solve_opts* o,
                              richm_solve_info* info, void* work, size_t work_bytes, void* stream) {
  clear_error();
  RICHM_ARG(b_host != nullptr && x_host != nullptr && info != nullptr, "null argument");
  size_t need = 0, sw = 0;
  RICHM_TRY(richm_solve_host_workspace(op, o, &need));
  RICHM_TRY(richm_solve_workspace(op, o, &sw));
  RICHM_ARG(work != nullptr, "null workspace");
  if (work_bytes < need) return set_error(RICHM_ERR_NOMEM, "workspace %zu < %zu bytes", work_bytes, need);
  size_t dense = 0;
  for (int b = 0; b < op->batch; ++b) dense += (size_t)op->h_inst[b].n * op->h_inst[b].n;
  char* p = reinterpret_cast<char*>(work) + sw;
  double* bd = reinterpret_cast<double*>(p);
  double* xd = reinterpret_cast<double*>(p + a256(op->elems * sizeof(double)));
  double* stage = reinterpret_cast<double*>(p + 2 * a256(op->elems * sizeof(double)));
  cudaStream_t s = (cudaStream_t)stream;
  RICHM_CUDA_TRY(cudaMemcpyAsync(stage, b_host, dense * sizeof(double), cudaMemcpyHostToDevice, s));
  RICHM_TRY(richm_pack(op, RICHM_F64, stage, bd, stream));
  richm_solver* S = nullptr;
  RICHM_TRY(oneshot_solver(op, o, w, alpha, alpha_t, work, sw, &S));
  richm_status st = richm_solver_start_zero(S, bd, xd, stream);
  if (st == RICHM_OK) st = run_to_completion(S, o->max_sweeps / o->refine_every + 2, s);
  if (st == RICHM_OK) st = richm_solver_finish(S, info, stream);
  oneshot_done(op, st);
  if (st != RICHM_OK && st != RICHM_ERR_NOT_CONVERGED && st != RICHM_ERR_DIVERGED) return st;
  const richm_status solve_st = st;
  RICHM_TRY(richm_unpack(op, RICHM_F64, xd, stage, stream));
  RICHM_CUDA_TRY(cudaMemcpyAsync(x_host, stage, dense * sizeof(double), cudaMemcpyDeviceToHost, s));
  RICHM_CUDA_TRY(cudaStreamSynchronize(s));
  return solve_st;
}

richm_status richm_solve(richm_operator* op, const double* b, double* x, const void* w, const void* alpha,
                         const void* alpha_t, const richm_solve_opts* o, richm_solve_info* info, void* work,
                         size_t work_bytes, void* stream) {
  clear_error();
  RICHM_ARG(info != nullptr, "null info");
  richm_solver* S = nullptr;
  RICHM_TRY(oneshot_solver(op, o, w, alpha, alpha_t, work, work_bytes, &S));
  richm_status st = richm_solver_start(S, b, x, stream);
  if (st == RICHM_OK) st = run_to_completion(S, o->max_sweeps / o->refine_every + 2, (cudaStream_t)stream);
  if (st == RICHM_OK) st = richm_solver_finish(S, info, stream);
  oneshot_done(op, st);
  return st;
}

}  // extern "C"

// ---------------------------------------------------------------- checkpoint / resume
// A solver session's state between steps, as one host byte image: a fixed header, then
// the iterate x, the second FP64 buffer (fused cycles), the four inner-state buffers,
// the inner right-hand side and the per-instance records. The header carries what a
// resumed session must share with the saved one (batch layout, options, a hash of the
// instances' stencils and of the weights) and the cycle count; the per-cycle norm
// partials are scratch and not saved. Resuming in another process continues the same
// arithmetic: the cycles that follow give the same bits as an uninterrupted session.

namespace {

struct SolverImageHeader {
  char magic[8];  // "RICHMSV1"
  unsigned version, header_bytes;
  int batch, inner, fuse, m, refine_every, precond;
  long long elems, cycles_run, max_sweeps, total_bytes;
  double tol;
  unsigned long long op_hash, weights_hash;
  int fp64_residual;
  char pad[28];
};
static_assert(sizeof(SolverImageHeader) == 128, "image header layout");

unsigned long long fnv1a(const void* p, size_t n, unsigned long long h = 1469598103934665603ull) {
  const unsigned char* c = static_cast<const unsigned char*>(p);
  for (size_t i = 0; i < n; ++i) h = (h ^ c[i]) * 1099511628211ull;
  return h;
}

unsigned long long operator_hash(const richm_operator* op) {
  unsigned long long h = fnv1a(&op->batch, sizeof(int));
  for (int b = 0; b < op->batch; ++b) {
    const Inst& I = op->h_inst[b];
    const double v[9] = {I.c, I.ax, I.ay, I.d1, I.d2, I.abc_re, I.abc_im, I.sp_im, I.sp_iw};
    const int k[3] = {I.n, I.pitch, I.kind};
    h = fnv1a(k, sizeof(k), h);
    h = fnv1a(v, sizeof(v), h);
  }
  return h;
}

richm_status weights_hash(const richm_solver* S, unsigned long long* out) {
  const size_t n = (size_t)S->op->batch * S->o.m * (S->o.inner == RICHM_F64 ? 8 : 4);
  std::vector<unsigned char> h(n);
  unsigned long long v = 1469598103934665603ull;
  for (const void* p : {S->w, S->a, S->at}) {
    const unsigned char tag = p ? 1 : 0;
    v = fnv1a(&tag, 1, v);
    if (!p) continue;
    RICHM_CUDA_TRY(cudaMemcpy(h.data(), p, n, cudaMemcpyDeviceToHost));
    v = fnv1a(h.data(), n, v);
  }
  *out = v;
  return RICHM_OK;
}

// (device pointer, bytes) of every saved part, in image order.
std::vector<std::pair<void*, size_t>> image_parts(const richm_solver* S, double* x) {
  const richm_operator* op = S->op;
  const size_t el = (size_t)op->elems, B = (size_t)op->batch;
  const size_t es = S->o.inner == RICHM_F64 ? 8 : (S->o.inner == RICHM_F32 ? 4 : 2);
  const size_t rs = S->o.inner == RICHM_F64 ? 8 : 4;
  std::vector<std::pair<void*, size_t>> v;
  v.push_back({x, el * sizeof(double)});
  if (S->x2) v.push_back({S->x2, el * sizeof(double)});
  for (int i = 0; i < 4; ++i) v.push_back({S->E[i], el * es});
  v.push_back({S->rhs, el * rs});
  v.push_back({S->bnorm, B * sizeof(double)});
  v.push_back({S->rel, B * sizeof(double)});
  v.push_back({S->sweeps, B * sizeof(long long)});
  v.push_back({S->status, B * sizeof(int)});
  v.push_back({S->active, B * sizeof(int)});
  v.push_back({S->xloc, B * sizeof(int)});
  v.push_back({S->count, sizeof(int)});
  return v;
}

size_t image_bytes(const richm_solver* S) {
  size_t n = sizeof(SolverImageHeader);
  for (const auto& p : image_parts(S, nullptr)) n += p.second;
  return n;
}

}  // namespace

extern "C" {

richm_status richm_solver_state_bytes(const richm_solver* S, size_t* bytes) {
  clear_error();
  RICHM_ARG(S != nullptr && bytes != nullptr, "null argument");
  *bytes = image_bytes(S);
  return RICHM_OK;
}

richm_status richm_solver_save(richm_solver* S, void* host, size_t bytes, void* stream) {
  clear_error();
  RICHM_ARG(S != nullptr && host != nullptr, "null argument");
  RICHM_ARG(S->started, "richm_solver_start has not been called");
  const size_t need = image_bytes(S);
  if (bytes < need) return set_error(RICHM_ERR_NOMEM, "image buffer %zu < %zu bytes", bytes, need);
  RICHM_CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
  RICHM_CUDA_TRY(cudaStreamSynchronize(S->s));
  SolverImageHeader h;
  std::memset(&h, 0, sizeof(h));
  std::memcpy(h.magic, "RICHMSV1", 8);
  h.version = 1;
  h.header_bytes = sizeof(h);
  h.batch = S->op->batch;
  h.inner = S->o.inner;
  h.fuse = S->o.fuse;
  h.m = S->o.m;
  h.refine_every = S->o.refine_every;
  h.precond = S->o.precond;
  h.fp64_residual = S->o.fp64_residual;
  h.elems = S->op->elems;
  h.cycles_run = S->cycles_run;
  h.max_sweeps = S->o.max_sweeps;
  h.total_bytes = (long long)need;
  h.tol = S->o.tol;
  h.op_hash = operator_hash(S->op);
  RICHM_TRY(weights_hash(S, &h.weights_hash));
  unsigned char* p = static_cast<unsigned char*>(host);
  std::memcpy(p, &h, sizeof(h));
  p += sizeof(h);
  for (const auto& part : image_parts(S, S->x)) {
    RICHM_CUDA_TRY(cudaMemcpy(p, part.first, part.second, cudaMemcpyDeviceToHost));
    p += part.second;
  }
  return RICHM_OK;
}

richm_status richm_solver_resume(richm_solver* S, const double* b, double* x, const void* host, size_t bytes,
                                 void* stream) {
  clear_error();
  RICHM_ARG(S != nullptr && b != nullptr && x != nullptr && host != nullptr, "null argument");
  RICHM_ARG(bytes >= sizeof(SolverImageHeader), "image of %zu bytes is shorter than its header", bytes);
  SolverImageHeader h;
  std::memcpy(&h, host, sizeof(h));
  RICHM_ARG(std::memcmp(h.magic, "RICHMSV1", 8) == 0 && h.version == 1 && h.header_bytes == sizeof(h),
            "not a solver image of this version");
  const size_t need = image_bytes(S);
  RICHM_ARG(h.total_bytes == (long long)need && bytes >= need, "image of %lld bytes, this session needs %zu",
            h.total_bytes, need);
  RICHM_ARG(h.batch == S->op->batch && h.elems == S->op->elems && h.op_hash == operator_hash(S->op),
            "the image was saved for other instances");
  RICHM_ARG(h.inner == S->o.inner && h.fuse == S->o.fuse && h.m == S->o.m && h.refine_every == S->o.refine_every &&
                h.precond == S->o.precond && h.tol == S->o.tol && h.max_sweeps == S->o.max_sweeps &&
                h.fp64_residual == S->o.fp64_residual,
            "the image was saved with other solve options (inner %d, fuse %d, m %d, refine_every %d)", h.inner,
            h.fuse, h.m, h.refine_every);
  unsigned long long wh = 0;
  RICHM_TRY(weights_hash(S, &wh));
  RICHM_ARG(wh == h.weights_hash, "the image was saved with other weights");
  RICHM_CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
  RICHM_CUDA_TRY(cudaStreamSynchronize(S->s));
  if (S->b != b || S->x != x) {
    for (auto& kv : S->execs) cudaGraphExecDestroy(kv.second);
    S->execs.clear();
  }
  S->b = b;
  S->x = x;
  const unsigned char* p = static_cast<const unsigned char*>(host) + sizeof(h);
  for (const auto& part : image_parts(S, x)) {
    RICHM_CUDA_TRY(cudaMemcpy(part.first, p, part.second, cudaMemcpyHostToDevice));
    p += part.second;
  }
  S->cycles_run = h.cycles_run;
  S->rows_now = S->rows_max;
  if (S->o.fuse > 1) {
    RICHM_CUDA_TRY(cudaMemcpy(S->h_count + 1, S->active, sizeof(int) * S->op->batch, cudaMemcpyDeviceToHost));
    int act = 0;
    for (int i = 0; i < S->op->batch; ++i) act += S->h_count[1 + i] != 0;
    if (act > 0) S->rows_now = choose_rows(S);
  }
  S->started = true;
  return RICHM_OK;
}

}  // extern "C"
