// SSOR-preconditioned sweeps (eq. 17 with B^{-1} = w (2 - w) (D - w U)^{-1} D (D - w L)^{-1},
// the SSOR member of the stationary preconditioners listed after eq. 17; w is the
// relaxation factor, A = D - L - U split in the row-major numbering of each instance).
//
// One sweep of the Table 1 iteration (velocity form, look-ahead at, momentum a, weight w_i)
//   y = x + at (x - x_prev),  r = b - A y,  x_new = x + a (x - x_prev) + w_i B^{-1} r
// is two passes over an instance, each a triangular solve with the 9-point stencil:
//   forward  (rows top to bottom):  z = (D - w L)^{-1} r, with r formed on the fly;
//   backward (rows bottom to top):  s = (D - w U)^{-1} D z, then x_new and x_prev_new = x.
// In the forward solve, z(i, j) = r(i, j)/c - (w/c) [ax z(i, j-1) + ay z(i-1, j)
// + d1 z(i-1, j-1) + d2 z(i-1, j+1)]: the previous row enters as known values, and along
// the row the recurrence z_j = q_j - kappa z_{j-1} (kappa = w ax / c, |kappa| < 1 for the
// Q1 stencil and 0 < w < 2) is a first-order linear recurrence with a constant
// coefficient. The instance's rows are walked in order; within a row each lane takes VW
// consecutive columns, composes the affine maps of its columns, and a log-depth scan of
// those maps across the lanes (shuffles) gives every lane its incoming value, after which
// it replays its columns. Rows of at most 32 VW columns run on two warps per instance
// (the row pipelines below); wider rows are taken in chunks by one warp, carrying the
// last value. The backward solve is the mirror image (rows and columns reversed, upper
// neighbours). The intermediate z lives in a padded buffer.
//
// With x == nullptr the same kernels apply the preconditioner alone, out = B^{-1} b
// (y = 0, no momentum, w = 1): the adjoint of a preconditioned sweep needs B^{-1} of
// the incoming gradient.
#include <algorithm>

#include "common.cuh"
#include "kernels.cuh"

namespace richm {

constexpr int kSsorWarps = 1;  // instances per block of the multi-chunk kernels (one warp each)

template <typename E> struct SsorVW;
template <> struct SsorVW<float> { static constexpr int v = 16; };
template <> struct SsorVW<double> { static constexpr int v = 8; };

// VW values of row `row` (1..n, else zeros) at columns c0.. of an instance's buffer,
// with the left and right neighbours of the lane's first and last column (zero outside
// 0..pitch-1; the lane's own loads and shuffles inside a chunk).
template <typename E, int VW>
struct RowVW {
  E v[VW];
  E l, r;
};

// 16-byte vector loads and stores of VW consecutive values (constant indices only, so
// the values stay in registers).
template <typename E, int VW>
__device__ __forceinline__ void ld16(const E* p, E* v) {
  if constexpr (sizeof(E) == 4) {
#pragma unroll
    for (int q = 0; q < VW / 4; ++q) {
      const float4 t = reinterpret_cast<const float4*>(p)[q];
      v[4 * q] = t.x;
      v[4 * q + 1] = t.y;
      v[4 * q + 2] = t.z;
      v[4 * q + 3] = t.w;
    }
  } else {
#pragma unroll
    for (int q = 0; q < VW / 2; ++q) {
      const double2 t = reinterpret_cast<const double2*>(p)[q];
      v[2 * q] = t.x;
      v[2 * q + 1] = t.y;
    }
  }
}
template <typename E, int VW>
__device__ __forceinline__ void st16(E* p, const E* v) {
  if constexpr (sizeof(E) == 4) {
#pragma unroll
    for (int q = 0; q < VW / 4; ++q)
      reinterpret_cast<float4*>(p)[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
  } else {
#pragma unroll
    for (int q = 0; q < VW / 2; ++q) reinterpret_cast<double2*>(p)[q] = make_double2(v[2 * q], v[2 * q + 1]);
  }
}

template <typename E, int VW>
__device__ __forceinline__ void load_vw(const E* base, int row, int n, int pitch, int c0, int lane, bool live,
                                        bool first_chunk, RowVW<E, VW>& R) {
  const bool in = row >= 1 && row <= n;
  const E* p = base + (long long)row * pitch + c0;
#pragma unroll
  for (int e = 0; e < VW; ++e) R.v[e] = E(0);
  if (in && live) ld16<E, VW>(p, R.v);
  E l = __shfl_up_sync(0xffffffffu, R.v[VW - 1], 1);
  E r = __shfl_down_sync(0xffffffffu, R.v[0], 1);
  if (lane == 0) l = (in && !first_chunk) ? p[-1] : E(0);
  if (lane == 31) r = (in && c0 + VW < pitch) ? p[VW] : E(0);
  R.l = l;
  R.r = r;
}

template <typename E, int VW>
__device__ __forceinline__ E left_of(const RowVW<E, VW>& R, int e) { return e == 0 ? R.l : R.v[e - 1]; }
template <typename E, int VW>
__device__ __forceinline__ E right_of(const RowVW<E, VW>& R, int e) { return e == VW - 1 ? R.r : R.v[e + 1]; }

// y = x + at (x - x_prev) on a row (neighbours included).
template <typename E, int VW>
__device__ __forceinline__ void lookahead(RowVW<E, VW>& X, const RowVW<E, VW>& XP, E at) {
#pragma unroll
  for (int e = 0; e < VW; ++e) X.v[e] = X.v[e] + at * (X.v[e] - XP.v[e]);
  X.l = X.l + at * (X.l - XP.l);
  X.r = X.r + at * (X.r - XP.r);
}

// Inclusive scan of affine maps z -> P + Q z over the lanes, in lane order (UP) or in
// reverse lane order; composing a map after the ones before it.
template <typename E, bool UP>
__device__ __forceinline__ void scan_maps(E& P, E& Q, int lane) {
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const E Pp = UP ? __shfl_up_sync(0xffffffffu, P, d) : __shfl_down_sync(0xffffffffu, P, d);
    const E Qp = UP ? __shfl_up_sync(0xffffffffu, Q, d) : __shfl_down_sync(0xffffffffu, Q, d);
    const bool has = UP ? lane >= d : lane + d < 32;
    if (has) {
      P = P + Q * Pp;
      Q = Q * Qp;
    }
  }
}

template <typename E>
struct SsorArgs {
  const Inst* insts;
  int batch;
  const E* x;   // null: apply B^{-1} to b (y = 0, out_x = B^{-1} b)
  const E* xp;  // null without momentum
  const E* b;
  E* z;         // intermediate (padded)
  E* out_x;
  E* out_xp;    // null without momentum
  const E* w;   // null: w = 1
  const E* a;   // null without momentum
  const E* at;  // null: at = a
  int m, kidx;
  E relax;
  const int* active;
};

template <typename E, int VW>
__global__ void __launch_bounds__(kSsorWarps * 32) ssor_forward_kernel(const SsorArgs<E> A) {
  const int lane = threadIdx.x & 31;
  const int inst = blockIdx.x * kSsorWarps + (threadIdx.x >> 5);
  if (inst >= A.batch) return;
  if (A.active && A.active[inst] == 0) return;
  const Inst& I = A.insts[inst];
  const int n = I.n, pitch = I.pitch;
  const E c = (E)I.c, ax = (E)I.ax, ay = (E)I.ay, d1 = (E)I.d1, d2 = (E)I.d2;
  const E rc = E(1) / c;
  const E kx = A.relax * ax * rc, ky = A.relax * ay * rc, k1 = A.relax * d1 * rc, k2 = A.relax * d2 * rc;
  const int ci = inst * A.m + A.kidx;
  const E ati = A.a ? (A.at ? A.at[ci] : A.a[ci]) : E(0);
  const E* xb = A.x ? A.x + I.off : nullptr;
  const E* xpb = A.xp ? A.xp + I.off : nullptr;
  const E* bb = A.b + I.off;
  E* zb = A.z + I.off;
  constexpr int CH = 32 * VW;
  const int nch = (pitch + CH - 1) / CH;
  for (int i = 1; i <= n; ++i) {
    E carry = E(0);
    for (int ch = 0; ch < nch; ++ch) {
      const int c0 = ch * CH + lane * VW;
      const bool live = c0 < pitch;
      RowVW<E, VW> YU{}, YC{}, YD{}, ZU, T;
      if (xb) {
        load_vw<E, VW>(xb, i - 1, n, pitch, c0, lane, live, ch == 0, YU);
        load_vw<E, VW>(xb, i, n, pitch, c0, lane, live, ch == 0, YC);
        load_vw<E, VW>(xb, i + 1, n, pitch, c0, lane, live, ch == 0, YD);
      }
      if (xb && xpb && ati != E(0)) {
        load_vw<E, VW>(xpb, i - 1, n, pitch, c0, lane, live, ch == 0, T);
        lookahead<E, VW>(YU, T, ati);
        load_vw<E, VW>(xpb, i, n, pitch, c0, lane, live, ch == 0, T);
        lookahead<E, VW>(YC, T, ati);
        load_vw<E, VW>(xpb, i + 1, n, pitch, c0, lane, live, ch == 0, T);
        lookahead<E, VW>(YD, T, ati);
      }
      load_vw<E, VW>(zb, i - 1, n, pitch, c0, lane, live, ch == 0, ZU);
      load_vw<E, VW>(bb, i, n, pitch, c0, lane, live, ch == 0, T);  // b (neighbours unused)
      E q[VW], k[VW];
      E P = E(0), Q = E(1);
#pragma unroll
      for (int e = 0; e < VW; ++e) {
        const E Ay = c * YC.v[e] + ax * (left_of(YC, e) + right_of(YC, e)) + ay * (YU.v[e] + YD.v[e]) +
                     d1 * (right_of(YD, e) + left_of(YU, e)) + d2 * (right_of(YU, e) + left_of(YD, e));
        const bool ok = c0 + e < n;
        q[e] = ok ? (T.v[e] - Ay) * rc - (ky * ZU.v[e] + k1 * left_of(ZU, e) + k2 * right_of(ZU, e)) : E(0);
        k[e] = ok ? -kx : E(0);
        P = q[e] + k[e] * P;
        Q = k[e] * Q;
      }
      scan_maps<E, true>(P, Q, lane);
      E Pe = __shfl_up_sync(0xffffffffu, P, 1), Qe = __shfl_up_sync(0xffffffffu, Q, 1);
      if (lane == 0) Pe = E(0), Qe = E(1);
      E zv = Pe + Qe * carry;
      E out[VW];
#pragma unroll
      for (int e = 0; e < VW; ++e) {
        zv = q[e] + k[e] * zv;
        out[e] = zv;
      }
      if (live) st16<E, VW>(zb + (long long)i * pitch + c0, out);
      carry = __shfl_sync(0xffffffffu, P + Q * carry, 31);
    }
    __syncwarp();  // row i of z is read by other lanes in the next row
  }
}

template <typename E, int VW>
__global__ void __launch_bounds__(kSsorWarps * 32) ssor_backward_kernel(const SsorArgs<E> A) {
  const int lane = threadIdx.x & 31;
  const int inst = blockIdx.x * kSsorWarps + (threadIdx.x >> 5);
  if (inst >= A.batch) return;
  if (A.active && A.active[inst] == 0) return;
  const Inst& I = A.insts[inst];
  const int n = I.n, pitch = I.pitch;
  const E c = (E)I.c, ax = (E)I.ax, ay = (E)I.ay, d1 = (E)I.d1, d2 = (E)I.d2;
  const E rc = E(1) / c;
  const E kx = A.relax * ax * rc, ky = A.relax * ay * rc, k1 = A.relax * d1 * rc, k2 = A.relax * d2 * rc;
  const int ci = inst * A.m + A.kidx;
  const E wi = (A.w ? A.w[ci] : E(1)) * A.relax * (E(2) - A.relax);
  const E ai = A.a ? A.a[ci] : E(0);
  const E* xb = A.x ? A.x + I.off : nullptr;
  const E* xpb = A.xp ? A.xp + I.off : nullptr;
  E* zb = A.z + I.off;
  E* ox = A.out_x + I.off;
  E* oxp = A.out_xp ? A.out_xp + I.off : nullptr;
  constexpr int CH = 32 * VW;
  const int nch = (pitch + CH - 1) / CH;
  {
    // the output's halo rows (the buffer may come uninitialised from a rotation)
    E zero[VW];
#pragma unroll
    for (int e = 0; e < VW; ++e) zero[e] = E(0);
    for (int ch = 0; ch < nch; ++ch) {
      const int c0 = ch * CH + lane * VW;
      if (c0 < pitch) {
        st16<E, VW>(ox + c0, zero);
        st16<E, VW>(ox + (long long)(n + 1) * pitch + c0, zero);
        if (oxp) {
          st16<E, VW>(oxp + c0, zero);
          st16<E, VW>(oxp + (long long)(n + 1) * pitch + c0, zero);
        }
      }
    }
  }
  for (int i = n; i >= 1; --i) {
    E carry = E(0);
    for (int ch = nch - 1; ch >= 0; --ch) {
      const int c0 = ch * CH + lane * VW;
      const bool live = c0 < pitch;
      RowVW<E, VW> SD, ZC;
      load_vw<E, VW>(zb, i + 1, n, pitch, c0, lane, live, ch == 0, SD);  // s of the row below
      load_vw<E, VW>(zb, i, n, pitch, c0, lane, live, ch == 0, ZC);      // z of this row
      E t[VW], k[VW];
      E P = E(0), Q = E(1);
#pragma unroll
      for (int e = VW - 1; e >= 0; --e) {
        const bool ok = c0 + e < n;
        t[e] = ok ? ZC.v[e] - (ky * SD.v[e] + k1 * right_of(SD, e) + k2 * left_of(SD, e)) : E(0);
        k[e] = ok ? -kx : E(0);
        P = t[e] + k[e] * P;
        Q = k[e] * Q;
      }
      scan_maps<E, false>(P, Q, lane);
      E Pe = __shfl_down_sync(0xffffffffu, P, 1), Qe = __shfl_down_sync(0xffffffffu, Q, 1);
      if (lane == 31) Pe = E(0), Qe = E(1);
      E sv = Pe + Qe * carry;
      E sr[VW];
#pragma unroll
      for (int e = VW - 1; e >= 0; --e) {
        sv = t[e] + k[e] * sv;
        sr[e] = sv;
      }
      carry = __shfl_sync(0xffffffffu, P + Q * carry, 0);
      if (live) {
        const long long o = (long long)i * pitch + c0;
        E xv[VW] = {}, xpv[VW], xn[VW];
        if (xb) ld16<E, VW>(xb + o, xv);
        if (xpb) ld16<E, VW>(xpb + o, xpv);
#pragma unroll
        for (int e = 0; e < VW; ++e) {
          const E v = xpb ? xv[e] - xpv[e] : E(0);
          xn[e] = xv[e] + ai * v + wi * sr[e];
        }
        st16<E, VW>(ox + o, xn);
        if (oxp) st16<E, VW>(oxp + o, xv);
        st16<E, VW>(zb + o, sr);
      }
    }
    __syncwarp();  // row i of s is read by other lanes in the next row
  }
}

// ---------------------------------------------------------------- single-chunk rows
// Rows of at most 32 VW columns (FP32: n <= 511, FP64: n <= 255) are one chunk, so the
// whole previous row of z (forward) or s (backward) and the three-row window of the
// look-ahead iterate stay in registers, and the inputs arrive through cp.async rings
// twelve rows ahead. With a single chunk the incoming value of the row is 0, so the scan needs only
// the P parts: the multiplier of a lane's map is (-kappa)^VW (lanes holding columns
// >= n have multiplier 0, but they only ever follow the interior lanes in the forward
// direction, and in the backward direction the lanes after them contribute P = 0).

// y of a row from x and x_prev values loaded as plain vectors (zeros outside 1..n).
template <typename E, int VW>
__device__ __forceinline__ void y_from(const E* xv, const E* xpv, E at, bool mom, RowVW<E, VW>& Y) {
#pragma unroll
  for (int e = 0; e < VW; ++e) Y.v[e] = mom ? xv[e] + at * (xv[e] - xpv[e]) : xv[e];
  Y.l = __shfl_up_sync(0xffffffffu, Y.v[VW - 1], 1);
  Y.r = __shfl_down_sync(0xffffffffu, Y.v[0], 1);
}

template <typename E, int VW>
__device__ __forceinline__ void edges_zero(RowVW<E, VW>& Y, int lane) {
  if (lane == 0) Y.l = E(0);   // column -1: boundary
  if (lane == 31) Y.r = E(0);  // beyond the pitch
}


namespace {

// Row steps between issuing a row's copies and using it. One row step of a single warp
// is ~0.25 us, and the copies took several of them to land on GB300: prefetching 3, 6,
// 12 and 16 rows ahead gave 0.92, 0.71, 0.52 and 0.52 ms per sweep of 511^2.
constexpr int kRowPF = 12;
constexpr int kRowSlots = kRowPF + 1;  // ring slots per array

__device__ __forceinline__ void row_cp16(void* smem, const void* gmem, bool valid) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(sa), "l"(gmem), "r"(valid ? 16 : 0)
               : "memory");
}
__device__ __forceinline__ void row_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void row_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(kRowPF - 1) : "memory"); }
__device__ __forceinline__ void row_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

}  // namespace

// A row of 32 lanes x VW values in shared memory, interleaved in 16-byte chunks: chunk q
// of lane l at (32 q + l) x 16 bytes, so that each 16-byte access of a warp covers 512
// consecutive bytes (no bank conflicts; a lane's own VW values contiguous would put
// eight lanes of a quarter warp on four banks).
template <typename E, int VW>
__device__ __forceinline__ void ld_il(const unsigned char* row, int lane, E* v) {
  constexpr int C = 16 / (int)sizeof(E);
#pragma unroll
  for (int q = 0; q < VW / C; ++q) {
    if constexpr (sizeof(E) == 4) {
      const float4 t = *reinterpret_cast<const float4*>(row + (32 * q + lane) * 16);
      v[4 * q] = t.x;
      v[4 * q + 1] = t.y;
      v[4 * q + 2] = t.z;
      v[4 * q + 3] = t.w;
    } else {
      const double2 t = *reinterpret_cast<const double2*>(row + (32 * q + lane) * 16);
      v[2 * q] = t.x;
      v[2 * q + 1] = t.y;
    }
  }
}
template <typename E, int VW>
__device__ __forceinline__ void st_il(unsigned char* row, int lane, const E* v) {
  constexpr int C = 16 / (int)sizeof(E);
#pragma unroll
  for (int q = 0; q < VW / C; ++q) {
    if constexpr (sizeof(E) == 4)
      *reinterpret_cast<float4*>(row + (32 * q + lane) * 16) = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2],
                                                                           v[4 * q + 3]);
    else
      *reinterpret_cast<double2*>(row + (32 * q + lane) * 16) = make_double2(v[2 * q], v[2 * q + 1]);
  }
}

// Shared-memory rings: NSLOT slots of three interleaved row arrays, filled with cp.async
// by the warp that reads them, or read by another warp after a barrier.
template <typename E, int VW, int NSLOT = kRowSlots>
struct RowRing {
  static constexpr int ROW = 32 * VW * (int)sizeof(E);  // bytes of one array row
  static constexpr int BYTES = 3 * NSLOT * ROW;
  unsigned char* base;
  int lane;
  __device__ unsigned char* row(int array, int slot) const { return base + (array * NSLOT + slot) * ROW; }
  __device__ void load(int array, int slot, E* v) const { ld_il<E, VW>(row(array, slot), lane, v); }
  // copy this lane's VW values of row `r` (zero-filled unless valid) into (array, slot)
  __device__ void issue(int array, int slot, const E* src_base, int r, int pitch, int c0, bool valid) const {
    const E* src = src_base + (long long)(valid ? r : 0) * pitch + c0;
    unsigned char* dst = row(array, slot);
#pragma unroll
    for (int q = 0; q < VW * (int)sizeof(E) / 16; ++q)
      row_cp16(dst + (32 * q + lane) * 16, src + q * (16 / (int)sizeof(E)), valid);
  }
};

// rp = b/c - (A y)/c at the centre row C, with coefficients already divided by c.
template <typename E, int VW>
__device__ __forceinline__ void scaled_rhs(const RowVW<E, VW>& U, const RowVW<E, VW>& C, const RowVW<E, VW>& D,
                                           const E* bv, E rc, E axr, E ayr, E d1r, E d2r, E* rp) {
#pragma unroll
  for (int e = 0; e < VW; ++e) {
    E t = fma(-axr, left_of(C, e) + right_of(C, e), -C.v[e]);
    t = fma(-ayr, U.v[e] + D.v[e], t);
    t = fma(-d1r, right_of(D, e) + left_of(U, e), t);
    t = fma(-d2r, right_of(U, e) + left_of(D, e), t);
    rp[e] = fma(bv[e], rc, t);
  }
}

// FP32 rows of VW columns per lane: the same on packed pairs of columns (sm_100's FFMA2
// and friends: one issue slot for two columns), with the horizontal couplings written
// per column as west / east terms W_j = axr C_j + d1r U_j + d2r D_j and
// E_j = axr C_j + d2r U_j + d1r D_j formed on pairs, so that only their shifted sum
// W_{e-1} + E_{e+1} needs per-column adds.
template <int VW>
__device__ __forceinline__ void scaled_rhs_f32(const RowVW<float, VW>& U, const RowVW<float, VW>& C,
                                               const RowVW<float, VW>& D, const float* bv, float rc, float axr,
                                               float ayr, float d1r, float d2r, float* rp) {
  constexpr int NP = VW / 2;
  const float2 ax2 = make_float2(axr, axr), d12 = make_float2(d1r, d1r), d22 = make_float2(d2r, d2r);
  const float2 nay2 = make_float2(-ayr, -ayr), rc2 = make_float2(rc, rc), m1 = make_float2(-1.f, -1.f);
  float W[VW], E[VW];
#pragma unroll
  for (int p = 0; p < NP; ++p) {
    const float2 c2 = make_float2(C.v[2 * p], C.v[2 * p + 1]);
    const float2 u2 = make_float2(U.v[2 * p], U.v[2 * p + 1]);
    const float2 d2 = make_float2(D.v[2 * p], D.v[2 * p + 1]);
    const float2 axc = __fmul2_rn(ax2, c2);
    const float2 w2 = __ffma2_rn(d22, d2, __ffma2_rn(d12, u2, axc));
    const float2 e2 = __ffma2_rn(d12, d2, __ffma2_rn(d22, u2, axc));
    W[2 * p] = w2.x;
    W[2 * p + 1] = w2.y;
    E[2 * p] = e2.x;
    E[2 * p + 1] = e2.y;
  }
  const float wl = fmaf(d2r, D.l, fmaf(d1r, U.l, axr * C.l));  // W of the column left of this lane
  const float er = fmaf(d1r, D.r, fmaf(d2r, U.r, axr * C.r));  // E of the column right of this lane
#pragma unroll
  for (int p = 0; p < NP; ++p) {
    const float2 c2 = make_float2(C.v[2 * p], C.v[2 * p + 1]);
    const float2 u2 = make_float2(U.v[2 * p], U.v[2 * p + 1]);
    const float2 d2 = make_float2(D.v[2 * p], D.v[2 * p + 1]);
    const float2 b2 = make_float2(bv[2 * p], bv[2 * p + 1]);
    const float2 s2 = make_float2((p == 0 ? wl : W[2 * p - 1]) + E[2 * p + 1],
                                  W[2 * p] + (p == NP - 1 ? er : E[2 * p + 2]));
    float2 t = __ffma2_rn(m1, c2, __fmul2_rn(b2, rc2));
    t = __ffma2_rn(nay2, __fadd2_rn(u2, d2), t);
    t = __ffma2_rn(m1, s2, t);
    rp[2 * p] = t.x;
    rp[2 * p + 1] = t.y;
  }
}

template <>
__device__ __forceinline__ void scaled_rhs<float, 16>(const RowVW<float, 16>& U, const RowVW<float, 16>& C,
                                                      const RowVW<float, 16>& D, const float* bv, float rc, float axr,
                                                      float ayr, float d1r, float d2r, float* rp) {
  scaled_rhs_f32<16>(U, C, D, bv, rc, axr, ayr, d1r, d2r, rp);
}
template <>
__device__ __forceinline__ void scaled_rhs<float, 8>(const RowVW<float, 8>& U, const RowVW<float, 8>& C,
                                                     const RowVW<float, 8>& D, const float* bv, float rc, float axr,
                                                     float ayr, float d1r, float d2r, float* rp) {
  scaled_rhs_f32<8>(U, C, D, bv, rc, axr, ayr, d1r, d2r, rp);
}
template <>
__device__ __forceinline__ void scaled_rhs<float, 4>(const RowVW<float, 4>& U, const RowVW<float, 4>& C,
                                                     const RowVW<float, 4>& D, const float* bv, float rc, float axr,
                                                     float ayr, float d1r, float d2r, float* rp) {
  scaled_rhs_f32<4>(U, C, D, bv, rc, axr, ayr, d1r, d2r, rp);
}

template <int VW>
__device__ __forceinline__ void y_from_f32(const float* xv, const float* xpv, float at, bool mom,
                                           RowVW<float, VW>& Y) {
  const float2 at2 = make_float2(at, at), m1 = make_float2(-1.f, -1.f);
#pragma unroll
  for (int p = 0; p < VW / 2; ++p) {
    const float2 x2 = make_float2(xv[2 * p], xv[2 * p + 1]);
    float2 y2 = x2;
    if (mom) y2 = __ffma2_rn(at2, __ffma2_rn(m1, make_float2(xpv[2 * p], xpv[2 * p + 1]), x2), x2);
    Y.v[2 * p] = y2.x;
    Y.v[2 * p + 1] = y2.y;
  }
  Y.l = __shfl_up_sync(0xffffffffu, Y.v[VW - 1], 1);
  Y.r = __shfl_down_sync(0xffffffffu, Y.v[0], 1);
}
template <>
__device__ __forceinline__ void y_from<float, 16>(const float* xv, const float* xpv, float at, bool mom,
                                                  RowVW<float, 16>& Y) {
  y_from_f32<16>(xv, xpv, at, mom, Y);
}
template <>
__device__ __forceinline__ void y_from<float, 8>(const float* xv, const float* xpv, float at, bool mom,
                                                 RowVW<float, 8>& Y) {
  y_from_f32<8>(xv, xpv, at, mom, Y);
}
template <>
__device__ __forceinline__ void y_from<float, 4>(const float* xv, const float* xpv, float at, bool mom,
                                                 RowVW<float, 4>& Y) {
  y_from_f32<4>(xv, xpv, at, mom, Y);
}

// ---------------------------------------------------------------- two-warp row pipelines
// The single-warp row kernels spend most of a row on work off the recurrence's critical
// path (loading and forming the next rows' right-hand sides, the Table 1 update), which
// one warp issues in order with the recurrence. Here each instance has two warps: the
// solver warp runs only the row recurrence, the helper warp streams the inputs and does
// the rest, and they meet once per row at a named barrier (`bar.sync 1, 64`; the block is
// the instance, both warps run the same number of iterations, and both leave together).
//   forward:  at iteration t the helper stores rp of row t + 1 (formed at t - 1) in a
//             two-slot ring and forms rp of row t + 2; the solver solves row t from rp.
//   backward: at iteration t the solver solves row n - t and leaves s in a two-slot ring;
//             the helper applies the update to row n - t + 1 with the s of iteration t - 1
//             and keeps the z rows the solver reads resident (its copies of a row land
//             before the barrier that precedes the solver's use).
constexpr int kPipeSlotsB = kRowPF + 2;  // backward ring: a slot is re-targeted one iteration after its last read

__device__ __forceinline__ void pipe_sync() { asm volatile("bar.sync 1, 64;" ::: "memory"); }

template <typename E, int VW>
struct PipeSizes {
  static constexpr int RPB = 2 * 32 * VW * (int)sizeof(E);  // two slots of one row
  static constexpr int FWD = RowRing<E, VW>::BYTES + RPB;
  static constexpr int BWD = RowRing<E, VW, kPipeSlotsB>::BYTES + RPB;
};

// Per-lane constants of the in-row recurrence v_e = q_e + k_e v_{e-1} over this lane's
// VW columns in recurrence order (the backward solve passes its columns reversed). The
// composed map's offset P = sum_e ce_e q_e (ce_e = product of k after e) is summed as
// four independent partial sums, and the replay runs in groups of four columns: local
// recurrences from 0, a carry chain over the groups, and a fix-up with pk_e = product
// of k from the group's first column to e. Dependent steps per row: 6 + 9 instead of
// 16 + 16 for VW = 16.
template <typename E, int VW>
struct RecCoef {
  E ce[VW];
  E pk[VW];
};

template <typename E, int VW>
__device__ __forceinline__ void rec_coef(const E* k, RecCoef<E, VW>& R) {
  E p = E(1);
#pragma unroll
  for (int e = VW - 1; e >= 0; --e) {
    R.ce[e] = p;
    p *= k[e];
  }
#pragma unroll
  for (int g = 0; g < VW / 4; ++g) {
    E q = E(1);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      q *= k[4 * g + j];
      R.pk[4 * g + j] = q;
    }
  }
}

template <typename E, int VW>
__device__ __forceinline__ E rec_compose(const E* q, const RecCoef<E, VW>& R) {
  E s[4] = {E(0), E(0), E(0), E(0)};
#pragma unroll
  for (int e = 0; e < VW; ++e) s[e % 4] = fma(R.ce[e], q[e], s[e % 4]);
  return (s[0] + s[1]) + (s[2] + s[3]);
}

template <typename E, int VW>
__device__ __forceinline__ void rec_replay(const E* q, const E* k, const RecCoef<E, VW>& R, E vin, E* v) {
  E loc[VW];
#pragma unroll
  for (int g = 0; g < VW / 4; ++g) {
    E u = E(0);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      u = fma(k[4 * g + j], u, q[4 * g + j]);
      loc[4 * g + j] = u;
    }
  }
  E carry = vin;
#pragma unroll
  for (int g = 0; g < VW / 4; ++g) {
#pragma unroll
    for (int j = 0; j < 4; ++j) v[4 * g + j] = fma(R.pk[4 * g + j], carry, loc[4 * g + j]);
    carry = v[4 * g + 3];
  }
}

// Solver warp, forward: row i from rp (this lane's VW values) and the previous row of z.
template <typename E, int VW>
__device__ __forceinline__ void fwd_solve_row(const E* rp, RowVW<E, VW>& Z, const E* k, const E* mk, const E* qd,
                                              const RecCoef<E, VW>& R, E ky, E k1, E k2, int lane, bool live,
                                              E* zrow) {
  E q[VW];
#pragma unroll
  for (int e = 0; e < VW; ++e)  // z = 0 beyond the domain (mask 0)
    q[e] = mk[e] * (rp[e] - (ky * Z.v[e] + k1 * left_of(Z, e) + k2 * right_of(Z, e)));
  E P = rec_compose<E, VW>(q, R);
#pragma unroll
  for (int d = 0; d < 5; ++d) {
    const E Pp = __shfl_up_sync(0xffffffffu, P, 1 << d);
    if (lane >= (1 << d)) P = P + qd[d] * Pp;
  }
  E zin = __shfl_up_sync(0xffffffffu, P, 1);
  if (lane == 0) zin = E(0);
  rec_replay<E, VW>(q, k, R, zin, Z.v);
  if (live) st16<E, VW>(zrow, Z.v);
  Z.l = __shfl_up_sync(0xffffffffu, Z.v[VW - 1], 1);
  Z.r = __shfl_down_sync(0xffffffffu, Z.v[0], 1);
  edges_zero<E, VW>(Z, lane);
}

// Helper warp, forward, iteration t at window phase PH (rows t, t + 1, t + 2 of y in
// slots PH, PH + 1, PH + 2 mod 3): publish rp of row t + 1, take step t + 2 (x, x_prev
// of row t + 3, b of row t + 2), put y of row t + 3 into slot PH and form rp of row t + 2.
template <typename E, int VW, int PH>
__device__ __forceinline__ void fwd_helper_iter(int t, RowVW<E, VW>* Y, E* rp, unsigned char* rpring, const RowRing<E, VW>& ring,
                                                int n, int pitch, int c0, bool live, bool hx, bool mom, E ati,
                                                E rc, E axr, E ayr, E d1r, E d2r, int lane, const E* xb,
                                                const E* xpb, const E* bb) {
  constexpr int S0 = PH, S1 = (PH + 1) % 3, S2 = (PH + 2) % 3;
  st_il<E, VW>(rpring + ((t + 1) & 1) * RowRing<E, VW>::ROW, lane, rp);
  row_wait();
  const int sl = (t + 2) % kRowSlots;
  E xv[VW], xpv[VW], bv[VW];
  ring.load(0, sl, xv);
  if (mom) ring.load(1, sl, xpv);
  ring.load(2, sl, bv);
  {
    const int s = t + 2 + kRowPF;
    const int sn = s % kRowSlots;
    const bool vx = hx && live && s + 1 <= n, vb = live && s >= 1 && s <= n;
    ring.issue(0, sn, xb, s + 1, pitch, c0, vx);
    if (mom) ring.issue(1, sn, xpb, s + 1, pitch, c0, vx);
    ring.issue(2, sn, bb, s, pitch, c0, vb);
    row_commit();
  }
  y_from<E, VW>(xv, xpv, ati, mom, Y[S0]);
  edges_zero<E, VW>(Y[S0], lane);
  scaled_rhs<E, VW>(Y[S1], Y[S2], Y[S0], bv, rc, axr, ayr, d1r, d2r, rp);
}

template <typename E, int VW>
__global__ void __launch_bounds__(64) ssor_forward_pipe_kernel(const SsorArgs<E> A) {
  extern __shared__ __align__(16) unsigned char ssor_smem[];
  const int lane = threadIdx.x & 31;
  const bool helper = threadIdx.x >= 32;
  const int inst = blockIdx.x;
  if (A.active && A.active[inst] == 0) return;  // both warps
  const Inst& I = A.insts[inst];
  const int n = I.n, pitch = I.pitch;
  const E rc = E(1) / (E)I.c;
  const E axr = (E)I.ax * rc, ayr = (E)I.ay * rc, d1r = (E)I.d1 * rc, d2r = (E)I.d2 * rc;
  const E kx = A.relax * axr, ky = A.relax * ayr, k1 = A.relax * d1r, k2 = A.relax * d2r;
  const int c0 = lane * VW;
  const bool live = c0 < pitch;
  unsigned char* rpring = ssor_smem + RowRing<E, VW>::BYTES;
  if (helper) {
    const int ci = inst * A.m + A.kidx;
    const E ati = A.a ? (A.at ? A.at[ci] : A.a[ci]) : E(0);
    const bool hx = A.x != nullptr;  // else y = 0: the x copies are zero fills from b's address
    const bool mom = hx && A.xp != nullptr && ati != E(0);
    const E* bb = A.b + I.off;
    const E* xb = hx ? A.x + I.off : bb;
    const E* xpb = A.xp ? A.xp + I.off : xb;
    RowRing<E, VW> ring{ssor_smem, lane};
    // step s brings x and x_prev of row s + 1 and b of row s
    auto issue = [&](int s) {
      const int sl = s % kRowSlots;
      const bool vx = hx && live && s + 1 <= n, vb = live && s >= 1 && s <= n;
      ring.issue(0, sl, xb, s + 1, pitch, c0, vx);
      if (mom) ring.issue(1, sl, xpb, s + 1, pitch, c0, vx);
      ring.issue(2, sl, bb, s, pitch, c0, vb);
      row_commit();
    };
    RowVW<E, VW> Y[3];  // slot 0: row 0 (zero), 1: row 1, 2: row 2
#pragma unroll
    for (int e = 0; e < VW; ++e) Y[0].v[e] = E(0);
    Y[0].l = Y[0].r = E(0);
#pragma unroll
    for (int s = 0; s < kRowPF; ++s) issue(s);
    E xv[VW], xpv[VW], bv[VW], rp[VW];
    row_wait();  // step 0: x, x_prev of row 1
    ring.load(0, 0, xv);
    if (mom) ring.load(1, 0, xpv);
    y_from<E, VW>(xv, xpv, ati, mom, Y[1]);
    edges_zero<E, VW>(Y[1], lane);
    issue(kRowPF);
    row_wait();  // step 1: x, x_prev of row 2, b of row 1
    ring.load(0, 1, xv);
    if (mom) ring.load(1, 1, xpv);
    ring.load(2, 1, bv);
    y_from<E, VW>(xv, xpv, ati, mom, Y[2]);
    edges_zero<E, VW>(Y[2], lane);
    issue(kRowPF + 1);
    scaled_rhs<E, VW>(Y[0], Y[1], Y[2], bv, rc, axr, ayr, d1r, d2r, rp);  // rp of row 1
    for (int t = 0; t <= n; t += 3) {
      fwd_helper_iter<E, VW, 0>(t, Y, rp, rpring, ring, n, pitch, c0, live, hx, mom, ati, rc, axr, ayr, d1r, d2r,
                                lane, xb, xpb, bb);
      pipe_sync();
      if (t + 1 > n) break;
      fwd_helper_iter<E, VW, 1>(t + 1, Y, rp, rpring, ring, n, pitch, c0, live, hx, mom, ati, rc, axr, ayr, d1r, d2r,
                                lane, xb, xpb, bb);
      pipe_sync();
      if (t + 2 > n) break;
      fwd_helper_iter<E, VW, 2>(t + 2, Y, rp, rpring, ring, n, pitch, c0, live, hx, mom, ati, rc, axr, ayr, d1r, d2r,
                                lane, xb, xpb, bb);
      pipe_sync();
    }
    row_wait_all();
  } else {
    E qd[5];  // multipliers of 2^d consecutive lanes' maps
    {
      E q = E(1);
#pragma unroll
      for (int e = 0; e < VW; ++e) q *= -kx;
#pragma unroll
      for (int d = 0; d < 5; ++d) {
        qd[d] = q;
        q *= q;
      }
    }
    E k[VW], mk[VW];  // recurrence coefficient and mask per column: 0 beyond the domain (z = 0 there)
#pragma unroll
    for (int e = 0; e < VW; ++e) {
      mk[e] = (c0 + e < n) ? E(1) : E(0);
      k[e] = -kx * mk[e];
    }
    RecCoef<E, VW> R;
    rec_coef<E, VW>(k, R);
    E* zb = A.z + I.off;
    RowVW<E, VW> Z;
#pragma unroll
    for (int e = 0; e < VW; ++e) Z.v[e] = E(0);
    Z.l = Z.r = E(0);
    for (int t = 0; t <= n; t += 3) {
      // iteration t: row t (none at t = 0), from the rp the helper published at t - 1
      if (t >= 1) {
        E rp[VW];
        ld_il<E, VW>(rpring + (t & 1) * RowRing<E, VW>::ROW, lane, rp);
        fwd_solve_row<E, VW>(rp, Z, k, mk, qd, R, ky, k1, k2, lane, live, zb + (long long)t * pitch + c0);
      }
      pipe_sync();
      if (t + 1 > n) break;
      {
        E rp[VW];
        ld_il<E, VW>(rpring + ((t + 1) & 1) * RowRing<E, VW>::ROW, lane, rp);
        fwd_solve_row<E, VW>(rp, Z, k, mk, qd, R, ky, k1, k2, lane, live, zb + (long long)(t + 1) * pitch + c0);
      }
      pipe_sync();
      if (t + 2 > n) break;
      {
        E rp[VW];
        ld_il<E, VW>(rpring + ((t + 2) & 1) * RowRing<E, VW>::ROW, lane, rp);
        fwd_solve_row<E, VW>(rp, Z, k, mk, qd, R, ky, k1, k2, lane, live, zb + (long long)(t + 2) * pitch + c0);
      }
      pipe_sync();
    }
  }
}

template <typename E, int VW>
__global__ void __launch_bounds__(64) ssor_backward_pipe_kernel(const SsorArgs<E> A) {
  extern __shared__ __align__(16) unsigned char ssor_smem[];
  using Ring = RowRing<E, VW, kPipeSlotsB>;
  const int lane = threadIdx.x & 31;
  const bool helper = threadIdx.x >= 32;
  const int inst = blockIdx.x;
  if (A.active && A.active[inst] == 0) return;  // both warps
  const Inst& I = A.insts[inst];
  const int n = I.n, pitch = I.pitch;
  const E rc = E(1) / (E)I.c;
  const E kx = A.relax * (E)I.ax * rc, ky = A.relax * (E)I.ay * rc, k1 = A.relax * (E)I.d1 * rc,
          k2 = A.relax * (E)I.d2 * rc;
  const int c0 = lane * VW;
  const bool live = c0 < pitch;
  Ring ring{ssor_smem, lane};
  unsigned char* sring = ssor_smem + Ring::BYTES;
  if (helper) {
    const int ci = inst * A.m + A.kidx;
    const E wi = (A.w ? A.w[ci] : E(1)) * A.relax * (E(2) - A.relax);
    const E ai = A.a ? A.a[ci] : E(0);
    const bool hx = A.x != nullptr;  // else x = 0: zero fills from z's address
    const bool mom = hx && A.xp != nullptr;
    const E* zb = A.z + I.off;
    const E* xb = hx ? A.x + I.off : zb;
    const E* xpb = A.xp ? A.xp + I.off : xb;
    E* ox = A.out_x + I.off;
    E* oxp = A.out_xp ? A.out_xp + I.off : nullptr;
    E zero[VW];
#pragma unroll
    for (int e = 0; e < VW; ++e) zero[e] = E(0);
    if (live) {  // the output's halo rows (the buffer may come uninitialised from a rotation)
      st16<E, VW>(ox + c0, zero);
      st16<E, VW>(ox + (long long)(n + 1) * pitch + c0, zero);
      if (oxp) {
        st16<E, VW>(oxp + c0, zero);
        st16<E, VW>(oxp + (long long)(n + 1) * pitch + c0, zero);
      }
    }
    // the copies of row r (z, x, x_prev) go to slot (n - r) mod slots
    auto issue = [&](int r) {
      const int sl = (n - r) % kPipeSlotsB;
      const bool v = live && r >= 1;
      ring.issue(0, sl, zb, r, pitch, c0, v);
      ring.issue(1, sl, xb, r, pitch, c0, v && hx);
      if (mom) ring.issue(2, sl, xpb, r, pitch, c0, v);
      row_commit();
    };
#pragma unroll
    for (int q = 0; q < kRowPF; ++q) issue(n - q);
    row_wait();  // row n for the solver's first iteration
    pipe_sync();
    for (int t = 0; t <= n; ++t) {
      if (t >= 1 && live) {  // the update of row n - t + 1 with the s of iteration t - 1
        const int r = n - t + 1;
        const int sl = (t - 1) % kPipeSlotsB;
        E xv[VW], xpv[VW], sv[VW], xn[VW];
        ring.load(1, sl, xv);
        if (mom) ring.load(2, sl, xpv);
        ld_il<E, VW>(sring + ((t - 1) & 1) * Ring::ROW, lane, sv);
#pragma unroll
        for (int e = 0; e < VW; ++e) xn[e] = xv[e] + ai * (mom ? xv[e] - xpv[e] : E(0)) + wi * sv[e];
        const long long o = (long long)r * pitch + c0;
        st16<E, VW>(ox + o, xn);
        if (oxp) st16<E, VW>(oxp + o, xv);
      }
      issue(n - t - kRowPF);
      row_wait();  // row n - t - 1 for the solver's next iteration
      pipe_sync();
    }
    row_wait_all();
  } else {
    E qd[5];
    {
      E q = E(1);
#pragma unroll
      for (int e = 0; e < VW; ++e) q *= -kx;
#pragma unroll
      for (int d = 0; d < 5; ++d) {
        qd[d] = q;
        q *= q;
      }
    }
    E k[VW], mk[VW];  // recurrence coefficient and mask per column: 0 beyond the domain
#pragma unroll
    for (int e = 0; e < VW; ++e) {
      mk[e] = (c0 + e < n) ? E(1) : E(0);
      k[e] = -kx * mk[e];
    }
    E kr[VW];  // the recurrence runs over the columns in reverse
#pragma unroll
    for (int e = 0; e < VW; ++e) kr[e] = k[VW - 1 - e];
    RecCoef<E, VW> R;
    rec_coef<E, VW>(kr, R);
    RowVW<E, VW> SD;  // s of the row below
#pragma unroll
    for (int e = 0; e < VW; ++e) SD.v[e] = E(0);
    SD.l = SD.r = E(0);
    pipe_sync();
    for (int t = 0; t <= n; ++t) {
      if (t < n) {  // row n - t
        E zc[VW];
        ring.load(0, t % kPipeSlotsB, zc);
        E tr[VW];  // t in reversed column order
#pragma unroll
        for (int e = VW - 1; e >= 0; --e)
          tr[VW - 1 - e] = mk[e] * (zc[e] - (ky * SD.v[e] + k1 * right_of(SD, e) + k2 * left_of(SD, e)));
        E P = rec_compose<E, VW>(tr, R);
#pragma unroll
        for (int d = 0; d < 5; ++d) {
          const E Pp = __shfl_down_sync(0xffffffffu, P, 1 << d);
          if (lane + (1 << d) < 32) P = P + qd[d] * Pp;
        }
        E sin = __shfl_down_sync(0xffffffffu, P, 1);
        if (lane == 31) sin = E(0);
        E sr[VW];
        rec_replay<E, VW>(tr, kr, R, sin, sr);
#pragma unroll
        for (int e = 0; e < VW; ++e) SD.v[e] = sr[VW - 1 - e];
        st_il<E, VW>(sring + (t & 1) * Ring::ROW, lane, SD.v);
        SD.l = __shfl_up_sync(0xffffffffu, SD.v[VW - 1], 1);
        SD.r = __shfl_down_sync(0xffffffffu, SD.v[0], 1);
        edges_zero<E, VW>(SD, lane);
      }
      pipe_sync();
    }
  }
}

// The row kernels' rings exceed the default 48 KB of dynamic shared memory per block.
template <typename E, int VW>
static cudaError_t ssor_row_attributes() {
  cudaError_t e = cudaFuncSetAttribute(ssor_forward_pipe_kernel<E, VW>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       PipeSizes<E, VW>::FWD);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(ssor_backward_pipe_kernel<E, VW>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             PipeSizes<E, VW>::BWD);
  return e;
}

cudaError_t init_ssor_attributes() {
  cudaError_t e = ssor_row_attributes<float, 16>();
  if (e == cudaSuccess) e = ssor_row_attributes<float, 8>();
  if (e == cudaSuccess) e = ssor_row_attributes<float, 4>();
  if (e == cudaSuccess) e = ssor_row_attributes<double, 8>();
  if (e == cudaSuccess) e = ssor_row_attributes<double, 4>();
  return e;
}

// The two-warp row pipelines with VW columns per lane (rows of at most 32 VW columns).
template <typename E, int VW>
static richm_status launch_ssor_pipes(richm_operator* op, const SsorArgs<E>& A, cudaStream_t s) {
  ssor_forward_pipe_kernel<E, VW><<<op->batch, 64, PipeSizes<E, VW>::FWD, s>>>(A);
  RICHM_LAUNCH_CHECK("SSOR forward solve");
  ssor_backward_pipe_kernel<E, VW><<<op->batch, 64, PipeSizes<E, VW>::BWD, s>>>(A);
  RICHM_LAUNCH_CHECK("SSOR backward solve");
  return RICHM_OK;
}

template <typename E>
richm_status launch_ssor_sweep(richm_operator* op, const E* x, const E* xp, const E* b, E* z, E* out_x, E* out_xp,
                               const E* w, const E* a, const E* at, int m, int kidx, double relax, const int* active,
                               cudaStream_t s) {
  constexpr int VW = SsorVW<E>::v;
  // out_xp (x_k copied for the caller) may be null when the caller keeps x_k in place
  SsorArgs<E> A{op->d_inst, op->batch, x, a ? xp : nullptr, b, z, out_x, a ? out_xp : nullptr,
                w, a, at, m, kidx, (E)relax, active};
  const int blocks = (op->batch + kSsorWarps - 1) / kSsorWarps;
  int max_pitch = 0;
  for (const Inst& I : op->h_inst) max_pitch = std::max(max_pitch, I.pitch);
  // every row is one chunk: two-warp row pipelines, one block per instance, with the
  // fewest columns per lane that cover the widest row (shorter lane chains per row)
  if (max_pitch <= 128) return launch_ssor_pipes<E, 4>(op, A, s);
  if (max_pitch <= 256) return launch_ssor_pipes<E, 8>(op, A, s);
  if constexpr (VW == 16) {
    if (max_pitch <= 512) return launch_ssor_pipes<E, 16>(op, A, s);
  }
  ssor_forward_kernel<E, VW><<<blocks, kSsorWarps * 32, 0, s>>>(A);
  RICHM_LAUNCH_CHECK("SSOR forward solve");
  ssor_backward_kernel<E, VW><<<blocks, kSsorWarps * 32, 0, s>>>(A);
  RICHM_LAUNCH_CHECK("SSOR backward solve");
  return RICHM_OK;
}

template <typename E>
richm_status launch_ssor_apply(richm_operator* op, const E* r, E* z, E* out, double relax, cudaStream_t s) {
  return launch_ssor_sweep<E>(op, nullptr, nullptr, r, z, out, nullptr, nullptr, nullptr, nullptr, 1, 0, relax,
                              nullptr, s);
}

template richm_status launch_ssor_apply<float>(richm_operator*, const float*, float*, float*, double, cudaStream_t);
template richm_status launch_ssor_apply<double>(richm_operator*, const double*, double*, double*, double,
                                                cudaStream_t);
template richm_status launch_ssor_sweep<float>(richm_operator*, const float*, const float*, const float*, float*,
                                               float*, float*, const float*, const float*, const float*, int, int,
                                               double, const int*, cudaStream_t);
template richm_status launch_ssor_sweep<double>(richm_operator*, const double*, const double*, const double*,
                                                double*, double*, double*, const double*, const double*,
                                                const double*, int, int, double, const int*, cudaStream_t);

}  // namespace richm
