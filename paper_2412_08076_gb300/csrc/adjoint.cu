// Differentiation of K unrolled sweeps ("backpropagate", Algorithm 1).
//
// Forward sweep k (i = k mod m):  v = x_k - x_{k-1},  y = x_k + at_i v,
//   x_{k+1} = x_k + a_i v + w_i d (b - A y)      (d = D^{-1} or 1)
// With lam_{k+1} = dL/dx_{k+1} and A symmetric, q = w_i A (d lam_{k+1}) and
//   lam_k  = (1 + a_i) lam_{k+1} - (1 + at_i) q + c_{k+1}
//   c_k    = -a_i lam_{k+1} + at_i q          (the part that reaches x_{k-1})
//   dL/dw_i += <lam_{k+1}, d (b - A y)>,  dL/da_i += <lam_{k+1}, v>,  dL/dat_i -= <q, v>
// and dL/dx_0 = lam_0 + c_0 because x_{-1} = x_0. One adjoint kernel applies the
// stencil twice (to d lam and to y), so each step streams lam, c, x_k, x_{k-1}, b
// once. States between checkpoints are recomputed from the checkpoint by the
// forward kernel, which is deterministic, so the recomputation is bitwise exact.
//
// With the SSOR preconditioner (d replaced by the symmetric matrix B^{-1}) the step
// first forms u = B^{-1} lam_{k+1} with the SSOR solves; then q = w_i A u and, because
// <lam, B^{-1} r> = <B^{-1} lam, r>, dL/dw_i += <u, b - A y> with no second solve.
//
// Complex states (the Helmholtz operators of eqs. 21-22, real weights): with the
// gradient of a real loss written g = dL/dRe x + i dL/dIm x, so that dL = Re<g, dx>
// with <u, v> = sum conj(u) v, the same recursion holds with A^T replaced by A^H. The
// 5-point Helmholtz matrix is complex symmetric (its absorbing and sponge terms sit on
// the diagonal), so A^H = conj(A): the stencil with the imaginary parts of its diagonal
// negated; the weight gradients are the real parts of the inner products above.
#include <type_traits>

#include "common.cuh"
#include "kernels.cuh"

namespace richm {

static size_t a256(size_t v) { return (v + 255) / 256 * 256; }

struct alignas(32) Dot3 {
  double v[4];
};

// Rows stream through per-warp shared-memory rings filled by cp.async two row steps
// ahead (each lane copies and reads back only its own 16-byte chunks; lanes 0 and 31
// also the chunks just outside the warp for the stencils' edge neighbours), as in the
// one-sweep kernel: x, x_prev and the stenciled array of the window row, b, the carry
// and (PM 2) lam of the output row.
constexpr int kAdjPF = 2;
constexpr int kAdjSlots = 4;
constexpr int kAdjXC = 34, kAdjBC = 32;  // chunks per stencil row (with the two edge chunks) and per plain row
__host__ __device__ constexpr int adj_ring_chunks() { return kAdjSlots * (3 * kAdjXC + 3 * kAdjBC); }

__device__ __forceinline__ void adj_cp(uint4* smem, const void* gmem, bool valid) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(sa), "l"(gmem), "r"(valid ? 16 : 0)
               : "memory");
}

// PM: 0 no preconditioner, 1 Jacobi (d = 1/c), 2 a matrix B^{-1} applied beforehand
// (u = B^{-1} lam in `ub`: the stencil and the weight gradient take u, the rest lam).
template <typename T, bool MOM, int PM>
__global__ void __launch_bounds__(kWarpsPerBlock * 32)
    adjoint_kernel(const Inst* insts, const Tile* tiles, int ntiles, const T* __restrict__ lam,
                   const T* __restrict__ ub, const T* __restrict__ carry, const T* __restrict__ x,
                   const T* __restrict__ xp, const T* __restrict__ b, T* __restrict__ lam_out,
                   T* __restrict__ carry_out, const T* __restrict__ w, const T* __restrict__ a,
                   const T* __restrict__ at, int m, int kidx, int final_step, Dot3* __restrict__ partials) {
  constexpr int VW = VecWidth<T>::value;
  extern __shared__ __align__(16) uint4 adj_ring[];
  const int lane = threadIdx.x & 31;
  const int wt = blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
  if (wt >= ntiles) return;
  const Tile t = tiles[wt];
  const Inst& I = insts[t.inst];
  const int n = I.n, pitch = I.pitch;
  const int cidx = t.inst * m + kidx;
  const T wi = w[cidx];
  T ai = 0, ati = 0;
  if (MOM) {
    ai = a[cidx];
    ati = at ? at[cidx] : ai;
  }
  const T sc = (T)I.c, sax = (T)I.ax, say = (T)I.ay, sd1 = (T)I.d1, sd2 = (T)I.d2;
  const T dv = PM == 1 ? (T)I.dinv : T(1);
  const T qs = wi * dv;  // q = w d A lam (d constant for Q1), or w A u
  const T* __restrict__ sl = PM == 2 ? ub : lam;  // the array the stencil is applied to
  const int c0 = t.tx * 32 * VW + lane * VW;
  const bool live = c0 < pitch;
  const int r0 = t.ty * kRows + 1;
  const int r1 = min(r0 + kRows - 1, n);
  const long long off = I.off;
  const bool has_left = c0 > 0, has_right = c0 + VW < pitch;
  const bool has_carry = MOM && carry != nullptr;
  uint4* ring = adj_ring + (threadIdx.x >> 5) * adj_ring_chunks();
  uint4* xr = ring;                        // [slot][XC]
  uint4* xpr = xr + kAdjSlots * kAdjXC;    // [slot][XC]
  uint4* lr = xpr + kAdjSlots * kAdjXC;    // [slot][XC] stenciled array
  uint4* br = lr + kAdjSlots * kAdjXC;     // [slot][BC]
  uint4* cr = br + kAdjSlots * kAdjBC;     // [slot][BC] carry
  uint4* mr = cr + kAdjSlots * kAdjBC;     // [slot][BC] lam (PM 2)

  // window row q of x, x_prev and the stenciled array; output row q - 1 of b, carry, lam
  auto issue = [&](int q) {
    const int so = q & (kAdjSlots - 1);
    const bool rv = (q >= 1) && (q <= n) && (q <= r1 + 1);
    const long long ro = off + (long long)(rv ? q : 0) * pitch;
    const int cc = live ? c0 : 0;
    adj_cp(xr + so * kAdjXC + 1 + lane, x + ro + cc, rv && live);
    if (MOM) adj_cp(xpr + so * kAdjXC + 1 + lane, xp + ro + cc, rv && live);
    adj_cp(lr + so * kAdjXC + 1 + lane, sl + ro + cc, rv && live);
    if (lane == 0) {
      const int lc = has_left ? c0 - VW : 0;
      adj_cp(xr + so * kAdjXC, x + ro + lc, rv && has_left);
      if (MOM) adj_cp(xpr + so * kAdjXC, xp + ro + lc, rv && has_left);
      adj_cp(lr + so * kAdjXC, sl + ro + lc, rv && has_left);
    }
    if (lane == 31) {
      const int rc = has_right ? c0 + VW : 0;
      adj_cp(xr + so * kAdjXC + 33, x + ro + rc, rv && has_right);
      if (MOM) adj_cp(xpr + so * kAdjXC + 33, xp + ro + rc, rv && has_right);
      adj_cp(lr + so * kAdjXC + 33, sl + ro + rc, rv && has_right);
    }
    const int qb = q - 1;
    const bool bv = (qb >= r0) && (qb <= r1) && live;
    const long long bo = off + (long long)(bv ? qb : 0) * pitch + (live ? c0 : 0);
    adj_cp(br + so * kAdjBC + lane, b + bo, bv);
    if (has_carry) adj_cp(cr + so * kAdjBC + lane, carry + bo, bv);
    if (PM == 2) adj_cp(mr + so * kAdjBC + lane, lam + bo, bv);
    asm volatile("cp.async.commit_group;\n" ::: "memory");
  };
  auto chunk = [&](const uint4* r, int i) {
    VecN<T, VW> v;
    *reinterpret_cast<uint4*>(&v) = r[i];
    return v;
  };
  // y = x + at (x - x_prev) of window row q with its neighbours; x, x_prev kept
  auto take_y = [&](int q, RowT<T, VW>& Y, T* xs, T* xps) {
    const int so = q & (kAdjSlots - 1);
    const VecN<T, VW> X = chunk(xr, so * kAdjXC + 1 + lane);
    VecN<T, VW> XP{};
    if (MOM) XP = chunk(xpr, so * kAdjXC + 1 + lane);
#pragma unroll
    for (int e = 0; e < VW; ++e) {
      Y.y[e] = MOM ? X.v[e] + ati * (X.v[e] - XP.v[e]) : X.v[e];
      xs[e] = X.v[e];
      xps[e] = XP.v[e];
    }
    T le = 0, re = 0;
    if (lane == 0) {
      const VecN<T, VW> L = chunk(xr, so * kAdjXC);
      le = L.v[VW - 1];
      if (MOM) le = le + ati * (le - chunk(xpr, so * kAdjXC).v[VW - 1]);
    }
    if (lane == 31) {
      const VecN<T, VW> R = chunk(xr, so * kAdjXC + 33);
      re = R.v[0];
      if (MOM) re = re + ati * (re - chunk(xpr, so * kAdjXC + 33).v[0]);
    }
    row_neighbours<T, VW>(Y, lane, le, re);
  };
  auto take_l = [&](int q, RowT<T, VW>& L) {
    const int so = q & (kAdjSlots - 1);
    const VecN<T, VW> Lv = chunk(lr, so * kAdjXC + 1 + lane);
#pragma unroll
    for (int e = 0; e < VW; ++e) L.y[e] = Lv.v[e];
    const T le = lane == 0 ? chunk(lr, so * kAdjXC).v[VW - 1] : T(0);
    const T re = lane == 31 ? chunk(lr, so * kAdjXC + 33).v[0] : T(0);
    row_neighbours<T, VW>(L, lane, le, re);
  };

  for (int q = r0 - 1; q <= r0 + kAdjPF; ++q) issue(q);
  asm volatile("cp.async.wait_group %0;\n" ::"n"(kAdjPF) : "memory");
  double s_w = 0.0, s_a = 0.0, s_at = 0.0;
  RowT<T, VW> YU, YC, YD, LU, LC, LD;
  T xC[VW], xpC[VW], xD[VW], xpD[VW], t0[VW], t1[VW];
  take_y(r0 - 1, YU, t0, t1);
  take_y(r0, YC, xC, xpC);
  take_l(r0 - 1, LU);
  take_l(r0, LC);
  for (int r = r0; r <= r1; ++r) {
    issue(r + 1 + kAdjPF);
    asm volatile("cp.async.wait_group %0;\n" ::"n"(kAdjPF) : "memory");
    take_y(r + 1, YD, xD, xpD);
    take_l(r + 1, LD);
    const int so = (r + 1) & (kAdjSlots - 1);
    const VecN<T, VW> Bv = chunk(br, so * kAdjBC + lane);
    VecN<T, VW> Cv{}, Lm{};
    if (has_carry) Cv = chunk(cr, so * kAdjBC + lane);
    if (PM == 2) Lm = chunk(mr, so * kAdjBC + lane);
    T Ay[VW], Al[VW];
    apply_q1<T, VW, T>(YU, YC, YD, sc, sax, say, sd1, sd2, Ay);
    apply_q1<T, VW, T>(LU, LC, LD, sc, sax, say, sd1, sd2, Al);
    VecN<T, VW> Lo, Co;
    // FP32 state: the row's few products are summed in FP32 and the row sums in FP64
    // (GB300's FP64 pipe would otherwise bound the kernel); FP64 state sums in FP64
    T rw = T(0), ra = T(0), rat = T(0);
#pragma unroll
    for (int e = 0; e < VW; ++e) {
      const bool ok = (c0 + e) < n;
      const T l = PM == 2 ? Lm.v[e] : LC.y[e];  // lam
      const T u = LC.y[e];                      // lam, d lam folded into dr, or B^{-1} lam
      const T q = qs * Al[e];
      const T dr = dv * (Bv.v[e] - Ay[e]);
      const T v = MOM ? xC[e] - xpC[e] : T(0);
      T ln = MOM ? (T(1) + ai) * l - (T(1) + ati) * q + Cv.v[e] : l - q;
      T cn = MOM ? -ai * l + ati * q : T(0);
      if (ok) {
        if constexpr (std::is_same<T, float>::value) {
          rw = fmaf(u, dr, rw);
          if (MOM) {
            ra = fmaf(l, v, ra);
            rat = fmaf(q, v, rat);
          }
        } else {
          s_w += (double)u * (double)dr;
          if (MOM) {
            s_a += (double)l * (double)v;
            s_at += (double)q * (double)v;
          }
        }
      }
      if (final_step) ln = ln + cn;
      Lo.v[e] = ok ? ln : T(0);
      Co.v[e] = ok ? cn : T(0);
    }
    if constexpr (std::is_same<T, float>::value) {
      s_w += f32_to_f64_exact(rw);
      if (MOM) {
        s_a += f32_to_f64_exact(ra);
        s_at += f32_to_f64_exact(rat);
      }
    }
    if (live) {
      const long long ro = off + (long long)r * pitch + c0;
      stv<T, VW>(lam_out + ro, Lo);
      if (MOM && !final_step) stv<T, VW>(carry_out + ro, Co);
    }
    YU = YC;
    YC = YD;
    LU = LC;
    LC = LD;
#pragma unroll
    for (int e = 0; e < VW; ++e) {
      xC[e] = xD[e];
      xpC[e] = xpD[e];
    }
  }
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
  s_w = warp_sum(s_w);
  s_a = warp_sum(s_a);
  s_at = warp_sum(s_at);
  if (lane == 0) {
    Dot3 d;
    d.v[0] = s_w;
    d.v[1] = s_a;
    d.v[2] = s_at;
    d.v[3] = 0.0;
    partials[wt] = d;
  }
}


// One adjoint step for complex states (no preconditioner): rows walk down a warp tile
// of 32 * VW columns with plain vector loads (the state of a complex tile row is 16
// bytes per lane), the stencils of y (for b - A y) and of lam (for A^H lam) kept as
// three-row windows.
template <typename C, bool MOM>
__global__ void __launch_bounds__(kWarpsPerBlock * 32)
    adjoint_cx_kernel(const Inst* insts, const Tile* tiles, int ntiles, const C* __restrict__ lam,
                      const C* __restrict__ carry, const C* __restrict__ x, const C* __restrict__ xp,
                      const C* __restrict__ b, C* __restrict__ lam_out, C* __restrict__ carry_out,
                      const typename RealOf<C>::type* __restrict__ w, const typename RealOf<C>::type* __restrict__ a,
                      const typename RealOf<C>::type* __restrict__ at, int m, int kidx, int final_step,
                      Dot3* __restrict__ partials) {
  using R = typename RealOf<C>::type;
  constexpr int VW = VecWidth<C>::value;
  const int lane = threadIdx.x & 31;
  const int wt = blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
  if (wt >= ntiles) return;
  const Tile t = tiles[wt];
  const Inst& I = insts[t.inst];
  const int n = I.n, pitch = I.pitch;
  const int cidx = t.inst * m + kidx;
  const R wi = w[cidx];
  R ai = 0, ati = 0;
  if (MOM) {
    ai = a[cidx];
    ati = at ? at[cidx] : ai;
  }
  const R sc = (R)I.c, soff = (R)I.ax, abr = (R)I.abc_re, abi = (R)I.abc_im, spi = (R)I.sp_im, spw = (R)I.sp_iw;
  const int c0 = t.tx * 32 * VW + lane * VW;
  const bool live = c0 < pitch;
  const int r0 = t.ty * kRows + 1;
  const int r1 = min(r0 + kRows - 1, n);
  const long long off = I.off;
  const bool has_carry = MOM && carry != nullptr;
  const C z{};
  // row pr of y = x + at (x - x_prev) with its neighbours; x, x_prev of the row kept
  auto load_y = [&](int pr, RowT<C, VW>& Y, C* xs, C* xps) {
    const bool in = (pr >= 1) && (pr <= n);
    const long long ro = off + (long long)pr * pitch;
    VecN<C, VW> X{}, XP{};
    if (in && live) {
      X = ldv<C, VW>(x + ro + c0);
      if (MOM) XP = ldv<C, VW>(xp + ro + c0);
    }
#pragma unroll
    for (int e = 0; e < VW; ++e) {
      Y.y[e] = MOM ? X.v[e] + ati * (X.v[e] - XP.v[e]) : X.v[e];
      xs[e] = X.v[e];
      xps[e] = XP.v[e];
    }
    C le = z, re = z;
    if (in) {
      if (lane == 0 && c0 > 0) {
        le = x[ro + c0 - 1];
        if (MOM) le = le + ati * (le - xp[ro + c0 - 1]);
      }
      if (lane == 31 && c0 + VW < pitch) {
        re = x[ro + c0 + VW];
        if (MOM) re = re + ati * (re - xp[ro + c0 + VW]);
      }
    }
    row_neighbours<C, VW>(Y, lane, le, re);
  };
  auto load_l = [&](int pr, RowT<C, VW>& L) {
    const bool in = (pr >= 1) && (pr <= n);
    const long long ro = off + (long long)pr * pitch;
    VecN<C, VW> Lv{};
    if (in && live) Lv = ldv<C, VW>(lam + ro + c0);
#pragma unroll
    for (int e = 0; e < VW; ++e) L.y[e] = Lv.v[e];
    C le = z, re = z;
    if (in) {
      if (lane == 0 && c0 > 0) le = lam[ro + c0 - 1];
      if (lane == 31 && c0 + VW < pitch) re = lam[ro + c0 + VW];
    }
    row_neighbours<C, VW>(L, lane, le, re);
  };
  double s_w = 0.0, s_a = 0.0, s_at = 0.0;
  RowT<C, VW> YU, YC, YD, LU, LC, LD;
  C xC[VW], xpC[VW], xD[VW], xpD[VW], t0[VW], t1[VW];
  load_y(r0 - 1, YU, t0, t1);
  load_y(r0, YC, xC, xpC);
  load_l(r0 - 1, LU);
  load_l(r0, LC);
  for (int r = r0; r <= r1; ++r) {
    load_y(r + 1, YD, xD, xpD);
    load_l(r + 1, LD);
    const long long ro = off + (long long)r * pitch + c0;
    VecN<C, VW> Bv{}, Cv{};
    if (live) {
      Bv = ldv<C, VW>(b + ro);
      if (has_carry) Cv = ldv<C, VW>(carry + ro);
    }
    C Ay[VW], Al[VW];
    apply_fd5<C, VW, R>(YU, YC, YD, r - 1, c0, n, sc, soff, abr, abi, spi, spw, Ay);
    apply_fd5<C, VW, R>(LU, LC, LD, r - 1, c0, n, sc, soff, abr, -abi, -spi, spw, Al);  // conj(A) lam
    VecN<C, VW> Lo, Co;
    // complex64: the row's products summed in FP32, the row sums in FP64 (GB300's FP64
    // pipe would otherwise bound the kernel); complex128 sums in FP64
    R rw = R(0), ra = R(0), rat = R(0);
#pragma unroll
    for (int e = 0; e < VW; ++e) {
      const bool ok = (c0 + e) < n;
      const C l = LC.y[e];
      const C q = wi * Al[e];
      const C dr = Bv.v[e] - Ay[e];
      const C v = MOM ? xC[e] - xpC[e] : z;
      C ln = MOM ? ((R(1) + ai) * l - (R(1) + ati) * q) + Cv.v[e] : l - q;
      const C cn = MOM ? (-ai) * l + ati * q : z;
      if (ok) {
        rw = fma(l.re, dr.re, fma(l.im, dr.im, rw));
        if (MOM) {
          ra = fma(l.re, v.re, fma(l.im, v.im, ra));
          rat = fma(q.re, v.re, fma(q.im, v.im, rat));
        }
      }
      if (final_step) ln = ln + cn;
      Lo.v[e] = ok ? ln : z;
      Co.v[e] = ok ? cn : z;
    }
    if constexpr (std::is_same<R, float>::value) {
      s_w += f32_to_f64_exact(rw);
      if (MOM) {
        s_a += f32_to_f64_exact(ra);
        s_at += f32_to_f64_exact(rat);
      }
    } else {
      s_w += rw;
      if (MOM) {
        s_a += ra;
        s_at += rat;
      }
    }
    if (live) {
      stv<C, VW>(lam_out + ro, Lo);
      if (MOM && !final_step) stv<C, VW>(carry_out + ro, Co);
    }
    YU = YC;
    YC = YD;
    LU = LC;
    LC = LD;
#pragma unroll
    for (int e = 0; e < VW; ++e) {
      xC[e] = xD[e];
      xpC[e] = xpD[e];
    }
  }
  s_w = warp_sum(s_w);
  s_a = warp_sum(s_a);
  s_at = warp_sum(s_at);
  if (lane == 0) {
    Dot3 d;
    d.v[0] = s_w;
    d.v[1] = s_a;
    d.v[2] = s_at;
    d.v[3] = 0.0;
    partials[wt] = d;
  }
}

// The adjoint kernels' rings exceed the default 48 KB of dynamic shared memory.
template <typename T>
static cudaError_t adjoint_attributes_t() {
  const int bytes = (int)(sizeof(uint4) * kWarpsPerBlock * adj_ring_chunks());
  cudaError_t e = cudaSuccess;
#define RICHM_ADJ_ATTR(M, P) \
  if (e == cudaSuccess)      \
    e = cudaFuncSetAttribute(adjoint_kernel<T, M, P>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  RICHM_ADJ_ATTR(true, 0)
  RICHM_ADJ_ATTR(true, 1)
  RICHM_ADJ_ATTR(true, 2)
  RICHM_ADJ_ATTR(false, 0)
  RICHM_ADJ_ATTR(false, 1)
  RICHM_ADJ_ATTR(false, 2)
#undef RICHM_ADJ_ATTR
  return e;
}

cudaError_t init_adjoint_attributes() {
  cudaError_t e = adjoint_attributes_t<float>();
  if (e == cudaSuccess) e = adjoint_attributes_t<double>();
  return e;
}

// acc[b][kidx][0..2] += per-instance sums of the tile partials (fixed order).
__global__ void adjoint_reduce_kernel(const Dot3* __restrict__ partials, const int* __restrict__ inst_begin,
                                      int batch, int m, int kidx, double* __restrict__ acc) {
  const int lane = threadIdx.x & 31;
  const int bi = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (bi >= batch) return;
  double s0 = 0.0, s1 = 0.0, s2 = 0.0;
  for (int t = inst_begin[bi] + lane; t < inst_begin[bi + 1]; t += 32) {
    const Dot3 p = partials[t];
    s0 += p.v[0];
    s1 += p.v[1];
    s2 += p.v[2];
  }
  s0 = warp_sum(s0);
  s1 = warp_sum(s1);
  s2 = warp_sum(s2);
  if (lane == 0) {
    double* A = acc + ((long long)bi * m + kidx) * 3;
    A[0] += s0;
    A[1] += s1;
    A[2] += s2;
  }
}

template <typename T>
__global__ void adjoint_finish_kernel(const double* __restrict__ acc, int count, T* g_w, T* g_a, T* g_at,
                                      int nag) {  // T: the weights' real type
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  const double dw = acc[3 * i], da = acc[3 * i + 1], dat = -acc[3 * i + 2];
  if (g_w) g_w[i] = (T)dw;
  if (g_a) g_a[i] = (T)(nag ? da + dat : da);
  if (g_at) g_at[i] = (T)dat;
}

template <typename T>
static richm_status launch_adjoint(richm_operator* op, const T* lam, const T* ub, const T* carry, const T* x,
                                   const T* xp, const T* b, T* lam_out, T* carry_out, const T* w, const T* a,
                                   const T* at, int m, int kidx, int precond, int final_step, Dot3* partials,
                                   double* acc, cudaStream_t s) {
  constexpr int VW = VecWidth<T>::value;
  const TileMap* tm = nullptr;
  RICHM_TRY(get_tiles(op, 32 * VW, kRows, &tm));
  const int blocks = (tm->ntiles + kWarpsPerBlock - 1) / kWarpsPerBlock;
  const int thr = kWarpsPerBlock * 32;
  const bool mom = a != nullptr;
  const size_t smem = sizeof(uint4) * kWarpsPerBlock * adj_ring_chunks();
#define RICHM_ADJ(M, P)                                                                                         \
  adjoint_kernel<T, M, P><<<blocks, thr, smem, s>>>(op->d_inst, tm->d_tiles, tm->ntiles, lam, ub, carry, x, xp, \
                                                    b, lam_out, carry_out, w, a, at, m, kidx, final_step, partials)
  if (mom) {
    if (precond == 2) RICHM_ADJ(true, 2);
    else if (precond == 1) RICHM_ADJ(true, 1);
    else RICHM_ADJ(true, 0);
  } else {
    if (precond == 2) RICHM_ADJ(false, 2);
    else if (precond == 1) RICHM_ADJ(false, 1);
    else RICHM_ADJ(false, 0);
  }
#undef RICHM_ADJ
  RICHM_LAUNCH_CHECK("adjoint sweep");
  const int wpb = 8;
  adjoint_reduce_kernel<<<(op->batch + wpb - 1) / wpb, wpb * 32, 0, s>>>(partials, tm->d_inst_begin, op->batch, m,
                                                                         kidx, acc);
  RICHM_LAUNCH_CHECK("adjoint reduce");
  return RICHM_OK;
}

template <typename C>
static richm_status launch_adjoint_cx(richm_operator* op, const C* lam, const C* carry, const C* x, const C* xp,
                                      const C* b, C* lam_out, C* carry_out, const typename RealOf<C>::type* w,
                                      const typename RealOf<C>::type* a, const typename RealOf<C>::type* at, int m,
                                      int kidx, int final_step, Dot3* partials, double* acc, cudaStream_t s) {
  constexpr int VW = VecWidth<C>::value;
  const TileMap* tm = nullptr;
  RICHM_TRY(get_tiles(op, 32 * VW, kRows, &tm));
  const int blocks = (tm->ntiles + kWarpsPerBlock - 1) / kWarpsPerBlock;
  const int thr = kWarpsPerBlock * 32;
  if (a != nullptr)
    adjoint_cx_kernel<C, true><<<blocks, thr, 0, s>>>(op->d_inst, tm->d_tiles, tm->ntiles, lam, carry, x, xp, b,
                                                      lam_out, carry_out, w, a, at, m, kidx, final_step, partials);
  else
    adjoint_cx_kernel<C, false><<<blocks, thr, 0, s>>>(op->d_inst, tm->d_tiles, tm->ntiles, lam, carry, x, xp, b,
                                                       lam_out, carry_out, w, a, at, m, kidx, final_step, partials);
  RICHM_LAUNCH_CHECK("complex adjoint sweep");
  const int wpb = 8;
  adjoint_reduce_kernel<<<(op->batch + wpb - 1) / wpb, wpb * 32, 0, s>>>(partials, tm->d_inst_begin, op->batch, m,
                                                                         kidx, acc);
  RICHM_LAUNCH_CHECK("adjoint reduce");
  return RICHM_OK;
}

// One forward sweep with any preconditioner (z: SSOR scratch; real states only).
template <typename T>
static richm_status sweep_any(richm_operator* op, const T* x, const T* xp, const T* b, T* out,
                              const typename RealOf<T>::type* w, const typename RealOf<T>::type* a,
                              const typename RealOf<T>::type* at, int m, int kidx, int precond, double relax, T* z,
                              cudaStream_t s) {
  if constexpr (!IsCplx<T>::value) {
    if (precond == 2)
      return launch_ssor_sweep<T>(op, x, xp, b, z, out, nullptr, w, a, at, m, kidx, relax, nullptr, s);
  }
  return launch_sweep<T>(op, x, xp, b, out, w, a, at, m, kidx, precond, nullptr, s);
}

template <typename T, typename WT = typename RealOf<T>::type>
static richm_status forward_ckpt_t(richm_operator* op, const T* x0, const T* b, const WT* w, const WT* a,
                                   const WT* at, int m, int K, int s_every, int precond, double relax, T* ckpts,
                                   T* xK, void* work, cudaStream_t s) {
  const size_t es = op->elems;
  const size_t bytes = es * sizeof(T);
  const size_t slot = 2 * es;
  // slot j holds (x_{js}, x_{js-1}); slot 0 = (x0, x0)
  RICHM_CUDA_TRY(cudaMemcpyAsync(ckpts, x0, bytes, cudaMemcpyDeviceToDevice, s));
  RICHM_CUDA_TRY(cudaMemcpyAsync(ckpts + es, x0, bytes, cudaMemcpyDeviceToDevice, s));
  T* W[4];  // three rotating states and the SSOR scratch
  for (int i = 0; i < 4; ++i) W[i] = reinterpret_cast<T*>(reinterpret_cast<char*>(work) + i * a256(bytes));
  const int nseg = K / s_every;
  // FP32 segments of 8 (or 4) sweeps without SSOR: one temporally blocked pass per
  // segment writes exactly the pair the next checkpoint holds (x_{k+TL}, x_{k+TL-1});
  // it agrees with the one-sweep kernels that recompute the segments backward to FP32
  // rounding (not bit for bit)
  int TL = 0;
  if constexpr (std::is_same<T, float>::value) {
    if (precond != 2 && a != nullptr && (s_every == 8 || s_every == 4)) TL = s_every;
  }
  for (int j = 0; j < nseg; ++j) {
    T* cx = ckpts + (size_t)j * slot;
    T* cxp = cx + es;
    T* nx = ckpts + (size_t)(j + 1) * slot;
    T* nxp = nx + es;
    if constexpr (std::is_same<T, float>::value) {
      if (TL) {
        RICHM_TRY(launch_sweep_fused(op, TL, cx, cxp, b, nx, nxp, w, a, at, m, (j * s_every) % m, precond, nullptr, s));
        continue;
      }
    }
    T* cur = cx;
    T* prev = cxp;
    for (int t = 0; t < s_every; ++t) {
      // the last two sweeps land in the next checkpoint slot; the others rotate
      // through three work buffers, never touching either checkpoint slot
      T* out = nullptr;
      if (t == s_every - 1) out = nx;
      else if (t == s_every - 2) out = nxp;
      else
        for (int i = 0; i < 3 && out == nullptr; ++i)
          if (W[i] != cur && W[i] != prev) out = W[i];
      const int kidx = (j * s_every + t) % m;
      RICHM_TRY(sweep_any<T>(op, cur, a ? prev : nullptr, b, out, w, a, at, m, kidx, precond, relax, W[3], s));
      prev = cur;
      cur = out;
    }
    if (s_every == 1) RICHM_CUDA_TRY(cudaMemcpyAsync(nxp, cx, bytes, cudaMemcpyDeviceToDevice, s));
  }
  if (xK) RICHM_CUDA_TRY(cudaMemcpyAsync(xK, ckpts + (size_t)nseg * slot, bytes, cudaMemcpyDeviceToDevice, s));
  return RICHM_OK;
}

template <typename T>
static size_t adjoint_ws(richm_operator* op, int s_every) {
  int nt = 0;
  residual_tiles<T>(op, &nt);
  const size_t buf = a256(op->elems * sizeof(T));
  // segment states, lam and carry pairs, u = B^{-1} lam and the SSOR scratch
  const size_t adj = (size_t)(s_every > 1 ? s_every - 1 : 0) * buf + 6 * buf + a256(sizeof(Dot3) * nt) +
                     a256(sizeof(double) * 3 * 64 * (size_t)op->batch);
  const size_t loss = loss_workspace_bytes(op, sizeof(T), nt);
  return adj > loss ? adj : loss;
}

template <typename T, typename W = typename RealOf<T>::type>
static richm_status adjoint_t(richm_operator* op, const T* ckpts, int s_every, const T* b, const T* gK, const W* w,
                              const W* a, const W* at, int m, int K, int precond, double relax, W* g_w, W* g_a,
                              W* g_at, T* g_x0, void* work, size_t work_bytes, cudaStream_t s) {
  if (work_bytes < adjoint_ws<T>(op, s_every)) return set_error(RICHM_ERR_NOMEM, "adjoint workspace too small");
  const size_t es = op->elems;
  const size_t buf = a256(es * sizeof(T));
  const size_t slot = 2 * es;
  int nt = 0;
  RICHM_TRY(residual_tiles<T>(op, &nt));
  char* p = reinterpret_cast<char*>(work);
  std::vector<T*> seg(s_every + 1, nullptr);
  for (int t = 2; t <= s_every; ++t) {
    seg[t] = reinterpret_cast<T*>(p);
    p += buf;
  }
  T* LB[2];
  T* CB[2];
  for (int i = 0; i < 2; ++i) {
    LB[i] = reinterpret_cast<T*>(p);
    p += buf;
  }
  for (int i = 0; i < 2; ++i) {
    CB[i] = reinterpret_cast<T*>(p);
    p += buf;
  }
  T* U = reinterpret_cast<T*>(p);  // B^{-1} lam (SSOR)
  p += buf;
  T* Z = reinterpret_cast<T*>(p);  // SSOR scratch
  p += buf;
  Dot3* partials = reinterpret_cast<Dot3*>(p);
  p += a256(sizeof(Dot3) * nt);
  double* acc = reinterpret_cast<double*>(p);
  RICHM_CUDA_TRY(cudaMemsetAsync(acc, 0, sizeof(double) * 3 * m * (size_t)op->batch, s));
  const T* lam = gK;
  const T* carry = nullptr;
  int pi = 0;
  const int nseg = K / s_every;
  for (int j = nseg - 1; j >= 0; --j) {
    const T* cx = ckpts + (size_t)j * slot;
    seg[0] = const_cast<T*>(cx + es);  // x_{js-1}
    seg[1] = const_cast<T*>(cx);       // x_{js}
    for (int t = 0; t + 2 <= s_every; ++t) {
      const int kidx = (j * s_every + t) % m;
      RICHM_TRY(sweep_any<T>(op, seg[t + 1], a ? seg[t] : nullptr, b, seg[t + 2], w, a, at, m, kidx, precond,
                             relax, Z, s));
    }
    for (int t = s_every - 1; t >= 0; --t) {
      const int k = j * s_every + t;
      const int fin = (k == 0) ? 1 : 0;
      T* lo = (fin && g_x0) ? g_x0 : LB[pi];
      if constexpr (IsCplx<T>::value) {
        RICHM_TRY(launch_adjoint_cx<T>(op, lam, carry, seg[t + 1], seg[t], b, lo, CB[pi], w, a, at, m, k % m, fin,
                                       partials, acc, s));
      } else {
        if (precond == 2) RICHM_TRY(launch_ssor_apply<T>(op, lam, Z, U, relax, s));
        RICHM_TRY(launch_adjoint<T>(op, lam, U, carry, seg[t + 1], seg[t], b, lo, CB[pi], w, a, at, m, k % m,
                                    precond, fin, partials, acc, s));
      }
      lam = LB[pi];
      carry = CB[pi];
      pi ^= 1;
    }
  }
  const int cnt = op->batch * m;
  adjoint_finish_kernel<W><<<(cnt + 255) / 256, 256, 0, s>>>(acc, cnt, g_w, g_a, g_at, at == nullptr ? 1 : 0);
  RICHM_LAUNCH_CHECK("adjoint finish");
  return RICHM_OK;
}

}  // namespace richm

using namespace richm;

extern "C" {

richm_status richm_checkpoint_elems(const richm_operator* op, int K, int ckpt_every, size_t* elems) {
  clear_error();
  RICHM_ARG(op && elems, "null argument");
  RICHM_ARG(ckpt_every >= 1 && K >= 0 && K % ckpt_every == 0, "K must be a multiple of ckpt_every >= 1");
  *elems = (size_t)(K / ckpt_every + 1) * 2 * op->elems;
  return RICHM_OK;
}

// Real (Q1) states take every preconditioner; complex (Helmholtz) states none.
static richm_status check_adjoint_dtype(richm_dtype dtype, int precond) {
  RICHM_ARG(dtype == RICHM_F32 || dtype == RICHM_F64 || dtype == RICHM_C64 || dtype == RICHM_C128,
            "invalid dtype %d", (int)dtype);
  RICHM_ARG(!dtype_complex(dtype) || precond == 0, "complex (Helmholtz) differentiation takes no preconditioner");
  return RICHM_OK;
}

static richm_status check_precond(int precond, double relax) {
  RICHM_ARG(precond >= 0 && precond <= 2, "precond must be 0, 1 or 2");
  RICHM_ARG(precond != 2 || (relax > 0.0 && relax < 2.0), "SSOR relaxation factor must lie in (0, 2)");
  return RICHM_OK;
}

richm_status richm_forward_checkpointed(richm_operator* op, richm_dtype dtype, const void* x0, const void* b,
                                        const void* w, const void* alpha, const void* alpha_t, int m, int K,
                                        int ckpt_every, int precond, double relax, void* ckpts, void* xK,
                                        void* work, size_t work_bytes, void* stream) {
  clear_error();
  RICHM_ARG(op != nullptr, "null operator");
  RICHM_TRY(check_dtype_for_op(op, dtype));
  RICHM_TRY(check_adjoint_dtype(dtype, precond));
  RICHM_ARG(x0 && b && w && ckpts, "null argument");
  RICHM_ARG(m >= 1 && m <= 64, "m out of range");
  RICHM_ARG(ckpt_every >= 1 && K >= 0 && K % ckpt_every == 0, "K must be a multiple of ckpt_every >= 1");
  RICHM_ARG(alpha != nullptr || alpha_t == nullptr, "alpha_t given without alpha");
  RICHM_TRY(check_precond(precond, relax));
  const size_t need = 4 * a256(op->elems * dtype_size(dtype));
  RICHM_ARG(work != nullptr, "null workspace");
  if (work_bytes < need) return set_error(RICHM_ERR_NOMEM, "workspace %zu < %zu bytes", work_bytes, need);
  cudaStream_t s = (cudaStream_t)stream;
  switch (dtype) {
    case RICHM_F32:
      return forward_ckpt_t<float>(op, (const float*)x0, (const float*)b, (const float*)w, (const float*)alpha,
                                   (const float*)alpha_t, m, K, ckpt_every, precond, relax, (float*)ckpts,
                                   (float*)xK, work, s);
    case RICHM_F64:
      return forward_ckpt_t<double>(op, (const double*)x0, (const double*)b, (const double*)w, (const double*)alpha,
                                    (const double*)alpha_t, m, K, ckpt_every, precond, relax, (double*)ckpts,
                                    (double*)xK, work, s);
    case RICHM_C64:
      return forward_ckpt_t<cplx<float>>(op, (const cplx<float>*)x0, (const cplx<float>*)b, (const float*)w,
                                         (const float*)alpha, (const float*)alpha_t, m, K, ckpt_every, precond,
                                         relax, (cplx<float>*)ckpts, (cplx<float>*)xK, work, s);
    default:
      return forward_ckpt_t<cplx<double>>(op, (const cplx<double>*)x0, (const cplx<double>*)b, (const double*)w,
                                          (const double*)alpha, (const double*)alpha_t, m, K, ckpt_every, precond,
                                          relax, (cplx<double>*)ckpts, (cplx<double>*)xK, work, s);
  }
}

richm_status richm_adjoint_workspace(const richm_operator* op, richm_dtype dtype, int ckpt_every, size_t* bytes) {
  clear_error();
  RICHM_ARG(op && bytes, "null argument");
  RICHM_TRY(check_adjoint_dtype(dtype, 0));
  RICHM_ARG(ckpt_every >= 1, "ckpt_every < 1");
  auto* o = const_cast<richm_operator*>(op);
  const size_t fwd = 4 * a256(op->elems * dtype_size(dtype));
  const size_t adj = dtype == RICHM_F32   ? adjoint_ws<float>(o, ckpt_every)
                     : dtype == RICHM_F64 ? adjoint_ws<double>(o, ckpt_every)
                     : dtype == RICHM_C64 ? adjoint_ws<cplx<float>>(o, ckpt_every)
                                          : adjoint_ws<cplx<double>>(o, ckpt_every);
  *bytes = adj > fwd ? adj : fwd;
  return RICHM_OK;
}

richm_status richm_sweeps_adjoint(richm_operator* op, richm_dtype dtype, const void* ckpts, int ckpt_every,
                                  const void* b, const void* gK, const void* w, const void* alpha,
                                  const void* alpha_t, int m, int K, int precond, double relax, void* g_w,
                                  void* g_alpha, void* g_alpha_t, void* g_x0, void* work, size_t work_bytes,
                                  void* stream) {
  clear_error();
  RICHM_ARG(op != nullptr, "null operator");
  RICHM_TRY(check_dtype_for_op(op, dtype));
  RICHM_TRY(check_adjoint_dtype(dtype, precond));
  RICHM_ARG(ckpts && b && gK && w && work, "null argument");
  RICHM_ARG(m >= 1 && m <= 64, "m out of range");
  RICHM_ARG(ckpt_every >= 1 && K >= 1 && K % ckpt_every == 0, "K must be a positive multiple of ckpt_every");
  RICHM_ARG(alpha != nullptr || alpha_t == nullptr, "alpha_t given without alpha");
  RICHM_TRY(check_precond(precond, relax));
  cudaStream_t s = (cudaStream_t)stream;
  switch (dtype) {
    case RICHM_F32:
      return adjoint_t<float>(op, (const float*)ckpts, ckpt_every, (const float*)b, (const float*)gK,
                              (const float*)w, (const float*)alpha, (const float*)alpha_t, m, K, precond, relax,
                              (float*)g_w, (float*)g_alpha, (float*)g_alpha_t, (float*)g_x0, work, work_bytes, s);
    case RICHM_F64:
      return adjoint_t<double>(op, (const double*)ckpts, ckpt_every, (const double*)b, (const double*)gK,
                               (const double*)w, (const double*)alpha, (const double*)alpha_t, m, K, precond, relax,
                               (double*)g_w, (double*)g_alpha, (double*)g_alpha_t, (double*)g_x0, work, work_bytes,
                               s);
    case RICHM_C64:
      return adjoint_t<cplx<float>>(op, (const cplx<float>*)ckpts, ckpt_every, (const cplx<float>*)b,
                                    (const cplx<float>*)gK, (const float*)w, (const float*)alpha,
                                    (const float*)alpha_t, m, K, precond, relax, (float*)g_w, (float*)g_alpha,
                                    (float*)g_alpha_t, (cplx<float>*)g_x0, work, work_bytes, s);
    default:
      return adjoint_t<cplx<double>>(op, (const cplx<double>*)ckpts, ckpt_every, (const cplx<double>*)b,
                                     (const cplx<double>*)gK, (const double*)w, (const double*)alpha,
                                     (const double*)alpha_t, m, K, precond, relax, (double*)g_w, (double*)g_alpha,
                                     (double*)g_alpha_t, (cplx<double>*)g_x0, work, work_bytes, s);
  }
}

}  // extern "C"
