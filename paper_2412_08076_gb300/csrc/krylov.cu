// Restarted flexible GMRES for batches of complex Helmholtz instances, preconditioned
// by the library's NAG-Richardson(m) sweeps (Sec. 3.2: the single-level solvers as
// smoothers inside a preconditioner of FGMRES restarted every 20 iterations, Table 9).
//
// FGMRES (Saad 1993): r = b - A x, v_1 = r / |r|; step j: z_j = M(v_j), w = A z_j,
// orthogonalise w against v_1..v_j, v_{j+1} = w / |w|; after the cycle
// x += Z y with y minimising |beta e_1 - H y|. Every instance has its own Krylov
// space; the batch moves in lockstep and an instance whose residual estimate reached
// the tolerance stops taking Arnoldi steps.
//
// GB300 form: the Arnoldi basis V (complex128 by default) and the iterate (complex128)
// are in the padded layout; the preconditioner (K smoother sweeps on A z = v from z = 0) runs in
// complex64 (or complex128), and the z_j are kept in that type: the flexible variant
// only needs w = A z_j for the z_j it keeps, so storing them narrow is exact. The
// orthogonalisation is classical Gram-Schmidt applied twice (two passes of one
// batched dot kernel over all previous vectors and one update kernel), which reads
// each basis vector twice per step instead of j times as modified Gram-Schmidt
// would, with the same stability. Dots and norms are summed in FP64 per warp tile and
// then per instance in a fixed order. The small Hessenberg problems are reduced by
// complex Givens rotations, one thread per instance.
//
// With a complex64 basis (opts->basis) the cycle's vectors, A z_j, the Gram-Schmidt
// products and updates are complex64 on the FP32 pipe (GB300 runs FP64 at 1/64 of the
// FP32 rate, and the complex128 passes are bound by it); the dots and norms are summed
// over a warp tile's rows in FP32 and over the tiles in FP64. The residual that starts
// every cycle stays b - A x in FP64 with x in complex128, so each restart refines the
// solution against the exact residual (the cycles of 20 steps reduce it by far less
// than the complex64 rounding).
#include <algorithm>
#include <cmath>
#include <type_traits>
#include <vector>

#include "common.cuh"
#include "kernels.cuh"

namespace richm {

using C128 = cplx<double>;
using C64 = cplx<float>;
constexpr int kMaxRestart = 64;
// Rows of a Krylov warp tile: short tiles give the streaming kernels (updates, products,
// scaling, the solution update) four times the warps of the residual geometry, more
// loads in flight per SM.
constexpr int kKryRows = 4;
// the dots keep the residual's 16-row tiles: one block row per basis vector already
// gives them enough warps, and fewer partial sums to reduce
constexpr int kDotRows = 16;

// the basis type of the options: complex128 unless opts->basis is RICHM_C64
static bool narrow_basis(const richm_fgmres_opts* o) { return o->basis == RICHM_C64; }

template <typename T>
__device__ __forceinline__ cplx<T> conj_mul(cplx<T> a, cplx<T> b) {  // conj(a) * b
  return {a.re * b.re + a.im * b.im, a.re * b.im - a.im * b.re};
}
__device__ __forceinline__ double widen_d(float v) { return f32_to_f64_exact(v); }
__device__ __forceinline__ double widen_d(double v) { return v; }
__device__ __forceinline__ double2 c2d(C128 v) { return make_double2(v.re, v.im); }
__device__ __forceinline__ C128 d2c(double2 v) { return {v.x, v.y}; }

// partials[i * ntiles + t] = sum over warp tile t of conj(V_i) w (32 columns x kDotRows
// rows of complex128; the padding columns and halo rows are zero in both)
template <typename VB>
__global__ void __launch_bounds__(kWarpsPerBlock * 32)
    kry_dot_kernel(const Inst* insts, const Tile* tiles, int ntiles, const VB* __restrict__ V, size_t vstride,
                   const VB* __restrict__ w, double2* __restrict__ partials, const int* __restrict__ active) {
  using T = typename RealOf<VB>::type;
  const int lane = threadIdx.x & 31;
  const int wt = blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
  if (wt >= ntiles) return;
  const int i = blockIdx.y;
  const Tile t = tiles[wt];
  T sre = T(0), sim = T(0);  // this lane's column of the tile (at most kDotRows terms)
  if (!active || active[t.inst]) {
    const Inst& I = insts[t.inst];
    const int c0 = t.tx * 32 + lane;
    if (c0 < I.n) {
      const int r0 = t.ty * kDotRows + 1;
      const int r1 = min(r0 + kDotRows - 1, I.n);
      const VB* vi = V + (size_t)i * vstride + I.off + c0;
      const VB* wb = w + I.off + c0;
      // eight rows' loads issued together at a time (the tile's rows are independent)
      constexpr int kBatch = 8;
#pragma unroll
      for (int h = 0; h < kDotRows; h += kBatch) {
        VB va[kBatch], wa[kBatch];
#pragma unroll
        for (int q = 0; q < kBatch; ++q) {
          const long long o = (long long)(r0 + h + q) * I.pitch;
          const bool ok = r0 + h + q <= r1;
          va[q] = ok ? vi[o] : VB{T(0), T(0)};
          wa[q] = ok ? wb[o] : VB{T(0), T(0)};
        }
#pragma unroll
        for (int q = 0; q < kBatch; ++q) {
          const VB p = conj_mul(va[q], wa[q]);
          sre += p.re;
          sim += p.im;
        }
      }
    }
  }
  const double dre = warp_sum(widen_d(sre));
  const double dim = warp_sum(widen_d(sim));
  if (lane == 0) partials[(size_t)i * ntiles + wt] = make_double2(dre, dim);
}

// h[b * ldh + i] = sum over instance b's tiles of partials[i * ntiles + t] (fixed order)
constexpr int kReduceThreads = 256;
__global__ void __launch_bounds__(kReduceThreads)
    kry_reduce_kernel(const double2* __restrict__ partials, const int* __restrict__ inst_begin, int ntiles,
                      int batch, double2* __restrict__ h, int ldh) {
  __shared__ double2 part[kReduceThreads / 32];
  const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
  const int b = blockIdx.x, i = blockIdx.y;
  if (b >= batch) return;
  double sre = 0.0, sim = 0.0;
  for (int t = inst_begin[b] + threadIdx.x; t < inst_begin[b + 1]; t += kReduceThreads) {
    const double2 p = partials[(size_t)i * ntiles + t];
    sre += p.x;
    sim += p.y;
  }
  sre = warp_sum(sre);
  sim = warp_sum(sim);
  if (lane == 0) part[wi] = make_double2(sre, sim);
  __syncthreads();
  if (threadIdx.x == 0) {
    double2 acc = make_double2(0.0, 0.0);
    for (int q = 0; q < kReduceThreads / 32; ++q) {
      acc.x += part[q].x;
      acc.y += part[q].y;
    }
    h[(size_t)b * ldh + i] = acc;
  }
}

// w -= sum_{i < nv} h[b][i] V_i over the tile; optionally the tile's sum |w|^2 in
// partials (as (|w|^2, 0), the layout of the residual norm partials)
// (complex64 basis: the coefficients narrowed once per warp into shared memory)
template <typename VB>
__global__ void __launch_bounds__(kWarpsPerBlock * 32)
    kry_update_kernel(const Inst* insts, const Tile* tiles, int ntiles, const VB* __restrict__ V, size_t vstride,
                      int nv, const double2* __restrict__ h, int ldh, VB* __restrict__ w,
                      double2* __restrict__ partials, const int* __restrict__ active) {
  using T = typename RealOf<VB>::type;
  constexpr bool NARROW = std::is_same<T, float>::value;
  __shared__ C64 hs[kWarpsPerBlock][kMaxRestart + 1];
  const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
  const int wt = blockIdx.x * kWarpsPerBlock + wi;
  if (wt >= ntiles) return;
  const Tile t = tiles[wt];
  T s2 = T(0);
  if (!active || active[t.inst]) {
    const Inst& I = insts[t.inst];
    const double2* hb = h + (size_t)t.inst * ldh;
    if constexpr (NARROW) {
      for (int i = lane; i < nv; i += 32) hs[wi][i] = C64{f64_to_f32_rn(hb[i].x), f64_to_f32_rn(hb[i].y)};
      __syncwarp();
    }
    const int c0 = t.tx * 32 + lane;
    if (c0 < I.n) {
      const int r0 = t.ty * kKryRows + 1;
      const int r1 = min(r0 + kKryRows - 1, I.n);
      VB* wb = w + I.off;
      for (int r = r0; r <= r1; ++r) {
        const long long o = (long long)r * I.pitch + c0;
        // two independent sums (even and odd vectors) halve the dependent chain
        VB acc = wb[o], acc2{T(0), T(0)};
        int i = 0;
#pragma unroll 2
        for (; i + 1 < nv; i += 2) {
          VB h0, h1;
          if constexpr (NARROW) {
            h0 = hs[wi][i];
            h1 = hs[wi][i + 1];
          } else {
            h0 = d2c(hb[i]);
            h1 = d2c(hb[i + 1]);
          }
          const VB v0 = V[(size_t)i * vstride + I.off + o], v1 = V[(size_t)(i + 1) * vstride + I.off + o];
          acc = acc - cmul(h0, v0);
          acc2 = acc2 + cmul(h1, v1);
        }
        if (i < nv) {
          VB h0;
          if constexpr (NARROW) h0 = hs[wi][i];
          else h0 = d2c(hb[i]);
          acc = acc - cmul(h0, V[(size_t)i * vstride + I.off + o]);
        }
        acc = acc - acc2;
        wb[o] = acc;
        s2 += acc.re * acc.re + acc.im * acc.im;
      }
    }
  }
  if (partials) {
    const double d2 = warp_sum(widen_d(s2));
    if (lane == 0) partials[wt] = make_double2(d2, 0.0);
  }
}

// w = A z in complex64 arithmetic over rows 1..n (columns >= n written as zero), one
// column per lane (the complex128 geometry), for the complex64 basis.
template <typename EZ>
__global__ void __launch_bounds__(kWarpsPerBlock * 32)
    kry_apply_kernel(const Inst* insts, const Tile* tiles, int ntiles, const EZ* __restrict__ z,
                     C64* __restrict__ out, const int* __restrict__ active) {
  const int lane = threadIdx.x & 31;
  const int wt = blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
  if (wt >= ntiles) return;
  const Tile t = tiles[wt];
  if (active && !active[t.inst]) return;
  const Inst& I = insts[t.inst];
  const int n = I.n, pitch = I.pitch;
  const int c0 = t.tx * 32 + lane;
  const bool live = c0 < pitch;
  const int r0 = t.ty * kKryRows + 1;
  const int r1 = min(r0 + kKryRows - 1, n);
  const EZ* zb = z + I.off;
  auto load = [&](int pr, RowT<C64, 1>& Y) {
    const bool in = (pr >= 1) && (pr <= n);
    const long long ro = (long long)pr * pitch;
    C64 v{0.f, 0.f};
    if (in && live) v = C64{(float)zb[ro + c0].re, (float)zb[ro + c0].im};
    Y.y[0] = v;
    C64 le{0.f, 0.f}, re{0.f, 0.f};
    if (in) {
      if (lane == 0 && c0 > 0) le = C64{(float)zb[ro + c0 - 1].re, (float)zb[ro + c0 - 1].im};
      if (lane == 31 && c0 + 1 < pitch) re = C64{(float)zb[ro + c0 + 1].re, (float)zb[ro + c0 + 1].im};
    }
    row_neighbours<C64, 1>(Y, lane, le, re);
  };
  RowT<C64, 1> U, C, D;
  load(r0 - 1, U);
  load(r0, C);
  for (int r = r0; r <= r1; ++r) {
    load(r + 1, D);
    C64 Ax[1];
    apply_fd5<C64, 1, float>(U, C, D, r - 1, c0, n, (float)I.c, (float)I.ax, (float)I.abc_re, (float)I.abc_im,
                             (float)I.sp_im, (float)I.sp_iw, Ax);
    if (live) out[I.off + (long long)r * pitch + c0] = c0 < n ? Ax[0] : C64{0.f, 0.f};
    U = C;
    C = D;
  }
}

// v = w / nrm[b] over rows 1..n (columns >= n stay zero), and the same narrowed to
// complex64 in vn when given
template <typename VB>
__global__ void __launch_bounds__(kWarpsPerBlock * 32)
    kry_scale_kernel(const Inst* insts, const Tile* tiles, int ntiles, const VB* __restrict__ w,
                     const double* __restrict__ nrm, VB* __restrict__ v, C64* __restrict__ vn,
                     const int* __restrict__ active) {
  using T = typename RealOf<VB>::type;
  const int lane = threadIdx.x & 31;
  const int wt = blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
  if (wt >= ntiles) return;
  const Tile t = tiles[wt];
  if (active && !active[t.inst]) return;
  const Inst& I = insts[t.inst];
  const int c0 = t.tx * 32 + lane;
  if (c0 >= I.pitch) return;
  const double sd = nrm[t.inst] > 0.0 ? 1.0 / nrm[t.inst] : 0.0;
  T s;
  if constexpr (std::is_same<T, float>::value) s = f64_to_f32_rn(sd);
  else s = sd;
  const int r0 = t.ty * kKryRows + 1;
  const int r1 = min(r0 + kKryRows - 1, I.n);
  for (int r = r0; r <= r1; ++r) {
    const long long o = I.off + (long long)r * I.pitch + c0;
    const VB q = c0 < I.n ? s * w[o] : VB{T(0), T(0)};
    v[o] = q;
    if (vn) vn[o] = C64{(float)q.re, (float)q.im};
  }
}

// Per-instance state of the small least-squares problems.
struct KryState {
  double2* H;       // [batch][R][R + 1]: column j of the rotated Hessenberg matrix
  double2* hcol;    // [batch][R + 1]: first Gram-Schmidt pass's coefficients
  double2* hcol2;   // [batch][R + 1]: second pass's
  double* cs;       // [batch][R]
  double2* sn;      // [batch][R]
  double2* g;       // [batch][R + 1]
  double2* y;       // [batch][R]
  double* beta;     // [batch] residual norm at the cycle's start
  double* bnorm;    // [batch]
  double* wnorm;    // [batch]
  double2* wn2;     // [batch]: (|w|^2, 0) after the second Gram-Schmidt pass
  double* rnorm;    // [batch] true residual norm
  int* iters;       // [batch] Arnoldi steps taken
  int* jend;        // [batch] steps of the current cycle
  int* in_cycle;    // [batch] 1 while the instance takes Arnoldi steps in this cycle
  int* done;        // [batch] 1 once converged
  int* count;       // [1]
};

// Start of a cycle: g = beta e_1; an instance continues if beta > tol |b| and it has
// steps left.
__global__ void kry_cycle_start_kernel(KryState S, int batch, int R, double tol, int max_iters) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= batch) return;
  for (int i = 0; i <= R; ++i) S.g[(size_t)b * (R + 1) + i] = make_double2(0.0, 0.0);
  S.g[(size_t)b * (R + 1)] = make_double2(S.beta[b], 0.0);
  S.jend[b] = 0;
  const bool conv = S.beta[b] <= tol * S.bnorm[b];
  if (conv) S.done[b] = 1;
  const int go = !conv && !S.done[b] && S.iters[b] < max_iters;
  S.in_cycle[b] = go;
  if (go) atomicAdd(S.count, 1);
}

// Step j of every instance still in its cycle: column j of H from the two
// Gram-Schmidt passes and |w|, the previous rotations, a new rotation, g, and the
// residual estimate |g_{j+1}|; the instance leaves the cycle when the estimate reaches
// tol |b|, after R steps, at max_iters, or on a breakdown (|w| = 0).
__global__ void kry_givens_kernel(KryState S, int batch, int R, int j, double tol, int max_iters) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= batch || !S.in_cycle[b]) return;
  const size_t ld = (size_t)(R + 1);
  double2* Hc = S.H + ((size_t)b * R + j) * ld;
  for (int i = 0; i <= j; ++i) {
    const double2 p = S.hcol[b * ld + i], q = S.hcol2[b * ld + i];
    Hc[i] = make_double2(p.x + q.x, p.y + q.y);
  }
  const double hn = sqrt(S.wn2[b].x);
  S.wnorm[b] = hn;
  Hc[j + 1] = make_double2(hn, 0.0);
  for (int i = 0; i < j; ++i) {  // earlier rotations
    const double c = S.cs[(size_t)b * R + i];
    const C128 s = d2c(S.sn[(size_t)b * R + i]);
    const C128 a = d2c(Hc[i]), e = d2c(Hc[i + 1]);
    const C128 na = c * a + cmul(s, e);
    const C128 ne = c * e - cmul(C128{s.re, -s.im}, a);
    Hc[i] = c2d(na);
    Hc[i + 1] = c2d(ne);
  }
  // rotation zeroing the real entry hn below a = H[j][j]
  const C128 a = d2c(Hc[j]);
  const double aa = hypot(a.re, a.im);
  double c;
  C128 s;
  if (aa == 0.0) {
    c = 0.0;
    s = {1.0, 0.0};
    Hc[j] = make_double2(hn, 0.0);
  } else {
    const double t = hypot(aa, hn);
    c = aa / t;
    const C128 ph = {a.re / aa, a.im / aa};
    s = (hn / t) * ph;
    Hc[j] = c2d(t * ph);
  }
  Hc[j + 1] = make_double2(0.0, 0.0);
  S.cs[(size_t)b * R + j] = c;
  S.sn[(size_t)b * R + j] = c2d(s);
  const C128 gj = d2c(S.g[b * ld + j]);
  S.g[b * ld + j] = c2d(c * gj);
  const C128 gn = -1.0 * cmul(C128{s.re, -s.im}, gj);
  S.g[b * ld + j + 1] = c2d(gn);
  S.iters[b] += 1;
  S.jend[b] = j + 1;
  const double est = hypot(gn.re, gn.im);
  const bool conv = est <= tol * S.bnorm[b];
  if (conv || j + 1 == R || S.iters[b] >= max_iters || hn == 0.0) {
    S.in_cycle[b] = 0;
  } else {
    atomicAdd(S.count, 1);
  }
}

// y = R^{-1} g over the cycle's steps (back substitution in the rotated H)
__global__ void kry_backsolve_kernel(KryState S, int batch, int R) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= batch) return;
  const size_t ld = (size_t)(R + 1);
  const int J = S.jend[b];
  for (int i = J - 1; i >= 0; --i) {
    C128 acc = d2c(S.g[b * ld + i]);
    for (int k = i + 1; k < J; ++k)
      acc = acc - cmul(d2c(S.H[((size_t)b * R + k) * ld + i]), d2c(S.y[(size_t)b * R + k]));
    const C128 d = d2c(S.H[((size_t)b * R + i) * ld + i]);
    S.y[(size_t)b * R + i] = c2d(cdiv(acc, d));
  }
}

// x += sum_{i < jend[b]} y[b][i] Z_i (Z in the preconditioner's type). NARROW (the
// complex64 basis): the sum formed in complex64 with y narrowed once per warp, then
// added to x in FP64; the next cycle's FP64 residual corrects its rounding.
template <typename EZ, bool NARROW>
__global__ void __launch_bounds__(kWarpsPerBlock * 32)
    kry_xupdate_kernel(const Inst* insts, const Tile* tiles, int ntiles, const EZ* __restrict__ Z, size_t zstride,
                       KryState S, int R, C128* __restrict__ x) {
  __shared__ C64 ys[kWarpsPerBlock][kMaxRestart];
  const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
  const int wt = blockIdx.x * kWarpsPerBlock + wi;
  if (wt >= ntiles) return;
  const Tile t = tiles[wt];
  const int J = S.jend[t.inst];
  if (J == 0) return;
  const Inst& I = insts[t.inst];
  const double2* yb = S.y + (size_t)t.inst * R;
  if constexpr (NARROW) {
    for (int i = lane; i < J; i += 32) ys[wi][i] = C64{f64_to_f32_rn(yb[i].x), f64_to_f32_rn(yb[i].y)};
    __syncwarp();
  }
  const int c0 = t.tx * 32 + lane;
  if (c0 >= I.n) return;
  const int r0 = t.ty * kKryRows + 1;
  const int r1 = min(r0 + kKryRows - 1, I.n);
  for (int r = r0; r <= r1; ++r) {
    const long long o = I.off + (long long)r * I.pitch + c0;
    if constexpr (NARROW) {
      C64 acc{0.f, 0.f};
#pragma unroll 4
      for (int i = 0; i < J; ++i) {
        const EZ z = Z[(size_t)i * zstride + o];
        acc = acc + cmul(ys[wi][i], C64{(float)z.re, (float)z.im});
      }
      const C128 xo = x[o];
      x[o] = C128{xo.re + f32_to_f64_exact(acc.re), xo.im + f32_to_f64_exact(acc.im)};
    } else {
      C128 acc = x[o];
      for (int i = 0; i < J; ++i) {
        const EZ z = Z[(size_t)i * zstride + o];
        acc = acc + cmul(d2c(yb[i]), C128{(double)z.re, (double)z.im});
      }
      x[o] = acc;
    }
  }
}

static size_t a256(size_t v) { return (v + 255) / 256 * 256; }

struct KryLayout {
  size_t V, Z, W, vin, zp, sw, dots, norms, H, hcol, hcol2, cs, sn, g, y, beta, bnorm, wnorm, wn2, rnorm, iters, jend,
      in_cycle, done, count, total;
};

static richm_status kry_layout(richm_operator* op, const richm_fgmres_opts* o, KryLayout* L) {
  const size_t el = op->elems;
  const size_t es = o->inner == RICHM_C64 ? 8 : 16;
  const size_t vs = narrow_basis(o) ? 8 : 16;  // basis element
  const size_t R = (size_t)o->restart, B = (size_t)op->batch;
  int nt_res = 0;
  RICHM_TRY(residual_tiles<C128>(op, &nt_res));
  const TileMap* tm = nullptr;
  RICHM_TRY(get_tiles(op, 32, kKryRows, &tm));
  const size_t nt = (size_t)tm->ntiles;
  RICHM_TRY(get_tiles(op, 32, kDotRows, &tm));
  const size_t nt_dot = (size_t)tm->ntiles;
  size_t sw = 0;
  RICHM_TRY(richm_sweeps_workspace(op, (richm_dtype)o->inner, &sw));
  size_t p = 0;
  auto take = [&](size_t bytes) {
    const size_t at = p;
    p += a256(bytes);
    return at;
  };
  L->V = take((R + 1) * a256(el * vs));
  L->Z = take(R * a256(el * es));
  L->W = take(el * vs);
  L->vin = take(o->inner == RICHM_C64 && !narrow_basis(o) ? el * 8 : 0);
  L->zp = take(el * es);
  L->sw = take(sw);
  L->dots = take((R + 1) * nt_dot * sizeof(double2));
  L->norms = take(std::max(nt, (size_t)nt_res) * sizeof(double2));  // the residual's partials or the Krylov tiles'

  L->H = take(B * R * (R + 1) * sizeof(double2));
  L->hcol = take(B * (R + 1) * sizeof(double2));
  L->hcol2 = take(B * (R + 1) * sizeof(double2));
  L->cs = take(B * R * sizeof(double));
  L->sn = take(B * R * sizeof(double2));
  L->g = take(B * (R + 1) * sizeof(double2));
  L->y = take(B * R * sizeof(double2));
  L->beta = take(B * sizeof(double));
  L->bnorm = take(B * sizeof(double));
  L->wnorm = take(B * sizeof(double));
  L->wn2 = take(B * sizeof(double2));
  L->rnorm = take(B * sizeof(double));
  L->iters = take(B * sizeof(int));
  L->jend = take(B * sizeof(int));
  L->in_cycle = take(B * sizeof(int));
  L->done = take(B * sizeof(int));
  L->count = take(sizeof(int));
  L->total = p;
  return RICHM_OK;
}

static richm_status check_fgmres(const richm_operator* op, const richm_fgmres_opts* o) {
  RICHM_ARG(op != nullptr && o != nullptr, "null operator or options");
  RICHM_ARG(o->restart >= 1 && o->restart <= kMaxRestart, "restart = %d out of range [1, 64]", o->restart);
  RICHM_ARG(o->tol >= 0.0, "tol < 0");
  RICHM_ARG(o->max_iters >= 0, "max_iters < 0");
  RICHM_ARG(o->m >= 1 && o->m <= 64, "m = %d out of range [1, 64]", o->m);
  RICHM_ARG(o->sweeps >= 0, "sweeps < 0");
  RICHM_ARG(o->inner == RICHM_C64 || o->inner == RICHM_C128, "inner must be RICHM_C64 or RICHM_C128");
  RICHM_ARG(o->precond == 0 || o->precond == 1, "precond must be 0 or 1");
  RICHM_ARG(o->basis == 0 || o->basis == RICHM_C128 || o->basis == RICHM_C64,
            "basis must be 0 (complex128), RICHM_C128 or RICHM_C64");
  RICHM_ARG(!narrow_basis(o) || o->inner == RICHM_C64, "a complex64 basis needs inner RICHM_C64");
  for (int b = 0; b < op->batch; ++b)
    if (op->h_inst[b].kind == RICHM_ANISO_Q1)
      return set_error(RICHM_ERR_UNSUPPORTED, "richm_fgmres takes Helmholtz instances (instance %d is Q1)", b);
  return RICHM_OK;
}

template <typename EZ, typename VB>
static richm_status fgmres_t(richm_operator* op, const C128* b, C128* x, const void* w, const void* alpha,
                             const void* alpha_t, const richm_fgmres_opts* o, richm_fgmres_info* info, char* work,
                             const KryLayout& L, cudaStream_t s) {
  constexpr bool NB = std::is_same<VB, C64>::value;  // complex64 basis
  const int R = o->restart, B = op->batch;
  const size_t el = op->elems;
  const size_t es = sizeof(EZ);
  const size_t vstride = a256(el * sizeof(VB)) / sizeof(VB), zstride = a256(el * es) / es;
  VB* V = reinterpret_cast<VB*>(work + L.V);
  EZ* Z = reinterpret_cast<EZ*>(work + L.Z);
  VB* W = reinterpret_cast<VB*>(work + L.W);
  C64* vin = (o->inner == RICHM_C64 && !NB) ? reinterpret_cast<C64*>(work + L.vin) : nullptr;
  EZ* zp = reinterpret_cast<EZ*>(work + L.zp);
  void* sw = work + L.sw;
  size_t swb = 0;
  RICHM_TRY(richm_sweeps_workspace(op, (richm_dtype)o->inner, &swb));
  double2* dots = reinterpret_cast<double2*>(work + L.dots);
  double2* norms = reinterpret_cast<double2*>(work + L.norms);
  KryState S{reinterpret_cast<double2*>(work + L.H),     reinterpret_cast<double2*>(work + L.hcol),
             reinterpret_cast<double2*>(work + L.hcol2), reinterpret_cast<double*>(work + L.cs),
             reinterpret_cast<double2*>(work + L.sn),    reinterpret_cast<double2*>(work + L.g),
             reinterpret_cast<double2*>(work + L.y),     reinterpret_cast<double*>(work + L.beta),
             reinterpret_cast<double*>(work + L.bnorm),  reinterpret_cast<double*>(work + L.wnorm),
             reinterpret_cast<double2*>(work + L.wn2),   reinterpret_cast<double*>(work + L.rnorm),  reinterpret_cast<int*>(work + L.iters),
             reinterpret_cast<int*>(work + L.jend),      reinterpret_cast<int*>(work + L.in_cycle),
             reinterpret_cast<int*>(work + L.done),      reinterpret_cast<int*>(work + L.count)};
  const TileMap* tm = nullptr;
  RICHM_TRY(get_tiles(op, 32, kKryRows, &tm));  // 32 columns (one per lane) x kKryRows rows
  const int nt = tm->ntiles;
  const TileMap* td = nullptr;  // the dots' 16-row tiles
  RICHM_TRY(get_tiles(op, 32, kDotRows, &td));
  const int ntd = td->ntiles;
  const int dblocks = (ntd + kWarpsPerBlock - 1) / kWarpsPerBlock;
  const int tblocks = (nt + kWarpsPerBlock - 1) / kWarpsPerBlock;
  const int ithr = 128, iblocks = (B + ithr - 1) / ithr;
  // the buffers' halo rows and padding must be zero: clear everything the kernels read
  RICHM_CUDA_TRY(cudaMemsetAsync(work, 0, L.total, s));
  int h_count = 0;
  auto read_count = [&]() -> richm_status {
    RICHM_CUDA_TRY(cudaMemcpyAsync(&h_count, S.count, sizeof(int), cudaMemcpyDeviceToHost, s));
    RICHM_CUDA_TRY(cudaStreamSynchronize(s));
    return RICHM_OK;
  };
  // the library's choice of pass length (complex64 without preconditioner: fused passes
  // of four sweeps, on tiles short enough to spread a small batch over the GPU)
  richm_sweep_opts so{o->m, 0, o->precond, 0, 1.0};
  for (int cycle = 0;; ++cycle) {
    // r = b - A x, beta = |r| (and |b| at the first cycle from the same pass)
    if constexpr (NB) RICHM_TRY((launch_residual_to<C128, C64>(op, x, b, W, norms, nullptr, s, false)));
    else RICHM_TRY(launch_residual<C128>(op, x, b, W, norms, s));
    RICHM_TRY(launch_norm_reduce(op, 1, norms, S.beta, cycle == 0 ? S.bnorm : nullptr, nullptr, s));
    RICHM_CUDA_TRY(cudaMemsetAsync(S.count, 0, sizeof(int), s));
    kry_cycle_start_kernel<<<iblocks, ithr, 0, s>>>(S, B, R, o->tol, o->max_iters);
    RICHM_LAUNCH_CHECK("FGMRES cycle start");
    RICHM_TRY(read_count());
    if (h_count == 0) break;
    kry_scale_kernel<VB><<<tblocks, kWarpsPerBlock * 32, 0, s>>>(op->d_inst, tm->d_tiles, nt, W, S.beta, V, vin,
                                                                 S.in_cycle);
    RICHM_LAUNCH_CHECK("FGMRES scale");
    for (int j = 0; j < R; ++j) {
      // z_j = M(v_j): K smoother sweeps on A z = v_j from z = 0
      EZ* zj = Z + (size_t)j * zstride;
      RICHM_CUDA_TRY(cudaMemsetAsync(zj, 0, el * es, s));
      RICHM_CUDA_TRY(cudaMemsetAsync(zp, 0, el * es, s));
      const void* rhs = vin ? (const void*)vin : (const void*)(V + (size_t)j * vstride);
      if (o->sweeps > 0)
        RICHM_TRY(richm_apply_sweeps(op, (richm_dtype)o->inner, zj, alpha ? zp : nullptr, rhs, w, alpha, alpha_t,
                                     o->sweeps, &so, sw, swb, s));
      else
        RICHM_CUDA_TRY(cudaMemcpyAsync(zj, rhs, el * es, cudaMemcpyDeviceToDevice, s));
      // w = A z_j, then two Gram-Schmidt passes against v_0..v_j
      if constexpr (NB) {
        kry_apply_kernel<EZ><<<tblocks, kWarpsPerBlock * 32, 0, s>>>(op->d_inst, tm->d_tiles, nt, zj, W, S.in_cycle);
        RICHM_LAUNCH_CHECK("FGMRES stencil");
      } else {
        RICHM_TRY((launch_apply_to<EZ, C128>(op, zj, W, s)));
      }
      for (int pass = 0; pass < 2; ++pass) {
        kry_dot_kernel<VB><<<dim3(dblocks, j + 1), kWarpsPerBlock * 32, 0, s>>>(op->d_inst, td->d_tiles, ntd, V,
                                                                               vstride, W, dots, S.in_cycle);
        RICHM_LAUNCH_CHECK("FGMRES dots");
        double2* hc = pass == 0 ? S.hcol : S.hcol2;
        kry_reduce_kernel<<<dim3(B, j + 1), kReduceThreads, 0, s>>>(dots, td->d_inst_begin, ntd, B, hc, R + 1);
        RICHM_LAUNCH_CHECK("FGMRES dot reduction");
        kry_update_kernel<VB><<<tblocks, kWarpsPerBlock * 32, 0, s>>>(op->d_inst, tm->d_tiles, nt, V, vstride,
                                                                      j + 1, hc, R + 1, W,
                                                                      pass == 1 ? norms : nullptr, S.in_cycle);
        RICHM_LAUNCH_CHECK("FGMRES update");
      }
      kry_reduce_kernel<<<dim3(B, 1), kReduceThreads, 0, s>>>(norms, tm->d_inst_begin, nt, B, S.wn2, 1);
      RICHM_LAUNCH_CHECK("FGMRES norm reduction");
      RICHM_CUDA_TRY(cudaMemsetAsync(S.count, 0, sizeof(int), s));
      kry_givens_kernel<<<iblocks, ithr, 0, s>>>(S, B, R, j, o->tol, o->max_iters);
      RICHM_LAUNCH_CHECK("FGMRES rotations");
      if (j + 1 < R) {
        kry_scale_kernel<VB><<<tblocks, kWarpsPerBlock * 32, 0, s>>>(op->d_inst, tm->d_tiles, nt, W, S.wnorm,
                                                                     V + (size_t)(j + 1) * vstride, vin,
                                                                     S.in_cycle);
        RICHM_LAUNCH_CHECK("FGMRES scale");
      }
      // the host looks at the count of instances still in the cycle every fourth step
      // (each look is a round trip that idles the GPU); steps taken after every instance
      // left the cycle change nothing, since every kernel but the preconditioner's skips
      // the instances outside it
      if ((j & 3) == 3 || j + 1 == R) {
        RICHM_TRY(read_count());
        if (h_count == 0) break;
      }
    }
    kry_backsolve_kernel<<<iblocks, ithr, 0, s>>>(S, B, R);
    RICHM_LAUNCH_CHECK("FGMRES back substitution");
    kry_xupdate_kernel<EZ, NB><<<tblocks, kWarpsPerBlock * 32, 0, s>>>(op->d_inst, tm->d_tiles, nt, Z, zstride, S, R,
                                                                       x);
    RICHM_LAUNCH_CHECK("FGMRES solution update");
  }
  // the final true residual of every instance
  if constexpr (NB) RICHM_TRY((launch_residual_to<C128, C64>(op, x, b, W, norms, nullptr, s, false)));
  else RICHM_TRY(launch_residual<C128>(op, x, b, W, norms, s));
  RICHM_TRY(launch_norm_reduce(op, 1, norms, S.rnorm, nullptr, nullptr, s));
  std::vector<double> hr(B), hb(B);
  std::vector<int> hi(B), hd(B);
  RICHM_CUDA_TRY(cudaMemcpyAsync(hr.data(), S.rnorm, B * sizeof(double), cudaMemcpyDeviceToHost, s));
  RICHM_CUDA_TRY(cudaMemcpyAsync(hb.data(), S.bnorm, B * sizeof(double), cudaMemcpyDeviceToHost, s));
  RICHM_CUDA_TRY(cudaMemcpyAsync(hi.data(), S.iters, B * sizeof(int), cudaMemcpyDeviceToHost, s));
  RICHM_CUDA_TRY(cudaMemcpyAsync(hd.data(), S.done, B * sizeof(int), cudaMemcpyDeviceToHost, s));
  RICHM_CUDA_TRY(cudaStreamSynchronize(s));
  richm_status st = RICHM_OK;
  for (int i = 0; i < B; ++i) {
    info[i].iters = hi[i];
    info[i].rel_res = hb[i] > 0.0 ? hr[i] / hb[i] : hr[i];
    if (!std::isfinite(info[i].rel_res)) {
      info[i].status = RICHM_ERR_DIVERGED;
      st = RICHM_ERR_DIVERGED;
    } else if (!hd[i] && info[i].rel_res > o->tol) {
      info[i].status = RICHM_ERR_NOT_CONVERGED;
      if (st == RICHM_OK) st = RICHM_ERR_NOT_CONVERGED;
    } else {
      info[i].status = RICHM_OK;
    }
  }
  return st;
}

}  // namespace richm

using namespace richm;

extern "C" {

richm_status richm_fgmres_workspace(const richm_operator* op, const richm_fgmres_opts* o, size_t* bytes) {
  clear_error();
  RICHM_TRY(check_fgmres(op, o));
  RICHM_ARG(bytes != nullptr, "null output");
  KryLayout L;
  RICHM_TRY(kry_layout(const_cast<richm_operator*>(op), o, &L));
  *bytes = L.total;
  return RICHM_OK;
}

richm_status richm_fgmres(richm_operator* op, const void* b, void* x, const void* w, const void* alpha,
                          const void* alpha_t, const richm_fgmres_opts* o, richm_fgmres_info* info, void* work,
                          size_t work_bytes, void* stream) {
  clear_error();
  RICHM_TRY(check_fgmres(op, o));
  RICHM_ARG(b != nullptr && x != nullptr && info != nullptr, "null b, x or info");
  RICHM_ARG(o->sweeps == 0 || w != nullptr, "null smoother weights");
  RICHM_ARG(alpha != nullptr || alpha_t == nullptr, "alpha_t given without alpha");
  KryLayout L;
  RICHM_TRY(kry_layout(op, o, &L));
  RICHM_ARG(work != nullptr, "null workspace");
  if (work_bytes < L.total) return set_error(RICHM_ERR_NOMEM, "workspace %zu < %zu bytes", work_bytes, L.total);
  cudaStream_t s = (cudaStream_t)stream;
  char* wk = reinterpret_cast<char*>(work);
  if (narrow_basis(o))
    return fgmres_t<C64, C64>(op, (const C128*)b, (C128*)x, w, alpha, alpha_t, o, info, wk, L, s);
  if (o->inner == RICHM_C64)
    return fgmres_t<C64, C128>(op, (const C128*)b, (C128*)x, w, alpha, alpha_t, o, info, wk, L, s);
  return fgmres_t<C128, C128>(op, (const C128*)b, (C128*)x, w, alpha, alpha_t, o, info, wk, L, s);
}

}  // extern "C"
