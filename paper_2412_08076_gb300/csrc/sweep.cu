// Forward sweeps of the Richardson(m) family (Table 1, eq. 17).
//
// One launch performs one sweep of
//   y       = x_k + at_i (x_k - x_{k-1})
//   x_{k+1} = x_k + a_i (x_k - x_{k-1}) + w_i B^{-1} (b - A y)
// over every tile of every active instance. The kernel is HBM-bound (per unknown:
// read x_k, x_{k-1}, b, write x_{k+1}); each warp streams R rows of a 32-lane x
// 16-byte column block, keeping the stencil's three rows of y in registers, so
// every input row is read once per warp tile and neighbours across lanes come
// from warp shuffles.
#include <type_traits>

#include "common.cuh"
#include "kernels.cuh"

namespace richm {

template <typename E>
struct SweepArgs {
  using S = typename RealOf<E>::type;
  const Inst* insts;
  const Tile* tiles;
  int ntiles;
  const E* x;
  const E* xp;
  const E* b;
  E* out;
  const S* w;
  const S* a;
  const S* at;
  int m;
  int kidx;
  const int* active;
};

template <typename E, bool MOM, bool PRE>
__global__ void __launch_bounds__(kWarpsPerBlock * 32, 4) sweep1_kernel(const SweepArgs<E> A) {
  using S = typename RealOf<E>::type;
  constexpr int VW = VecWidth<E>::value;
  constexpr bool CPLX = IsCplx<E>::value;
  const int lane = threadIdx.x & 31;
  const int wt = blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
  if (wt >= A.ntiles) return;
  const Tile t = A.tiles[wt];
  if (A.active && A.active[t.inst] == 0) return;
  const Inst& I = A.insts[t.inst];
  const int n = I.n, pitch = I.pitch;
  const int cidx = t.inst * A.m + A.kidx;
  const S wi = A.w[cidx];
  S ai = 0, ati = 0;
  if (MOM) {
    ai = A.a[cidx];
    ati = A.at ? A.at[cidx] : ai;
  }
  const S sc = (S)I.c, sax = (S)I.ax, say = (S)I.ay, sd1 = (S)I.d1, sd2 = (S)I.d2;
  const S sabr = (S)I.abc_re, sabi = (S)I.abc_im, sdinv = (S)I.dinv;
  const int c0 = t.tx * 32 * VW + lane * VW;
  const bool live = c0 < pitch;
  const int r0 = t.ty * kRows + 1;
  const int r1 = min(r0 + kRows - 1, n);
  const E* xb = A.x + I.off;
  const E* xpb = MOM ? A.xp + I.off : nullptr;
  const E* bb = A.b + I.off;
  E* ob = A.out + I.off;

  auto load = [&](int pr, RowT<E, VW>& Y, E* xs, E* xps) {
    const bool in = (pr >= 1) && (pr <= n);
    VecN<E, VW> X{}, XP{};
    const long long ro = (long long)pr * pitch;
    if (in && live) {
      X = ldv<E, VW>(xb + ro + c0);
      if (MOM) XP = ldv<E, VW>(xpb + ro + c0);
    }
#pragma unroll
    for (int e = 0; e < VW; ++e) {
      Y.y[e] = MOM ? X.v[e] + ati * (X.v[e] - XP.v[e]) : X.v[e];
      xs[e] = X.v[e];
      xps[e] = XP.v[e];
    }
    E le{}, re{};
    if (in) {
      if (lane == 0 && c0 > 0) {
        E xv = xb[ro + c0 - 1];
        le = xv;
        if (MOM) {
          E pv = xpb[ro + c0 - 1];
          le = xv + ati * (xv - pv);
        }
      }
      if (lane == 31 && c0 + VW < pitch) {
        E xv = xb[ro + c0 + VW];
        re = xv;
        if (MOM) {
          E pv = xpb[ro + c0 + VW];
          re = xv + ati * (xv - pv);
        }
      }
    }
    row_neighbours<E, VW>(Y, lane, le, re);
  };

  RowT<E, VW> U, C, D;
  E xC[VW], xpC[VW], xD[VW], xpD[VW], tmp0[VW], tmp1[VW];
  load(r0 - 1, U, tmp0, tmp1);
  load(r0, C, xC, xpC);
  for (int r = r0; r <= r1; ++r) {
    load(r + 1, D, xD, xpD);
    VecN<E, VW> Bv{};
    if (live) Bv = ldv<E, VW>(bb + (long long)r * pitch + c0);
    E Ay[VW];
    if constexpr (CPLX) {
      apply_fd5<E, VW, S>(U, C, D, r - 1, c0, n, sc, sax, sabr, sabi, Ay);
    } else {
      apply_q1<E, VW, S>(U, C, D, sc, sax, say, sd1, sd2, Ay);
    }
    VecN<E, VW> O;
#pragma unroll
    for (int e = 0; e < VW; ++e) {
      const int col = c0 + e;
      E res = Bv.v[e] - Ay[e];
      if (PRE) {
        if constexpr (CPLX) {
          int miss = (r == 1) + (r == n) + (col == 0) + (col == n - 1);
          E diag = {sc + (S)miss * sabr, (S)miss * sabi};
          res = cdiv(res, diag);
        } else {
          res = sdinv * res;
        }
      }
      E nx = xC[e] + wi * res;
      if (MOM) nx = nx + ai * (xC[e] - xpC[e]);
      O.v[e] = (col < n) ? nx : E{};
    }
    if (live) stv<E, VW>(ob + (long long)r * pitch + c0, O);
    U = C;
    C = D;
#pragma unroll
    for (int e = 0; e < VW; ++e) {
      xC[e] = xD[e];
      xpC[e] = xpD[e];
    }
  }
}

template <typename E>
richm_status launch_sweep(richm_operator* op, const E* x, const E* xp, const E* b, E* out,
                          const typename RealOf<E>::type* w, const typename RealOf<E>::type* a,
                          const typename RealOf<E>::type* at, int m, int kidx, int precond, const int* active,
                          cudaStream_t s) {
  constexpr int VW = VecWidth<E>::value;
  const TileMap* tm = nullptr;
  RICHM_TRY(get_tiles(op, 32 * VW, kRows, &tm));
  SweepArgs<E> A{op->d_inst, tm->d_tiles, tm->ntiles, x, xp, b, out, w, a, at, m, kidx, active};
  const int blocks = (tm->ntiles + kWarpsPerBlock - 1) / kWarpsPerBlock;
  const dim3 block(kWarpsPerBlock * 32);
  const bool mom = (a != nullptr);
  if (mom && precond) sweep1_kernel<E, true, true><<<blocks, block, 0, s>>>(A);
  else if (mom) sweep1_kernel<E, true, false><<<blocks, block, 0, s>>>(A);
  else if (precond) sweep1_kernel<E, false, true><<<blocks, block, 0, s>>>(A);
  else sweep1_kernel<E, false, false><<<blocks, block, 0, s>>>(A);
  RICHM_LAUNCH_CHECK("sweep");
  return RICHM_OK;
}

#define RICHM_INST_SWEEP(E)                                                                                  \
  template richm_status launch_sweep<E>(richm_operator*, const E*, const E*, const E*, E*,                   \
                                        const RealOf<E>::type*, const RealOf<E>::type*,                      \
                                        const RealOf<E>::type*, int, int, int, const int*, cudaStream_t);
RICHM_INST_SWEEP(float)
RICHM_INST_SWEEP(double)
RICHM_INST_SWEEP(cplx<float>)
RICHM_INST_SWEEP(cplx<double>)

// K sweeps with a three-buffer rotation (x_k, x_{k-1}, free); the results are
// moved back into (x, x_prev) at the end when the rotation left them elsewhere.
template <typename E>
static richm_status apply_sweeps_t(richm_operator* op, E* x, E* xp, const E* b, const void* w, const void* a,
                                   const void* at, int K, const richm_sweep_opts* o, void* work, cudaStream_t s) {
  using S = typename RealOf<E>::type;
  const size_t bytes = op->elems * sizeof(E);
  E* W0 = reinterpret_cast<E*>(work);
  E* W1 = reinterpret_cast<E*>(reinterpret_cast<char*>(work) + ((bytes + 255) / 256) * 256);
  const bool mom = (a != nullptr);
  E* cur = x;
  E* prev = mom ? xp : nullptr;
  int k = 0;
  if constexpr (std::is_same<E, float>::value) {
    // fused passes of TL sweeps: (cur, prev) -> the other pair of buffers
    const int TL = (o->fuse == 4 || o->fuse == 8) ? o->fuse : 0;
    for (; TL > 0 && k + TL <= K; k += TL) {
      E* ox = (cur == x) ? W0 : x;
      E* oxp = (cur == x) ? W1 : xp;
      if (!mom && oxp == nullptr) oxp = W1;
      const int kidx0 = (int)(((long long)o->k_start + k) % o->m);
      RICHM_TRY(launch_sweep_fused(op, TL, cur, prev, b, ox, oxp, (const S*)w, (const S*)a, (const S*)at, o->m,
                                   kidx0, o->precond, nullptr, s));
      cur = ox;
      prev = mom ? oxp : nullptr;
    }
  }
  for (; k < K; ++k) {
    E* outb = nullptr;
    E* cand[4] = {W0, W1, x, xp};
    for (E* c : cand)
      if (c != nullptr && c != cur && c != prev) {
        outb = c;
        break;
      }
    const int kidx = (int)(((long long)o->k_start + k) % o->m);
    RICHM_TRY(launch_sweep<E>(op, cur, prev, b, outb, (const S*)w, (const S*)a, (const S*)at, o->m, kidx,
                              o->precond, nullptr, s));
    prev = mom ? cur : nullptr;
    cur = outb;
  }
  if (cur != x || (mom && prev != xp)) {
    if (mom) {
      // the final pair (cur, prev) lives in two of {x, xp, W0, W1}
      if (prev == x) {  // must move x -> xp before overwriting x
        RICHM_CUDA_TRY(cudaMemcpyAsync(xp, prev, bytes, cudaMemcpyDeviceToDevice, s));
        RICHM_CUDA_TRY(cudaMemcpyAsync(x, cur, bytes, cudaMemcpyDeviceToDevice, s));
      } else {
        if (cur != x) RICHM_CUDA_TRY(cudaMemcpyAsync(x, cur, bytes, cudaMemcpyDeviceToDevice, s));
        if (prev != xp) RICHM_CUDA_TRY(cudaMemcpyAsync(xp, prev, bytes, cudaMemcpyDeviceToDevice, s));
      }
    } else {
      RICHM_CUDA_TRY(cudaMemcpyAsync(x, cur, bytes, cudaMemcpyDeviceToDevice, s));
    }
  }
  return RICHM_OK;
}

}  // namespace richm

using namespace richm;

extern "C" {

richm_status richm_sweeps_workspace(const richm_operator* op, richm_dtype dtype, size_t* bytes) {
  clear_error();
  RICHM_ARG(op && bytes, "null argument");
  RICHM_ARG(dtype_valid(dtype), "invalid dtype %d", (int)dtype);
  const size_t one = ((op->elems * dtype_size(dtype) + 255) / 256) * 256;
  *bytes = 2 * one;
  return RICHM_OK;
}

richm_status richm_autotune_workspace(const richm_operator* op, size_t* bytes) {
  clear_error();
  RICHM_ARG(op && bytes, "null argument");
  const size_t one = ((op->elems * sizeof(float) + 255) / 256) * 256;
  *bytes = 5 * one + 256 * 3 * 64 * sizeof(float) * (size_t)((op->batch + 255) / 256);
  return RICHM_OK;
}

richm_status richm_autotune(richm_operator* op, int m, int momentum, void* work, size_t work_bytes, void* stream,
                            int* best_fuse, float* ms_per_sweep) {
  clear_error();
  RICHM_ARG(op != nullptr && work != nullptr, "null argument");
  RICHM_TRY(check_dtype_for_op(op, RICHM_F32));
  RICHM_ARG(m >= 1 && m <= 64, "m out of range");
  size_t need = 0;
  richm_autotune_workspace(op, &need);
  if (work_bytes < need) return set_error(RICHM_ERR_NOMEM, "workspace %zu < %zu bytes", work_bytes, need);
  cudaStream_t s = (cudaStream_t)stream;
  const size_t one = ((op->elems * sizeof(float) + 255) / 256) * 256;
  char* p = reinterpret_cast<char*>(work);
  float* x = reinterpret_cast<float*>(p);
  float* xp = reinterpret_cast<float*>(p + one);
  float* b = reinterpret_cast<float*>(p + 2 * one);
  void* W = p + 3 * one;
  float* coef = reinterpret_cast<float*>(p + 5 * one);
  const size_t nc = (size_t)op->batch * m;
  RICHM_CUDA_TRY(cudaMemsetAsync(x, 0, 3 * one, s));
  // small weights and momentum: values do not affect timing, only stay finite
  std::vector<float> hc(2 * nc);
  for (size_t i = 0; i < nc; ++i) {
    hc[i] = (float)(0.5 / op->h_inst[i / m].G);
    hc[nc + i] = 0.3f;
  }
  RICHM_CUDA_TRY(cudaMemcpyAsync(coef, hc.data(), sizeof(float) * 2 * nc, cudaMemcpyHostToDevice, s));
  const float* w = coef;
  const float* a = momentum ? coef + nc : nullptr;
  cudaEvent_t e0, e1;
  RICHM_CUDA_TRY(cudaEventCreate(&e0));
  RICHM_CUDA_TRY(cudaEventCreate(&e1));
  const int cands[3] = {1, 4, 8};
  int best = 1;
  float best_ms = 1e30f;
  for (int c : cands) {
    richm_sweep_opts o{m, 0, 0, c};
    const int K = 16;
    richm_status st = apply_sweeps_t<float>(op, x, xp, b, w, a, nullptr, K, &o, W, s);  // warm-up
    if (st != RICHM_OK) break;
    cudaEventRecord(e0, s);
    for (int r = 0; r < 3 && st == RICHM_OK; ++r) st = apply_sweeps_t<float>(op, x, xp, b, w, a, nullptr, K, &o, W, s);
    cudaEventRecord(e1, s);
    cudaError_t ce = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (st == RICHM_OK && ce == cudaSuccess && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess) {
      ms /= 3.0f * K;
      if (ms < best_ms) {
        best_ms = ms;
        best = c;
      }
    }
    if (st != RICHM_OK) {
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      return st;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  op->best_fuse = best;
  if (best_fuse) *best_fuse = best;
  if (ms_per_sweep) *ms_per_sweep = best_ms;
  return RICHM_OK;
}

richm_status richm_apply_sweeps(richm_operator* op, richm_dtype dtype, void* x, void* x_prev, const void* b,
                                const void* w, const void* alpha, const void* alpha_t, int K,
                                const richm_sweep_opts* opts, void* work, size_t work_bytes, void* stream) {
  clear_error();
  RICHM_ARG(op != nullptr && opts != nullptr, "null operator or options");
  RICHM_TRY(check_dtype_for_op(op, dtype));
  RICHM_ARG(K >= 0, "K = %d < 0", K);
  RICHM_ARG(opts->m >= 1 && opts->m <= 64, "m = %d out of range [1, 64]", opts->m);
  RICHM_ARG(opts->k_start >= 0, "k_start < 0");
  RICHM_ARG(opts->precond == 0 || opts->precond == 1, "precond must be 0 or 1");
  RICHM_ARG(opts->fuse == 0 || opts->fuse == 1 || opts->fuse == 2 || opts->fuse == 4 || opts->fuse == 8,
            "fuse must be 0, 1, 2, 4 or 8");
  RICHM_ARG(x != nullptr && b != nullptr && w != nullptr, "null x, b or w");
  RICHM_ARG(alpha != nullptr || alpha_t == nullptr, "alpha_t given without alpha");
  RICHM_ARG(alpha == nullptr || x_prev != nullptr, "momentum needs x_prev");
  if (K == 0) return RICHM_OK;
  size_t need = 0;
  richm_sweeps_workspace(op, dtype, &need);
  RICHM_ARG(work != nullptr, "null workspace");
  if (work_bytes < need) return set_error(RICHM_ERR_NOMEM, "workspace %zu < %zu bytes", work_bytes, need);
  cudaStream_t s = (cudaStream_t)stream;
  richm_sweep_opts o = *opts;
  if (o.fuse == 0) o.fuse = (dtype == RICHM_F32) ? op->best_fuse : 1;
  opts = &o;
  switch (dtype) {
    case RICHM_F32:
      return apply_sweeps_t<float>(op, (float*)x, (float*)x_prev, (const float*)b, w, alpha, alpha_t, K, opts, work, s);
    case RICHM_F64:
      return apply_sweeps_t<double>(op, (double*)x, (double*)x_prev, (const double*)b, w, alpha, alpha_t, K, opts, work, s);
    case RICHM_C64:
      return apply_sweeps_t<cplx<float>>(op, (cplx<float>*)x, (cplx<float>*)x_prev, (const cplx<float>*)b, w, alpha,
                                         alpha_t, K, opts, work, s);
    case RICHM_C128:
      return apply_sweeps_t<cplx<double>>(op, (cplx<double>*)x, (cplx<double>*)x_prev, (const cplx<double>*)b, w,
                                          alpha, alpha_t, K, opts, work, s);
  }
  return set_error(RICHM_ERR_ARG, "invalid dtype");
}

}  // extern "C"
