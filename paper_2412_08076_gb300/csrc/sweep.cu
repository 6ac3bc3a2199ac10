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

// Rows are prefetched kS1Prefetch row steps ahead with cp.async into per-warp
// shared-memory rings. A ring row holds the warp's 32 lane chunks of 16 bytes plus
// one chunk on each side (copied by lanes 0 and 31), so every lane reads back only
// what it copied itself: no barrier is needed.
constexpr int kS1Prefetch = 2;
constexpr int kS1Slots = 4;  // prefetched rows in flight + the row being consumed
__host__ __device__ constexpr int s1_ring_chunks(bool mom) { return kS1Slots * (34 + (mom ? 34 : 0) + 32); }

__device__ __forceinline__ void cp_async_chunk(uint4* smem, const void* gmem, bool valid) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  const int nbytes = valid ? 16 : 0;  // 0: zero-fill without reading global memory
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(sa), "l"(gmem), "r"(nbytes) : "memory");
}

template <typename E, bool MOM, bool PRE>
__global__ void __launch_bounds__(kWarpsPerBlock * 32, 3) sweep1_kernel(const SweepArgs<E> A) {
  using S = typename RealOf<E>::type;
  constexpr int VW = VecWidth<E>::value;
  constexpr bool CPLX = IsCplx<E>::value;
  constexpr int XC = 34, BC = 32;  // chunks per x row (with the two edge chunks) and per b row
  extern __shared__ __align__(16) uint4 s1_ring[];
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
  const S sspi = (S)I.sp_im, sspw = (S)I.sp_iw;
  const int c0 = t.tx * 32 * VW + lane * VW;
  const bool live = c0 < pitch;
  const int r0 = t.ty * kRows + 1;
  const int r1 = min(r0 + kRows - 1, n);
  const E* xb = A.x + I.off;
  const E* xpb = MOM ? A.xp + I.off : A.x + I.off;
  const E* bb = A.b + I.off;
  E* ob = A.out + I.off;
  uint4* ring = s1_ring + (threadIdx.x >> 5) * s1_ring_chunks(MOM);
  uint4* xr = ring;                                        // [slot][XC]
  uint4* xpr = ring + kS1Slots * XC;                       // [slot][XC] (MOM)
  uint4* br = ring + kS1Slots * (XC + (MOM ? XC : 0));     // [slot][BC]
  const bool has_left = c0 > 0, has_right = c0 + VW < pitch;

  // copies of x[q], x_{k-1}[q] (the next window row) and b[q - 1] (the next output row)
  auto issue = [&](int q) {
    const int sl = q & (kS1Slots - 1);
    const bool rv = (q >= 1) && (q <= n) && (q <= r1 + 1);
    const long long ro = (long long)(rv ? q : 0) * pitch;
    cp_async_chunk(xr + sl * XC + 1 + lane, xb + ro + (live ? c0 : 0), rv && live);
    if (MOM) cp_async_chunk(xpr + sl * XC + 1 + lane, xpb + ro + (live ? c0 : 0), rv && live);
    if (lane == 0) {
      cp_async_chunk(xr + sl * XC, xb + ro + (has_left ? c0 - VW : 0), rv && has_left);
      if (MOM) cp_async_chunk(xpr + sl * XC, xpb + ro + (has_left ? c0 - VW : 0), rv && has_left);
    }
    if (lane == 31) {
      cp_async_chunk(xr + sl * XC + 33, xb + ro + (has_right ? c0 + VW : 0), rv && has_right);
      if (MOM) cp_async_chunk(xpr + sl * XC + 33, xpb + ro + (has_right ? c0 + VW : 0), rv && has_right);
    }
    const int qb = q - 1;
    const bool bv = (qb >= r0) && (qb <= r1) && live;
    cp_async_chunk(br + sl * BC + lane, bb + (long long)(bv ? qb : 0) * pitch + (live ? c0 : 0), bv);
    asm volatile("cp.async.commit_group;\n" ::: "memory");
  };

  // y row of x[q] from ring slot q (neighbours across lanes by shuffles, edges from
  // the edge chunks); keeps x and x_{k-1} of the row for the update
  auto take = [&](int q, RowT<E, VW>& Y, E* xs, E* xps) {
    const int sl = q & (kS1Slots - 1);
    VecN<E, VW> X, XP;
    *reinterpret_cast<uint4*>(&X) = xr[sl * XC + 1 + lane];
    if (MOM) *reinterpret_cast<uint4*>(&XP) = xpr[sl * XC + 1 + lane];
#pragma unroll
    for (int e = 0; e < VW; ++e) {
      Y.y[e] = MOM ? X.v[e] + ati * (X.v[e] - XP.v[e]) : X.v[e];
      xs[e] = X.v[e];
      xps[e] = MOM ? XP.v[e] : E{};
    }
    E le{}, re{};
    if (lane == 0) {
      VecN<E, VW> L, LP;
      *reinterpret_cast<uint4*>(&L) = xr[sl * XC];
      le = L.v[VW - 1];
      if (MOM) {
        *reinterpret_cast<uint4*>(&LP) = xpr[sl * XC];
        le = le + ati * (le - LP.v[VW - 1]);
      }
    }
    if (lane == 31) {
      VecN<E, VW> R, RP;
      *reinterpret_cast<uint4*>(&R) = xr[sl * XC + 33];
      re = R.v[0];
      if (MOM) {
        *reinterpret_cast<uint4*>(&RP) = xpr[sl * XC + 33];
        re = re + ati * (re - RP.v[0]);
      }
    }
    row_neighbours<E, VW>(Y, lane, le, re);
  };

  for (int q = r0 - 1; q <= r0 + kS1Prefetch; ++q) issue(q);
  asm volatile("cp.async.wait_group %0;\n" ::"n"(kS1Prefetch) : "memory");
  RowT<E, VW> U, C, D;
  E xC[VW], xpC[VW], xD[VW], xpD[VW], tmp0[VW], tmp1[VW];
  take(r0 - 1, U, tmp0, tmp1);
  take(r0, C, xC, xpC);
  for (int r = r0; r <= r1; ++r) {
    issue(r + 1 + kS1Prefetch);
    asm volatile("cp.async.wait_group %0;\n" ::"n"(kS1Prefetch) : "memory");
    take(r + 1, D, xD, xpD);
    VecN<E, VW> Bv;
    *reinterpret_cast<uint4*>(&Bv) = br[((r + 1) & (kS1Slots - 1)) * BC + lane];
    E Ay[VW];
    if constexpr (CPLX) {
      apply_fd5<E, VW, S>(U, C, D, r - 1, c0, n, sc, sax, sabr, sabi, sspi, sspw, Ay);
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
          E diag = {sc + (S)miss * sabr, (S)miss * sabi + sponge_im<S>(r - 1, col, n, sspi, sspw)};
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
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
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
  const size_t sm_mom = sizeof(uint4) * kWarpsPerBlock * s1_ring_chunks(true);
  const size_t sm_plain = sizeof(uint4) * kWarpsPerBlock * s1_ring_chunks(false);
  if (mom && precond) sweep1_kernel<E, true, true><<<blocks, block, sm_mom, s>>>(A);
  else if (mom) sweep1_kernel<E, true, false><<<blocks, block, sm_mom, s>>>(A);
  else if (precond) sweep1_kernel<E, false, true><<<blocks, block, sm_plain, s>>>(A);
  else sweep1_kernel<E, false, false><<<blocks, block, sm_plain, s>>>(A);
  RICHM_LAUNCH_CHECK("sweep");
  return RICHM_OK;
}

// The one-sweep kernels use more than the default 48 KB of dynamic shared memory.
template <typename E>
static cudaError_t sweep1_attributes() {
  const int mom = (int)(sizeof(uint4) * kWarpsPerBlock * s1_ring_chunks(true));
  const int plain = (int)(sizeof(uint4) * kWarpsPerBlock * s1_ring_chunks(false));
  cudaError_t e = cudaFuncSetAttribute(sweep1_kernel<E, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, mom);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(sweep1_kernel<E, true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, mom);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(sweep1_kernel<E, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, plain);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(sweep1_kernel<E, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, plain);
  return e;
}

cudaError_t init_sweep_attributes() {
  cudaError_t e = sweep1_attributes<float>();
  if (e == cudaSuccess) e = sweep1_attributes<double>();
  if (e == cudaSuccess) e = sweep1_attributes<cplx<float>>();
  if (e == cudaSuccess) e = sweep1_attributes<cplx<double>>();
  if (e == cudaSuccess) e = init_fused_attributes();
  if (e == cudaSuccess) e = init_ssor_attributes();
  if (e == cudaSuccess) e = init_adjoint_attributes();
  return e;
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
  // the rotation may end in a workspace buffer that is copied back whole
  RICHM_TRY(launch_zero_halo(op, W0, sizeof(E), s));
  RICHM_TRY(launch_zero_halo(op, W1, sizeof(E), s));
  if constexpr (std::is_same<E, float>::value || std::is_same<E, double>::value) {
    if (o->precond == 2) {
      // SSOR: one forward and one backward solve per sweep; the third buffer holds z
      E* Z = reinterpret_cast<E*>(reinterpret_cast<char*>(work) + 2 * (((bytes + 255) / 256) * 256));
      for (; k < K; ++k) {
        E* outb = nullptr;
        E* cand[4] = {W0, W1, x, xp};
        for (E* c : cand)
          if (c != nullptr && c != cur && c != prev) {
            outb = c;
            break;
          }
        const int kidx = (int)(((long long)o->k_start + k) % o->m);
        // x_{k+1} -> outb; x_k stays where it is and becomes the new previous iterate
        RICHM_TRY(launch_ssor_sweep<E>(op, cur, prev, b, Z, outb, nullptr, (const S*)w, (const S*)a,
                                       (const S*)at, o->m, kidx, o->relax, nullptr, s));
        prev = mom ? cur : nullptr;
        cur = outb;
      }
    }
  }
  if constexpr (std::is_same<E, cplx<float>>::value) {
    // complex Helmholtz: fused passes of 4 sweeps (no preconditioner)
    const int TL = (o->fuse == 4 && o->precond == 0) ? 4 : 0;
    for (; TL > 0 && k + TL <= K; k += TL) {
      E* ox = (cur == x) ? W0 : x;
      E* oxp = (cur == x) ? W1 : xp;
      if (!mom && oxp == nullptr) oxp = W1;
      const int kidx0 = (int)(((long long)o->k_start + k) % o->m);
      RICHM_TRY(launch_sweep_fused_cx(op, TL, cur, prev, b, ox, oxp, (const float*)w, (const float*)a,
                                      (const float*)at, o->m, kidx0, nullptr, s));
      cur = ox;
      prev = mom ? oxp : nullptr;
    }
  }
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
  *bytes = 3 * one;  // two rotation buffers and the SSOR intermediate
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
  // candidates: (sweeps per pass, rows of a fused warp tile)
  const int cands[7][2] = {{1, 0}, {4, 64}, {4, 128}, {4, 256}, {8, 64}, {8, 128}, {8, 256}};
  int best = 1, best_rows = op->best_rows;
  float best_ms = 1e30f;
  for (const auto& cr : cands) {
    const int c = cr[0];
    if (c > 1) op->best_rows = cr[1];
    richm_sweep_opts o{m, 0, 0, c, 1.0};
    const int K = 16;
    richm_status st = apply_sweeps_t<float>(op, x, xp, b, w, a, nullptr, K, &o, W, s);  // warm-up
    if (st == RICHM_OK) cudaEventRecord(e0, s);
    for (int r = 0; r < 3 && st == RICHM_OK; ++r) st = apply_sweeps_t<float>(op, x, xp, b, w, a, nullptr, K, &o, W, s);
    if (st != RICHM_OK) {
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      return st;
    }
    cudaEventRecord(e1, s);
    float ms = 0.f;
    if (cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess) {
      ms /= 3.0f * K;
      if (ms < best_ms) {
        best_ms = ms;
        best = c;
        if (c > 1) best_rows = cr[1];
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  op->best_rows = best_rows;
  op->best_fuse = best;
  if (best_fuse) *best_fuse = best;
  if (ms_per_sweep) *ms_per_sweep = best_ms;
  return RICHM_OK;
}

richm_status richm_tuned(const richm_operator* op, int* fuse, int* rows) {
  clear_error();
  RICHM_ARG(op != nullptr, "null operator");
  if (fuse) *fuse = op->best_fuse;
  if (rows) *rows = op->best_rows;
  return RICHM_OK;
}

richm_status richm_set_tuning(richm_operator* op, int fuse, int rows) {
  clear_error();
  RICHM_ARG(op != nullptr, "null operator");
  RICHM_ARG(fuse == 1 || fuse == 4 || fuse == 8, "fuse must be 1, 4 or 8");
  RICHM_ARG(rows >= 16 && rows <= 256 && rows % 16 == 0, "rows must be a multiple of 16 from 16 to 256");
  op->best_fuse = fuse;
  op->best_rows = rows;
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
  RICHM_ARG(opts->precond == 0 || opts->precond == 1 || opts->precond == 2, "precond must be 0, 1 or 2");
  if (opts->precond == 2) {
    RICHM_ARG(opts->relax > 0.0 && opts->relax < 2.0, "SSOR relaxation factor %g outside (0, 2)", opts->relax);
    if (dtype != RICHM_F32 && dtype != RICHM_F64)
      return set_error(RICHM_ERR_UNSUPPORTED, "SSOR preconditioning takes RICHM_F32 or RICHM_F64 Q1 state");
  }
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
  if (o.fuse == 0) {
    if (dtype == RICHM_F32 || dtype == RICHM_BF16) o.fuse = op->best_fuse;
    else if (dtype == RICHM_C64 && o.precond == 0) o.fuse = 4;
    else o.fuse = 1;
  }
  if (o.precond == 2) o.fuse = 1;  // the triangular solves cannot be fused in time
  opts = &o;
  switch (dtype) {
    case RICHM_BF16: {
      // fused passes only: (x, x_prev) -> (W0, W1) -> (x, x_prev) ...
      const int TL = o.fuse;
      if (TL != 4 && TL != 8)
        return set_error(RICHM_ERR_UNSUPPORTED, "bfloat16 state needs fused passes (fuse 4 or 8)");
      if (K % TL != 0) return set_error(RICHM_ERR_UNSUPPORTED, "bfloat16 state: K must be a multiple of %d", TL);
      using B16 = __nv_bfloat16;
      const size_t bytes = op->elems * sizeof(B16);
      B16* W0 = reinterpret_cast<B16*>(work);
      B16* W1 = reinterpret_cast<B16*>(reinterpret_cast<char*>(work) + ((bytes + 255) / 256) * 256);
      B16* cur = (B16*)x;
      B16* prev = (B16*)x_prev;
      const bool mom = alpha != nullptr;
      RICHM_TRY(launch_zero_halo(op, W0, sizeof(B16), s));
      RICHM_TRY(launch_zero_halo(op, W1, sizeof(B16), s));
      for (int k = 0; k < K; k += TL) {
        B16* ox = (cur == (B16*)x) ? W0 : (B16*)x;
        B16* oxp = (cur == (B16*)x) ? W1 : (mom ? (B16*)x_prev : W1);
        RICHM_TRY(launch_sweep_fused_bf16(op, TL, cur, mom ? prev : nullptr, (const float*)b, ox, oxp,
                                          (const float*)w, (const float*)alpha, (const float*)alpha_t, o.m,
                                          (int)(((long long)o.k_start + k) % o.m), o.precond, nullptr, s));
        cur = ox;
        prev = oxp;
      }
      if (cur != (B16*)x) {
        RICHM_CUDA_TRY(cudaMemcpyAsync(x, cur, bytes, cudaMemcpyDeviceToDevice, s));
        if (mom) RICHM_CUDA_TRY(cudaMemcpyAsync(x_prev, prev, bytes, cudaMemcpyDeviceToDevice, s));
      }
      return RICHM_OK;
    }
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
