// Temporally blocked forward sweeps: TL sweeps of the Table 1 iteration per pass
// over HBM (real Q1, FP32 state).
//
// One warp owns 128 columns (a float4 per lane) of one instance and streams its
// rows top to bottom through a pipeline of TL time levels: while input row r is
// loaded, level s (s = 1..TL) computes row r - s of x_{k+s} from the three-row
// register window of y_{k+s-1} = x_{k+s-1} + at (x_{k+s-1} - x_{k+s-2}) that level
// s-1 has just extended. Right-hand-side rows wait in a TL-row delay line. Columns
// outside the domain are exactly zero at every level (Dirichlet), so tiles that touch
// the physical boundary need no halo there; at interior tile edges the result of
// level s is wrong in the s outermost columns, so neighbouring tiles overlap by TL
// columns on each side and only the inner columns are stored. Each pass reads x_k,
// x_{k-1}, b once (plus the overlaps and TL halo rows above and below each row-block
// tile) and writes the last two levels: 20 bytes per unknown per TL sweeps.
// Input rows are prefetched PF row steps ahead with cp.async into per-warp
// shared-memory rings (each lane copies and later reads only its own 16 bytes, so no
// barrier is needed), which keeps HBM latency out of the level pipeline; the b rows
// stay in their ring until the last level has used them. Each b row is copied into
// two slots NB apart, so that every level reads its row at a fixed offset from the
// step's slot, without wrapping.
//
// Nothing outside the domain needs clearing at any level: rows outside 1..n get the
// weight 0 (their inputs are zero, so they stay zero), and the lanes' stencil
// couplings into columns >= n are masked, so those columns (zero in every input, b
// included) stay zero as well.
//
// The real kernel is bound by instruction issue, so its arithmetic runs on pairs of
// columns with the packed FP32 instructions of sm_100 and later (one issue slot for
// two multiply-adds): a lane's four columns are two aligned pairs, and the stencil is
// arranged so that only the sum of the horizontal couplings needs per-column
// (unpaired) adds.
#include "common.cuh"
#include "kernels.cuh"

namespace richm {

constexpr int kFuseWarps = 4;

struct SweepTArgs {
  const Inst* insts;
  const Tile* tiles;
  int ntiles;
  const void* x;     // state storage type ST (float or bf16)
  const void* xp;
  const float* b;
  void* out_x;       // x_{k+TL}
  void* out_xp;      // x_{k+TL-1}
  const float* w;
  const float* a;
  const float* at;
  int m;
  int kidx0;  // coefficient index of the first sweep of the pass
  const int* active;
  int rows;   // output rows of a warp tile
};

// Per-warp state of the pipeline. Window slots rotate by phase: at phase p the new
// row of every level goes into slot p; after it, U = slot (p+1)%3, C = slot (p+2)%3,
// D = slot p. Unrolling the row loop by three makes every slot index a constant.
// Each lane keeps only its own values per row; what crosses lanes is exchanged by
// shuffles when the stencil is applied. Complex kernel: four floats (two complex
// columns) per row.
template <int TL>
struct FusedState {
  float Y[TL + 1][3][4];   // level s: rows of y_{s-1} (this lane's four values)
  float xc[TL + 1][4];     // level s: x_{s-1} on the centre row (MOM and NAGex only)
  float vc[TL + 1][4];     // level s: x_{s-1} - x_{s-2} on the centre row
  float prevx[2][TL + 1][4];  // outputs of level s at the last row steps (two slots)
};

// The real kernel's state: the same rows, this lane's four columns as two pairs.
template <int TL>
struct PairState {
  float2 Y[TL + 1][3][2];
  float2 xc[TL + 1][2];
  float2 vc[TL + 1][2];
  float2 prevx[2][TL + 1][2];
};

__device__ __forceinline__ float2 pair(float v) { return make_float2(v, v); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
  unsigned long long A, B, D;
  asm("mov.b64 %0, {%1, %2};" : "=l"(A) : "f"(a.x), "f"(a.y));
  asm("mov.b64 %0, {%1, %2};" : "=l"(B) : "f"(b.x), "f"(b.y));
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(D) : "l"(A), "l"(B));
  float2 r;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(D));
  return r;
}

constexpr int kPrefetch = 2;  // row steps between issuing a row's copies and using it

// XB: extra b slots for a pipeline that reads b rows further back (the skewed kernel).
template <typename ST, int TL, int XB = 0>
struct FusedRings {
  // one spare slot in each ring: a slot is re-targeted two row steps after its last read
  static constexpr int NS = kPrefetch + 2;            // x_k and x_{k-1} row slots
  static constexpr int NB = TL + kPrefetch + 2 + XB;  // b row slots (kept until level TL), each held twice
  static constexpr int XROW = 128 * (int)sizeof(ST);  // bytes of one state row (128 columns)
  static constexpr int BOFF = 2 * NS * XROW;          // start of the b ring
  static constexpr int BYTES = BOFF + 2 * NB * 128 * 4;
};

// State storage: FP32, or bfloat16 (arithmetic stays FP32; values are rounded to
// nearest-even when a pass stores its result).
__device__ __forceinline__ void st4_to_float(const float* p, float* v) {
  const float4 q = *reinterpret_cast<const float4*>(p);
  v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
}
__device__ __forceinline__ void st4_to_float(const __nv_bfloat16* p, float* v) {
  const uint2 q = *reinterpret_cast<const uint2*>(p);
  const __nv_bfloat162 lo = *reinterpret_cast<const __nv_bfloat162*>(&q.x);
  const __nv_bfloat162 hi = *reinterpret_cast<const __nv_bfloat162*>(&q.y);
  const float2 a = __bfloat1622float2(lo), b = __bfloat1622float2(hi);
  v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}
__device__ __forceinline__ void float_to_st4(float* p, const float* v) {
  *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
__device__ __forceinline__ void float_to_st4(__nv_bfloat16* p, const float* v) {
  const __nv_bfloat162 lo = __floats2bfloat162_rn(v[0], v[1]);
  const __nv_bfloat162 hi = __floats2bfloat162_rn(v[2], v[3]);
  uint2 q;
  q.x = *reinterpret_cast<const unsigned*>(&lo);
  q.y = *reinterpret_cast<const unsigned*>(&hi);
  *reinterpret_cast<uint2*>(p) = q;
}

template <typename ST>
struct FusedCtx {
  const ST* xb;
  const ST* xpb;
  const float* bb;
  ST* ox;
  ST* oxp;
  unsigned char* ring;  // this warp's rings: x[NS] rows, xp[NS] rows (ST), b[NB] rows (float)
  int n, pitch, c0, lane;
  // Rows are counted in the frame of the tile's first row band (lanes 0-15 of a tail
  // pair hold band ty, lanes 16-31 band pad - 2, whose pointers are shifted by the
  // band offset): this lane's rows 1..n are rlo .. rlo + n - 1, its inputs are
  // loaded up to row vhi and its results stored for rows r0 .. shi.
  int rlo, vhi, r0, shi;
  bool live, store_cols;
  float2 nc2, nay2;        // (-c, -c), (-ay, -ay)
  float2 ax2, d12, d22;    // (ax, ax), (d1, d1), (d2, d2)
  float2 negm[2];          // -1 per column of this lane inside the domain, 0 for columns >= n
  float ml, mr;   // 0 where this lane's left / right neighbour lies beyond the warp, else 1
};

// b - A y of the 9-point Q1 stencil at this lane's four columns (two pairs) from the
// window rows U, C, D:  A y = c C + ay (U + D) + S,  S_e = W_{e-1} + E_{e+1}, with
//   W_j = ax C_j + d1 U_j + d2 D_j   (column j's coupling to column j + 1),
//   E_j = ax C_j + d2 U_j + d1 D_j   (column j's coupling to column j - 1).
// W and E are formed on aligned pairs; only S needs per-column adds. The warp's edge
// lanes take 0 from beyond the warp (outside the domain, hence 0, or in the tile
// overlap, whose values are discarded); the masks are multiplies.
template <typename ST>
__device__ __forceinline__ void resid_pairs(const float2* U, const float2* C, const float2* D, const float2* b,
                                            const FusedCtx<ST>& c, float2* out) {
  float2 W[2], E[2];
#pragma unroll
  for (int p = 0; p < 2; ++p) {
    const float2 axc = __fmul2_rn(c.ax2, C[p]);
    W[p] = __ffma2_rn(c.d22, D[p], __ffma2_rn(c.d12, U[p], axc));
    E[p] = __ffma2_rn(c.d12, D[p], __ffma2_rn(c.d22, U[p], axc));
  }
  const float wm1 = c.ml * __shfl_up_sync(0xffffffffu, W[1].y, 1);  // W of column -1
  const float e4 = c.mr * __shfl_down_sync(0xffffffffu, E[0].x, 1);  // E of column 4
  const float2 S[2] = {make_float2(wm1 + E[0].y, W[0].x + E[1].x), make_float2(W[0].y + E[1].y, W[1].x + e4)};
#pragma unroll
  for (int p = 0; p < 2; ++p) {
    float2 t = __ffma2_rn(c.nc2, C[p], b[p]);
    t = __ffma2_rn(c.nay2, __fadd2_rn(U[p], D[p]), t);
    out[p] = __ffma2_rn(c.negm[p], S[p], t);
  }
}

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, bool valid) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  const int nbytes = valid ? 16 : 0;  // 0: zero-fill, no global read
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(sa), "l"(gmem), "r"(nbytes) : "memory");
}
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem, bool valid) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  const int nbytes = valid ? 8 : 0;
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(sa), "l"(gmem), "r"(nbytes) : "memory");
}
template <typename ST>
__device__ __forceinline__ void cp_async_state(void* smem, const ST* gmem, bool valid) {
  if constexpr (sizeof(ST) == 4) cp_async16(smem, gmem, valid);  // four FP32 values
  else cp_async8(smem, gmem, valid);                               // four bf16 values
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

__device__ __forceinline__ int ring_slot(int r, int nslots) { return (r + 64 * nslots) % nslots; }

// Issue the copies of input row r (x_k, x_{k-1}, b) into the rings (zero-filled
// outside rows 1..n, beyond the tile's last needed row, or beyond the row pitch).
template <typename ST, int TL, bool MOM, int XB = 0>
__device__ __forceinline__ void issue_row(const FusedCtx<ST>& c, int r) {
  using R = FusedRings<ST, TL, XB>;
  const bool valid = ((unsigned)(r - c.rlo) <= (unsigned)(c.vhi - c.rlo)) && c.live;
  const long long ro = (long long)(valid ? r : 0) * c.pitch + (c.live ? c.c0 : 0);
  const int xs = ring_slot(r, R::NS);
  cp_async_state<ST>(c.ring + xs * R::XROW + c.lane * 4 * (int)sizeof(ST), c.xb + ro, valid);
  if (MOM)
    cp_async_state<ST>(c.ring + (R::NS + xs) * R::XROW + c.lane * 4 * (int)sizeof(ST), c.xpb + ro, valid);
  unsigned char* bs = c.ring + R::BOFF + ring_slot(r, R::NB) * 512 + c.lane * 16;
  cp_async16(bs, c.bb + ro, valid);
  cp_async16(bs + R::NB * 512, c.bb + ro, valid);
  cp_async_commit();
}

// The first level's inputs of row step rr: issue the copies of row rr + kPrefetch, wait
// for those of row rr, and read x_k and x_{k-1} of row rr from the rings.
template <typename ST, int TL, bool MOM, bool ABS>
__device__ __forceinline__ void step_inputs(int rr, const FusedCtx<ST>& c, float2* x0, float2* xm) {
  using R = FusedRings<ST, TL>;
  issue_row<ST, TL, MOM>(c, rr + kPrefetch);
  cp_async_wait<kPrefetch>();  // the copies of row rr have landed
  const int xs = ring_slot(rr, R::NS);
  float v[4];
  st4_to_float(reinterpret_cast<const ST*>(c.ring + xs * R::XROW) + c.lane * 4, v);
  x0[0] = make_float2(v[0], v[1]);
  x0[1] = make_float2(v[2], v[3]);
  if (MOM) {
    st4_to_float(reinterpret_cast<const ST*>(c.ring + (R::NS + xs) * R::XROW) + c.lane * 4, v);
    xm[0] = make_float2(v[0], v[1]);
    xm[1] = make_float2(v[2], v[3]);
  } else {
    xm[0] = xm[1] = pair(0.f);
  }
  if constexpr (ABS) {
    // the stored pair (e, e_prev) stands for (0, e_prev - e): e has been added to the
    // FP64 solution, the difference keeps the velocity
#pragma unroll
    for (int p = 0; p < 2; ++p) {
      xm[p] = MOM ? sub2(xm[p], x0[p]) : pair(0.f);
      x0[p] = pair(0.f);
    }
  }
}

// Levels S0..S1 of row step rr at window phase PH: level s computes row rr - s of
// x_{k+s}. in1: the row entering level S0 (level S0 - 1's output of this step, row
// rr - S0 + 1); in2: the level S0 - 2 row of the previous step (row rr - S0 + 1 of
// x_{k+S0-2}), the look-ahead's other input. NAGF: at == a, so x_{k+1} = y + w (b - A y)
// needs only the window. The outputs that the next step needs (levels S0 - 1 .. DL)
// go to prevx[PW], the previous step's are read from prevx[1 - PW]; the three unrolled
// phases write slots 0, 1, 0, and the loop copies slot 0 to slot 1 once per three steps.
template <typename ST, int TL, int S0, int S1, int DL, bool MOM, bool NAGF, int PH, int PW>
__device__ __forceinline__ void step_levels(int rr, const FusedCtx<ST>& c, PairState<TL>& st, const float2* in1,
                                            const float2* in2, const float2* wl, const float2* al,
                                            const float2* atl, float2 (*newx)[2]) {
  using R = FusedRings<ST, TL>;
  constexpr int SD = PH, SU = (PH + 1) % 3, SC = (PH + 2) % 3;
  newx[S0 - 1][0] = in1[0];
  newx[S0 - 1][1] = in1[1];
  // b row rr - s sits at slot (rr mod NB) + NB - s: one of its two copies, never wrapped
  const unsigned char* bstep = c.ring + R::BOFF + (ring_slot(rr, R::NB) + R::NB) * 512 + c.lane * 16;
#pragma unroll
  for (int s = S0; s <= S1; ++s) {
    const int row = rr - s;
    const float4 B4 = *reinterpret_cast<const float4*>(bstep - s * 512);
    const float2 Bv[2] = {make_float2(B4.x, B4.y), make_float2(B4.z, B4.w)};
    // rows outside 1..n keep their (zero) values: weight 0
    const float2 ws = ((unsigned)(row - c.rlo) < (unsigned)c.n) ? wl[s] : pair(0.f);
    // extend level s's window with row rr - s + 1 of y_{s-1}
    float2* Yn = st.Y[s][SD];
    float2 vn[2];
#pragma unroll
    for (int p = 0; p < 2; ++p) {
      const float2 xs1 = newx[s - 1][p];
      const float2 xs2 = (s == S0) ? in2[p] : st.prevx[1 - PW][s - 2][p];
      vn[p] = MOM ? sub2(xs1, xs2) : pair(0.f);
      Yn[p] = MOM ? __ffma2_rn(atl[s], vn[p], xs1) : xs1;
    }
    float2 ry[2];
    resid_pairs<ST>(st.Y[s][SU], st.Y[s][SC], Yn, Bv, c, ry);
#pragma unroll
    for (int p = 0; p < 2; ++p) {
      if (!MOM || NAGF) {
        newx[s][p] = __ffma2_rn(ws, ry[p], st.Y[s][SC][p]);  // NAG: y = x + a v is the window centre
      } else {
        newx[s][p] = __ffma2_rn(ws, ry[p], __ffma2_rn(al[s], st.vc[s][p], st.xc[s][p]));
        st.xc[s][p] = newx[s - 1][p];
        st.vc[s][p] = vn[p];
      }
    }
  }
  if (MOM) {
#pragma unroll
    for (int s = S0 - 1; s <= DL; ++s)
#pragma unroll
      for (int p = 0; p < 2; ++p) st.prevx[PW][s][p] = newx[s][p];
  }
}

// Store rows rr - TL of x_{k+TL} and rr - TL + 1 of x_{k+TL-1} (this lane's columns).
template <typename ST, int TL, bool MOM>
__device__ __forceinline__ void step_store(int rr, const FusedCtx<ST>& c, const float2* last, const float2* prev) {
  if (c.store_cols) {
    const int ra = rr - TL, rb = rr - TL + 1;
    if (ra >= c.r0 && ra <= c.shi) {
      const float v[4] = {last[0].x, last[0].y, last[1].x, last[1].y};
      float_to_st4(c.ox + (long long)ra * c.pitch + c.c0, v);
    }
    if (MOM && rb >= c.r0 && rb <= c.shi) {
      const float v[4] = {prev[0].x, prev[0].y, prev[1].x, prev[1].y};
      float_to_st4(c.oxp + (long long)rb * c.pitch + c.c0, v);
    }
  }
}

// One row step of the whole pipeline (levels 1..TL) in one warp.
template <typename ST, int TL, bool MOM, bool NAGF, bool ABS, int PH, int PW>
__device__ __forceinline__ void fused_step(int rr, const FusedCtx<ST>& c, PairState<TL>& st, const float2* wl,
                                           const float2* al, const float2* atl) {
  float2 x0[2], xm[2];
  step_inputs<ST, TL, MOM, ABS>(rr, c, x0, xm);
  float2 newx[TL + 1][2];
  step_levels<ST, TL, 1, TL, TL - 2, MOM, NAGF, PH, PW>(rr, c, st, x0, xm, wl, al, atl, newx);
  step_store<ST, TL, MOM>(rr, c, newx[TL], newx[TL - 1]);
}

// Per-warp setup of a fused tile: coefficients of the TL levels, row and column frames,
// pointers (the ring pointer is the caller's). Returns the last input row step.
template <typename ST, int TL, bool MOM, bool PRE>
__device__ __forceinline__ int fused_setup(const SweepTArgs& A, const Tile& t, int lane, FusedCtx<ST>& c,
                                           float2* wl, float2* al, float2* atl) {
  constexpr int VW = 4;
  constexpr int STRIDE = 128 - 2 * TL;
  const Inst& I = A.insts[t.inst];
  const float dv = PRE ? (float)I.dinv : 1.f;
#pragma unroll
  for (int s = 1; s <= TL; ++s) {
    const int ci = t.inst * A.m + (A.kidx0 + s - 1) % A.m;
    const float as = MOM ? A.a[ci] : 0.f;
    wl[s] = pair(A.w[ci] * dv);
    al[s] = pair(as);
    atl[s] = pair(MOM ? (A.at ? A.at[ci] : as) : 0.f);
  }
  c.n = I.n;
  c.pitch = I.pitch;
  c.lane = lane;
  c.nc2 = pair(-(float)I.c);
  c.nay2 = pair(-(float)I.ay);
  c.ax2 = pair((float)I.ax);
  c.d12 = pair((float)I.d1);
  c.d22 = pair((float)I.d2);
  // a tail pair: 16 lanes per 64-column tile, lanes 16-31 on row band pad - 2
  const bool tail = t.pad > 0;
  const int tlane = tail ? (lane & 15) : lane;
  const bool idle = tail && lane >= 16 && t.pad == 1;
  const int band = (tail && lane >= 16 && !idle) ? t.pad - 2 : t.ty;
  const int dr = (band - t.ty) * A.rows;  // this lane's row offset from band ty
  const int cs = t.tx * STRIDE;    // first column of the tile
  c.c0 = cs + tlane * VW;          // this lane's first column
  c.live = c.c0 < c.pitch && !idle;
  c.ml = (tlane == 0) ? 0.f : 1.f;
  c.mr = (tlane == (tail ? 15 : 31)) ? 0.f : 1.f;
#pragma unroll
  for (int p = 0; p < 2; ++p)
    c.negm[p] = make_float2(c.c0 + 2 * p < c.n ? -1.f : 0.f, c.c0 + 2 * p + 1 < c.n ? -1.f : 0.f);
  const bool last_tile = tail || (cs + 128 >= c.n);
  const int clo = cs + (t.tx > 0 ? TL : 0);
  const int chi = last_tile ? c.pitch : cs + 128 - TL;
  c.store_cols = c.live && c.c0 >= clo && c.c0 + VW <= chi;
  c.r0 = t.ty * A.rows + 1;
  const int r1 = min(c.r0 + dr + A.rows - 1, c.n);  // this lane's last row (own frame)
  c.rlo = 1 - dr;
  c.vhi = min(r1 + TL, c.n) - dr;
  c.shi = r1 - dr;
  const long long sh = (long long)dr * c.pitch;
  c.xb = reinterpret_cast<const ST*>(A.x) + I.off + sh;
  c.xpb = reinterpret_cast<const ST*>(MOM ? A.xp : A.x) + I.off + sh;
  c.bb = A.b + I.off + sh;
  c.ox = reinterpret_cast<ST*>(A.out_x) + I.off + sh;
  c.oxp = MOM ? reinterpret_cast<ST*>(A.out_xp) + I.off + sh : nullptr;
  // the loop covers the longer of the two bands of a tail pair
  const int endA = min(c.r0 + A.rows - 1, c.n) + TL;
  const int endB = (tail && t.pad > 1) ? min((t.pad - 2) * A.rows + A.rows, c.n) + TL - (t.pad - 2 - t.ty) * A.rows
                                       : endA;
  return max(endA, endB);
}

template <int TL>
__device__ __forceinline__ void zero_state(PairState<TL>& st) {
#pragma unroll
  for (int s = 0; s <= TL; ++s) {
#pragma unroll
    for (int q = 0; q < 3; ++q)
#pragma unroll
      for (int p = 0; p < 2; ++p) st.Y[s][q][p] = pair(0.f);
#pragma unroll
    for (int p = 0; p < 2; ++p) st.xc[s][p] = st.vc[s][p] = st.prevx[0][s][p] = st.prevx[1][s][p] = pair(0.f);
  }
}

// b rows above the tile's first input row are never loaded: zero their slots
template <typename ST, int TL, int XB = 0>
__device__ __forceinline__ void zero_b_ring(const FusedCtx<ST>& c) {
  using R = FusedRings<ST, TL, XB>;
  for (int q = 0; q < 2 * R::NB; ++q)
    *reinterpret_cast<float4*>(c.ring + R::BOFF + q * 512 + c.lane * 16) = make_float4(0.f, 0.f, 0.f, 0.f);
}

template <typename ST, int TL, bool MOM, bool PRE, bool NAGF, bool ABS>
__global__ void __launch_bounds__(kFuseWarps * 32, TL == 4 ? 4 : 2) sweepT_kernel(const SweepTArgs A) {
  extern __shared__ __align__(16) unsigned char fused_smem[];
  const int lane = threadIdx.x & 31;
  const int wt = blockIdx.x * kFuseWarps + (threadIdx.x >> 5);
  if (wt >= A.ntiles) return;
  const Tile t = A.tiles[wt];
  if (A.active && A.active[t.inst] == 0) return;
  float2 wl[TL + 1], al[TL + 1], atl[TL + 1];
  FusedCtx<ST> c;
  const int rend = fused_setup<ST, TL, MOM, PRE>(A, t, lane, c, wl, al, atl);
  c.ring = fused_smem + (threadIdx.x >> 5) * FusedRings<ST, TL>::BYTES;
  PairState<TL> st;
  zero_state<TL>(st);
  zero_b_ring<ST, TL>(c);
  const int rstart = c.r0 - TL;
#pragma unroll
  for (int d = 0; d < kPrefetch; ++d) issue_row<ST, TL, MOM>(c, rstart + d);
  // rows r0-TL .. r1+TL in steps of three (a few extra steps at the end only
  // compute rows that are neither stored nor used)
  for (int rr = rstart; rr <= rend; rr += 3) {
    fused_step<ST, TL, MOM, NAGF, ABS, 0, 0>(rr, c, st, wl, al, atl);
    fused_step<ST, TL, MOM, NAGF, ABS, 1, 1>(rr + 1, c, st, wl, al, atl);
    fused_step<ST, TL, MOM, NAGF, ABS, 2, 0>(rr + 2, c, st, wl, al, atl);
    if (MOM) {
#pragma unroll
      for (int s = 0; s + 2 <= TL; ++s)
#pragma unroll
        for (int p = 0; p < 2; ++p) st.prevx[1][s][p] = st.prevx[0][s][p];
    }
  }
  cp_async_wait<0>();
}

// ---------------------------------------------------------------- 8 levels on two warps
// The 8-level pipeline of a tile split over two warps of one block: the lower warp runs
// levels 1-4 (and all loads), the upper warp levels 5-8 (and the stores). Each warp
// holds the state of four levels, so three blocks of two tiles (12 warps) fit an SM
// where the one-warp kernel fits two blocks of four warps, while HBM traffic stays that
// of eight sweeps per pass.
//
// The levels are skewed by two rows: level s at row step rr inserts the row that level
// s - 1 produced at the previous step (row rr - 2s + 1) and updates row rr - 2s. The
// levels of one step then depend only on the previous step, so a warp's four levels are
// four independent chains (processed top level first, so that each level takes its
// pending row before the level below replaces it). A level hands the next one
// (x_s, x_{s-1}) of the row it updated; the last level stores both. The lower warp
// passes level 4's pair to the upper warp through a two-slot exchange in shared memory,
// which level 5 inserts at the next step, and the upper warp reads the b rows from the
// lower warp's ring (kept for the 16-row skew). A named barrier of the two warps per
// row step orders the exchange and the ring reuse. Both warps of a tile leave together
// or not at all, and pass the same barriers.
constexpr int kSplitTiles = 2;  // tiles per block, two warps each

__device__ __forceinline__ void pair_sync(int id) { asm volatile("bar.sync %0, 64;" ::"r"(id) : "memory"); }

constexpr int kSkewXB = 8;             // b rows back to rr - 16
constexpr int kSkewXch = 2 * 2 * 512;  // two slots of (x_4, x_3) rows

template <typename ST>
__host__ __device__ constexpr int skew_tile_bytes() { return FusedRings<ST, 8, kSkewXB>::BYTES + kSkewXch; }

// Four levels of one warp. Level j: window rows of y_{s-1} (slots rotate by phase),
// x_{s-1} and x_{s-1} - x_{s-2} of the centre row; P[j]: the (x_{s-1}, x_{s-2}) row that
// level j inserts at the next step (j >= 1; level 0's comes from the loads or the exchange).
struct SkewState {
  float2 Y[4][3][2];
  float2 XC[4][2];
  float2 VC[4][2];
  float2 P[4][2][2];
};

// Level s of step rr (state slot j): insert the row (px, pxo), update the centre row
// rr - 2s; the new (x_s, x_{s-1}) of that row go to xo, xl.
template <typename ST, bool MOM, bool NAGF, int PH>
__device__ __forceinline__ void skew_level(int rr, int s, int j, const FusedCtx<ST>& c, SkewState& st,
                                           const float2* px, const float2* pxo, const unsigned char* bstep,
                                           float2 w2, float2 a2, float2 at2, float2* xo, float2* xl) {
  constexpr int SD = PH, SU = (PH + 1) % 3, SC = (PH + 2) % 3;
  float2 vn[2];
#pragma unroll
  for (int p = 0; p < 2; ++p) {
    vn[p] = MOM ? sub2(px[p], pxo[p]) : pair(0.f);
    st.Y[j][SD][p] = MOM ? __ffma2_rn(at2, vn[p], px[p]) : px[p];
  }
  const int row = rr - 2 * s;
  const float4 B4 = *reinterpret_cast<const float4*>(bstep - 2 * s * 512);
  const float2 Bv[2] = {make_float2(B4.x, B4.y), make_float2(B4.z, B4.w)};
  const float2 ws = ((unsigned)(row - c.rlo) < (unsigned)c.n) ? w2 : pair(0.f);
  float2 ry[2];
  resid_pairs<ST>(st.Y[j][SU], st.Y[j][SC], st.Y[j][SD], Bv, c, ry);
#pragma unroll
  for (int p = 0; p < 2; ++p) {
    if (!MOM || NAGF) xo[p] = __ffma2_rn(ws, ry[p], st.Y[j][SC][p]);  // y = x + a v is the window centre
    else xo[p] = __ffma2_rn(ws, ry[p], __ffma2_rn(a2, st.VC[j][p], st.XC[j][p]));
    xl[p] = st.XC[j][p];
    st.XC[j][p] = px[p];
    if (MOM && !NAGF) st.VC[j][p] = vn[p];
  }
}

template <typename ST, bool MOM, bool NAGF, bool ABS, int PH>
__device__ __forceinline__ void skew_lower_step(int rr, int it, const FusedCtx<ST>& c, SkewState& st,
                                                unsigned char* xch, const float2* wl, const float2* al,
                                                const float2* atl) {
  using R = FusedRings<ST, 8, kSkewXB>;
  issue_row<ST, 8, MOM, kSkewXB>(c, rr + kPrefetch);
  cp_async_wait<kPrefetch + 1>();  // the copies of row rr - 1 have landed
  const unsigned char* bstep = c.ring + R::BOFF + (ring_slot(rr, R::NB) + R::NB) * 512 + c.lane * 16;
  float2 xo[2], xl[2];
  // level 4: its row goes to the upper warp
  skew_level<ST, MOM, NAGF, PH>(rr, 4, 3, c, st, st.P[3][0], st.P[3][1], bstep, wl[4], al[4], atl[4], xo, xl);
  {
    unsigned char* xs = xch + (it & 1) * 1024 + c.lane * 16;
    *reinterpret_cast<float4*>(xs) = make_float4(xo[0].x, xo[0].y, xo[1].x, xo[1].y);
    *reinterpret_cast<float4*>(xs + 512) = make_float4(xl[0].x, xl[0].y, xl[1].x, xl[1].y);
  }
  // levels 3, 2
#pragma unroll
  for (int j = 2; j >= 1; --j) {
    skew_level<ST, MOM, NAGF, PH>(rr, 1 + j, j, c, st, st.P[j][0], st.P[j][1], bstep, wl[1 + j], al[1 + j],
                                  atl[1 + j], st.P[j + 1][0], st.P[j + 1][1]);
  }
  // level 1 inserts the loaded row rr - 1
  float2 x0[2], xm[2];
  {
    const int xs = ring_slot(rr - 1, R::NS);
    float v[4];
    st4_to_float(reinterpret_cast<const ST*>(c.ring + xs * R::XROW) + c.lane * 4, v);
    x0[0] = make_float2(v[0], v[1]);
    x0[1] = make_float2(v[2], v[3]);
    if (MOM) {
      st4_to_float(reinterpret_cast<const ST*>(c.ring + (R::NS + xs) * R::XROW) + c.lane * 4, v);
      xm[0] = make_float2(v[0], v[1]);
      xm[1] = make_float2(v[2], v[3]);
    } else {
      xm[0] = xm[1] = pair(0.f);
    }
    if constexpr (ABS) {
      // the stored pair (e, e_prev) stands for (0, e_prev - e)
#pragma unroll
      for (int p = 0; p < 2; ++p) {
        xm[p] = MOM ? sub2(xm[p], x0[p]) : pair(0.f);
        x0[p] = pair(0.f);
      }
    }
  }
  skew_level<ST, MOM, NAGF, PH>(rr, 1, 0, c, st, x0, xm, bstep, wl[1], al[1], atl[1], st.P[1][0], st.P[1][1]);
}

template <typename ST, bool MOM, bool NAGF, int PH>
__device__ __forceinline__ void skew_upper_step(int rr, int it, const FusedCtx<ST>& c, SkewState& st,
                                                const unsigned char* xch, const float2* wl, const float2* al,
                                                const float2* atl) {
  using R = FusedRings<ST, 8, kSkewXB>;
  const unsigned char* bstep = c.ring + R::BOFF + (ring_slot(rr, R::NB) + R::NB) * 512 + c.lane * 16;
  float2 xo[2], xl[2];
  // level 8: store row rr - 16 of x_{k+8} and x_{k+7}
  skew_level<ST, MOM, NAGF, PH>(rr, 8, 3, c, st, st.P[3][0], st.P[3][1], bstep, wl[8], al[8], atl[8], xo, xl);
  if (c.store_cols) {
    const int ra = rr - 16;
    if (ra >= c.r0 && ra <= c.shi) {
      const float v8[4] = {xo[0].x, xo[0].y, xo[1].x, xo[1].y};
      float_to_st4(c.ox + (long long)ra * c.pitch + c.c0, v8);
      if (MOM) {
        const float v7[4] = {xl[0].x, xl[0].y, xl[1].x, xl[1].y};
        float_to_st4(c.oxp + (long long)ra * c.pitch + c.c0, v7);
      }
    }
  }
  // levels 7, 6
#pragma unroll
  for (int j = 2; j >= 1; --j) {
    skew_level<ST, MOM, NAGF, PH>(rr, 5 + j, j, c, st, st.P[j][0], st.P[j][1], bstep, wl[5 + j], al[5 + j],
                                  atl[5 + j], st.P[j + 1][0], st.P[j + 1][1]);
  }
  // level 5 inserts the row the lower warp's level 4 produced at the previous step
  float2 xi[2], xim[2];
  {
    const unsigned char* xs = xch + ((it - 1) & 1) * 1024 + c.lane * 16;
    const float4 x4 = *reinterpret_cast<const float4*>(xs);
    const float4 x3 = *reinterpret_cast<const float4*>(xs + 512);
    xi[0] = make_float2(x4.x, x4.y);
    xi[1] = make_float2(x4.z, x4.w);
    xim[0] = make_float2(x3.x, x3.y);
    xim[1] = make_float2(x3.z, x3.w);
  }
  skew_level<ST, MOM, NAGF, PH>(rr, 5, 0, c, st, xi, xim, bstep, wl[5], al[5], atl[5], st.P[1][0], st.P[1][1]);
}

template <typename ST, bool MOM, bool PRE, bool NAGF, bool ABS>
__global__ void __launch_bounds__(kSplitTiles * 64, 3) sweepT8_kernel(const SweepTArgs A) {
  constexpr int TL = 8;
  extern __shared__ __align__(16) unsigned char fused_smem[];
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int pid = warp >> 1;           // this block's tile
  const bool upper = (warp & 1) != 0;  // levels 5-8, else 1-4
  const int wt = blockIdx.x * kSplitTiles + pid;
  if (wt >= A.ntiles) return;  // both warps of the tile
  const Tile t = A.tiles[wt];
  if (A.active && A.active[t.inst] == 0) return;  // both warps of the tile
  float2 wl[TL + 1], al[TL + 1], atl[TL + 1];
  FusedCtx<ST> c;
  const int rend = fused_setup<ST, TL, MOM, PRE>(A, t, lane, c, wl, al, atl) + TL;  // TL more steps of skew
  c.ring = fused_smem + pid * skew_tile_bytes<ST>();
  unsigned char* xch = c.ring + FusedRings<ST, TL, kSkewXB>::BYTES;
  const int bar = 1 + pid;
  const int rstart = c.r0 - TL + 1;  // level 1's window starts with row r0 - 8
  SkewState st;
#pragma unroll
  for (int j = 0; j < 4; ++j)
#pragma unroll
    for (int p = 0; p < 2; ++p) {
      st.Y[j][0][p] = st.Y[j][1][p] = st.Y[j][2][p] = pair(0.f);
      st.XC[j][p] = st.VC[j][p] = st.P[j][0][p] = st.P[j][1][p] = pair(0.f);
    }
  if (!upper) {
    zero_b_ring<ST, TL, kSkewXB>(c);
    for (int q = 0; q < 4; ++q)
      *reinterpret_cast<float4*>(xch + q * 512 + lane * 16) = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int d = 0; d <= kPrefetch; ++d) issue_row<ST, TL, MOM, kSkewXB>(c, rstart - 1 + d);
  }
  pair_sync(bar);
  // Both warps pass the barriers of every step rstart .. rstart + nsteps - 1 (whole groups
  // of three, the last steps only compute rows that are neither stored nor used). Level s
  // is first needed at step r0 - 8 + 3s (its window fills two steps earlier) and last at
  // r1 + 8 + s, so the lower warp has no work in the last four steps and the upper warp
  // none in the first twelve (before r0 + 5); they only pass those barriers. Step q from
  // rstart runs at window phase q mod 3 in both warps.
  const int nsteps = 3 * ((rend - rstart + 3) / 3);
  if (!upper) {
    const int nl = 3 * ((rend - 4 - rstart + 3) / 3);
    int q = 0;
    for (; q < nl; q += 3) {
      skew_lower_step<ST, MOM, NAGF, ABS, 0>(rstart + q, q, c, st, xch, wl, al, atl);
      pair_sync(bar);
      skew_lower_step<ST, MOM, NAGF, ABS, 1>(rstart + q + 1, q + 1, c, st, xch, wl, al, atl);
      pair_sync(bar);
      skew_lower_step<ST, MOM, NAGF, ABS, 2>(rstart + q + 2, q + 2, c, st, xch, wl, al, atl);
      pair_sync(bar);
    }
    for (; q < nsteps; ++q) pair_sync(bar);
    cp_async_wait<0>();
  } else {
    constexpr int kIdle = 12;  // r0 + 5 - rstart, a multiple of three
    int q = 0;
    for (; q < kIdle; ++q) pair_sync(bar);
    for (; q < nsteps; q += 3) {
      skew_upper_step<ST, MOM, NAGF, 0>(rstart + q, q, c, st, xch, wl, al, atl);
      pair_sync(bar);
      skew_upper_step<ST, MOM, NAGF, 1>(rstart + q + 1, q + 1, c, st, xch, wl, al, atl);
      pair_sync(bar);
      skew_upper_step<ST, MOM, NAGF, 2>(rstart + q + 2, q + 2, c, st, xch, wl, al, atl);
      pair_sync(bar);
    }
  }
}

// ---------------------------------------------------------------- complex Helmholtz
// The same row pipeline for the 5-point complex Helmholtz operator (eq. 22) with a
// first-order absorbing (or Dirichlet) boundary and complex64 state. A lane holds two
// complex columns (16 bytes), so a warp tile is 64 columns wide (tails 32); the ring
// and row bookkeeping of FusedCtx run in float units (pitch and columns doubled). Only
// the centre row of a level's window needs cross-lane neighbours. The diagonal of a row
// next to the boundary gains the absorbing term per missing neighbour: rows 1 and n
// through the level's row index, columns 0 and n - 1 through per-lane column terms.
// Columns from n on stay zero through a zero neighbour coefficient, rows outside 1..n
// through the zero weight, as in the Q1 kernel.
struct CxCoef {
  float nb[2];        // neighbour coefficient per column of this lane (0 from column n on)
  float dre[2], dim[2];  // diagonal of an interior row per column (with the column terms)
  float abre, abim;   // added to the diagonal per missing row neighbour
  float spim, spiw;   // sponge layer (eq. 21): i spim max(0, 1 - d spiw) at distance d
  float dcol[2];      // distance of this lane's columns from the left / right boundary
};

template <int TL, bool MOM, bool NAGF, bool SP, int PH, int PW>
__device__ __forceinline__ void fused_step_cx(int rr, const FusedCtx<float>& c, const CxCoef& k,
                                              FusedState<TL>& st, const float* wl, const float* al,
                                              const float* atl) {
  using R = FusedRings<float, TL>;
  constexpr int SD = PH, SU = (PH + 1) % 3, SC = (PH + 2) % 3;
  issue_row<float, TL, MOM>(c, rr + kPrefetch);
  cp_async_wait<kPrefetch>();
  float x0[4], xm[4];
  {
    const int xs = ring_slot(rr, R::NS);
    st4_to_float(reinterpret_cast<const float*>(c.ring + xs * R::XROW) + c.lane * 4, x0);
    if (MOM) st4_to_float(reinterpret_cast<const float*>(c.ring + (R::NS + xs) * R::XROW) + c.lane * 4, xm);
    else xm[0] = xm[1] = xm[2] = xm[3] = 0.f;
  }
  float newx[TL + 1][4];
#pragma unroll
  for (int e = 0; e < 4; ++e) newx[0][e] = x0[e];
  const unsigned char* bstep = c.ring + R::BOFF + (ring_slot(rr, R::NB) + R::NB) * 512 + c.lane * 16;
#pragma unroll
  for (int s = 1; s <= TL; ++s) {
    const int row = rr - s;
    const float4 B4 = *reinterpret_cast<const float4*>(bstep - s * 512);
    const float Bv[4] = {B4.x, B4.y, B4.z, B4.w};
    const float ws = ((unsigned)(row - c.rlo) < (unsigned)c.n) ? wl[s] : 0.f;
    const float rm = (float)((row == c.rlo) + (row == c.rlo + c.n - 1));  // missing row neighbours
    // the row's distance from the top / bottom boundary (sponge layer)
    const float drow = SP ? (float)min(row - c.rlo + 1, c.n - (row - c.rlo)) : 0.f;
    float* Yn = st.Y[s][SD];
    float vn[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const float xs1 = newx[s - 1][e];
      const float xs2 = (s == 1) ? xm[e] : st.prevx[1 - PW][s - 2][e];
      vn[e] = MOM ? xs1 - xs2 : 0.f;
      Yn[e] = MOM ? fmaf(atl[s], vn[e], xs1) : xs1;
    }
    const float* YU = st.Y[s][SU];
    const float* YC = st.Y[s][SC];
    // complex neighbours of the centre row across lanes (zero beyond the tile's lanes)
    const float lre = c.ml * __shfl_up_sync(0xffffffffu, YC[2], 1);
    const float lim = c.ml * __shfl_up_sync(0xffffffffu, YC[3], 1);
    const float rre = c.mr * __shfl_down_sync(0xffffffffu, YC[0], 1);
    const float rim = c.mr * __shfl_down_sync(0xffffffffu, YC[1], 1);
    float ry[4];
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      const float yre = YC[2 * e], yim = YC[2 * e + 1];
      const float wre = e == 0 ? lre : YC[0], wim = e == 0 ? lim : YC[1];
      const float ere = e == 1 ? rre : YC[2], eim = e == 1 ? rim : YC[3];
      const float sre = (wre + ere) + (YU[2 * e] + Yn[2 * e]);
      const float sim = (wim + eim) + (YU[2 * e + 1] + Yn[2 * e + 1]);
      const float dre = fmaf(rm, k.abre, k.dre[e]);
      float dim = fmaf(rm, k.abim, k.dim[e]);
      if constexpr (SP) dim = fmaf(k.spim, fmaxf(0.f, fmaf(-fminf(drow, k.dcol[e]), k.spiw, 1.f)), dim);
      ry[2 * e] = fmaf(-k.nb[e], sre, fmaf(dim, yim, fmaf(-dre, yre, Bv[2 * e])));
      ry[2 * e + 1] = fmaf(-k.nb[e], sim, fmaf(-dim, yre, fmaf(-dre, yim, Bv[2 * e + 1])));
    }
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      if (!MOM || NAGF) {
        newx[s][e] = fmaf(ws, ry[e], YC[e]);
      } else {
        newx[s][e] = fmaf(ws, ry[e], fmaf(al[s], st.vc[s][e], st.xc[s][e]));
        st.xc[s][e] = newx[s - 1][e];
        st.vc[s][e] = vn[e];
      }
    }
  }
  if (c.store_cols) {
    const int ra = rr - TL, rb = rr - TL + 1;
    if (ra >= c.r0 && ra <= c.shi) float_to_st4(c.ox + (long long)ra * c.pitch + c.c0, newx[TL]);
    if (MOM && rb >= c.r0 && rb <= c.shi) float_to_st4(c.oxp + (long long)rb * c.pitch + c.c0, newx[TL - 1]);
  }
  if (MOM) {
#pragma unroll
    for (int s = 0; s + 2 <= TL; ++s)
#pragma unroll
      for (int e = 0; e < 4; ++e) st.prevx[PW][s][e] = newx[s][e];
  }
}

template <int TL, bool MOM, bool NAGF, bool SP>
__global__ void __launch_bounds__(kFuseWarps * 32, 3) sweepT_cx_kernel(const SweepTArgs A) {
  constexpr int STRIDE = 64 - 2 * TL;
  extern __shared__ __align__(16) unsigned char fused_smem[];
  const int lane = threadIdx.x & 31;
  const int wt = blockIdx.x * kFuseWarps + (threadIdx.x >> 5);
  if (wt >= A.ntiles) return;
  const Tile t = A.tiles[wt];
  if (A.active && A.active[t.inst] == 0) return;
  const Inst& I = A.insts[t.inst];
  float wl[TL + 1], al[TL + 1], atl[TL + 1];
#pragma unroll
  for (int s = 1; s <= TL; ++s) {
    const int ci = t.inst * A.m + (A.kidx0 + s - 1) % A.m;
    wl[s] = A.w[ci];
    al[s] = MOM ? A.a[ci] : 0.f;
    atl[s] = MOM ? (A.at ? A.at[ci] : al[s]) : 0.f;
  }
  const int n = I.n;
  const bool tail = t.pad > 0;
  const int tlane = tail ? (lane & 15) : lane;
  const bool idle = tail && lane >= 16 && t.pad == 1;
  const int band = (tail && lane >= 16 && !idle) ? t.pad - 2 : t.ty;
  const int dr = (band - t.ty) * A.rows;
  const int cs = t.tx * STRIDE;         // first complex column of the tile
  const int cc = cs + tlane * 2;        // this lane's first complex column
  FusedCtx<float> c;
  c.n = n;
  c.pitch = 2 * I.pitch;                // float units
  c.lane = lane;
  c.c0 = 2 * cc;
  c.live = cc < I.pitch && !idle;
  c.ml = (tlane == 0) ? 0.f : 1.f;
  c.mr = (tlane == (tail ? 15 : 31)) ? 0.f : 1.f;
  CxCoef k;
#pragma unroll
  for (int e = 0; e < 2; ++e) {
    const int col = cc + e;
    const float cm = (float)((col == 0) + (col == n - 1));
    k.nb[e] = col < n ? (float)I.ax : 0.f;
    k.dre[e] = (float)I.c + cm * (float)I.abc_re;
    k.dim[e] = cm * (float)I.abc_im;
    k.dcol[e] = (float)min(col + 1, n - col);
  }
  k.abre = (float)I.abc_re;
  k.abim = (float)I.abc_im;
  k.spim = (float)I.sp_im;
  k.spiw = (float)I.sp_iw;
  const bool last_tile = tail || (cs + 64 >= n);
  const int clo = cs + (t.tx > 0 ? TL : 0);
  const int chi = last_tile ? I.pitch : cs + 64 - TL;
  c.store_cols = c.live && cc >= clo && cc + 2 <= chi;
  c.r0 = t.ty * A.rows + 1;
  const int r1 = min(c.r0 + dr + A.rows - 1, n);
  c.rlo = 1 - dr;
  c.vhi = min(r1 + TL, n) - dr;
  c.shi = r1 - dr;
  const int endA = min(c.r0 + A.rows - 1, n) + TL;
  const int endB = (tail && t.pad > 1) ? min((t.pad - 2) * A.rows + A.rows, n) + TL - (t.pad - 2 - t.ty) * A.rows
                                       : endA;
  const int rend = max(endA, endB);
  const long long off = 2 * (I.off + (long long)dr * I.pitch);
  c.xb = reinterpret_cast<const float*>(A.x) + off;
  c.xpb = reinterpret_cast<const float*>(MOM ? A.xp : A.x) + off;
  c.bb = A.b + off;
  c.ox = reinterpret_cast<float*>(A.out_x) + off;
  c.oxp = MOM ? reinterpret_cast<float*>(A.out_xp) + off : nullptr;
  c.ring = fused_smem + (threadIdx.x >> 5) * FusedRings<float, TL>::BYTES;
  FusedState<TL> st;
#pragma unroll
  for (int s = 0; s <= TL; ++s) {
#pragma unroll
    for (int q = 0; q < 3; ++q)
#pragma unroll
      for (int e = 0; e < 4; ++e) st.Y[s][q][e] = 0.f;
#pragma unroll
    for (int e = 0; e < 4; ++e) st.xc[s][e] = st.vc[s][e] = st.prevx[0][s][e] = st.prevx[1][s][e] = 0.f;
  }
  for (int q = 0; q < 2 * FusedRings<float, TL>::NB; ++q)
    *reinterpret_cast<float4*>(c.ring + FusedRings<float, TL>::BOFF + q * 512 + lane * 16) =
        make_float4(0.f, 0.f, 0.f, 0.f);
  const int rstart = c.r0 - TL;
#pragma unroll
  for (int d = 0; d < kPrefetch; ++d) issue_row<float, TL, MOM>(c, rstart + d);
  for (int rr = rstart; rr <= rend; rr += 3) {
    fused_step_cx<TL, MOM, NAGF, SP, 0, 0>(rr, c, k, st, wl, al, atl);
    fused_step_cx<TL, MOM, NAGF, SP, 1, 1>(rr + 1, c, k, st, wl, al, atl);
    fused_step_cx<TL, MOM, NAGF, SP, 2, 0>(rr + 2, c, k, st, wl, al, atl);
    if (MOM) {
#pragma unroll
      for (int s = 0; s + 2 <= TL; ++s)
#pragma unroll
        for (int e = 0; e < 4; ++e) st.prevx[1][s][e] = st.prevx[0][s][e];
    }
  }
  cp_async_wait<0>();
}

template <typename ST>
static cudaError_t skew_attributes() {
  const int bytes = skew_tile_bytes<ST>() * kSplitTiles;
  cudaError_t e = cudaSuccess;
#define RICHM_SKEW_ATTR(MOM, PRE, NAGF, ABS)                                                                  \
  if (e == cudaSuccess)                                                                                      \
    e = cudaFuncSetAttribute(sweepT8_kernel<ST, MOM, PRE, NAGF, ABS>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                             bytes);
  RICHM_SKEW_ATTR(true, true, true, false)
  RICHM_SKEW_ATTR(true, false, true, false)
  RICHM_SKEW_ATTR(true, true, false, false)
  RICHM_SKEW_ATTR(true, false, false, false)
  RICHM_SKEW_ATTR(false, true, false, false)
  RICHM_SKEW_ATTR(false, false, false, false)
  RICHM_SKEW_ATTR(true, true, true, true)
  RICHM_SKEW_ATTR(true, false, true, true)
  RICHM_SKEW_ATTR(true, true, false, true)
  RICHM_SKEW_ATTR(true, false, false, true)
  RICHM_SKEW_ATTR(false, true, false, true)
  RICHM_SKEW_ATTR(false, false, false, true)
#undef RICHM_SKEW_ATTR
  return e;
}

template <typename ST, int TL>
static cudaError_t fused_attributes_tl() {
  const int bytes = FusedRings<ST, TL>::BYTES * kFuseWarps;
  cudaError_t e = cudaSuccess;
#define RICHM_FUSED_ATTR(MOM, PRE, NAGF, ABS)                                                               \
  if (e == cudaSuccess)                                                                                      \
    e = cudaFuncSetAttribute(sweepT_kernel<ST, TL, MOM, PRE, NAGF, ABS>,                                      \
                             cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  RICHM_FUSED_ATTR(true, true, true, false)
  RICHM_FUSED_ATTR(true, false, true, false)
  RICHM_FUSED_ATTR(true, true, false, false)
  RICHM_FUSED_ATTR(true, false, false, false)
  RICHM_FUSED_ATTR(false, true, false, false)
  RICHM_FUSED_ATTR(false, false, false, false)
  RICHM_FUSED_ATTR(true, true, true, true)
  RICHM_FUSED_ATTR(true, false, true, true)
  RICHM_FUSED_ATTR(true, true, false, true)
  RICHM_FUSED_ATTR(true, false, false, true)
  RICHM_FUSED_ATTR(false, true, false, true)
  RICHM_FUSED_ATTR(false, false, false, true)
#undef RICHM_FUSED_ATTR
  return e;
}

// The fused kernels' rings can exceed the default 48 KB of dynamic shared memory.
cudaError_t init_fused_attributes() {
  const int cx_bytes = FusedRings<float, 4>::BYTES * kFuseWarps;
  cudaError_t e = cudaSuccess;
#define RICHM_CX_ATTR(M, N, SP)                                                                                 \
  if (e == cudaSuccess)                                                                                         \
    e = cudaFuncSetAttribute(sweepT_cx_kernel<4, M, N, SP>, cudaFuncAttributeMaxDynamicSharedMemorySize, cx_bytes);
  RICHM_CX_ATTR(true, true, false)
  RICHM_CX_ATTR(true, false, false)
  RICHM_CX_ATTR(false, false, false)
  RICHM_CX_ATTR(true, true, true)
  RICHM_CX_ATTR(true, false, true)
  RICHM_CX_ATTR(false, false, true)
#undef RICHM_CX_ATTR
  if (e == cudaSuccess) e = fused_attributes_tl<float, 4>();
  if (e == cudaSuccess) e = skew_attributes<float>();
  if (e == cudaSuccess) e = fused_attributes_tl<__nv_bfloat16, 4>();
  if (e == cudaSuccess) e = skew_attributes<__nv_bfloat16>();
  return e;
}

template <typename ST>
static richm_status launch_fused_t(richm_operator* op, int TL, const ST* x, const ST* xp, const float* b, ST* out_x,
                                   ST* out_xp, const float* w, const float* a, const float* at, int m, int kidx0,
                                   int precond, const int* active, cudaStream_t s, int rows, bool absorb) {
  if (rows <= 0) rows = op->best_rows;
  const TileMap* tm = nullptr;
  RICHM_TRY(get_tiles(op, -TL, rows, &tm));
  SweepTArgs A{op->d_inst, tm->d_tiles, tm->ntiles, x, xp, b, out_x, out_xp, w, a, at, m, kidx0, active, rows};
  const bool mom = a != nullptr;
  const bool nag = mom && at == nullptr;  // at = a
  if (TL == 8) {  // two warps per tile, two tiles per block
    const int blocks = (tm->ntiles + kSplitTiles - 1) / kSplitTiles;
    const int thr = kSplitTiles * 64;
    const size_t smem = (size_t)skew_tile_bytes<ST>() * kSplitTiles;
#define RICHM_SKEW(ABS)                                                                                    \
  if (nag && precond) sweepT8_kernel<ST, true, true, true, ABS><<<blocks, thr, smem, s>>>(A);             \
  else if (nag) sweepT8_kernel<ST, true, false, true, ABS><<<blocks, thr, smem, s>>>(A);                  \
  else if (mom && precond) sweepT8_kernel<ST, true, true, false, ABS><<<blocks, thr, smem, s>>>(A);       \
  else if (mom) sweepT8_kernel<ST, true, false, false, ABS><<<blocks, thr, smem, s>>>(A);                 \
  else if (precond) sweepT8_kernel<ST, false, true, false, ABS><<<blocks, thr, smem, s>>>(A);             \
  else sweepT8_kernel<ST, false, false, false, ABS><<<blocks, thr, smem, s>>>(A);
    if (absorb) {
      RICHM_SKEW(true)
    } else {
      RICHM_SKEW(false)
    }
#undef RICHM_SKEW
    RICHM_LAUNCH_CHECK("fused sweep");
    return RICHM_OK;
  }
  const int blocks = (tm->ntiles + kFuseWarps - 1) / kFuseWarps;
  const int thr = kFuseWarps * 32;
  const size_t smem = (size_t)FusedRings<ST, 4>::BYTES * kFuseWarps;
#define RICHM_FUSED(TLV, ABS)                                                                              \
  if (nag && precond) sweepT_kernel<ST, TLV, true, true, true, ABS><<<blocks, thr, smem, s>>>(A);         \
  else if (nag) sweepT_kernel<ST, TLV, true, false, true, ABS><<<blocks, thr, smem, s>>>(A);              \
  else if (mom && precond) sweepT_kernel<ST, TLV, true, true, false, ABS><<<blocks, thr, smem, s>>>(A);   \
  else if (mom) sweepT_kernel<ST, TLV, true, false, false, ABS><<<blocks, thr, smem, s>>>(A);             \
  else if (precond) sweepT_kernel<ST, TLV, false, true, false, ABS><<<blocks, thr, smem, s>>>(A);         \
  else sweepT_kernel<ST, TLV, false, false, false, ABS><<<blocks, thr, smem, s>>>(A);
  if (TL != 4 && TL != 8) return set_error(RICHM_ERR_ARG, "fused sweeps support 4 or 8 sweeps per pass");
  if (!absorb) {
    RICHM_FUSED(4, false)
  } else {
    RICHM_FUSED(4, true)
  }
#undef RICHM_FUSED
  RICHM_LAUNCH_CHECK("fused sweep");
  return RICHM_OK;
}

richm_status launch_sweep_fused(richm_operator* op, int TL, const float* x, const float* xp, const float* b,
                                float* out_x, float* out_xp, const float* w, const float* a, const float* at, int m,
                                int kidx0, int precond, const int* active, cudaStream_t s, int rows, bool absorb) {
  return launch_fused_t<float>(op, TL, x, xp, b, out_x, out_xp, w, a, at, m, kidx0, precond, active, s, rows,
                               absorb);
}

richm_status launch_sweep_fused_cx(richm_operator* op, int TL, const cplx<float>* x, const cplx<float>* xp,
                                   const cplx<float>* b, cplx<float>* out_x, cplx<float>* out_xp, const float* w,
                                   const float* a, const float* at, int m, int kidx0, const int* active,
                                   cudaStream_t s, int rows) {
  if (TL != 4) return set_error(RICHM_ERR_ARG, "complex fused sweeps take 4 sweeps per pass");
  const TileMap* tm = nullptr;
  if (rows <= 0) {
    // the operator's tile height, halved (down to 16 rows) while the batch has fewer
    // warp tiles than two blocks per SM take: a small batch then still spreads over the
    // GPU (4 x 511^2: 5 sweeps in 49 instead of 112 us)
    rows = op->best_rows;
    RICHM_TRY(get_tiles(op, -100 - TL, rows, &tm));
    while (rows > 16 && tm->ntiles < 2 * kFuseWarps * op->sms) {
      rows /= 2;
      RICHM_TRY(get_tiles(op, -100 - TL, rows, &tm));
    }
  } else {
    RICHM_TRY(get_tiles(op, -100 - TL, rows, &tm));
  }
  SweepTArgs A{op->d_inst, tm->d_tiles, tm->ntiles, x, xp, reinterpret_cast<const float*>(b), out_x, out_xp,
               w, a, at, m, kidx0, active, rows};
  const int blocks = (tm->ntiles + kFuseWarps - 1) / kFuseWarps;
  const size_t smem = (size_t)FusedRings<float, 4>::BYTES * kFuseWarps;
  const bool mom = a != nullptr;
  const bool nag = mom && at == nullptr;
  bool sp = false;  // a sponge layer in the batch: the per-node diagonal term
  for (const Inst& I : op->h_inst) sp = sp || I.sp_im != 0.0;
#define RICHM_CX(SP)                                                                          \
  if (nag) sweepT_cx_kernel<4, true, true, SP><<<blocks, kFuseWarps * 32, smem, s>>>(A);      \
  else if (mom) sweepT_cx_kernel<4, true, false, SP><<<blocks, kFuseWarps * 32, smem, s>>>(A); \
  else sweepT_cx_kernel<4, false, false, SP><<<blocks, kFuseWarps * 32, smem, s>>>(A);
  if (sp) {
    RICHM_CX(true)
  } else {
    RICHM_CX(false)
  }
#undef RICHM_CX
  RICHM_LAUNCH_CHECK("complex fused sweep");
  return RICHM_OK;
}

richm_status launch_sweep_fused_bf16(richm_operator* op, int TL, const __nv_bfloat16* x, const __nv_bfloat16* xp,
                                     const float* b, __nv_bfloat16* out_x, __nv_bfloat16* out_xp, const float* w,
                                     const float* a, const float* at, int m, int kidx0, int precond,
                                     const int* active, cudaStream_t s, int rows, bool absorb) {
  return launch_fused_t<__nv_bfloat16>(op, TL, x, xp, b, out_x, out_xp, w, a, at, m, kidx0, precond, active, s,
                                       rows, absorb);
}

}  // namespace richm
