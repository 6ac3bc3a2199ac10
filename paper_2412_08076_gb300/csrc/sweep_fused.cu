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
// x_{k-1}, b once (plus the overlaps and TL halo rows above and below each 64-row
// tile) and writes the last two levels: 20 bytes per unknown per TL sweeps.
#include "common.cuh"
#include "kernels.cuh"

namespace richm {

constexpr int kFuseWarps = 4;

struct SweepTArgs {
  const Inst* insts;
  const Tile* tiles;
  int ntiles;
  const float* x;
  const float* xp;
  const float* b;
  float* out_x;   // x_{k+TL}
  float* out_xp;  // x_{k+TL-1}
  const float* w;
  const float* a;
  const float* at;
  int m;
  int kidx0;  // coefficient index of the first sweep of the pass
  const int* active;
};

template <int TL, bool MOM, bool PRE>
__global__ void __launch_bounds__(kFuseWarps * 32) sweepT_kernel(const SweepTArgs A) {
  constexpr int VW = 4;
  constexpr int STRIDE = 128 - 2 * TL;
  const int lane = threadIdx.x & 31;
  const int wt = blockIdx.x * kFuseWarps + (threadIdx.x >> 5);
  if (wt >= A.ntiles) return;
  const Tile t = A.tiles[wt];
  if (A.active && A.active[t.inst] == 0) return;
  const Inst& I = A.insts[t.inst];
  const int n = I.n, pitch = I.pitch;
  const float sc = (float)I.c, sax = (float)I.ax, say = (float)I.ay, sd1 = (float)I.d1, sd2 = (float)I.d2;
  const float dv = PRE ? (float)I.dinv : 1.f;

  float wl[TL + 1], al[TL + 1], atl[TL + 1];
#pragma unroll
  for (int s = 1; s <= TL; ++s) {
    const int ci = t.inst * A.m + (A.kidx0 + s - 1) % A.m;
    wl[s] = A.w[ci] * dv;
    al[s] = MOM ? A.a[ci] : 0.f;
    atl[s] = MOM ? (A.at ? A.at[ci] : al[s]) : 0.f;
  }

  const int cs = t.tx * STRIDE;            // first column of the tile
  const int c0 = cs + lane * VW;           // this lane's first column
  const bool live = c0 < pitch;
  const bool last_tile = (cs + 128 >= n);
  const int vlo = cs + (t.tx > 0 ? TL : 0);
  const int vhi = last_tile ? pitch : cs + 128 - TL;
  const bool store_cols = live && c0 >= vlo && c0 + VW <= vhi;
  const int r0 = t.ty * kFuseRows + 1;
  const int r1 = min(r0 + kFuseRows - 1, n);
  const float* xb = A.x + I.off;
  const float* xpb = MOM ? A.xp + I.off : nullptr;
  const float* bb = A.b + I.off;
  float* ox = A.out_x + I.off;
  float* oxp = MOM ? A.out_xp + I.off : nullptr;

  // per-level state
  RowT<float, VW> YU[TL + 1], YC[TL + 1], YD[TL + 1];
  float xc[TL + 1][VW], vc[TL + 1][VW];   // centre row of level s: x_{s-1}, v_{s-1}
  float prevx[TL + 1][VW];                // level s output of the previous iteration
  float bd[TL + 1][VW];                   // b delay line: bd[s] = b[rr - s]
#pragma unroll
  for (int s = 0; s <= TL; ++s) {
#pragma unroll
    for (int e = 0; e < VW; ++e) {
      YU[s].y[e] = YC[s].y[e] = YD[s].y[e] = 0.f;
      xc[s][e] = vc[s][e] = prevx[s][e] = bd[s][e] = 0.f;
    }
    YU[s].yl = YU[s].yr = YC[s].yl = YC[s].yr = YD[s].yl = YD[s].yr = 0.f;
  }

  for (int rr = r0 - TL; rr <= r1 + TL; ++rr) {
#pragma unroll
    for (int s = TL; s >= 1; --s)
#pragma unroll
      for (int e = 0; e < VW; ++e) bd[s][e] = bd[s - 1][e];
    float x0[VW], xm[VW];
    {
      VecN<float, VW> X{}, XP{}, Bv{};
      if (rr >= 1 && rr <= n && live) {
        const long long ro = (long long)rr * pitch + c0;
        X = ldv<float, VW>(xb + ro);
        if (MOM) XP = ldv<float, VW>(xpb + ro);
        Bv = ldv<float, VW>(bb + ro);
      }
#pragma unroll
      for (int e = 0; e < VW; ++e) {
        x0[e] = X.v[e];
        xm[e] = XP.v[e];
        bd[0][e] = Bv.v[e];
      }
    }
    float newx[TL + 1][VW];
#pragma unroll
    for (int e = 0; e < VW; ++e) newx[0][e] = x0[e];
#pragma unroll
    for (int s = 1; s <= TL; ++s) {
      // extend level s's window with row rr - s + 1 of y_{s-1}
      RowT<float, VW> Yn;
      float vn[VW];
#pragma unroll
      for (int e = 0; e < VW; ++e) {
        const float xs1 = newx[s - 1][e];
        const float xs2 = (s == 1) ? xm[e] : prevx[s - 2][e];
        vn[e] = MOM ? xs1 - xs2 : 0.f;
        Yn.y[e] = MOM ? xs1 + atl[s] * vn[e] : xs1;
      }
      row_neighbours<float, VW>(Yn, lane, 0.f, 0.f);
      YU[s] = YC[s];
      YC[s] = YD[s];
      YD[s] = Yn;
      // level s at row rr - s (centre of the window)
      float Ay[VW];
      apply_q1<float, VW, float>(YU[s], YC[s], YD[s], sc, sax, say, sd1, sd2, Ay);
      const int row = rr - s;
      const bool row_in = (row >= 1) && (row <= n);
#pragma unroll
      for (int e = 0; e < VW; ++e) {
        float nx = xc[s][e] + wl[s] * (bd[s][e] - Ay[e]);
        if (MOM) nx = nx + al[s] * vc[s][e];
        newx[s][e] = (row_in && (c0 + e) < n) ? nx : 0.f;
        xc[s][e] = newx[s - 1][e];
        vc[s][e] = vn[e];
      }
    }
    // outputs: x_{k+TL} at row rr - TL, x_{k+TL-1} at row rr - TL + 1
    if (store_cols) {
      const int ra = rr - TL, rb = rr - TL + 1;
      if (ra >= r0 && ra <= r1) {
        VecN<float, VW> O;
#pragma unroll
        for (int e = 0; e < VW; ++e) O.v[e] = newx[TL][e];
        stv<float, VW>(ox + (long long)ra * pitch + c0, O);
      }
      if (MOM && rb >= r0 && rb <= r1) {
        VecN<float, VW> O;
#pragma unroll
        for (int e = 0; e < VW; ++e) O.v[e] = newx[TL - 1][e];
        stv<float, VW>(oxp + (long long)rb * pitch + c0, O);
      }
    }
#pragma unroll
    for (int s = 0; s <= TL; ++s)
#pragma unroll
      for (int e = 0; e < VW; ++e) prevx[s][e] = newx[s][e];
  }
}

richm_status launch_sweep_fused(richm_operator* op, int TL, const float* x, const float* xp, const float* b,
                                float* out_x, float* out_xp, const float* w, const float* a, const float* at, int m,
                                int kidx0, int precond, const int* active, cudaStream_t s) {
  const TileMap* tm = nullptr;
  RICHM_TRY(get_tiles(op, -TL, kFuseRows, &tm));
  SweepTArgs A{op->d_inst, tm->d_tiles, tm->ntiles, x, xp, b, out_x, out_xp, w, a, at, m, kidx0, active};
  const int blocks = (tm->ntiles + kFuseWarps - 1) / kFuseWarps;
  const int thr = kFuseWarps * 32;
  const bool mom = a != nullptr;
#define RICHM_FUSED(TLV)                                                                         \
  if (mom && precond) sweepT_kernel<TLV, true, true><<<blocks, thr, 0, s>>>(A);                 \
  else if (mom) sweepT_kernel<TLV, true, false><<<blocks, thr, 0, s>>>(A);                      \
  else if (precond) sweepT_kernel<TLV, false, true><<<blocks, thr, 0, s>>>(A);                  \
  else sweepT_kernel<TLV, false, false><<<blocks, thr, 0, s>>>(A);
  if (TL == 4) {
    RICHM_FUSED(4)
  } else if (TL == 8) {
    RICHM_FUSED(8)
  } else {
    return set_error(RICHM_ERR_ARG, "fused sweeps support 4 or 8 sweeps per pass");
  }
#undef RICHM_FUSED
  RICHM_LAUNCH_CHECK("fused sweep");
  return RICHM_OK;
}

}  // namespace richm
