// Operator construction, layout, packing, weights and error reporting.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <mutex>

#include "common.cuh"
#include "kernels.cuh"

namespace richm {

namespace {
thread_local std::string g_last_error;
}

richm_status set_error(richm_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return s;
}

void clear_error() { g_last_error.clear(); }

static long long round_up(long long v, long long m) { return (v + m - 1) / m * m; }

// Closed form of the element-assembled Q1 row (Sec. 2.4, eq. 18): q[0..4] = centre,
// x-neighbour, y-neighbour, corner (+1,+1), corner (+1,-1); q[5] = Gershgorin bound.
static void q1_stencil(double eps, double theta, double* q) {
  const double cs = std::cos(theta), sn = std::sin(theta);
  const double c11 = cs * cs + eps * sn * sn;
  const double c22 = sn * sn + eps * cs * cs;
  const double c12 = (1.0 - eps) * sn * cs;
  q[0] = 4.0 * (c11 + c22) / 3.0;
  q[1] = (c22 - 2.0 * c11) / 3.0;
  q[2] = (c11 - 2.0 * c22) / 3.0;
  q[3] = -(c11 + c22) / 6.0 - 0.5 * c12;
  q[4] = -(c11 + c22) / 6.0 + 0.5 * c12;
  q[5] = std::fabs(q[0]) + 2.0 * (std::fabs(q[1]) + std::fabs(q[2]) + std::fabs(q[3]) + std::fabs(q[4]));
}

richm_status get_tiles(richm_operator* op, int tw, int rows, const TileMap** out) {
  long long key = (long long)tw * 1000003LL + rows;
  auto it = op->tiles.find(key);
  if (it != op->tiles.end()) {
    *out = &it->second;
    return RICHM_OK;
  }
  TileMap tm;
  tm.tw = tw;
  tm.rows = rows;
  std::vector<Tile> h;
  tm.h_inst_begin.resize(op->batch + 1);
  for (int b = 0; b < op->batch; ++b) {
    tm.h_inst_begin[b] = (int)h.size();
    const Inst& I = op->h_inst[b];
    const int ty_n = (I.n + rows - 1) / rows;
    if (tw > 0) {  // plain tiles of tw columns
      const int tx_n = (I.pitch + tw - 1) / tw;
      for (int ty = 0; ty < ty_n; ++ty)
        for (int tx = 0; tx < tx_n; ++tx) h.push_back(Tile{b, ty, tx, 0});
    } else {  // fused tiles: 128 columns overlapping by 2*TL at interior edges, and a tail
      int full = 0, half = 0;
      if (tw <= -100) fused_columns(I.n, -tw - 100, &full, &half, 64);  // complex: two columns per lane
      else fused_columns(I.n, -tw, &full, &half);
      for (int ty = 0; ty < ty_n; ++ty)
        for (int tx = 0; tx < full; ++tx) h.push_back(Tile{b, ty, tx, 0});
      if (half)
        for (int ty = 0; ty < ty_n; ty += 2) h.push_back(Tile{b, ty, full, ty + 1 < ty_n ? ty + 3 : 1});
    }
  }
  tm.h_inst_begin[op->batch] = (int)h.size();
  tm.ntiles = (int)h.size();
  RICHM_CUDA_TRY(cudaMalloc(&tm.d_tiles, sizeof(Tile) * h.size()));
  RICHM_CUDA_TRY(cudaMemcpy(tm.d_tiles, h.data(), sizeof(Tile) * h.size(), cudaMemcpyHostToDevice));
  RICHM_CUDA_TRY(cudaMalloc(&tm.d_inst_begin, sizeof(int) * (op->batch + 1)));
  RICHM_CUDA_TRY(cudaMemcpy(tm.d_inst_begin, tm.h_inst_begin.data(), sizeof(int) * (op->batch + 1),
                            cudaMemcpyHostToDevice));
  auto res = op->tiles.emplace(key, tm);
  *out = &res.first->second;
  return RICHM_OK;
}

richm_status check_dtype_for_op(const richm_operator* op, richm_dtype t) {
  RICHM_ARG(dtype_valid(t), "invalid dtype %d", (int)t);
  bool cplx_t = dtype_complex(t);
  for (int b = 0; b < op->batch; ++b) {
    bool helm = op->h_inst[b].kind != RICHM_ANISO_Q1;
    if (helm != cplx_t)
      return set_error(RICHM_ERR_UNSUPPORTED,
                       "instance %d: %s problems use %s dtypes", b, helm ? "Helmholtz" : "Q1",
                       helm ? "complex" : "real");
  }
  return RICHM_OK;
}

// ---------------------------------------------------------------- pack / unpack

template <typename W>
__global__ void pack_kernel(const Inst* insts, const W* __restrict__ dense, W* __restrict__ padded) {
  const Inst I = insts[blockIdx.y];
  int r = blockIdx.x;
  if (r >= I.n + 2) return;
  W* row = padded + I.off + (long long)r * I.pitch;
  bool inner = (r >= 1 && r <= I.n);
  const W* src = dense + I.dense_off + (long long)(r - 1) * I.n;
  for (int c = threadIdx.x; c < I.pitch; c += blockDim.x) {
    W v{};
    if (inner && c < I.n) v = src[c];
    row[c] = v;
  }
}

template <typename W>
__global__ void unpack_kernel(const Inst* insts, const W* __restrict__ padded, W* __restrict__ dense) {
  const Inst I = insts[blockIdx.y];
  int r = blockIdx.x;
  if (r >= I.n) return;
  const W* row = padded + I.off + (long long)(r + 1) * I.pitch;
  W* dst = dense + I.dense_off + (long long)r * I.n;
  for (int c = threadIdx.x; c < I.n; c += blockDim.x) dst[c] = row[c];
}

struct alignas(16) W16 {
  unsigned long long a, b;
};

// Rows 0 and n + 1 of every instance of a padded buffer of `esize`-byte elements.
__global__ void zero_halo_rows_kernel(const Inst* insts, unsigned char* buf, int esize) {
  const Inst& I = insts[blockIdx.x];
  const long long row = blockIdx.y == 0 ? 0 : (long long)(I.n + 1);
  uint4* p = reinterpret_cast<uint4*>(buf + (I.off + row * I.pitch) * esize);
  const int chunks = I.pitch * esize / 16;  // pitch is a multiple of 32 elements
  for (int q = threadIdx.x; q < chunks; q += blockDim.x) p[q] = make_uint4(0u, 0u, 0u, 0u);
}

richm_status launch_zero_halo(const richm_operator* op, void* buf, size_t esize, cudaStream_t s) {
  zero_halo_rows_kernel<<<dim3(op->batch, 2), 128, 0, s>>>(op->d_inst, reinterpret_cast<unsigned char*>(buf),
                                                           (int)esize);
  RICHM_LAUNCH_CHECK("zero halo rows");
  return RICHM_OK;
}

template <bool PACK>
static richm_status pack_dispatch(const richm_operator* op, richm_dtype dt, const void* src, void* dst,
                                  void* stream) {
  RICHM_ARG(op != nullptr, "null operator");
  RICHM_ARG(dtype_valid(dt), "invalid dtype %d", (int)dt);
  RICHM_ARG(src != nullptr && dst != nullptr, "null buffer");
  dim3 grid(op->max_n + 2, op->batch);
  cudaStream_t s = (cudaStream_t)stream;
  size_t es = dtype_size(dt);
  if (PACK) {
    if (es == 2) pack_kernel<uint16_t><<<grid, 256, 0, s>>>(op->d_inst, (const uint16_t*)src, (uint16_t*)dst);
    else if (es == 4) pack_kernel<uint32_t><<<grid, 256, 0, s>>>(op->d_inst, (const uint32_t*)src, (uint32_t*)dst);
    else if (es == 8) pack_kernel<unsigned long long><<<grid, 256, 0, s>>>(op->d_inst, (const unsigned long long*)src, (unsigned long long*)dst);
    else pack_kernel<W16><<<grid, 256, 0, s>>>(op->d_inst, (const W16*)src, (W16*)dst);
  } else {
    if (es == 2) unpack_kernel<uint16_t><<<grid, 256, 0, s>>>(op->d_inst, (const uint16_t*)src, (uint16_t*)dst);
    else if (es == 4) unpack_kernel<uint32_t><<<grid, 256, 0, s>>>(op->d_inst, (const uint32_t*)src, (uint32_t*)dst);
    else if (es == 8) unpack_kernel<unsigned long long><<<grid, 256, 0, s>>>(op->d_inst, (const unsigned long long*)src, (unsigned long long*)dst);
    else unpack_kernel<W16><<<grid, 256, 0, s>>>(op->d_inst, (const W16*)src, (W16*)dst);
  }
  RICHM_LAUNCH_CHECK(PACK ? "pack" : "unpack");
  return RICHM_OK;
}

}  // namespace richm

using namespace richm;

extern "C" {

const char* richm_last_error(void) { return g_last_error.c_str(); }

const char* richm_version(void) { return "richm 0.1 (sm_103a)"; }

richm_status richm_operator_create(const richm_pde* pdes, int batch, richm_operator** out) {
  clear_error();
  RICHM_ARG(out != nullptr, "null output handle");
  *out = nullptr;
  RICHM_ARG(pdes != nullptr, "null pde array");
  RICHM_ARG(batch >= 1 && batch <= (1 << 20), "batch %d out of range", batch);
  auto* op = new (std::nothrow) richm_operator();
  if (!op) return set_error(RICHM_ERR_NOMEM, "host allocation failed");
  op->batch = batch;
  op->pdes.assign(pdes, pdes + batch);
  op->h_inst.resize(batch);
  long long off = 0, doff = 0;
  for (int b = 0; b < batch; ++b) {
    const richm_pde& p = pdes[b];
    if (p.n < 1 || p.n > 16383) {
      delete op;
      return set_error(RICHM_ERR_ARG, "instance %d: n = %d out of range [1, 16383]", b, p.n);
    }
    Inst I{};
    I.n = p.n;
    I.kind = p.kind;
    I.pitch = (int)round_up(p.n + 1, 32);
    I.off = off;
    I.dense_off = doff;
    off = round_up(off + (long long)(p.n + 2) * I.pitch, 64);
    doff += (long long)p.n * p.n;
    if (p.kind == RICHM_ANISO_Q1) {
      if (!(p.eps > 0.0 && p.eps <= 1.0) || !std::isfinite(p.theta)) {
        delete op;
        return set_error(RICHM_ERR_ARG, "instance %d: need 0 < eps <= 1 and finite theta", b);
      }
      double q[6];
      q1_stencil(p.eps, p.theta, q);
      I.c = q[0];
      I.ax = q[1];
      I.ay = q[2];
      I.d1 = q[3];
      I.d2 = q[4];
      I.dinv = 1.0 / I.c;
      I.G = q[5];
    } else if (p.kind == RICHM_HELMHOLTZ_FD5_ABC || p.kind == RICHM_HELMHOLTZ_FD5_DIRICHLET ||
               p.kind == RICHM_HELMHOLTZ_FD5_SPONGE) {
      if (!(p.k >= 0.0) || !std::isfinite(p.k)) {
        delete op;
        return set_error(RICHM_ERR_ARG, "instance %d: need finite k >= 0", b);
      }
      double h = 1.0 / (p.n + 1);
      double kh = p.k * h;
      I.c = (4.0 - kh * kh) / (h * h);
      I.ax = I.ay = -1.0 / (h * h);
      I.d1 = I.d2 = 0.0;
      if (p.kind == RICHM_HELMHOLTZ_FD5_ABC) {
        // -g/h^2 with g = 1/(1 - i k h) = (1 + i k h)/(1 + k^2 h^2)
        double den = 1.0 + kh * kh;
        I.abc_re = -(1.0 / den) / (h * h);
        I.abc_im = -(kh / den) / (h * h);
      }
      if (p.kind == RICHM_HELMHOLTZ_FD5_SPONGE && p.k > 0.0) {
        // eq. 21 with c = 1: i gamma omega on the diagonal, gamma = k max(0, 1 - d / L),
        // L = 2 pi / k one wavelength, d the distance to the boundary
        I.sp_im = p.k * p.k;
        I.sp_iw = h * p.k / (2.0 * 3.14159265358979323846);  // h / L
      }
      // Gershgorin: largest row sum over the row types that exist for this n (a node at
      // distance d >= 2 from the boundary has four neighbours, and its sponge term is at
      // most that of d = 2)
      double off1 = 1.0 / (h * h);
      auto rowsum = [&](int missing, int d) {
        double dr = I.c + missing * I.abc_re;
        double di = missing * I.abc_im + I.sp_im * std::max(0.0, 1.0 - d * I.sp_iw);
        return std::sqrt(dr * dr + di * di) + (4 - missing) * off1;
      };
      double G = 0.0;
      if (p.n == 1) G = rowsum(4, 1);
      else {
        G = std::max(G, rowsum(2, 1));
        G = std::max(G, rowsum(p.n >= 3 ? 1 : 2, 1));
        if (p.n >= 3) G = std::max(G, rowsum(0, 2));
      }
      I.G = G;
      I.dinv = 0.0;
    } else {
      delete op;
      return set_error(RICHM_ERR_ARG, "instance %d: unknown problem kind %d", b, p.kind);
    }
    op->max_n = std::max(op->max_n, p.n);
    op->h_inst[b] = I;
  }
  op->elems = (size_t)off;
  cudaError_t e = cudaGetDevice(&op->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&op->sms, cudaDevAttrMultiProcessorCount, op->device);
  if (e == cudaSuccess) {
    // kernel attributes, once per device (a stream capture may follow later calls)
    static std::mutex mu;
    static std::vector<int> done;
    std::lock_guard<std::mutex> lock(mu);
    if (std::find(done.begin(), done.end(), op->device) == done.end()) {
      e = init_sweep_attributes();
      if (e == cudaSuccess) done.push_back(op->device);
    }
  }
  if (e == cudaSuccess) e = cudaMalloc(&op->d_inst, sizeof(Inst) * batch);
  if (e == cudaSuccess)
    e = cudaMemcpy(op->d_inst, op->h_inst.data(), sizeof(Inst) * batch, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    if (op->d_inst) cudaFree(op->d_inst);
    delete op;
    return set_error(e == cudaErrorMemoryAllocation ? RICHM_ERR_NOMEM : RICHM_ERR_CUDA,
                     "descriptor upload failed: %s", cudaGetErrorString(e));
  }
  *out = op;
  return RICHM_OK;
}

void richm_operator_destroy(richm_operator* op) {
  if (!op) return;
  for (auto& kv : op->tiles) {
    cudaFree(kv.second.d_tiles);
    cudaFree(kv.second.d_inst_begin);
  }
  richm::solver_release_oneshot(op);
  if (op->d_inst) cudaFree(op->d_inst);
  richm::fourier_release(op);
  delete op;
}

richm_status richm_operator_batch(const richm_operator* op, int* batch) {
  RICHM_ARG(op && batch, "null argument");
  *batch = op->batch;
  return RICHM_OK;
}

richm_status richm_stencil(const richm_operator* op, int instance, double* coef) {
  RICHM_ARG(op && coef, "null argument");
  RICHM_ARG(instance >= 0 && instance < op->batch, "instance %d out of range", instance);
  const Inst& I = op->h_inst[instance];
  for (int i = 0; i < 8; ++i) coef[i] = 0.0;
  if (I.kind == RICHM_ANISO_Q1) {
    coef[0] = I.c; coef[1] = I.ax; coef[2] = I.ay; coef[3] = I.d1; coef[4] = I.d2;
  } else {
    coef[0] = I.c; coef[1] = I.ax; coef[2] = I.abc_re; coef[3] = I.abc_im;
    coef[4] = I.sp_im; coef[5] = I.sp_iw > 0.0 ? 1.0 / I.sp_iw : 0.0;
  }
  return RICHM_OK;
}

richm_status richm_q1_stencil(double eps, double theta, double* coef) {
  clear_error();
  RICHM_ARG(coef != nullptr, "null output");
  RICHM_ARG(eps > 0.0 && eps <= 1.0 && std::isfinite(theta), "need 0 < eps <= 1 and finite theta");
  q1_stencil(eps, theta, coef);
  return RICHM_OK;
}

richm_status richm_gershgorin(const richm_operator* op, double* lmax) {
  RICHM_ARG(op && lmax, "null argument");
  for (int b = 0; b < op->batch; ++b) lmax[b] = op->h_inst[b].G;
  return RICHM_OK;
}

richm_status richm_chebyshev_weights(double lmax, double lmin, int m, double* w) {
  RICHM_ARG(w != nullptr, "null output");
  RICHM_ARG(m >= 1, "m = %d < 1", m);
  RICHM_ARG(lmin > 0.0 && lmax > lmin && std::isfinite(lmax), "need 0 < lmin < lmax");
  const double pi = 3.14159265358979323846;
  for (int i = 1; i <= m; ++i) {
    double x = std::cos((2.0 * i - 1.0) * pi / (2.0 * m));
    w[i - 1] = 2.0 / (lmax + lmin + (lmax - lmin) * x);
  }
  return RICHM_OK;
}

richm_status richm_layout(const richm_operator* op, int instance, size_t* offset, int* pitch, int* rows) {
  RICHM_ARG(op != nullptr, "null operator");
  RICHM_ARG(instance >= 0 && instance < op->batch, "instance %d out of range", instance);
  const Inst& I = op->h_inst[instance];
  if (offset) *offset = (size_t)I.off;
  if (pitch) *pitch = I.pitch;
  if (rows) *rows = I.n + 2;
  return RICHM_OK;
}

richm_status richm_buffer_elems(const richm_operator* op, size_t* elems) {
  RICHM_ARG(op && elems, "null argument");
  *elems = op->elems;
  return RICHM_OK;
}

richm_status richm_pack(const richm_operator* op, richm_dtype dtype, const void* dense, void* padded,
                        void* stream) {
  clear_error();
  return pack_dispatch<true>(op, dtype, dense, padded, stream);
}

richm_status richm_unpack(const richm_operator* op, richm_dtype dtype, const void* padded, void* dense,
                          void* stream) {
  clear_error();
  return pack_dispatch<false>(op, dtype, padded, dense, stream);
}

}  // extern "C"
