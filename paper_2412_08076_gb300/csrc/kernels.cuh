// Internal launchers shared between the library's translation units.
#pragma once

#include "common.cuh"

namespace richm {

// Kernel attributes that must be set before the first launch (called once per
// process and device by richm_operator_create).
cudaError_t init_sweep_attributes();  // also the fused, SSOR and adjoint kernels
cudaError_t init_fused_attributes();
cudaError_t init_ssor_attributes();
cudaError_t init_adjoint_attributes();

// One forward sweep (see sweep.cu). `a == nullptr`: no momentum (xp unused);
// `at == nullptr`: at = a. `active`: per-instance flags or nullptr (all active).
template <typename E>
richm_status launch_sweep(richm_operator* op, const E* x, const E* xp, const E* b, E* out,
                          const typename RealOf<E>::type* w, const typename RealOf<E>::type* a,
                          const typename RealOf<E>::type* at, int m, int kidx, int precond, const int* active,
                          cudaStream_t s);

// TL (4 or 8) fused FP32 sweeps of a real Q1 batch: reads (x_k, x_{k-1}) from
// (x, xp), writes (x_{k+TL}, x_{k+TL-1}) to (out_x, out_xp); the outputs must not
// alias the inputs. kidx0 = coefficient index of the first sweep.
// rows: output rows of a warp tile (a multiple of 16 up to 256); <= 0 takes the operator's
// tuned value. absorb: the input pair (x, xp) stands for (0, xp - x), the state after
// the mixed-precision refinement moved x into the FP64 solution (the solver's first
// pass of a cycle).
richm_status launch_sweep_fused(richm_operator* op, int TL, const float* x, const float* xp, const float* b,
                                float* out_x, float* out_xp, const float* w, const float* a, const float* at, int m,
                                int kidx0, int precond, const int* active, cudaStream_t s, int rows = 0,
                                bool absorb = false);

// TL (4) fused complex64 sweeps of a Helmholtz batch (no preconditioner), same
// conventions as launch_sweep_fused.
richm_status launch_sweep_fused_cx(richm_operator* op, int TL, const cplx<float>* x, const cplx<float>* xp,
                                   const cplx<float>* b, cplx<float>* out_x, cplx<float>* out_xp, const float* w,
                                   const float* a, const float* at, int m, int kidx0, const int* active,
                                   cudaStream_t s, int rows = 0);

// The same with bfloat16 state (x, x_prev and the outputs); b and the arithmetic are FP32.
richm_status launch_sweep_fused_bf16(richm_operator* op, int TL, const __nv_bfloat16* x, const __nv_bfloat16* xp,
                                     const float* b, __nv_bfloat16* out_x, __nv_bfloat16* out_xp, const float* w,
                                     const float* a, const float* at, int m, int kidx0, int precond,
                                     const int* active, cudaStream_t s, int rows = 0, bool absorb = false);

// Zero rows 0 and n + 1 of every instance of a padded buffer (esize-byte elements). The
// sweep kernels write rows 1..n of their outputs only; a workspace buffer whose result
// is copied back to the caller gets its halo rows cleared first.
richm_status launch_zero_halo(const richm_operator* op, void* buf, size_t esize, cudaStream_t s);

// One SSOR-preconditioned sweep of a Q1 batch (E = float or double): forward triangular
// solve into z, backward solve and the Table 1 update into (out_x, out_xp). z: a padded
// scratch buffer (no initial contents needed); the outputs must not alias the inputs.
template <typename E>
richm_status launch_ssor_sweep(richm_operator* op, const E* x, const E* xp, const E* b, E* z, E* out_x, E* out_xp,
                               const E* w, const E* a, const E* at, int m, int kidx, double relax, const int* active,
                               cudaStream_t s);

// out = B^{-1} r with the SSOR B^{-1} of relaxation factor `relax` (the same two
// triangular solves, y = 0); z: padded scratch. out must alias neither r nor z.
template <typename E>
richm_status launch_ssor_apply(richm_operator* op, const E* r, E* z, E* out, double relax, cudaStream_t s);

// r = b - A x in FP64 with per-tile partial sums (sum |r|^2, sum |b|^2) written to
// `partials` (one double2 per warp tile of the residual geometry); r_out may be null.
template <typename E>
richm_status launch_residual(richm_operator* op, const E* x, const E* b, E* r_out, double2* partials,
                             cudaStream_t s);

// Residual of an FP64 state written in another type (the mixed-precision solver's
// inner right-hand side); instances with active[b] == 0 are skipped. With
// `refinement` the partials hold (|r|^2, 0): the solver knows |b| from its first
// residual and skips that sum.
template <typename E, typename RO>
richm_status launch_residual_to(richm_operator* op, const E* x, const E* b, RO* r_out, double2* partials,
                                const int* active, cudaStream_t s, bool refinement);

// out = A x in FP64 (written in RO) over rows 1..n of every instance (columns >= n
// written as zero); the halo rows of out are not touched.
template <typename E, typename RO>
richm_status launch_apply_to(richm_operator* op, const E* x, RO* out, cudaStream_t s);

// Bytes of the loss workspace (residual buffer, partials, three per-instance arrays).
size_t loss_workspace_bytes(richm_operator* op, size_t elem_size, int ntiles);

// Per-instance reduction of residual partials into norms (each output may be null).
richm_status launch_norm_reduce(richm_operator* op, int residual_vw, const double2* partials, double* rnorm,
                                double* bnorm, double* rel, cudaStream_t s);

// Number of warp tiles of the residual kernel for state type E.
template <typename E>
richm_status residual_tiles(richm_operator* op, int* ntiles);

}  // namespace richm
