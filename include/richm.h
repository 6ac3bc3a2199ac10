/*
 * richm.h - C ABI of the GB300 Richardson(m) stencil library (librichm.so).
 *
 * The library solves batches of linear systems A u = f (eq. 1 of "Momentum-
 * Accelerated Richardson(m) and Their Multilevel Neural Solvers") arising from
 *   - the anisotropic diffusion problem -div(C grad u) = f, u = 0 on the boundary,
 *     C = R(theta) diag(1, eps) R(theta)^T, bilinear (Q1) elements on a uniform
 *     mesh of the unit square (eq. 18 and Sec. 2.4), and
 *   - the Helmholtz problem -Lap(u) - k^2 u = f with the 5-point stencil of eq. 22,
 * with the long-step iterations of Table 1 (Richardson(m), MOM-, NAG- and
 * NAGex-Richardson(m)) and the preconditioned form of eq. 17 with B^{-1} = D^{-1}.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Grids. Instance b has n_b x n_b interior unknowns, h = 1/(n_b + 1). Unknown
 *   (i, j) sits at x = (j + 1) h, y = (i + 1) h (column index = x, row index = y).
 * Padded layout. Grid arrays live in one device buffer per field holding every
 *   instance. Instance b occupies rows 0 .. n_b+1 of width `pitch_b` elements
 *   starting at element `offset_b` (richm_layout): row 0 and row n_b+1 are zero
 *   halo rows, unknown (i, j) is element offset_b + (i+1)*pitch_b + j, and the
 *   columns n_b .. pitch_b-1 of every row are zero padding (pitch_b >= n_b + 1, a
 *   multiple of 32; offset_b a multiple of 64). The layout in elements is the same
 *   for every dtype. Every element outside the interior MUST be zero on input;
 *   the library keeps it zero on output. richm_pack / richm_unpack convert from /
 *   to dense row-major n_b x n_b blocks.
 * Ownership. Grid buffers, weights, outputs and workspaces are caller-owned
 *   device memory unless a parameter says "host". The operator handle is
 *   library-owned (richm_operator_create / richm_operator_destroy) and holds a
 *   small device copy of the instance descriptors. All device pointers must
 *   belong to the device that was current when the operator was created, and
 *   that device must be current in every call.
 * Streams. `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *   stream). Calls are stream-ordered and asynchronous unless documented
 *   otherwise; the library synchronises only where an entry point returns host
 *   results (richm_solve).
 * Weights. Sweep k (0-based, global) uses coefficient index (k mod m), i.e. the
 *   paper's w_{(k mod m)+1}. Coefficient arrays are [batch][m], row-major, in the
 *   real type of the state dtype (float for RICHM_F32/RICHM_C64, double for
 *   RICHM_F64/RICHM_C128).
 * Errors. Every call returns a richm_status. Argument errors are detected before
 *   any work is queued and leave every buffer untouched. RICHM_ERR_CUDA reports a
 *   failed launch or CUDA call; richm_last_error() gives a message (thread-local,
 *   valid until the next call from the same thread). No C++ exception crosses
 *   this interface.
 */
#ifndef RICHM_H
#define RICHM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  RICHM_OK = 0,
  RICHM_ERR_ARG = 1,           /* invalid argument (null pointer, bad size, bad enum) */
  RICHM_ERR_CUDA = 2,          /* a CUDA runtime / cuFFT call or kernel launch failed */
  RICHM_ERR_NOMEM = 3,         /* workspace too small or a library allocation failed */
  RICHM_ERR_NOT_CONVERGED = 4, /* richm_solve: an instance reached max_sweeps */
  RICHM_ERR_DIVERGED = 5,      /* richm_solve: an instance's residual became non-finite or > 1e30 ||f|| */
  RICHM_ERR_UNSUPPORTED = 6    /* valid request the library does not implement (e.g. dtype/problem mix) */
} richm_status;

typedef enum {
  RICHM_ANISO_Q1 = 0,              /* eq. 18, bilinear elements, Dirichlet eliminated (Sec. 2.4) */
  RICHM_HELMHOLTZ_FD5_ABC = 1,     /* eq. 22 interior rows; first-order absorbing boundary */
  RICHM_HELMHOLTZ_FD5_DIRICHLET = 2,/* eq. 22 interior rows; u = 0 on the boundary */
  RICHM_HELMHOLTZ_FD5_SPONGE = 3   /* eq. 21: eq. 22's stencil, u = 0 on the boundary, and the damping
                                      term i gamma(x) omega / c^2 on the diagonal, with c = 1 (omega = k),
                                      gamma = k max(0, 1 - d(x)/L), d(x) the distance to the boundary and
                                      L = 2 pi / k one wavelength (a linear ramp: the paper gives the layer's
                                      thickness and end values only) */
} richm_problem;

typedef enum {
  RICHM_F64 = 0,   /* double */
  RICHM_F32 = 1,   /* float */
  RICHM_C64 = 2,   /* complex64: interleaved {float re, float im} */
  RICHM_C128 = 3,  /* complex128: interleaved {double re, double im} */
  RICHM_BF16 = 4   /* bfloat16 storage of the iterate with FP32 arithmetic (Q1 sweeps and the solver's
                      inner state only; the right-hand side and the weights stay FP32) */
} richm_dtype;

/* Output head of the meta network (Sec. 2.3): which Table 1 method its outputs
 * parametrise, and how many there are for m steps. */
typedef enum {
  RICHM_HEAD_NAG_SHARED = 0, /* m + 1: w_i and one momentum a for every step (NAG, at = a) */
  RICHM_HEAD_RICHARDSON = 1, /* m: w_i only (Richardson(m)) */
  RICHM_HEAD_MOM = 2,        /* 2m: w_i, a_i; at_i = 0 (MOM) */
  RICHM_HEAD_NAG = 3,        /* 2m: w_i, a_i; at_i = a_i (NAG) */
  RICHM_HEAD_NAGEX = 4,      /* 3m: w_i, a_i, at_i (NAGex) */
  RICHM_HEAD_RAW = 5         /* m outputs o_i written as they are (w_out[b][i] = o_i; G unused): the
                                parameters of the FNS symbol and transition maps (richm_symbol_from_stencil,
                                richm_transition_from_band) */
} richm_meta_head;

/* One PDE instance. eps, theta: anisotropy strength (0 < eps <= 1) and angle for
 * RICHM_ANISO_Q1; k: wavenumber for the Helmholtz kinds (k >= 0). */
typedef struct {
  int kind;      /* richm_problem */
  int n;         /* interior unknowns per direction, 1 <= n <= 16383 */
  double eps;
  double theta;
  double k;
} richm_pde;

typedef struct richm_operator richm_operator;

/* ------------------------------------------------------------------ setup */

/* Build the discrete operators of `batch` instances (eq. 18 / eq. 22).
 * Q1 stencil (closed form of the element-assembled matrix, Sec. 2.4): with
 * c11 = cos^2 t + eps sin^2 t, c22 = sin^2 t + eps cos^2 t, c12 = (1-eps) sin t cos t,
 *   centre 4(c11+c22)/3, x-neighbours (c22-2c11)/3, y-neighbours (c11-2c22)/3,
 *   corners (+1,+1),(-1,-1): -(c11+c22)/6 - c12/2; (+1,-1),(-1,+1): -(c11+c22)/6 + c12/2.
 * Helmholtz (eq. 22): centre (4 - k^2 h^2)/h^2, neighbours -1/h^2; with the
 *   absorbing boundary each missing neighbour adds -1/((1 - i k h) h^2) to the
 *   diagonal (ghost value u_0 = u_1/(1 - i k h) from du/dn - i k u = 0).
 * pdes: host [batch]. *out receives a library-owned handle. Errors: RICHM_ERR_ARG
 * for batch < 1 or an invalid instance; RICHM_ERR_NOMEM / RICHM_ERR_CUDA if the
 * device copy of the descriptors cannot be made. */
richm_status richm_operator_create(const richm_pde* pdes, int batch, richm_operator** out);
void richm_operator_destroy(richm_operator* op);

/* Number of instances. */
richm_status richm_operator_batch(const richm_operator* op, int* batch);

/* Host FP64 stencil coefficients of one instance.
 * Q1: coef[0..4] = centre, x-neighbour, y-neighbour, corner(+1,+1), corner(+1,-1).
 * Helmholtz: coef[0] = centre, coef[1] = neighbour, coef[2..3] = (re, im) added to the
 * diagonal per missing neighbour (0 for Dirichlet and the sponge layer); sponge layer:
 * coef[4] = the imaginary diagonal term on the boundary (k^2) and coef[5] = the layer's
 * width L/h in grid spacings, so that a node at distance d h from the boundary gains
 * i coef[4] max(0, 1 - d / coef[5]). coef: host [8]. */
richm_status richm_stencil(const richm_operator* op, int instance, double* coef);

/* The Q1 stencil of richm_operator_create for one (eps, theta) without an operator
 * (host only, no device memory): coef[0..4] = centre, x-neighbour, y-neighbour,
 * corner(+1,+1), corner(+1,-1); coef[5] = the Gershgorin bound |c| + 2 sum |off|.
 * coef: host [6]. Errors: RICHM_ERR_ARG unless 0 < eps <= 1 and theta is finite. */
richm_status richm_q1_stencil(double eps, double theta, double* coef);

/* Gershgorin bound max_i sum_j |a_ij| per instance (the lmax estimate used with
 * eqs. 8-9 in the Chebyshev semi-iteration, Sec. 2.1). lmax: host [batch]. */
richm_status richm_gershgorin(const richm_operator* op, double* lmax);

/* Chebyshev-optimal weights (eqs. 8-9): w_i = 2/(lmax + lmin + (lmax - lmin) x_i),
 * x_i = cos((2i-1) pi / 2m), i = 1..m, returned in index order. w: host [m].
 * Errors: RICHM_ERR_ARG unless 0 < lmin < lmax and m >= 1. */
richm_status richm_chebyshev_weights(double lmax, double lmin, int m, double* w);

/* Order of the steps inside a period. Eqs. 8-9 fix the set of weights of a period,
 * not the order of its steps; in FP32 the order decides how much the rounding made at
 * one step is amplified by the later (long) steps of the same period. This reorders
 * them by a Leja ordering of the nodes z_i = 1/w_i (the roots of the period's residual
 * polynomial): first the node of largest |z|, then repeatedly the node maximising the
 * product (FP64, in the order taken) of its distances to the nodes already taken, ties
 * to the smaller index (Reichel 1990). The paper has no counterpart; it is an option
 * of this library.
 * richm_leja_order (host): w: host [m] (nonzero, finite), perm: host [m] receives the
 * permutation, perm[s] = index of the step that runs at position s; 1 <= m <= 64.
 * richm_leja_permute (device, stream-ordered): for every instance b of the operator,
 * w_out[b][s] = w[b][perm_b[s]] with perm_b the Leja order of w[b][:], and alpha_out,
 * alpha_t_out the same permutation of alpha, alpha_t (a step's coefficients move
 * together); arrays [batch][m] in the real type of dtype (float for RICHM_F32,
 * RICHM_C64, RICHM_BF16; double for RICHM_F64, RICHM_C128). alpha / alpha_t and their
 * outputs are both given or both NULL. Not in place. Errors: RICHM_ERR_ARG. */
richm_status richm_leja_order(const double* w, int m, int* perm);
richm_status richm_leja_permute(const richm_operator* op, richm_dtype dtype, const void* w, const void* alpha,
                                const void* alpha_t, int m, void* w_out, void* alpha_out, void* alpha_t_out,
                                void* stream);

/* Padded layout of one instance (see the header comment): element offset of its
 * row 0, row pitch in elements, and number of rows (n + 2). Host outputs. */
richm_status richm_layout(const richm_operator* op, int instance, size_t* offset, int* pitch, int* rows);

/* Elements of one padded field buffer holding every instance. Host output. */
richm_status richm_buffer_elems(const richm_operator* op, size_t* elems);

/* Dense <-> padded conversion on the device. dense: instances concatenated, each
 * n_b*n_b row-major. richm_pack writes every element of `padded` (zeros outside
 * the interior). Buffers must not overlap. */
richm_status richm_pack(const richm_operator* op, richm_dtype dtype, const void* dense, void* padded, void* stream);
richm_status richm_unpack(const richm_operator* op, richm_dtype dtype, const void* padded, void* dense, void* stream);

/* ------------------------------------------------------------------ sweeps */

typedef struct {
  int m;        /* period length, 1 <= m <= 64 */
  int k_start;  /* global index of the first sweep */
  int precond;  /* 0: B^{-1} = I; 1: B^{-1} = D^{-1} (eq. 17 with the Jacobi preconditioner);
                   2: B^{-1} = relax (2 - relax) (D - relax U)^{-1} D (D - relax L)^{-1}, the SSOR
                   preconditioner listed after eq. 17, with A = D - L - U split in the row-major
                   numbering of each instance's unknowns (Q1, RICHM_F32 or RICHM_F64, one sweep per
                   pass) */
  int fuse;     /* sweeps per pass over HBM (temporal blocking): 0 = library choice, else 1, 2, 4 or 8
                   (RICHM_F32 / RICHM_BF16 Q1: 4 or 8; RICHM_C64 Helmholtz without preconditioner,
                   absorbing, Dirichlet or sponge boundary: 4; other cases run one sweep per pass) */
  double relax; /* SSOR relaxation factor, 0 < relax < 2 (precond = 2 only) */
} richm_sweep_opts;

/* Workspace bytes richm_apply_sweeps needs for `dtype` (three padded buffers). */
richm_status richm_sweeps_workspace(const richm_operator* op, richm_dtype dtype, size_t* bytes);

/* K sweeps of the Table 1 iteration in the two-level form
 *   y       = x_k + at_i (x_k - x_{k-1})
 *   x_{k+1} = x_k + a_i (x_k - x_{k-1}) + w_i B^{-1} (b - A y),   i = k mod m,
 * which is Table 1's velocity form with v_k = x_k - x_{k-1}: a = at = 0 gives
 * Richardson(m) (eqs. 2-5), at = 0 MOM-, at = a NAG- and general at NAGex-
 * Richardson(m); precond = 1 applies eq. 17 with B^{-1} = D^{-1}.
 * x (in: x_{k_start}, out: x_{k_start+K}) and x_prev (in: x_{k_start-1}, out:
 * x_{k_start+K-1}) are padded buffers; b is the padded right-hand side.
 * w: [batch][m] (required); alpha: [batch][m] or NULL (no momentum; x_prev may then
 * be NULL and is not written); alpha_t: [batch][m] or NULL (= alpha, i.e. NAG).
 * dtype: RICHM_F32/RICHM_F64 for Q1, RICHM_C64/RICHM_C128 for Helmholtz (weights real).
 * RICHM_BF16 (Q1): x and x_prev hold bfloat16, b and the weights are FP32, the sweeps
 * run in FP32 in fused passes only (fuse 4 or 8, or 0 with a tuned pass length > 1;
 * K must be a multiple of it) and each pass rounds its two output levels to bfloat16.
 * work: at least richm_sweeps_workspace bytes. K = 0 is a no-op. */
richm_status richm_apply_sweeps(richm_operator* op, richm_dtype dtype, void* x, void* x_prev, const void* b,
                                const void* w, const void* alpha, const void* alpha_t, int K,
                                const richm_sweep_opts* opts, void* work, size_t work_bytes, void* stream);

/* Autotuner: times 16 FP32 sweeps of this operator's batch with 1 sweep per launch
 * and with 4 or 8 sweeps per pass (richm_apply_sweeps' fuse) on warp tiles of 64,
 * 128 or 256 rows, and stores the fastest pair in the operator. Every fused launch
 * then uses the tuned tile height, and calls with fuse = 0 (richm_apply_sweeps on
 * RICHM_F32, richm_solve / richm_solver_create with inner RICHM_F32) the tuned pass
 * length (before any tuning: 4 sweeps per pass, 256 rows). momentum: 1 times the NAG
 * kernels, 0 the plain ones. Synchronises `stream`. best_fuse (host, may be NULL)
 * receives the pass length and ms_per_sweep (host, may be NULL) its time per sweep.
 * work: at least richm_autotune_workspace bytes (overwritten). Q1 operators only. */
richm_status richm_autotune_workspace(const richm_operator* op, size_t* bytes);
richm_status richm_autotune(richm_operator* op, int m, int momentum, void* work, size_t work_bytes, void* stream,
                            int* best_fuse, float* ms_per_sweep);

/* The operator's current pass length and fused tile height (host outputs, may be NULL). */
richm_status richm_tuned(const richm_operator* op, int* fuse, int* rows);

/* Set them without timing (fuse: 1, 4 or 8; rows: a multiple of 16 from 16 to 256).
 * Affects later calls. */
richm_status richm_set_tuning(richm_operator* op, int fuse, int rows);

/* ------------------------------------------------------------------ residual */

/* Workspace bytes richm_residual_norm needs (per-tile FP64 partial sums). */
richm_status richm_residual_workspace(const richm_operator* op, size_t* bytes);

/* r = b - A x and its norms (eq. 15 and the stopping test of Sec. 2.4), summed in
 * FP64 whatever the state dtype (complex: |r|^2). Outputs are device [batch]
 * arrays; each may be NULL: rnorm = ||r||_2, bnorm = ||b||_2, rel = rnorm / bnorm.
 * r_out: padded buffer of the same dtype receiving r, or NULL. Deterministic:
 * partial sums are combined in a fixed order. */
richm_status richm_residual_norm(richm_operator* op, richm_dtype dtype, const void* x, const void* b,
                                 double* rnorm, double* bnorm, double* rel, void* r_out,
                                 void* work, size_t work_bytes, void* stream);

/* The same residual and norms as richm_residual_norm for callers that cannot
 * allocate device memory where they need them: code running inside a memory pool or
 * allocator callback it does not own, or a process whose device memory another
 * framework reserved up front. The paper has no counterpart; this is an interface
 * convenience. The scratch (per-tile partial sums and per-instance tile offsets)
 * lives in file-scope device arrays of the library, present on every GPU that loads
 * it until the process exits (1 MiB + 256 KiB); the call allocates nothing.
 * Limits: at most 65536 warp tiles (tiles of 16 rows x 32 lanes x one 16-byte vector:
 * about 134 M FP32, 67 M FP64 or complex64 and 33 M complex128 unknowns, less the
 * padding of each row to its 32-element pitch) and 65536 instances; larger batches
 * return RICHM_ERR_NOMEM before any work is queued. Every call looks up the arrays'
 * device addresses on the current device (cudaGetSymbolAddress, host-side; no address
 * is kept between calls, so a context that is destroyed and made again is safe); the
 * first call on a device may load the library's module there, so make it before any
 * stream capture. Every call shares the arrays and rewrites all
 * the entries it reads, so nothing needs clearing, but calls that overlap on the GPU
 * (different streams, threads or devices' contexts racing on one array) race: order
 * them. Outputs and error behaviour are those of richm_residual_norm. */
richm_status richm_residual_norm_static(richm_operator* op, richm_dtype dtype, const void* x, const void* b,
                                        double* rnorm, double* bnorm, double* rel, void* r_out, void* stream);

/* ------------------------------------------------------------------ solve */

typedef struct {
  int m;                 /* period length */
  double tol;            /* stop an instance once ||b - A x|| / ||b|| <= tol (FP64 residual) */
  long long max_sweeps;  /* per instance */
  int refine_every;      /* sweeps between FP64 refinement steps / convergence checks (>= 1) */
  int inner;             /* richm_dtype of the inner sweeps: RICHM_F32 (mixed precision), RICHM_F64, or
                            RICHM_BF16 (bfloat16 inner state, FP32 arithmetic and rhs; fused sweeps) */
  int precond;           /* as in richm_sweep_opts (2, SSOR: one sweep per launch, fuse 0 or 1) */
  int fuse;              /* as in richm_sweep_opts */
  int use_graph;         /* 1: replay the refinement cycle as a CUDA graph */
  double relax;          /* as in richm_sweep_opts */
  int fp64_residual;     /* fused FP32 / BF16 cycles: 0 (default) forms each refinement's r = b - A x in
                            64-bit fixed point (error below the FP64 evaluation's, see rel_res), 1 in
                            FP64 arithmetic (slower on GB300); other solves always use FP64 */
} richm_solve_opts;

typedef struct {
  long long sweeps;  /* sweeps applied to this instance */
  double rel_res;    /* final relative residual ||b - A x|| / ||b||: r = b - A x in FP64, or, after
                        fused FP32 cycles, in 64-bit fixed point per tile (error below FP64
                        evaluation's) with |r|^2 summed as FP32 pairs (relative error below 1e-12) */
  int status;        /* RICHM_OK, RICHM_ERR_NOT_CONVERGED or RICHM_ERR_DIVERGED */
} richm_solve_info;

/* Workspace bytes of richm_solve / richm_solver_create: four inner-state buffers, the
 * inner right-hand side, per-tile partial sums, per-instance arrays and, for an FP32 or
 * bfloat16 inner state, a second padded FP64 solution buffer (fused cycles alternate
 * between it and x). Layout, for inspecting a session between steps (with
 * E = elems x the inner state's element size rounded up to 256 bytes): inner-state
 * buffer j (padded, inner dtype) at byte j*E, j = 0..3; the inner right-hand side
 * (padded, FP64 for an FP64 inner state, else FP32) at 4*E; the second FP64 solution
 * buffer in the last elems*8 bytes rounded up to 256. After cycle c of a fused session
 * (refine_every/fuse passes per cycle) the cycle's final pair (e_k, e_{k-1}) is in
 * buffers (0, 1) when (c + 1) * refine_every/fuse is even, else (2, 3), and the
 * refinement has written x + e_k to the second buffer for even c, to x for odd c. */
richm_status richm_solve_workspace(const richm_operator* op, const richm_solve_opts* opts, size_t* bytes);

/* Solve every instance of a Q1 batch to tolerance ("iterate until a tolerance or the
 * maximum number of iterations", Sec. 2.3) with FP64 iterative refinement around the
 * inner sweeps: every refine_every sweeps, x += e (FP64), r = b - A x (FP64), the
 * inner right-hand side becomes r, e restarts at 0 and the inner velocity and weight
 * index carry over (so the split is the same iteration in exact arithmetic).
 * b: padded FP64 right-hand side; x: padded FP64, in = initial guess, out = solution.
 * w / alpha / alpha_t: [batch][m] in the real type of opts->inner (alpha, alpha_t as in
 * richm_apply_sweeps). info: host [batch]. Synchronises `stream` before returning.
 * Returns RICHM_OK if every instance converged, else RICHM_ERR_DIVERGED if any
 * diverged, else RICHM_ERR_NOT_CONVERGED. The operator keeps the call's session (the
 * richm_solver below: its stream, events, pinned words and captured cycle graphs) for
 * the next richm_solve or richm_solve_host with the same options, the same weight and
 * workspace pointers and the same tuned fused settings, so repeated solves skip that
 * setup; it is released with the operator or replaced by the next call that differs.
 * One-call solves on one operator must therefore not run from several host threads
 * at once. */
richm_status richm_solve(richm_operator* op, const double* b, double* x, const void* w, const void* alpha,
                         const void* alpha_t, const richm_solve_opts* opts, richm_solve_info* info,
                         void* work, size_t work_bytes, void* stream);

/* Session form of richm_solve for callers that drive the refinement cycles
 * themselves (progress reporting, fixed-cycle timing, resuming). The handle keeps
 * pointers to the caller's weights and workspace (which must stay valid until
 * richm_solver_destroy) and owns a CUDA stream, two events, pinned host words for the
 * active count and flags and, once steps have run with use_graph, the instantiated
 * graphs of a cycle. richm_solver_start binds b and x, zeroes the inner state and
 * evaluates the initial residual; richm_solver_step runs `cycles` refinement cycles
 * (each: refine_every sweeps, the FP64 update, the FP64 residual and the per-instance
 * test) ordered after the work already queued on `stream`, and, when active_out is
 * not NULL, waits and returns the number of instances still iterating;
 * richm_solver_finish waits for `stream`, fills info (host [batch]) and leaves the
 * current FP64 iterate of every instance in x. Between steps, fused cycles may hold the
 * newest iterate of an instance in the workspace's second FP64 buffer: call
 * richm_solver_finish (it may be called between steps as well) before reading x.
 * Without fused cycles x is current after every step. Instances that converged, diverged or
 * reached max_sweeps are skipped by later cycles. With fused sweeps, the start and
 * every step that reports active_out pick the fused tile height for the instances
 * still iterating (the operator's tuned height halved down to 16 rows, whichever a model of
 * the pass's waves of blocks over the SMs estimates fastest); the arithmetic per
 * unknown does not depend on the tile height. */
typedef struct richm_solver richm_solver;
richm_status richm_solver_create(richm_operator* op, const richm_solve_opts* opts, const void* w, const void* alpha,
                                 const void* alpha_t, void* work, size_t work_bytes, richm_solver** out);
richm_status richm_solver_start(richm_solver* s, const double* b, double* x, void* stream);
/* As richm_solver_start with the initial guess x = 0 (written by the call): the
 * initial residual is b, so no stencil is applied. */
richm_status richm_solver_start_zero(richm_solver* s, const double* b, double* x, void* stream);
richm_status richm_solver_step(richm_solver* s, int cycles, int* active_out, void* stream);
richm_status richm_solver_finish(richm_solver* s, richm_solve_info* info, void* stream);
void richm_solver_destroy(richm_solver* s);

/* Checkpoint and resume of a solver session between steps (no counterpart in the
 * paper; the solve of eq. 15's iteration to tolerance run in several processes).
 * richm_solver_state_bytes gives the size of the session's image; richm_solver_save
 * waits for `stream` and the session's own stream and copies the image into `host`
 * (bytes at least that size; pageable or pinned host memory, owned by the caller): a
 * 128-byte header (magic "RICHMSV1", version 1, batch, elems, opts->inner, the resolved
 * fuse, m, refine_every, precond, tol, max_sweeps, the cycle count, an FNV-1a hash of
 * every instance's kind, sizes and stencil, an FNV-1a hash of the weights' bytes), then
 * the current x (FP64, padded), the second FP64 buffer (inner RICHM_F32 / RICHM_BF16),
 * the four inner-state buffers, the inner right-hand side and the per-instance norms,
 * sweep counts, statuses and active flags. The caller may write it to a file.
 * richm_solver_resume binds b and x like richm_solver_start and restores the image into
 * a session created (in this process or another) for the same instances, options and
 * weights; it returns RICHM_ERR_ARG, restoring nothing, if the header does not match.
 * richm_solver_step then continues with the saved cycle count, and the cycles give the
 * same bits as in the uninterrupted session. Both calls are synchronous and must not run
 * during stream capture. Errors: RICHM_ERR_ARG (null, not started, mismatch),
 * RICHM_ERR_NOMEM (host buffer too small), RICHM_ERR_CUDA. */
richm_status richm_solver_state_bytes(const richm_solver* s, size_t* bytes);
richm_status richm_solver_save(richm_solver* s, void* host, size_t bytes, void* stream);
richm_status richm_solver_resume(richm_solver* s, const double* b, double* x, const void* host, size_t bytes,
                                 void* stream);

/* richm_solve from host memory, from the initial guess 0: copies b_host (dense,
 * instances concatenated, n_b*n_b row-major, FP64; pinned memory makes the copy
 * asynchronous and fast) to the device, packs it, solves as richm_solve, unpacks the
 * solution and copies it to x_host (same dense layout), then synchronises `stream`.
 * w / alpha / alpha_t are device arrays as in richm_solve. work: at least
 * richm_solve_host_workspace bytes (the solve workspace, two padded FP64 buffers and a
 * dense staging buffer). Returns as richm_solve. */
richm_status richm_solve_host_workspace(const richm_operator* op, const richm_solve_opts* opts, size_t* bytes);
richm_status richm_solve_host(richm_operator* op, const double* b_host, double* x_host, const void* w,
                              const void* alpha, const void* alpha_t, const richm_solve_opts* opts,
                              richm_solve_info* info, void* work, size_t work_bytes, void* stream);

/* One FP64 refinement step of a mixed-precision iteration on a Q1 batch:
 *   x += e;  e_prev -= e (if e_prev is not NULL);  e = 0;  rhs_out = b - A x,
 * with x, b FP64 padded buffers, e, e_prev and rhs_out padded buffers of the
 * inner dtype (RICHM_F32 or RICHM_F64); e may be NULL (no update, residual only).
 * rel: device [batch] relative residual ||b - A x|| / ||b|| (FP64), or NULL.
 * work: at least richm_residual_workspace bytes. */
richm_status richm_refine(richm_operator* op, double* x, const double* b, void* e, void* e_prev, int inner,
                          void* rhs_out, double* rel, void* work, size_t work_bytes, void* stream);

/* ------------------------------------------------------------------ Krylov outer solver */

/* Restarted flexible GMRES with the Table 1 sweeps as its preconditioner (Sec. 3.2: the
 * single-level solvers as smoothers of a preconditioner for FGMRES restarted every 20
 * iterations, Table 9; FGMRES after Saad, SIAM J. Sci. Comput. 14 (1993) 461-469). */
typedef struct {
  int restart;    /* Arnoldi steps per cycle, 1..64 (the paper's 20) */
  double tol;     /* an instance stops once its residual estimate reaches tol * ||b|| */
  int max_iters;  /* Arnoldi steps per instance at most */
  int m;          /* period of the smoother's coefficients ([batch][m] arrays) */
  int sweeps;     /* smoother sweeps per preconditioner application (0: no preconditioner) */
  int inner;      /* the smoother's state: RICHM_C64 (mixed precision) or RICHM_C128 */
  int precond;    /* the smoother's B^{-1}: 0 none, 1 Jacobi (D^{-1}) */
  int basis;      /* the Arnoldi basis: 0 or RICHM_C128 (complex128), or RICHM_C64 (with inner
                     RICHM_C64: the cycle's vectors, products and Gram-Schmidt passes in
                     complex64, dots and norms summed over tiles in FP64; every cycle
                     still starts from b - A x in FP64) */
} richm_fgmres_opts;

typedef struct {
  int iters;       /* Arnoldi steps taken (the iteration count of Table 9) */
  double rel_res;  /* final ||b - A x|| / ||b|| (FP64, recomputed) */
  int status;      /* RICHM_OK, RICHM_ERR_NOT_CONVERGED or RICHM_ERR_DIVERGED */
} richm_fgmres_info;

/* Workspace bytes of richm_fgmres: restart + 1 basis vectors (opts->basis), restart
 * preconditioned vectors of the inner type, the smoother's state and workspace, and the
 * per-instance Hessenberg systems. */
richm_status richm_fgmres_workspace(const richm_operator* op, const richm_fgmres_opts* opts, size_t* bytes);

/* Solve A x = b for every (Helmholtz) instance of the batch: each cycle starts from
 * r = b - A x, builds an orthonormal basis v_1..v_j of complex128 vectors with
 * z_i = M(v_i), A z_i = sum_k h_ki v_k (classical Gram-Schmidt applied twice), reduces
 * the Hessenberg system by complex Givens rotations, stops an instance once the
 * least-squares residual reaches tol * ||b||, and updates x += sum_i y_i z_i. M(v) is
 * opts->sweeps sweeps of the Table 1 iteration on A z = v from z = 0 (coefficients w,
 * alpha, alpha_t as in richm_apply_sweeps, in the real type of opts->inner), run in
 * opts->inner precision; the z_i are kept in that type. b, x: padded complex128
 * buffers (x: initial guess in, solution out). info: host [batch]. Synchronises
 * `stream` (the host reads the number of instances still iterating after every step).
 * Returns RICHM_OK if every instance converged, else RICHM_ERR_DIVERGED if any
 * diverged, else RICHM_ERR_NOT_CONVERGED; RICHM_ERR_UNSUPPORTED for Q1 instances. */
richm_status richm_fgmres(richm_operator* op, const void* b, void* x, const void* w, const void* alpha,
                          const void* alpha_t, const richm_fgmres_opts* opts, richm_fgmres_info* info, void* work,
                          size_t work_bytes, void* stream);

/* ------------------------------------------------------------------ differentiation */

/* Checkpoint store for K unrolled sweeps with a checkpoint every s sweeps:
 * (K/s + 1) slots of two padded buffers (x_k, x_{k-1}) for k = 0, s, 2s, ...; slot j
 * starts at element 2*j*elems. Returns the element count (x dtype). */
richm_status richm_checkpoint_elems(const richm_operator* op, int K, int ckpt_every, size_t* elems);

/* Forward K sweeps from x0 with zero initial velocity (x_{-1} = x0), storing the
 * checkpoints; xK receives x_K (padded). dtype: RICHM_F32 / RICHM_F64 (Q1) or
 * RICHM_C64 / RICHM_C128 (Helmholtz, precond 0 only; the weights in the real type).
 * Same coefficient conventions as richm_apply_sweeps: precond 0 none, 1 Jacobi, 2 SSOR with relaxation factor relax
 * in (0, 2) (ignored otherwise). Requires K % ckpt_every == 0. work: at least
 * richm_adjoint_workspace bytes (four padded buffers suffice). Only the interior rows
 * (and their padding columns) of the slots after slot 0 are written, and xK is a copy
 * of the last slot: pass a zeroed store for xK to be a padded buffer with zero halos. */
richm_status richm_forward_checkpointed(richm_operator* op, richm_dtype dtype, const void* x0, const void* b,
                                        const void* w, const void* alpha, const void* alpha_t, int m, int K,
                                        int ckpt_every, int precond, double relax, void* ckpts, void* xK,
                                        void* work, size_t work_bytes, void* stream);

/* Workspace bytes for richm_loss_log_residual and richm_sweeps_adjoint. */
richm_status richm_adjoint_workspace(const richm_operator* op, richm_dtype dtype, int ckpt_every, size_t* bytes);

/* Training loss (the log form of eq. 15, the L2 loss of Algorithm 1):
 *   L = (1/B) sum_b ln(||b_b - A_b x_b|| / ||b_b||),
 * and its gradient g = dL/dx = -(1/B) A^H r / ||r||^2, r = b - A x (A^H = A for Q1; for
 * the complex Helmholtz dtypes g = dL/dRe x + i dL/dIm x and A^H = conj(A), the 5-point
 * matrix being complex symmetric). loss: device scalar (FP64); g: padded buffer (dtype
 * of x) or NULL. */
richm_status richm_loss_log_residual(richm_operator* op, richm_dtype dtype, const void* x, const void* b,
                                     double* loss, void* g, void* work, size_t work_bytes, void* stream);

/* Reverse-mode sweep ("backpropagate", Algorithm 1) over the K sweeps recorded by
 * richm_forward_checkpointed (same precond and relax), with A and B^{-1} symmetric so
 * the adjoint applies the same stencil and preconditioner. Complex (Helmholtz) dtypes
 * (precond 0, real weights) use A^H = conj(A) in place of A for q and the real parts
 * of the complex inner products <u, v> = sum conj(u) v; lam and the gradients with
 * respect to x0 are dL/dRe + i dL/dIm. For k = K-1 .. 0
 * (i = k mod m), with lam_{k+1} = dL/dx_{k+1}, u = B^{-1} lam_{k+1} (for SSOR one
 * forward and one backward triangular solve per step) and q = w_i A u,
 *   dL/dw_i   += <lam_{k+1}, B^{-1}(b - A y_k)> = <u, b - A y_k>
 *   dL/da_i   += <lam_{k+1}, x_k - x_{k-1}>
 *   dL/dat_i  += -<q, x_k - x_{k-1}>
 *   lam_k      = (1 + a_i) lam_{k+1} - (1 + at_i) q + c_{k+1},  c_k = -a_i lam_{k+1} + at_i q,
 * and dL/dx0 = lam_0 + c_0 (x_{-1} = x0). Segments between checkpoints are recomputed.
 * gK: dL/dx_K (padded). g_w, g_alpha, g_alpha_t: device [batch][m] (real type), each
 * may be NULL; when alpha_t is NULL (NAG, at = a) the at-gradient is added into
 * g_alpha. g_x0: padded or NULL. Gradients are written, not accumulated. */
richm_status richm_sweeps_adjoint(richm_operator* op, richm_dtype dtype, const void* ckpts, int ckpt_every,
                                  const void* b, const void* gK, const void* w, const void* alpha,
                                  const void* alpha_t, int m, int K, int precond, double relax, void* g_w,
                                  void* g_alpha, void* g_alpha_t, void* g_x0, void* work, size_t work_bytes,
                                  void* stream);

/* ------------------------------------------------------------------ meta network */

/* Meta(theta; mu) of Sec. 2.3: an MLP 2 -> 64 -> 64 -> nout with ReLU, FP32, nout the
 * head's output count (richm_meta_head, at most 64), parameters packed as W1[64][2],
 * b1[64], W2[64][64], b2[64], W3[nout][64], b3[nout] (W[out][in]);
 * richm_meta_param_count gives the total (5457 for m = 16 and the shared-momentum head).
 * Output map: w_i = exp(o_i) / G_b (i < m); the shared head writes a = sigmoid(o_m) to
 * every alpha_out[b][i]; the per-step heads write alpha_out[b][i] = sigmoid(o_{m+i}); the
 * NAGex head writes alpha_t_out[b][i] = sigmoid(o_{2m+i}); the MOM head writes zeros to
 * alpha_t_out if it is not NULL (the sweeps' at = 0). inputs: [B][2] = (log10 eps,
 * theta). G: [B] spectral scales (the Gershgorin bounds, or 1 for an SSOR-preconditioned
 * spectrum). acts: [B][2*64 + nout] saved pre-activations for the backward pass, or
 * NULL. alpha_out may be NULL for the Richardson head, alpha_t_out for every head but
 * NAGex. All arrays device, FP32. Errors: RICHM_ERR_ARG for an unknown head, m < 1 or
 * more than 64 outputs, or a null array the head needs. */
richm_status richm_meta_param_count(int m, int head, int* count);
richm_status richm_meta_forward(const float* params, const float* inputs, const float* G, int B, int m, int head,
                                float* w_out, float* alpha_out, float* alpha_t_out, float* acts, void* stream);

/* Backward of richm_meta_forward given dL/dw, dL/dalpha and (NAGex head) dL/dalpha_t,
 * each [B][m] (dL/dalpha summed over the steps for the shared momentum; g_alpha may be
 * NULL for the Richardson head, g_alpha_t for every head but NAGex). g_params: [count],
 * written (batch sum, fixed order). work: at least B * count floats. */
richm_status richm_meta_backward(const float* params, const float* inputs, const float* G, const float* acts,
                                 int B, int m, int head, const float* g_w, const float* g_alpha,
                                 const float* g_alpha_t, float* g_params, void* work, size_t work_bytes,
                                 void* stream);

/* One Adam step (Kingma & Ba 2015) over `count` parameters in place; t is 1-based. */
richm_status richm_adam_step(float* params, const float* grads, float* m1, float* m2, int count, int t,
                             float lr, float beta1, float beta2, float eps, void* stream);

/* ------------------------------------------------------------------ two-level step */

/* Workspace bytes for richm_fourier_correction: the real residual, its half spectrum
 * (n x (n/2 + 1) per instance) and the cuFFT work area. */
richm_status richm_fourier_workspace(const richm_operator* op, size_t* bytes);

/* Fourier-domain correction of the FNS iteration (eqs. 19-20 with T = I):
 *   x += Re( IFFT2( S .* FFT2(b - A x) ) ),
 * forward transform unnormalised, inverse scaled by 1/n^2 (computed with real-to-complex
 * and complex-to-real transforms and the symmetrised symbol (S(k) + conj S(-k)) / 2,
 * which gives the same real part). Every instance of the
 * operator must be Q1 with the same n. dtype RICHM_F32. symbol: device complex64
 * [n][n] shared by the batch. x, b: padded. */
richm_status richm_fourier_correction(richm_operator* op, richm_dtype dtype, void* x, const void* b,
                                      const void* symbol, void* work, size_t work_bytes, void* stream);

/* Workspace bytes for richm_fourier_correction_vjp: two real n x n fields and two half
 * spectra per instance, and the cuFFT work area. */
richm_status richm_fourier_vjp_workspace(const richm_operator* op, size_t* bytes);

/* Reverse mode of richm_fourier_correction, for learning the symbol of the FNS neural
 * iteration (Sec. 3.1, eq. 20 with T = I; the Meta-Lambda step of Algorithm 2). With
 * x, b the forward call's inputs (x before the correction), g = dL/dx' for its output
 * x' = x + Re(IFFT2(S .* FFT2(b - A x))), R and G the spectra of b - A x and of g:
 *   dsymbol[k] = sum over the batch of conj(R(k)) G(k) / n^2
 *              = dL/dRe S(k) + i dL/dIm S(k)   (complex64 [n][n], written), or NULL;
 *   g_x = g - A Re(IFFT2(conj(S) .* G)) = dL/dx   (padded, may alias g), or NULL.
 * x and b may be NULL when dsymbol is. Same instance rules as the forward call; dtype
 * RICHM_F32 (FP32 transforms and arithmetic). work: at least richm_fourier_vjp_workspace
 * bytes. Errors: RICHM_ERR_ARG for a null g, symbol or work, or a symbol gradient
 * without x and b; RICHM_ERR_NOMEM for a short workspace. */
richm_status richm_fourier_correction_vjp(richm_operator* op, richm_dtype dtype, const void* x, const void* b,
                                          const void* g, const void* symbol, void* dsymbol, void* g_x, void* work,
                                          size_t work_bytes, void* stream);

/* The FNS correction with a transition (Sec. 3.1, eq. 20, H = F T Lambda T^* F^{-1}): T
 * mixes every frequency with its neighbours in a band by one kernel tau, which is the
 * same as multiplying by the field t(x) = sum_d tau_d exp(2 pi i d.x / n) on the grid; the
 * library takes t directly, real (tau Hermitian-symmetric), [n][n] FP32 device, shared
 * by the batch:
 *   x += t .* Re(IFFT2(S .* FFT2(t .* (b - A x)))).
 * transition NULL is T = I (richm_fourier_correction). Same instance rules, dtype and
 * workspace as richm_fourier_correction. */
richm_status richm_fourier_correction_t(richm_operator* op, richm_dtype dtype, void* x, const void* b,
                                        const void* symbol, const void* transition, void* work, size_t work_bytes,
                                        void* stream);

/* Workspace bytes for richm_fourier_correction_t_vjp: three real n x n fields and three
 * half spectra per instance, and the cuFFT work area. */
richm_status richm_fourier_t_vjp_workspace(const richm_operator* op, size_t* bytes);

/* Reverse mode of richm_fourier_correction_t (the Meta-Lambda and Meta-T steps of
 * Algorithm 2). With r = b - A x, q = t r, Q = FFT2(q), p = Re(IFFT2(S Q)) (so
 * x' = x + t p), g = dL/dx', G^ = FFT2(t g) and h = Re(IFFT2(conj(S) G^)):
 *   dsymbol     = sum over the batch of conj(Q) G^ / n^2   (complex64 [n][n]) or NULL,
 *   dtransition = sum over the batch of g p + r h           (FP32 [n][n]) or NULL,
 *   g_x         = g - A (t h) = dL/dx                       (padded, may alias g) or NULL.
 * x, b are needed for either parameter gradient; transition NULL is t = 1 (and then
 * dtransition must be NULL). work: at least richm_fourier_t_vjp_workspace bytes. */
richm_status richm_fourier_correction_t_vjp(richm_operator* op, richm_dtype dtype, const void* x, const void* b,
                                            const void* g, const void* symbol, const void* transition,
                                            void* dsymbol, void* dtransition, void* g_x, void* work,
                                            size_t work_bytes, void* stream);

/* Parameter maps of the FNS neural iteration (Sec. 3.1: Meta-Lambda produces the diagonal
 * Lambda approximating the inverses of A's eigenvalues, Meta-T the transition's kernel;
 * their architectures are not given, so the library maps a few network outputs, o,
 * to the symbol and the transition field, and the meta network with the RICHM_HEAD_RAW
 * head produces o).
 * Symbol: p_m = q_m exp(o_m) (m < 5) with q the instance's Q1 stencil (centre,
 * x-neighbour, y-neighbour, corner(+1,+1), corner(+1,-1)), delta = q_5 exp(o_5), and
 *   sigma(k) = p0 + 2 p1 cos t2 + 2 p2 cos t1 + 2 p3 cos(t1 + t2) + 2 p4 cos(t1 - t2),
 *   S(k) = sigma / (sigma^2 + delta^2),  t = 2 pi k / n  (k = (row, column) frequency),
 * the regularised inverse of the periodic symbol (o = 0: the instance's own stencil).
 * q: host double [6]; o: device FP32 [6]; symbol: device complex64 [n][n] (imaginary 0).
 * Transition: tau = device FP32 [9] = (tau_0, then (re, im) of the band offsets (0,1),
 * (1,0), (1,1), (1,-1)) of a Hermitian-symmetric kernel; the field is
 *   t(i, j) = tau_0 + 2 sum_d (re_d cos(2 pi d.x / n) - im_d sin(2 pi d.x / n)),
 * written to transition: device FP32 [n][n] (the input of richm_fourier_correction_t).
 * Reverse modes: d_o[m] = dL/do_m from dsymbol (the complex gradient
 * richm_fourier_correction_t_vjp gives; S is real, so its real part), dtau[q] = dL/dtau_q
 * from dtransition; outputs device FP32, written; summed in FP64 in a fixed order.
 * work: at least richm_fns_map_workspace bytes. Errors: RICHM_ERR_ARG, RICHM_ERR_NOMEM. */
richm_status richm_fns_map_workspace(size_t* bytes);
richm_status richm_symbol_from_stencil(int n, const double* q, const float* o, void* symbol, void* stream);
richm_status richm_symbol_from_stencil_vjp(int n, const double* q, const float* o, const void* dsymbol, float* d_o,
                                           void* work, size_t work_bytes, void* stream);
richm_status richm_transition_from_band(int n, const float* tau, float* transition, void* stream);
richm_status richm_transition_from_band_vjp(int n, const float* dtransition, float* dtau, void* work,
                                            size_t work_bytes, void* stream);

/* ------------------------------------------------------------------ misc */

/* FMA throughput microbenchmark for the arithmetic ceilings of the roofline (no
 * counterpart in the paper): kind 0 = FP32 FMA, 1 = packed FP32 pairs (two FMAs per
 * instruction), 2 = FP64 FMA. Eight independent multiply-add chains in every thread of
 * 8 blocks of 256 threads per SM, one warm-up and five timed launches on the legacy
 * default stream of the current device (synchronous); *tflops = 2 flops per FMA over
 * the timed launches. Allocates and frees a small output buffer. Errors: RICHM_ERR_ARG
 * for another kind or a null output, RICHM_ERR_CUDA for a failed launch. */
richm_status richm_fma_peak(int kind, double* tflops);

/* Self-test of the library's own FP32 <-> FP64 conversions (no counterpart in the
 * paper: GB300 runs conversions to and from FP64 on its reduced-rate FP64 pipe, so
 * the refinement residual and update move the IEEE 754 fields with integer
 * operations instead). Compares them bit for bit with the hardware conversions:
 * widening on all 2^32 binary32 inputs, round-to-nearest-even narrowing on every
 * binary64 high word (sign, exponent, top 20 fraction bits) combined with eight low
 * words at and around the rounding boundary (2^35 inputs). Writes the mismatch
 * counts (widening, narrowing; 0 and 0 when correct) to host mismatches[2].
 * Allocates 16 bytes of device memory, runs on the legacy default stream of the
 * current device and blocks until done (tens of milliseconds on a GB300). */
richm_status richm_selftest_conversions(long long* mismatches);

/* Thread-local description of the last error ("" if none). */
const char* richm_last_error(void);

/* Library version string. */
const char* richm_version(void);

#ifdef __cplusplus
}
#endif

#endif /* RICHM_H */
