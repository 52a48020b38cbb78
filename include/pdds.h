/*
 * pdds.h -- C ABI of the GB300 (sm_103a) PDDSparse assembly library.
 *
 * PDDSparse (Bernal, Moron-Vidal & Acebron, arXiv 2301.05780) turns a 2-D
 * linear elliptic Dirichlet problem (Eq. 6) on a domain cut into square
 * subdomains into a sparse "interfacial" system G(w) u = b(w) (Eq. 23) whose
 * unknowns are the solution values at knots on the subdomain interfaces
 * (Sec. 3.1).  Row k of G and b_k are Monte Carlo expectations over
 * Feynman-Kac paths started at knot k and stopped when they leave the knot's
 * patch (Eq. 19-25); this library computes them on one GPU and solves the
 * system.
 *
 * Conventions shared by every entry point:
 *  - Every function returns a pdds_status; no exception crosses the ABI.  On
 *    failure the context's error text (pdds_last_error) says why; failures
 *    before a context exists are described by pdds_last_error(NULL).
 *  - "device" pointers are CUDA device (or managed) memory on the current
 *    device; "host" pointers are ordinary host memory.  Caller-owned buffers
 *    are borrowed for the duration of the call only, unless stated otherwise.
 *  - Work is enqueued on the CUDA stream passed as `cuda_stream`
 *    (a cudaStream_t; NULL = legacy default stream) and is asynchronous with
 *    respect to the host, unless the entry point says it synchronizes.
 *  - Knot order is lexicographic in (y, x) over the interior knots, i.e. the
 *    knots on interior grid lines that are not on the boundary of Omega.  Knots
 *    on the boundary are not unknowns: their known values g enter b.
 *  - CSR matrices use int32 row pointers / column indices, columns ascending
 *    within a row, the diagonal included.
 */
#ifndef PDDS_H
#define PDDS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  PDDS_OK = 0,
  PDDS_EINVAL = 1,   /* invalid argument (size, pointer, range)                      */
  PDDS_ENOMEM = 2,   /* device or host allocation failed                             */
  PDDS_ECUDA = 3,    /* a CUDA runtime call failed (text in pdds_last_error)         */
  PDDS_ENOCONV = 4,  /* the iterative solve hit maxit before reaching rtol            */
  PDDS_ETIMEOUT = 5, /* a bounded device-side wait gave up (reported by pdds_stats)   */
  PDDS_ETRUNC = 6    /* informational: some paths reached the step cap                */
} pdds_status;

typedef struct pdds_ctx pdds_ctx; /* opaque; owns the device-side problem tables */

/* Domain and its subdomain grid (Sec. 3.1, Eq. 12-18).
 * Omega = [x0,x1] x [y0,y1] is cut into Hx x Hy equal rectangles; every
 * subdomain edge carries m knot intervals.  `ext` knots are added to each
 * patch-side stencil past both segment ends (clipped to the closure of
 * Omega), so that a diagonal overshoot near a patch corner can be projected
 * on the extended stencil instead of onto the corner (Sec. 3.3, Fig. 3). */
typedef struct {
  double x0, x1, y0, y1;
  int32_t Hx, Hy; /* >= 1 each, and Hx >= 2 or Hy >= 2 (otherwise no knots)   */
  int32_t m;      /* >= 1                                                     */
  int32_t ext;    /* >= 0                                                     */
} pdds_grid;

/* Coefficients of Eq. 6 with diffusion sigma(x) = s(x) I (so A = s^2 I).
 * Built-in sets (kind = PDDS_COEF_BUILTIN, builtin_id):                        */
enum {
  PDDS_COEF_LAPLACE_EXPSIN = 0, /* s = sqrt2, d = 0, c = 0, f = 0, g = e^x sin y      */
  PDDS_COEF_MANUFACTURED = 1,   /* s = sqrt2, d = (sin 2pi y, cos 2pi x), c = -(1+x^2),
                                   f = L u for u = sin(pi x)cos(pi y) + x y, g = u      */
  PDDS_COEF_VARSIGMA = 2,       /* s = sqrt2 (1 + 0.3 sin 2pi x sin 2pi y), d = 0, c = -1,
                                   f = L u for u = e^{x/4} cos(y/2), g = u              */
  PDDS_COEF_TABLE = 3,          /* s and c bilinear in FP32 tables, d = 0,
                                   f = params[0], g = params[1] (constants); every c
                                   value <= 0, every s value finite and nonzero      */
  PDDS_COEF_CONSTANT = 4,       /* s = p0 != 0, d = (p1, p2), c = p3 <= 0, f = p4, g = p5 */
  PDDS_COEF_POISSON_E1 = 5      /* Sec. 5.1, Eq. 42-43: Lap u = f on [-100,100]^2, i.e.
                                   s = sqrt2, d = 0, c = 0, f = Lap u and g = u for
                                   u = 3 + sin(r)/3 + tanh(q)/3, r = sqrt(1 + x^2/100
                                   + y^2/50), q = sin(3x/25 + y/20) + sin(x/20 - 3y/25) */
};
enum { PDDS_COEF_BUILTIN = 0 };

typedef struct {
  int32_t kind;         /* PDDS_COEF_BUILTIN                                          */
  int32_t builtin_id;   /* PDDS_COEF_*                                                 */
  const float* sigma_tab; /* TABLE only: host or device, [tab_ny][tab_nx] row-major,    */
  const float* c_tab;     /*   nodes spanning Omega; copied at pdds_create (not kept)   */
  int32_t tab_nx, tab_ny; /* >= 2 each                                                  */
  double params[8];
} pdds_coeffs;

/* CSR matrix in caller-owned DEVICE memory: row_ptr[n+1], col[nnz], val[nnz]. */
typedef struct {
  int64_t n, nnz;
  int32_t* row_ptr;
  int32_t* col;
  double* val;
} pdds_csr;

/* Per-path record written by pdds_assemble_records (40 bytes). */
typedef struct {
  int32_t steps;      /* K, Euler-Maruyama steps taken                                */
  int32_t side_flags; /* exit side (0 E, 1 N, 2 W, 3 S) | flags << 8: bit0 step cap,
                         bit1 along-line clamp                                         */
  int32_t col_a, col_b; /* knots receiving w_a, w_b; -1 = none or boundary point      */
  float w_a, w_b;     /* Y_K times the interpolation weight                           */
  float b_contrib;    /* Z_K + xi_K + boundary terms: the path's share of b_k times N */
  float Y;            /* Y_K = exp(int c dt)                                          */
  float xi;           /* xi_K alone (0 without a control variate)                     */
  float s_line;       /* interface exit: coordinate along the side's grid line, in
                         lattice spacings from the line's start (0 on the boundary of
                         Omega); with RBF stencils col_a = col_b = -1, w_a = w_b = 0 and
                         the weights are H_j(s_line) of the side's stencil           */
} pdds_path_record;

typedef struct {
  int64_t path_steps;       /* sum over paths of K (last assemble call)                */
  int64_t paths;            /* paths completed                                         */
  int64_t truncated;        /* paths that reached the step cap                          */
  int64_t clamped;          /* interface exits clamped to the stencil ends              */
  int64_t units;            /* work units processed                                     */
  int32_t device_error;     /* PDDS_OK, PDDS_ETIMEOUT, or PDDS_EINVAL (an RBF exit found no
                               table for its stencil: nothing deposited; or a per-knot budget
                               outside [0, 2^31): counted as 0) from the last assembly      */
  int32_t solve_iters;      /* iterations of the last pdds_solve                        */
  double solve_relres;      /* ||b - G u|| / ||b|| of the last pdds_solve               */
  float path_kernel_ms;     /* CUDA-event time of the last path kernel (timing on)     */
  int32_t kernel_launches;  /* kernels launched by the last assemble + solve calls      */
  int32_t path_grid;        /* CTAs of the last path kernel                             */
  int32_t path_block;       /* threads per CTA of the last path kernel                  */
} pdds_stats_t;

/* ------------------------------------------------------------------------ */
/* Host-only geometry (no CUDA call): the knot set, patches and stencils of  */
/* Sec. 3.1 (Eq. 13-18).  Pass NULL arrays to query sizes only.  xy_host is  */
/* [n][2]; row_ptr_host [n+1]; col_host [nnz].                                */
pdds_status pdds_geometry_host(const pdds_grid* grid, int64_t* n, int64_t* nnz,
                               double* xy_host, int32_t* row_ptr_host, int32_t* col_host);

/* Builds the problem on the current device: knot table, patch boxes, stencil
 * slots, CSR pattern (Sec. 3.1) and, for PDDS_COEF_TABLE, padded device copies
 * of the coefficient tables with their TMA descriptors.  Synchronizes the
 * device.  Errors: EINVAL (grid/coeffs; also a potential c > 0 anywhere: the
 * paper's setting takes c <= 0, and the path weights Y = exp(int c dt) <= 1
 * are summed as exact 2^-30 fixed point), ENOMEM, ECUDA. */
pdds_status pdds_create(const pdds_grid* grid, const pdds_coeffs* coeffs, pdds_ctx** out);
void pdds_destroy(pdds_ctx* ctx);

pdds_status pdds_num_knots(const pdds_ctx* ctx, int64_t* n, int64_t* nnz);
pdds_status pdds_knot_coords(const pdds_ctx* ctx, double* xy_host /* [n][2] */);

/* Step cap per path (K_max).  Default: 40 x the strip bound on the mean exit
 * time of the largest patch, w^2 / (4 s_min^2) with w = 2 min(Lx, Ly), over dt. */
pdds_status pdds_set_step_cap(pdds_ctx* ctx, int64_t k_max);

/* Launch shape of the path kernel: threads per CTA (multiple of 32, <= 1024),
 * CTAs per SM (0 = occupancy maximum), paths per work unit (>= 32) and the
 * number of exited lanes a warp gathers before resolving exits (1..32).
 * Zeros keep the current value.  pdds_autotune picks them by measurement. */
pdds_status pdds_set_launch(pdds_ctx* ctx, int32_t block, int32_t ctas_per_sm,
                            int32_t unit_paths, int32_t exit_batch);
pdds_status pdds_get_launch(const pdds_ctx* ctx, int32_t* block, int32_t* ctas_per_sm,
                            int32_t* unit_paths, int32_t* exit_batch);
/* Autotuner: times short assemblies of a sample of the knots (every k-th,
 * k >= 8 chosen so that the sample has at most 2e8 paths, each at the full
 * per-knot budget n_paths, time step dt) for every combination of block in
 * {64, 128, 256, 512}, unit_paths in {256, 1024, 4096, 16384} and exit_batch in
 * {2, 4, 8, 16}; the twelve fastest are timed again; the three fastest of those
 * are timed twice on the whole problem (on every k2-th knot when it has more
 * than 1e9 paths) and the fastest is kept.  The launch shape
 * only reorders floating-point additions, never the estimator.  Results are
 * cached for the process per (device, coefficient set, control variate on/off,
 * grid, n_paths); a cached shape is applied without timing.  Allocates and
 * frees its own scratch and synchronizes the device. */
pdds_status pdds_autotune(pdds_ctx* ctx, int64_t n_paths, double dt, uint64_t seed,
                          void* cuda_stream);

/* Philox tag of the single-problem calls on ctx (pdds_assemble,
 * pdds_assemble_records, pdds_assemble_solve_host, pdds_calibrate,
 * pdds_autotune): the fourth counter word of every path's stream, (q, p, k,
 * tag).  Default 0.  pdds_assemble_batch gives problem i the tag i whatever
 * this setting, so a single-problem call with tag i on the context of problem
 * i draws the same Gaussians as that problem does in a batch (used to check a
 * batch row by row with per-path records).  Applies to later calls. */
pdds_status pdds_set_philox_tag(pdds_ctx* ctx, uint32_t tag);

/* Bound, in seconds, on every device-side wait of the path kernel (a warp
 * waiting for the next work unit of its CTA, or for the TMA copy of a
 * tabulated-coefficient tile).  When a wait runs out the kernel stops taking
 * work, returns, and pdds_stats reports PDDS_ETIMEOUT; the results of that
 * call (G, b, records, counters) are then incomplete and must be discarded.
 * What a timeout leaves behind: nothing on the device beyond those partial
 * results (no memory, no pending work); a tile copy that had not landed when
 * its wait ran out is given a further max(limit, 1 s) to land before its CTA
 * returns, so that no copy is left writing into released shared memory.
 * The context stays usable.  0 restores the default: 10 s plus 4 us per step
 * of the step cap (40 us per step with the in-path network). */
pdds_status pdds_set_wait_limit(pdds_ctx* ctx, double seconds);

/* When on, the path kernel is bracketed by CUDA events on the caller's stream
 * (pdds_assemble_batch: the whole batched graph).  The assembly does not wait
 * for them; pdds_stats, which synchronizes, reports the duration of the last
 * timed assembly in path_kernel_ms. */
pdds_status pdds_set_timing(pdds_ctx* ctx, int32_t on);

/* Monte Carlo assembly of G and b (Eq. 24-25), the hot path.
 * For every knot k, N_k paths of dX = d dt + s dW (naive Euler-Maruyama, Sec.
 * 2.3) carry Y = exp(int c dt) and Z = -int f Y dt (Eq. 9) until they leave the
 * closed patch (Eq. 15); an exit on the boundary of Omega adds g Y to b_k, an
 * exit on an interface interpolates linearly between the two nearest stencil
 * knots of the side crossed (Eq. 21-22 with a linear scheme; boundary points of
 * the stencil add their known g).  Then G_kk = 1, G_kj = -sum/N_k, b_k = sum/N_k.
 *   n_per_knot: DEVICE int64[n] budgets, or NULL to use n_paths for every knot
 *   n_paths   : >= 1 when n_per_knot is NULL; every N_k must be in [0, 2^31) (a
 *               knot with N_k = 0 keeps row e_k and b_k = 0; the device counts
 *               any other value as 0 and records PDDS_EINVAL for pdds_stats)
 *   dt        : time step h > 0
 *   seed      : 64-bit Philox4x32-10 key; the normal pair for step 2q and 2q+1 of
 *               path p from knot k comes from counter (q, p, k, tag)
 *   G         : caller-owned device CSR sized by pdds_num_knots; row_ptr, col and
 *               val are all written
 *   b         : device double[n]
 * Asynchronous (unless timing is on).  Device-side errors surface in pdds_stats. */
pdds_status pdds_assemble(pdds_ctx* ctx, const int64_t* n_per_knot, int64_t n_paths,
                          double dt, uint64_t seed, pdds_csr* G, double* b, void* cuda_stream);

/* Same as pdds_assemble, plus one pdds_path_record per path written to the
 * DEVICE array `records`, laid out knot by knot (knot-major, then path index);
 * it must hold sum_k N_k records (a budget outside [0, 2^31) counts as 0
 * there too). */
pdds_status pdds_assemble_records(pdds_ctx* ctx, const int64_t* n_per_knot, int64_t n_paths,
                                  double dt, uint64_t seed, pdds_csr* G, double* b,
                                  pdds_path_record* records, void* cuda_stream);

/* Interpolation on the patch-side stencils (Eq. 21):
 *  PDDS_INTERP_LINEAR  piecewise linear between the two nearest stencil knots
 *                      (footnote 8; the default);
 *  PDDS_INTERP_RBF     1-D inverse-multiquadric RBF interpolation over the whole
 *                      stencil (Sec. 2.1, Eq. 1-5, phi_c(r) = 1/sqrt(r^2 + c^2)):
 *                      an exit at z gives every stencil knot j the weight Y H_j(z),
 *                      H_j the cardinal functions (Eq. 5).  The library tabulates
 *                      the H_j of every stencil length as per-interval Chebyshev
 *                      series (FP64 construction, FP32 coefficients, truncation error
 *                      below 2e-7 max|H|) and evaluates them at each exit.
 * rbf_shape: c in the units of Omega; <= 0 picks the c at which the spectral
 * condition number of the longest stencil's matrix Phi is 1e10 (the choice of
 * Sec. 5.1).  shape_used / table_err (nullable, host): the c in use and the
 * tables' truncation bound.  Applies to later assemble / calibrate calls on ctx
 * (not to batches); synchronizes.  Errors: EINVAL (kind, or Phi not positive
 * definite in FP64 for a too-large c), ENOMEM, ECUDA. */
enum { PDDS_INTERP_LINEAR = 0, PDDS_INTERP_RBF = 1 };
pdds_status pdds_set_interpolation(pdds_ctx* ctx, int32_t kind, double rbf_shape,
                                   double* shape_used, double* table_err);

/* Exit scheme of the path kernel (Sec. 2.3):
 *  PDDS_SCHEME_EM  naive Euler-Maruyama: exit at the first step outside the
 *                  closed patch (weak order 1/2; the default);
 *  PDDS_SCHEME_GM  Gobet-Menozzi: every patch side is moved inwards by
 *                  0.5826 |s(P)| sqrt(h), P the normal projection of the
 *                  current point on that side, and the path exits at the first
 *                  step beyond a moved side (weak order 1).  The exit side is the
 *                  one of smallest positive overshoot past its moved line; the
 *                  exit point is the normal projection on the true side.
 * Applies to every later assemble / calibrate call on ctx (not to batches). */
enum { PDDS_SCHEME_EM = 0, PDDS_SCHEME_GM = 1 };
pdds_status pdds_set_scheme(pdds_ctx* ctx, int32_t scheme);

/* Per-knot time steps h_k (Sec. 4.2, Eq. 40).  h_per_knot: DEVICE double[n],
 * every h_k > 0 and finite, copied into the context (synchronizes; the caller
 * may free it afterwards); NULL returns to the single dt of each call.  While
 * set, knot k steps with h_k and the dt argument of assemble / calibrate only
 * fixes the time horizon of the step cap: knot k stops after
 * ceil(k_max dt / h_k) steps.  Not used by pdds_assemble_batch. */
pdds_status pdds_set_knot_steps(pdds_ctx* ctx, const double* h_per_knot);

/* Calibration run of Sec. 4.1 (Phase II): N_k "mixed GM/EM" paths per knot
 * with the warm-up nodal solution u0 as the data on the patch boundary.  Every
 * path yields a Gobet-Menozzi score phi_GM (first step beyond a moved side)
 * and a naive score phi_EM (first step outside the patch) from one trajectory
 * (the same Philox counters as pdds_assemble with `seed`), where
 * phi = Y u0(P) + Z, u0(P) being the stencil interpolation of the nodal u0 on
 * an interface side and g on the boundary of Omega; with a control variate
 * attached, xi (Eq. 37, up to the GM exit) is drawn alongside.  Per knot:
 *   moments[k][0..7] = N_k, sum d, sum d^2, sum phi_GM, sum phi_GM^2,
 *                      sum xi, sum xi^2, sum phi_GM xi      (d = phi_EM - phi_GM)
 * in FP64 (DEVICE double[n][8]).  u0: DEVICE double[n]; n_per_knot / n_paths /
 * dt / seed as for pdds_assemble (per-knot steps apply when set).  The scheme
 * setting is ignored.  One launch of the path kernel: each path records its
 * GM exit and steps on to its naive exit, so the run costs the naive paths'
 * steps.  Allocates context-owned record scratch (two 40-byte records per
 * path, kept for reuse) and synchronizes the stream. */
pdds_status pdds_calibrate(pdds_ctx* ctx, const double* u0, const int64_t* n_per_knot,
                           int64_t n_paths, double dt, uint64_t seed, double* moments,
                           void* cuda_stream);

/* Eq. 40-41: per-knot steps and path budgets for accuracy eps from the
 * calibration moments (DEVICE double[n][8], as written by pdds_calibrate):
 *   gap_k = mean d,  V_k = sample variance of phi_GM,  rho_k^2 = corr(phi_GM, xi)^2
 *   h_out[k] = min(h0, 2 h0' eps / (3 |gap_k|))        (h0 when gap_k = 0)
 *   N_out[k] = N_job * max(1, round(9 V_k (1 - rho_k^2) / (eps^2 N_job)))
 * (rounding half to even), capped at the largest multiple of N_job below 2^31
 * so that it is a valid budget (a NaN V_k gives N_job).  h_out: DEVICE
 * double[n]; N_out: DEVICE int64[n]; diag (nullable): DEVICE double[n][3] =
 * gap_k, V_k, rho_k^2.  No context; asynchronous.  EINVAL for n < 1, eps, h0
 * or h0' not > 0, or N_job outside [1, 2^31). */
pdds_status pdds_plan(const double* moments, int64_t n, double eps, double h0, double h0p,
                      int64_t n_job, double* h_out, int64_t* n_out, double* diag,
                      void* cuda_stream);

/* Several independent problems (same coefficient set id) in ONE persistent
 * launch: paths of all problems share one work queue.  Arrays have `count`
 * entries; n_per_knot[i] may be NULL (then n_paths is used).  Problem i uses
 * Philox tag i, so its streams differ from problem 0's.  The sequence is
 * captured once into a CUDA graph per (count, ctxs) and replayed.  Budgets
 * follow pdds_assemble (outside [0, 2^31): no paths, PDDS_EINVAL recorded).
 * The launch's counters, device error and time are those of ctxs[0]: read
 * them with pdds_stats(ctxs[0]). */
pdds_status pdds_assemble_batch(pdds_ctx* const* ctxs, int32_t count,
                                const int64_t* const* n_per_knot, int64_t n_paths, double dt,
                                uint64_t seed, pdds_csr* const* G, double* const* b,
                                void* cuda_stream);

/* FP64 BiCGSTAB for G u = b (Eq. 23), all on the device; u (device double[n])
 * is overwritten (initial guess 0).  Synchronizes the stream to read the
 * residual every few iterations.  Returns ENOCONV if ||b - G u|| > rtol ||b||
 * after maxit iterations; *iters (nullable) gets the iteration count. */
pdds_status pdds_solve(pdds_ctx* ctx, const pdds_csr* G, const double* b, double* u,
                       double rtol, int32_t maxit, int32_t* iters, void* cuda_stream);

/* ------------------------------------------------------------------------ */
/* Learned control variate (Eq. 11, 37-39).  The paper adds to each score the */
/* Ito integral xi = -int Y F . dW with F = sigma^T grad u0, u0 a warm-up     */
/* solution (Sec. 4.2); here u0 is a small network v_theta : R^2 -> R,        */
/* 2 -> 64 -> 64 -> 1 with SiLU, fitted to warm-up nodal values and boundary  */
/* samples.  theta is FP32, PDDS_MLP_NPARAM values: W1[64][2], b1[64],         */
/* W2[64][64] (row = output unit), b2[64], w3[64], b3.                        */
#define PDDS_MLP_NPARAM 4417

/* Mean-squared-error loss (1/N) sum_p (v(x_p) - target_p)^2 and its gradient
 * w.r.t. theta (FP32 forward/backward kernels).  All pointers DEVICE:
 * theta[NPARAM], xy[npts][2], target[npts], grad[NPARAM] (overwritten),
 * loss (one double, overwritten).  Asynchronous. */
pdds_status pdds_mlp_loss_grad(const float* theta, const float* xy, const float* target,
                               int64_t npts, float* grad, double* loss, void* cuda_stream);

/* `steps` full-batch Adam steps (beta1 0.9, beta2 0.999, eps 1e-8, rate lr)
 * on the loss above; theta (DEVICE) is updated in place; loss_history_host
 * (nullable) receives the loss before each step.  Allocates and frees its own
 * scratch (gradient, Adam moments, step state, loss history) and a private
 * stream on which the steps run as a replayed CUDA graph, ordered after the
 * work already queued on cuda_stream; synchronizes.  One kernel launch per
 * step: 64-point tiles on at most two CTAs per SM, FP32 throughout, the
 * CTA partial gradients added with FP32 atomics (the summation order, and so
 * the last bits, vary from run to run).
 * Errors: EINVAL (NULL pointer, npts < 1, steps < 1, lr <= 0), ECUDA. */
pdds_status pdds_mlp_train(float* theta, const float* xy, const float* target, int64_t npts,
                           int32_t steps, double lr, double* loss_history_host,
                           void* cuda_stream);

/* The same loss gradient and training on the fifth-generation tensor cores
 * (the fit of Phase I, Sec. 4.3): tiles of 128 points, one 256-thread CTA
 * per tile at a time (two warpgroups, each half of the hidden units; at most
 * two CTAs per SM: ~107 KB of shared memory and 256 TMEM columns each); the
 * forward product h1 W2^T, the backward product
 * g2 W2 and the weight gradient [g2 | g1]^T [h1 | x | y | 1] (contracted over
 * the tile's points, accumulated in TMEM over the CTA's tiles) run as
 * tcgen05.mma kind::f16 with BF16 operands and FP32 accumulation; the rest
 * is FP32.  The loss and the gradient carry the BF16 rounding of the
 * products' operands (within 1e-2 of the FP64 loss and gradient norm).
 * Arguments, the Adam step, scratch, graph replay and synchronisation as for
 * pdds_mlp_loss_grad / pdds_mlp_train.  A bounded tensor-core wait (2 s) that
 * runs out makes that step's loss NaN (loss, loss_history_host).
 * Errors: EINVAL, ECUDA. */
pdds_status pdds_mlp_loss_grad_tc(const float* theta, const float* xy, const float* target,
                                  int64_t npts, float* grad, double* loss, void* cuda_stream);
pdds_status pdds_mlp_train_tc(float* theta, const float* xy, const float* target, int64_t npts,
                              int32_t steps, double lr, double* loss_history_host,
                              void* cuda_stream);

/* v_theta and grad v_theta at npts DEVICE points with the in-path evaluation
 * (64x64 layer on the tensor cores with BF16 operands and FP32 accumulation;
 * the rest FP32).  v (nullable) [npts], grad_xy [npts][2].  Synchronizes. */
pdds_status pdds_mlp_eval(const float* theta, const float* xy, int64_t npts, float* v,
                          float* grad_xy, void* cuda_stream);

/* Samples of the boundary data g of Eq. 6 on the boundary of Omega, for the
 * fit of v_theta (the warm-up nodal values say nothing about u between the
 * outermost knots and the boundary, where g is known exactly): n_per_side
 * points on each side, E (x = x1), N (y = y1), W (x = x0), S (y = y0) in that
 * order, at the midpoints of n_per_side equal intervals (corners excluded),
 * with g evaluated on the device as the path kernel evaluates it at a
 * boundary exit.  xy: DEVICE float [4 n_per_side][2]; g: DEVICE float
 * [4 n_per_side].  Asynchronous.  EINVAL for n_per_side outside [1, 2^26]. */
pdds_status pdds_boundary_samples(const pdds_ctx* ctx, int32_t n_per_side, float* xy, float* g,
                                  void* cuda_stream);

/* v_theta and grad v_theta at npts DEVICE points on the fifth-generation
 * tensor cores (tcgen05.mma kind::tf32 with TMEM accumulators): tiles of 128
 * points, the two 64 x 64 products (forward h1 W2^T and backward g2 W2 of
 * Eq. 37's grad v) each as three TF32 products of the hi / lo split of both
 * operands (FP32-accurate), the rest FP32.  Used to tabulate grad v_theta for
 * the look-up-table control variate (Sec. 4.2).  theta, xy [npts][2], v
 * (nullable) [npts], grad_xy [npts][2]: DEVICE.  One CTA of two 128-thread
 * warpgroups per SM (~195 KB of shared memory, 256 TMEM columns).
 * Synchronizes the stream.
 * Errors: EINVAL, ECUDA, ETIMEOUT (a bounded tensor-core wait ran out). */
pdds_status pdds_mlp_eval_tc(const float* theta, const float* xy, int64_t npts, float* v,
                             float* grad_xy, void* cuda_stream);

/* Attach v_theta (DEVICE theta, copied and staged) to the context: from then
 * on pdds_assemble adds xi_K = -sum_n Y_n s(X_n) grad v(X_n) . dW_n to every
 * path's b contribution (Eq. 37, left-point Ito sum), which leaves E[b]
 * unchanged and lowers its variance as v approaches u.  NULL detaches it.
 * Available for PDDS_COEF_LAPLACE_EXPSIN, _MANUFACTURED, _CONSTANT and
 * _POISSON_E1 (EINVAL otherwise, nothing changed); a staging error (ECUDA)
 * leaves no control variate attached. */
pdds_status pdds_set_control_variate(pdds_ctx* ctx, const float* theta);

/* Tensor-core engine of the in-path network of Eq. 37 (pdds_set_control_variate;
 * the estimator, the streams and the BF16 rounding points are the same with
 * both, so G and b differ only in the rounding of the network's products):
 *  PDDS_NET_TCGEN05 (default): the paths of a 128-thread warpgroup step
 *    together; at each step the 128 positions form one M = 128 tile, h1 W2^T
 *    and g2 W2 run as tcgen05.mma (kind::f16, BF16 operands, FP32 in TMEM),
 *    SiLU'(a1) waits in TMEM as BF16 pairs.  Launch: 128 threads per CTA
 *    (the block setting of pdds_set_launch does not apply), up to five CTAs
 *    per SM (96 TMEM columns, 96 registers per thread).
 *    Both exits (naive and extended: Gobet-Menozzi, per-knot steps, RBF
 *    stencils, the calibration's mixed run).  Each wait for a product is
 *    bounded by max(wait limit, 1 s) (pdds_set_wait_limit).
 *  PDDS_NET_MMA_SYNC: each warp evaluates its 32 lanes on its own with
 *    mma.sync.m16n8k16 (BF16, FP32 accumulation in registers).
 * Applies to later calls.  EINVAL for another value. */
enum { PDDS_NET_MMA_SYNC = 0, PDDS_NET_TCGEN05 = 1 };
pdds_status pdds_set_network_engine(pdds_ctx* ctx, int32_t engine);

/* Tabulated control variate (Sec. 4.2: F = sigma^T grad u0 stored as an
 * interpolatory look-up table): grad_xy is a DEVICE (or host) float array
 * [ny][nx][2] of (du0/dx, du0/dy) at the nodes of an nx x ny grid spanning
 * Omega (corners included); the context keeps it cell by cell (the four
 * corners of each cell together, 32 bytes, 4x the node table's size).  From
 * then on the path kernel adds xi = -sum_n Y_n s(X_n) g(X_n) . dW_n, g the
 * bilinear interpolation of the table (replaces an attached network; NULL
 * detaches).  Per step it costs one 32-byte cell read instead of the
 * network's two 64 x 64 products.  Available for every coefficient set.
 * Synchronizes (the device).  On an error no control variate is attached.
 * Errors: EINVAL (nx, ny < 2 or nx ny > 2^28), ENOMEM, ECUDA. */
pdds_status pdds_set_control_variate_grid(pdds_ctx* ctx, const float* grad_xy, int32_t nx,
                                          int32_t ny);

/* Allocation-free variant of pdds_solve (the paper has no counterpart; this
 * is a service to callers).  For callers that cannot allocate device memory:
 * applications that own all device memory through their own pool or arena
 * under a fixed budget, where a library-side cudaMalloc would bypass their
 * accounting or fail, and latency-critical code that cannot accept the implicit
 * synchronization of cudaMalloc/cudaFree.  It needs no context and calls no
 * cudaMalloc, cudaFree or allocating library routine: its scratch (six work
 * vectors and the recurrence scalars) is a static device array of
 * 6 * 131072 + 32 doubles (6.3 MB) that every GPU loading this library holds
 * until the process exits.
 *   G, b, u, rtol, maxit, iters, cuda_stream: as for pdds_solve (all device
 *     pointers; u is overwritten, initial guess 0; the stream is synchronized
 *     every few iterations to read the residual).
 *   G->n must be in [1, 131072]; larger systems are rejected with PDDS_EINVAL
 *     before any device work (use pdds_solve).
 * The first call on each device looks up the array's device address with that
 * device current; make that first call before any stream capture.  The address
 * is kept for the life of the process: after a cudaDeviceReset (or any other
 * teardown of the device's primary context) it is stale, so a process that
 * resets a device must not call pdds_solve_noalloc on that device again.  All calls
 * in the process share the one array per device: calls that overlap on the
 * GPU (other host threads or other streams) race and corrupt each other's
 * results -- serialize them.  Each call re-initialises every part of the array
 * it reads, so nothing carries over from the previous call.
 * Errors: EINVAL, ENOCONV, ECUDA; text via pdds_last_error(NULL). */
pdds_status pdds_solve_noalloc(const pdds_csr* G, const double* b, double* u, double rtol,
                               int32_t maxit, int32_t* iters, void* cuda_stream);

/* End-to-end call with HOST buffers: uploads the per-knot budgets, assembles,
 * solves and downloads G (row_ptr, col, val), b and u.  Device scratch is owned
 * by the context.  n_per_knot_host may be NULL; EINVAL (nothing launched) if a
 * budget is outside [0, 2^31).  Synchronizes the stream. */
pdds_status pdds_assemble_solve_host(pdds_ctx* ctx, const int64_t* n_per_knot_host,
                                     int64_t n_paths, double dt, uint64_t seed, double rtol,
                                     int32_t maxit, int32_t* row_ptr_host, int32_t* col_host,
                                     double* val_host, double* b_host, double* u_host,
                                     void* cuda_stream);

/* End-to-end batch with HOST buffers: the `count` problems of
 * pdds_assemble_batch in ONE persistent launch (replayed from its CUDA graph),
 * then each problem's FP64 BiCGSTAB solve (Eq. 23), all on the device.  Per
 * call: the per-knot budgets go up (n_per_knot_host[i]: int64[n_i], or NULL /
 * a NULL array for n_paths everywhere) and G (row_ptr[n_i+1], col[nnz_i],
 * val[nnz_i]), b[n_i] and u[n_i] of every problem come down.  Every array has
 * `count` entries of HOST pointers (pinned memory copies fastest); row_ptr_host
 * and col_host (or their entries) may be NULL to skip the pattern, val, b and
 * u may not.  Device buffers are each context's own scratch (allocated on the
 * first call and kept).  Budgets outside [0, 2^31) are rejected (EINVAL)
 * before any copy or launch.  Restrictions and counters as for
 * pdds_assemble_batch (the launch's counters and time are read with
 * pdds_stats(ctxs[0]); its kernel_launches then counts the batch and all
 * solves).  Returns ENOCONV if some solve did not reach rtol (every result is
 * still copied back).  Synchronizes the stream. */
pdds_status pdds_assemble_solve_batch_host(pdds_ctx* const* ctxs, int32_t count,
                                           const int64_t* const* n_per_knot_host, int64_t n_paths,
                                           double dt, uint64_t seed, double rtol, int32_t maxit,
                                           int32_t* const* row_ptr_host, int32_t* const* col_host,
                                           double* const* val_host, double* const* b_host,
                                           double* const* u_host, void* cuda_stream);

/* Counters of the last assemble / solve (synchronizes the device).  Returns
 * the device error the last assembly recorded (out->device_error: PDDS_ETIMEOUT
 * or PDDS_EINVAL), else PDDS_OK; the counters are filled in either case. */
pdds_status pdds_stats(pdds_ctx* ctx, pdds_stats_t* out);

/* Text of the last error on ctx (or of the last failed pdds_create when ctx is
 * NULL).  Never NULL; valid until the next call on the same context. */
const char* pdds_last_error(const pdds_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* PDDS_H */
