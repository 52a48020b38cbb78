/*
 * Oracle for the Monte Carlo assembly of the PDDSparse interfacial system
 * G(w) u = b(w)  (Bernal, Moron-Vidal & Acebron, "A hybrid probabilistic domain
 * decomposition algorithm suited for very large-scale elliptic PDEs",
 * arXiv 2301.05780).
 *
 * TEST INFRASTRUCTURE ONLY.  This is a plain, slow, obviously-correct FP64 CPU
 * restatement of the estimator of Sec. 3.2 (Eq. 8-9, 19-25), the naive
 * Euler-Maruyama integrator of Sec. 2.3, the extended-stencil exit rule of
 * Sec. 3.3 (Fig. 3), the control variate of Eq. 11 / Eq. 37-39 and the linear
 * solve of Eq. 23.  It exists to check the CUDA library against.  Only the
 * test suite, the smoke check and the CPU-baseline leg of the benchmark may
 * load it.  It shares no code, header, table or helper with the CUDA library;
 * only the seeded input generators (workload module) feed both.
 *
 * Parity status per function (what pins it is in the test suite):
 *   orc_philox4x32_10      pinned: avalanche + uniformity + normal moments/KS
 *   orc_geometry           pinned: knot-count closed form, n = 11277 of Sec. 5.1,
 *                                  stencil rules i)-iii) of Eq. 17
 *   orc_assemble           pinned: G.1 = b invariant (c=f=0, g=1), rectangle
 *                                  exit-time and harmonic-measure series (Eq. 26),
 *                                  Lambda^2 scaling, whole-domain patch = plain
 *                                  Feynman-Kac (Eq. 8) on manufactured solutions,
 *                                  drift-only deterministic exit, sqrt(h) bias
 *   orc_assemble_ex (GM)   pinned: G.1 = b invariant, rectangle exit-time
 *                                  series (bias O(h) against O(sqrt h) for EM),
 *                                  harmonic measure of an off-centre point
 *   orc_calibrate          pinned: EM / GM means equal the rows of the EM / GM
 *                                  systems applied to u0, constant data give
 *                                  zero variance, v = 0 gives rho = 0
 *   orc_plan               pinned: Eq. 40-41 on hand-worked values
 *   RBF stencils (orc_rbf_*, ORC_INTERP_RBF)
 *                          pinned: cardinal property, a library RBF
 *                                  interpolator on the same points, spectral
 *                                  accuracy on smooth data, the assembled
 *                                  weights against the cardinal functions
 *   POISSON_E1 coefficients pinned: f against a finite-difference Laplacian
 *                                  of g = u of Eq. 43
 *   tabulated control variate (cv_tab)
 *                          pinned: a constant table equals the linear network
 *                                  path for path; a table of grad u collapses
 *                                  the score variance; unbiased
 *   orc_mlp_*              pinned: finite differences, closed-form special cases
 *   orc_lu_solve           pinned: residual and a library dense solve
 *   orc_bicgstab           pinned: agreement with orc_lu_solve and residual
 *   TABLE coefficients     parity unpinned for absolute u (no exact solution);
 *                          pinned only through the G.1 = b invariant (c = 0).
 */
#ifndef PDDS_ORACLE_H
#define PDDS_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Coefficient sets (Eq. 6-7 with A = sigma sigma^T, sigma = s(x) I). */
enum {
  ORC_COEF_LAPLACE_EXPSIN = 0, /* s=sqrt2, d=0, c=0, f=0, g=e^x sin y            */
  ORC_COEF_MANUFACTURED   = 1, /* s=sqrt2, d=(sin2pi y, cos2pi x), c=-(1+x^2),
                                  u=sin(pi x)cos(pi y)+xy, f=Lu, g=u             */
  ORC_COEF_VARSIGMA       = 2, /* s=sqrt2(1+0.3 sin2pi x sin2pi y), d=0, c=-1,
                                  u=e^{x/4}cos(y/2), f=Lu, g=u                   */
  ORC_COEF_TABLE          = 3, /* s, c bilinear in FP32 tables, d=0,
                                  f=params[0], g=params[1]                       */
  ORC_COEF_CONSTANT       = 4, /* s=p0, d=(p1,p2), c=p3, f=p4, g=p5              */
  ORC_COEF_POISSON_E1     = 5  /* Sec. 5.1: Lap u = f (s=sqrt2, d=0, c=0), u of
                                  Eq. 43 on [-100,100]^2, f = Lap u, g = u       */
};

/* Exit schemes (Sec. 2.3). */
enum {
  ORC_SCHEME_EM = 0,           /* naive: first step outside the closed patch     */
  ORC_SCHEME_GM = 1            /* Gobet-Menozzi: sides moved inwards by
                                  ORC_GM_SHIFT |sigma N| sqrt(h)                  */
};
#define ORC_GM_SHIFT 0.5826

/* Interpolation on the patch-side stencils (Eq. 21). */
enum {
  ORC_INTERP_LINEAR = 0,       /* piecewise linear (footnote 8)                   */
  ORC_INTERP_RBF = 1           /* 1-D inverse-multiquadric RBF cardinal functions
                                  over the whole stencil (Sec. 2.1, Eq. 1-5)        */
};
#define ORC_MAX_STENCIL 1024

typedef struct {
  double x0, x1, y0, y1; /* Omega = [x0,x1] x [y0,y1]                              */
  int32_t Hx, Hy;        /* subdomain grid                                          */
  int32_t m;             /* knot intervals per subdomain edge                       */
  int32_t ext;           /* stencil extension (knots) past each segment end         */
} orc_grid;

typedef struct {
  int32_t id;            /* ORC_COEF_*                                              */
  int32_t tab_nx, tab_ny;/* table nodes (TABLE), spanning Omega                     */
  int32_t pad_;
  double params[8];
  const float* sigma_tab;/* [tab_ny][tab_nx] row-major, host                        */
  const float* c_tab;
  const double* mlp;     /* NULL = plain estimator; else ORC_MLP_NPARAM values      */
  const float* cv_tab;   /* tabulated control variate (Sec. 4.2): grad u0 at the
                            [cv_ny][cv_nx] nodes spanning Omega, (gx, gy) pairs,
                            bilinear in between; used when mlp is NULL           */
  int32_t cv_nx, cv_ny;
} orc_coeffs;

/* One record per simulated path (optional output of orc_assemble). */
typedef struct {
  int32_t steps;         /* K: number of EM steps taken                              */
  int32_t side;          /* exit side 0=E 1=N 2=W 3=S                                */
  int32_t flags;         /* bit0 truncated at k_max, bit1 along-line clamp applied   */
  int32_t col_a, col_b;  /* knot columns receiving w_a, w_b (-1: none / Dirichlet)    */
  int32_t pad_;
  double w_a, w_b;       /* Y_K * interpolation weight (linear; 0 for RBF)           */
  double b_contrib;      /* Z_K + xi_K + Dirichlet terms (goes to b)                 */
  double Y;              /* Y_K = exp(S_K)                                           */
  double s_line;         /* interface exit: lattice coordinate along the side's line */
} orc_record;

/* One path of the mixed GM/EM calibration run (optional output). */
typedef struct {
  int32_t steps_gm, side_gm, flags_gm;
  int32_t steps_em, side_em, flags_em;
  double phi_gm, phi_em;  /* scores with u0 as patch data (xi excluded)         */
  double xi_gm;           /* control-variate integral at the GM exit            */
  double pad_;
} orc_cal_record;
#define ORC_CAL_NMOM 8

/* Run parameters of orc_assemble_ex / orc_calibrate. */
typedef struct {
  const int64_t* n_per_knot;  /* paths per knot (length n) or NULL: n_paths     */
  int64_t n_paths;
  double dt;                  /* reference step                                 */
  const double* h_per_knot;   /* per-knot step h_k (length n) or NULL: dt        */
  int64_t k_max;              /* step cap at dt; knot k stops after
                                 ceil(k_max dt / h_k) steps                     */
  uint64_t seed;
  uint32_t tag_word;
  int32_t scheme;             /* ORC_SCHEME_* (orc_assemble_ex only)            */
  int32_t interp;             /* ORC_INTERP_*                                   */
  int32_t pad_;
  double rbf_c;               /* IMQ shape parameter c (absolute units), RBF only */
} orc_run;

#define ORC_MLP_HIDDEN 64
#define ORC_MLP_NPARAM (64 * 2 + 64 + 64 * 64 + 64 + 64 + 1)

/* ---- RNG ---------------------------------------------------------------- */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
/* Box-Muller pair from two uniform words (FP64). */
void orc_box_muller(uint32_t a, uint32_t b, double* z0, double* z1);

/* ---- geometry (Sec. 3.1) ------------------------------------------------- */
/* Sizes of the unknown-knot system. */
int orc_geometry_size(const orc_grid* g, int64_t* n, int64_t* nnz);
/* Knot coordinates xy[2n] (lexicographic y then x), CSR pattern (columns
 * ascending, diagonal included). */
int orc_geometry(const orc_grid* g, double* xy, int64_t* row_ptr, int32_t* col);

/* ---- estimator (Eq. 24-25) ------------------------------------------------ */
/* Assembles rows `rows[0..nrows)` of G and b.  val[] (length nnz, layout of
 * orc_geometry) and b[] (length n) are written only for those rows.
 * n_per_knot: paths per knot (length n) or NULL to use n_paths for all.
 * records (may be NULL): per path, rows in request order, paths ascending.
 * stats[0] += total steps, stats[1] += truncated paths, stats[2] += clamps. */
int orc_assemble(const orc_grid* g, const orc_coeffs* cf,
                 const int64_t* n_per_knot, int64_t n_paths,
                 double dt, uint64_t seed, uint32_t tag_word, int64_t k_max,
                 const int32_t* rows, int32_t nrows, int32_t threads,
                 double* val, double* b, orc_record* records, int64_t* stats);

/* The same with the exit scheme and per-knot steps of `run`. */
int orc_assemble_ex(const orc_grid* g, const orc_coeffs* cf, const orc_run* run,
                    const int32_t* rows, int32_t nrows, int32_t threads,
                    double* val, double* b, orc_record* records, int64_t* stats);

/* Mixed GM/EM calibration run (Sec. 4.1): moments[r][ORC_CAL_NMOM] of
 * requested row r = [N, sum d, sum d^2, sum phi_GM, sum phi_GM^2, sum xi,
 * sum xi^2, sum phi_GM xi] with d = phi_EM - phi_GM and u0 (length n) as the
 * patch data; records (may be NULL) per path as in orc_assemble. */
int orc_calibrate(const orc_grid* g, const orc_coeffs* cf, const orc_run* run, const double* u0,
                  const int32_t* rows, int32_t nrows, int32_t threads, double* moments,
                  orc_cal_record* records, int64_t* stats);

/* Eq. 40-41: per-knot step h_out[i] and path budget n_out[i] from moments
 * [n][ORC_CAL_NMOM]; diag[3i..3i+2] = mean(phi_EM - phi_GM), var(phi_GM),
 * rho^2(phi_GM, xi) (diag may be NULL). */
void orc_plan(int64_t n, const double* moments, double eps, double h0, double h0p,
              int64_t n_job, double* h_out, int64_t* n_out, double* diag);

/* Cardinal functions H_0..H_{m-1} (Eq. 5) of the IMQ RBF (Eq. 3 read with
 * + c^2) on the stencil 0, 1, ..., m-1 (lattice units) at z; c_lat is the
 * shape parameter in lattice units.  0, or -1 for a bad size or singular Phi. */
int orc_rbf_cardinal(int32_t m, double c_lat, double z, double* H);
/* Spectral condition number of Phi for that stencil (Jacobi eigenvalues). */
double orc_rbf_cond(int32_t m, double c_lat);
/* c_lat at which that condition number equals `cond` (bisection). */
double orc_rbf_shape_for_cond(int32_t m, double cond);

/* Finalize: the raw sums in val/b for the given rows become Eq. 24-25 entries. */
void orc_finalize_rows(const orc_grid* g, const int64_t* row_ptr, const int32_t* col,
                       const int64_t* n_per_knot, int64_t n_paths,
                       const int32_t* rows, int32_t nrows, double* val, double* b);

/* ---- coefficients and exact solutions (for tests) ------------------------- */
void orc_coeffs_eval(const orc_grid* g, const orc_coeffs* cf, double x, double y,
                     double* s, double* dx, double* dy, double* c, double* f);
double orc_boundary_g(const orc_coeffs* cf, double x, double y);

/* ---- linear solve (Eq. 23) ----------------------------------------------- */
int orc_lu_solve(int64_t n, const double* A_dense, const double* b, double* x);
int orc_bicgstab(int64_t n, const int64_t* row_ptr, const int32_t* col, const double* val,
                 const double* b, double* x, double rtol, int32_t maxit, int32_t* iters,
                 double* relres);

/* ---- control-variate network v_theta (Eq. 11, 37-39) --------------------- */
double orc_mlp_value(const double* theta, double x, double y);
void   orc_mlp_grad_x(const double* theta, double x, double y, double* gx, double* gy);
/* Mean-squared-error loss over npts points and its gradient w.r.t. theta. */
double orc_mlp_loss_grad(const double* theta, const double* xy, const double* target,
                         int64_t npts, double* grad);
/* One Adam step (Kingma & Ba 2015) on theta with moments m, v at step t >= 1. */
void   orc_adam_step(double* theta, const double* grad, double* m, double* v, int64_t t,
                     int64_t nparam, double lr, double beta1, double beta2, double eps);

#ifdef __cplusplus
}
#endif
#endif
