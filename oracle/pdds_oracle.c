/*
 * Oracle for the Monte Carlo assembly of the PDDSparse system G(w) u = b(w)
 * (arXiv 2301.05780).  TEST INFRASTRUCTURE ONLY: see pdds_oracle.h.
 *
 * Everything here is FP64, single-path-at-a-time, in the order the paper states
 * the method.  Threads split the requested rows; within a row, paths are
 * simulated and summed in ascending path index, so results do not depend on
 * the thread count.
 */
#include "pdds_oracle.h"

#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* ========================================================================= *
 * Philox4x32-10 (Salmon, Moraes, Dror & Shaw, "Parallel random numbers: as   *
 * easy as 1, 2, 3", SC'11).  Each round multiplies words 0 and 2 by the two  *
 * round multipliers, and the high halves are xored with the other two words  *
 * and the round key; the key advances by the two Weyl constants per round.   *
 * ========================================================================= */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int r = 0; r < 10; ++r) {
    if (r > 0) { k0 += W0; k1 += W1; }
    uint64_t p0 = (uint64_t)M0 * (uint64_t)c0;
    uint64_t p1 = (uint64_t)M1 * (uint64_t)c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    uint32_t n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Uniform in (0,1) from a 32-bit word: (w + 1/2) 2^-32.  Box-Muller (1958):
 * rho = sqrt(-2 ln u_a), theta = 2 pi u_b, z0 = rho cos theta, z1 = rho sin theta. */
void orc_box_muller(uint32_t a, uint32_t b, double* z0, double* z1) {
  const double two32 = 4294967296.0;
  double ua = ((double)a + 0.5) / two32;
  double ub = ((double)b + 0.5) / two32;
  double rho = sqrt(-2.0 * log(ua));
  double th = 2.0 * M_PI * ub;
  *z0 = rho * cos(th);
  *z1 = rho * sin(th);
}

/* ========================================================================= *
 * Geometry (Sec. 3.1, Eq. 12-18).                                            *
 * Omega is the rectangle [x0,x1]x[y0,y1] cut into Hx x Hy subdomains; every   *
 * subdomain edge carries m knot intervals, so knots live on the integer       *
 * lattice (i, j), 0 <= i <= LX = Hx m, 0 <= j <= LY = Hy m, on the grid lines  *
 * (i % m == 0 or j % m == 0).  Unknown knots are the interior ones; knots on   *
 * the boundary of Omega carry g and are folded into b.  Order: j, then i.     *
 * ========================================================================= */
typedef struct {
  orc_grid g;
  int LX, LY;
  double dx, dy;
  int n;
  int *ki, *kj;   /* lattice coords of knot k  */
  int *grid;      /* (LX+1)*(LY+1): knot index or -1 */
  int64_t nnz;
  int64_t* row_ptr;
  int32_t* col;
} geom_t;

typedef struct {
  int ilo, ihi, jlo, jhi;  /* patch (slab) box in lattice units, Eq. 13-15 */
  /* per side O in E,N,W,S: */
  int dirichlet[4];        /* the side lies on the boundary of Omega       */
  int line[4];             /* fixed lattice coordinate of the side's line   */
  int a[4], b[4];          /* stencil lattice range along the line, Eq. 17 */
} patch_t;

static int is_knot(const geom_t* G, int i, int j) {
  if (i <= 0 || i >= G->LX || j <= 0 || j >= G->LY) return 0;
  return (i % G->g.m == 0) || (j % G->g.m == 0);
}

/* Slab Q(x_k) = union of the closed grid squares whose boundary holds x_k
 * (Eq. 13).  Omega is a grid-aligned rectangle, so the patch Pi = Q (Eq. 15). */
static void make_patch(const geom_t* G, int k, patch_t* P) {
  int m = G->g.m, E = G->g.ext;
  int i = G->ki[k], j = G->kj[k];
  if (i % m == 0) { P->ilo = i - m; P->ihi = i + m; }
  else            { P->ilo = (i / m) * m; P->ihi = P->ilo + m; }
  if (j % m == 0) { P->jlo = j - m; P->jhi = j + m; }
  else            { P->jlo = (j / m) * m; P->jhi = P->jlo + m; }
  /* E: x = ihi, along y.  N: y = jhi, along x.  W: x = ilo.  S: y = jlo. */
  P->line[0] = P->ihi; P->dirichlet[0] = (P->ihi == G->LX);
  P->line[1] = P->jhi; P->dirichlet[1] = (P->jhi == G->LY);
  P->line[2] = P->ilo; P->dirichlet[2] = (P->ilo == 0);
  P->line[3] = P->jlo; P->dirichlet[3] = (P->jlo == 0);
  for (int o = 0; o < 4; ++o) {
    int vertical = (o == 0 || o == 2);
    int lo = vertical ? P->jlo : P->ilo;
    int hi = vertical ? P->jhi : P->ihi;
    int lmax = vertical ? G->LY : G->LX;
    /* Segment knots plus `ext` knots past each end, kept inside the closure
     * of Omega (Eq. 17 i-iii; extension as in Fig. 3). */
    P->a[o] = lo - E < 0 ? 0 : lo - E;
    P->b[o] = hi + E > lmax ? lmax : hi + E;
  }
}

static int cmp_int(const void* a, const void* b) {
  int x = *(const int*)a, y = *(const int*)b;
  return (x > y) - (x < y);
}

/* Columns of row k: the knot itself and every unknown knot of its stencils. */
static int row_columns(const geom_t* G, int k, int* cols) {
  patch_t P; make_patch(G, k, &P);
  int nc = 0;
  cols[nc++] = k;
  for (int o = 0; o < 4; ++o) {
    if (P.dirichlet[o]) continue;
    int vertical = (o == 0 || o == 2);
    for (int t = P.a[o]; t <= P.b[o]; ++t) {
      int i = vertical ? P.line[o] : t;
      int j = vertical ? t : P.line[o];
      if (is_knot(G, i, j)) cols[nc++] = G->grid[(size_t)j * (G->LX + 1) + i];
    }
  }
  qsort(cols, nc, sizeof(int), cmp_int);
  int u = 0;
  for (int q = 0; q < nc; ++q)
    if (u == 0 || cols[q] != cols[u - 1]) cols[u++] = cols[q];
  return u;
}

static void geom_free(geom_t* G) {
  free(G->ki); free(G->kj); free(G->grid); free(G->row_ptr); free(G->col);
  memset(G, 0, sizeof(*G));
}

static int geom_build(const orc_grid* g, geom_t* G, int with_csr) {
  memset(G, 0, sizeof(*G));
  if (g->Hx < 1 || g->Hy < 1 || g->m < 1 || g->ext < 0 || !(g->x1 > g->x0) || !(g->y1 > g->y0))
    return -1;
  G->g = *g;
  G->LX = g->Hx * g->m; G->LY = g->Hy * g->m;
  G->dx = (g->x1 - g->x0) / G->LX;
  G->dy = (g->y1 - g->y0) / G->LY;
  size_t np = (size_t)(G->LX + 1) * (G->LY + 1);
  G->grid = (int*)malloc(np * sizeof(int));
  int cnt = 0;
  for (int j = 0; j <= G->LY; ++j)
    for (int i = 0; i <= G->LX; ++i) {
      int kk = is_knot(G, i, j) ? cnt++ : -1;
      G->grid[(size_t)j * (G->LX + 1) + i] = kk;
    }
  G->n = cnt;
  G->ki = (int*)malloc((size_t)(cnt > 0 ? cnt : 1) * sizeof(int));
  G->kj = (int*)malloc((size_t)(cnt > 0 ? cnt : 1) * sizeof(int));
  for (int j = 0; j <= G->LY; ++j)
    for (int i = 0; i <= G->LX; ++i) {
      int kk = G->grid[(size_t)j * (G->LX + 1) + i];
      if (kk >= 0) { G->ki[kk] = i; G->kj[kk] = j; }
    }
  if (!with_csr) return 0;
  G->row_ptr = (int64_t*)malloc((size_t)(cnt + 1) * sizeof(int64_t));
  int maxc = 1 + 4 * (2 * g->m + 2 * g->ext + 1);
  int* cols = (int*)malloc((size_t)maxc * sizeof(int));
  G->row_ptr[0] = 0;
  for (int k = 0; k < cnt; ++k) G->row_ptr[k + 1] = G->row_ptr[k] + row_columns(G, k, cols);
  G->nnz = G->row_ptr[cnt];
  G->col = (int32_t*)malloc((size_t)(G->nnz > 0 ? G->nnz : 1) * sizeof(int32_t));
  for (int k = 0; k < cnt; ++k) {
    int nc = row_columns(G, k, cols);
    for (int q = 0; q < nc; ++q) G->col[G->row_ptr[k] + q] = cols[q];
  }
  free(cols);
  return 0;
}

int orc_geometry_size(const orc_grid* g, int64_t* n, int64_t* nnz) {
  geom_t G;
  if (geom_build(g, &G, 1)) return -1;
  *n = G.n; *nnz = G.nnz;
  geom_free(&G);
  return 0;
}

int orc_geometry(const orc_grid* g, double* xy, int64_t* row_ptr, int32_t* col) {
  geom_t G;
  if (geom_build(g, &G, 1)) return -1;
  for (int k = 0; k < G.n; ++k) {
    if (xy) {
      xy[2 * k] = g->x0 + G.ki[k] * G.dx;
      xy[2 * k + 1] = g->y0 + G.kj[k] * G.dy;
    }
  }
  if (row_ptr) memcpy(row_ptr, G.row_ptr, (size_t)(G.n + 1) * sizeof(int64_t));
  if (col) memcpy(col, G.col, (size_t)G.nnz * sizeof(int32_t));
  geom_free(&G);
  return 0;
}

/* ========================================================================= *
 * Coefficients of Eq. 6 (sigma = s I, so A = s^2 I and the generator is       *
 * (s^2/2) Lap + d . grad), and the boundary data g.                           *
 * ========================================================================= */
static double table_bilinear(const orc_grid* g, const float* T, int nx, int ny, double x, double y) {
  double fx = (x - g->x0) / (g->x1 - g->x0) * (nx - 1);
  double fy = (y - g->y0) / (g->y1 - g->y0) * (ny - 1);
  int i = (int)floor(fx), j = (int)floor(fy);
  if (i < 0) i = 0;
  if (i > nx - 2) i = nx - 2;
  if (j < 0) j = 0;
  if (j > ny - 2) j = ny - 2;
  double tx = fx - i, ty = fy - j;
  double v00 = T[(size_t)j * nx + i], v10 = T[(size_t)j * nx + i + 1];
  double v01 = T[(size_t)(j + 1) * nx + i], v11 = T[(size_t)(j + 1) * nx + i + 1];
  return (1 - tx) * (1 - ty) * v00 + tx * (1 - ty) * v10 + (1 - tx) * ty * v01 + tx * ty * v11;
}

/* Eq. 43: u = 3 + sin(r)/3 + tanh(q)/3 with r = sqrt(1 + x^2/100 + y^2/50) and
 * q = sin(3x/25 + y/20) + sin(x/20 - 3y/25). */
static double e1_u(double x, double y) {
  double r = sqrt(1.0 + x * x / 100.0 + y * y / 50.0);
  double q = sin(3.0 * x / 25.0 + y / 20.0) + sin(x / 20.0 - 3.0 * y / 25.0);
  return 3.0 + sin(r) / 3.0 + tanh(q) / 3.0;
}

/* Lap u of Eq. 43, by the chain rule:
 *   Lap sin r = cos r Lap r - sin r |grad r|^2,  |grad r|^2 = G / r^2,
 *   Lap r = (1/100 + 1/50) / r - G / r^3,         G = x^2/100^2 + y^2/50^2;
 *   Lap tanh q = (1 - T^2) Lap q - 2 T (1 - T^2) |grad q|^2,  T = tanh q,
 *   Lap q = -((3/25)^2 + (1/20)^2) q,
 *   grad q = ((3/25) cos a + (1/20) cos b, (1/20) cos a - (3/25) cos b). */
static double e1_laplacian(double x, double y) {
  double r = sqrt(1.0 + x * x / 100.0 + y * y / 50.0);
  double G = x * x / 1.0e4 + y * y / 2.5e3;
  double lap_r = (1.0 / 100.0 + 1.0 / 50.0) / r - G / (r * r * r);
  double lap_sin = cos(r) * lap_r - sin(r) * G / (r * r);
  double a = 3.0 * x / 25.0 + y / 20.0, bb = x / 20.0 - 3.0 * y / 25.0;
  double q = sin(a) + sin(bb);
  double qx = 3.0 / 25.0 * cos(a) + cos(bb) / 20.0;
  double qy = cos(a) / 20.0 - 3.0 / 25.0 * cos(bb);
  double T = tanh(q);
  double lap_q = -((3.0 / 25.0) * (3.0 / 25.0) + (1.0 / 20.0) * (1.0 / 20.0)) * q;
  double lap_tanh = (1.0 - T * T) * lap_q - 2.0 * T * (1.0 - T * T) * (qx * qx + qy * qy);
  return (lap_sin + lap_tanh) / 3.0;
}

/* Tabulated grad u0 (Sec. 4.2's interpolatory look-up table of F / sigma):
 * bilinear between the nodes of a [cv_ny][cv_nx] grid spanning Omega, the
 * point clamped to the closure of Omega. */
static void cv_table_grad(const orc_grid* g, const orc_coeffs* cf, double x, double y,
                          double* gx, double* gy) {
  const int nx = cf->cv_nx, ny = cf->cv_ny;
  double fx = (x - g->x0) / (g->x1 - g->x0) * (nx - 1);
  double fy = (y - g->y0) / (g->y1 - g->y0) * (ny - 1);
  int i = (int)floor(fx), j = (int)floor(fy);
  if (i < 0) i = 0;
  if (i > nx - 2) i = nx - 2;
  if (j < 0) j = 0;
  if (j > ny - 2) j = ny - 2;
  double tx = fx - i, ty = fy - j;
  if (tx < 0) tx = 0;
  if (tx > 1) tx = 1;
  if (ty < 0) ty = 0;
  if (ty > 1) ty = 1;
  for (int q = 0; q < 2; ++q) {
    const float* T = cf->cv_tab + q;
    double v00 = T[2 * ((size_t)j * nx + i)], v10 = T[2 * ((size_t)j * nx + i + 1)];
    double v01 = T[2 * ((size_t)(j + 1) * nx + i)], v11 = T[2 * ((size_t)(j + 1) * nx + i + 1)];
    double v = (1 - tx) * (1 - ty) * v00 + tx * (1 - ty) * v10 + (1 - tx) * ty * v01 + tx * ty * v11;
    if (q == 0) *gx = v; else *gy = v;
  }
}

void orc_coeffs_eval(const orc_grid* g, const orc_coeffs* cf, double x, double y,
                     double* s, double* dx, double* dy, double* c, double* f) {
  const double pi = M_PI;
  switch (cf->id) {
  case ORC_COEF_LAPLACE_EXPSIN:
    *s = sqrt(2.0); *dx = 0; *dy = 0; *c = 0; *f = 0;
    break;
  case ORC_COEF_MANUFACTURED: {
    /* u = sin(pi x) cos(pi y) + x y;  Lap u = -2 pi^2 sin(pi x) cos(pi y). */
    double sx = sin(pi * x), cx = cos(pi * x), sy = sin(pi * y), cy = cos(pi * y);
    double u = sx * cy + x * y;
    double ux = pi * cx * cy + y;
    double uy = -pi * sx * sy + x;
    double lap = -2.0 * pi * pi * sx * cy;
    *s = sqrt(2.0);
    *dx = sin(2.0 * pi * y);
    *dy = cos(2.0 * pi * x);
    *c = -(1.0 + x * x);
    *f = lap + (*dx) * ux + (*dy) * uy + (*c) * u;  /* (s^2/2) = 1 */
    break;
  }
  case ORC_COEF_VARSIGMA: {
    /* u = e^{x/4} cos(y/2);  Lap u = (1/16 - 1/4) u. */
    double sg = sqrt(2.0) * (1.0 + 0.3 * sin(2.0 * pi * x) * sin(2.0 * pi * y));
    double u = exp(x / 4.0) * cos(y / 2.0);
    *s = sg; *dx = 0; *dy = 0; *c = -1.0;
    *f = 0.5 * sg * sg * (1.0 / 16.0 - 1.0 / 4.0) * u + (*c) * u;
    break;
  }
  case ORC_COEF_TABLE:
    *s = table_bilinear(g, cf->sigma_tab, cf->tab_nx, cf->tab_ny, x, y);
    *c = table_bilinear(g, cf->c_tab, cf->tab_nx, cf->tab_ny, x, y);
    *dx = 0; *dy = 0; *f = cf->params[0];
    break;
  case ORC_COEF_POISSON_E1:
    /* Eq. 42 reads Lap u = f; with s = sqrt2 the generator (s^2/2) Lap is Lap,
     * so f is Eq. 42's right-hand side, Lap of the u of Eq. 43. */
    *s = sqrt(2.0); *dx = 0; *dy = 0; *c = 0; *f = e1_laplacian(x, y);
    break;
  default: /* ORC_COEF_CONSTANT */
    *s = cf->params[0]; *dx = cf->params[1]; *dy = cf->params[2];
    *c = cf->params[3]; *f = cf->params[4];
    break;
  }
}

double orc_boundary_g(const orc_coeffs* cf, double x, double y) {
  const double pi = M_PI;
  switch (cf->id) {
  case ORC_COEF_LAPLACE_EXPSIN: return exp(x) * sin(y);
  case ORC_COEF_MANUFACTURED:   return sin(pi * x) * cos(pi * y) + x * y;
  case ORC_COEF_VARSIGMA:       return exp(x / 4.0) * cos(y / 2.0);
  case ORC_COEF_TABLE:          return cf->params[1];
  case ORC_COEF_POISSON_E1:     return e1_u(x, y);
  default:                      return cf->params[5];
  }
}

/* ========================================================================= *
 * v_theta : R^2 -> R, 2 -> 64 -> 64 -> 1 with SiLU (a * logistic(a)).         *
 * theta layout: W1[64][2], b1[64], W2[64][64] (row = output), b2[64], w3[64], *
 * b3.                                                                         *
 * ========================================================================= */
#define HID ORC_MLP_HIDDEN
static double logistic(double a) { return 1.0 / (1.0 + exp(-a)); }

typedef struct { double a1[HID], h1[HID], a2[HID], h2[HID], v; } mlp_fwd_t;

static void mlp_forward(const double* th, double x, double y, mlp_fwd_t* F) {
  const double *W1 = th, *b1 = W1 + 2 * HID, *W2 = b1 + HID, *b2 = W2 + HID * HID,
               *w3 = b2 + HID, *b3 = w3 + HID;
  for (int i = 0; i < HID; ++i) {
    F->a1[i] = W1[2 * i] * x + W1[2 * i + 1] * y + b1[i];
    F->h1[i] = F->a1[i] * logistic(F->a1[i]);
  }
  for (int i = 0; i < HID; ++i) {
    double s = b2[i];
    for (int j = 0; j < HID; ++j) s += W2[i * HID + j] * F->h1[j];
    F->a2[i] = s;
    F->h2[i] = s * logistic(s);
  }
  double v = b3[0];
  for (int i = 0; i < HID; ++i) v += w3[i] * F->h2[i];
  F->v = v;
}

/* d/da [a logistic(a)] = logistic(a) (1 + a (1 - logistic(a))). */
static double dsilu(double a) { double s = logistic(a); return s * (1.0 + a * (1.0 - s)); }

double orc_mlp_value(const double* th, double x, double y) {
  mlp_fwd_t F; mlp_forward(th, x, y, &F); return F.v;
}

void orc_mlp_grad_x(const double* th, double x, double y, double* gx, double* gy) {
  const double *W1 = th, *b1 = W1 + 2 * HID, *W2 = b1 + HID, *b2 = W2 + HID * HID, *w3 = b2 + HID;
  mlp_fwd_t F; mlp_forward(th, x, y, &F);
  double g2[HID], g1[HID];
  for (int i = 0; i < HID; ++i) g2[i] = w3[i] * dsilu(F.a2[i]);            /* dv/da2 */
  for (int j = 0; j < HID; ++j) {                                           /* dv/da1 */
    double s = 0;
    for (int i = 0; i < HID; ++i) s += W2[i * HID + j] * g2[i];
    g1[j] = s * dsilu(F.a1[j]);
  }
  double sx = 0, sy = 0;
  for (int j = 0; j < HID; ++j) { sx += W1[2 * j] * g1[j]; sy += W1[2 * j + 1] * g1[j]; }
  *gx = sx; *gy = sy;
}

double orc_mlp_loss_grad(const double* th, const double* xy, const double* target,
                         int64_t npts, double* grad) {
  const double *W2 = th + 2 * HID + HID, *w3 = W2 + HID * HID + HID;
  double *gW1 = grad, *gb1 = gW1 + 2 * HID, *gW2 = gb1 + HID, *gb2 = gW2 + HID * HID,
         *gw3 = gb2 + HID, *gb3 = gw3 + HID;
  memset(grad, 0, sizeof(double) * ORC_MLP_NPARAM);
  double loss = 0;
  for (int64_t p = 0; p < npts; ++p) {
    double x = xy[2 * p], y = xy[2 * p + 1];
    mlp_fwd_t F; mlp_forward(th, x, y, &F);
    double r = F.v - target[p];
    loss += r * r;
    double dv = 2.0 * r / (double)npts;                   /* dL/dv */
    double d2[HID], d1[HID];
    gb3[0] += dv;
    for (int i = 0; i < HID; ++i) { gw3[i] += dv * F.h2[i]; d2[i] = dv * w3[i] * dsilu(F.a2[i]); }
    for (int i = 0; i < HID; ++i) {
      gb2[i] += d2[i];
      for (int j = 0; j < HID; ++j) gW2[i * HID + j] += d2[i] * F.h1[j];
    }
    for (int j = 0; j < HID; ++j) {
      double s = 0;
      for (int i = 0; i < HID; ++i) s += W2[i * HID + j] * d2[i];
      d1[j] = s * dsilu(F.a1[j]);
      gb1[j] += d1[j];
      gW1[2 * j] += d1[j] * x;
      gW1[2 * j + 1] += d1[j] * y;
    }
  }
  return loss / (double)npts;
}

void orc_adam_step(double* th, const double* g, double* m, double* v, int64_t t,
                   int64_t np, double lr, double b1, double b2, double eps) {
  double c1 = 1.0 - pow(b1, (double)t), c2 = 1.0 - pow(b2, (double)t);
  for (int64_t i = 0; i < np; ++i) {
    m[i] = b1 * m[i] + (1.0 - b1) * g[i];
    v[i] = b2 * v[i] + (1.0 - b2) * g[i] * g[i];
    th[i] -= lr * (m[i] / c1) / (sqrt(v[i] / c2) + eps);
  }
}

/* ========================================================================= *
 * One Feynman-Kac path inside the patch of knot k (Eq. 9, naive EM, Sec. 2.3) *
 * and its exit resolution (Eq. 22-25, corner rule of Sec. 3.3).               *
 * ========================================================================= */
typedef struct {
  const geom_t* G;
  const orc_coeffs* cf;
  double dt;                 /* reference step (the step cap k_max is given at dt) */
  const double* h_per_knot;  /* per-knot steps h_k, or NULL for dt everywhere      */
  uint32_t key[2];
  uint32_t tag;
  int64_t k_max;
  int interp;                /* ORC_INTERP_*                                     */
  double rbf_c;              /* IMQ shape parameter (absolute units)              */
  struct rbf_cache_s* rbf[2];/* factorised RBF matrices: [0] lines along x,
                                [1] lines along y (lattice spacing dx, dy)       */
} sim_t;

/* ========================================================================= *
 * 1-D RBF interpolation on a stencil (Sec. 2.1, Eq. 1-5) with the inverse     *
 * multiquadric phi_c(r) = 1 / sqrt(r^2 + c^2) (Eq. 3, read with + c^2).        *
 * On an equispaced stencil of m points the cardinal functions, in lattice     *
 * units, depend only on m and c / spacing: H(z) = Phi^{-1} phi(z) with        *
 * phi(z)_i = phi_c(|z - z_i|) (Eq. 5, Phi symmetric), computed by LU with      *
 * partial pivoting in FP64.                                                   *
 * ========================================================================= */
typedef struct rbf_cache_s {
  double c_lat;              /* shape parameter in lattice units                */
  double* lu[ORC_MAX_STENCIL + 1];   /* LU factors of Phi for stencil length m  */
  int* piv[ORC_MAX_STENCIL + 1];
  pthread_mutex_t mu;
} rbf_cache_t;

static double imq(double r, double c) { return 1.0 / sqrt(r * r + c * c); }

/* In-place LU with partial pivoting of the m x m row-major A; 0 or -1 if singular. */
static int lu_factor(int m, double* A, int* piv) {
  for (int k = 0; k < m; ++k) {
    int p = k;
    for (int i = k + 1; i < m; ++i)
      if (fabs(A[(size_t)i * m + k]) > fabs(A[(size_t)p * m + k])) p = i;
    piv[k] = p;
    if (A[(size_t)p * m + k] == 0.0) return -1;
    if (p != k)
      for (int j = 0; j < m; ++j) {
        double t = A[(size_t)k * m + j];
        A[(size_t)k * m + j] = A[(size_t)p * m + j];
        A[(size_t)p * m + j] = t;
      }
    for (int i = k + 1; i < m; ++i) {
      double l = A[(size_t)i * m + k] / A[(size_t)k * m + k];
      A[(size_t)i * m + k] = l;
      for (int j = k + 1; j < m; ++j) A[(size_t)i * m + j] -= l * A[(size_t)k * m + j];
    }
  }
  return 0;
}

static void lu_solve_inplace(int m, const double* LU, const int* piv, double* x) {
  /* whole rows (multipliers included) were swapped: P A = L U */
  for (int k = 0; k < m; ++k)
    if (piv[k] != k) { double t = x[k]; x[k] = x[piv[k]]; x[piv[k]] = t; }
  for (int k = 0; k < m; ++k)
    for (int i = k + 1; i < m; ++i) x[i] -= LU[(size_t)i * m + k] * x[k];
  for (int i = m - 1; i >= 0; --i) {
    double v = x[i];
    for (int j = i + 1; j < m; ++j) v -= LU[(size_t)i * m + j] * x[j];
    x[i] = v / LU[(size_t)i * m + i];
  }
}

static void rbf_matrix(int m, double c, double* A) {
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < m; ++j) A[(size_t)i * m + j] = imq((double)(i - j), c);
}

/* Cardinal functions H_0..H_{m-1} at z (lattice units from the first point). */
static int rbf_eval(const double* LU, const int* piv, int m, double c, double z, double* H) {
  for (int i = 0; i < m; ++i) H[i] = imq(z - (double)i, c);
  lu_solve_inplace(m, LU, piv, H);
  return 0;
}

static int rbf_get(rbf_cache_t* C, int m, const double** LU, const int** piv) {
  pthread_mutex_lock(&C->mu);
  if (!C->lu[m]) {
    double* A = (double*)malloc((size_t)m * m * sizeof(double));
    int* p = (int*)malloc((size_t)m * sizeof(int));
    rbf_matrix(m, C->c_lat, A);
    if (lu_factor(m, A, p)) { free(A); free(p); pthread_mutex_unlock(&C->mu); return -1; }
    C->lu[m] = A;
    C->piv[m] = p;
  }
  *LU = C->lu[m];
  *piv = C->piv[m];
  pthread_mutex_unlock(&C->mu);
  return 0;
}

static void rbf_cache_free(rbf_cache_t* C) {
  if (!C) return;
  for (int m = 0; m <= ORC_MAX_STENCIL; ++m) { free(C->lu[m]); free(C->piv[m]); }
  pthread_mutex_destroy(&C->mu);
  free(C);
}

int orc_rbf_cardinal(int32_t m, double c_lat, double z, double* H) {
  if (m < 2 || m > ORC_MAX_STENCIL || !(c_lat > 0)) return -1;
  double* A = (double*)malloc((size_t)m * m * sizeof(double));
  int* p = (int*)malloc((size_t)m * sizeof(int));
  rbf_matrix(m, c_lat, A);
  int rc = lu_factor(m, A, p);
  if (!rc) rbf_eval(A, p, m, c_lat, z, H);
  free(A);
  free(p);
  return rc;
}

/* Eigenvalues of the symmetric m x m matrix A (destroyed) by cyclic Jacobi
 * rotations; returns the spectral condition number max|l| / min|l|. */
static double sym_cond(int m, double* A) {
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0;
    for (int i = 0; i < m; ++i)
      for (int j = i + 1; j < m; ++j) off += A[(size_t)i * m + j] * A[(size_t)i * m + j];
    if (off < 1e-300) break;
    for (int p = 0; p < m; ++p)
      for (int q = p + 1; q < m; ++q) {
        double apq = A[(size_t)p * m + q];
        if (fabs(apq) < 1e-300) continue;
        double app = A[(size_t)p * m + p], aqq = A[(size_t)q * m + q];
        double th = (aqq - app) / (2.0 * apq);
        double t = (th >= 0 ? 1.0 : -1.0) / (fabs(th) + sqrt(th * th + 1.0));
        double cs = 1.0 / sqrt(t * t + 1.0), sn = t * cs;
        for (int k = 0; k < m; ++k) {
          double akp = A[(size_t)k * m + p], akq = A[(size_t)k * m + q];
          A[(size_t)k * m + p] = cs * akp - sn * akq;
          A[(size_t)k * m + q] = sn * akp + cs * akq;
        }
        for (int k = 0; k < m; ++k) {
          double apk = A[(size_t)p * m + k], aqk = A[(size_t)q * m + k];
          A[(size_t)p * m + k] = cs * apk - sn * aqk;
          A[(size_t)q * m + k] = sn * apk + cs * aqk;
        }
      }
  }
  double lo = 1e300, hi = 0.0;
  for (int i = 0; i < m; ++i) {
    double v = fabs(A[(size_t)i * m + i]);
    if (v < lo) lo = v;
    if (v > hi) hi = v;
  }
  return hi / lo;
}

double orc_rbf_cond(int32_t m, double c_lat) {
  double* A = (double*)malloc((size_t)m * m * sizeof(double));
  rbf_matrix(m, c_lat, A);
  double k = sym_cond(m, A);
  free(A);
  return k;
}

/* The shape parameter (lattice units) at which the spectral condition number
 * of Phi for an m-point stencil equals `cond` (Sec. 5.1 fixes c that way):
 * bisection on log c, the condition number growing with c. */
double orc_rbf_shape_for_cond(int32_t m, double cond) {
  double lo = 1e-3, hi = 1e2;
  for (int it = 0; it < 200; ++it) {
    double mid = sqrt(lo * hi);
    if (orc_rbf_cond(m, mid) < cond) lo = mid; else hi = mid;
    if (hi / lo < 1.0 + 1e-12) break;
  }
  return sqrt(lo * hi);
}

typedef struct {
  int steps, side, flags;
  int nw;                        /* entries used in col[] / w[]          */
  int col[ORC_MAX_STENCIL];      /* unknown-knot columns, -1 if none     */
  double w[ORC_MAX_STENCIL];     /* Y * interpolation weight for col[]   */
  double bsum;         /* everything that goes to b (Z + xi + Dirichlet terms) */
  double Y;
  double xi;           /* the control-variate integral alone (0 without one) */
  double s_line;       /* exit coordinate along the side's line, lattice units */
} path_out_t;

typedef struct { double xlo, xhi, ylo, yhi; } box_t;

/* Step of knot k and its step cap: the cap covers the same time horizon as
 * k_max steps of dt, i.e. ceil(k_max dt / h_k) steps. */
static double knot_h(const sim_t* S, int k) {
  return S->h_per_knot ? S->h_per_knot[k] : S->dt;
}
static int64_t knot_cap(const sim_t* S, double h) {
  if (h == S->dt) return S->k_max;
  double c = ceil((double)S->k_max * S->dt / h);
  return c < 1.0 ? 1 : (int64_t)c;
}

/* Gobet-Menozzi shift (Sec. 2.3): every side of the patch moves inwards by
 * 0.5826 |sigma(P) N| sqrt(h), with P the normal projection of the current
 * point on that side (kept on the closed side) and N its normal.  With
 * sigma = s I this is 0.5826 |s(P)| sqrt(h). */
static void gm_shifts(const sim_t* S, const box_t* B, double X, double Yp, double h,
                      double shift[4]) {
  double cx = X < B->xlo ? B->xlo : (X > B->xhi ? B->xhi : X);
  double cy = Yp < B->ylo ? B->ylo : (Yp > B->yhi ? B->yhi : Yp);
  const double px[4] = {B->xhi, cx, B->xlo, cx};
  const double py[4] = {cy, B->yhi, cy, B->ylo};
  for (int o = 0; o < 4; ++o) {
    double s, dxv, dyv, c, f;
    orc_coeffs_eval(&S->G->g, S->cf, px[o], py[o], &s, &dxv, &dyv, &c, &f);
    shift[o] = ORC_GM_SHIFT * fabs(s) * sqrt(h);
  }
}

/* Exit resolution (Eq. 22-25, corner rule of Sec. 3.3) of the state
 * (X, Yp, Y = exp(Sacc), Z, xi) after n steps.  The exit side is the side
 * with the smallest positive overshoot past its line moved inwards by
 * shift[o] (all zero for naive EM; ties E < N < W < S); a truncated path that
 * is inside every moved line goes to the nearest one.  The exit point is the
 * normal projection on the side's true line. */
static void resolve_exit(const sim_t* S, const patch_t* P, const box_t* B, double X, double Yp,
                         double Sacc, double Z, double xi, int truncated, int64_t n,
                         const double shift[4], path_out_t* out) {
  const geom_t* G = S->G;
  const orc_grid* g = &G->g;
  double Yk = exp(Sacc);
  /* Signed overshoot past each (moved) side, E N W S. */
  double ov[4] = {X - B->xhi + shift[0], Yp - B->yhi + shift[1], B->xlo - X + shift[2],
                  B->ylo - Yp + shift[3]};
  int side = -1;
  for (int o = 0; o < 4; ++o)          /* smallest positive overshoot */
    if (ov[o] > 0 && (side < 0 || ov[o] < ov[side])) side = o;
  if (side < 0)                         /* truncated inside: nearest side */
    for (int o = 0; o < 4; ++o)
      if (side < 0 || ov[o] > ov[side]) side = o;

  out->steps = (int)n;
  out->side = side;
  out->flags = truncated ? 1 : 0;
  out->nw = 2;
  out->col[0] = out->col[1] = -1;
  out->w[0] = out->w[1] = 0;
  out->s_line = 0.0;
  out->Y = Yk;
  out->xi = xi;
  double bsum = Z + xi;
  int vertical = (side == 0 || side == 2);
  double line_xy = vertical ? (side == 0 ? B->xhi : B->xlo) : (side == 1 ? B->yhi : B->ylo);
  double along = vertical ? Yp : X;
  if (P->dirichlet[side]) {
    /* Exit on the boundary of Omega: score g(P) Y (Eq. 25), P projected
     * normally and kept in the closure of Omega. */
    double lo = vertical ? g->y0 : g->x0, hi = vertical ? g->y1 : g->x1;
    if (along < lo) along = lo;
    if (along > hi) along = hi;
    double px = vertical ? line_xy : along, py = vertical ? along : line_xy;
    bsum += Yk * orc_boundary_g(S->cf, px, py);
  } else {
    /* Exit on an interface: piecewise-linear interpolation over the side's
     * extended stencil (Eq. 21-22 with a linear scheme, footnote 8). */
    double origin = vertical ? g->y0 : g->x0, step = vertical ? G->dy : G->dx;
    int lmax = vertical ? G->LY : G->LX;
    double s = (along - origin) / step;
    if (s < P->a[side]) { s = P->a[side]; out->flags |= 2; }
    if (s > P->b[side]) { s = P->b[side]; out->flags |= 2; }
    out->s_line = s;
    if (S->interp == ORC_INTERP_RBF) {
      /* Eq. 21-22: every stencil knot j gets the cardinal weight H_j(P). */
      int m = P->b[side] - P->a[side] + 1;
      const double* LU;
      const int* piv;
      double H[ORC_MAX_STENCIL];
      rbf_cache_t* C = S->rbf[vertical ? 1 : 0];
      if (rbf_get(C, m, &LU, &piv) == 0) {
        rbf_eval(LU, piv, m, C->c_lat, s - P->a[side], H);
      } else {
        for (int q = 0; q < m; ++q) H[q] = 0.0;
      }
      out->nw = m;
      for (int q = 0; q < m; ++q) {
        int tl = P->a[side] + q;
        int i = vertical ? P->line[side] : tl;
        int j = vertical ? tl : P->line[side];
        out->col[q] = -1;
        out->w[q] = 0.0;
        if (tl == 0 || tl == lmax)
          bsum += Yk * H[q] * orc_boundary_g(S->cf, g->x0 + i * G->dx, g->y0 + j * G->dy);
        else {
          out->col[q] = G->grid[(size_t)j * (G->LX + 1) + i];
          out->w[q] = Yk * H[q];
        }
      }
    } else {
      int t = (int)floor(s);
      if (t >= P->b[side]) t = P->b[side] - 1;
      double lam = s - t;
      double w[2] = {1.0 - lam, lam};
      for (int q = 0; q < 2; ++q) {
        int tl = t + q;
        int i = vertical ? P->line[side] : tl;
        int j = vertical ? tl : P->line[side];
        if (tl == 0 || tl == lmax) {
          /* Stencil end on the boundary of Omega: known value g there. */
          bsum += Yk * w[q] * orc_boundary_g(S->cf, g->x0 + i * G->dx, g->y0 + j * G->dy);
        } else {
          out->col[q] = G->grid[(size_t)j * (G->LX + 1) + i];
          out->w[q] = Yk * w[q];
        }
      }
    }
  }
  out->bsum = bsum;
}

/* One Feynman-Kac path inside the patch of knot k (Eq. 9, Euler-Maruyama with
 * the knot's step h_k).  mode bit 0 asks for the naive exit (first step
 * outside the closed patch), bit 1 for the Gobet-Menozzi exit (first step
 * outside the patch with its sides moved inwards, Sec. 2.3).  With both bits
 * the path is the "mixed GM/EM" trajectory of Sec. 4.1: after the GM exit it
 * simply goes on until the naive exit, so both scores come from one path. */
static void simulate(const sim_t* S, int k, int64_t p, int mode, path_out_t* em, path_out_t* gm) {
  const geom_t* G = S->G;
  const orc_grid* g = &G->g;
  patch_t P; make_patch(G, k, &P);
  box_t B = {g->x0 + P.ilo * G->dx, g->x0 + P.ihi * G->dx,
             g->y0 + P.jlo * G->dy, g->y0 + P.jhi * G->dy};
  const double h = knot_h(S, k), sqh = sqrt(h);
  const int64_t cap = knot_cap(S, h);
  const double zero[4] = {0, 0, 0, 0};
  double X = g->x0 + G->ki[k] * G->dx, Yp = g->y0 + G->kj[k] * G->dy;
  double Sacc = 0.0, Z = 0.0, xi = 0.0;   /* Y = exp(S) */
  int64_t n = 0;
  int need_em = mode & 1, need_gm = (mode >> 1) & 1;
  double z[4] = {0, 0, 0, 0};
  for (;;) {
    if ((n & 1) == 0) {
      /* One Philox call per two steps: counter (step pair, path, knot, tag). */
      uint32_t ctr[4] = {(uint32_t)(n >> 1), (uint32_t)p, (uint32_t)k, S->tag}, r[4];
      orc_philox4x32_10(ctr, S->key, r);
      orc_box_muller(r[0], r[1], &z[0], &z[1]);
      orc_box_muller(r[2], r[3], &z[2], &z[3]);
    }
    double zx = z[(n & 1) * 2], zy = z[(n & 1) * 2 + 1];
    double s, dxv, dyv, c, f;
    orc_coeffs_eval(g, S->cf, X, Yp, &s, &dxv, &dyv, &c, &f);
    double Yw = exp(Sacc);
    double dWx = sqh * zx, dWy = sqh * zy;
    Z -= f * Yw * h;                                     /* dZ = -f Y dt      */
    if (S->cf->mlp) {                                    /* dxi = -Y F . dW   */
      double gx, gy;
      orc_mlp_grad_x(S->cf->mlp, X, Yp, &gx, &gy);
      xi -= Yw * s * (gx * dWx + gy * dWy);              /* F = sigma^T grad v */
    } else if (S->cf->cv_tab) {                          /* F from the table  */
      double gx, gy;
      cv_table_grad(g, S->cf, X, Yp, &gx, &gy);
      xi -= Yw * s * (gx * dWx + gy * dWy);
    }
    Sacc += c * h;                                       /* dY = c Y dt       */
    X += dxv * h + s * dWx;                              /* dX = d dt + s dW  */
    Yp += dyv * h + s * dWy;
    ++n;
    if (need_gm) {                                       /* left the moved patch */
      double sh[4];
      gm_shifts(S, &B, X, Yp, h, sh);
      if (X > B.xhi - sh[0] || Yp > B.yhi - sh[1] || X < B.xlo + sh[2] || Yp < B.ylo + sh[3]) {
        resolve_exit(S, &P, &B, X, Yp, Sacc, Z, xi, 0, n, sh, gm);
        need_gm = 0;
      }
    }
    if (need_em && (X > B.xhi || X < B.xlo || Yp > B.yhi || Yp < B.ylo)) {  /* left closed patch */
      resolve_exit(S, &P, &B, X, Yp, Sacc, Z, xi, 0, n, zero, em);
      need_em = 0;
    }
    if (!need_em && !need_gm) break;
    if (n >= cap) {                                      /* truncated */
      if (need_gm) {
        double sh[4];
        gm_shifts(S, &B, X, Yp, h, sh);
        resolve_exit(S, &P, &B, X, Yp, Sacc, Z, xi, 1, n, sh, gm);
      }
      if (need_em) resolve_exit(S, &P, &B, X, Yp, Sacc, Z, xi, 1, n, zero, em);
      break;
    }
  }
}

/* ========================================================================= *
 * Row assembly (Eq. 24-25).  Raw sums: val holds sum_p Y w for each column,   *
 * b holds sum_p of the b contributions; orc_finalize_rows divides by N_k.     *
 * ========================================================================= */
typedef struct job_s job_t;
struct job_s {
  sim_t S;
  int scheme;
  void (*row_fn)(job_t*, int, int64_t*);
  const double* u0;          /* calibration: nodal warm-up solution */
  double* moments;           /* calibration: [nrows][ORC_CAL_NMOM] */
  orc_cal_record* cal_records;
  const int64_t* n_per_knot;
  int64_t n_paths;
  const int32_t* rows;
  int32_t nrows;
  double* val;
  double* b;
  orc_record* records;
  const int64_t* rec_off;     /* record offset per requested row */
  int next;                    /* shared row counter */
  pthread_mutex_t mu;
  int64_t stats[3];
};

static int64_t paths_of(const job_t* J, int k) {
  return J->n_per_knot ? J->n_per_knot[k] : J->n_paths;
}

static void assemble_row(job_t* J, int r, int64_t* st) {
  const geom_t* G = J->S.G;
  int k = J->rows[r];
  int64_t N = paths_of(J, k);
  int64_t rb = G->row_ptr[k], re = G->row_ptr[k + 1];
  int nc = (int)(re - rb);
  double* acc = (double*)calloc((size_t)nc, sizeof(double));
  double bacc = 0.0;
  for (int64_t p = 0; p < N; ++p) {
    path_out_t o;
    if (J->scheme == ORC_SCHEME_GM) simulate(&J->S, k, p, 2, NULL, &o);
    else simulate(&J->S, k, p, 1, &o, NULL);
    st[0] += o.steps;
    st[1] += (o.flags & 1) ? 1 : 0;
    st[2] += (o.flags & 2) ? 1 : 0;
    for (int q = 0; q < o.nw; ++q) {
      if (o.col[q] < 0) continue;
      int lo = 0, hi = nc - 1, pos = -1;       /* column search in the row */
      while (lo <= hi) {
        int mid = (lo + hi) / 2;
        int cm = G->col[rb + mid];
        if (cm == o.col[q]) { pos = mid; break; }
        if (cm < o.col[q]) lo = mid + 1; else hi = mid - 1;
      }
      if (pos >= 0) acc[pos] += o.w[q];
    }
    bacc += o.bsum;
    if (J->records) {
      orc_record* R = &J->records[J->rec_off[r] + p];
      R->steps = o.steps; R->side = o.side; R->flags = o.flags;
      const int lin = J->S.interp != ORC_INTERP_RBF;  /* RBF: weights from s_line */
      R->col_a = lin ? o.col[0] : -1; R->col_b = lin ? o.col[1] : -1; R->pad_ = 0;
      R->w_a = lin ? o.w[0] : 0.0; R->w_b = lin ? o.w[1] : 0.0;
      R->b_contrib = o.bsum; R->Y = o.Y; R->s_line = o.s_line;
    }
  }
  for (int q = 0; q < nc; ++q) J->val[rb + q] = acc[q];
  J->b[k] = bacc;
  free(acc);
}

static void* worker(void* arg) {
  job_t* J = (job_t*)arg;
  int64_t st[3] = {0, 0, 0};
  for (;;) {
    pthread_mutex_lock(&J->mu);
    int r = J->next++;
    pthread_mutex_unlock(&J->mu);
    if (r >= J->nrows) break;
    J->row_fn(J, r, st);
  }
  pthread_mutex_lock(&J->mu);
  for (int i = 0; i < 3; ++i) J->stats[i] += st[i];
  pthread_mutex_unlock(&J->mu);
  return NULL;
}

/* Common set-up of a threaded run over the requested rows; returns 0 or an
 * error code (invalid step, cap or row). */
static int job_begin(job_t* J, geom_t* G, const orc_grid* g, const orc_coeffs* cf,
                     const orc_run* run, const int32_t* rows, int32_t nrows) {
  if (!(run->dt > 0) || run->k_max < 1) return -1;
  /* the tabulated set reads both tables at every step */
  if (cf->id == ORC_COEF_TABLE &&
      (!cf->sigma_tab || !cf->c_tab || cf->tab_nx < 2 || cf->tab_ny < 2))
    return -1;
  if (geom_build(g, G, 1)) return -1;
  for (int r = 0; r < nrows; ++r)
    if (rows[r] < 0 || rows[r] >= G->n) { geom_free(G); return -2; }
  if (run->h_per_knot)
    for (int r = 0; r < nrows; ++r)
      if (!(run->h_per_knot[rows[r]] > 0)) { geom_free(G); return -1; }
  memset(J, 0, sizeof(*J));
  J->S.G = G; J->S.cf = cf; J->S.dt = run->dt; J->S.h_per_knot = run->h_per_knot;
  J->S.key[0] = (uint32_t)run->seed; J->S.key[1] = (uint32_t)(run->seed >> 32);
  J->S.tag = run->tag_word; J->S.k_max = run->k_max;
  J->S.interp = run->interp;
  J->S.rbf_c = run->rbf_c;
  J->S.rbf[0] = J->S.rbf[1] = NULL;
  if (run->interp == ORC_INTERP_RBF) {
    if (!(run->rbf_c > 0) || 2 * g->m + 1 + 2 * g->ext > ORC_MAX_STENCIL) {
      geom_free(G);
      return -1;
    }
    for (int o = 0; o < 2; ++o) {
      J->S.rbf[o] = (rbf_cache_t*)calloc(1, sizeof(rbf_cache_t));
      J->S.rbf[o]->c_lat = run->rbf_c / (o == 0 ? G->dx : G->dy);
      pthread_mutex_init(&J->S.rbf[o]->mu, NULL);
    }
  } else if (run->interp != ORC_INTERP_LINEAR) {
    geom_free(G);
    return -1;
  }
  J->scheme = run->scheme;
  J->n_per_knot = run->n_per_knot; J->n_paths = run->n_paths;
  J->rows = rows; J->nrows = nrows;
  return 0;
}

static int64_t* record_offsets(const job_t* J) {
  int64_t* off = (int64_t*)malloc((size_t)(J->nrows + 1) * sizeof(int64_t));
  off[0] = 0;
  for (int r = 0; r < J->nrows; ++r) off[r + 1] = off[r] + paths_of(J, J->rows[r]);
  return off;
}

static void job_run(job_t* J, int32_t threads, int64_t* stats) {
  pthread_mutex_init(&J->mu, NULL);
  if (threads < 1) threads = 1;
  pthread_t* th = (pthread_t*)malloc((size_t)threads * sizeof(pthread_t));
  for (int t = 0; t < threads; ++t) pthread_create(&th[t], NULL, worker, J);
  for (int t = 0; t < threads; ++t) pthread_join(th[t], NULL);
  free(th);
  pthread_mutex_destroy(&J->mu);
  if (stats) for (int i = 0; i < 3; ++i) stats[i] += J->stats[i];
}

int orc_assemble_ex(const orc_grid* g, const orc_coeffs* cf, const orc_run* run,
                    const int32_t* rows, int32_t nrows, int32_t threads,
                    double* val, double* b, orc_record* records, int64_t* stats) {
  if (run->scheme != ORC_SCHEME_EM && run->scheme != ORC_SCHEME_GM) return -1;
  geom_t G;
  job_t J;
  int rc = job_begin(&J, &G, g, cf, run, rows, nrows);
  if (rc) return rc;
  J.row_fn = assemble_row;
  J.val = val; J.b = b; J.records = records;
  int64_t* off = records ? record_offsets(&J) : NULL;
  J.rec_off = off;
  job_run(&J, threads, stats);
  free(off);
  rbf_cache_free(J.S.rbf[0]);
  rbf_cache_free(J.S.rbf[1]);
  geom_free(&G);
  return 0;
}

int orc_assemble(const orc_grid* g, const orc_coeffs* cf,
                 const int64_t* n_per_knot, int64_t n_paths,
                 double dt, uint64_t seed, uint32_t tag_word, int64_t k_max,
                 const int32_t* rows, int32_t nrows, int32_t threads,
                 double* val, double* b, orc_record* records, int64_t* stats) {
  orc_run run;
  memset(&run, 0, sizeof(run));
  run.n_per_knot = n_per_knot; run.n_paths = n_paths; run.dt = dt; run.h_per_knot = NULL;
  run.scheme = ORC_SCHEME_EM; run.tag_word = tag_word; run.seed = seed; run.k_max = k_max;
  return orc_assemble_ex(g, cf, &run, rows, nrows, threads, val, b, records, stats);
}

/* ========================================================================= *
 * Calibration (Sec. 4.1, Phase II): N'_0 mixed GM/EM paths per knot with the  *
 * warm-up solution u0 as Dirichlet data on the patch boundary.  A score is    *
 * phi = Y u0(P) + Z, where u0(P) is the stencil interpolation of the nodal    *
 * u0 on an interface side (the same weights as row k of G) or g on the        *
 * boundary of Omega; xi (Eq. 37) is kept apart.  Per knot the moments         *
 *   [N, sum d, sum d^2, sum phi_GM, sum phi_GM^2, sum xi, sum xi^2,           *
 *    sum phi_GM xi],  d = phi_EM - phi_GM,                                    *
 * are summed in ascending path order (xi is taken at the GM exit).            *
 * ========================================================================= */
static double score_of(const path_out_t* o, const double* u0) {
  double phi = o->bsum - o->xi;
  for (int q = 0; q < o->nw; ++q)
    if (o->col[q] >= 0) phi += o->w[q] * u0[o->col[q]];
  return phi;
}

static void calibrate_row(job_t* J, int r, int64_t* st) {
  int k = J->rows[r];
  int64_t N = paths_of(J, k);
  double m[ORC_CAL_NMOM];
  for (int i = 0; i < ORC_CAL_NMOM; ++i) m[i] = 0.0;
  for (int64_t p = 0; p < N; ++p) {
    path_out_t em, gm;
    simulate(&J->S, k, p, 3, &em, &gm);
    st[0] += em.steps;
    st[1] += (em.flags & 1) ? 1 : 0;
    st[2] += ((em.flags | gm.flags) & 2) ? 1 : 0;
    double pe = score_of(&em, J->u0), pg = score_of(&gm, J->u0), x = gm.xi;
    double d = pe - pg;
    m[0] += 1.0;
    m[1] += d;      m[2] += d * d;
    m[3] += pg;     m[4] += pg * pg;
    m[5] += x;      m[6] += x * x;
    m[7] += pg * x;
    if (J->cal_records) {
      orc_cal_record* R = &J->cal_records[J->rec_off[r] + p];
      R->steps_gm = gm.steps; R->side_gm = gm.side; R->flags_gm = gm.flags;
      R->steps_em = em.steps; R->side_em = em.side; R->flags_em = em.flags;
      R->phi_gm = pg; R->phi_em = pe; R->xi_gm = x; R->pad_ = 0.0;
    }
  }
  for (int i = 0; i < ORC_CAL_NMOM; ++i) J->moments[(size_t)r * ORC_CAL_NMOM + i] = m[i];
}

int orc_calibrate(const orc_grid* g, const orc_coeffs* cf, const orc_run* run, const double* u0,
                  const int32_t* rows, int32_t nrows, int32_t threads, double* moments,
                  orc_cal_record* records, int64_t* stats) {
  geom_t G;
  job_t J;
  int rc = job_begin(&J, &G, g, cf, run, rows, nrows);
  if (rc) return rc;
  J.row_fn = calibrate_row;
  J.u0 = u0; J.moments = moments; J.cal_records = records;
  int64_t* off = records ? record_offsets(&J) : NULL;
  J.rec_off = off;
  job_run(&J, threads, stats);
  free(off);
  rbf_cache_free(J.S.rbf[0]);
  rbf_cache_free(J.S.rbf[1]);
  geom_free(&G);
  return 0;
}

/* ========================================================================= *
 * Setting h_i and N_i from the calibration moments (Sec. 4.2).              *
 *  gap_i  = mean(phi_EM - phi_GM)            (Eq. 36; the GM bias at h'_0 is   *
 *                                             bounded by |gap_i| / 2, Eq. 35) *
 *  V_i    = sample variance of phi_GM,  rho_i^2 = corr(phi_GM, xi)^2 (Eq. 39) *
 *  h_i    = min(h_0, 2 h'_0 eps / (3 |gap_i|))                       (Eq. 40) *
 *  N_i    from (2/3) eps = 2 sqrt(V_i (1 - rho_i^2) / N_i), i.e.             *
 *           N_i = 9 V_i (1 - rho_i^2) / eps^2, rounded to the closest        *
 *           multiple k N_job with k >= 1                             (Eq. 41) *
 * diag[3i..3i+2] = gap_i, V_i, rho_i^2 (may be NULL).                        *
 * ========================================================================= */
void orc_plan(int64_t n, const double* mom, double eps, double h0, double h0p, int64_t n_job,
              double* h_out, int64_t* n_out, double* diag) {
  for (int64_t i = 0; i < n; ++i) {
    const double* m = mom + (size_t)i * ORC_CAL_NMOM;
    double N = m[0];
    double gap = N > 0 ? m[1] / N : 0.0;
    double var = 0.0, vx = 0.0, cov = 0.0;
    if (N > 1) {
      var = (m[4] - m[3] * m[3] / N) / (N - 1.0);
      vx = (m[6] - m[5] * m[5] / N) / (N - 1.0);
      cov = (m[7] - m[3] * m[5] / N) / (N - 1.0);
    }
    if (var < 0) var = 0;
    double rho2 = (var > 0 && vx > 0) ? cov * cov / (var * vx) : 0.0;
    if (rho2 > 1.0) rho2 = 1.0;
    double h = h0;
    if (gap != 0.0) {
      double hb = 2.0 * h0p * eps / (3.0 * fabs(gap));
      if (hb < h) h = hb;
    }
    double nraw = 9.0 * var * (1.0 - rho2) / (eps * eps);
    double k = nearbyint(nraw / (double)n_job);
    if (k < 1.0) k = 1.0;
    h_out[i] = h;
    n_out[i] = (int64_t)k * n_job;
    if (diag) { diag[3 * i] = gap; diag[3 * i + 1] = var; diag[3 * i + 2] = rho2; }
  }
}

void orc_finalize_rows(const orc_grid* g, const int64_t* row_ptr, const int32_t* col,
                       const int64_t* n_per_knot, int64_t n_paths,
                       const int32_t* rows, int32_t nrows, double* val, double* b) {
  (void)g;
  for (int r = 0; r < nrows; ++r) {
    int k = rows[r];
    double N = (double)(n_per_knot ? n_per_knot[k] : n_paths);
    for (int64_t q = row_ptr[k]; q < row_ptr[k + 1]; ++q)
      val[q] = (col[q] == k) ? 1.0 : -val[q] / N;       /* Eq. 24 */
    b[k] = b[k] / N;                                     /* Eq. 25 */
  }
}

/* ========================================================================= *
 * Linear solves for Eq. 23.                                                   *
 * ========================================================================= */
int orc_lu_solve(int64_t n, const double* A_in, const double* b, double* x) {
  /* Gaussian elimination with partial pivoting on a copy. */
  double* A = (double*)malloc((size_t)(n * n) * sizeof(double));
  double* r = (double*)malloc((size_t)n * sizeof(double));
  memcpy(A, A_in, (size_t)(n * n) * sizeof(double));
  memcpy(r, b, (size_t)n * sizeof(double));
  int rc = 0;
  for (int64_t c = 0; c < n; ++c) {
    int64_t piv = c;
    for (int64_t i = c + 1; i < n; ++i)
      if (fabs(A[i * n + c]) > fabs(A[piv * n + c])) piv = i;
    if (A[piv * n + c] == 0.0) { rc = -1; break; }
    if (piv != c) {
      for (int64_t j = 0; j < n; ++j) { double t = A[c * n + j]; A[c * n + j] = A[piv * n + j]; A[piv * n + j] = t; }
      double t = r[c]; r[c] = r[piv]; r[piv] = t;
    }
    for (int64_t i = c + 1; i < n; ++i) {
      double l = A[i * n + c] / A[c * n + c];
      if (l == 0.0) continue;
      for (int64_t j = c; j < n; ++j) A[i * n + j] -= l * A[c * n + j];
      r[i] -= l * r[c];
    }
  }
  if (rc == 0)
    for (int64_t i = n - 1; i >= 0; --i) {
      double s = r[i];
      for (int64_t j = i + 1; j < n; ++j) s -= A[i * n + j] * x[j];
      x[i] = s / A[i * n + i];
    }
  free(A); free(r);
  return rc;
}

static void spmv(int64_t n, const int64_t* rp, const int32_t* ci, const double* v,
                 const double* x, double* y) {
  for (int64_t i = 0; i < n; ++i) {
    double s = 0;
    for (int64_t q = rp[i]; q < rp[i + 1]; ++q) s += v[q] * x[ci[q]];
    y[i] = s;
  }
}
static double dot(int64_t n, const double* a, const double* b) {
  double s = 0;
  for (int64_t i = 0; i < n; ++i) s += a[i] * b[i];
  return s;
}

/* BiCGSTAB (van der Vorst 1992), x0 = 0, stop at ||r|| <= rtol ||b||. */
int orc_bicgstab(int64_t n, const int64_t* rp, const int32_t* ci, const double* val,
                 const double* b, double* x, double rtol, int32_t maxit, int32_t* iters,
                 double* relres) {
  double *r = calloc(n, 8), *rh = calloc(n, 8), *p = calloc(n, 8), *v = calloc(n, 8),
         *s = calloc(n, 8), *t = calloc(n, 8);
  for (int64_t i = 0; i < n; ++i) { x[i] = 0; r[i] = b[i]; rh[i] = b[i]; }
  double bn = sqrt(dot(n, b, b));
  if (bn == 0) bn = 1;
  double rho = 1, alpha = 1, omega = 1;
  int it = 0, rc = -1;
  double res = sqrt(dot(n, r, r)) / bn;
  if (res <= rtol) rc = 0;
  while (rc != 0 && it < maxit) {
    ++it;
    double rho1 = dot(n, rh, r);
    if (rho1 == 0) break;
    double beta = (rho1 / rho) * (alpha / omega);
    for (int64_t i = 0; i < n; ++i) p[i] = r[i] + beta * (p[i] - omega * v[i]);
    spmv(n, rp, ci, val, p, v);
    alpha = rho1 / dot(n, rh, v);
    for (int64_t i = 0; i < n; ++i) s[i] = r[i] - alpha * v[i];
    double sn = sqrt(dot(n, s, s)) / bn;
    if (sn <= rtol) {
      for (int64_t i = 0; i < n; ++i) x[i] += alpha * p[i];
      res = sn; rc = 0; break;
    }
    spmv(n, rp, ci, val, s, t);
    omega = dot(n, t, s) / dot(n, t, t);
    for (int64_t i = 0; i < n; ++i) { x[i] += alpha * p[i] + omega * s[i]; r[i] = s[i] - omega * t[i]; }
    rho = rho1;
    res = sqrt(dot(n, r, r)) / bn;
    if (res <= rtol) rc = 0;
  }
  if (iters) *iters = it;
  if (relres) *relres = res;
  free(r); free(rh); free(p); free(v); free(s); free(t);
  return rc;
}
