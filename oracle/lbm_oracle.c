/*
 * lbm_oracle.c -- TEST INFRASTRUCTURE, NOT THE PRODUCT.
 *
 * A plain, slow, double-precision CPU restatement of the coupled lattice
 * Boltzmann (LB) step of Xiong, Wang & Liu, "Local volume-conserving lattice
 * Boltzmann model for incompressible multiphase flows" (arXiv 2505.10899):
 * the hydrodynamic MRT-LB of Sec. 3.1 (Eqs. 20-29) coupled to the
 * interface-capturing MRT-LB of Sec. 3.2 (Eqs. 30-37) for the modified,
 * volume-conserving Cahn-Hilliard equation (Eq. 17).
 *
 * Only the test-suite, the smoke check and the CPU-baseline leg of the
 * benchmark may load this file.  It shares no code with the CUDA library.
 *
 * Style: every quantity is formed exactly as the paper writes it -- the
 * equilibria and sources in velocity space (Eqs. 21-23, 31-32), the
 * collision in moment space with the literal 9x9 matrix of Eq. 24 and its
 * Gauss-Jordan inverse (Eqs. 25, 33), the isotropic stencils as the
 * weighted sums of Sec. 3.2, the level-set variable and the sharpening
 * factor through log and tanh (Eqs. 32, 37).  No blocking, no fusion, no
 * algebraic shortcut.  Lattice units: dt = dx = 1.
 *
 * State convention: f, g hold the distributions f_i(x,t), g_i(x,t) *after*
 * streaming, i.e. the left-hand sides of Eqs. 20 and 30 at time t; jprev
 * holds phi*u at t-1 for the backward difference of d_t(phi u) (Sec. 3.2).
 * Arrays are [component][y][x] with x fastest; the grid is periodic in x,
 * and in y either periodic or closed by walls (walls = 1).
 *
 * Readings where the paper is silent (listed with reasons in the design
 * notes of the repository):
 *   - unspecified MRT rates are taken from the caller (default 1);
 *     s7^f = s8^f = 1/tau_f (Eq. 27) and s3^g = s5^g = 1/tau_g (Eq. 34)
 *     always overwrite the caller's entries;
 *   - rho(phi) and mu(phi) are linear in the unclipped phi, and
 *     tau_f(x) = mu/(rho c_s^2) + 1/2 from Eq. 27;
 *   - F in Eqs. 21 and 28 is the surface force hbar*grad(phi) (Eq. 18);
 *   - n = grad(psi)/|grad(psi)| where |grad(psi)| >= 0.1, else 0 (psi of
 *     Eq. 14, a signed distance with |grad(psi)| = 1 on the equilibrium
 *     profile): |grad(psi)| < 0.1 only on ridges of psi (droplet centres,
 *     thread axes, mid-planes of necks) and in the clipped bulk, where a
 *     unit vector would take its direction from rounding;
 *   - the backward difference starts from phi0*u0 (d_t(phi u) = 0 at t=0);
 *   - prescribed single-vortex velocity: u = -U sin^2(pi X) sin(2 pi Y)
 *     cos(pi t/T), v = U sin^2(pi Y) sin(2 pi X) cos(pi t/T) with node-centred
 *     X = (x+1/2)/nx, Y = (y+1/2)/ny and t the step index (Eqs. 43-44 with
 *     the sign of the benchmark configuration; U < 0 gives the paper's sign);
 *   - walls (the shear-flow set-up of Sec. 4.4; the paper gives no boundary
 *     scheme): halfway bounce-back below y = 0 and above y = ny - 1; f gains
 *     the moving-wall term 2 w_i rho (c_i . u_w)/c_s^2 with rho = rho(phi) of
 *     the receiving node after streaming; g bounces back without a term (no
 *     flux of phi through a wall); the stencils see a ghost row that mirrors
 *     the wall row (zero normal gradient: neutral wetting, 90 degrees).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* |grad(psi)| below which n of Eq. 17 is 0 (see the header). */
#define NORMAL_MIN 0.1

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* ORC_PLANT (1-10, 21-22, 24-27) selects a deliberately wrong variant of one formula, for the
 * mutation test that shows the pins catch it (0 = the oracle as written). */
#ifndef ORC_PLANT
#define ORC_PLANT 0
#endif

/* ---- D2Q9 lattice, Eq. 19 evaluated (c = 1), and its weights ---------- */
static const int CX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int CY[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
static const double WT[9] = {4.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0,
                             1.0 / 9.0,  1.0 / 9.0,  1.0 / 36.0,
                             1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};
static const double CS2 = 1.0 / 3.0; /* c_s^2 = c^2/3 */

/* ---- Transformation matrix M, Eq. 24 (also used for g, Sec. 3.2) ------ */
static const double MM[9][9] = {
    {1, 1, 1, 1, 1, 1, 1, 1, 1},         {-4, -1, -1, -1, -1, 2, 2, 2, 2},
    {4, -2, -2, -2, -2, 1, 1, 1, 1},     {0, 1, 0, -1, 0, 1, -1, -1, 1},
    {0, -2, 0, 2, 0, 1, -1, -1, 1},      {0, 0, 1, 0, -1, 1, 1, -1, -1},
    {0, 0, -2, 0, 2, 1, 1, -1, -1},      {0, 1, -1, 1, -1, 0, 0, 0, 0},
    {0, 0, 0, 0, 0, 1, -1, 1, -1}};

static double MINV[9][9];
static int minv_ready = 0;

/* Gauss-Jordan elimination with partial pivoting on [M | I]. */
static void build_minv(void) {
  double a[9][18];
  for (int r = 0; r < 9; ++r)
    for (int c = 0; c < 18; ++c)
      a[r][c] = (c < 9) ? MM[r][c] : (c - 9 == r ? 1.0 : 0.0);
  for (int col = 0; col < 9; ++col) {
    int piv = col;
    for (int r = col + 1; r < 9; ++r)
      if (fabs(a[r][col]) > fabs(a[piv][col])) piv = r;
    if (piv != col)
      for (int c = 0; c < 18; ++c) {
        double t = a[col][c];
        a[col][c] = a[piv][c];
        a[piv][c] = t;
      }
    double d = a[col][col];
    for (int c = 0; c < 18; ++c) a[col][c] /= d;
    for (int r = 0; r < 9; ++r) {
      if (r == col) continue;
      double m = a[r][col];
      if (m == 0.0) continue;
      for (int c = 0; c < 18; ++c) a[r][c] -= m * a[col][c];
    }
  }
  for (int r = 0; r < 9; ++r)
    for (int c = 0; c < 9; ++c) MINV[r][c] = a[r][c + 9];
  minv_ready = 1;
}

/* ---- Parameters ---------------------------------------------------------- */
typedef struct {
  int32_t nx, ny;
  int32_t flow;  /* 0: coupled f-g step; 1: g only, prescribed single vortex */
  int32_t walls; /* 0: periodic in y; 1: walls below y = 0 and above y = ny-1 */
  double W;      /* interface width */
  double sigma;  /* surface tension (gamma in Sec. 2) */
  double lambda; /* penalty constant, Eq. 6; 0 gives the classical model */
  double xi;     /* regulariser of Eq. 37 */
  double tau_g;  /* phase-field relaxation time, Eq. 34 */
  double rho_l, rho_g;     /* densities of the phi=1 and phi=0 fluids */
  double tau_f_l, tau_f_g; /* f relaxation times in the two bulks, Eq. 27 */
  double s_f[9], s_g[9];   /* MRT rates, Eq. 26; tied entries overwritten */
  double vortex_U, vortex_T;
  double u_top, u_bot; /* wall velocities along x (walls = 1) */
} orc_params;

void orc_lattice(int32_t *cx, int32_t *cy, double *w) {
  for (int i = 0; i < 9; ++i) {
    cx[i] = CX[i];
    cy[i] = CY[i];
    w[i] = WT[i];
  }
}

void orc_matrices(double *m, double *minv) {
  if (!minv_ready) build_minv();
  for (int r = 0; r < 9; ++r)
    for (int c = 0; c < 9; ++c) {
      m[r * 9 + c] = MM[r][c];
      minv[r * 9 + c] = MINV[r][c];
    }
}

/* ---- Per-node formulas ---------------------------------------------------- */

/* Eq. 23 */
static double s_u(int i, double ux, double uy) {
  double cu = CX[i] * ux + CY[i] * uy;
  double uu = ux * ux + uy * uy;
  return WT[i] * (cu / CS2 + cu * cu / (2.0 * CS2 * CS2) - uu / (2.0 * CS2));
}

/* Eq. 22: incompressible, pressure-based equilibrium of f. */
void orc_feq(double p, double rho, double ux, double uy, double *out) {
  for (int i = 0; i < 9; ++i) {
    double wp = (i == 0) ? (WT[0] - 1.0) : WT[i];
    out[i] = wp * p / CS2 + rho * s_u(i, ux, uy);
  }
}

/* Eq. 21: discrete forcing term; gr = grad(rho), (Fx,Fy) = total force. */
void orc_force(double ux, double uy, double Fx, double Fy, double grx,
               double gry, double *out) {
  double u[2] = {ux, uy}, gr[2] = {grx, gry};
  for (int i = 0; i < 9; ++i) {
    double c[2] = {(double)CX[i], (double)CY[i]};
    double u_gr = ux * grx + uy * gry; /* not const: see ORC_PLANT 1 */
    double c_F = c[0] * Fx + c[1] * Fy;
    double tens = 0.0; /* (u grad rho) : (c_i c_i - c_s^2 I) */
    for (int a = 0; a < 2; ++a)
      for (int b = 0; b < 2; ++b)
        tens += u[a] * gr[b] * (c[a] * c[b] - CS2 * (a == b ? 1.0 : 0.0));
#if ORC_PLANT == 1
    u_gr = 0.0;
#endif
    out[i] = WT[i] * (u_gr + c_F / CS2 + tens / CS2);
  }
}

/* Eq. 31: equilibrium of g; mu is the chemical potential hbar of Eq. 2. */
void orc_geq(double phi, double mu, double lambda, double ux, double uy,
             double *out) {
  double lam = mu + lambda * phi;
#if ORC_PLANT == 3
  out[0] = phi + WT[0] * lam;
#else
  out[0] = phi + (WT[0] - 1.0) * lam;
#endif
  for (int i = 1; i < 9; ++i)
    out[i] = WT[i] * lam + WT[i] * (CX[i] * phi * ux + CY[i] * phi * uy) / CS2;
}

/* Eq. 32: source of the phase-field LB; (dJx,dJy) = d_t(phi u),
 * (nx_,ny_) = grad(psi)/|grad(psi)|. */
void orc_gsrc(double dJx, double dJy, double lambda, double W, double psi,
              double nx_, double ny_, double *out) { /* arguments reassigned by ORC_PLANT 6 */
  double th = tanh(2.0 * psi / W);
#if ORC_PLANT == 10
  double sharp = -(lambda / W) * (1.0 - th * th);
#else
  double sharp = (lambda / W) * (1.0 - th * th);
#endif
#if ORC_PLANT == 6
  dJx = dJy = 0.0;
#endif
  double vx = dJx / CS2 + sharp * nx_;
  double vy = dJy / CS2 + sharp * ny_;
  for (int i = 0; i < 9; ++i) out[i] = WT[i] * (CX[i] * vx + CY[i] * vy);
}

/* Eq. 37 with the clip of phi to [0,1] stated after it. */
double orc_psi(double phi, double W, double xi) {
#if ORC_PLANT == 8
  double pc = phi;
#else
  double pc = phi < 0.0 ? 0.0 : (phi > 1.0 ? 1.0 : phi);
#endif
  return 0.25 * W * log((pc + xi) / (1.0 - pc + xi));
}

/* Eq. 2 */
double orc_chem(double phi, double lap_phi, double W, double sigma) {
#if ORC_PLANT == 7
  double beta = 12.0 * sigma / W, kappa = 3.0 * sigma * W;
#else
  double beta = 12.0 * sigma / W, kappa = 1.5 * sigma * W; /* Sec. 2 */
#endif
  return 4.0 * beta * phi * (phi - 1.0) * (phi - 0.5) - kappa * lap_phi;
}

/* Eqs. 25 / 33: m* = m - S(m - m_eq) + (I - S/2) Mbar_F, back with M^-1. */
void orc_mrt(const double *f, const double *feq, const double *F,
             const double *s, double *out) {
  if (!minv_ready) build_minv();
  double m[9], meq[9], mF[9], ms[9];
  for (int k = 0; k < 9; ++k) {
    m[k] = meq[k] = mF[k] = 0.0;
    for (int j = 0; j < 9; ++j) {
#if ORC_PLANT == 4
      m[k] += MM[j][k] * f[j];
#else
      m[k] += MM[k][j] * f[j];
#endif
      meq[k] += MM[k][j] * feq[j];
      mF[k] += MM[k][j] * F[j];
    }
  }
  for (int k = 0; k < 9; ++k)
    ms[k] = m[k] - s[k] * (m[k] - meq[k]) + (1.0 - 0.5 * s[k]) * mF[k];
  for (int i = 0; i < 9; ++i) {
    out[i] = 0.0;
    for (int k = 0; k < 9; ++k) out[i] += MINV[i][k] * ms[k];
  }
}

/* Isotropic gradient and Laplacian of Sec. 3.2 (Thampi et al.), periodic in
 * x; in y periodic, or with walls a ghost row that mirrors the wall row
 * (chi(x, -1) = chi(x, 0), chi(x, ny) = chi(x, ny-1): zero normal gradient). */
static void stencil_w(const double *chi, int nx, int ny, int walls, int x, int y,
                      double *gx, double *gy, double *lap) {
  double c0 = chi[(size_t)y * nx + x];
  double sx = 0.0, sy = 0.0, sl = 0.0;
  for (int i = 1; i < 9; ++i) {
    int xn = ((x + CX[i]) % nx + nx) % nx;
    int yn = y + CY[i];
#if ORC_PLANT == 22
    if (0)
#else
    if (walls)
#endif
      yn = yn < 0 ? 0 : (yn >= ny ? ny - 1 : yn);
    else
      yn = (yn % ny + ny) % ny;
    double v = chi[(size_t)yn * nx + xn];
    sx += WT[i] * CX[i] * v / CS2;
#if ORC_PLANT == 2
    sy -= WT[i] * CY[i] * v / CS2;
#else
    sy += WT[i] * CY[i] * v / CS2;
#endif
    sl += 2.0 * WT[i] * (v - c0) / CS2;
  }
  if (gx) *gx = sx;
  if (gy) *gy = sy;
  if (lap) *lap = sl;
}

static void stencil(const double *chi, int nx, int ny, int x, int y, double *gx,
                    double *gy, double *lap) {
  stencil_w(chi, nx, ny, 0, x, y, gx, gy, lap);
}

void orc_stencil(const double *chi, int32_t nx, int32_t ny, double *gx,
                 double *gy, double *lap) {
  for (int y = 0; y < ny; ++y)
    for (int x = 0; x < nx; ++x) {
      size_t k = (size_t)y * nx + x;
      stencil(chi, nx, ny, x, y, gx + k, gy + k, lap + k);
    }
}

/* Prescribed single-vortex velocity (Eqs. 43-44, reading in the header). */
static void vortex_u(const orc_params *p, int x, int y, int64_t t, double *ux,
                     double *uy) {
#if ORC_PLANT == 26
  double X = (double)x / p->nx, Y = (double)y / p->ny;
#elif ORC_PLANT == 25
  double Y = (x + 0.5) / p->nx, X = (y + 0.5) / p->ny;
#else
  double X = (x + 0.5) / p->nx, Y = (y + 0.5) / p->ny;
#endif
#if ORC_PLANT == 24
  double ct = cos(2.0 * M_PI * (double)t / p->vortex_T);
#else
  double ct = cos(M_PI * (double)t / p->vortex_T);
#endif
  double sx = sin(M_PI * X), sy = sin(M_PI * Y);
#if ORC_PLANT == 27
  *ux = -p->vortex_U * sx * sin(2.0 * M_PI * Y) * ct;
#else
  *ux = -p->vortex_U * sx * sx * sin(2.0 * M_PI * Y) * ct;
#endif
  *uy = p->vortex_U * sy * sy * sin(2.0 * M_PI * X) * ct;
}

/* Linear rho(phi), mu(phi) (reading) and tau_f from Eq. 27. */
static double rho_of(const orc_params *p, double phi) {
  return p->rho_g + phi * (p->rho_l - p->rho_g);
}
static double tau_f_of(const orc_params *p, double phi) {
  double mu_l = p->rho_l * CS2 * (p->tau_f_l - 0.5);
  double mu_g = p->rho_g * CS2 * (p->tau_f_g - 0.5);
  double mu = mu_g + phi * (mu_l - mu_g);
  return mu / (rho_of(p, phi) * CS2) + 0.5;
}

/* ---- Macroscopic fields of a post-streaming state (Eqs. 2, 28-29, 35-37) */
typedef struct {
  double *phi, *psi;               /* Eq. 35, Eq. 37 */
  double *gpx, *gpy, *lap;         /* grad phi, lap phi */
  double *gsx, *gsy;               /* grad psi */
} work_t;

static int work_alloc(work_t *w, size_t n) {
  double *base = (double *)malloc(sizeof(double) * n * 7);
  if (!base) return -1;
  w->phi = base;
  w->psi = base + n;
  w->gpx = base + 2 * n;
  w->gpy = base + 3 * n;
  w->lap = base + 4 * n;
  w->gsx = base + 5 * n;
  w->gsy = base + 6 * n;
  return 0;
}

static void phase_fields(const orc_params *p, const double *g, work_t *w) {
  int nx = p->nx, ny = p->ny;
  size_t n = (size_t)nx * ny;
  for (size_t k = 0; k < n; ++k) {
    double s = 0.0;
    for (int i = 0; i < 9; ++i) s += g[i * n + k]; /* Eq. 35 */
    w->phi[k] = s;
    w->psi[k] = orc_psi(s, p->W, p->xi); /* Eq. 37 */
  }
#pragma omp parallel for schedule(static)
  for (int y = 0; y < ny; ++y)
    for (int x = 0; x < nx; ++x) {
      size_t k = (size_t)y * nx + x;
      stencil_w(w->phi, nx, ny, p->walls, x, y, w->gpx + k, w->gpy + k, w->lap + k);
      stencil_w(w->psi, nx, ny, p->walls, x, y, w->gsx + k, w->gsy + k, NULL);
    }
}

/* Hydrodynamic macroscopics at one node: Eqs. 2, 18 (F = hbar grad phi),
 * 28 and 29.  Returns hbar; fills u, p, rho, grad rho, F. */
typedef struct {
  double mu, rho, grx, gry, Fx, Fy, ux, uy, p;
} node_macro;

static void node_macros(const orc_params *p, const double *f, size_t n,
                        size_t k, const work_t *w, int64_t t, int x, int y,
                        node_macro *o) {
  double phi = w->phi[k];
  o->mu = orc_chem(phi, w->lap[k], p->W, p->sigma);
  o->Fx = o->mu * w->gpx[k];
  o->Fy = o->mu * w->gpy[k];
  o->rho = rho_of(p, phi);
  o->grx = (p->rho_l - p->rho_g) * w->gpx[k];
  o->gry = (p->rho_l - p->rho_g) * w->gpy[k];
  if (p->flow == 0) {
    double jx = 0.0, jy = 0.0, sum_nz = 0.0;
    for (int i = 0; i < 9; ++i) {
      jx += CX[i] * f[i * n + k];
      jy += CY[i] * f[i * n + k];
      if (i != 0) sum_nz += f[i * n + k];
    }
#if ORC_PLANT == 5
    o->ux = (jx + o->Fx) / o->rho;
    o->uy = (jy + o->Fy) / o->rho;
#else
    o->ux = (jx + 0.5 * o->Fx) / o->rho; /* Eq. 28 */
    o->uy = (jy + 0.5 * o->Fy) / o->rho;
#endif
    double u_gr = o->ux * o->grx + o->uy * o->gry;
#if ORC_PLANT == 9
    o->p = CS2 / (1.0 - WT[0]) * (sum_nz + 0.5 * u_gr);
#else
    o->p = CS2 / (1.0 - WT[0]) *
           (sum_nz + 0.5 * u_gr + o->rho * s_u(0, o->ux, o->uy)); /* Eq. 29 */
#endif
  } else {
    vortex_u(p, x, y, t, &o->ux, &o->uy);
    o->p = 0.0;
  }
}

static void fill_rates(const orc_params *p, double phi, double *sf, double *sg) {
  for (int k = 0; k < 9; ++k) {
    sf[k] = p->s_f[k];
    sg[k] = p->s_g[k];
  }
  sf[7] = sf[8] = 1.0 / tau_f_of(p, phi); /* Eq. 27 */
  sg[3] = sg[5] = 1.0 / p->tau_g;         /* Eq. 34 */
}

/* ---- Public entry points --------------------------------------------------
 * All return 0 on success, -1 on bad arguments, -2 on allocation failure.   */

static int check_params(const orc_params *p) {
  if (!p || p->nx < 1 || p->ny < 1) return -1;
  if (p->flow != 0 && p->flow != 1) return -1;
  if (!(p->W > 0.0) || !(p->tau_g > 0.5)) return -1;
  if (p->flow == 0 && (!(p->rho_l > 0.0) || !(p->rho_g > 0.0) ||
                       !(p->tau_f_l > 0.5) || !(p->tau_f_g > 0.5)))
    return -1;
  if (p->flow == 1 && !(p->vortex_T != 0.0)) return -1;
  if (p->walls != 0 && (p->walls != 1 || p->flow != 0)) return -1;
  return 0;
}

/* Initial state (Sec. 4 set-ups: tanh profiles, velocity given, p = 0):
 * hbar0 from Eq. 2 on phi0, g = g_eq(phi0, hbar0, u0) (Eq. 31),
 * f = f_eq(p=0, rho(phi0), u0) (Eq. 22), jprev = phi0 u0.
 * u0 may be NULL (fluid at rest); in vortex mode u0 is ignored and the
 * prescribed velocity at t = 0 is used. */
int orc_init(const orc_params *p, const double *phi0, const double *u0,
             double *f, double *g, double *jprev) {
  if (check_params(p) || !phi0 || !g || !jprev || (p->flow == 0 && !f))
    return -1;
  int nx = p->nx, ny = p->ny;
  size_t n = (size_t)nx * ny;
  double *lap = (double *)malloc(sizeof(double) * n);
  if (!lap) return -2;
  for (int y = 0; y < ny; ++y)
    for (int x = 0; x < nx; ++x)
      stencil_w(phi0, nx, ny, p->walls, x, y, NULL, NULL, lap + (size_t)y * nx + x);
  for (int y = 0; y < ny; ++y)
    for (int x = 0; x < nx; ++x) {
      size_t k = (size_t)y * nx + x;
      double ux = 0.0, uy = 0.0;
      if (p->flow == 1) {
        vortex_u(p, x, y, 0, &ux, &uy);
      } else if (u0) {
        ux = u0[k];
        uy = u0[n + k];
      }
      double mu = orc_chem(phi0[k], lap[k], p->W, p->sigma);
      double ge[9], fe[9];
      orc_geq(phi0[k], mu, p->lambda, ux, uy, ge);
      for (int i = 0; i < 9; ++i) g[i * n + k] = ge[i];
      if (p->flow == 0) {
        orc_feq(0.0, rho_of(p, phi0[k]), ux, uy, fe);
        for (int i = 0; i < 9; ++i) f[i * n + k] = fe[i];
      }
      jprev[k] = phi0[k] * ux;
      jprev[n + k] = phi0[k] * uy;
    }
  free(lap);
  return 0;
}

/* Opposite directions of Eq. 19. */
static const int OPP[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};

/* Moving-wall term of the halfway bounce-back for f: a population returning
 * from a wall moving at u_w along x gains 2 w_i rho_w (c_i . u_w) / c_s^2,
 * with rho_w = rho(phi) of the receiving wall node after streaming (phi from
 * its g, which bounce back without a term: no flux of phi through a wall). */
static void wall_momentum(const orc_params *p, double *f, const double *g) {
  int nx = p->nx, ny = p->ny;
  size_t n = (size_t)nx * ny;
  for (int side = 0; side < 2; ++side) {
    int y = side == 0 ? 0 : ny - 1;
    int cy_in = side == 0 ? 1 : -1; /* directions entering from the wall */
    double uw = side == 0 ? p->u_bot : p->u_top;
    for (int x = 0; x < nx; ++x) {
      size_t k = (size_t)y * nx + x;
      double phi = 0.0;
      for (int i = 0; i < 9; ++i) phi += g[i * n + k];
      double rho = rho_of(p, phi);
      for (int i = 0; i < 9; ++i)
#if ORC_PLANT == 21
        if (CY[i] == cy_in) f[i * n + k] -= 2.0 * WT[i] * rho * (CX[i] * uw) / CS2;
#else
        if (CY[i] == cy_in) f[i * n + k] += 2.0 * WT[i] * rho * (CX[i] * uw) / CS2;
#endif
    }
  }
}

/* One collision at one node, given its macroscopic context. */
static void collide_node(const orc_params *p, const double *f, const double *g,
                         const double *jprev, size_t n, size_t k,
                         const work_t *w, const node_macro *m, double *fstar,
                         double *gstar, double *jnew) {
  double phi = w->phi[k];
  double sf[9], sg[9];
  fill_rates(p, phi, sf, sg);

  if (p->flow == 0) {
    double fl[9], fe[9], Fi[9];
    for (int i = 0; i < 9; ++i) fl[i] = f[i * n + k];
    orc_feq(m->p, m->rho, m->ux, m->uy, fe);                      /* Eq. 22 */
    orc_force(m->ux, m->uy, m->Fx, m->Fy, m->grx, m->gry, Fi);    /* Eq. 21 */
    orc_mrt(fl, fe, Fi, sf, fstar);                               /* Eq. 25 */
  }

  double Jx = phi * m->ux, Jy = phi * m->uy;
  double dJx = Jx - jprev[k], dJy = Jy - jprev[n + k]; /* backward difference */
  double gsx = w->gsx[k], gsy = w->gsy[k];
  double nrm2 = gsx * gsx + gsy * gsy;
  double nx_ = 0.0, ny_ = 0.0;
  if (nrm2 >= NORMAL_MIN * NORMAL_MIN) {
    double nrm = sqrt(nrm2);
    nx_ = gsx / nrm;
    ny_ = gsy / nrm;
  }
  double gl[9], ge[9], Gi[9];
  for (int i = 0; i < 9; ++i) gl[i] = g[i * n + k];
  orc_geq(phi, m->mu, p->lambda, m->ux, m->uy, ge);                 /* Eq. 31 */
  orc_gsrc(dJx, dJy, p->lambda, p->W, w->psi[k], nx_, ny_, Gi);     /* Eq. 32 */
  orc_mrt(gl, ge, Gi, sg, gstar);                                   /* Eq. 33 */
  jnew[0] = Jx;
  jnew[1] = Jy;
}

/* Advance nsteps from time t0.  f, g, jprev are updated in place. */
int orc_step(const orc_params *p, double *f, double *g, double *jprev,
             int64_t t0, int64_t nsteps) {
  if (check_params(p) || !g || !jprev || (p->flow == 0 && !f) || nsteps < 0)
    return -1;
  int nx = p->nx, ny = p->ny;
  size_t n = (size_t)nx * ny;
  work_t w;
  if (work_alloc(&w, n)) return -2;
  double *fs = (double *)malloc(sizeof(double) * 9 * n);
  double *gs = (double *)malloc(sizeof(double) * 9 * n);
  if (!fs || !gs) {
    free(w.phi);
    free(fs);
    free(gs);
    return -2;
  }
  for (int64_t s = 0; s < nsteps; ++s) {
    int64_t t = t0 + s;
    phase_fields(p, g, &w);
#pragma omp parallel for schedule(static)
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nx; ++x) {
        size_t k = (size_t)y * nx + x;
        node_macro m;
        node_macros(p, f, n, k, &w, t, x, y, &m);
        double fst[9], gst[9], jn[2];
        collide_node(p, f, g, jprev, n, k, &w, &m, fst, gst, jn);
        for (int i = 0; i < 9; ++i) {
          if (p->flow == 0) fs[i * n + k] = fst[i];
          gs[i * n + k] = gst[i];
        }
        jprev[k] = jn[0];
        jprev[n + k] = jn[1];
      }
    /* Streaming, left-hand sides of Eqs. 20 and 30: value moves to x + c_i.
     * With walls, a value that would cross y = -1/2 or y = ny - 1/2 returns to
     * its node in the opposite direction (halfway bounce-back). */
    for (int i = 0; i < 9; ++i)
      for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
          int xd = ((x + CX[i]) % nx + nx) % nx;
          int yd = y + CY[i];
          size_t src = (size_t)i * n + (size_t)y * nx + x;
          size_t dst;
          if (p->walls && (yd < 0 || yd >= ny))
            dst = (size_t)OPP[i] * n + (size_t)y * nx + x;
          else
            dst = (size_t)i * n + (size_t)((yd % ny + ny) % ny) * nx + xd;
          if (p->flow == 0) f[dst] = fs[src];
          g[dst] = gs[src];
        }
    if (p->walls) wall_momentum(p, f, g);
  }
  free(w.phi);
  free(fs);
  free(gs);
  return 0;
}

/* Macroscopic fields phi, u, p of the state at time t (Eqs. 28-29, 35).
 * Any output pointer may be NULL. */
int orc_fields(const orc_params *p, const double *f, const double *g,
               int64_t t, double *phi, double *ux, double *uy, double *pr) {
  if (check_params(p) || !g || (p->flow == 0 && !f)) return -1;
  int nx = p->nx, ny = p->ny;
  size_t n = (size_t)nx * ny;
  work_t w;
  if (work_alloc(&w, n)) return -2;
  phase_fields(p, g, &w);
  for (int y = 0; y < ny; ++y)
    for (int x = 0; x < nx; ++x) {
      size_t k = (size_t)y * nx + x;
      node_macro m;
      node_macros(p, f, n, k, &w, t, x, y, &m);
      if (phi) phi[k] = w.phi[k];
      if (ux) ux[k] = m.ux;
      if (uy) uy[k] = m.uy;
      if (pr) pr[k] = m.p;
    }
  free(w.phi);
  return 0;
}

/* Collision products at every node of a post-streaming state, before
 * streaming: f*, g* and the new phi*u.  Used by the tests to check single
 * nodes.  fstar may be NULL in vortex mode. */
int orc_collide(const orc_params *p, const double *f, const double *g,
                const double *jprev, int64_t t, double *fstar, double *gstar,
                double *jnew) {
  if (check_params(p) || !g || !jprev || !gstar || !jnew ||
      (p->flow == 0 && (!f || !fstar)))
    return -1;
  int nx = p->nx, ny = p->ny;
  size_t n = (size_t)nx * ny;
  work_t w;
  if (work_alloc(&w, n)) return -2;
  phase_fields(p, g, &w);
  for (int y = 0; y < ny; ++y)
    for (int x = 0; x < nx; ++x) {
      size_t k = (size_t)y * nx + x;
      node_macro m;
      node_macros(p, f, n, k, &w, t, x, y, &m);
      double fst[9], gst[9], jn[2];
      collide_node(p, f, g, jprev, n, k, &w, &m, fst, gst, jn);
      for (int i = 0; i < 9; ++i) {
        if (p->flow == 0) fstar[i * n + k] = fst[i];
        gstar[i * n + k] = gst[i];
      }
      jnew[k] = jn[0];
      jnew[n + k] = jn[1];
    }
  free(w.phi);
  return 0;
}

/* Phase volumes V_r = sum of phi over the nodes labelled r (the droplet
 * volumes plotted in Fig. 3b), with Kahan summation in FP64.  labels may be
 * NULL (one region, the whole grid); label < 0 belongs to no region. */
int orc_volume(const orc_params *p, const double *g, const int8_t *labels,
               int32_t nregions, double *out) {
  if (!p || p->nx < 1 || p->ny < 1 || !g || !out || nregions < 1) return -1;
  size_t n = (size_t)p->nx * p->ny;
  double *sum = (double *)calloc((size_t)nregions, sizeof(double));
  double *cmp = (double *)calloc((size_t)nregions, sizeof(double));
  if (!sum || !cmp) {
    free(sum);
    free(cmp);
    return -2;
  }
  for (size_t k = 0; k < n; ++k) {
    int r = labels ? labels[k] : 0;
    if (r < 0 || r >= nregions) continue;
    double phi = 0.0;
    for (int i = 0; i < 9; ++i) phi += g[i * n + k];
    double yv = phi - cmp[r];
    double tv = sum[r] + yv;
    cmp[r] = (tv - sum[r]) - yv;
    sum[r] = tv;
  }
  for (int r = 0; r < nregions; ++r) out[r] = sum[r];
  free(sum);
  free(cmp);
  return 0;
}

int orc_num_threads(void) {
#ifdef _OPENMP
  extern int omp_get_max_threads(void);
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* Threads of the OpenMP loops over rows (the runtime is shared by every
 * oracle library in the process).  Each node is computed by one thread with
 * no reduction across nodes, so the results do not depend on the count. */
void orc_set_num_threads(int n) {
#ifdef _OPENMP
  extern void omp_set_num_threads(int);
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}
