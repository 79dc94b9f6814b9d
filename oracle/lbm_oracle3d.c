/*
 * lbm_oracle3d.c -- TEST INFRASTRUCTURE, NOT THE PRODUCT.
 *
 * FP64 CPU restatement of the three-dimensional extension of the coupled LB
 * step of Xiong, Wang & Liu (arXiv 2505.10899).  The paper is two-dimensional
 * (D2Q9, MRT); in three dimensions this follows its own statement that the
 * MRT model reduces to the single-relaxation-time model when all rates are
 * equal (Sec. 3.1, text after Eq. 26), written on the textbook lattices:
 *   - hydrodynamics: D3Q19, c_s^2 = 1/3, weights 1/3, 1/18 (6), 1/36 (12);
 *     f* = f - (f - f_eq)/tau_f + (1 - 1/(2 tau_f)) F_i            (Eq. 20)
 *     with f_eq of Eqs. 22-23, F_i of Eq. 21, u of Eq. 28 and p of Eq. 29
 *     (c_s^2/(1 - w_0) = 1/2);
 *   - phase field: D3Q7, c_s^2 = 1/4, weights 1/4, 1/8 (6);
 *     g* = g - (g - g_eq)/tau_g + (1 - 1/(2 tau_g)) G_i            (Eq. 30)
 *     with g_eq of Eq. 31 and G_i of Eq. 32 on that lattice, so that the
 *     mobility is M = (tau_g - 1/2)/4 (Eq. 34 with c_s^2 = 1/4);
 *   - the isotropic gradient and Laplacian of Sec. 3.2 with the D3Q19 set;
 *   - psi, its clip and xi as Eq. 37; phi = sum g (Eq. 35);
 *   - n = grad(psi)/|grad(psi)| where |grad(psi)| >= 0.1, else 0, as in the
 *     2-D oracle.
 * Only the test-suite, the smoke check and the CPU-baseline leg of the
 * benchmark may load this file.  It shares no code with the CUDA library.
 *
 * State: f [19][z][y][x], g [7][z][y][x] after streaming, jprev [3][z][y][x];
 * periodic in x, y and z.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* |grad(psi)| below which n of Eq. 17 is 0. */
#define NORMAL_MIN 0.1

/* ORC_PLANT (11-20, 23) selects a deliberately wrong variant of one formula, for
 * the mutation test of the pins only; 0 (the default) is the method. */
#ifndef ORC_PLANT
#define ORC_PLANT 0
#endif

/* D3Q19: rest, 6 axis, 12 face diagonals */
static const int C19[19][3] = {{0, 0, 0},  {1, 0, 0},   {-1, 0, 0}, {0, 1, 0},   {0, -1, 0},
                               {0, 0, 1},  {0, 0, -1},  {1, 1, 0},  {-1, -1, 0}, {1, -1, 0},
                               {-1, 1, 0}, {1, 0, 1},   {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
                               {0, 1, 1},  {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};
static double W19(int i) { return i == 0 ? 1.0 / 3.0 : (i < 7 ? 1.0 / 18.0 : 1.0 / 36.0); }
static const double CS2F = 1.0 / 3.0;

/* D3Q7: rest, 6 axis */
static const int C7[7][3] = {{0, 0, 0}, {1, 0, 0},  {-1, 0, 0}, {0, 1, 0},
                             {0, -1, 0}, {0, 0, 1}, {0, 0, -1}};
static double W7(int i) { return i == 0 ? 0.25 : 0.125; }
static const double CS2G = 0.25;

typedef struct {
  int32_t nx, ny, nz, pad_;
  double W, sigma, lambda, xi;
  double tau_g, rho_l, rho_g, tau_f_l, tau_f_g;
} orc3_params;

void orc3_lattices(int32_t *c19, double *w19, int32_t *c7, double *w7) {
  for (int i = 0; i < 19; ++i) {
    for (int a = 0; a < 3; ++a) c19[3 * i + a] = C19[i][a];
    w19[i] = W19(i);
  }
  for (int i = 0; i < 7; ++i) {
    for (int a = 0; a < 3; ++a) c7[3 * i + a] = C7[i][a];
    w7[i] = W7(i);
  }
}

static size_t idx(const orc3_params *p, int x, int y, int z) {
  x = ((x % p->nx) + p->nx) % p->nx;
  y = ((y % p->ny) + p->ny) % p->ny;
  z = ((z % p->nz) + p->nz) % p->nz;
  return ((size_t)z * p->ny + y) * p->nx + x;
}

/* Eqs. 22-23 on D3Q19 */
void orc3_feq(double pr, double rho, const double *u, double *out) {
  double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  for (int i = 0; i < 19; ++i) {
    double cu = C19[i][0] * u[0] + C19[i][1] * u[1] + C19[i][2] * u[2];
    double s = W19(i) * (cu / CS2F + cu * cu / (2 * CS2F * CS2F) - uu / (2 * CS2F));
    double wp = i == 0 ? W19(0) - 1.0 : W19(i);
    out[i] = wp * pr / CS2F + rho * s;
  }
}

/* Eq. 21 on D3Q19 */
void orc3_force(const double *u, const double *F, const double *gr, double *out) {
  double ugr = u[0] * gr[0] + u[1] * gr[1] + u[2] * gr[2];
  for (int i = 0; i < 19; ++i) {
    double cF = C19[i][0] * F[0] + C19[i][1] * F[1] + C19[i][2] * F[2];
    double tens = 0.0;
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b)
#if ORC_PLANT == 11
        tens += u[a] * gr[b] * (C19[i][a] * C19[i][b]);
#else
        tens += u[a] * gr[b] * (C19[i][a] * C19[i][b] - CS2F * (a == b ? 1.0 : 0.0));
#endif
    out[i] = W19(i) * (ugr + cF / CS2F + tens / CS2F);
  }
}

/* Eq. 31 on D3Q7 */
void orc3_geq(double phi, double mu, double lambda, const double *u, double *out) {
  double lam = mu + lambda * phi;
  out[0] = phi + (W7(0) - 1.0) * lam;
  for (int i = 1; i < 7; ++i) {
    double cJ = C7[i][0] * phi * u[0] + C7[i][1] * phi * u[1] + C7[i][2] * phi * u[2];
#if ORC_PLANT == 12
    out[i] = W7(i) * lam + W7(i) * cJ / CS2F;
#else
    out[i] = W7(i) * lam + W7(i) * cJ / CS2G;
#endif
  }
}

/* Eq. 32 on D3Q7 */
void orc3_gsrc(const double *dJ, double lambda, double W, double psi, const double *n,
               double *out) {
  double th = tanh(2.0 * psi / W);
  double sharp = (lambda / W) * (1.0 - th * th);
#if ORC_PLANT == 16
  sharp = -sharp;
#endif
  double v[3];
  for (int a = 0; a < 3; ++a) v[a] = dJ[a] / CS2G + sharp * n[a];
  for (int i = 0; i < 7; ++i)
    out[i] = W7(i) * (C7[i][0] * v[0] + C7[i][1] * v[1] + C7[i][2] * v[2]);
}

static double psi_of(double phi, double W, double xi) {
  double pc = phi < 0.0 ? 0.0 : (phi > 1.0 ? 1.0 : phi);
  return 0.25 * W * log((pc + xi) / (1.0 - pc + xi));
}

/* Isotropic stencils of Sec. 3.2 on the D3Q19 set. */
static void stencil(const orc3_params *p, const double *chi, int x, int y, int z, double *g,
                    double *lap) {
  double c0 = chi[idx(p, x, y, z)];
  double s[3] = {0, 0, 0}, sl = 0.0;
  for (int i = 1; i < 19; ++i) {
    double v = chi[idx(p, x + C19[i][0], y + C19[i][1], z + C19[i][2])];
#if ORC_PLANT == 18
    double wi = 1.0 / 18.0 * (i < 7 ? 1.0 : 0.0) + 1.0 / 36.0 * (i >= 7 ? 1.0 : 0.0) * 1.5;
#else
    double wi = W19(i);
#endif
    for (int a = 0; a < 3; ++a) s[a] += wi * C19[i][a] * v / CS2F;
    sl += 2.0 * wi * (v - c0) / CS2F;
  }
#if ORC_PLANT == 13
  s[2] = -s[2];
#endif
  if (g)
    for (int a = 0; a < 3; ++a) g[a] = s[a];
  if (lap) *lap = sl;
}

void orc3_stencil(const orc3_params *p, const double *chi, double *gx, double *gy, double *gz,
                  double *lap) {
  for (int z = 0; z < p->nz; ++z)
    for (int y = 0; y < p->ny; ++y)
      for (int x = 0; x < p->nx; ++x) {
        size_t k = idx(p, x, y, z);
        double g[3], l;
        stencil(p, chi, x, y, z, g, &l);
        gx[k] = g[0];
        gy[k] = g[1];
        gz[k] = g[2];
        lap[k] = l;
      }
}

static double chem(const orc3_params *p, double phi, double lap) {
  double beta = 12.0 * p->sigma / p->W, kappa = 1.5 * p->sigma * p->W; /* Sec. 2 */
  return 4.0 * beta * phi * (phi - 1.0) * (phi - 0.5) - kappa * lap;
}

static double rho_of(const orc3_params *p, double phi) {
  return p->rho_g + phi * (p->rho_l - p->rho_g);
}

static double tau_f_of(const orc3_params *p, double phi) {
  double mu_l = p->rho_l * CS2F * (p->tau_f_l - 0.5), mu_g = p->rho_g * CS2F * (p->tau_f_g - 0.5);
#if ORC_PLANT == 20
  return (mu_g + phi * (mu_l - mu_g)) / (p->rho_l * CS2F) + 0.5;
#else
  return (mu_g + phi * (mu_l - mu_g)) / (rho_of(p, phi) * CS2F) + 0.5;
#endif
}

typedef struct {
  double *phi, *psi;
} phase_t;

static void phase_fields(const orc3_params *p, const double *g, phase_t *w) {
  size_t n = (size_t)p->nx * p->ny * p->nz;
  for (size_t k = 0; k < n; ++k) {
    double s = 0.0;
    for (int i = 0; i < 7; ++i) s += g[i * n + k]; /* Eq. 35 */
    w->phi[k] = s;
    w->psi[k] = psi_of(s, p->W, p->xi); /* Eq. 37 */
  }
}

typedef struct {
  double mu, rho, gp[3], lap, F[3], gr[3], u[3], pr, gs[3];
} macro3;

static void node_macros(const orc3_params *p, const double *f, size_t n, int x, int y, int z,
                        const phase_t *w, macro3 *m) {
  size_t k = idx(p, x, y, z);
  double phi = w->phi[k];
  stencil(p, w->phi, x, y, z, m->gp, &m->lap);
  stencil(p, w->psi, x, y, z, m->gs, NULL);
  m->mu = chem(p, phi, m->lap);
  m->rho = rho_of(p, phi);
  double j[3] = {0, 0, 0}, sum_nz = 0.0;
  for (int i = 0; i < 19; ++i) {
    for (int a = 0; a < 3; ++a) j[a] += C19[i][a] * f[i * n + k];
    if (i) sum_nz += f[i * n + k];
  }
  for (int a = 0; a < 3; ++a) {
    m->F[a] = m->mu * m->gp[a]; /* F = hbar grad phi */
    m->gr[a] = (p->rho_l - p->rho_g) * m->gp[a];
#if ORC_PLANT == 14
    m->u[a] = (j[a] + m->F[a]) / m->rho;
#else
    m->u[a] = (j[a] + 0.5 * m->F[a]) / m->rho; /* Eq. 28 */
#endif
  }
  double ugr = m->u[0] * m->gr[0] + m->u[1] * m->gr[1] + m->u[2] * m->gr[2];
  double uu = m->u[0] * m->u[0] + m->u[1] * m->u[1] + m->u[2] * m->u[2];
  double s0 = W19(0) * (-uu / (2 * CS2F));
#if ORC_PLANT == 17
  m->pr = CS2F / (1.0 - 4.0 / 9.0) * (sum_nz + 0.5 * ugr + m->rho * s0);
#else
  m->pr = CS2F / (1.0 - W19(0)) * (sum_nz + 0.5 * ugr + m->rho * s0); /* Eq. 29 */
#endif
}

static int check(const orc3_params *p) {
  if (!p || p->nx < 1 || p->ny < 1 || p->nz < 1) return -1;
  if (!(p->W > 0) || !(p->tau_g > 0.5) || !(p->tau_f_l > 0.5) || !(p->tau_f_g > 0.5)) return -1;
  if (!(p->rho_l > 0) || !(p->rho_g > 0)) return -1;
  return 0;
}

int orc3_init(const orc3_params *p, const double *phi0, const double *u0, double *f, double *g,
              double *j) {
  if (check(p) || !phi0 || !f || !g || !j) return -1;
  size_t n = (size_t)p->nx * p->ny * p->nz;
  for (int z = 0; z < p->nz; ++z)
    for (int y = 0; y < p->ny; ++y)
      for (int x = 0; x < p->nx; ++x) {
        size_t k = idx(p, x, y, z);
        double lap;
        stencil(p, phi0, x, y, z, NULL, &lap);
        double u[3] = {0, 0, 0};
        if (u0)
          for (int a = 0; a < 3; ++a) u[a] = u0[a * n + k];
        double ge[7], fe[19];
        orc3_geq(phi0[k], chem(p, phi0[k], lap), p->lambda, u, ge);
        orc3_feq(0.0, rho_of(p, phi0[k]), u, fe);
        for (int i = 0; i < 7; ++i) g[i * n + k] = ge[i];
        for (int i = 0; i < 19; ++i) f[i * n + k] = fe[i];
        for (int a = 0; a < 3; ++a) j[a * n + k] = phi0[k] * u[a];
      }
  return 0;
}

int orc3_step(const orc3_params *p, double *f, double *g, double *j, int64_t nsteps) {
  if (check(p) || !f || !g || !j || nsteps < 0) return -1;
  size_t n = (size_t)p->nx * p->ny * p->nz;
  phase_t w;
  w.phi = (double *)malloc(sizeof(double) * n);
  w.psi = (double *)malloc(sizeof(double) * n);
  double *fs = (double *)malloc(sizeof(double) * 19 * n);
  double *gs = (double *)malloc(sizeof(double) * 7 * n);
  if (!w.phi || !w.psi || !fs || !gs) {
    free(w.phi);
    free(w.psi);
    free(fs);
    free(gs);
    return -2;
  }
  for (int64_t s = 0; s < nsteps; ++s) {
    phase_fields(p, g, &w);
#pragma omp parallel for schedule(static)
    for (int z = 0; z < p->nz; ++z)
      for (int y = 0; y < p->ny; ++y)
        for (int x = 0; x < p->nx; ++x) {
          size_t k = idx(p, x, y, z);
          macro3 m;
          node_macros(p, f, n, x, y, z, &w, &m);
          double phi = w.phi[k];
          /* hydrodynamics, SRT limit of Eq. 25 */
          double tf = tau_f_of(p, phi), fe[19], Fi[19];
          orc3_feq(m.pr, m.rho, m.u, fe);
          orc3_force(m.u, m.F, m.gr, Fi);
          for (int i = 0; i < 19; ++i)
            fs[i * n + k] = f[i * n + k] - (f[i * n + k] - fe[i]) / tf + (1.0 - 0.5 / tf) * Fi[i];
          /* phase field, SRT limit of Eq. 33 */
          double J[3], dJ[3], nn[3] = {0, 0, 0};
          for (int a = 0; a < 3; ++a) {
            J[a] = phi * m.u[a];
#if ORC_PLANT == 15
            dJ[a] = 0.0;
#else
            dJ[a] = J[a] - j[a * n + k];
#endif
          }
          double g2 = m.gs[0] * m.gs[0] + m.gs[1] * m.gs[1] + m.gs[2] * m.gs[2];
#if ORC_PLANT == 23
          if (g2 != 0.0)
#else
          if (g2 >= NORMAL_MIN * NORMAL_MIN)
#endif
            for (int a = 0; a < 3; ++a) nn[a] = m.gs[a] / sqrt(g2);
          double ge[7], Gi[7];
          orc3_geq(phi, m.mu, p->lambda, m.u, ge);
          orc3_gsrc(dJ, p->lambda, p->W, w.psi[k], nn, Gi);
          double tg = p->tau_g;
          for (int i = 0; i < 7; ++i)
            gs[i * n + k] = g[i * n + k] - (g[i * n + k] - ge[i]) / tg + (1.0 - 0.5 / tg) * Gi[i];
          for (int a = 0; a < 3; ++a) j[a * n + k] = J[a];
        }
    /* streaming (push) */
    for (int z = 0; z < p->nz; ++z)
      for (int y = 0; y < p->ny; ++y)
        for (int x = 0; x < p->nx; ++x) {
          size_t k = idx(p, x, y, z);
          for (int i = 0; i < 19; ++i)
            f[i * n + idx(p, x + C19[i][0], y + C19[i][1], z + C19[i][2])] = fs[i * n + k];
          for (int i = 0; i < 7; ++i)
#if ORC_PLANT == 19
            g[i * n + idx(p, x + C7[i][0], y + C7[i][1], z - C7[i][2])] = gs[i * n + k];
#else
            g[i * n + idx(p, x + C7[i][0], y + C7[i][1], z + C7[i][2])] = gs[i * n + k];
#endif
        }
  }
  free(w.phi);
  free(w.psi);
  free(fs);
  free(gs);
  return 0;
}

int orc3_fields(const orc3_params *p, const double *f, const double *g, double *phi, double *u,
                double *pr) {
  if (check(p) || !f || !g) return -1;
  size_t n = (size_t)p->nx * p->ny * p->nz;
  phase_t w;
  w.phi = (double *)malloc(sizeof(double) * n);
  w.psi = (double *)malloc(sizeof(double) * n);
  if (!w.phi || !w.psi) {
    free(w.phi);
    free(w.psi);
    return -2;
  }
  phase_fields(p, g, &w);
  for (int z = 0; z < p->nz; ++z)
    for (int y = 0; y < p->ny; ++y)
      for (int x = 0; x < p->nx; ++x) {
        size_t k = idx(p, x, y, z);
        macro3 m;
        node_macros(p, f, n, x, y, z, &w, &m);
        if (phi) phi[k] = w.phi[k];
        if (u)
          for (int a = 0; a < 3; ++a) u[a * n + k] = m.u[a];
        if (pr) pr[k] = m.pr;
      }
  free(w.phi);
  free(w.psi);
  return 0;
}
