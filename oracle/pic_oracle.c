/*
 * Plain FP64 CPU oracle of the patch-decomposed 2D3V particle-in-cell step.
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, the smoke check and the
 * benchmark's CPU-baseline leg; never by the product library.
 *
 * Every step follows the order of the SDMD loop (Section 2.2, steps (i) and
 * (ii); Section 3.3 "Particles" / "Fields" phases):
 *   1. per patch (OpenMP over patches): interpolate E^n and Bm^n at x^n,
 *      Boris push u^{n-1/2} -> u^{n+1/2}, move x^n -> x^{n+1}, Esirkepov
 *      deposition of J^{n+1/2} into a private patch current buffer;
 *   2. SDMD step (i): the patch buffers are added into the region (domain)
 *      current in ascending patch order, so the result does not depend on
 *      the number of threads;
 *   3. particle boundary conditions and re-binning into patches;
 *   4. Yee update of the region: E^{n+1}, B^{n+3/2}, Bm^{n+1} = time average,
 *      Silver-Mueller open boundaries (with laser injection at x_min);
 *   5. moving window shift, when due.
 * SDMD step (ii) is the interpolation itself: patches read the region's
 * fields directly.
 */
#include "pic_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define G 4 /* ghost cells stored on every side of every axis */
#define NF 12

/* Yee stagger of each stored component: 1 = dual (half-integer) along axis. */
static const int STAG_X[NF] = {1, 0, 0, 0, 1, 1, 0, 1, 1, 1, 0, 0};
static const int STAG_Y[NF] = {0, 1, 0, 1, 0, 1, 1, 0, 1, 0, 1, 0};

struct orc_state {
  orc_config c;
  long sx, ntot;          /* row stride, elements per array */
  double *F[NF];
  double *rho_bg, *rho_prev;
  int have_rho_prev;
  long np, cap;
  double *x, *y, *ux, *uy, *uz, *w;
  int *pid;               /* patch of each particle */
  long *pstart;           /* particles of patch p: [pstart[p], pstart[p+1]) */
  int npx, npy;
  long step;
  double t;
  int nshift;
};

static int imod(int a, int n) { int r = a % n; return r < 0 ? r + n : r; }

/* Address of component array element at grid index (i, j); periodic axes
 * wrap, open axes address the ghost cells directly. */
static double *at(const orc_state *s, double *a, int i, int j) {
  if (s->c.fbc_x == ORC_FBC_PERIODIC) i = imod(i, s->c.nx);
  if (s->c.fbc_y == ORC_FBC_PERIODIC) j = imod(j, s->c.ny);
  return &a[(long)(j + G) * s->sx + (i + G)];
}

static int in_store(const orc_state *s, int i, int j) {
  int okx = s->c.fbc_x == ORC_FBC_PERIODIC || (i >= -G && i < s->c.nx + G);
  int oky = s->c.fbc_y == ORC_FBC_PERIODIC || (j >= -G && j < s->c.ny + G);
  return okx && oky;
}

/* Second-order (quadratic B-spline) shape, Section 3.2 ("second order shape
 * function, 5 points stencil" for the Esirkepov scheme): nearest node
 * i0 = floor(xi + 1/2), delta = xi - i0 in [-1/2, 1/2); weights of nodes
 * i0-1, i0, i0+1. */
void orc_shape2(double xi, int *i0, double S[3]) {
  int i = (int)floor(xi + 0.5);
  double d = xi - (double)i;
  S[0] = 0.5 * (0.5 - d) * (0.5 - d);
  S[1] = 0.75 - d * d;
  S[2] = 0.5 * (0.5 + d) * (0.5 + d);
  *i0 = i;
}

/* Boris rotation push (pusher not named in the paper).  u is u^{n-1/2} on
 * input and u^{n+1/2} on output. */
void orc_boris(double q, double m, double dt, const double E[3],
               const double B[3], double u[3]) {
  double eps = q * dt / (2.0 * m);
  double um[3], up[3], uprime[3], tv[3], sv[3];
  int k;
  for (k = 0; k < 3; ++k) um[k] = u[k] + eps * E[k];
  double gm = sqrt(1.0 + um[0] * um[0] + um[1] * um[1] + um[2] * um[2]);
  for (k = 0; k < 3; ++k) tv[k] = eps * B[k] / gm;
  double t2 = tv[0] * tv[0] + tv[1] * tv[1] + tv[2] * tv[2];
  for (k = 0; k < 3; ++k) sv[k] = 2.0 * tv[k] / (1.0 + t2);
  uprime[0] = um[0] + (um[1] * tv[2] - um[2] * tv[1]);
  uprime[1] = um[1] + (um[2] * tv[0] - um[0] * tv[2]);
  uprime[2] = um[2] + (um[0] * tv[1] - um[1] * tv[0]);
  up[0] = um[0] + (uprime[1] * sv[2] - uprime[2] * sv[1]);
  up[1] = um[1] + (uprime[2] * sv[0] - uprime[0] * sv[2]);
  up[2] = um[2] + (uprime[0] * sv[1] - uprime[1] * sv[0]);
  for (k = 0; k < 3; ++k) u[k] = up[k] + eps * E[k];
}

/* Interpolate component comp at (x, y) with the quadratic shape of its own
 * stagger. */
static double gather(const orc_state *s, int comp, double x, double y) {
  int ix, iy, a, b;
  double Sx[3], Sy[3], v = 0.0;
  orc_shape2(x / s->c.dx - 0.5 * STAG_X[comp], &ix, Sx);
  orc_shape2(y / s->c.dy - 0.5 * STAG_Y[comp], &iy, Sy);
  for (b = 0; b < 3; ++b)
    for (a = 0; a < 3; ++a)
      v += Sx[a] * Sy[b] * *at(s, s->F[comp], ix - 1 + a, iy - 1 + b);
  return v;
}

double orc_gather(const orc_state *s, int comp, double x, double y) {
  if (comp < 0 || comp >= NF) return NAN;
  return gather(s, comp, x, y);
}

/* Esirkepov (2001) charge-conserving current of one particle, 2D3V, on the
 * 5-node window that starts two nodes below the nearest node of x^n.  Jw[0]
 * holds Jx at dual x-index ix+k, primal y-index iy+l; Jw[1] Jy at primal
 * ix+k, dual iy+l; Jw[2] Jz at primal (ix+k, iy+l). */
int orc_esirkepov(const orc_state *s, double x0, double y0, double x1,
                  double y1, double w, double vz, int *ix, int *iy,
                  double Jw[3][5][5]) {
  double S0x[5] = {0}, S1x[5] = {0}, S0y[5] = {0}, S1y[5] = {0};
  double DSx[5], DSy[5], S[3];
  int i0, j0, i1, j1, k, l;
  const double q = s->c.q;
  orc_shape2(x0 / s->c.dx, &i0, S);
  for (k = 0; k < 3; ++k) S0x[1 + k] = S[k];
  orc_shape2(y0 / s->c.dy, &j0, S);
  for (k = 0; k < 3; ++k) S0y[1 + k] = S[k];
  orc_shape2(x1 / s->c.dx, &i1, S);
  if (i1 - i0 < -1 || i1 - i0 > 1) return -1; /* moved more than one cell */
  for (k = 0; k < 3; ++k) S1x[1 + (i1 - i0) + k] = S[k];
  orc_shape2(y1 / s->c.dy, &j1, S);
  if (j1 - j0 < -1 || j1 - j0 > 1) return -1;
  for (k = 0; k < 3; ++k) S1y[1 + (j1 - j0) + k] = S[k];
  for (k = 0; k < 5; ++k) {
    DSx[k] = S1x[k] - S0x[k];
    DSy[k] = S1y[k] - S0y[k];
  }
  *ix = i0 - 2;
  *iy = j0 - 2;
  /* Jx: prefix sum of W_x = DSx (S0y + DSy/2) along x. */
  for (l = 0; l < 5; ++l) {
    double acc = 0.0;
    for (k = 0; k < 5; ++k) {
      acc += DSx[k] * (S0y[l] + 0.5 * DSy[l]);
      Jw[0][l][k] += -q * w * (s->c.dx / s->c.dt) * acc;
    }
  }
  /* Jy: prefix sum of W_y = DSy (S0x + DSx/2) along y. */
  for (k = 0; k < 5; ++k) {
    double acc = 0.0;
    for (l = 0; l < 5; ++l) {
      acc += DSy[l] * (S0x[k] + 0.5 * DSx[k]);
      Jw[1][l][k] += -q * w * (s->c.dy / s->c.dt) * acc;
    }
  }
  /* Jz = q w v_z W_z, W_z the time average of Sx Sy along the straight
   * path. */
  for (l = 0; l < 5; ++l)
    for (k = 0; k < 5; ++k) {
      double Wz = S0x[k] * S0y[l] + 0.5 * DSx[k] * S0y[l] +
                  0.5 * S0x[k] * DSy[l] + (1.0 / 3.0) * DSx[k] * DSy[l];
      Jw[2][l][k] += q * w * vz * Wz;
    }
  return 0;
}

/* Laser field entering through x_min: y-polarised Gaussian beam focused on
 * the boundary, Gaussian envelope with intensity FWHM tau, carrier w0 = 1,
 * evaluated at the retarded time of the (possibly moved) boundary. */
int orc_laser_field(const orc_state *s, double y, double t, double *ey) {
  const orc_config *c = &s->c;
  double tr = t - s->nshift * c->px * c->dx - c->t_peak;
  double r = (y - c->y_center) / c->waist;
  *ey = c->a0 * exp(-r * r) * exp(-2.0 * log(2.0) * tr * tr / (c->tau * c->tau)) *
        sin(tr);
  return 0;
}

static double profile(const orc_config *c, double xphys) {
  if (c->inj_ramp <= 0.0) return xphys >= c->inj_x0 ? c->inj_n0 : 0.0;
  double f = (xphys - c->inj_x0) / c->inj_ramp;
  if (f < 0.0) f = 0.0;
  if (f > 1.0) f = 1.0;
  return c->inj_n0 * f;
}

static int patch_of(const orc_state *s, double x, double y) {
  int cx = (int)floor(x / s->c.dx), cy = (int)floor(y / s->c.dy);
  int px = cx / s->c.px, py = cy / s->c.py;
  if (px < 0) px = 0;
  if (px >= s->npx) px = s->npx - 1;
  if (py < 0) py = 0;
  if (py >= s->npy) py = s->npy - 1;
  return py * s->npx + px;
}

/* Stable counting sort of the particles by patch. */
static void rebin(orc_state *s) {
  long np = s->np, i;
  int npatch = s->npx * s->npy, p;
  long *cnt = calloc(npatch + 1, sizeof(long));
  for (i = 0; i < np; ++i) {
    s->pid[i] = patch_of(s, s->x[i], s->y[i]);
    cnt[s->pid[i] + 1]++;
  }
  for (p = 0; p < npatch; ++p) cnt[p + 1] += cnt[p];
  memcpy(s->pstart, cnt, (npatch + 1) * sizeof(long));
  double *arr[6] = {s->x, s->y, s->ux, s->uy, s->uz, s->w};
  double *tmp = malloc((np > 0 ? np : 1) * sizeof(double));
  long *dst = malloc((np > 0 ? np : 1) * sizeof(long));
  int *pid2 = malloc((np > 0 ? np : 1) * sizeof(int));
  for (i = 0; i < np; ++i) dst[i] = cnt[s->pid[i]]++;
  for (int a = 0; a < 6; ++a) {
    for (i = 0; i < np; ++i) tmp[dst[i]] = arr[a][i];
    memcpy(arr[a], tmp, np * sizeof(double));
  }
  for (i = 0; i < np; ++i) pid2[dst[i]] = s->pid[i];
  memcpy(s->pid, pid2, np * sizeof(int));
  free(tmp);
  free(dst);
  free(pid2);
  free(cnt);
}

static int grow(orc_state *s, long need) {
  if (need <= s->cap) return 0;
  long cap = need + need / 2 + 16;
  double **arr[6] = {&s->x, &s->y, &s->ux, &s->uy, &s->uz, &s->w};
  for (int a = 0; a < 6; ++a) {
    double *p = realloc(*arr[a], cap * sizeof(double));
    if (!p) return -1;
    *arr[a] = p;
  }
  int *pp = realloc(s->pid, cap * sizeof(int));
  if (!pp) return -1;
  s->pid = pp;
  s->cap = cap;
  return 0;
}

orc_state *orc_create(const orc_config *c) {
  if (c->nx <= 0 || c->ny <= 0 || c->px <= 0 || c->py <= 0) return NULL;
  if (c->nx % c->px || c->ny % c->py) return NULL;
  orc_state *s = calloc(1, sizeof(orc_state));
  s->c = *c;
  s->sx = c->nx + 2 * G;
  s->ntot = s->sx * (c->ny + 2 * G);
  for (int k = 0; k < NF; ++k) s->F[k] = calloc(s->ntot, sizeof(double));
  s->rho_bg = calloc(s->ntot, sizeof(double));
  s->rho_prev = calloc(s->ntot, sizeof(double));
  s->npx = c->nx / c->px;
  s->npy = c->ny / c->py;
  s->pstart = calloc(s->npx * s->npy + 1, sizeof(long));
  return s;
}

void orc_destroy(orc_state *s) {
  if (!s) return;
  for (int k = 0; k < NF; ++k) free(s->F[k]);
  free(s->rho_bg);
  free(s->rho_prev);
  free(s->x); free(s->y); free(s->ux); free(s->uy); free(s->uz); free(s->w);
  free(s->pid);
  free(s->pstart);
  free(s);
}

int orc_load(orc_state *s, const double *x, const double *y, const double *ux,
             const double *uy, const double *uz, const double *w, long n) {
  if (grow(s, s->np + n)) return -1;
  for (long i = 0; i < n; ++i) {
    long k = s->np + i;
    s->x[k] = x[i]; s->y[k] = y[i];
    s->ux[k] = ux[i]; s->uy[k] = uy[i]; s->uz[k] = uz[i];
    s->w[k] = w[i];
  }
  s->np += n;
  rebin(s);
  return 0;
}

long orc_num_particles(const orc_state *s) { return s->np; }

long orc_get_particles(const orc_state *s, double *out) {
  long n = s->np;
  const double *arr[6] = {s->x, s->y, s->ux, s->uy, s->uz, s->w};
  for (int a = 0; a < 6; ++a) memcpy(out + a * n, arr[a], n * sizeof(double));
  return n;
}

static void out_range(int fbc, int n, int *lo, int *cnt) {
  if (fbc == ORC_FBC_PERIODIC) { *lo = 0; *cnt = n; }
  else { *lo = -1; *cnt = n + 2; }
}

static void deposit_rho(const orc_state *s, double *rho, double sign);

static double *comp_array(orc_state *s, int comp, int *tmp_owned) {
  *tmp_owned = 0;
  if (comp < NF) return s->F[comp];
  if (comp == ORC_RHO_BG) return s->rho_bg;
  if (comp == ORC_RHO) {
    double *r = calloc(s->ntot, sizeof(double));
    deposit_rho(s, r, 1.0);
    *tmp_owned = 1;
    return r;
  }
  return NULL;
}

int orc_set_field(orc_state *s, int comp, const double *src) {
  int lx, nxo, ly, nyo;
  if (comp < 0 || comp >= ORC_NOUT || comp == ORC_RHO) return -1;
  double *a = comp == ORC_RHO_BG ? s->rho_bg : s->F[comp];
  out_range(s->c.fbc_x, s->c.nx, &lx, &nxo);
  out_range(s->c.fbc_y, s->c.ny, &ly, &nyo);
  for (int j = 0; j < nyo; ++j)
    for (int i = 0; i < nxo; ++i)
      *at(s, a, lx + i, ly + j) = src[(long)j * nxo + i];
  return 0;
}

int orc_get_field(orc_state *s, int comp, double *dst) {
  int lx, nxo, ly, nyo, own;
  if (comp < 0 || comp >= ORC_NOUT) return -1;
  double *a = comp_array(s, comp, &own);
  out_range(s->c.fbc_x, s->c.nx, &lx, &nxo);
  out_range(s->c.fbc_y, s->c.ny, &ly, &nyo);
  for (int j = 0; j < nyo; ++j)
    for (int i = 0; i < nxo; ++i)
      dst[(long)j * nxo + i] = *at(s, a, lx + i, ly + j);
  if (own) free(a);
  return 0;
}

/* rho += sign * q w S(x) S(y) at primal nodes. */
static void deposit_rho(const orc_state *s, double *rho, double sign) {
  for (long p = 0; p < s->np; ++p) {
    int ix, iy;
    double Sx[3], Sy[3];
    orc_shape2(s->x[p] / s->c.dx, &ix, Sx);
    orc_shape2(s->y[p] / s->c.dy, &iy, Sy);
    for (int b = 0; b < 3; ++b)
      for (int a = 0; a < 3; ++a)
        if (in_store(s, ix - 1 + a, iy - 1 + b))
          *at(s, rho, ix - 1 + a, iy - 1 + b) +=
              sign * s->c.q * s->w[p] * Sx[a] * Sy[b];
  }
}

int orc_set_background(orc_state *s, int mode, double value) {
  memset(s->rho_bg, 0, s->ntot * sizeof(double));
  if (mode == 1) {
    for (long k = 0; k < s->ntot; ++k) s->rho_bg[k] = value;
  } else if (mode == 2) {
    deposit_rho(s, s->rho_bg, -1.0);
  } else if (mode != 0) {
    return -1;
  }
  return 0;
}

/* Update range of a component along one axis: periodic axes update [0, n);
 * open axes update primal nodes [0, n] and dual points [0, n-1]. */
static void upd_range(int fbc, int n, int dual, int *lo, int *hi) {
  *lo = 0;
  *hi = (fbc == ORC_FBC_PERIODIC) ? n : (dual ? n : n + 1);
}

/* Binomial current filter (Section 3.2: "two-pass binomial filter" on the
 * current densities every iteration): each pass replaces J(i) by
 * (J(i-1) + 2 J(i) + J(i+1)) / 4 along x, then the same along y, for every
 * stored index; periodic axes wrap, open axes read zero outside the stored
 * range. */
static void filter_current(orc_state *s) {
  const orc_config *c = &s->c;
  double *tmp = malloc(s->ntot * sizeof(double));
  const int xl = c->fbc_x == ORC_FBC_PERIODIC ? 0 : -G, xh = c->fbc_x == ORC_FBC_PERIODIC ? c->nx : c->nx + G;
  const int yl = c->fbc_y == ORC_FBC_PERIODIC ? 0 : -G, yh = c->fbc_y == ORC_FBC_PERIODIC ? c->ny : c->ny + G;
  for (int pass = 0; pass < c->filter_passes; ++pass)
    for (int k = ORC_JX; k <= ORC_JZ; ++k)
      for (int axis = 0; axis < 2; ++axis) {
        double *J = s->F[k];
        memcpy(tmp, J, s->ntot * sizeof(double));
        for (int j = yl; j < yh; ++j)
          for (int i = xl; i < xh; ++i) {
            const int di = axis == 0, dj = axis == 1;
            double lo = 0.0, hi = 0.0;
            if (in_store(s, i - di, j - dj)) lo = *at(s, tmp, i - di, j - dj);
            if (in_store(s, i + di, j + dj)) hi = *at(s, tmp, i + di, j + dj);
            *at(s, J, i, j) = 0.25 * (lo + 2.0 * *at(s, tmp, i, j) + hi);
          }
      }
  free(tmp);
}

void orc_apply_filter(orc_state *s) { filter_current(s); }

/* Yee finite-difference update of the region (Section 3.2):
 * E^{n+1} = E^n + dt (curl B^{n+1/2} - J^{n+1/2}),
 * B^{n+3/2} = B^{n+1/2} - dt curl E^{n+1}, Bm^{n+1} = (B^{n+1/2}+B^{n+3/2})/2,
 * followed by the Silver-Mueller boundary values of B on open axes. */
static void maxwell(orc_state *s) {
  const orc_config *c = &s->c;
  const double dt = c->dt, dx = c->dx, dy = c->dy;
  double *Ex = s->F[ORC_EX], *Ey = s->F[ORC_EY], *Ez = s->F[ORC_EZ];
  double *Bx = s->F[ORC_BX], *By = s->F[ORC_BY], *Bz = s->F[ORC_BZ];
  double *Jx = s->F[ORC_JX], *Jy = s->F[ORC_JY], *Jz = s->F[ORC_JZ];
  int i, j, xl, xh, yl, yh;

  upd_range(c->fbc_x, c->nx, 1, &xl, &xh);
  upd_range(c->fbc_y, c->ny, 0, &yl, &yh);
#pragma omp parallel for private(i)
  for (j = yl; j < yh; ++j)
    for (i = xl; i < xh; ++i)
      *at(s, Ex, i, j) += dt * ((*at(s, Bz, i, j) - *at(s, Bz, i, j - 1)) / dy -
                                *at(s, Jx, i, j));
  upd_range(c->fbc_x, c->nx, 0, &xl, &xh);
  upd_range(c->fbc_y, c->ny, 1, &yl, &yh);
#pragma omp parallel for private(i)
  for (j = yl; j < yh; ++j)
    for (i = xl; i < xh; ++i)
      *at(s, Ey, i, j) += dt * (-(*at(s, Bz, i, j) - *at(s, Bz, i - 1, j)) / dx -
                                *at(s, Jy, i, j));
  upd_range(c->fbc_x, c->nx, 0, &xl, &xh);
  upd_range(c->fbc_y, c->ny, 0, &yl, &yh);
#pragma omp parallel for private(i)
  for (j = yl; j < yh; ++j)
    for (i = xl; i < xh; ++i)
      *at(s, Ez, i, j) += dt * ((*at(s, By, i, j) - *at(s, By, i - 1, j)) / dx -
                                (*at(s, Bx, i, j) - *at(s, Bx, i, j - 1)) / dy -
                                *at(s, Jz, i, j));

  /* Keep B^{n+1/2} in Bm, then advance B. */
  memcpy(s->F[ORC_BMX], Bx, s->ntot * sizeof(double));
  memcpy(s->F[ORC_BMY], By, s->ntot * sizeof(double));
  memcpy(s->F[ORC_BMZ], Bz, s->ntot * sizeof(double));

  upd_range(c->fbc_x, c->nx, 0, &xl, &xh);
  upd_range(c->fbc_y, c->ny, 1, &yl, &yh);
#pragma omp parallel for private(i)
  for (j = yl; j < yh; ++j)
    for (i = xl; i < xh; ++i)
      *at(s, Bx, i, j) -= dt * (*at(s, Ez, i, j + 1) - *at(s, Ez, i, j)) / dy;
  upd_range(c->fbc_x, c->nx, 1, &xl, &xh);
  upd_range(c->fbc_y, c->ny, 0, &yl, &yh);
#pragma omp parallel for private(i)
  for (j = yl; j < yh; ++j)
    for (i = xl; i < xh; ++i)
      *at(s, By, i, j) += dt * (*at(s, Ez, i + 1, j) - *at(s, Ez, i, j)) / dx;
  upd_range(c->fbc_x, c->nx, 1, &xl, &xh);
  upd_range(c->fbc_y, c->ny, 1, &yl, &yh);
#pragma omp parallel for private(i)
  for (j = yl; j < yh; ++j)
    for (i = xl; i < xh; ++i)
      *at(s, Bz, i, j) -= dt * ((*at(s, Ey, i + 1, j) - *at(s, Ey, i, j)) / dx -
                                (*at(s, Ex, i, j + 1) - *at(s, Ex, i, j)) / dy);

  /* Silver-Mueller: the first-order absorbing condition E_t -/+ n x B =
   * 2 E_inc, centred half a step back and combined with Ampere's law on the
   * boundary node, gives the ghost B^{n+3/2} just outside each open face.
   * Transverse differences that would need a ghost of the other open axis
   * (corner nodes) are taken as zero. */
  const double tB = s->t + 1.5 * dt; /* time level of B^{n+3/2} */
  if (c->fbc_x == ORC_FBC_SM) {
    const double r = dt / dx;
    const int nx = c->nx, ny = c->ny;
    int jlo = 0, jhi = (c->fbc_y == ORC_FBC_PERIODIC) ? ny : ny + 1;
    for (j = jlo; j < jhi; ++j) {
      double dBx0 = 0.0, dBxn = 0.0;
      int interior = c->fbc_y == ORC_FBC_PERIODIC || (j >= 1 && j <= ny - 1);
      if (interior) {
        dBx0 = *at(s, Bx, 0, j) - *at(s, Bx, 0, j - 1);
        dBxn = *at(s, Bx, nx, j) - *at(s, Bx, nx, j - 1);
      }
      double ezinc = 0.0;
      /* By at x = -dx/2 (pairs with Ez; the laser has no z component). */
      *at(s, By, -1, j) = (-4.0 * ezinc + 2.0 * *at(s, Ez, 0, j) -
                           (1.0 - r) * *at(s, By, 0, j) - (dt / dy) * dBx0) /
                          (1.0 + r);
      *at(s, By, nx, j) = (-2.0 * *at(s, Ez, nx, j) -
                           (1.0 - r) * *at(s, By, nx - 1, j) + (dt / dy) * dBxn) /
                          (1.0 + r);
    }
    jhi = ny; /* Bz is dual along y */
    for (j = 0; j < jhi; ++j) {
      double eyinc = 0.0;
      if (c->laser_on) orc_laser_field(s, (j + 0.5) * dy, tB, &eyinc);
      *at(s, Bz, -1, j) = (4.0 * eyinc - 2.0 * *at(s, Ey, 0, j) -
                           (1.0 - r) * *at(s, Bz, 0, j)) / (1.0 + r);
      *at(s, Bz, nx, j) = (2.0 * *at(s, Ey, nx, j) -
                           (1.0 - r) * *at(s, Bz, nx - 1, j)) / (1.0 + r);
    }
  }
  if (c->fbc_y == ORC_FBC_SM) {
    const double r = dt / dy;
    const int nx = c->nx, ny = c->ny;
    int ihi = (c->fbc_x == ORC_FBC_PERIODIC) ? nx : nx + 1;
    for (i = 0; i < ihi; ++i) {
      double dBy0 = 0.0, dByn = 0.0;
      int interior = c->fbc_x == ORC_FBC_PERIODIC || (i >= 1 && i <= nx - 1);
      if (interior) {
        dBy0 = *at(s, By, i, 0) - *at(s, By, i - 1, 0);
        dByn = *at(s, By, i, ny) - *at(s, By, i - 1, ny);
      }
      *at(s, Bx, i, -1) = (-2.0 * *at(s, Ez, i, 0) - (1.0 - r) * *at(s, Bx, i, 0) -
                           (dt / dx) * dBy0) / (1.0 + r);
      *at(s, Bx, i, ny) = (2.0 * *at(s, Ez, i, ny) -
                           (1.0 - r) * *at(s, Bx, i, ny - 1) + (dt / dx) * dByn) /
                          (1.0 + r);
    }
    for (i = 0; i < nx; ++i) {
      *at(s, Bz, i, -1) = (2.0 * *at(s, Ex, i, 0) - (1.0 - r) * *at(s, Bz, i, 0)) /
                          (1.0 + r);
      *at(s, Bz, i, ny) = (-2.0 * *at(s, Ex, i, ny) -
                           (1.0 - r) * *at(s, Bz, i, ny - 1)) / (1.0 + r);
    }
  }

  /* Bm^{n+1} = (B^{n+1/2} + B^{n+3/2}) / 2 everywhere (ghosts included). */
  for (int k = 0; k < 3; ++k) {
    double *bm = s->F[ORC_BMX + k], *b = s->F[ORC_BX + k];
    for (long e = 0; e < s->ntot; ++e) bm[e] = 0.5 * (bm[e] + b[e]);
  }
}

/* Shift the window by one patch column (px cells) towards +x: every stored
 * value (boundary and ghost nodes included, so that the charge of particles
 * near the old x_max keeps its whole stencil) moves px cells down in index;
 * stored indices with no source become vacuum; particles of the leaving
 * column are dropped and the new column is filled with plasma of the
 * configured profile, regularly placed, at rest. */
static void shift_window(orc_state *s) {
  const orc_config *c = &s->c;
  const int P = c->px, nx = c->nx;
  double *arrs[NF + 1];
  for (int k = 0; k < NF; ++k) arrs[k] = s->F[k];
  arrs[NF] = s->rho_bg;
  for (int k = 0; k < NF + 1; ++k) {
    double *a = arrs[k];
    for (int j = -G; j < c->ny + G; ++j) {
      double *row = &a[(long)(j + G) * s->sx];
      for (int i = -G; i < nx + G; ++i)
        row[i + G] = (i + P < nx + G) ? row[i + P + G] : 0.0;
    }
  }
  s->nshift++;
  /* Move and drop particles. */
  long k = 0;
  for (long p = 0; p < s->np; ++p) {
    double xn = s->x[p] - P * c->dx;
    if (xn < 0.0) continue;
    s->x[k] = xn; s->y[k] = s->y[p];
    s->ux[k] = s->ux[p]; s->uy[k] = s->uy[p]; s->uz[k] = s->uz[p];
    s->w[k] = s->w[p];
    ++k;
  }
  long kept = k;
  long nnew = (long)P * c->ny * c->inj_ppcx * c->inj_ppcy;
  grow(s, kept + nnew);
  const int ppc = c->inj_ppcx * c->inj_ppcy;
  for (int j = 0; j < c->ny; ++j)
    for (int i = nx - P; i < nx; ++i)
      for (int b = 0; b < c->inj_ppcy; ++b)
        for (int a = 0; a < c->inj_ppcx; ++a) {
          double xl = (i + (a + 0.5) / c->inj_ppcx) * c->dx;
          double yl = (j + (b + 0.5) / c->inj_ppcy) * c->dy;
          double xphys = xl + (double)s->nshift * P * c->dx;
          s->x[k] = xl; s->y[k] = yl;
          s->ux[k] = 0.0; s->uy[k] = 0.0; s->uz[k] = 0.0;
          s->w[k] = profile(c, xphys) / ppc;
          ++k;
        }
  /* Immobile ions of the new plasma, co-located with the new electrons. */
  s->np = k;
  {
    orc_state tmp = *s;
    tmp.x = s->x + kept; tmp.y = s->y + kept; tmp.w = s->w + kept;
    tmp.np = k - kept;
    deposit_rho(&tmp, s->rho_bg, -1.0);
  }
  rebin(s);
}

static void apply_particle_bc(orc_state *s) {
  const orc_config *c = &s->c;
  const double Lx = c->nx * c->dx, Ly = c->ny * c->dy;
  long k = 0;
  for (long p = 0; p < s->np; ++p) {
    double x = s->x[p], y = s->y[p];
    int drop = 0;
    if (x < 0.0 || x >= Lx) {
      int bc = x < 0.0 ? c->pbc_x[0] : c->pbc_x[1];
      if (bc == ORC_PBC_PERIODIC) x += (x < 0.0 ? Lx : -Lx);
      else if (bc == ORC_PBC_REFLECT) { x = x < 0.0 ? -x : 2.0 * Lx - x; s->ux[p] = -s->ux[p]; }
      else drop = 1;
    }
    if (!drop && (y < 0.0 || y >= Ly)) {
      int bc = y < 0.0 ? c->pbc_y[0] : c->pbc_y[1];
      if (bc == ORC_PBC_PERIODIC) y += (y < 0.0 ? Ly : -Ly);
      else if (bc == ORC_PBC_REFLECT) { y = y < 0.0 ? -y : 2.0 * Ly - y; s->uy[p] = -s->uy[p]; }
      else drop = 1;
    }
    if (drop) continue;
    s->x[k] = x; s->y[k] = y;
    s->ux[k] = s->ux[p]; s->uy[k] = s->uy[p]; s->uz[k] = s->uz[p];
    s->w[k] = s->w[p];
    ++k;
  }
  s->np = k;
}

int orc_step(orc_state *s, int nsteps) {
  const orc_config *c = &s->c;
  const int P = c->px, Q = c->py, W = P + 5, H = Q + 5;
  const int npatch = s->npx * s->npy;
  double *Jbuf = malloc((size_t)npatch * 3 * W * H * sizeof(double));
  int bad = 0;
#ifdef _OPENMP
  if (c->nthreads > 0) omp_set_num_threads(c->nthreads);
#endif
  for (int n = 0; n < nsteps; ++n) {
    if (c->track_continuity) {
      memset(s->rho_prev, 0, s->ntot * sizeof(double));
      deposit_rho(s, s->rho_prev, 1.0);
      s->have_rho_prev = 1;
    }
    for (int k = ORC_JX; k <= ORC_JZ; ++k) memset(s->F[k], 0, s->ntot * sizeof(double));
    memset(Jbuf, 0, (size_t)npatch * 3 * W * H * sizeof(double));

    /* Particle phase: each patch interpolates, pushes and deposits into its
     * own current buffer covering nodes [X0-2, X0+P+2] x [Y0-2, Y0+Q+2]. */
#pragma omp parallel for schedule(dynamic) reduction(| : bad)
    for (int p = 0; p < npatch; ++p) {
      const int X0 = (p % s->npx) * P, Y0 = (p / s->npx) * Q;
      double *Jp = Jbuf + (size_t)p * 3 * W * H;
      for (long k = s->pstart[p]; k < s->pstart[p + 1]; ++k) {
        double E[3], B[3], u[3] = {s->ux[k], s->uy[k], s->uz[k]};
        double x0 = s->x[k], y0 = s->y[k];
        for (int a = 0; a < 3; ++a) {
          E[a] = gather(s, ORC_EX + a, x0, y0);
          B[a] = gather(s, ORC_BMX + a, x0, y0);
        }
        orc_boris(c->q, c->m, c->dt, E, B, u);
        double g = sqrt(1.0 + u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
        double x1 = x0 + c->dt * u[0] / g, y1 = y0 + c->dt * u[1] / g;
        double Jw[3][5][5];
        int ix, iy;
        memset(Jw, 0, sizeof Jw);
        if (orc_esirkepov(s, x0, y0, x1, y1, s->w[k], u[2] / g, &ix, &iy, Jw)) {
          bad = 1;
          continue;
        }
        int ox = ix - (X0 - 2), oy = iy - (Y0 - 2);
        if (ox < 0 || oy < 0 || ox + 5 > W || oy + 5 > H) { bad = 1; continue; }
        for (int cc = 0; cc < 3; ++cc)
          for (int l = 0; l < 5; ++l)
            for (int m = 0; m < 5; ++m)
              Jp[(size_t)cc * W * H + (oy + l) * W + ox + m] += Jw[cc][l][m];
        s->x[k] = x1; s->y[k] = y1;
        s->ux[k] = u[0]; s->uy[k] = u[1]; s->uz[k] = u[2];
      }
    }
    /* SDMD step (i): patch currents -> region current, ascending patch
     * order. */
    for (int p = 0; p < npatch; ++p) {
      const int X0 = (p % s->npx) * P, Y0 = (p / s->npx) * Q;
      double *Jp = Jbuf + (size_t)p * 3 * W * H;
      for (int cc = 0; cc < 3; ++cc)
        for (int l = 0; l < H; ++l)
          for (int m = 0; m < W; ++m) {
            int i = X0 - 2 + m, j = Y0 - 2 + l;
            if (in_store(s, i, j))
              *at(s, s->F[ORC_JX + cc], i, j) += Jp[(size_t)cc * W * H + l * W + m];
          }
    }
    apply_particle_bc(s);
    rebin(s);
    if (c->filter_passes > 0) filter_current(s);
    maxwell(s);
    s->step++;
    s->t += c->dt;
    if (c->mw_on && s->t > c->mw_t0 &&
        s->t - c->mw_t0 >= (s->nshift + 1) * (double)P * c->dx) {
      shift_window(s);
      s->have_rho_prev = 0;
    }
  }
  free(Jbuf);
  return bad ? -2 : 0;
}

int orc_diag(orc_state *s, double *out) {
  const orc_config *c = &s->c;
  const double dV = c->dx * c->dy;
  double UE = 0, UB = 0, UK = 0, qtot = 0;
  for (int j = 0; j < c->ny; ++j)
    for (int i = 0; i < c->nx; ++i)
      for (int k = 0; k < 3; ++k) {
        double e = *at(s, s->F[ORC_EX + k], i, j), b = *at(s, s->F[ORC_BMX + k], i, j);
        UE += 0.5 * e * e * dV;
        UB += 0.5 * b * b * dV;
      }
  for (long p = 0; p < s->np; ++p) {
    double g = sqrt(1.0 + s->ux[p] * s->ux[p] + s->uy[p] * s->uy[p] + s->uz[p] * s->uz[p]);
    UK += s->w[p] * (g - 1.0) * c->m * dV;
    qtot += c->q * s->w[p] * dV;
  }
  double *rho = calloc(s->ntot, sizeof(double));
  deposit_rho(s, rho, 1.0);
  int xl = c->fbc_x == ORC_FBC_PERIODIC ? 0 : 3, xh = c->fbc_x == ORC_FBC_PERIODIC ? c->nx : c->nx - 3;
  int yl = c->fbc_y == ORC_FBC_PERIODIC ? 0 : 3, yh = c->fbc_y == ORC_FBC_PERIODIC ? c->ny : c->ny - 3;
  double gauss = 0.0, cont = s->have_rho_prev ? 0.0 : NAN;
  for (int j = yl; j < yh; ++j)
    for (int i = xl; i < xh; ++i) {
      double divE = (*at(s, s->F[ORC_EX], i, j) - *at(s, s->F[ORC_EX], i - 1, j)) / c->dx +
                    (*at(s, s->F[ORC_EY], i, j) - *at(s, s->F[ORC_EY], i, j - 1)) / c->dy;
      double r = *at(s, rho, i, j) + *at(s, s->rho_bg, i, j);
      double gres = fabs(divE - r);
      if (gres > gauss) gauss = gres;
      if (s->have_rho_prev) {
        double divJ = (*at(s, s->F[ORC_JX], i, j) - *at(s, s->F[ORC_JX], i - 1, j)) / c->dx +
                      (*at(s, s->F[ORC_JY], i, j) - *at(s, s->F[ORC_JY], i, j - 1)) / c->dy;
        double cr = fabs((*at(s, rho, i, j) - *at(s, s->rho_prev, i, j)) / c->dt + divJ);
        if (cr > cont) cont = cr;
      }
    }
  free(rho);
  out[0] = (double)s->step;
  out[1] = s->t;
  out[2] = (double)s->np;
  out[3] = UE;
  out[4] = UB;
  out[5] = UK;
  out[6] = gauss;
  out[7] = cont;
  out[8] = (double)s->nshift;
  out[9] = qtot;
  return 0;
}
