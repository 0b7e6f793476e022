/*
 * Plain FP64 CPU oracle of the patch-decomposed 3D3V particle-in-cell step.
 * TEST INFRASTRUCTURE ONLY (see pic_oracle3d.h).
 *
 * One step, in the order of the SDMD loop (Section 2.2, Section 3.3):
 *   1. per patch (OpenMP over patches): interpolate E^n, Bm^n at x^n with
 *      the quadratic shape of each component's stagger, Boris push
 *      u^{n-1/2} -> u^{n+1/2}, move x^n -> x^{n+1}, Esirkepov current of
 *      the move into the patch's private buffer;
 *   2. SDMD step (i): patch buffers added into the region current in
 *      ascending patch order (independent of the thread count);
 *   3. particle boundary conditions, re-binning;
 *   4. Yee update of the region (E^{n+1}, B^{n+3/2}, Bm^{n+1}), then the
 *      Silver-Mueller ghost B of every open face, with the laser at x_min;
 *   5. moving-window shift when due.
 * SDMD step (ii) is the interpolation: patches read the region directly.
 */
#include "pic_oracle3d.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#include "pic_oracle.h" /* orc_shape2, orc_boris */

#define G 4
#define NF 12

/* stagger of component c along axis a: 1 = dual (half-integer) */
static const int STAG[NF][3] = {
    {1, 0, 0}, {0, 1, 0}, {0, 0, 1},  /* Ex Ey Ez */
    {0, 1, 1}, {1, 0, 1}, {1, 1, 0},  /* Bx By Bz */
    {0, 1, 1}, {1, 0, 1}, {1, 1, 0},  /* Bmx Bmy Bmz */
    {1, 0, 0}, {0, 1, 0}, {0, 0, 1}}; /* Jx Jy Jz */

struct o3_state {
  o3_config c;
  long sx, sy, ntot;  /* strides: x fastest, then y, then z */
  double *F[NF];
  double *rho_bg, *rho_prev;
  int have_rho_prev;
  long np, cap;
  double *x[3], *u[3], *w;
  int *pid;
  long *pstart;
  int np_[3], npatch;
  long step;
  double t;
  int nshift;
};

static int imod(int a, int n) { int r = a % n; return r < 0 ? r + n : r; }

static long idx(const o3_state *s, int i, int j, int k) {
  if (s->c.fbc[0] == 0) i = imod(i, s->c.n[0]);
  if (s->c.fbc[1] == 0) j = imod(j, s->c.n[1]);
  if (s->c.fbc[2] == 0) k = imod(k, s->c.n[2]);
  return ((long)(k + G) * s->sy + (j + G)) * s->sx + (i + G);
}

static int in_store(const o3_state *s, int i, int j, int k) {
  const int v[3] = {i, j, k};
  for (int a = 0; a < 3; ++a)
    if (s->c.fbc[a] != 0 && (v[a] < -G || v[a] >= s->c.n[a] + G)) return 0;
  return 1;
}

#define AT(s, arr, i, j, k) ((arr)[idx((s), (i), (j), (k))])

static double gather(const o3_state *s, int comp, const double x[3]) {
  int i0[3];
  double S[3][3], v = 0.0;
  for (int a = 0; a < 3; ++a) orc_shape2(x[a] / s->c.d[a] - 0.5 * STAG[comp][a], &i0[a], S[a]);
  for (int c = 0; c < 3; ++c)
    for (int b = 0; b < 3; ++b)
      for (int a = 0; a < 3; ++a)
        v += S[0][a] * S[1][b] * S[2][c] *
             AT(s, s->F[comp], i0[0] - 1 + a, i0[1] - 1 + b, i0[2] - 1 + c);
  return v;
}

double o3_gather(const o3_state *s, int comp, double x, double y, double z) {
  if (comp < 0 || comp >= NF) return NAN;
  const double p[3] = {x, y, z};
  return gather(s, comp, p);
}

/* Esirkepov (2001) in 3D: with S0, S1 the shapes at x^n, x^{n+1} on a
 * common 5-node window per axis and DS = S1 - S0,
 *   W_x = DSx (S0y S0z + DSy S0z / 2 + S0y DSz / 2 + DSy DSz / 3)
 * (and cyclically W_y, W_z); J_a = -q w (d_a / dt) x prefix sum of W_a
 * along axis a. */
int o3_esirkepov(const o3_state *s, const double x0[3], const double x1[3], double w,
                 int ix[3], double Jw[3][5][5][5]) {
  double S0[3][5], S1[3][5], DS[3][5], S[3];
  int i0, i1;
  for (int a = 0; a < 3; ++a) {
    for (int k = 0; k < 5; ++k) S0[a][k] = S1[a][k] = 0.0;
    orc_shape2(x0[a] / s->c.d[a], &i0, S);
    for (int k = 0; k < 3; ++k) S0[a][1 + k] = S[k];
    orc_shape2(x1[a] / s->c.d[a], &i1, S);
    if (i1 - i0 < -1 || i1 - i0 > 1) return -1;
    for (int k = 0; k < 3; ++k) S1[a][1 + (i1 - i0) + k] = S[k];
    for (int k = 0; k < 5; ++k) DS[a][k] = S1[a][k] - S0[a][k];
    ix[a] = i0 - 2;
  }
  const double q = s->c.q;
  for (int c = 0; c < 3; ++c) {
    const int b = (c + 1) % 3, e = (c + 2) % 3; /* the two other axes */
    const double coef = -q * w * s->c.d[c] / s->c.dt;
    /* n[c] runs along the prefix-sum axis, n[b], n[e] across it */
    for (int nb = 0; nb < 5; ++nb)
      for (int ne = 0; ne < 5; ++ne) {
        const double A = S0[b][nb] * S0[e][ne] + 0.5 * DS[b][nb] * S0[e][ne] +
                         0.5 * S0[b][nb] * DS[e][ne] + (1.0 / 3.0) * DS[b][nb] * DS[e][ne];
        double acc = 0.0;
        for (int nc = 0; nc < 5; ++nc) {
          acc += DS[c][nc] * A;
          int n3[3];
          n3[c] = nc;
          n3[b] = nb;
          n3[e] = ne;
          Jw[c][n3[2]][n3[1]][n3[0]] += coef * acc;
        }
      }
  }
  return 0;
}

int o3_laser_field(const o3_state *s, double y, double z, double t, double *ey) {
  const o3_config *c = &s->c;
  const double tr = t - s->nshift * c->p[0] * c->d[0] - c->t_peak;
  const double ry = (y - c->y_center) / c->waist, rz = (z - c->z_center) / c->waist;
  *ey = c->a0 * exp(-(ry * ry + rz * rz)) * exp(-2.0 * log(2.0) * tr * tr / (c->tau * c->tau)) *
        sin(tr);
  return 0;
}

static double profile(const o3_config *c, double xphys) {
  if (c->inj_ramp <= 0.0) return xphys >= c->inj_x0 ? c->inj_n0 : 0.0;
  double f = (xphys - c->inj_x0) / c->inj_ramp;
  if (f < 0.0) f = 0.0;
  if (f > 1.0) f = 1.0;
  return c->inj_n0 * f;
}

static int patch_of(const o3_state *s, long p) {
  int pc[3];
  for (int a = 0; a < 3; ++a) {
    int cell = (int)floor(s->x[a][p] / s->c.d[a]);
    int q = cell / s->c.p[a];
    if (q < 0) q = 0;
    if (q >= s->np_[a]) q = s->np_[a] - 1;
    pc[a] = q;
  }
  return (pc[2] * s->np_[1] + pc[1]) * s->np_[0] + pc[0];
}

static double **arrays(o3_state *s, double *out[7]) {
  out[0] = s->x[0]; out[1] = s->x[1]; out[2] = s->x[2];
  out[3] = s->u[0]; out[4] = s->u[1]; out[5] = s->u[2];
  out[6] = s->w;
  return out;
}

static void rebin(o3_state *s) {
  const long np = s->np;
  long *cnt = calloc(s->npatch + 1, sizeof(long));
  for (long i = 0; i < np; ++i) {
    s->pid[i] = patch_of(s, i);
    cnt[s->pid[i] + 1]++;
  }
  for (int p = 0; p < s->npatch; ++p) cnt[p + 1] += cnt[p];
  memcpy(s->pstart, cnt, (s->npatch + 1) * sizeof(long));
  double *arr[7];
  arrays(s, arr);
  const long m = np > 0 ? np : 1;
  double *tmp = malloc(m * sizeof(double));
  long *dst = malloc(m * sizeof(long));
  int *pid2 = malloc(m * sizeof(int));
  for (long i = 0; i < np; ++i) dst[i] = cnt[s->pid[i]]++;
  for (int a = 0; a < 7; ++a) {
    for (long i = 0; i < np; ++i) tmp[dst[i]] = arr[a][i];
    memcpy(arr[a], tmp, np * sizeof(double));
  }
  for (long i = 0; i < np; ++i) pid2[dst[i]] = s->pid[i];
  memcpy(s->pid, pid2, np * sizeof(int));
  free(tmp);
  free(dst);
  free(pid2);
  free(cnt);
}

static int grow(o3_state *s, long need) {
  if (need <= s->cap) return 0;
  const long cap = need + need / 2 + 16;
  double **arr[7] = {&s->x[0], &s->x[1], &s->x[2], &s->u[0], &s->u[1], &s->u[2], &s->w};
  for (int a = 0; a < 7; ++a) {
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

o3_state *o3_create(const o3_config *c) {
  for (int a = 0; a < 3; ++a)
    if (c->n[a] <= 0 || c->p[a] <= 0 || c->n[a] % c->p[a]) return NULL;
  o3_state *s = calloc(1, sizeof(o3_state));
  s->c = *c;
  s->sx = c->n[0] + 2 * G;
  s->sy = c->n[1] + 2 * G;
  s->ntot = s->sx * s->sy * (c->n[2] + 2 * G);
  for (int k = 0; k < NF; ++k) s->F[k] = calloc(s->ntot, sizeof(double));
  s->rho_bg = calloc(s->ntot, sizeof(double));
  s->rho_prev = calloc(s->ntot, sizeof(double));
  for (int a = 0; a < 3; ++a) s->np_[a] = c->n[a] / c->p[a];
  s->npatch = s->np_[0] * s->np_[1] * s->np_[2];
  s->pstart = calloc(s->npatch + 1, sizeof(long));
  return s;
}

void o3_destroy(o3_state *s) {
  if (!s) return;
  for (int k = 0; k < NF; ++k) free(s->F[k]);
  free(s->rho_bg);
  free(s->rho_prev);
  for (int a = 0; a < 3; ++a) { free(s->x[a]); free(s->u[a]); }
  free(s->w);
  free(s->pid);
  free(s->pstart);
  free(s);
}

int o3_load(o3_state *s, const double *x, const double *y, const double *z, const double *ux,
            const double *uy, const double *uz, const double *w, long n) {
  if (grow(s, s->np + n)) return -1;
  for (long i = 0; i < n; ++i) {
    const long k = s->np + i;
    s->x[0][k] = x[i]; s->x[1][k] = y[i]; s->x[2][k] = z[i];
    s->u[0][k] = ux[i]; s->u[1][k] = uy[i]; s->u[2][k] = uz[i];
    s->w[k] = w[i];
  }
  s->np += n;
  rebin(s);
  return 0;
}

long o3_num_particles(const o3_state *s) { return s->np; }

long o3_get_particles(const o3_state *s, double *out) {
  double *arr[7];
  arrays((o3_state *)s, arr);
  for (int a = 0; a < 7; ++a) memcpy(out + a * s->np, arr[a], s->np * sizeof(double));
  return s->np;
}

static void out_range(int fbc, int n, int *lo, int *cnt) {
  if (fbc == 0) { *lo = 0; *cnt = n; }
  else { *lo = -1; *cnt = n + 2; }
}

/* rho += sign q w S(x) S(y) S(z) at nodes, for particles [first, last). */
static void deposit_rho(const o3_state *s, double *rho, double sign, long first, long last) {
  for (long p = first; p < last; ++p) {
    int i0[3];
    double S[3][3];
    for (int a = 0; a < 3; ++a) orc_shape2(s->x[a][p] / s->c.d[a], &i0[a], S[a]);
    for (int c = 0; c < 3; ++c)
      for (int b = 0; b < 3; ++b)
        for (int a = 0; a < 3; ++a) {
          const int i = i0[0] - 1 + a, j = i0[1] - 1 + b, k = i0[2] - 1 + c;
          if (in_store(s, i, j, k))
            AT(s, rho, i, j, k) += sign * s->c.q * s->w[p] * S[0][a] * S[1][b] * S[2][c];
        }
  }
}

static double *comp_array(o3_state *s, int comp, int *owned) {
  *owned = 0;
  if (comp < NF) return s->F[comp];
  if (comp == O3_RHO_BG) return s->rho_bg;
  if (comp == O3_RHO) {
    double *r = calloc(s->ntot, sizeof(double));
    deposit_rho(s, r, 1.0, 0, s->np);
    *owned = 1;
    return r;
  }
  return NULL;
}

int o3_set_field(o3_state *s, int comp, const double *src) {
  if (comp < 0 || comp >= O3_NOUT || comp == O3_RHO) return -1;
  double *a = comp == O3_RHO_BG ? s->rho_bg : s->F[comp];
  int lo[3], cnt[3];
  for (int d = 0; d < 3; ++d) out_range(s->c.fbc[d], s->c.n[d], &lo[d], &cnt[d]);
  for (int k = 0; k < cnt[2]; ++k)
    for (int j = 0; j < cnt[1]; ++j)
      for (int i = 0; i < cnt[0]; ++i)
        AT(s, a, lo[0] + i, lo[1] + j, lo[2] + k) = src[((long)k * cnt[1] + j) * cnt[0] + i];
  return 0;
}

int o3_get_field(o3_state *s, int comp, double *dst) {
  int owned;
  if (comp < 0 || comp >= O3_NOUT) return -1;
  double *a = comp_array(s, comp, &owned);
  int lo[3], cnt[3];
  for (int d = 0; d < 3; ++d) out_range(s->c.fbc[d], s->c.n[d], &lo[d], &cnt[d]);
  for (int k = 0; k < cnt[2]; ++k)
    for (int j = 0; j < cnt[1]; ++j)
      for (int i = 0; i < cnt[0]; ++i)
        dst[((long)k * cnt[1] + j) * cnt[0] + i] = AT(s, a, lo[0] + i, lo[1] + j, lo[2] + k);
  if (owned) free(a);
  return 0;
}

int o3_set_background(o3_state *s, int mode, double value) {
  memset(s->rho_bg, 0, s->ntot * sizeof(double));
  if (mode == 1) {
    for (long e = 0; e < s->ntot; ++e) s->rho_bg[e] = value;
  } else if (mode == 2) {
    deposit_rho(s, s->rho_bg, -1.0, 0, s->np);
  } else if (mode != 0) {
    return -1;
  }
  return 0;
}

/* Regular plasma at rest in cells [i_lo, i_hi) x all y with centre
 * y >= inj_ymin x all z, weight n(x_lab) / ppc; appended to the particles,
 * and its immobile ions added to the background charge. */
static void add_plasma(o3_state *s, int i_lo, int i_hi) {
  const o3_config *c = &s->c;
  const int ppc = c->inj_ppc[0] * c->inj_ppc[1] * c->inj_ppc[2];
  const long first = s->np;
  long n = 0;
  for (int j = 0; j < c->n[1]; ++j)
    if ((j + 0.5) * c->d[1] >= c->inj_ymin) n += (long)(i_hi - i_lo) * c->n[2] * ppc;
  grow(s, s->np + n);
  long k = s->np;
  const double shift = (double)s->nshift * c->p[0] * c->d[0];
  for (int kk = 0; kk < c->n[2]; ++kk)
    for (int j = 0; j < c->n[1]; ++j) {
      if (!((j + 0.5) * c->d[1] >= c->inj_ymin)) continue;
      for (int i = i_lo; i < i_hi; ++i)
        for (int cz = 0; cz < c->inj_ppc[2]; ++cz)
          for (int cy = 0; cy < c->inj_ppc[1]; ++cy)
            for (int cx = 0; cx < c->inj_ppc[0]; ++cx) {
              const double xl = (i + (cx + 0.5) / c->inj_ppc[0]) * c->d[0];
              s->x[0][k] = xl;
              s->x[1][k] = (j + (cy + 0.5) / c->inj_ppc[1]) * c->d[1];
              s->x[2][k] = (kk + (cz + 0.5) / c->inj_ppc[2]) * c->d[2];
              s->u[0][k] = s->u[1][k] = s->u[2][k] = 0.0;
              s->w[k] = profile(c, xl + shift) / ppc;
              ++k;
            }
    }
  s->np = k;
  deposit_rho(s, s->rho_bg, -1.0, first, s->np);
}

int o3_fill_plasma(o3_state *s) {
  add_plasma(s, 0, s->c.n[0]);
  rebin(s);
  return 0;
}

static void upd_range(int fbc, int n, int dual, int *lo, int *hi) {
  *lo = 0;
  *hi = fbc == 0 ? n : (dual ? n : n + 1);
}

/* Loop over the update range of component comp. */
#define FOR_RANGE(s, comp, i, j, k)                                              \
  int lo_[3], hi_[3];                                                            \
  for (int a_ = 0; a_ < 3; ++a_)                                                 \
    upd_range((s)->c.fbc[a_], (s)->c.n[a_], STAG[comp][a_], &lo_[a_], &hi_[a_]); \
  _Pragma("omp parallel for") for (int k = lo_[2]; k < hi_[2]; ++k)              \
    for (int j = lo_[1]; j < hi_[1]; ++j)                                        \
      for (int i = lo_[0]; i < hi_[0]; ++i)

/* Ghost B of one open face (axis a, lower or upper) for the pair (E_c,
 * B_d), from the first-order Silver-Mueller condition taken half a step
 * ahead of E^{n+1} with Ampere's law on the boundary node:
 *   lower: G = [2 e + dt T - s (1 - r) I - 4 e_inc] / (s (1 + r))
 *   upper: G = -[2 e + dt T + s (1 - r) I] / (s (1 + r))
 * with r = dt / d_a, s = +1 when (curl B)_c holds +d_a B_d, -1 when it holds
 * -d_a B_d, T = -s d_b B_a the transverse part of (curl B)_c (b the third
 * axis; taken as zero where it would need a ghost of another open axis),
 * I the B_d value just inside, e = E_c^{n+1} on the face. */
static void sm_face(o3_state *s, int a, int upper, int c, double tB) {
  const o3_config *cf = &s->c;
  /* the ghost component's axis d is the third axis (neither a nor c) */
  int s_sign, d;
  if ((c + 1) % 3 == a) { s_sign = 1; d = (c + 2) % 3; }
  else { s_sign = -1; d = (c + 1) % 3; }
  const int b = d;
  const double r = cf->dt / cf->d[a];
  double *E = s->F[O3_EX + c], *Bd = s->F[O3_BX + d], *Ba = s->F[O3_BX + a];
  /* transverse ranges of the ghost B_d: primal along its own axis d */
  int lo[3] = {0, 0, 0}, hi[3];
  for (int e = 0; e < 3; ++e) hi[e] = (cf->fbc[e] == 0 || e != d) ? cf->n[e] : cf->n[e] + 1;
  lo[a] = hi[a] = 0;
  hi[a] = 1;
  for (int k = lo[2]; k < hi[2]; ++k)
    for (int j = lo[1]; j < hi[1]; ++j)
      for (int i = lo[0]; i < hi[0]; ++i) {
        int node[3] = {i, j, k}, gh[3] = {i, j, k}, in[3] = {i, j, k};
        node[a] = upper ? cf->n[a] : 0;
        gh[a] = upper ? cf->n[a] : -1;
        in[a] = upper ? cf->n[a] - 1 : 0;
        double T = 0.0;
        const int nb = node[b];
        const int interior = cf->fbc[b] == 0 || (nb >= 1 && nb <= cf->n[b] - 1);
        if (interior) {
          int m[3] = {node[0], node[1], node[2]};
          m[b] -= 1;
          T = -s_sign * (AT(s, Ba, node[0], node[1], node[2]) - AT(s, Ba, m[0], m[1], m[2])) /
              cf->d[b];
        }
        const double e = AT(s, E, node[0], node[1], node[2]);
        const double I = AT(s, Bd, in[0], in[1], in[2]);
        double ghost;
        if (!upper) {
          double einc = 0.0;
          if (cf->laser_on && a == 0 && c == 1)
            o3_laser_field(s, (node[1] + 0.5) * cf->d[1], node[2] * cf->d[2], tB, &einc);
          ghost = (2.0 * e + cf->dt * T - s_sign * (1.0 - r) * I - 4.0 * einc) / (s_sign * (1.0 + r));
        } else {
          ghost = -(2.0 * e + cf->dt * T + s_sign * (1.0 - r) * I) / (s_sign * (1.0 + r));
        }
        AT(s, Bd, gh[0], gh[1], gh[2]) = ghost;
      }
}

/* Yee update of the region (Section 3.2), 3D:
 *   E^{n+1} = E^n + dt (curl B^{n+1/2} - J^{n+1/2}),
 *   B^{n+3/2} = B^{n+1/2} - dt curl E^{n+1},  Bm^{n+1} = average,
 * then the Silver-Mueller ghosts of the open faces. */
static void maxwell(o3_state *s) {
  const o3_config *c = &s->c;
  const double dt = c->dt, dx = c->d[0], dy = c->d[1], dz = c->d[2];
  double *Ex = s->F[O3_EX], *Ey = s->F[O3_EY], *Ez = s->F[O3_EZ];
  double *Bx = s->F[O3_BX], *By = s->F[O3_BY], *Bz = s->F[O3_BZ];
  double *Jx = s->F[O3_JX], *Jy = s->F[O3_JY], *Jz = s->F[O3_JZ];
  {
    FOR_RANGE(s, O3_EX, i, j, k)
    AT(s, Ex, i, j, k) += dt * ((AT(s, Bz, i, j, k) - AT(s, Bz, i, j - 1, k)) / dy -
                                (AT(s, By, i, j, k) - AT(s, By, i, j, k - 1)) / dz -
                                AT(s, Jx, i, j, k));
  }
  {
    FOR_RANGE(s, O3_EY, i, j, k)
    AT(s, Ey, i, j, k) += dt * ((AT(s, Bx, i, j, k) - AT(s, Bx, i, j, k - 1)) / dz -
                                (AT(s, Bz, i, j, k) - AT(s, Bz, i - 1, j, k)) / dx -
                                AT(s, Jy, i, j, k));
  }
  {
    FOR_RANGE(s, O3_EZ, i, j, k)
    AT(s, Ez, i, j, k) += dt * ((AT(s, By, i, j, k) - AT(s, By, i - 1, j, k)) / dx -
                                (AT(s, Bx, i, j, k) - AT(s, Bx, i, j - 1, k)) / dy -
                                AT(s, Jz, i, j, k));
  }
  memcpy(s->F[O3_BMX], Bx, s->ntot * sizeof(double));
  memcpy(s->F[O3_BMY], By, s->ntot * sizeof(double));
  memcpy(s->F[O3_BMZ], Bz, s->ntot * sizeof(double));
  {
    FOR_RANGE(s, O3_BX, i, j, k)
    AT(s, Bx, i, j, k) -= dt * ((AT(s, Ez, i, j + 1, k) - AT(s, Ez, i, j, k)) / dy -
                                (AT(s, Ey, i, j, k + 1) - AT(s, Ey, i, j, k)) / dz);
  }
  {
    FOR_RANGE(s, O3_BY, i, j, k)
    AT(s, By, i, j, k) -= dt * ((AT(s, Ex, i, j, k + 1) - AT(s, Ex, i, j, k)) / dz -
                                (AT(s, Ez, i + 1, j, k) - AT(s, Ez, i, j, k)) / dx);
  }
  {
    FOR_RANGE(s, O3_BZ, i, j, k)
    AT(s, Bz, i, j, k) -= dt * ((AT(s, Ey, i + 1, j, k) - AT(s, Ey, i, j, k)) / dx -
                                (AT(s, Ex, i, j + 1, k) - AT(s, Ex, i, j, k)) / dy);
  }
  const double tB = s->t + 1.5 * dt;
  for (int a = 0; a < 3; ++a) {
    if (c->fbc[a] == 0) continue;
    for (int upper = 0; upper < 2; ++upper)
      for (int comp = 0; comp < 3; ++comp)
        if (comp != a) sm_face(s, a, upper, comp, tB);
  }
  for (int k = 0; k < 3; ++k) {
    double *bm = s->F[O3_BMX + k], *b = s->F[O3_BX + k];
    for (long e = 0; e < s->ntot; ++e) bm[e] = 0.5 * (bm[e] + b[e]);
  }
}

static void shift_window(o3_state *s) {
  const o3_config *c = &s->c;
  const int P = c->p[0], nx = c->n[0];
  double *arrs[NF + 1];
  for (int k = 0; k < NF; ++k) arrs[k] = s->F[k];
  arrs[NF] = s->rho_bg;
  for (int q = 0; q < NF + 1; ++q)
    for (int k = -G; k < c->n[2] + G; ++k)
      for (int j = -G; j < c->n[1] + G; ++j) {
        double *row = &arrs[q][((long)(k + G) * s->sy + (j + G)) * s->sx];
        for (int i = -G; i < nx + G; ++i) row[i + G] = (i + P < nx + G) ? row[i + P + G] : 0.0;
      }
  s->nshift++;
  long k = 0;
  for (long p = 0; p < s->np; ++p) {
    const double xn = s->x[0][p] - P * c->d[0];
    if (xn < 0.0) continue;
    s->x[0][k] = xn; s->x[1][k] = s->x[1][p]; s->x[2][k] = s->x[2][p];
    s->u[0][k] = s->u[0][p]; s->u[1][k] = s->u[1][p]; s->u[2][k] = s->u[2][p];
    s->w[k] = s->w[p];
    ++k;
  }
  s->np = k;
  add_plasma(s, nx - P, nx);
  rebin(s);
}

static void apply_particle_bc(o3_state *s) {
  const o3_config *c = &s->c;
  long k = 0;
  for (long p = 0; p < s->np; ++p) {
    int drop = 0;
    double v[3] = {s->x[0][p], s->x[1][p], s->x[2][p]};
    for (int a = 0; a < 3 && !drop; ++a) {
      const double L = c->n[a] * c->d[a];
      if (v[a] < 0.0 || v[a] >= L) {
        const int bc = v[a] < 0.0 ? c->pbc[a][0] : c->pbc[a][1];
        if (bc == 0) v[a] += (v[a] < 0.0 ? L : -L);
        else if (bc == 1) { v[a] = v[a] < 0.0 ? -v[a] : 2.0 * L - v[a]; s->u[a][p] = -s->u[a][p]; }
        else drop = 1;
      }
    }
    if (drop) continue;
    for (int a = 0; a < 3; ++a) { s->x[a][k] = v[a]; s->u[a][k] = s->u[a][p]; }
    s->w[k] = s->w[p];
    ++k;
  }
  s->np = k;
}

int o3_step(o3_state *s, int nsteps) {
  const o3_config *c = &s->c;
  const int W[3] = {c->p[0] + 5, c->p[1] + 5, c->p[2] + 5};
  const size_t per = (size_t)W[0] * W[1] * W[2];
  double *Jbuf = malloc((size_t)s->npatch * 3 * per * sizeof(double));
  int bad = 0;
#ifdef _OPENMP
  if (c->nthreads > 0) omp_set_num_threads(c->nthreads);
#endif
  if (!Jbuf) return -3;
  for (int n = 0; n < nsteps; ++n) {
    if (c->track_continuity) {
      memset(s->rho_prev, 0, s->ntot * sizeof(double));
      deposit_rho(s, s->rho_prev, 1.0, 0, s->np);
      s->have_rho_prev = 1;
    }
    for (int q = O3_JX; q <= O3_JZ; ++q) memset(s->F[q], 0, s->ntot * sizeof(double));
    memset(Jbuf, 0, (size_t)s->npatch * 3 * per * sizeof(double));
#pragma omp parallel for schedule(dynamic) reduction(| : bad)
    for (int p = 0; p < s->npatch; ++p) {
      const int pc[3] = {p % s->np_[0], (p / s->np_[0]) % s->np_[1], p / (s->np_[0] * s->np_[1])};
      int X0[3];
      for (int a = 0; a < 3; ++a) X0[a] = pc[a] * c->p[a];
      double *Jp = Jbuf + (size_t)p * 3 * per;
      for (long q = s->pstart[p]; q < s->pstart[p + 1]; ++q) {
        double E[3], B[3], u[3] = {s->u[0][q], s->u[1][q], s->u[2][q]};
        const double x0[3] = {s->x[0][q], s->x[1][q], s->x[2][q]};
        for (int a = 0; a < 3; ++a) {
          E[a] = gather(s, O3_EX + a, x0);
          B[a] = gather(s, O3_BMX + a, x0);
        }
        orc_boris(c->q, c->m, c->dt, E, B, u);
        const double g = sqrt(1.0 + u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
        double x1[3];
        for (int a = 0; a < 3; ++a) x1[a] = x0[a] + c->dt * u[a] / g;
        double Jw[3][5][5][5];
        int ix[3];
        memset(Jw, 0, sizeof Jw);
        if (o3_esirkepov(s, x0, x1, s->w[q], ix, Jw)) { bad = 1; continue; }
        int o[3], outside = 0;
        for (int a = 0; a < 3; ++a) {
          o[a] = ix[a] - (X0[a] - 2);
          if (o[a] < 0 || o[a] + 5 > W[a]) outside = 1;
        }
        if (outside) { bad = 1; continue; }
        for (int cc = 0; cc < 3; ++cc)
          for (int kk = 0; kk < 5; ++kk)
            for (int jj = 0; jj < 5; ++jj)
              for (int ii = 0; ii < 5; ++ii)
                Jp[cc * per + ((size_t)(o[2] + kk) * W[1] + o[1] + jj) * W[0] + o[0] + ii] +=
                    Jw[cc][kk][jj][ii];
        for (int a = 0; a < 3; ++a) { s->x[a][q] = x1[a]; s->u[a][q] = u[a]; }
      }
    }
    /* SDMD step (i): patch buffers -> region, ascending patch order */
    for (int p = 0; p < s->npatch; ++p) {
      const int pc[3] = {p % s->np_[0], (p / s->np_[0]) % s->np_[1], p / (s->np_[0] * s->np_[1])};
      const double *Jp = Jbuf + (size_t)p * 3 * per;
      for (int cc = 0; cc < 3; ++cc)
        for (int kk = 0; kk < W[2]; ++kk)
          for (int jj = 0; jj < W[1]; ++jj)
            for (int ii = 0; ii < W[0]; ++ii) {
              const int i = pc[0] * c->p[0] - 2 + ii, j = pc[1] * c->p[1] - 2 + jj,
                        k = pc[2] * c->p[2] - 2 + kk;
              if (in_store(s, i, j, k))
                AT(s, s->F[O3_JX + cc], i, j, k) += Jp[cc * per + ((size_t)kk * W[1] + jj) * W[0] + ii];
            }
    }
    apply_particle_bc(s);
    rebin(s);
    maxwell(s);
    s->step++;
    s->t += c->dt;
    if (c->mw_on && s->t > c->mw_t0 &&
        s->t - c->mw_t0 >= (s->nshift + 1) * (double)c->p[0] * c->d[0]) {
      shift_window(s);
      s->have_rho_prev = 0;
    }
  }
  free(Jbuf);
  return bad ? -2 : 0;
}

int o3_diag(o3_state *s, double *out) {
  const o3_config *c = &s->c;
  const double dV = c->d[0] * c->d[1] * c->d[2];
  double UE = 0, UB = 0, UK = 0, qtot = 0;
  for (int k = 0; k < c->n[2]; ++k)
    for (int j = 0; j < c->n[1]; ++j)
      for (int i = 0; i < c->n[0]; ++i)
        for (int q = 0; q < 3; ++q) {
          const double e = AT(s, s->F[O3_EX + q], i, j, k), b = AT(s, s->F[O3_BMX + q], i, j, k);
          UE += 0.5 * e * e * dV;
          UB += 0.5 * b * b * dV;
        }
  for (long p = 0; p < s->np; ++p) {
    const double g = sqrt(1.0 + s->u[0][p] * s->u[0][p] + s->u[1][p] * s->u[1][p] +
                          s->u[2][p] * s->u[2][p]);
    UK += s->w[p] * (g - 1.0) * c->m * dV;
    qtot += c->q * s->w[p] * dV;
  }
  double *rho = calloc(s->ntot, sizeof(double));
  deposit_rho(s, rho, 1.0, 0, s->np);
  int lo[3], hi[3];
  for (int a = 0; a < 3; ++a) {
    lo[a] = c->fbc[a] == 0 ? 0 : 3;
    hi[a] = c->fbc[a] == 0 ? c->n[a] : c->n[a] - 3;
  }
  double gauss = 0.0, cont = s->have_rho_prev ? 0.0 : NAN;
  for (int k = lo[2]; k < hi[2]; ++k)
    for (int j = lo[1]; j < hi[1]; ++j)
      for (int i = lo[0]; i < hi[0]; ++i) {
        const double divE =
            (AT(s, s->F[O3_EX], i, j, k) - AT(s, s->F[O3_EX], i - 1, j, k)) / c->d[0] +
            (AT(s, s->F[O3_EY], i, j, k) - AT(s, s->F[O3_EY], i, j - 1, k)) / c->d[1] +
            (AT(s, s->F[O3_EZ], i, j, k) - AT(s, s->F[O3_EZ], i, j, k - 1)) / c->d[2];
        const double g = fabs(divE - AT(s, rho, i, j, k) - AT(s, s->rho_bg, i, j, k));
        if (g > gauss) gauss = g;
        if (s->have_rho_prev) {
          const double divJ =
              (AT(s, s->F[O3_JX], i, j, k) - AT(s, s->F[O3_JX], i - 1, j, k)) / c->d[0] +
              (AT(s, s->F[O3_JY], i, j, k) - AT(s, s->F[O3_JY], i, j - 1, k)) / c->d[1] +
              (AT(s, s->F[O3_JZ], i, j, k) - AT(s, s->F[O3_JZ], i, j, k - 1)) / c->d[2];
          const double cr = fabs((AT(s, rho, i, j, k) - AT(s, s->rho_prev, i, j, k)) / c->dt + divJ);
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
