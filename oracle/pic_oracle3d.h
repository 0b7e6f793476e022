/*
 * Plain FP64 CPU oracle of the patch-decomposed 3D3V particle-in-cell step.
 *
 * TEST INFRASTRUCTURE ONLY, like pic_oracle.h: loaded by the test-suite, the
 * smoke check and the CPU-baseline leg of the benchmark; never by the
 * product library, with which it shares no code, header, table or helper.
 *
 * The 3D restatement of the same loop (Section 2.2 steps (i) and (ii),
 * Section 3.2 operators, Section 3.3 phases): Yee lattice with E and J on
 * cell edges and B on cell faces, quadratic shape per axis, Boris push,
 * Esirkepov charge-conserving current with prefix sums along each axis,
 * per-patch current buffers reduced into the region in ascending patch
 * order, Silver-Mueller open faces with a y-polarised laser at x_min,
 * moving window along x.  The quadratic shape and the Boris push are the
 * 2D oracle's (orc_shape2, orc_boris), which its pins fix.
 *
 * Stagger (1 = dual along that axis):
 *   Ex (1,0,0) Ey (0,1,0) Ez (0,0,1); Bx (0,1,1) By (1,0,1) Bz (1,1,0);
 *   J like E, Bm like B, rho at nodes.
 * Field layout of o3_get_field / o3_set_field: (nz_e, ny_e, nx_e) row-major,
 * per axis n_e = n (periodic, indices [0, n)) or n + 2 (open, [-1, n]).
 */
#ifndef PIC_ORACLE3D_H
#define PIC_ORACLE3D_H
#ifdef __cplusplus
extern "C" {
#endif

enum { O3_EX = 0, O3_EY, O3_EZ, O3_BX, O3_BY, O3_BZ, O3_BMX, O3_BMY, O3_BMZ,
       O3_JX, O3_JY, O3_JZ, O3_RHO, O3_RHO_BG, O3_NOUT };

typedef struct {
  int n[3];              /* cells per axis */
  double d[3], dt;
  int p[3];              /* patch size in cells per axis */
  int fbc[3];            /* field BC per axis: 0 periodic, 1 Silver-Mueller */
  int pbc[3][2];         /* particle BC per face: 0 periodic, 1 reflect, 2 remove */
  double q, m;
  int laser_on;          /* y-polarised Gaussian laser through x_min */
  double a0, waist, tau, t_peak, y_center, z_center;
  int mw_on;             /* moving window along +x at c */
  double mw_t0;
  double inj_n0, inj_x0, inj_ramp;  /* plasma profile along x (lab frame) */
  double inj_ymin;       /* plasma only in cells whose centre has y >= inj_ymin */
  int inj_ppc[3];        /* regularly placed particles per cell per axis */
  int track_continuity;
  int nthreads;
} o3_config;

typedef struct o3_state o3_state;

o3_state *o3_create(const o3_config *c);
void o3_destroy(o3_state *s);
int o3_load(o3_state *s, const double *x, const double *y, const double *z,
            const double *ux, const double *uy, const double *uz, const double *w, long n);
/* Fill the whole domain with the configured plasma at rest (the profile the
 * moving window injects) and add its immobile ions to the background. */
int o3_fill_plasma(o3_state *s);
long o3_num_particles(const o3_state *s);
/* out: 7 x n rows (x, y, z, ux, uy, uz, w), in patch order.  Returns n. */
long o3_get_particles(const o3_state *s, double *out);
int o3_set_field(o3_state *s, int comp, const double *src);
int o3_get_field(o3_state *s, int comp, double *dst);
/* mode 0 none, 1 uniform value, 2 neutralising the loaded particles */
int o3_set_background(o3_state *s, int mode, double value);
int o3_step(o3_state *s, int nsteps);
/* out[0..9]: step, t, Np, U_E, U_B, U_K, gauss, continuity (NaN if not
 * available), window shifts, total charge */
int o3_diag(o3_state *s, double *out);
/* Esirkepov current of one particle moving x0 -> x1 (global positions) on
 * the 5-node windows starting at i0(x0) - 2 per axis: Jw[c][k][j][i] is
 * component c at window node (i, j, k) (dual along c); ix receives the
 * window's first node per axis.  -1 if a move exceeds one cell. */
int o3_esirkepov(const o3_state *s, const double x0[3], const double x1[3], double w,
                 int ix[3], double Jw[3][5][5][5]);
double o3_gather(const o3_state *s, int comp, double x, double y, double z);
int o3_laser_field(const o3_state *s, double y, double z, double t, double *ey);

#ifdef __cplusplus
}
#endif
#endif
