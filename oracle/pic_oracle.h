/*
 * Plain FP64 CPU oracle of the patch-decomposed 2D3V particle-in-cell step.
 *
 * TEST INFRASTRUCTURE ONLY.  This file and pic_oracle.c are the slow,
 * obviously-correct restatement of the method against which the CUDA path is
 * checked.  Only the test-suite, the smoke check and the CPU-baseline leg of
 * the benchmark may load it; the product library never links or calls it, and
 * the two share no code, header, table or helper.
 *
 * What it computes (the paper names the operators, it does not write them):
 *   - Section 2.2: particles live in small patches, fields in one region;
 *     two extra steps: (i) patch -> region current reduction after
 *     deposition, (ii) region -> patch field communication after Maxwell.
 *   - Section 3.2: Yee-lattice finite-difference Maxwell solver; Esirkepov
 *     charge-conserving deposition with the second-order (3-node, "5-point
 *     stencil") shape; interpolation / push / deposition as the particle
 *     phase (Section 3.3).
 *   - The pusher is not named in the paper; the Boris scheme is used.
 * Normalised units: lengths c/w, time 1/w, u = p/(mc), fields m c w / e,
 * densities n_c; dE/dt = curl B - J, dB/dt = -curl E, div E = rho.
 *
 * Field layout returned by orc_get_field: (ny_e, nx_e) row-major, where per
 * axis n_e = n (periodic) covering indices [0, n) or n_e = n + 2 (open,
 * Silver-Mueller) covering indices [-1, n].  Index i of a component that is
 * dual (staggered) along an axis sits at (i + 1/2) d, otherwise at i d.
 */
#ifndef PIC_ORACLE_H
#define PIC_ORACLE_H
#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_EX = 0, ORC_EY, ORC_EZ, ORC_BX, ORC_BY, ORC_BZ, ORC_BMX, ORC_BMY,
       ORC_BMZ, ORC_JX, ORC_JY, ORC_JZ, ORC_RHO, ORC_RHO_BG, ORC_NOUT };
enum { ORC_FBC_PERIODIC = 0, ORC_FBC_SM = 1 };
enum { ORC_PBC_PERIODIC = 0, ORC_PBC_REFLECT = 1, ORC_PBC_REMOVE = 2 };

typedef struct {
  int nx, ny;            /* cells */
  double dx, dy, dt;
  int px, py;            /* patch size in cells */
  int fbc_x, fbc_y;      /* field BC per axis */
  int pbc_x[2], pbc_y[2];/* particle BC per face (lo, hi) */
  double q, m;           /* species charge and mass */
  int laser_on;          /* y-polarised laser injected through x_min */
  double a0, waist, tau, t_peak, y_center;
  int mw_on;             /* moving window along +x at c */
  double mw_t0;
  double inj_n0, inj_x0, inj_ramp; /* density profile of injected plasma */
  int inj_ppcx, inj_ppcy;
  int track_continuity;  /* keep rho^n of the last step for the residual */
  int filter_passes;     /* binomial (1,2,1)/4 passes on J, each along x then y */
  int nthreads;          /* OpenMP threads for the patch loop (0 = default) */
} orc_config;

typedef struct orc_state orc_state;

orc_state *orc_create(const orc_config *c);
void orc_destroy(orc_state *s);
/* Load particles: global positions in c/w, momenta u = p/mc, weights. */
int orc_load(orc_state *s, const double *x, const double *y, const double *ux,
             const double *uy, const double *uz, const double *w, long n);
long orc_num_particles(const orc_state *s);
/* out: 6 x n (x, y, ux, uy, uz, w), in patch order. Returns n. */
long orc_get_particles(const orc_state *s, double *out);
int orc_set_field(orc_state *s, int comp, const double *src);
int orc_get_field(orc_state *s, int comp, double *dst);
/* Background charge: mode 0 none, 1 uniform value, 2 neutralising the
 * currently loaded particles (immobile ions co-located with them). */
int orc_set_background(orc_state *s, int mode, double value);
int orc_step(orc_state *s, int nsteps);
/* out[0..9]: step, t, Np, U_E, U_B, U_K, gauss residual, continuity
 * residual (NaN when unavailable), window shifts, total charge. */
int orc_diag(orc_state *s, double *out);
/* Single-particle primitives exposed for the pins. */
void orc_shape2(double xi, int *i0, double S[3]);
void orc_boris(double q, double m, double dt, const double E[3],
               const double B[3], double u[3]);
/* Deposit one particle moving from (x0,y0) to (x1,y1) with momentum u (for
 * v_z) into a zero-initialised (5 x 5 x 3) window; returns the window's first
 * node indices; returns -1 if the move exceeds one cell. */
int orc_esirkepov(const orc_state *s, double x0, double y0, double x1,
                  double y1, double w, double vz, int *ix, int *iy,
                  double Jw[3][5][5]);
/* Apply the configured binomial filter passes to the stored J (test hook). */
void orc_apply_filter(orc_state *s);
/* Interpolated value of component comp (< ORC_RHO) at (x, y). */
double orc_gather(const orc_state *s, int comp, double x, double y);
int orc_laser_field(const orc_state *s, double y, double t, double *ey);

#ifdef __cplusplus
}
#endif
#endif
