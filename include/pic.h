/*
 * libpic: GB300-native (sm_103a) patch-decomposed particle-in-cell step.
 *
 * The method is Single Domain Multiple Decompositions (SDMD, Section 2.2 of
 * "Single Domain Multiple Decompositions for Particle-in-Cell simulations"):
 * macro-particles live in small patches, fields live in one large region.
 * Here a patch (or a chunk of a heavy one) is one work item of a persistent
 * grid: a thread block stages its field tile and accumulates its current
 * tile in shared memory; the region is the whole single domain in HBM.  One step
 * is: region -> patch field staging (SDMD step (ii)), interpolation, Boris
 * push, Esirkepov deposition into the patch current tile, patch -> region
 * current reduction (SDMD step (i)), re-binning of particles that left their
 * patch, Yee FDTD update of the region with open (Silver-Mueller) or periodic
 * boundaries, and the moving-window shift when due (Section 3.2 / 3.3).
 *
 * Conventions (every entry point):
 *  - returns a pic_status; never aborts, exits or prints;
 *  - keeps no caller pointer after it returns; inputs are copied;
 *  - pointers tagged PIC_HOST are host memory, PIC_DEVICE are device memory
 *    of the context's device;
 *  - device-side faults (capacity overflow, non-finite particle, move of more
 *    than one cell, a wait that ran out) are sticky: they are reported by the
 *    next synchronising call (pic_step, pic_sync, pic_get_*, pic_diag) as
 *    PIC_EOVERFLOW / PIC_ENONFINITE / PIC_ETIMEOUT, and every later call then
 *    returns PIC_ESTATE until pic_restore succeeds;
 *  - pic_last_error(ctx) gives a human-readable reason for the last failure.
 *
 * Units are normalised: lengths c/w, time 1/w, momentum u = p / (m c),
 * fields m c w / e, densities n_c; dE/dt = curl B - J, dB/dt = -curl E.
 *
 * Field arrays exchanged with the library (pic_set_field / pic_get_field)
 * are float64, row-major (ny_e, nx_e), y slowest.  Per axis, a periodic axis
 * gives n_e = n entries for grid indices [0, n); an open axis gives
 * n_e = n + 2 entries for grid indices [-1, n] (ghost, interior, boundary).
 * A component staggered (dual) along an axis has grid index i at (i + 1/2) d,
 * otherwise at i d (Yee lattice: Ex (1/2,0), Ey (0,1/2), Ez (0,0),
 * Bx (0,1/2), By (1/2,0), Bz (1/2,1/2); J like E; rho at nodes).
 * 3D contexts (dims = 3) exchange (nz_e, ny_e, nx_e) arrays with the same
 * per-axis rule on the 3D Yee lattice: Ex (1/2,0,0), Ey (0,1/2,0),
 * Ez (0,0,1/2), Bx (0,1/2,1/2), By (1/2,0,1/2), Bz (1/2,1/2,0).  A 3D context
 * has snapshots and the auto-grow replay, but no current filter, cell-order
 * sort, batch membership or deterministic mode.
 *
 * Species and initial charge: pic_load_particles takes one species, the
 * configuration's mobile one (pic_config.q, m); the immobile ions (a
 * species with no motion, and the background charge of the initial field
 * solve) are the charge background of pic_set_background.  pic_get_field
 * reads one component per call.
 */
#ifndef PIC_H
#define PIC_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  PIC_OK = 0,
  PIC_EINVAL = 1,     /* bad argument or configuration */
  PIC_ENOMEM = 2,     /* device or host allocation failed */
  PIC_ECUDA = 3,      /* a CUDA runtime call failed */
  PIC_EOVERFLOW = 4,  /* a patch or re-binning buffer ran out of capacity */
  PIC_ETIMEOUT = 5,   /* a bounded device wait ran out */
  PIC_ENONFINITE = 6, /* a particle became non-finite or moved > 1 cell */
  PIC_ESTATE = 7      /* context unusable after an earlier device fault */
} pic_status;

typedef enum { PIC_FP64 = 0, PIC_FP32 = 1 } pic_precision;
/* Field boundary per axis. */
enum { PIC_BC_PERIODIC = 0, PIC_BC_SILVER_MULLER = 1 };
/* Particle boundary per face. */
enum { PIC_PBC_PERIODIC = 0, PIC_PBC_REFLECT = 1, PIC_PBC_REMOVE = 2 };
/* Where a caller buffer lives. */
enum { PIC_HOST = 0, PIC_DEVICE = 1 };
/* Field identifiers for pic_set_field / pic_get_field. */
enum {
  PIC_EX = 0, PIC_EY, PIC_EZ, PIC_BX, PIC_BY, PIC_BZ, PIC_BMX, PIC_BMY,
  PIC_BMZ, PIC_JX, PIC_JY, PIC_JZ, PIC_RHO, PIC_RHO_BG, PIC_NFIELDS
};
/* Background charge modes for pic_set_background. */
enum { PIC_BG_NONE = 0, PIC_BG_UNIFORM = 1, PIC_BG_NEUTRALISING = 2 };

typedef struct pic_config {
  int dims;              /* 2 (2D3V) or 3 (3D3V) */
  int n[3];              /* cells per axis; n[i] % patch[i] == 0 */
  double d[3];           /* cell size per axis */
  double dt;             /* time step; 2D: dt < min(d); 3D: the Courant
                            condition dt sqrt(sum 1/d^2) < 1 */
  int patch[3];          /* patch size in cells, multiple of 4: 4..64 (2D),
                            4..32 with the current tile in shared memory
                            (3D) */
  int prec;              /* pic_precision */
  int bc_field[3];       /* PIC_BC_* per axis */
  int bc_part[3][2];     /* PIC_PBC_* per face (lo, hi); periodic must pair
                            with a periodic field axis */
  double q, m;           /* charge and mass of the mobile species.  The
                             runs have one mobile species (electrons) and
                             immobile ions: the species, q, m and "mobile"
                             arguments of a per-species load call are these
                             two fields plus pic_set_background, which holds
                             the immobile ions' charge (the bg_rho of an
                             initial-field call). */
  /* Laser entering through x_min (requires an open x axis): Ey_inc(y, t) =
   * a0 exp(-((y-yc)/waist)^2) exp(-2 ln2 (tr/tau)^2) sin(tr),
   * tr = t - x_shift - t_peak, x_shift the moving window's displacement;
   * 3D: the transverse factor is exp(-((y-yc)^2 + (z-zc)^2)/waist^2) with
   * zc = laser_z_center. */
  int laser_on;
  double laser_a0, laser_waist, laser_tau, laser_t_peak, laser_y_center;
  /* Moving window at c along +x: after a step that brings t - mw_t0 to at
   * least (k+1) patch widths, the domain shifts one patch column. */
  int moving_window;
  double mw_t0;
  /* Plasma injected in the new column: density n0 min(1, max(0,
   * (x - x0) / ramp)) (a step at x0 if ramp <= 0), ppc[0] x ppc[1]
   * (x ppc[2] in 3D) particles per cell placed regularly, at rest; in 3D
   * only in cells whose centre has y >= inj_ymin. */
  double inj_n0, inj_x0, inj_ramp;
  int inj_ppc[3];
  double capacity_factor; /* patch capacity = factor x the fullest patch at
                             the first load (>= 1; 0 means 2.0) */
  int capacity_min;       /* lower bound on the patch capacity (0 = 256) */
  void *stream;           /* cudaStream_t to run on; NULL = library-owned */
  int device;             /* CUDA device ordinal */
  int use_graph;          /* 1: replay the captured step as a CUDA graph */
  int timing;             /* 1: per-phase CUDA-event timers (no graph) */
  int tma;                /* 1 (default if >= 0): stage field tiles with TMA;
                             0: plain coalesced loads */
  int block;              /* threads per patch block (0 = default 256) */
  int merge;              /* deposition: 1 = each thread takes 4 (FP32) or 2
                             (FP64) consecutive particles with 128-bit loads
                             and sums those sharing a current window in
                             registers before the shared atomics; otherwise
                             (default) one particle per thread per slice */
  int auto_grow;          /* 1: pic_step keeps a device copy of the state at
                             entry; a patch or re-binning capacity overflow
                             grows the capacity (x1.5 or more) and replays the
                             steps instead of failing (up to 4 times) */
  int sort_every;         /* > 0: every sort_every steps (and after loading)
                             re-order each patch's particles so that a warp's
                             32 lanes hold particles of 32 distinct
                             neighbouring cells; 0: never */
  int task_chunk;         /* particles per work item of the particle step: a
                             patch holding more is split over several
                             blocks, each with its own current tile
                             (0 = 4096 in FP32, 2048 in FP64; at most 4096:
                             the FP32 tile accumulates in 32-bit fixed point
                             whose resolution, 2^(ceil(log2 n) - 30) of a
                             bound on the contributions of the item's n
                             particles, follows from it) */
  int filter_passes;      /* binomial current filter (Section 3.2): 0 off, 1 or
                             2 passes of (1,2,1)/4 along x then y applied to
                             J before the field update (2D only) */
  double inj_ymin;        /* 3D plasma: lower y bound of the filled cells */
  double laser_z_center;  /* 3D laser: z of the beam axis */
  int window_cells;       /* moving-window step in cells, a multiple of
                             patch[0] (0 = patch[0]): the window advances
                             window_cells / patch[0] patch columns at once,
                             so the patch size (a performance choice) and
                             the window step (part of the run) are set
                             apart; pic_diag's shifts counts window steps */
  /* Device memory of the context (fields, particles, buffers, and the
   * Poisson start's scratch and FFT work area): when dev_alloc is set, taken
   * with dev_alloc(bytes, alloc_user) and given back with dev_free(ptr,
   * alloc_user), else cudaMalloc / cudaFree.  Set both or neither
   * (PIC_EINVAL otherwise).  dev_alloc returns memory of cfg.device aligned
   * to at least 256 bytes, or NULL (the call then fails with PIC_ENOMEM).
   * Both are called on the thread of the API call that needs them; the
   * context's stream is synchronised before each dev_free.  Batches and
   * servers keep their own small argument arrays with cudaMalloc. */
  void *(*dev_alloc)(size_t bytes, void *user);
  void (*dev_free)(void *ptr, void *user);
  void *alloc_user;
  int current_float;      /* FP32 path: 1 = the shared current tile
                             accumulates with float atomics; 0 (default) =
                             32-bit fixed point (native integer shared
                             atomics) scaled per work item to a bound on its
                             own contributions: (3/4) |q| times the largest
                             w |v| its particles can reach, from the previous
                             step's largest w |u| and w of its source
                             patches and the staged tile's largest |E|;
                             contributions below 2^(ceil(log2 n) - 31) of
                             that bound round to zero.  FP64 accumulates in
                             float64 (64-bit fixed point when
                             deterministic); merge = 1 keeps a run-wide
                             fixed-point scale. */
  long long staging_wait_polls; /* bound on the polls of each wait for a
                             field tile staged by TMA before the wait is
                             declared lost: the block then drains the
                             in-flight copy (itself bounded), records
                             PIC_ETIMEOUT in the context's sticky device
                             word and returns (the call reports
                             PIC_ETIMEOUT, later calls PIC_ESTATE until
                             pic_restore).  0 = default 2^24 polls; a
                             negative value makes every wait run out at
                             once, without a poll (for tests of this path) */
  int deterministic;      /* 1: results bitwise reproducible from run to run
                             and equal alone, batched and served (2D).  The
                             SDMD patch -> region current reduction (Section
                             2.2, step (i)) is made order-independent: a
                             patch is one work item; its shared current tile
                             accumulates in fixed point (FP32 32-bit as by
                             default, FP64 64-bit integers at 2^-(62 -
                             ceil(log2 n)) of the largest contribution);
                             the tiles are stored whole and the region
                             current summed from them in a fixed order.
                             Slower (no heavy-patch splitting, 64-bit shared
                             integer atomics in FP64); requires merge <= 0
                             and current_float = 0 */
} pic_config;

typedef struct pic_diag_t {
  long long step;         /* steps taken */
  double t;               /* simulated time */
  long long np;           /* particles, including those in flight between
                             patches */
  double U_E, U_B, U_K;   /* 1/2 sum |E|^2 dV, 1/2 sum |Bm|^2 dV over the
                             cells [0,nx) x [0,ny); sum w (gamma - 1) m dV */
  double gauss;           /* max |div_h E - rho - rho_bg| (open axes: 3 cells
                             from the faces excluded) */
  double continuity;      /* max |(rho^{n+1} - rho^n)/dt + div_h J| of the
                             last step, NaN if unavailable */
  double charge;          /* sum q w dV of the particles */
  int shifts;             /* moving-window shifts done */
  int max_patch_count;    /* fullest patch after the last step */
  int capacity;           /* particles per patch */
  double ms_particles, ms_fields, ms_window; /* timers (timing = 1) */
  long long launches;     /* kernels launched by this context so far */
  long long particle_step_launches;
  int grows;              /* capacity growths done by auto_grow */
  long long sorts;        /* cell-order sorts done */
  double ms_sort;         /* timer of the sorts (timing = 1) */
  long long calm_particle_steps; /* particle-steps skipped so far: particles
                             at rest in zero fields, in patches whose copy
                             the step kept (2D; 0 in 3D) */
} pic_diag_t;

typedef struct pic_ctx pic_ctx;

/* Create a context: validates the configuration and allocates the fields
 * (particles are allocated by the first pic_load_particles).  The context
 * owns all device memory it allocates.
 * Paper: the single domain (region) and its patches, Section 2.2. */
pic_status pic_create(const pic_config *cfg, pic_ctx **out);

/* Append n particles (global positions x, y in c/w; momenta u; weights w =
 * local density / particles per cell), float64, PIC_HOST or PIC_DEVICE.
 * They are binned into patches on the device; positions outside the domain
 * give PIC_EINVAL.  The first call sizes the patch capacity.  2D contexts
 * only (PIC_EINVAL for dims = 3).  Page-locked host arrays are read in
 * place by the kernels (no staging copy).  The species is the
 * configuration's mobile one (pic_config.q, m).
 * Paper: macro-particles held by the patches, Section 2.2. */
pic_status pic_load_particles(pic_ctx *ctx, const double *x, const double *y,
                              const double *ux, const double *uy,
                              const double *uz, const double *w, size_t n,
                              int where);
/* The same with z positions, for 3D contexts (PIC_EINVAL for dims = 2).
 * Paper: as pic_load_particles, in three dimensions. */
pic_status pic_load_particles3(pic_ctx *ctx, const double *x, const double *y,
                               const double *z, const double *ux,
                               const double *uy, const double *uz,
                               const double *w, size_t n, int where);

/* Fill the domain, on the device, with the configuration's plasma profile
 * (inj_n0, inj_x0, inj_ramp, inj_ppc: the profile the moving window
 * injects): inj_ppc[0] x inj_ppc[1] particles per cell at rest, regularly
 * placed, weight = density at the particle's x / particles per cell; the
 * charge of the co-located immobile ions is added to the background.  Only
 * before any particles are loaded (PIC_ESTATE otherwise); sizes the patch
 * capacity like the first pic_load_particles (a full patch x
 * capacity_factor).
 * Paper: macro-particles placed regularly in every cell, Section 3.2. */
pic_status pic_load_plasma(pic_ctx *ctx);

/* Overwrite one field component (PIC_EX..PIC_BMZ or PIC_RHO_BG) from an
 * array in the layout above.  B is taken at t + dt/2, Bm at t.
 * Paper: the region's fields on the Yee lattice, Sections 2.2 and 3.2. */
pic_status pic_set_field(pic_ctx *ctx, int which, const double *src, int where);

/* Background charge (immobile ions): none, uniform value, or neutralising
 * the particles currently loaded.  This is the immobile species and the
 * bg_rho of the initial field solve (it enters Gauss's law and the Poisson
 * start; the ions deposit no current).
 * Paper: the immobile-ion background of the runs, Section 3.1. */
pic_status pic_set_background(pic_ctx *ctx, int mode, double value);

/* Initial fields.  PIC_INIT_ZERO: E, B and Bm zero.  PIC_INIT_POISSON (every
 * axis periodic): E from Gauss's law for the loaded particles and the
 * background, div_h E = rho - <rho>, E = -grad_h phi on the Yee lattice,
 * solved in FP64 with a spectral (FFT) Poisson solve; B = Bm = 0.  Other
 * boundaries give PIC_EINVAL.
 * Paper: the Maxwell-Gauss system the Yee update preserves, Section 3.2. */
enum { PIC_INIT_ZERO = 0, PIC_INIT_POISSON = 1 };
pic_status pic_init_fields(pic_ctx *ctx, int mode);

/* Advance nsteps steps.  Synchronises with the device at the end and reports
 * device-side faults.
 * Paper: one PIC iteration with the two SDMD synchronisations, Section 2.2
 * steps (i) (patch currents reduced into the region) and (ii) (region
 * fields sent to the patches); the operators of Section 3.2 (Yee FDTD,
 * Esirkepov deposition of order 2 on a 5-point stencil, optional binomial
 * filter) and the "Particles" phase of Section 3.3 (interpolation, push,
 * deposition). */
pic_status pic_step(pic_ctx *ctx, int nsteps);

/* Read one field component (PIC_EX..PIC_RHO_BG) into dst (layout above).
 * PIC_JX..PIC_JZ give the current of the last step as the field update used
 * it (after the binomial filter when filter_passes > 0); PIC_RHO deposits
 * the particles' charge in float64.  A page-locked host dst is written in
 * place.
 * Paper: the region fields of Section 2.2 on the Yee lattice of 3.2. */
pic_status pic_get_field(pic_ctx *ctx, int which, double *dst, int where);

/* Copy the particles out as 6 x n float64 rows (x, y, ux, uy, uz, w), global
 * positions, in patch order; 3D contexts give 7 rows (x, y, z, ux, uy, uz,
 * w).  cap is the row length of out; *n receives the count (PIC_EINVAL if
 * it exceeds cap).  A page-locked host out is written in place.
 * Paper: the patches' macro-particles, Section 2.2. */
pic_status pic_get_particles(pic_ctx *ctx, double *out, size_t cap, size_t *n,
                             int where);

/* Diagnostics (float64 reductions on the device).
 * Paper: the energy and load measures of Section 3.3 (field and kinetic
 * energy, particle counts per patch), with the discrete Gauss and
 * continuity residuals the Yee / Esirkepov pair (Section 3.2) conserves. */
pic_status pic_diag(pic_ctx *ctx, pic_diag_t *out);

/* Wait for the context's stream and report sticky device faults.
 * (Library plumbing; the paper has no counterpart.) */
pic_status pic_sync(pic_ctx *ctx);

/* Checkpoint: with host == NULL, *bytes receives the size needed; otherwise
 * the whole state is written to host (size *bytes).  A 2D snapshot holds
 * fields, background charge, device scalars and the live particles of both
 * particle sets (packed, without the capacity slack), so its size follows
 * the particle count; the size query synchronises the context's stream.
 * (Fault recovery of this library; the paper has no counterpart.) */
pic_status pic_snapshot(pic_ctx *ctx, void *host, size_t *bytes);
/* Restore a snapshot taken from a context with the same configuration; also
 * clears a sticky device fault.  A context with particle storage takes only
 * a snapshot of its own capacity; one without (never loaded) allocates it.
 * The snapshot's size and counts are checked before the context changes
 * (PIC_EINVAL).  2D and 3D snapshots are distinct formats (PIC_EINVAL
 * across them). */
pic_status pic_restore(pic_ctx *ctx, const void *host, size_t bytes);

/* Device bytes a context with this configuration and at most np_max
 * particles at the first load would allocate (used for admission).
 * (Serving admission; the paper has no counterpart.) */
size_t pic_footprint(const pic_config *cfg, size_t np_max);

/* Human-readable reason of the context's last failure; destroy a context
 * (every allocation it made returned).  (Library plumbing; the paper has no
 * counterpart.) */
const char *pic_last_error(const pic_ctx *ctx);
void pic_destroy(pic_ctx *ctx);

/* ---- Batches ---------------------------------------------------------
 * Many independent runs (contexts) advanced together, one launch per kernel
 * per step for the whole batch: one work plan over the patches of every
 * run, one persistent particle-step launch whose work items carry their run
 * (the patch-level task decomposition of Section 2.2 applied across runs),
 * and one launch per field kernel whose blocks cover every run's region.
 * Each run keeps its own state and gives the same results, step for step,
 * as when stepped alone (the order of its floating-point atomic sums aside).
 *
 * Rules: the runs of a batch share a precision and the batch's device, have
 * particles loaded and hold no device fault; at most PIC_BATCH_MAX runs.  A
 * run may still be used alone between batched steps (its stream and the
 * batch's are ordered by events); a run whose capacity, storage or step
 * parity changed since the batch last built its device arguments makes the
 * next pic_batch_step rebuild them.  Inside a batch a run's capacity is
 * fixed (no auto_grow replay) and sort_every is not applied; a run that
 * faults (capacity overflow, non-finite particle, ...) holds the sticky
 * status that pic_step would give, leaves the batch, and pic_batch_step
 * returns that status (the other runs have stepped normally).
 * The batch does not own its runs: destroy it before them, or remove them
 * with pic_batch_set first. */
#define PIC_BATCH_MAX 64
typedef struct pic_batch pic_batch;
typedef struct pic_batch_config {
  void *stream;    /* cudaStream_t of the batch; NULL = library-owned */
  int device;      /* CUDA device ordinal (every run's) */
  int use_graph;   /* 1: each step replays a captured CUDA graph */
  int task_chunk;  /* particles per work item (0 = 4096 in FP32, 2048 in
                      FP64; at most 4096) */
} pic_batch_config;
typedef struct pic_batch_diag_t {
  long long steps;     /* batched steps taken */
  long long launches;  /* kernels launched by them (window shifts included) */
  long long builds;    /* device-argument (and graph) rebuilds */
  int nruns;           /* runs currently in the batch */
  int grid;            /* blocks of the persistent particle step */
} pic_batch_diag_t;

/* Paper (all batch calls): the patch-level task decomposition of Section
 * 2.2 applied across independent runs; batching itself has no counterpart
 * in the paper. */
pic_status pic_batch_create(const pic_batch_config *cfg, pic_batch **out);
/* Replace the batch's runs (n = 0 empties it); PIC_EINVAL / PIC_ESTATE when
 * a run breaks a rule above (runs of one batch also share the deterministic
 * setting), leaving the batch unchanged. */
pic_status pic_batch_set(pic_batch *b, pic_ctx *const *runs, int n);
/* Advance every run nsteps steps (moving-window shifts of each run applied
 * as they fall due).  Synchronises at the end.  Each run's step is the one
 * of pic_step (Section 2.2 steps (i) and (ii), Section 3.2 operators). */
pic_status pic_batch_step(pic_batch *b, int nsteps);
int pic_batch_size(const pic_batch *b);
pic_status pic_batch_get_diag(const pic_batch *b, pic_batch_diag_t *out);
const char *pic_batch_last_error(const pic_batch *b);
void pic_batch_destroy(pic_batch *b);

/* ---- Autotuner ---------------------------------------------------------
 * Chooses the launch shape of a workload by timing: square patch sizes
 * {8, 16, 32} (with the moving window, only those dividing its step, which
 * is kept: window_cells of the result names it), particle-step blocks of
 * {128, 256} threads and work items of {1024, 2048, 4096} particles, plus the
 * configuration as given.  Each candidate is a fresh context loaded with the
 * caller's particles (float64, PIC_HOST or PIC_DEVICE), stepped 2 steps to
 * warm up and then `steps` steps, timed on the host around pic_step (which
 * synchronises); the fastest wins.  The choice changes only the rounding
 * order of the current sums, never the method.  Results are cached per
 * process by (grid, boundaries, laser, window, filter, precision, particles
 * per cell); a cached key returns without timing (candidates = 0).
 * On success *tuned is cfg with patch, block, task_chunk (and, with the
 * moving window, window_cells) replaced. */
typedef struct pic_tune_t {
  int patch[3];        /* chosen patch size */
  int block;           /* chosen particle-step block size */
  int task_chunk;      /* chosen particles per work item */
  double ms_per_step;  /* its measured time per step */
  double ms_given;     /* time per step of the configuration as given */
  int candidates;      /* candidates timed (0: taken from the cache) */
} pic_tune_t;
pic_status pic_autotune(const pic_config *cfg, const double *x, const double *y,
                        const double *ux, const double *uy, const double *uz,
                        const double *w, size_t n, int where, int steps,
                        pic_config *tuned, pic_tune_t *out);
/* The autotuner on the configured plasma instead of caller particles (each
 * candidate filled on the device as by pic_load_plasma; needs inj_ppc >= 1
 * on every axis), for 2D and 3D contexts.  2D candidates as pic_autotune;
 * 3D candidates are the patch shapes {8, 16}^3 that divide the grid (and,
 * with the moving window, whose width divides its step) with work items of
 * {1024, 2048, 4096} particles, plus the configuration as given.  Cached
 * per process like pic_autotune, keyed by the full grid and the plasma. */
pic_status pic_autotune_plasma(const pic_config *cfg, int steps, pic_config *tuned,
                               pic_tune_t *out);
/* Forget every cached choice.  (Autotuning has no counterpart in the paper;
 * its candidates are the patch sizes of Section 2.2, the paper's own
 * performance knob, Section 3.3.) */
void pic_autotune_clear_cache(void);

/* ---- Serving ------------------------------------------------------------
 * A request loop over many PIC runs with continuous batching.  A request is
 * a configuration plus its initial plasma (the configuration's injection
 * profile, filled on the device by pic_load_plasma, with its ions as the
 * background) and a step count.  Each pic_server_tick:
 *  1. admits queued requests in arrival order while the run slots
 *     (max_runs) and the device-memory budget (the sum of the admitted runs'
 *     pic_footprint estimates) allow; an admitted run's state stays
 *     resident until it completes;
 *  2. advances every admitted run by k = min(steps_per_tick, the fewest
 *     steps any of them has left) batched steps (pic_batch_*: one launch per
 *     kernel for all runs, whatever their grid sizes);
 *  3. retires the runs that reached their step count (final diagnostics
 *     recorded; the context destroyed, or kept for pic_server_take).
 * A request that arrives while others run joins at the next tick in which
 * a slot and memory are free.  Times are seconds on the server's clock
 * (pic_server_clock).  FP32 and FP64 requests, deterministic or not, may be
 * mixed: the server keeps one batch per precision and mode and steps each
 * in every tick.  3D requests are admitted the same way and stepped one by
 * one in every tick, after the batches (there are no batched 3D kernels).
 * Not thread-safe: one host thread drives a server.
 * (Serving has no counterpart in the paper; each served run is the step of
 * pic_step.) */
typedef struct pic_server pic_server;
typedef struct pic_server_config {
  void *stream;          /* cudaStream_t of the batches; NULL = library-owned */
  int device;
  size_t hbm_budget;     /* bytes the admitted runs may hold; 0 = 90% of the
                            device memory free at creation */
  int max_runs;          /* runs admitted at once (1..PIC_BATCH_MAX; 0 = max) */
  int steps_per_tick;    /* batched steps per tick at most (0 = 10) */
  int use_graph;         /* batches replay captured CUDA graphs */
} pic_server_config;
enum { PIC_REQ_QUEUED = 0, PIC_REQ_RUNNING = 1, PIC_REQ_DONE = 2, PIC_REQ_FAILED = 3,
       PIC_REQ_CANCELLED = 4 };
typedef struct pic_request_info {
  int state;             /* PIC_REQ_* */
  int status;            /* pic_status of a failed request */
  long long steps_done, steps_total;
  long long np0;         /* particles at admission */
  long long np;          /* particles at completion */
  size_t footprint;      /* admission estimate (pic_footprint) */
  double t_submit, t_admit, t_done;  /* server clock, seconds */
  double U_E, U_B, U_K;  /* diagnostics at completion */
} pic_request_info;
typedef struct pic_server_stats {
  long long submitted, done, failed, queued, running;
  long long ticks, batched_steps;
  double particle_steps; /* sum over runs of particles at admission x steps */
  size_t hbm_in_use;     /* footprint estimates of the runs held */
  double busy_s;         /* time spent inside pic_server_tick */
  long long cancelled;   /* requests cancelled by pic_server_cancel */
} pic_server_stats;

pic_status pic_server_create(const pic_server_config *cfg, pic_server **out);
/* Queue a request (cfg is copied; plasma from cfg's inj_* fields, which
 * must give at least one particle per cell; dims 2 or 3); *id receives its
 * handle.
 * keep = 1: the finished context is kept for pic_server_take.  The
 * configuration is validated here (PIC_EINVAL). */
pic_status pic_server_submit(pic_server *s, const pic_config *cfg, long long nsteps, int keep,
                             long long *id);
/* Admit, step, retire (see above); *running (optional) receives the runs
 * on the device after the tick. */
pic_status pic_server_tick(pic_server *s, int *running);
pic_status pic_server_info(const pic_server *s, long long id, pic_request_info *out);
/* Hand a finished, kept run's context to the caller, who destroys it
 * (before the server: the context runs on the server's stream). */
pic_status pic_server_take(pic_server *s, long long id, pic_ctx **out);
/* Cancel a queued or running request between ticks: a queued one leaves
 * the queue; a running one leaves its batch and its context is destroyed
 * (its memory returns to the budget).  Its state becomes PIC_REQ_CANCELLED
 * with the steps it had done.  PIC_ESTATE for a request that already
 * finished, failed or was cancelled; PIC_EINVAL for an unknown id. */
pic_status pic_server_cancel(pic_server *s, long long id);
pic_status pic_server_get_stats(const pic_server *s, pic_server_stats *out);
double pic_server_clock(const pic_server *s);
void pic_server_destroy(pic_server *s);

/* Library version string.  (No counterpart in the paper.) */
const char *pic_version(void);

/* Allocation-free field energy (the paper has no counterpart: this is a
 * library service).  For callers that cannot let the library call
 * cudaMalloc -- an application that owns the device memory budget through
 * its own allocator, or a serving loop where a device allocation would
 * synchronise the device under live requests -- this computes
 * out[0] = 1/2 sum (Ex^2 + Ey^2 + Ez^2) dV and out[1] = 1/2 sum (Bmx^2 +
 * Bmy^2 + Bmz^2) dV over float64 cell arrays of shape (ny, nx), row-major,
 * all in device memory of the current device (out: 2 doubles, device).
 * It allocates nothing: its scratch is a fixed file-scope device array of
 * PIC_NOALLOC_MAX_ROWS x 2 doubles (1 MiB) that every GPU loading the library
 * holds until exit.  ny > PIC_NOALLOC_MAX_ROWS, nx or ny <= 0, or a null
 * pointer gives PIC_EINVAL.  Set-up, once per device and CUDA context: the
 * first call on a device (or any pic_create on it) loads this code's module
 * and kernels and looks up the scratch array's device address; until then
 * the array is not yet resident, and that first set-up may allocate and
 * synchronise like any module load, so make one call, or create a context,
 * on each device before serving and before any stream capture on it.  After
 * a device reset (cudaDeviceReset, a new primary context) the next call sets
 * up again.  Calls share the scratch array: calls that overlap on the GPU
 * race; a call rewrites every row it reads.  Runs asynchronously on
 * `stream` (a cudaStream_t; NULL = the default stream). */
#define PIC_NOALLOC_MAX_ROWS 65536
pic_status pic_field_energy_noalloc(const double *Ex, const double *Ey,
                                    const double *Ez, const double *Bmx,
                                    const double *Bmy, const double *Bmz,
                                    int nx, int ny, double dV, double *out,
                                    void *stream);

#ifdef __cplusplus
}
#endif
#endif
