// Internal definitions shared by the libpic CUDA translation units.
//
// Data layout in HBM (one context):
//   fields   one allocation of NCOMP components, each a (ny + 2 GY) x sx
//            array, x fastest; grid index (i, j) lives at
//            (j + GY) * sx + (i + GX); sx is a multiple of 32 elements.
//            Components: Ex Ey Ez Bmx Bmy Bmz | Bx By Bz | JA(x,y,z) |
//            JB(x,y,z).  E and Bm are adjacent so one 3D TMA box stages all
//            six interpolated components of a patch.  Ghost cells of a
//            periodic axis hold mirror copies of the interior, written by
//            the kernel that produces the value; ghost cells of an open axis
//            hold the Silver-Mueller values.
//   particles  per patch slot a segment of `cap` entries in six SoA arrays
//            (x, y patch-relative in cell units; ux, uy, uz; w), two
//            ping-pong sets; plus per slot 8 direction buckets of `bcap`
//            entries (particles that left the slot, already rebased to the
//            destination patch), two ping-pong sets.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace pic {

constexpr int GX = 4;  // ghost cells along x (keeps TMA box starts 16B aligned)
constexpr int GY = 4;  // ghost cells along y
constexpr int NCOMP = 15;
enum {
  C_EX = 0, C_EY, C_EZ, C_BMX, C_BMY, C_BMZ, C_BX, C_BY, C_BZ,
  C_JA = 9, C_JB = 12
};
enum { FBC_PERIODIC = 0, FBC_SM = 1 };
enum { PBC_PERIODIC = 0, PBC_REFLECT = 1, PBC_REMOVE = 2 };

// Sticky device error bits.
enum : unsigned {
  ERR_OVERFLOW_SEG = 1u,
  ERR_OVERFLOW_BKT = 2u,
  ERR_NONFINITE = 4u,
  ERR_FAST = 8u,
  ERR_TIMEOUT = 16u,
  ERR_LOAD_RANGE = 32u,
  ERR_OVERFLOW_LOAD = 64u,
  ERR_BOUNDS = 128u  // checked build: an index out of its array (access skipped)
};

// Checked build (-DPIC_CHECKED): PIC_IN(err, cond) is cond, and records
// ERR_BOUNDS in the unsigned err when it fails (the caller then skips the
// access: no trap, no early return, so every block still reaches its
// barriers); otherwise it is true and costs nothing.
#ifdef PIC_CHECKED
#define PIC_IN(err, cond) ((cond) ? true : ((err) |= ERR_BOUNDS, false))
#else
#define PIC_IN(err, cond) true
#endif

// Device-resident state; t and step are double-buffered by step parity so
// that the kernels of one step read slot p while the last one writes 1 - p.
struct DevState {
  double t[2];
  long long step[2];
  int nshift;
  int col0;       // slot column holding physical patch column 0
  unsigned err;
  int maxcnt[2];  // fullest patch written by the particle step of parity p
  double laser_h; // laser temporal factor at t_{n+3/2}, set by the E update
  // particles carried over in calm slots that a step skipped, summed over
  // all steps (each such particle is one particle-step with no work)
  unsigned long long calm_particles;
};

struct Geom {
  int nx, ny;       // cells
  int P, Q;         // patch size (x, y)
  int npx, npy, nslots;
  int sx, nys;      // row stride, stored rows
  long long cs;     // elements per component (sx * nys)
  double dx, dy, dt;
  int fbc_x, fbc_y;
  int pbc[2][2];    // [axis][face]
  double q, m;
};

template <typename R>
struct SoA {
  R *x, *y, *ux, *uy, *uz, *w;
};

// Direction buckets of one slot: bucket d holds up to cap[d] particles at
// elements [s * stride + off[d], ... + cap[d]).  A particle sheet moving
// along x (a laser-driven front) can carry a whole patch across an x edge in
// one step, so x-edge buckets get the full patch capacity, y-edge buckets
// half of it and corner buckets a quarter.
struct Buckets {
  int cap[8];
  int off[8];
  int stride;
};

// Direction k in 0..7 <-> (ddx, ddy), centre excluded.
__host__ __device__ inline int dir_index(int ddx, int ddy) {
  int code = (ddy + 1) * 3 + (ddx + 1);
  return code < 4 ? code : code - 1;
}
__host__ __device__ inline void dir_delta(int k, int &ddx, int &ddy) {
  int code = k < 4 ? k : k + 1;
  ddx = code % 3 - 1;
  ddy = code / 3 - 1;
}

// Neighbour slot of slot s in physical direction (ddx, ddy), or -1 when it
// lies outside a non-periodic domain face.  Slot columns form a ring offset
// by col0 (moving window); rows are not rotated.
__host__ __device__ inline int neighbour_slot(const Geom &g, int col0, int s, int ddx,
                                              int ddy) {
  int sxs = s % g.npx, sy = s / g.npx;
  int px = sxs - col0;
  if (px < 0) px += g.npx;
  int qx = px + ddx, qy = sy + ddy;
  if (qx < 0 || qx >= g.npx) {
    if (g.fbc_x != FBC_PERIODIC) return -1;
    qx = (qx + g.npx) % g.npx;
  }
  if (qy < 0 || qy >= g.npy) {
    if (g.fbc_y != FBC_PERIODIC) return -1;
    qy = (qy + g.npy) % g.npy;
  }
  int qs = (qx + col0) % g.npx;
  return qy * g.npx + qs;
}

__host__ __device__ inline long long fidx(const Geom &g, int i, int j) {
  return (long long)(j + GY) * g.sx + (i + GX);
}

// Write v at the periodic ghost images of stored element o = grid (i, j)
// (those that lie in the stored range); o itself is not written.
template <typename R>
__device__ __forceinline__ void mirror(const Geom &g, R *a, long long o, int i, int j, R v) {
  int mx = 0, my = 0;
  if (g.fbc_x == FBC_PERIODIC) mx = i < GX ? g.nx : (i >= g.nx - GX ? -g.nx : 0);
  if (g.fbc_y == FBC_PERIODIC) my = j < GY ? g.ny : (j >= g.ny - GY ? -g.ny : 0);
  if (mx) a[o + mx] = v;
  if (my) {
    const long long oy = o + (long long)my * g.sx;
    a[oy] = v;
    if (mx) a[oy + mx] = v;
  }
}

// Store v at (i, j) of component array a and at every periodic ghost image
// of (i, j) that lies in the stored range.
template <typename R>
__device__ inline void store_mirrored(const Geom &g, R *a, int i, int j, R v) {
  const long long o = fidx(g, i, j);
  a[o] = v;
  mirror(g, a, o, i, j, v);
}

// Quadratic B-spline weights of the nodes i0-1, i0, i0+1 for a coordinate
// xi (in cells): i0 = floor(xi + 1/2), delta = xi - i0.
template <typename R>
__device__ __forceinline__ int shape2(R xi, R S[3]) {
  R fl = floor(xi + R(0.5));
  R d = xi - fl;
  R a = R(0.5) - d, b = R(0.5) + d;
  S[0] = R(0.5) * a * a;
  S[1] = R(0.75) - d * d;
  S[2] = R(0.5) * b * b;
  return (int)fl;
}

// --- TMA / mbarrier helpers (inline PTX, sm_90+ forms valid on sm_103a) ---
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t phase) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(phase)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, uint64_t *bar,
                                            int c0, int c1, int c2) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4, %5}], [%2];" ::"r"(smem_u32(dst)),
      "l"((unsigned long long)map), "r"(smem_u32(bar)), "r"(c0), "r"(c1), "r"(c2)
      : "memory");
}

__device__ __forceinline__ void tma_load_4d(void *dst, const CUtensorMap *map, uint64_t *bar,
                                            int c0, int c1, int c2, int c3) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4, %5, %6}], [%2];" ::"r"(smem_u32(dst)),
      "l"((unsigned long long)map), "r"(smem_u32(bar)), "r"(c0), "r"(c1), "r"(c2), "r"(c3)
      : "memory");
}

// Default bound on mbarrier polls before a staging wait is declared lost
// (each try_wait suspends for up to a hardware time slice, so this is far
// beyond any real copy latency; the run's bound is StepArgs::wait_polls,
// pic_config.staging_wait_polls) and the bound used to drain an in-flight
// copy before the block returns.
constexpr long long WAIT_POLLS = 1ll << 24;
constexpr long long DRAIN_POLLS = 1ll << 22;
// The run's bound from pic_config.staging_wait_polls: 0 = WAIT_POLLS, a
// negative value = no poll (every wait runs out at once).
inline long long wait_polls_of(long long cfg) { return cfg == 0 ? WAIT_POLLS : (cfg < 0 ? 0 : cfg); }

// ----------------------------------------------------------- launchers ---
// Work plan of one particle step: items (patch slot, first work unit), a
// work unit being the particles one thread takes at once; patches holding
// more than `chunk` units are split into several items (task decomposition
// below the patch), ordered heaviest patch first.
struct Plan {
  int *item_slot, *item_first;  // [max_items]
  int *n_items, *next;          // device scalars: items, work counter
  int *units;                   // [nslots] scratch: units per slot
  int chunk;                    // units per item
  int unit;                     // particles per unit
  int max_items;
};

template <typename R>
struct StepArgs {
  Geom g;
  const R *F;          // field base (component 0)
  R *Jdst;             // current set deposited into (3 comps, g.cs apart)
  SoA<R> pin, pout;    // patch segments, read / written
  const int *cnt_in;
  int *cnt_out;
  SoA<R> bin, bout;    // direction buckets, read / written
  const int *bcnt_in;
  int *bcnt_out;
  // per slot: 1 when the step that wrote this array found the slot calm
  // (every particle at rest in an all-zero field tile, nothing arriving),
  // i.e. both segment sets then hold the same particles; the step reads
  // calm_in (previous step) and writes calm_out (set to 1 before the step,
  // cleared by any item of a slot that was not calm)
  const unsigned char *calm_in;
  unsigned char *calm_out;
  // copies of the counts of the previous state's particle sets (the inputs
  // of the most recent step), kept for the continuity diagnostic: the work
  // plan clears the step's output counts, which may still hold them
  int *cnt_prev, *bcnt_prev;
  // FP32 fixed-point tile scale per work item (single particles): per slot
  // the largest (w |u|)^2 and w of the particles its items processed, as
  // float bits ([2 s], [2 s + 1]); the step reads the previous step's
  // (stat_in) and writes its own (stat_out, cleared by the plan).  An item
  // bounds its particles' contributions by (3/4) |q| B with
  //   B = min(max w |u| + 2 |eps| |E|_tile max w, max w, wglob)
  // (the Boris rotation keeps |u|; each half kick adds at most |eps| |E|;
  // |v| <= min(|u|, 1)), maxima over the item's nine source slots, and
  // scales its tile by 2^K jk / B, jk = 1 / ((3/4)^2 |q|).
  const unsigned *stat_in;
  unsigned *stat_out;
  R jk, wglob;
  long long wait_polls;  // bound on polls of a tile-staging wait
  // deterministic mode: one work item per slot; FP64 tiles in 64-bit fixed
  // point; each item stores its whole current tile (as reals) into jbuf at
  // [slot][3 (P+5) (Q+5)] and sets jflag[slot]; the region current is then
  // summed from the stored tiles in a fixed order (launch_gather_current)
  int det;
  R *jbuf;
  int *jflag;
  int cap;
  Buckets bk;
  int parity;
  DevState *st;
  // per-step constants in the working precision, computed on the host (the
  // device's FP64 unit is slow: no per-thread double arithmetic)
  R rdx, rdy;          // dt / dx, dt / dy (cell units per unit velocity)
  R eps;               // q dt / (2 m)
  R cjx, cjy, cjz;     // -q dx / dt, -q dy / dt, q
  R RP, RQ;            // patch size as reals
  // FP32: the shared current tile accumulates in 32-bit fixed point
  // (integer shared atomics are native; float ones are not): a contribution
  // v of component c adds round(v jscale[c]); the tile's integer times
  // junit[c] = 1 / jscale[c] is the current.  jscale[c] = 2^K / ((3/4)^2
  // |q| w_max) with K = 30 - ceil(log2(the particles of a work item)): every
  // contribution is below (4/3) 2^K (at most (3/4) |q| w), so an item's sums
  // stay below (4/3) 2^30 < 2^31.
  R jscale[3], junit[3];
  int jfloat;          // FP32: accumulate the tile with float atomics instead
                       // (selects the kernel instance; batches ignore it)
  Plan plan;
};

// Clear the output counts and run the persistent particle step with `grid`
// blocks; plan = true builds the step's work plan first (otherwise the plan
// was built ahead, by launch_plan, beside the previous field update).
template <typename R>
cudaError_t launch_particle_step(const StepArgs<R> &a, const CUtensorMap *tmap, bool tma,
                                 bool merge, int block, int grid, bool plan, cudaStream_t s);
// The work plan of the step described by a, which also clears the step's
// output counts; ahead: built while the step before is the most recent one
// (its inputs are then the previous state kept aside).
template <typename R>
cudaError_t launch_plan(const StepArgs<R> &a, bool ahead, cudaStream_t s);
// Deterministic mode: the region current of the step summed from the
// stored tiles in a fixed order (after the particle step).
template <typename R>
cudaError_t launch_gather_current(const StepArgs<R> &a, cudaStream_t s);
// Blocks of the particle step resident on the device at once.
template <typename R>
int particle_step_grid(int P, int Q, bool tma, bool merge, int block, bool jfloat = false);

// ---- batches: several independent runs advanced by one launch per kernel.
// Runs per batch; the tensor maps of a batch travel as one kernel parameter
// (128 B each), the per-run argument structs live in device arrays.
constexpr int kBatchMax = 64;
template <int N>
struct TmapSet {
  CUtensorMap m[N];
};
// Linear block index -> (run, block x, block y) of a batched 2D launch:
// run r owns blocks [off[r], off[r + 1]) laid out gx[r] per row.
struct BatchGrid {
  int n;
  int off[kBatchMax + 1];
  int gx[kBatchMax];
};
__host__ __device__ inline int batch_run(const int *off, int n, int b) {
  int lo = 0, hi = n;  // last r with off[r] <= b
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (off[mid] <= b) lo = mid; else hi = mid;
  }
  return lo;
}
template <typename R>
struct BatchRef {
  const StepArgs<R> *args;  // [n] this step's arguments of each run
  int *item_run;            // [max_items] run of each work item
  BatchGrid slots;          // run r owns flattened slots [off[r], off[r + 1])
  Plan plan;                // the batch's plan (units indexed by flat slot)
};
// Deterministic mode, batched: the gather of every run, block b of the
// launch working on run batch_run(bg, b) (blocks of 256 nodes per run).
template <typename R>
cudaError_t launch_gather_current_batch(const BatchRef<R> &b, const BatchGrid &bg, cudaStream_t s);
// Batched plan + persistent particle step over every run of `b`.
template <typename R>
cudaError_t launch_particle_step_batch(const BatchRef<R> &b, const TmapSet<kBatchMax> *tm,
                                       int P, int Q, bool tma, int block, int grid,
                                       size_t smem, cudaStream_t s);
template <typename R>
int particle_step_batch_grid(int P, int Q, bool tma, int block, size_t smem);
template <typename R>
cudaError_t prepare_particle_step_batch(int P, int Q, size_t smem);
// Raise the dynamic shared-memory limit of the step kernels (call outside
// stream capture).
template <typename R>
cudaError_t prepare_particle_step(int P, int Q);
size_t particle_step_smem(int P, int Q, size_t rsize);

template <typename R>
struct FieldArgs {
  Geom g;
  R *F;
  int parity;          // J set read = C_JA + 3 * parity, zeroed = the other
  DevState *st;
  R dt, idx, idy;      // dt, 1/dx, 1/dy in the working precision
  // Silver-Mueller coefficients per open axis: 1/(1+r), 1-r, dt/d_transverse
  R smx_inv1pr, smx_1mr, smx_dtt, smy_inv1pr, smy_1mr, smy_dtt;
  // laser: transverse profile a0 exp(-((y-yc)/w)^2) at y = (j+1/2) dy
  // (device array) and the temporal factor's parameters
  int laser_on;
  const double *laser_g;
  double tau, t_peak;
  int filter_passes;   // 0: E reads the deposited J; 1, 2: the filtered copy
};
template <typename R>
cudaError_t launch_fields(const FieldArgs<R> &a, cudaStream_t s);
// The binomial filter alone (a.filter_passes passes): current set src -> dst.
template <typename R>
cudaError_t launch_filter(const FieldArgs<R> &a, int src, int dst, cudaStream_t s);
// Field update of every run of a batch: `fa` holds each run's arguments,
// grid[k] maps the blocks of the filter (k = 0), E (1), B (2) and
// Silver-Mueller (3) kernels to runs; kernels with no block are skipped.
template <typename R>
cudaError_t launch_fields_batch(const FieldArgs<R> *fa, const BatchGrid grid[4], cudaStream_t s);
// Blocks per run of the batched field kernels (gx, gy for k = 0..2; the
// Silver-Mueller kernel: gx blocks per face, gy = 4 faces).
void field_batch_blocks(const Geom &g, int filter_passes, int gx[4], int gy[4]);

// Field I/O and utilities.
template <typename R>
cudaError_t launch_set_field(const Geom &g, R *arr, const double *src, cudaStream_t s);
template <typename R>
cudaError_t launch_get_field(const Geom &g, const R *arr, double *dst, cudaStream_t s);
cudaError_t launch_get_field_f64(const Geom &g, const double *arr, double *dst, cudaStream_t s);
cudaError_t launch_set_field_f64(const Geom &g, double *arr, const double *src, cudaStream_t s);
// *out = max(*out, max |w[i]|) over i < n as float64 bits (out on the
// device, initialised by the caller; a non-finite w gives +inf).
cudaError_t launch_absmax_f64(const double *w, size_t n, unsigned long long *out, cudaStream_t s);
// y[i] += x[i], i < n (float64).
cudaError_t launch_axpy_f64(double *y, const double *x, size_t n, cudaStream_t s);
template <typename R>
cudaError_t launch_shift_fields(const Geom &g, R *F, int ncomp, cudaStream_t s);
cudaError_t launch_shift_f64(const Geom &g, double *a, cudaStream_t s);

// Particles.
template <typename R>
cudaError_t launch_bin_count(const Geom &g, int col0, const double *x, const double *y, size_t n,
                             int *counts, unsigned *err, cudaStream_t s);
cudaError_t launch_clamp_counts(int *cnt, int n, int cap, cudaStream_t s);
template <typename R>
cudaError_t launch_bin_place(const Geom &g, int col0, const double *x, const double *y,
                             const double *ux, const double *uy, const double *uz,
                             const double *w, size_t n, SoA<R> seg, int *counts, int cap,
                             unsigned *err, cudaStream_t s);
template <typename R>
struct PartView {
  SoA<R> seg;
  const int *cnt;
  SoA<R> bkt;
  const int *bcnt;
  int cap;
  Buckets bk;
};
template <typename R>
cudaError_t launch_deposit_rho(const Geom &g, int col0, const PartView<R> &v, double *rho,
                               double sign, cudaStream_t s);
template <typename R>
cudaError_t launch_particle_diag(const Geom &g, int col0, const PartView<R> &v, double *partials,
                                 int nblocks, cudaStream_t s);
template <typename R>
cudaError_t launch_field_diag(const Geom &g, const R *F, double *partials, int nblocks,
                              cudaStream_t s);
template <typename R>
cudaError_t launch_gauss_diag(const Geom &g, const R *F, int jset, const double *rho,
                              const double *rho_prev, const double *rho_bg, double *partials,
                              int nblocks, cudaStream_t s);
template <typename R>
cudaError_t launch_get_particles(const Geom &g, int col0, const PartView<R> &v,
                                 const long long *offsets, double *out, size_t stride,
                                 cudaStream_t s);
// Copy the live particles of every slot (segment and 8 buckets) between two
// storage layouts (capacities may differ); counts are copied, clamped to the
// destination capacities.
template <typename R>
cudaError_t launch_repack(const Geom &g, SoA<R> src, const int *cnt_src, int cap_src,
                          SoA<R> bsrc, const int *bcnt_src, Buckets bk_src, SoA<R> dst,
                          int *cnt_dst, int cap_dst, SoA<R> bdst, int *bcnt_dst, Buckets bk_dst,
                          cudaStream_t s);

// Sort every patch's particles (segment plus incoming buckets, which are
// absorbed) into the interleaved cell order, through the scratch set.
template <typename R>
cudaError_t launch_sort_cells(const Geom &g, int col0, SoA<R> seg, int *cnt, SoA<R> scratch,
                              int *cnt_scratch, int cap, SoA<R> bkt, int *bcnt, Buckets bk,
                              unsigned *err, cudaStream_t s);

// old_col0: ring offset before the shift; nshift: shifts including this one.
template <typename R>
cudaError_t launch_window_particles(const Geom &g, int old_col0, int nshift, SoA<R> seg,
                                    int *cnt, SoA<R> bkt, int *bcnt, int cap, Buckets bk,
                                    double n0, double x0, double ramp, int ppcx, int ppcy,
                                    double *rho_bg, unsigned *err, cudaStream_t s);
// Initial plasma of a run: every patch filled as the window fills its new
// column (the same placement, weights and ion background).
template <typename R>
cudaError_t launch_fill_plasma(const Geom &g, int col0, int nshift, SoA<R> seg, int *cnt, int cap,
                               double n0, double x0, double ramp, int ppcx, int ppcy,
                               double *rho_bg, unsigned *err, cudaStream_t s);

}  // namespace pic
