// C-ABI of libpic (declared in include/pic.h): context, particle loading,
// the step loop (optionally replayed as CUDA graphs), moving window, field
// and particle I/O, float64 diagnostics and checkpoint/restore.
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <type_traits>
#include <vector>

#include "../../include/pic.h"
#include "alloc.h"
#include "common.cuh"
#include "noalloc.h"
#include "pack.h"
#include "pic3d.h"
#include "poisson.h"

using namespace pic;

struct pic_ctx {
  pic_config cfg;
  Geom g;
  bool fp32;
  size_t rs;  // bytes per real
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  void *F = nullptr;
  double *rho_bg = nullptr, *rho_a = nullptr, *rho_b = nullptr;
  double *laser_g = nullptr;  // transverse laser profile at y = (j + 1/2) dy
  void *seg[2][6] = {};
  int *cnt[2] = {};
  void *bkt[2][6] = {};
  int *bcnt[2] = {};
  // per-slot calm flags of the particle step (StepArgs::calm_in/out), and
  // whether they still describe the particle sets (any change of the
  // particles outside a step clears them before the next step)
  unsigned char *calm[2] = {};
  bool calm_ok = false;
  // counts of the previous state's particle sets (the inputs of the most
  // recent step), copied aside by the work plan that clears the arrays
  int *cnt_prev = nullptr, *bcnt_prev = nullptr;
  // per-slot maxima of (w |u|)^2 and w for the FP32 tile scale
  // (StepArgs::stat_in / stat_out), by step parity like calm
  unsigned *stat[2] = {};
  void *parena = nullptr;  // the one allocation all particle arrays live in
  // deterministic mode: the stored current tiles and their flags
  void *jbuf = nullptr;
  int *jflag = nullptr;
  int cap = 0;
  Buckets bk{};
  Plan plan{};
  int ps_grid = 0;
  DevState *st = nullptr;
  double *partials = nullptr;
  int npartials = 0;
  long long *offsets = nullptr;
  double *staging = nullptr;
  size_t staging_n = 0;
  // host mirrors of the device state
  long long step = 0;
  double t = 0.0;
  int nshift = 0, col0 = 0;
  // largest |w| the context holds or injects (scales the FP32 fixed-point
  // current tile; weights never change once loaded)
  double wmax = 0.0;
  bool prev_valid = false;  // previous particle state + last J usable
  CUtensorMap tmap;
  bool tmap_ok = false;
  cudaGraphExec_t gexec[2] = {nullptr, nullptr};
  // kGraphSteps consecutive steps from parity p in one graph (used when no
  // window shift or sort falls inside them)
  cudaGraphExec_t gexec_n[2] = {nullptr, nullptr};
  double ms_particles = 0, ms_fields = 0, ms_window = 0, ms_sort = 0;
  long long launches = 0, ps_launches = 0;
  int sticky = PIC_OK;
  std::string err;
  // device copy of the live state taken at the start of pic_step when the
  // capacity may grow (auto_grow): replayed after an overflow
  struct Backup {
    void *F = nullptr;        // components 0..8 (E, Bm, B)
    double *rho_bg = nullptr;
    void *seg[6] = {}, *bkt[6] = {};
    int *cnt = nullptr, *bcnt = nullptr;
    DevState *st = nullptr;
    int cap = 0;
    Buckets bk{};
    long long step = 0;
    double t = 0;
    int nshift = 0, col0 = 0;
  } bak;
  int grows = 0;
  long long sorts = 0;
  long long since_sort = 0;
  Ctx3 *c3 = nullptr;  // dims = 3: the 3D context (pic3d.cu)
  // the next step's work plan is built beside the field update on `aux`
  cudaStream_t aux = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  bool plan_ready = false;  // the plan for the current parity is built
};

namespace {
// Device memory of a 2D context (the caller's allocator when configured).
template <typename T>
cudaError_t cmalloc(pic_ctx *c, T **p, size_t bytes) {
  return dev_malloc(c->cfg, p, bytes);
}
void cfree(pic_ctx *c, void *p) { dev_free(c->cfg, c->stream, p); }
}  // namespace

namespace {

const char *kVersion = "libpic 0.2 (sm_103a, 2D3V and 3D3V SDMD patch PIC; FP64, FP32 with fixed-point current tiles)";

pic_status fail(pic_ctx *c, pic_status s, const std::string &msg) {
  if (c) c->err = msg;
  return s;
}

#define CK(call)                                                                     \
  do {                                                                               \
    cudaError_t e_ = (call);                                                         \
    if (e_ != cudaSuccess)                                                           \
      return fail(ctx, PIC_ECUDA, std::string(#call ": ") + cudaGetErrorString(e_)); \
  } while (0)

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
  }
  return fn;
}

bool valid_config(const pic_config *c, std::string &why) {
  if (!c) { why = "null config"; return false; }
  if (c->dims != 2 && c->dims != 3) { why = "dims must be 2 (2D3V) or 3 (3D3V)"; return false; }
  if (!c->dev_alloc != !c->dev_free) { why = "dev_alloc and dev_free are set together"; return false; }
  if (c->task_chunk < 0 || c->task_chunk > 4096) { why = "task_chunk must be in [0, 4096]"; return false; }
  if (c->deterministic && (c->dims != 2 || c->merge > 0 || c->current_float)) {
    why = "deterministic mode is 2D, without merge and float current accumulation";
    return false;
  }
  if (c->window_cells < 0 || (c->window_cells > 0 && c->window_cells % c->patch[0])) {
    why = "window_cells must be a multiple of patch[0]";
    return false;
  }
  if (c->dims == 3) {
    if (!valid_config3(c, why)) return false;
    if (c->prec != PIC_FP64 && c->prec != PIC_FP32) { why = "bad precision"; return false; }
    if (!(c->m > 0) || c->q == 0) { why = "mass must be positive and charge nonzero"; return false; }
    if (c->laser_on && c->bc_field[0] != PIC_BC_SILVER_MULLER) { why = "the laser needs an open x axis"; return false; }
    if (c->laser_on && !(c->laser_waist > 0 && c->laser_tau > 0)) { why = "laser waist and duration must be positive"; return false; }
    if (c->moving_window) {
      if (c->bc_field[0] != PIC_BC_SILVER_MULLER) { why = "the moving window needs an open x axis"; return false; }
      if (c->n[0] / c->patch[0] < 2) { why = "the moving window needs two patch columns"; return false; }
      if (c->inj_ppc[0] < 1 || c->inj_ppc[1] < 1 || c->inj_ppc[2] < 1) { why = "injected particles per cell must be >= 1"; return false; }
    }
    if (c->capacity_factor < 0) { why = "capacity factor must be >= 0"; return false; }
    return true;
  }
  for (int a = 0; a < 2; ++a) {
    if (c->n[a] <= 0 || c->patch[a] <= 0) { why = "cells and patch sizes must be positive"; return false; }
    if (c->patch[a] % 4 || c->patch[a] < 4 || c->patch[a] > 64) { why = "patch sizes must be multiples of 4 in [4, 64]"; return false; }
    if (c->n[a] % c->patch[a]) { why = "cells must be a multiple of the patch size"; return false; }
    if (!(c->d[a] > 0)) { why = "cell sizes must be positive"; return false; }
    if (c->bc_field[a] != PIC_BC_PERIODIC && c->bc_field[a] != PIC_BC_SILVER_MULLER) { why = "bad field boundary"; return false; }
    for (int f = 0; f < 2; ++f) {
      int b = c->bc_part[a][f];
      if (b < 0 || b > 2) { why = "bad particle boundary"; return false; }
      if ((b == PIC_PBC_PERIODIC) != (c->bc_field[a] == PIC_BC_PERIODIC)) { why = "periodic particle and field boundaries must pair"; return false; }
    }
  }
  if (c->n[0] / c->patch[0] < 1) { why = "no patches"; return false; }
  if (!(c->dt > 0) || !(c->dt < std::min(c->d[0], c->d[1]))) { why = "dt must be in (0, min(d))"; return false; }
  if (c->prec != PIC_FP64 && c->prec != PIC_FP32) { why = "bad precision"; return false; }
  if (!(c->m > 0) || c->q == 0) { why = "mass must be positive and charge nonzero"; return false; }
  if (c->laser_on && c->bc_field[0] != PIC_BC_SILVER_MULLER) { why = "the laser needs an open x axis"; return false; }
  if (c->laser_on && !(c->laser_waist > 0 && c->laser_tau > 0)) { why = "laser waist and duration must be positive"; return false; }
  if (c->moving_window) {
    if (c->bc_field[0] != PIC_BC_SILVER_MULLER) { why = "the moving window needs an open x axis"; return false; }
    if (c->n[0] / c->patch[0] < 2) { why = "the moving window needs two patch columns"; return false; }
    if (c->inj_ppc[0] < 1 || c->inj_ppc[1] < 1) { why = "injected particles per cell must be >= 1"; return false; }
  }
  if (c->capacity_factor < 0) { why = "capacity factor must be >= 0"; return false; }
  if (c->block && (c->block % 32 || c->block < 64 || c->block > 256)) { why = "block must be 64..256, a multiple of 32"; return false; }
  if (c->filter_passes < 0 || c->filter_passes > 2) { why = "filter_passes must be 0, 1 or 2"; return false; }
  return true;
}

Geom make_geom(const pic_config *c) {
  Geom g{};
  g.nx = c->n[0];
  g.ny = c->n[1];
  g.P = c->patch[0];
  g.Q = c->patch[1];
  g.npx = g.nx / g.P;
  g.npy = g.ny / g.Q;
  g.nslots = g.npx * g.npy;
  g.sx = ((g.nx + 2 * GX) + 31) / 32 * 32;
  g.nys = g.ny + 2 * GY;
  g.cs = (long long)g.sx * g.nys;
  g.dx = c->d[0];
  g.dy = c->d[1];
  g.dt = c->dt;
  g.fbc_x = c->bc_field[0];
  g.fbc_y = c->bc_field[1];
  for (int a = 0; a < 2; ++a)
    for (int f = 0; f < 2; ++f) g.pbc[a][f] = c->bc_part[a][f];
  g.q = c->q;
  g.m = c->m;
  return g;
}

size_t field_bytes(const Geom &g, size_t rs) { return (size_t)NCOMP * g.cs * rs; }
Buckets bucket_layout(int cap) {
  Buckets b{};
  int off = 0;
  for (int d = 0; d < 8; ++d) {
    int ddx, ddy;
    dir_delta(d, ddx, ddy);
    const int div = (ddx != 0 && ddy != 0) ? 4 : (ddx != 0 ? 1 : 2);
    b.cap[d] = std::max(32, (cap / div + 31) / 32 * 32);
    b.off[d] = off;
    off += b.cap[d];
  }
  b.stride = off;
  return b;
}
size_t particle_bytes(const Geom &g, int cap, size_t rs) {
  const Buckets b = bucket_layout(cap);
  return 2 * (6 * rs * ((size_t)g.nslots * cap + (size_t)g.nslots * b.stride) +
              sizeof(int) * ((size_t)g.nslots + (size_t)g.nslots * 8));
}

template <typename R>
SoA<R> soa(void *const a[6]) {
  return SoA<R>{(R *)a[0], (R *)a[1], (R *)a[2], (R *)a[3], (R *)a[4], (R *)a[5]};
}

template <typename R>
PartView<R> view(pic_ctx *c, int segset, int bktset) {
  PartView<R> v;
  v.seg = soa<R>(c->seg[segset]);
  v.cnt = c->cnt[segset];
  v.bkt = soa<R>(c->bkt[bktset]);
  v.bcnt = c->bcnt[bktset];
  v.cap = c->cap;
  v.bk = c->bk;
  return v;
}

pic_status check_usable(pic_ctx *ctx) {
  if (!ctx) return PIC_EINVAL;
  if (ctx->sticky != PIC_OK) return fail(ctx, PIC_ESTATE, "context holds a device fault: restore a snapshot");
  return PIC_OK;
}

// Read the sticky device word; convert it to a status.
pic_status poll_device(pic_ctx *ctx) {
  CK(cudaStreamSynchronize(ctx->stream));
  DevState h;
  CK(cudaMemcpy(&h, ctx->st, sizeof h, cudaMemcpyDeviceToHost));
  if (h.err) {
    pic_status s = PIC_ENONFINITE;
    std::string m = "device fault:";
    if (h.err & ERR_TIMEOUT) { s = PIC_ETIMEOUT; m += " staging wait ran out;"; }
    if (h.err & (ERR_OVERFLOW_SEG | ERR_OVERFLOW_BKT | ERR_OVERFLOW_LOAD)) {
      if (s != PIC_ETIMEOUT) s = PIC_EOVERFLOW;
      m += " patch capacity exceeded (raise capacity_factor);";
    }
    if (h.err & ERR_NONFINITE) m += " non-finite particle;";
    if (h.err & ERR_FAST) m += " particle moved more than one cell;";
    if (h.err & ERR_LOAD_RANGE) { s = PIC_EINVAL; m += " particle outside the domain;"; }
    if (h.err & ERR_BOUNDS) { s = PIC_ECUDA; m += " index out of bounds (checked build);"; }
    ctx->sticky = s;
    return fail(ctx, s, m);
  }
  return PIC_OK;
}

// Particles per work item of the 2D particle step unless configured: a
// whole 32 x 32-cell patch at 4 per cell in FP32 (the per-item fixed-point
// scale keeps the current resolution), 2048 in FP64 (one block per SM; more
// items balance better).
template <typename R>
constexpr int default_chunk() { return sizeof(R) == 4 ? 4096 : 2048; }

template <typename R>
pic_status alloc_particles(pic_ctx *ctx, int cap) {
  ctx->cap = cap;
  ctx->bk = bucket_layout(cap);
  const Geom &g = ctx->g;
  const bool merge = ctx->cfg.merge > 0;
  Plan &pl = ctx->plan;
  pl.unit = merge ? (int)(16 / sizeof(R)) : 1;
  const int chunk_particles = ctx->cfg.task_chunk > 0 ? ctx->cfg.task_chunk : default_chunk<R>();
  pl.chunk = std::max(1, chunk_particles / pl.unit);
  // work plan: a slot holds at most cap + bucket stride particles per step
  const long long units_max = (long long)(cap + ctx->bk.stride) / pl.unit + 9;
  const bool det = ctx->cfg.deterministic != 0;
  if (det) pl.chunk = (int)units_max;  // one work item per patch
  pl.max_items = (int)std::min<long long>((long long)g.nslots * ((units_max + pl.chunk - 1) / pl.chunk),
                                          1ll << 30);
  // every array of the particle storage carved from one allocation (one
  // allocator call for the load), 256-byte aligned
  char *base = nullptr;
  size_t used = 0;
  auto carve = [&](auto **p, size_t bytes) {
    used = (used + 255) & ~(size_t)255;
    *p = reinterpret_cast<std::remove_reference_t<decltype(*p)>>(base ? base + used : nullptr);
    used += bytes;
  };
  for (int pass = 0; pass < 2; ++pass) {
    used = 0;
    for (int s = 0; s < 2; ++s) {
      for (int a = 0; a < 6; ++a) {
        carve(reinterpret_cast<R **>(&ctx->seg[s][a]), sizeof(R) * (size_t)g.nslots * cap);
        carve(reinterpret_cast<R **>(&ctx->bkt[s][a]), sizeof(R) * (size_t)g.nslots * ctx->bk.stride);
      }
      carve(&ctx->cnt[s], sizeof(int) * g.nslots);
      carve(&ctx->bcnt[s], sizeof(int) * g.nslots * 8);
      carve(&ctx->calm[s], (size_t)g.nslots);
      carve(&ctx->stat[s], sizeof(unsigned) * 2 * g.nslots);
    }
    carve(&ctx->cnt_prev, sizeof(int) * g.nslots);
    carve(&ctx->bcnt_prev, sizeof(int) * g.nslots * 8);
    carve(&ctx->offsets, sizeof(long long) * (g.nslots * 9 + 1));
    carve(&pl.item_slot, sizeof(int) * pl.max_items);
    carve(&pl.item_first, sizeof(int) * pl.max_items);
    carve(&pl.n_items, sizeof(int) * 2);
    carve(&pl.units, sizeof(int) * g.nslots);
    if (det) {
      carve(reinterpret_cast<R **>(&ctx->jbuf), sizeof(R) * (size_t)g.nslots * 3 * (g.P + 5) * (g.Q + 5));
      carve(&ctx->jflag, sizeof(int) * g.nslots);
    }
    if (pass == 0) {
      CK(cmalloc(ctx, &ctx->parena, used));
      base = static_cast<char *>(ctx->parena);
    }
  }
  pl.next = pl.n_items + 1;
  for (int s = 0; s < 2; ++s) {
    CK(cudaMemsetAsync(ctx->cnt[s], 0, sizeof(int) * g.nslots, ctx->stream));
    CK(cudaMemsetAsync(ctx->bcnt[s], 0, sizeof(int) * g.nslots * 8, ctx->stream));
  }
  CK(cudaMemsetAsync(ctx->cnt_prev, 0, sizeof(int) * g.nslots, ctx->stream));
  CK(cudaMemsetAsync(ctx->bcnt_prev, 0, sizeof(int) * g.nslots * 8, ctx->stream));
  ctx->calm_ok = false;
  return PIC_OK;
}

void free_graphs(pic_ctx *c) {
  for (int p = 0; p < 2; ++p)
    if (c->gexec_n[p]) {
      cudaGraphExecDestroy(c->gexec_n[p]);
      c->gexec_n[p] = nullptr;
    }
  for (int p = 0; p < 2; ++p)
    if (c->gexec[p]) {
      cudaGraphExecDestroy(c->gexec[p]);
      c->gexec[p] = nullptr;
    }
}

template <typename R>
pic_status build_tmap(pic_ctx *ctx) {
  if (ctx->cfg.tma == 0) return PIC_OK;
  auto enc = encode_fn();
  if (!enc) return fail(ctx, PIC_ECUDA, "cuTensorMapEncodeTiled is not available");
  const Geom &g = ctx->g;
  cuuint64_t dims[3] = {(cuuint64_t)g.sx, (cuuint64_t)g.nys, 6};
  cuuint64_t strides[2] = {(cuuint64_t)g.sx * sizeof(R), (cuuint64_t)g.cs * sizeof(R)};
  cuuint32_t box[3] = {(cuuint32_t)(g.P + 8), (cuuint32_t)(g.Q + 3), 6};
  cuuint32_t es[3] = {1, 1, 1};
  CUresult r = enc(&ctx->tmap,
                   sizeof(R) == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64,
                   3, ctx->F, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(ctx, PIC_ECUDA, "cuTensorMapEncodeTiled failed");
  ctx->tmap_ok = true;
  return PIC_OK;
}

// Arguments of the particle step of parity p: reads segment set p and the
// bucket set 1 - p, writes segment set 1 - p, bucket set p and current set p.
// Fixed-point scales of the FP32 current tile for work items of at most
// per_item particles (see StepArgs::jscale).  Every contribution of a
// particle of weight w is below (3/4) |q| w in magnitude:
//   x: (q dx/dt) w P A with P a prefix sum of S1 - S0.  The prefix sum of
//      the quadratic shape weights changes with position at a rate equal to
//      a linear hat, at most 1, so |P| <= |dx_cells| = |v_x| dt/dx < dt/dx;
//      A = (S0 + S1)/2 <= 3/4.  y alike;
//   z: q w v_z W_z with |v_z| < 1 and W_z <= (3/4)^2.
// The scale 2^K / ((3/4)^2 |q| w_max) therefore keeps each contribution
// below (4/3) 2^K and an item's sums below (4/3) per_item 2^K <= (4/3) 2^30,
// inside the 32-bit range.  K <= 20 keeps every contribution below 2^22,
// the range in which the 2D kernel rounds it by adding 1.5 * 2^23.
template <typename R>
void set_current_scale(StepArgs<R> &a, const Geom &g, double wmax, int per_item) {
  int lg = 0;
  while ((1 << lg) < per_item) ++lg;
  const double two_k = std::ldexp(1.0, std::min(30 - lg, 20));
  const double c = 0.5625 * std::fabs(g.q);
  // a floor on w_max keeps the scale finite in FP32 (tinier weights only
  // lose resolution)
  const double wm = c > 0 ? std::max(wmax, two_k / (c * 1e30)) : 0.0;
  const double sc = c > 0 ? two_k / (c * wm) : 0.0;
  for (int k = 0; k < 3; ++k) {
    a.jscale[k] = R(sc);
    a.junit[k] = sc > 0 ? R(1.0 / sc) : R(0);
  }
}

template <typename R>
StepArgs<R> step_args(const pic_ctx *ctx, int p) {
  const Geom &g = ctx->g;
  StepArgs<R> a;
  a.g = g;
  a.F = (const R *)ctx->F;
  a.Jdst = (R *)ctx->F + (C_JA + 3 * p) * g.cs;
  a.pin = soa<R>(ctx->seg[p]);
  a.pout = soa<R>(ctx->seg[1 - p]);
  a.cnt_in = ctx->cnt[p];
  a.cnt_out = ctx->cnt[1 - p];
  a.bin = soa<R>(ctx->bkt[1 - p]);
  a.bout = soa<R>(ctx->bkt[p]);
  a.bcnt_in = ctx->bcnt[1 - p];
  a.bcnt_out = ctx->bcnt[p];
  a.calm_in = ctx->calm[p];
  a.calm_out = ctx->calm[1 - p];
  a.cnt_prev = ctx->cnt_prev;
  a.bcnt_prev = ctx->bcnt_prev;
  a.stat_in = ctx->stat[p];
  a.stat_out = ctx->stat[1 - p];
  a.jk = R(g.q != 0.0 ? 1.0 / (0.5625 * std::fabs(g.q)) : 0.0);
  a.wait_polls = wait_polls_of(ctx->cfg.staging_wait_polls);
  a.det = ctx->cfg.deterministic != 0;
  a.jbuf = (R *)ctx->jbuf;
  a.jflag = ctx->jflag;
  a.wglob = R(ctx->wmax);
  a.cap = ctx->cap;
  a.bk = ctx->bk;
  a.parity = p;
  a.st = ctx->st;
  a.rdx = R(g.dt / g.dx);
  a.rdy = R(g.dt / g.dy);
  a.eps = R(g.q * g.dt / (2.0 * g.m));
  a.cjx = R(-g.q * g.dx / g.dt);
  a.cjy = R(-g.q * g.dy / g.dt);
  a.cjz = R(g.q);
  a.RP = R(g.P);
  a.RQ = R(g.Q);
  a.plan = ctx->plan;
  set_current_scale(a, g, ctx->wmax,
                    ctx->plan.chunk > 0 ? ctx->plan.chunk * ctx->plan.unit : 2048);
  a.jfloat = ctx->cfg.current_float != 0;
  return a;
}

// Arguments of the field update of parity p (constants in the working
// precision computed here, on the host).
template <typename R>
FieldArgs<R> field_args(const pic_ctx *ctx, int p) {
  const Geom &g = ctx->g;
  FieldArgs<R> f;
  f.g = g;
  f.F = (R *)ctx->F;
  f.parity = p;
  f.st = ctx->st;
  f.dt = R(g.dt);
  f.idx = R(1.0 / g.dx);
  f.idy = R(1.0 / g.dy);
  const double rx = g.dt / g.dx, ry = g.dt / g.dy;
  f.smx_inv1pr = R(1.0 / (1.0 + rx));
  f.smx_1mr = R(1.0 - rx);
  f.smx_dtt = R(g.dt / g.dy);
  f.smy_inv1pr = R(1.0 / (1.0 + ry));
  f.smy_1mr = R(1.0 - ry);
  f.smy_dtt = R(g.dt / g.dx);
  f.laser_on = ctx->cfg.laser_on;
  f.laser_g = ctx->laser_g;
  f.tau = ctx->cfg.laser_tau;
  f.t_peak = ctx->cfg.laser_t_peak;
  f.filter_passes = ctx->cfg.filter_passes;
  return f;
}

// One step on the context's stream: the patch particle step (its work plan
// first when with_plan), then the region field update, beside which the
// next step's work plan is built on the auxiliary stream (it reads only the
// particle counts the step just wrote).  `mid` (optional) is recorded
// between the two phases.
template <typename R>
pic_status enqueue_step(pic_ctx *ctx, int parity, bool with_plan, cudaEvent_t mid = nullptr) {
  const Geom &g = ctx->g;
  const StepArgs<R> a = step_args<R>(ctx, parity);
  const int block = ctx->cfg.block ? ctx->cfg.block : 256;
  const bool merge = ctx->cfg.merge > 0;
  if (!ctx->ps_grid) {
    ctx->ps_grid = particle_step_grid<R>(g.P, g.Q, ctx->cfg.tma != 0, merge, block,
                                         ctx->cfg.current_float != 0);
    if (ctx->ps_grid <= 0) return fail(ctx, PIC_ECUDA, "particle step occupancy query failed");
  }
  CK(launch_particle_step<R>(a, &ctx->tmap, ctx->cfg.tma != 0, merge, block, ctx->ps_grid,
                             with_plan, ctx->stream));
  if (a.det) CK(launch_gather_current<R>(a, ctx->stream));
  if (mid) CK(cudaEventRecord(mid, ctx->stream));
  CK(cudaEventRecord(ctx->ev_fork, ctx->stream));
  CK(cudaStreamWaitEvent(ctx->aux, ctx->ev_fork, 0));
  CK(launch_plan<R>(step_args<R>(ctx, 1 - parity), true, ctx->aux));
  CK(cudaEventRecord(ctx->ev_join, ctx->aux));
  CK(launch_fields<R>(field_args<R>(ctx, parity), ctx->stream));
  CK(cudaStreamWaitEvent(ctx->stream, ctx->ev_join, 0));
  return PIC_OK;
}

int kernels_per_step(const pic_ctx *c) {
  return 4 + ((c->g.fbc_x == FBC_SM || c->g.fbc_y == FBC_SM) ? 1 : 0) +
         (c->cfg.filter_passes > 0 ? 1 : 0) + (c->cfg.deterministic ? 1 : 0);
}

__global__ void k_window_state(DevState *st, int col0, int nshift) {
  st->col0 = col0;
  st->nshift = nshift;
}

// After a window shift only two slot columns hold changed particles: c0
// (refilled with the new plasma column) and c1 (which received the
// in-flight particles of the dropped column).  Their calm flags and scale
// statistics (both parities) are reset; every other slot keeps its
// particles, and the fields moved with the frame, so its flags stay valid.
__global__ void k_calm_columns(unsigned char *calm0, unsigned char *calm1, unsigned *stat0,
                               unsigned *stat1, int npx, int npy, int c0, int c1) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 2 * npy) return;
  const int slot = (t >> 1) * npx + ((t & 1) ? c1 : c0);
  calm0[slot] = 0;
  calm1[slot] = 0;
  stat0[2 * slot] = stat0[2 * slot + 1] = 0x7f7f7f7fu;  // unknown: see ensure_calm
  stat1[2 * slot] = stat1[2 * slot + 1] = 0x7f7f7f7fu;
}

template <typename R>
pic_status window_shift(pic_ctx *ctx) {
  const Geom &g = ctx->g;
  const int q = (int)(ctx->step & 1);     // current segment set
  const int bset = 1 - q;                 // current bucket set
  const int last_j = 1 - q;               // J set of the step just taken
  R *F = (R *)ctx->F;
  CK(launch_shift_fields<R>(g, F, 9, ctx->stream));
  CK(launch_shift_fields<R>(g, F + (C_JA + 3 * last_j) * g.cs, 3, ctx->stream));
  CK(launch_shift_f64(g, ctx->rho_bg, ctx->stream));
  const int old_col0 = ctx->col0;
  ctx->nshift += 1;
  ctx->col0 = (old_col0 + 1) % g.npx;
  CK(launch_window_particles<R>(g, old_col0, ctx->nshift, soa<R>(ctx->seg[q]), ctx->cnt[q],
                                soa<R>(ctx->bkt[bset]), ctx->bcnt[bset], ctx->cap, ctx->bk,
                                ctx->cfg.inj_n0, ctx->cfg.inj_x0, ctx->cfg.inj_ramp,
                                ctx->cfg.inj_ppc[0], ctx->cfg.inj_ppc[1], ctx->rho_bg,
                                &ctx->st->err, ctx->stream));
  k_window_state<<<1, 1, 0, ctx->stream>>>(ctx->st, ctx->col0, ctx->nshift);
  ctx->launches += 7;
  if (ctx->calm_ok) {
    k_calm_columns<<<(2 * g.npy + 255) / 256, 256, 0, ctx->stream>>>(
        ctx->calm[0], ctx->calm[1], ctx->stat[0], ctx->stat[1], g.npx, g.npy, old_col0, ctx->col0);
    ctx->launches += 1;
  }
  CK(cudaGetLastError());
  ctx->prev_valid = false;
  ctx->plan_ready = false;  // particle counts changed
  return PIC_OK;
}

// Patch columns per window step.
int window_columns(const pic_config &c) {
  return c.window_cells > 0 ? c.window_cells / c.patch[0] : 1;
}

bool window_due_at(const pic_ctx *c, double t) {
  const int m = window_columns(c->cfg);
  return c->cfg.moving_window && t > c->cfg.mw_t0 &&
         t - c->cfg.mw_t0 >= (c->nshift / m + 1) * (double)m * c->g.P * c->g.dx;
}
bool window_due(const pic_ctx *c) { return window_due_at(c, c->t); }
// Steps of one multi-step graph replay.
constexpr int kGraphSteps = 8;
// True when the next kGraphSteps steps may run as one graph: no window shift
// due after any but the last of them (the time advanced as the steps
// advance it) and no cell-order sort due before the last.
bool graph_run_ok(const pic_ctx *c) {
  double t = c->t;
  for (int k = 1; k < kGraphSteps; ++k) {
    t += c->g.dt;
    if (window_due_at(c, t)) return false;
  }
  return !(c->cfg.sort_every > 0 && c->since_sort + kGraphSteps > c->cfg.sort_every);
}

template <typename R>
pic_status capture_graphs(pic_ctx *ctx) {
  for (int n : {1, kGraphSteps})
    for (int p = 0; p < 2; ++p) {
      cudaGraph_t gr;
      CK(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
      pic_status s = PIC_OK;
      for (int k = 0; k < n && s == PIC_OK; ++k)
        s = enqueue_step<R>(ctx, p ^ (k & 1), false);  // replays follow a built plan
      cudaError_t e = cudaStreamEndCapture(ctx->stream, &gr);
      if (s != PIC_OK) return s;
      CK(e);
      e = cudaGraphInstantiate(n == 1 ? &ctx->gexec[p] : &ctx->gexec_n[p], gr, 0);
      cudaGraphDestroy(gr);
      CK(e);
    }
  return PIC_OK;
}

void free_backup(pic_ctx *c) {
  auto &b = c->bak;
  cfree(c, b.F);
  cfree(c, b.rho_bg);
  for (int a = 0; a < 6; ++a) {
    cfree(c, b.seg[a]);
    cfree(c, b.bkt[a]);
  }
  cfree(c, b.cnt);
  cfree(c, b.bcnt);
  cfree(c, b.st);
  b = pic_ctx::Backup{};
}

void free_particles(pic_ctx *c) {
  cfree(c, c->parena);  // every array of the particle storage (alloc_particles)
  c->parena = nullptr;
  for (int s = 0; s < 2; ++s) {
    for (int a = 0; a < 6; ++a) c->seg[s][a] = c->bkt[s][a] = nullptr;
    c->cnt[s] = c->bcnt[s] = nullptr;
    c->calm[s] = nullptr;
    c->stat[s] = nullptr;
  }
  c->cnt_prev = c->bcnt_prev = nullptr;
  c->offsets = nullptr;
  c->jbuf = nullptr;
  c->jflag = nullptr;
  c->plan = Plan{};
}

// Copy the live state (current particle set and in-flight buckets, E, Bm,
// B, background charge, device scalars) into the backup.
template <typename R>
pic_status take_backup(pic_ctx *ctx) {
  auto &b = ctx->bak;
  const Geom &g = ctx->g;
  if (b.cap != ctx->cap) free_backup(ctx);
  if (!b.F) {
    b.cap = ctx->cap;
    b.bk = ctx->bk;
    CK(cmalloc(ctx, &b.F, 9 * g.cs * sizeof(R)));
    CK(cmalloc(ctx, &b.rho_bg, g.cs * sizeof(double)));
    for (int a = 0; a < 6; ++a) {
      CK(cmalloc(ctx, &b.seg[a], sizeof(R) * (size_t)g.nslots * b.cap));
      CK(cmalloc(ctx, &b.bkt[a], sizeof(R) * (size_t)g.nslots * b.bk.stride));
    }
    CK(cmalloc(ctx, &b.cnt, sizeof(int) * g.nslots));
    CK(cmalloc(ctx, &b.bcnt, sizeof(int) * g.nslots * 8));
    CK(cmalloc(ctx, &b.st, sizeof(DevState)));
  }
  const int q = (int)(ctx->step & 1);
  CK(cudaMemcpyAsync(b.F, ctx->F, 9 * g.cs * sizeof(R), cudaMemcpyDeviceToDevice, ctx->stream));
  CK(cudaMemcpyAsync(b.rho_bg, ctx->rho_bg, g.cs * sizeof(double), cudaMemcpyDeviceToDevice,
                     ctx->stream));
  CK(launch_repack<R>(g, soa<R>(ctx->seg[q]), ctx->cnt[q], ctx->cap, soa<R>(ctx->bkt[1 - q]),
                      ctx->bcnt[1 - q], ctx->bk, soa<R>(b.seg), b.cnt, b.cap, soa<R>(b.bkt),
                      b.bcnt, b.bk, ctx->stream));
  CK(cudaMemcpyAsync(b.st, ctx->st, sizeof(DevState), cudaMemcpyDeviceToDevice, ctx->stream));
  b.step = ctx->step;
  b.t = ctx->t;
  b.nshift = ctx->nshift;
  b.col0 = ctx->col0;
  ctx->launches += 1;
  return PIC_OK;
}

// Return to the backup with a patch capacity of new_cap (particle storage
// reallocated and repacked when it changes); clears the device fault.
template <typename R>
pic_status restore_backup(pic_ctx *ctx, int new_cap) {
  auto &b = ctx->bak;
  const Geom &g = ctx->g;
  CK(cudaStreamSynchronize(ctx->stream));
  if (new_cap != ctx->cap) {
    free_graphs(ctx);
    free_particles(ctx);
    pic_status s = alloc_particles<R>(ctx, new_cap);
    if (s) return s;
  }
  const int q = (int)(b.step & 1);
  CK(cudaMemcpyAsync(ctx->F, b.F, 9 * g.cs * sizeof(R), cudaMemcpyDeviceToDevice, ctx->stream));
  CK(cudaMemsetAsync((R *)ctx->F + C_JA * g.cs, 0, 6 * g.cs * sizeof(R), ctx->stream));
  CK(cudaMemcpyAsync(ctx->rho_bg, b.rho_bg, g.cs * sizeof(double), cudaMemcpyDeviceToDevice,
                     ctx->stream));
  CK(cudaMemsetAsync(ctx->cnt[1 - q], 0, sizeof(int) * g.nslots, ctx->stream));
  CK(cudaMemsetAsync(ctx->bcnt[q], 0, sizeof(int) * g.nslots * 8, ctx->stream));
  CK(launch_repack<R>(g, soa<R>(b.seg), b.cnt, b.cap, soa<R>(b.bkt), b.bcnt, b.bk,
                      soa<R>(ctx->seg[q]), ctx->cnt[q], ctx->cap, soa<R>(ctx->bkt[1 - q]),
                      ctx->bcnt[1 - q], ctx->bk, ctx->stream));
  DevState ds;
  CK(cudaMemcpyAsync(&ds, b.st, sizeof ds, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  ds.err = 0;
  CK(cudaMemcpy(ctx->st, &ds, sizeof ds, cudaMemcpyHostToDevice));
  ctx->step = b.step;
  ctx->t = b.t;
  ctx->nshift = b.nshift;
  ctx->col0 = b.col0;
  ctx->prev_valid = false;
  ctx->plan_ready = false;
  ctx->calm_ok = false;
  ctx->sticky = PIC_OK;
  ctx->launches += 1;
  return PIC_OK;
}

// Sort the live particles into the interleaved cell order (the other
// segment set is scratch at this point; in-flight buckets are absorbed).
template <typename R>
pic_status sort_particles(pic_ctx *ctx) {
  const int q = (int)(ctx->step & 1);
  CK(launch_sort_cells<R>(ctx->g, ctx->col0, soa<R>(ctx->seg[q]), ctx->cnt[q],
                          soa<R>(ctx->seg[1 - q]), ctx->cnt[1 - q], ctx->cap,
                          soa<R>(ctx->bkt[1 - q]), ctx->bcnt[1 - q], ctx->bk, &ctx->st->err,
                          ctx->stream));
  ctx->launches += 2;
  ctx->sorts += 1;
  ctx->prev_valid = false;
  ctx->plan_ready = false;
  ctx->calm_ok = false;
  return PIC_OK;
}

template <typename R>
pic_status run_steps(pic_ctx *ctx, int nsteps);

// Clear the calm flags when the particles changed outside a step since
// they were written (load, restore, window shift, sort, regrow).
pic_status ensure_calm(pic_ctx *ctx, cudaStream_t s) {
  if (ctx->calm_ok) return PIC_OK;
  for (int k = 0; k < 2; ++k) {
    CK(cudaMemsetAsync(ctx->calm[k], 0, ctx->g.nslots, s));
    // unknown maxima: huge (0x7f7f7f7f), so the FP32 tile bound falls back
    // to the run's largest weight with |v| <= 1
    CK(cudaMemsetAsync(ctx->stat[k], 0x7f, sizeof(unsigned) * 2 * ctx->g.nslots, s));
  }
  ctx->calm_ok = true;
  return PIC_OK;
}

// Advance nsteps; with auto_grow, an overflow of a patch or bucket capacity
// grows the capacity and replays the steps from the state at entry.
template <typename R>
pic_status do_step(pic_ctx *ctx, int nsteps) {
  if (!ctx->cap) return fail(ctx, PIC_ESTATE, "no particles loaded");
  if (!ctx->cfg.auto_grow) return run_steps<R>(ctx, nsteps);
  pic_status s = take_backup<R>(ctx);
  if (s) return s;
  for (int attempt = 0;; ++attempt) {
    s = run_steps<R>(ctx, nsteps);
    if (s != PIC_EOVERFLOW || attempt >= 4) return s;
    DevState h;
    CK(cudaMemcpy(&h, ctx->st, sizeof h, cudaMemcpyDeviceToHost));
    const int seen = std::max(h.maxcnt[0], h.maxcnt[1]);
    int cap = std::max((int)(1.5 * ctx->cap), (int)(1.25 * seen));
    cap = (cap + 31) / 32 * 32;
    s = restore_backup<R>(ctx, cap);
    if (s) return s;
    ctx->grows += 1;
  }
}

template <typename R>
pic_status run_steps(pic_ctx *ctx, int nsteps) {
  if (!ctx->cap) return fail(ctx, PIC_ESTATE, "no particles loaded");
  if (ctx->cfg.tma && !ctx->tmap_ok) {
    pic_status s = build_tmap<R>(ctx);
    if (s) return s;
  }
  CK(prepare_particle_step<R>(ctx->g.P, ctx->g.Q));
  const bool timing = ctx->cfg.timing != 0;
  const bool use_graph = ctx->cfg.use_graph && !timing;
  if (use_graph && !ctx->gexec[0]) {
    pic_status s = capture_graphs<R>(ctx);
    if (s) return s;
  }
  // timing: three events per step (start, between phases, end) and two per
  // window shift, read back once after the loop
  std::vector<cudaEvent_t> ev;
  std::vector<int> kind;  // 0: step triple, 1: window pair, 2: sort pair
  auto new_event = [&](cudaEvent_t *e) -> cudaError_t { return cudaEventCreate(e); };
  pic_status rs = PIC_OK;
  for (int n = 0; n < nsteps && rs == PIC_OK; ++n) {
    const int p = (int)(ctx->step & 1);
    if (ctx->cfg.sort_every > 0 && ctx->since_sort >= ctx->cfg.sort_every) {
      cudaEvent_t e[2];
      if (timing) {
        for (int k = 0; k < 2; ++k) CK(new_event(&e[k]));
        CK(cudaEventRecord(e[0], ctx->stream));
      }
      rs = sort_particles<R>(ctx);
      if (timing) {
        CK(cudaEventRecord(e[1], ctx->stream));
        ev.push_back(e[0]);
        ev.push_back(e[1]);
        kind.push_back(2);
      }
      if (rs) break;
      ctx->since_sort = 0;
    }
    ctx->since_sort += 1;
    {
      const pic_status cs = ensure_calm(ctx, ctx->stream);
      if (cs) return cs;
    }
    int adv = 1;  // steps this iteration advances
    if (use_graph) {
      if (!ctx->plan_ready) {
        CK(launch_plan<R>(step_args<R>(ctx, p), false, ctx->stream));
        ctx->launches += 1;
      }
      if (nsteps - n >= kGraphSteps && graph_run_ok(ctx)) {
        CK(cudaGraphLaunch(ctx->gexec_n[p], ctx->stream));
        adv = kGraphSteps;
      } else {
        CK(cudaGraphLaunch(ctx->gexec[p], ctx->stream));
      }
    } else if (timing) {
      cudaEvent_t e[3];
      for (int k = 0; k < 3; ++k) CK(new_event(&e[k]));
      CK(cudaEventRecord(e[0], ctx->stream));
      rs = enqueue_step<R>(ctx, p, !ctx->plan_ready, e[1]);
      CK(cudaEventRecord(e[2], ctx->stream));
      for (int k = 0; k < 3; ++k) ev.push_back(e[k]);
      kind.push_back(0);
      if (!ctx->plan_ready) ctx->launches += 1;
    } else {
      rs = enqueue_step<R>(ctx, p, !ctx->plan_ready);
      if (!ctx->plan_ready) ctx->launches += 1;
    }
    ctx->plan_ready = true;
    for (int k = 0; k < adv; ++k) {
      ctx->launches += kernels_per_step(ctx);
      ctx->ps_launches += 1;
      ctx->step += 1;
      ctx->t += ctx->g.dt;
    }
    ctx->since_sort += adv - 1;
    n += adv - 1;
    ctx->prev_valid = true;
    if (rs == PIC_OK && window_due(ctx)) {
      cudaEvent_t e[2];
      if (timing) {
        for (int k = 0; k < 2; ++k) CK(new_event(&e[k]));
        CK(cudaEventRecord(e[0], ctx->stream));
      }
      for (int k = 0; k < window_columns(ctx->cfg) && rs == PIC_OK; ++k) rs = window_shift<R>(ctx);
      if (timing) {
        CK(cudaEventRecord(e[1], ctx->stream));
        ev.push_back(e[0]);
        ev.push_back(e[1]);
        kind.push_back(1);
      }
    }
  }
  if (!ev.empty()) {
    CK(cudaStreamSynchronize(ctx->stream));
    size_t k = 0;
    for (int t : kind) {
      float a = 0, b = 0;
      if (t == 0) {
        CK(cudaEventElapsedTime(&a, ev[k], ev[k + 1]));
        CK(cudaEventElapsedTime(&b, ev[k + 1], ev[k + 2]));
        ctx->ms_particles += a;
        ctx->ms_fields += b;
        k += 3;
      } else {
        CK(cudaEventElapsedTime(&a, ev[k], ev[k + 1]));
        (t == 1 ? ctx->ms_window : ctx->ms_sort) += a;
        k += 2;
      }
    }
    for (cudaEvent_t e : ev) cudaEventDestroy(e);
  }
  if (rs) return rs;
  return poll_device(ctx);
}

const void *pinned_view(const void *host);
pic_status ensure_staging(pic_ctx *ctx, size_t n);

template <typename R>
pic_status do_load(pic_ctx *ctx, const double *x, const double *y, const double *ux,
                   const double *uy, const double *uz, const double *w, size_t n, int where) {
  const Geom &g = ctx->g;
  const double *src[6] = {x, y, ux, uy, uz, w};
  const double *d[6];
  double *tmp = nullptr;  // a staging copy for pageable host arrays
  if (where == PIC_HOST) {
    bool pinned = true;
    for (int a = 0; a < 6 && pinned; ++a) pinned = (d[a] = (const double *)pinned_view(src[a])) != nullptr;
    if (!pinned) {
      // (device memory of this call only: a load is not on the stepping path)
      CK(cmalloc(ctx, &tmp, sizeof(double) * 6 * std::max<size_t>(n, 1)));
      for (int a = 0; a < 6; ++a) {
        CK(cudaMemcpyAsync(tmp + a * n, src[a], sizeof(double) * n, cudaMemcpyHostToDevice,
                           ctx->stream));
        d[a] = tmp + a * n;
      }
    }
  } else {
    for (int a = 0; a < 6; ++a) d[a] = src[a];
  }
  const int q = (int)(ctx->step & 1);
  pic_status rs = PIC_OK;
  // validation / counting pass: particles outside the domain reject the
  // whole call without touching the stored particles
  int *cnt = nullptr;
  CK(cmalloc(ctx, &cnt, sizeof(int) * g.nslots));
  CK(cudaMemsetAsync(cnt, 0, sizeof(int) * g.nslots, ctx->stream));
  CK(launch_bin_count<R>(g, ctx->col0, d[0], d[1], n, cnt, &ctx->st->err, ctx->stream));
  // largest |w| of the call (float64 bits; +inf for a non-finite weight)
  unsigned long long *wbits = reinterpret_cast<unsigned long long *>(ctx->partials);
  CK(cudaMemsetAsync(wbits, 0, sizeof *wbits, ctx->stream));
  CK(launch_absmax_f64(d[5], n, wbits, ctx->stream));
  unsigned long long hw = 0;
  CK(cudaMemcpyAsync(&hw, wbits, sizeof hw, cudaMemcpyDeviceToHost, ctx->stream));
  std::vector<int> h(g.nslots);
  CK(cudaMemcpyAsync(h.data(), cnt, sizeof(int) * g.nslots, cudaMemcpyDeviceToHost, ctx->stream));
  DevState hs;
  CK(cudaMemcpyAsync(&hs, ctx->st, sizeof hs, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  cfree(ctx, cnt);
  ctx->launches += 2;
  if (hs.err & ERR_LOAD_RANGE) {
    unsigned zero = hs.err & ~ERR_LOAD_RANGE;
    CK(cudaMemcpy(&ctx->st->err, &zero, sizeof zero, cudaMemcpyHostToDevice));
    if (tmp) cfree(ctx, tmp);
    return fail(ctx, PIC_EINVAL, "particle position outside the domain");
  }
  double wl = 0.0;
  memcpy(&wl, &hw, sizeof wl);
  if (!std::isfinite(wl)) {
    if (tmp) cfree(ctx, tmp);
    return fail(ctx, PIC_EINVAL, "non-finite particle weight");
  }
  ctx->wmax = std::max(ctx->wmax, wl);
  if (!ctx->cap) {
    int mx = *std::max_element(h.begin(), h.end());
    double cf = ctx->cfg.capacity_factor > 0 ? ctx->cfg.capacity_factor : 2.0;
    int cmin = ctx->cfg.capacity_min > 0 ? ctx->cfg.capacity_min : 256;
    if (ctx->cfg.moving_window) {
      int inj = g.P * g.Q * ctx->cfg.inj_ppc[0] * ctx->cfg.inj_ppc[1];
      mx = std::max(mx, inj);
    }
    int cap = std::max(cmin, (int)std::ceil(cf * mx));
    cap = (cap + 31) / 32 * 32;
    rs = alloc_particles<R>(ctx, cap);
    if (rs) return rs;
  }
  CK(launch_bin_place<R>(g, ctx->col0, d[0], d[1], d[2], d[3], d[4], d[5], n,
                         soa<R>(ctx->seg[q]), ctx->cnt[q], ctx->cap, &ctx->st->err, ctx->stream));
  CK(launch_clamp_counts(ctx->cnt[q], g.nslots, ctx->cap, ctx->stream));
  ctx->launches += 2;
  if (ctx->cfg.sort_every > 0) {
    pic_status ss = sort_particles<R>(ctx);
    if (ss) return ss;
    ctx->since_sort = 0;
  }
  // clamp counts of overflowing slots happens via the error word
  if (tmp) {
    CK(cudaStreamSynchronize(ctx->stream));
    cfree(ctx, tmp);
  }
  ctx->prev_valid = false;
  ctx->plan_ready = false;
  ctx->calm_ok = false;
  free_graphs(ctx);  // capacity and buffers are baked into captured graphs
  return poll_device(ctx);
}

// Initial plasma filled on the device (the moving window's injection profile
// over every patch column); capacity sized like the first load.
template <typename R>
pic_status do_fill(pic_ctx *ctx) {
  const Geom &g = ctx->g;
  const pic_config &c = ctx->cfg;
  const int total = g.P * g.Q * c.inj_ppc[0] * c.inj_ppc[1];
  const double cf = c.capacity_factor > 0 ? c.capacity_factor : 2.0;
  const int cmin = c.capacity_min > 0 ? c.capacity_min : 256;
  int cap = std::max(cmin, (int)std::ceil(cf * total));
  cap = (cap + 31) / 32 * 32;
  pic_status rs = alloc_particles<R>(ctx, cap);
  if (rs) return rs;
  const int q = (int)(ctx->step & 1);
  CK(launch_fill_plasma<R>(g, ctx->col0, ctx->nshift, soa<R>(ctx->seg[q]), ctx->cnt[q], ctx->cap,
                           c.inj_n0, c.inj_x0, c.inj_ramp, c.inj_ppc[0], c.inj_ppc[1],
                           ctx->rho_bg, &ctx->st->err, ctx->stream));
  ctx->launches += 1;
  if (c.sort_every > 0) {
    pic_status ss = sort_particles<R>(ctx);
    if (ss) return ss;
    ctx->since_sort = 0;
  }
  ctx->prev_valid = false;
  ctx->plan_ready = false;
  ctx->calm_ok = false;
  free_graphs(ctx);
  return poll_device(ctx);
}

template <typename R>
pic_status do_get_particles(pic_ctx *ctx, double *out, size_t cap, size_t *n, int where) {
  const Geom &g = ctx->g;
  if (!ctx->cap) {
    *n = 0;
    return PIC_OK;
  }
  const int q = (int)(ctx->step & 1);
  std::vector<int> c(g.nslots), b((size_t)g.nslots * 8);
  CK(cudaMemcpyAsync(c.data(), ctx->cnt[q], sizeof(int) * g.nslots, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaMemcpyAsync(b.data(), ctx->bcnt[1 - q], sizeof(int) * g.nslots * 8, cudaMemcpyDeviceToHost,
                     ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  std::vector<long long> off((size_t)g.nslots * 9 + 1, 0);
  long long tot = 0;
  for (int pp = 0; pp < g.nslots; ++pp) {
    const int slot = (pp / g.npx) * g.npx + (pp % g.npx + ctx->col0) % g.npx;
    off[pp] = tot;
    tot += std::min(c[slot], ctx->cap);
  }
  for (int pp = 0; pp < g.nslots; ++pp) {
    const int slot = (pp / g.npx) * g.npx + (pp % g.npx + ctx->col0) % g.npx;
    for (int d = 0; d < 8; ++d) {
      int ddx, ddy;
      dir_delta(d, ddx, ddy);
      off[g.nslots + (size_t)pp * 8 + d] = tot;
      if (neighbour_slot(g, ctx->col0, slot, ddx, ddy) >= 0)
        tot += std::min(b[(size_t)slot * 8 + d], ctx->bk.cap[d]);
    }
  }
  *n = (size_t)tot;
  if (!out) return PIC_OK;
  if ((size_t)tot > cap) return fail(ctx, PIC_EINVAL, "output capacity too small");
  CK(cudaMemcpyAsync(ctx->offsets, off.data(), sizeof(long long) * off.size(), cudaMemcpyHostToDevice,
                     ctx->stream));
  double *dst = out;
  bool copy_out = false;
  if (where == PIC_HOST) {
    dst = (double *)pinned_view(out);  // written in place when page-locked
    if (!dst) {
      const pic_status s = ensure_staging(ctx, 6 * std::max<size_t>(cap, 1));
      if (s) return s;
      dst = ctx->staging;
      copy_out = true;
    }
  }
  CK(launch_get_particles<R>(g, ctx->col0, view<R>(ctx, q, 1 - q), ctx->offsets, dst, cap,
                             ctx->stream));
  ctx->launches += 1;
  if (copy_out)
    CK(cudaMemcpyAsync(out, dst, sizeof(double) * 6 * cap, cudaMemcpyDeviceToHost, ctx->stream));
  return poll_device(ctx);
}

// Device address of a host buffer the GPU can reach directly (page-locked
// memory of this process: on GB300 the kernels read and write it over the
// coherent CPU-GPU link, with no staging copy), or null for pageable memory.
const void *pinned_view(const void *host) {
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, host) != cudaSuccess) {
    cudaGetLastError();  // pageable memory on older drivers reports an error
    return nullptr;
  }
  return at.type == cudaMemoryTypeHost ? at.devicePointer : nullptr;
}

pic_status ensure_staging(pic_ctx *ctx, size_t n) {
  if (ctx->staging_n >= n) return PIC_OK;
  if (ctx->staging) cfree(ctx, ctx->staging);
  ctx->staging = nullptr;
  CK(cmalloc(ctx, &ctx->staging, sizeof(double) * n));
  ctx->staging_n = n;
  return PIC_OK;
}

void out_shape(const Geom &g, int &nxo, int &nyo) {
  nxo = g.fbc_x == FBC_PERIODIC ? g.nx : g.nx + 2;
  nyo = g.fbc_y == FBC_PERIODIC ? g.ny : g.ny + 2;
}

int comp_of(int which) {
  switch (which) {
    case PIC_EX: return C_EX;
    case PIC_EY: return C_EY;
    case PIC_EZ: return C_EZ;
    case PIC_BX: return C_BX;
    case PIC_BY: return C_BY;
    case PIC_BZ: return C_BZ;
    case PIC_BMX: return C_BMX;
    case PIC_BMY: return C_BMY;
    case PIC_BMZ: return C_BMZ;
    default: return -1;
  }
}

template <typename R>
pic_status deposit_current_rho(pic_ctx *ctx, double *rho, bool previous) {
  const Geom &g = ctx->g;
  CK(cudaMemsetAsync(rho, 0, sizeof(double) * g.cs, ctx->stream));
  if (!ctx->cap) return PIC_OK;
  const int q = (int)(ctx->step & 1);
  const int segset = previous ? 1 - q : q;
  const int bktset = previous ? q : 1 - q;
  PartView<R> v = view<R>(ctx, segset, bktset);
  if (previous) {  // the arrays may have been cleared for the coming step
    v.cnt = ctx->cnt_prev;
    v.bcnt = ctx->bcnt_prev;
  }
  CK(launch_deposit_rho<R>(g, ctx->col0, v, rho, 1.0, ctx->stream));
  ctx->launches += 1;
  return PIC_OK;
}

template <typename R>
pic_status do_get_field(pic_ctx *ctx, int which, double *dst, int where) {
  const Geom &g = ctx->g;
  int nxo, nyo;
  out_shape(g, nxo, nyo);
  const size_t n = (size_t)nxo * nyo;
  double *d = dst;
  bool copy_out = false;
  if (where == PIC_HOST) {
    d = (double *)pinned_view(dst);
    if (!d) {
      pic_status s = ensure_staging(ctx, n);
      if (s) return s;
      d = ctx->staging;
      copy_out = true;
    }
  }
  if (which == PIC_RHO || which == PIC_RHO_BG) {
    const double *src = ctx->rho_bg;
    if (which == PIC_RHO) {
      pic_status s = deposit_current_rho<R>(ctx, ctx->rho_a, false);
      if (s) return s;
      src = ctx->rho_a;
    }
    CK(launch_get_field_f64(g, src, d, ctx->stream));
  } else {
    int c = comp_of(which);
    int filtered = -1;
    if (which >= PIC_JX && which <= PIC_JZ) {
      const int jset = (int)((ctx->step + 1) & 1);  // set of the last step
      c = C_JA + 3 * jset + (which - PIC_JX);
      if (ctx->cfg.filter_passes > 0) {
        // the field update used the filtered current, which the step does
        // not keep: filter the deposited set again into the other set (zero
        // between steps), read it, and clear it again
        filtered = 1 - jset;
        CK(launch_filter<R>(field_args<R>(ctx, jset), jset, filtered, ctx->stream));
        c = C_JA + 3 * filtered + (which - PIC_JX);
        ctx->launches += 1;
      }
    }
    if (c < 0) return fail(ctx, PIC_EINVAL, "bad field id");
    CK(launch_get_field<R>(g, (const R *)ctx->F + c * g.cs, d, ctx->stream));
    if (filtered >= 0)
      CK(cudaMemsetAsync((R *)ctx->F + (C_JA + 3 * filtered) * g.cs, 0, 3 * g.cs * sizeof(R),
                         ctx->stream));
  }
  ctx->launches += 1;
  if (copy_out) {
    CK(cudaMemcpyAsync(dst, d, sizeof(double) * n, cudaMemcpyDeviceToHost, ctx->stream));
  }
  return poll_device(ctx);
}

template <typename R>
pic_status do_set_field(pic_ctx *ctx, int which, const double *src, int where) {
  const Geom &g = ctx->g;
  int nxo, nyo;
  out_shape(g, nxo, nyo);
  const size_t n = (size_t)nxo * nyo;
  const double *s = src;
  if (where == PIC_HOST) {
    pic_status r = ensure_staging(ctx, n);
    if (r) return r;
    CK(cudaMemcpyAsync(ctx->staging, src, sizeof(double) * n, cudaMemcpyHostToDevice, ctx->stream));
    s = ctx->staging;
  }
  if (which == PIC_RHO_BG) {
    CK(launch_set_field_f64(g, ctx->rho_bg, s, ctx->stream));
  } else {
    const int c = comp_of(which);
    if (c < 0) return fail(ctx, PIC_EINVAL, "field id not settable");
    CK(launch_set_field<R>(g, (R *)ctx->F + c * g.cs, s, ctx->stream));
  }
  ctx->launches += 1;
  ctx->prev_valid = false;
  return poll_device(ctx);
}

template <typename R>
pic_status do_diag(pic_ctx *ctx, pic_diag_t *out) {
  const Geom &g = ctx->g;
  memset(out, 0, sizeof *out);
  const int nb = ctx->npartials;
  std::vector<double> h(3 * nb);
  const double dV = g.dx * g.dy;
  CK(launch_field_diag<R>(g, (const R *)ctx->F, ctx->partials, nb, ctx->stream));
  CK(cudaMemcpyAsync(h.data(), ctx->partials, sizeof(double) * 2 * nb, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  double ue = 0, ub = 0;
  for (int b = 0; b < nb; ++b) {
    ue += h[2 * b];
    ub += h[2 * b + 1];
  }
  out->U_E = 0.5 * ue * dV;
  out->U_B = 0.5 * ub * dV;
  double ek = 0, ws = 0, cnt = 0;
  if (ctx->cap) {
    const int q = (int)(ctx->step & 1);
    CK(launch_particle_diag<R>(g, ctx->col0, view<R>(ctx, q, 1 - q), ctx->partials, nb, ctx->stream));
    CK(cudaMemcpyAsync(h.data(), ctx->partials, sizeof(double) * 3 * nb, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    for (int b = 0; b < nb; ++b) {
      ek += h[3 * b];
      ws += h[3 * b + 1];
      cnt += h[3 * b + 2];
    }
  }
  out->U_K = ek * g.m * dV;
  out->charge = g.q * ws * dV;
  out->np = (long long)llround(cnt);
  pic_status s = deposit_current_rho<R>(ctx, ctx->rho_a, false);
  if (s) return s;
  const bool cont = ctx->prev_valid && ctx->cap;
  if (cont) {
    s = deposit_current_rho<R>(ctx, ctx->rho_b, true);
    if (s) return s;
  }
  const int jset = (int)((ctx->step + 1) & 1);
  CK(launch_gauss_diag<R>(g, (const R *)ctx->F, jset, ctx->rho_a, cont ? ctx->rho_b : nullptr,
                          ctx->rho_bg, ctx->partials, nb, ctx->stream));
  CK(cudaMemcpyAsync(h.data(), ctx->partials, sizeof(double) * 2 * nb, cudaMemcpyDeviceToHost, ctx->stream));
  DevState hs;
  CK(cudaMemcpyAsync(&hs, ctx->st, sizeof hs, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  double gm = 0, cm = 0;
  for (int b = 0; b < nb; ++b) {
    gm = std::max(gm, h[2 * b]);
    cm = std::max(cm, h[2 * b + 1]);
  }
  out->gauss = gm;
  out->continuity = cont ? cm : NAN;
  out->step = ctx->step;
  out->t = ctx->t;
  out->shifts = ctx->nshift / window_columns(ctx->cfg);
  out->max_patch_count = hs.maxcnt[(ctx->step + 1) & 1];
  out->capacity = ctx->cap;
  out->grows = ctx->grows;
  out->calm_particle_steps = (long long)hs.calm_particles;
  out->sorts = ctx->sorts;
  out->ms_particles = ctx->ms_particles;
  out->ms_fields = ctx->ms_fields;
  out->ms_window = ctx->ms_window;
  out->ms_sort = ctx->ms_sort;
  ctx->launches += 5 + (cont ? 1 : 0);
  out->launches = ctx->launches;
  out->particle_step_launches = ctx->ps_launches;
  return poll_device(ctx);
}

// ---- snapshot layout: header, fields, rho_bg, segments, counts, buckets,
// bucket counts, device state
struct SnapHeader {
  char magic[8];
  int nx, ny, P, Q, fp32, cap, nshift, col0;
  long long step;
  double t;
  int prev_valid, sticky_pad;
  double wmax;
};

// ================================================================ batches
//
// A batch advances several independent contexts with one launch per kernel
// per step: one plan over the flattened patch slots of every run, one
// persistent particle step over the work items of every run (each item
// names its run; the run's arguments come from a device array and its
// tensor map from the launch's TmapSet parameter), then one launch per
// field kernel whose blocks map to (run, block) through BatchGrid.  Every
// run flips its step parity each step, so the device argument arrays are
// built for two phases and the step of phase k uses set k.

}  // namespace

struct pic_batch {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int use_graph = 1;
  int task_chunk = 0;
  std::vector<pic_ctx *> runs;
  bool fp32 = false;
  // state of the last build: membership, per-run capacity / storage / parity
  bool dirty = true;
  std::vector<int> cap_built;
  std::vector<void *> seg_built;
  std::vector<double> wmax_built;  // the runs' weight bounds the scales were set for
  std::vector<int> parity0;  // run parity at phase 0
  int phase = 0;
  // device arrays: step / field arguments per phase, plan
  void *sargs[2] = {nullptr, nullptr};
  void *fargs[2] = {nullptr, nullptr};
  Plan plan{};
  int *item_run = nullptr;
  int plan_items_alloc = 0, plan_slots_alloc = 0;
  BatchGrid slots{};
  BatchGrid fgrid[4]{};
  bool det = false;   // runs in deterministic mode (all or none)
  BatchGrid ggrid{};  // deterministic mode: blocks of the current gather per run
  TmapSet<kBatchMax> *tm = nullptr;  // host copy: the launch parameter
  int P = 0, Q = 0;                  // common patch shape, 0 when mixed
  bool tma = true;
  size_t smem = 0;
  int grid = 0;
  cudaGraphExec_t gexec[2] = {nullptr, nullptr};
  cudaEvent_t ev = nullptr;
  long long steps = 0, launches = 0, builds = 0;
  std::string err;
};

namespace {

pic_status bfail(pic_batch *b, pic_status s, const std::string &m) {
  b->err = m;
  return s;
}

#define BCK(call)                                                                       \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess)                                                              \
      return bfail(b, PIC_ECUDA, std::string(#call ": ") + cudaGetErrorString(e_));     \
  } while (0)

void batch_free_graphs(pic_batch *b) {
  for (int p = 0; p < 2; ++p)
    if (b->gexec[p]) {
      cudaGraphExecDestroy(b->gexec[p]);
      b->gexec[p] = nullptr;
    }
}

// True when a run changed since the last build (capacity regrown, storage
// reallocated, or stepped alone so that its parity no longer follows the
// batch's phase).
bool batch_stale(const pic_batch *b) {
  if (b->dirty) return true;
  for (size_t r = 0; r < b->runs.size(); ++r) {
    const pic_ctx *c = b->runs[r];
    if (c->cap != b->cap_built[r] || c->seg[0][0] != b->seg_built[r] ||
        c->wmax != b->wmax_built[r])
      return true;
    if ((int)(c->step & 1) != (b->parity0[r] ^ b->phase)) return true;
  }
  return false;
}

template <typename R>
pic_status batch_enqueue(pic_batch *b, int k) {
  BatchRef<R> br;
  br.args = (const StepArgs<R> *)b->sargs[k];
  br.item_run = b->item_run;
  br.slots = b->slots;
  br.plan = b->plan;
  BCK(launch_particle_step_batch<R>(br, b->tm, b->P, b->Q, b->tma, 256, b->grid, b->smem,
                                    b->stream));
  if (b->det) BCK(launch_gather_current_batch<R>(br, b->ggrid, b->stream));
  BCK(launch_fields_batch<R>((const FieldArgs<R> *)b->fargs[k], b->fgrid, b->stream));
  return PIC_OK;
}

int batch_kernels_per_step(const pic_batch *b) {
  int n = 4 + (b->det ? 1 : 0);  // plan, particle step, (gather), E, B
  if (b->fgrid[0].off[b->fgrid[0].n] > 0) ++n;
  if (b->fgrid[3].off[b->fgrid[3].n] > 0) ++n;
  return n;
}

template <typename R>
pic_status batch_build(pic_batch *b) {
  const int n = (int)b->runs.size();
  BCK(cudaStreamSynchronize(b->stream));  // argument arrays may be in use
  batch_free_graphs(b);
  b->cap_built.assign(n, 0);
  b->seg_built.assign(n, nullptr);
  b->wmax_built.assign(n, 0.0);
  b->parity0.assign(n, 0);
  b->phase = 0;
  b->P = b->runs[0]->g.P;
  b->Q = b->runs[0]->g.Q;
  b->tma = true;
  b->smem = 0;
  std::vector<StepArgs<R>> sa[2];
  std::vector<FieldArgs<R>> fa[2];
  BatchGrid slots{};
  BatchGrid fg[4]{};
  slots.n = n;
  for (int k = 0; k < 4; ++k) fg[k].n = n;
  long long max_items = 0;
  b->det = n > 0 && b->runs[0]->cfg.deterministic != 0;
  int chunk = std::max(1, b->task_chunk > 0 ? b->task_chunk : default_chunk<R>());
  if (b->det) {  // one work item per patch
    chunk = 1;
    for (int r = 0; r < n; ++r)
      chunk = std::max(chunk, b->runs[r]->cap + b->runs[r]->bk.stride + 9);
  }
  b->ggrid = BatchGrid{};
  b->ggrid.n = n;
  for (int r = 0; r < n; ++r) {
    const Geom &g = b->runs[r]->g;
    const int ni = g.fbc_x == FBC_PERIODIC ? g.nx : g.nx + 2 * GX;
    const int nj = g.fbc_y == FBC_PERIODIC ? g.ny : g.ny + 2 * GY;
    b->ggrid.off[r + 1] = b->ggrid.off[r] + (b->det ? (ni * nj + 255) / 256 : 0);
  }
  for (int r = 0; r < n; ++r) {
    pic_ctx *c = b->runs[r];
    const Geom &g = c->g;
    if (g.P != b->P || g.Q != b->Q) b->P = b->Q = 0;
    if (!c->cfg.tma) b->tma = false;
    b->smem = std::max(b->smem, particle_step_smem(g.P, g.Q, sizeof(R)));
    const int p0 = (int)(c->step & 1);
    b->parity0[r] = p0;
    b->cap_built[r] = c->cap;
    b->seg_built[r] = c->seg[0][0];
    b->wmax_built[r] = c->wmax;
    for (int k = 0; k < 2; ++k) {
      sa[k].push_back(step_args<R>(c, p0 ^ k));
      set_current_scale(sa[k].back(), g, c->wmax, chunk);  // the batch plan's items
      fa[k].push_back(field_args<R>(c, p0 ^ k));
    }
    slots.off[r + 1] = slots.off[r] + g.nslots;
    int gx[4], gy[4];
    field_batch_blocks(g, c->cfg.filter_passes, gx, gy);
    for (int k = 0; k < 4; ++k) {
      fg[k].gx[r] = std::max(gx[k], 1);
      fg[k].off[r + 1] = fg[k].off[r] + gx[k] * gy[k];
    }
    const long long units_max = (long long)c->cap + c->bk.stride + 9;
    max_items += (long long)g.nslots * ((units_max + chunk - 1) / chunk);
  }
  if (b->tma) {
    for (int r = 0; r < n; ++r) {
      pic_ctx *c = b->runs[r];
      if (!c->tmap_ok) {
        pic_status s = build_tmap<R>(c);
        if (s) return bfail(b, s, c->err);
      }
      b->tm->m[r] = c->tmap;
    }
  }
  if (max_items > (1ll << 30)) return bfail(b, PIC_EINVAL, "batch too large");
  // plan storage: grows, never shrinks
  if (max_items > b->plan_items_alloc || slots.off[n] > b->plan_slots_alloc) {
    cudaFree(b->plan.item_slot);
    cudaFree(b->plan.item_first);
    cudaFree(b->plan.units);
    cudaFree(b->item_run);
    b->plan_items_alloc = (int)std::max<long long>(max_items, b->plan_items_alloc);
    b->plan_slots_alloc = std::max(slots.off[n], b->plan_slots_alloc);
    BCK(cudaMalloc(&b->plan.item_slot, sizeof(int) * b->plan_items_alloc));
    BCK(cudaMalloc(&b->plan.item_first, sizeof(int) * b->plan_items_alloc));
    BCK(cudaMalloc(&b->item_run, sizeof(int) * b->plan_items_alloc));
    BCK(cudaMalloc(&b->plan.units, sizeof(int) * b->plan_slots_alloc));
  }
  b->plan.unit = 1;
  b->plan.chunk = chunk;
  b->plan.max_items = (int)max_items;
  b->slots = slots;
  for (int k = 0; k < 4; ++k) b->fgrid[k] = fg[k];
  for (int k = 0; k < 2; ++k) {
    BCK(cudaMemcpy(b->sargs[k], sa[k].data(), sizeof(StepArgs<R>) * n, cudaMemcpyHostToDevice));
    BCK(cudaMemcpy(b->fargs[k], fa[k].data(), sizeof(FieldArgs<R>) * n, cudaMemcpyHostToDevice));
  }
  BCK(prepare_particle_step_batch<R>(b->P, b->Q, b->smem));
  b->grid = particle_step_batch_grid<R>(b->P, b->Q, b->tma, 256, b->smem);
  if (b->grid <= 0) return bfail(b, PIC_ECUDA, "particle step occupancy query failed");
  if (b->use_graph) {
    for (int k = 0; k < 2; ++k) {
      cudaGraph_t gr;
      BCK(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
      pic_status s = batch_enqueue<R>(b, k);
      cudaError_t e = cudaStreamEndCapture(b->stream, &gr);
      if (s != PIC_OK) return s;
      BCK(e);
      e = cudaGraphInstantiate(&b->gexec[k], gr, 0);
      cudaGraphDestroy(gr);
      BCK(e);
    }
  }
  b->dirty = false;
  b->builds += 1;
  return PIC_OK;
}

// Make `waiter` wait for the work queued so far on `on`.
pic_status order_after(pic_batch *b, cudaStream_t waiter, cudaStream_t on) {
  if (waiter == on) return PIC_OK;
  BCK(cudaEventRecord(b->ev, on));
  BCK(cudaStreamWaitEvent(waiter, b->ev, 0));
  return PIC_OK;
}

template <typename R>
pic_status batch_step(pic_batch *b, int nsteps) {
  if (batch_stale(b)) {
    pic_status s = batch_build<R>(b);
    if (s) return s;
  }
  for (pic_ctx *c : b->runs) {
    pic_status s = order_after(b, b->stream, c->stream);
    if (s) return s;
  }
  pic_status rs = PIC_OK;
  for (int it = 0; it < nsteps && rs == PIC_OK; ++it) {
    const int k = b->phase;
    for (pic_ctx *c : b->runs) {
      const pic_status cs = ensure_calm(c, b->stream);
      if (cs) return bfail(b, cs, c->err);
    }
    if (b->use_graph) BCK(cudaGraphLaunch(b->gexec[k], b->stream));
    else rs = batch_enqueue<R>(b, k);
    b->launches += batch_kernels_per_step(b);
    b->steps += 1;
    b->phase ^= 1;
    for (pic_ctx *c : b->runs) {
      c->step += 1;
      c->t += c->g.dt;
      c->prev_valid = true;
      c->plan_ready = false;
      c->ps_launches += 1;
      if (rs == PIC_OK && window_due(c)) {
        // the shift runs on the batch's stream, between batched steps
        cudaStream_t own = c->stream;
        c->stream = b->stream;
        for (int k = 0; k < window_columns(c->cfg) && rs == PIC_OK; ++k) rs = window_shift<R>(c);
        c->stream = own;
        if (rs) rs = bfail(b, rs, c->err);
        b->launches += 7;
      }
    }
  }
  BCK(cudaStreamSynchronize(b->stream));
  // per-run device faults: sticky on the run, which leaves the batch
  pic_status first = rs;
  std::vector<pic_ctx *> keep;
  for (pic_ctx *c : b->runs) {
    pic_status s = order_after(b, c->stream, b->stream);
    if (s) return s;
    s = poll_device(c);
    if (s == PIC_OK) {
      keep.push_back(c);
    } else if (first == PIC_OK) {
      first = bfail(b, s, c->err);
    }
  }
  if (keep.size() != b->runs.size()) {
    b->runs = keep;
    b->dirty = true;
  }
  return first;
}

}  // namespace

// =================================================================== C ABI

extern "C" {

const char *pic_version(void) { return kVersion; }

size_t pic_footprint(const pic_config *cfg, size_t np_max) {
  std::string why;
  if (!valid_config(cfg, why)) return 0;
  if (cfg->dims == 3) return footprint3(cfg, np_max);
  Geom g = make_geom(cfg);
  const size_t rs = cfg->prec == PIC_FP32 ? 4 : 8;
  double cf = cfg->capacity_factor > 0 ? cfg->capacity_factor : 2.0;
  int cmin = cfg->capacity_min > 0 ? cfg->capacity_min : 256;
  // the fullest patch is not known before loading: assume a uniform load
  size_t per = (np_max + g.nslots - 1) / g.nslots;
  if (cfg->moving_window)
    per = std::max(per, (size_t)g.P * g.Q * cfg->inj_ppc[0] * cfg->inj_ppc[1]);
  int cap = std::max(cmin, (int)std::ceil(cf * (double)per));
  cap = (cap + 31) / 32 * 32;
  return field_bytes(g, rs) + 3 * sizeof(double) * g.cs + particle_bytes(g, cap, rs) +
         sizeof(long long) * (g.nslots * 9 + 1) + sizeof(double) * 3 * 1024 + sizeof(DevState);
}

pic_status pic_create(const pic_config *cfg, pic_ctx **out) {
  if (!out) return PIC_EINVAL;
  *out = nullptr;
  std::string why;
  if (!valid_config(cfg, why)) {
    // no context exists yet: report through a throw-away context-free path
    return PIC_EINVAL;
  }
  pic_ctx *ctx = new (std::nothrow) pic_ctx();
  if (!ctx) return PIC_ENOMEM;
  ctx->cfg = *cfg;
  if (ctx->cfg.tma < 0) ctx->cfg.tma = 1;
  ctx->g = make_geom(cfg);
  ctx->fp32 = cfg->prec == PIC_FP32;
  {
    // weights the injection (window, pic_load_plasma) can create
    const int ppc = cfg->inj_ppc[0] * cfg->inj_ppc[1];
    if (ppc > 0 && std::isfinite(cfg->inj_n0)) ctx->wmax = std::fabs(cfg->inj_n0) / ppc;
  }
  ctx->rs = ctx->fp32 ? 4 : 8;
  const Geom &g = ctx->g;
  auto bail = [&](pic_status s) {
    pic_destroy(ctx);
    return s;
  };
  if (cudaSetDevice(cfg->device) != cudaSuccess) return bail(PIC_ECUDA);
  // the allocation-free entry point made ready on this device, so that its
  // calls never load code or allocate
  if (noalloc_setup(cfg->device) != PIC_OK) return bail(PIC_ECUDA);
  if (cfg->stream) {
    ctx->stream = (cudaStream_t)cfg->stream;
  } else {
    if (cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking) != cudaSuccess) return bail(PIC_ECUDA);
    ctx->own_stream = true;
  }
  if (cfg->dims == 3) {
    const pic_status s = c3_create(cfg, ctx->stream, &ctx->c3, ctx->err);
    if (s) return bail(s);
    *out = ctx;
    return PIC_OK;
  }
  if (cudaStreamCreateWithFlags(&ctx->aux, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&ctx->ev_join, cudaEventDisableTiming) != cudaSuccess)
    return bail(PIC_ECUDA);
  if (cmalloc(ctx, &ctx->F, field_bytes(g, ctx->rs)) != cudaSuccess) return bail(PIC_ENOMEM);
  if (cmalloc(ctx, &ctx->rho_bg, sizeof(double) * g.cs) != cudaSuccess) return bail(PIC_ENOMEM);
  if (cmalloc(ctx, &ctx->rho_a, sizeof(double) * g.cs) != cudaSuccess) return bail(PIC_ENOMEM);
  if (cmalloc(ctx, &ctx->rho_b, sizeof(double) * g.cs) != cudaSuccess) return bail(PIC_ENOMEM);
  if (cmalloc(ctx, &ctx->st, sizeof(DevState)) != cudaSuccess) return bail(PIC_ENOMEM);
  ctx->npartials = 1024;
  if (cmalloc(ctx, &ctx->partials, sizeof(double) * 3 * ctx->npartials) != cudaSuccess) return bail(PIC_ENOMEM);
  if (cfg->laser_on) {
    std::vector<double> prof(g.ny + 1);
    for (int j = 0; j <= g.ny; ++j) {
      const double r = ((j + 0.5) * g.dy - cfg->laser_y_center) / cfg->laser_waist;
      prof[j] = cfg->laser_a0 * std::exp(-r * r);
    }
    if (cmalloc(ctx, &ctx->laser_g, sizeof(double) * prof.size()) != cudaSuccess) return bail(PIC_ENOMEM);
    if (cudaMemcpy(ctx->laser_g, prof.data(), sizeof(double) * prof.size(), cudaMemcpyHostToDevice) !=
        cudaSuccess)
      return bail(PIC_ECUDA);
  }
  if (cudaMemsetAsync(ctx->F, 0, field_bytes(g, ctx->rs), ctx->stream) != cudaSuccess ||
      cudaMemsetAsync(ctx->rho_bg, 0, sizeof(double) * g.cs, ctx->stream) != cudaSuccess ||
      cudaMemsetAsync(ctx->st, 0, sizeof(DevState), ctx->stream) != cudaSuccess ||
      cudaStreamSynchronize(ctx->stream) != cudaSuccess)
    return bail(PIC_ECUDA);
  *out = ctx;
  return PIC_OK;
}

void pic_destroy(pic_ctx *ctx) {
  if (!ctx) return;
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  c3_destroy(ctx->c3);
  ctx->c3 = nullptr;
  if (ctx->aux) {
    cudaStreamSynchronize(ctx->aux);
    cudaStreamDestroy(ctx->aux);
  }
  if (ctx->ev_fork) cudaEventDestroy(ctx->ev_fork);
  if (ctx->ev_join) cudaEventDestroy(ctx->ev_join);
  free_graphs(ctx);
  cfree(ctx, ctx->F);
  cfree(ctx, ctx->rho_bg);
  cfree(ctx, ctx->rho_a);
  cfree(ctx, ctx->rho_b);
  cfree(ctx, ctx->laser_g);
  cfree(ctx, ctx->st);
  cfree(ctx, ctx->partials);
  cfree(ctx, ctx->staging);
  free_particles(ctx);
  free_backup(ctx);
  if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
  delete ctx;
}

const char *pic_last_error(const pic_ctx *ctx) {
  if (!ctx) return "no context";
  return ctx->c3 ? c3_error(ctx->c3) : ctx->err.c_str();
}

pic_status pic_load_particles(pic_ctx *ctx, const double *x, const double *y, const double *ux,
                              const double *uy, const double *uz, const double *w, size_t n,
                              int where) {
  NvtxRange range("pic_load_particles");
  pic_status s = check_usable(ctx);
  if (s) return s;
  if (n && (!x || !y || !ux || !uy || !uz || !w)) return fail(ctx, PIC_EINVAL, "null particle array");
  if (where != PIC_HOST && where != PIC_DEVICE) return fail(ctx, PIC_EINVAL, "bad location");
  if (ctx->c3) return fail(ctx, PIC_EINVAL, "3D contexts load particles with pic_load_particles3");
  CK(cudaSetDevice(ctx->cfg.device));
  return ctx->fp32 ? do_load<float>(ctx, x, y, ux, uy, uz, w, n, where)
                   : do_load<double>(ctx, x, y, ux, uy, uz, w, n, where);
}

pic_status pic_load_particles3(pic_ctx *ctx, const double *x, const double *y, const double *z,
                               const double *ux, const double *uy, const double *uz,
                               const double *w, size_t n, int where) {
  pic_status s = check_usable(ctx);
  if (s) return s;
  if (!ctx->c3) return fail(ctx, PIC_EINVAL, "pic_load_particles3 needs a 3D context");
  if (n && (!x || !y || !z || !ux || !uy || !uz || !w)) return fail(ctx, PIC_EINVAL, "null particle array");
  if (where != PIC_HOST && where != PIC_DEVICE) return fail(ctx, PIC_EINVAL, "bad location");
  CK(cudaSetDevice(ctx->cfg.device));
  return c3_load(ctx->c3, x, y, z, ux, uy, uz, w, n, where);
}

pic_status pic_load_plasma(pic_ctx *ctx) {
  pic_status s = check_usable(ctx);
  if (s) return s;
  if (ctx->c3) {
    CK(cudaSetDevice(ctx->cfg.device));
    return c3_fill_plasma(ctx->c3);
  }
  if (ctx->cap) return fail(ctx, PIC_ESTATE, "particles are already loaded");
  if (ctx->cfg.inj_ppc[0] < 1 || ctx->cfg.inj_ppc[1] < 1 || !(ctx->cfg.inj_n0 >= 0))
    return fail(ctx, PIC_EINVAL, "plasma needs inj_ppc >= 1 and inj_n0 >= 0");
  CK(cudaSetDevice(ctx->cfg.device));
  return ctx->fp32 ? do_fill<float>(ctx) : do_fill<double>(ctx);
}

pic_status pic_set_field(pic_ctx *ctx, int which, const double *src, int where) {
  pic_status s = check_usable(ctx);
  if (s) return s;
  if (!src || (where != PIC_HOST && where != PIC_DEVICE)) return fail(ctx, PIC_EINVAL, "bad source");
  CK(cudaSetDevice(ctx->cfg.device));
  if (ctx->c3) return c3_set_field(ctx->c3, which, src, where);
  return ctx->fp32 ? do_set_field<float>(ctx, which, src, where)
                   : do_set_field<double>(ctx, which, src, where);
}

pic_status pic_set_background(pic_ctx *ctx, int mode, double value) {
  pic_status s = check_usable(ctx);
  if (s) return s;
  CK(cudaSetDevice(ctx->cfg.device));
  if (ctx->c3) return c3_set_background(ctx->c3, mode, value);
  const Geom &g = ctx->g;
  if (mode == PIC_BG_NONE) {
    CK(cudaMemsetAsync(ctx->rho_bg, 0, sizeof(double) * g.cs, ctx->stream));
  } else if (mode == PIC_BG_UNIFORM) {
    std::vector<double> h((size_t)g.cs, value);
    CK(cudaMemcpyAsync(ctx->rho_bg, h.data(), sizeof(double) * g.cs, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
  } else if (mode == PIC_BG_NEUTRALISING) {
    CK(cudaMemsetAsync(ctx->rho_bg, 0, sizeof(double) * g.cs, ctx->stream));
    if (ctx->cap) {
      const int q = (int)(ctx->step & 1);
      if (ctx->fp32)
        CK(launch_deposit_rho<float>(g, ctx->col0, view<float>(ctx, q, 1 - q), ctx->rho_bg, -1.0, ctx->stream));
      else
        CK(launch_deposit_rho<double>(g, ctx->col0, view<double>(ctx, q, 1 - q), ctx->rho_bg, -1.0, ctx->stream));
      ctx->launches += 1;
    }
  } else {
    return fail(ctx, PIC_EINVAL, "bad background mode");
  }
  return poll_device(ctx);
}

pic_status pic_init_fields(pic_ctx *ctx, int mode) {
  NvtxRange range("pic_init_fields");
  pic_status s = check_usable(ctx);
  if (s) return s;
  if (mode != PIC_INIT_ZERO && mode != PIC_INIT_POISSON) return fail(ctx, PIC_EINVAL, "bad init mode");
  CK(cudaSetDevice(ctx->cfg.device));
  if (ctx->c3) return c3_init_fields(ctx->c3, mode);
  const Geom &g = ctx->g;
  CK(cudaStreamSynchronize(ctx->stream));
  CK(cudaMemsetAsync(ctx->F, 0, 9 * g.cs * ctx->rs, ctx->stream));  // E, Bm, B
  ctx->prev_valid = false;
  if (mode == PIC_INIT_ZERO) return poll_device(ctx);
  if (g.fbc_x != FBC_PERIODIC || g.fbc_y != FBC_PERIODIC)
    return fail(ctx, PIC_EINVAL, "the Poisson start needs periodic axes");
  const size_t n = (size_t)g.nx * g.ny;
  double *buf = nullptr;
  CK(cmalloc(ctx, &buf, sizeof(double) * 5 * n));
  double *rho = buf, *bg = buf + n, *ex = buf + 2 * n, *ey = buf + 3 * n, *ez = buf + 4 * n;
  s = ctx->fp32 ? deposit_current_rho<float>(ctx, ctx->rho_a, false)
                : deposit_current_rho<double>(ctx, ctx->rho_a, false);
  if (s) { cfree(ctx, buf); return s; }
  CK(launch_get_field_f64(g, ctx->rho_a, rho, ctx->stream));
  CK(launch_get_field_f64(g, ctx->rho_bg, bg, ctx->stream));
  CK(launch_axpy_f64(rho, bg, n, ctx->stream));
  CK(cudaMemsetAsync(ez, 0, sizeof(double) * n, ctx->stream));
  const int nn[3] = {g.nx, g.ny, 1};
  const double dd[3] = {g.dx, g.dy, 1.0};
  s = poisson_fields(ctx->cfg, 2, nn, dd, rho, ex, ey, nullptr, ctx->stream, ctx->err);
  if (!s) {
    const double *src[3] = {ex, ey, ez};
    for (int c = 0; c < 3 && !s; ++c)
      s = ctx->fp32 ? do_set_field<float>(ctx, PIC_EX + c, src[c], PIC_DEVICE)
                    : do_set_field<double>(ctx, PIC_EX + c, src[c], PIC_DEVICE);
  }
  cudaStreamSynchronize(ctx->stream);
  cfree(ctx, buf);
  ctx->launches += 6;
  if (s) return s;
  return poll_device(ctx);
}

pic_status pic_step(pic_ctx *ctx, int nsteps) {
  NvtxRange range("pic_step");
  pic_status s = check_usable(ctx);
  if (s) return s;
  if (nsteps < 0) return fail(ctx, PIC_EINVAL, "negative step count");
  if (nsteps == 0) return PIC_OK;
  CK(cudaSetDevice(ctx->cfg.device));
  if (ctx->c3) return c3_step(ctx->c3, nsteps);
  return ctx->fp32 ? do_step<float>(ctx, nsteps) : do_step<double>(ctx, nsteps);
}

pic_status pic_get_field(pic_ctx *ctx, int which, double *dst, int where) {
  pic_status s = check_usable(ctx);
  if (s) return s;
  if (!dst || which < 0 || which >= PIC_NFIELDS || (where != PIC_HOST && where != PIC_DEVICE))
    return fail(ctx, PIC_EINVAL, "bad destination or field id");
  CK(cudaSetDevice(ctx->cfg.device));
  if (ctx->c3) return c3_get_field(ctx->c3, which, dst, where);
  return ctx->fp32 ? do_get_field<float>(ctx, which, dst, where)
                   : do_get_field<double>(ctx, which, dst, where);
}

pic_status pic_get_particles(pic_ctx *ctx, double *out, size_t cap, size_t *n, int where) {
  pic_status s = check_usable(ctx);
  if (s) return s;
  if (!n || (where != PIC_HOST && where != PIC_DEVICE)) return fail(ctx, PIC_EINVAL, "bad arguments");
  CK(cudaSetDevice(ctx->cfg.device));
  if (ctx->c3) return c3_get_particles(ctx->c3, out, cap, n, where);
  return ctx->fp32 ? do_get_particles<float>(ctx, out, cap, n, where)
                   : do_get_particles<double>(ctx, out, cap, n, where);
}

pic_status pic_diag(pic_ctx *ctx, pic_diag_t *out) {
  pic_status s = check_usable(ctx);
  if (s) return s;
  if (!out) return fail(ctx, PIC_EINVAL, "null output");
  CK(cudaSetDevice(ctx->cfg.device));
  if (ctx->c3) return c3_diag(ctx->c3, out);
  return ctx->fp32 ? do_diag<float>(ctx, out) : do_diag<double>(ctx, out);
}

pic_status pic_sync(pic_ctx *ctx) {
  pic_status s = check_usable(ctx);
  if (s) return s;
  CK(cudaSetDevice(ctx->cfg.device));
  if (ctx->c3) return c3_sync(ctx->c3);
  return poll_device(ctx);
}

// Snapshot layout (2D): SnapHeader, the 15 field components, the
// background charge, the device scalars, then for each particle set st = 0, 1
// (segments seg[st] with buckets bkt[st]): its segment counts (nslots ints),
// its bucket counts (8 nslots ints) and its live particles packed into six
// arrays (pack.h), slot by slot, segment then buckets.  Capacity slack is
// not stored.  Set q = step % 2 holds the current particles in its segments
// and the previous state's arrivals in its buckets; set 1 - q the previous
// state's particles and the current in-flight buckets; each is saved with
// the counts that describe it (the previous state's were kept aside).

// Offsets of one set's packed arrays from its counts; returns the total.
long long pack_offsets(const Geom &g, int cap, const Buckets &bk, const int *cnt, const int *bcnt,
                       std::vector<long long> &off) {
  off.assign((size_t)g.nslots * 9 + 1, 0);
  long long o = 0;
  for (int s = 0; s < g.nslots; ++s) {
    off[9 * (size_t)s] = o;
    o += std::min(std::max(cnt[s], 0), cap);
    for (int d = 0; d < 8; ++d) {
      off[9 * (size_t)s + 1 + d] = o;
      o += std::min(std::max(bcnt[(size_t)s * 8 + d], 0), bk.cap[d]);
    }
  }
  off.back() = o;
  return o;
}

pic_status pic_snapshot(pic_ctx *ctx, void *host, size_t *bytes) {
  pic_status s = check_usable(ctx);
  if (s) return s;
  if (!bytes) return fail(ctx, PIC_EINVAL, "null size");
  CK(cudaSetDevice(ctx->cfg.device));
  if (ctx->c3) return c3_snapshot(ctx->c3, host, bytes);
  CK(cudaStreamSynchronize(ctx->stream));
  const Geom &g = ctx->g;
  const int q = (int)(ctx->step & 1);
  // the counts that describe each set
  std::vector<int> cnt[2], bcnt[2];
  std::vector<long long> off[2];
  long long total[2] = {0, 0};
  if (ctx->cap) {
    for (int st = 0; st < 2; ++st) {
      cnt[st].resize(g.nslots);
      bcnt[st].resize((size_t)g.nslots * 8);
      CK(cudaMemcpy(cnt[st].data(), st == q ? ctx->cnt[st] : ctx->cnt_prev,
                    sizeof(int) * g.nslots, cudaMemcpyDeviceToHost));
      CK(cudaMemcpy(bcnt[st].data(), st == q ? ctx->bcnt_prev : ctx->bcnt[st],
                    sizeof(int) * g.nslots * 8, cudaMemcpyDeviceToHost));
      total[st] = pack_offsets(g, ctx->cap, ctx->bk, cnt[st].data(), bcnt[st].data(), off[st]);
    }
  }
  size_t need = sizeof(SnapHeader) + field_bytes(g, ctx->rs) + sizeof(double) * g.cs +
                sizeof(DevState);
  if (ctx->cap)
    for (int st = 0; st < 2; ++st)
      need += sizeof(int) * (size_t)g.nslots * 9 + 6 * ctx->rs * (size_t)total[st];
  if (!host) {
    *bytes = need;
    return PIC_OK;
  }
  if (*bytes < need) return fail(ctx, PIC_EINVAL, "snapshot buffer too small");
  char *p = (char *)host;
  SnapHeader h{};
  memcpy(h.magic, "PICSNAP4", 8);
  h.nx = g.nx; h.ny = g.ny; h.P = g.P; h.Q = g.Q; h.fp32 = ctx->fp32;
  h.cap = ctx->cap; h.nshift = ctx->nshift; h.col0 = ctx->col0;
  h.step = ctx->step; h.t = ctx->t; h.prev_valid = ctx->prev_valid; h.wmax = ctx->wmax;
  memcpy(p, &h, sizeof h);
  p += sizeof h;
  auto d2h = [&](const void *src, size_t n) -> cudaError_t {
    cudaError_t e = cudaMemcpy(p, src, n, cudaMemcpyDeviceToHost);
    p += n;
    return e;
  };
  CK(d2h(ctx->F, field_bytes(g, ctx->rs)));
  CK(d2h(ctx->rho_bg, sizeof(double) * g.cs));
  CK(d2h(ctx->st, sizeof(DevState)));
  if (ctx->cap) {
    void *flat = nullptr;
    const long long most = std::max(total[0], total[1]);
    if (most > 0) CK(cmalloc(ctx, &flat, 6 * ctx->rs * (size_t)most));
    pic_status rs = PIC_OK;
    for (int st = 0; st < 2 && rs == PIC_OK; ++st) {
      memcpy(p, cnt[st].data(), sizeof(int) * g.nslots);
      p += sizeof(int) * g.nslots;
      memcpy(p, bcnt[st].data(), sizeof(int) * g.nslots * 8);
      p += sizeof(int) * g.nslots * 8;
      if (total[st] == 0) continue;
      cudaError_t e = cudaMemcpyAsync(ctx->offsets, off[st].data(), sizeof(long long) * off[st].size(),
                                      cudaMemcpyHostToDevice, ctx->stream);
      if (e == cudaSuccess)
        e = ctx->fp32 ? launch_pack<float>(g, soa<float>(ctx->seg[st]),
                                           st == q ? ctx->cnt[st] : ctx->cnt_prev, ctx->cap,
                                           soa<float>(ctx->bkt[st]),
                                           st == q ? ctx->bcnt_prev : ctx->bcnt[st], ctx->bk,
                                           ctx->offsets, (float *)flat, total[st], ctx->stream)
                      : launch_pack<double>(g, soa<double>(ctx->seg[st]),
                                            st == q ? ctx->cnt[st] : ctx->cnt_prev, ctx->cap,
                                            soa<double>(ctx->bkt[st]),
                                            st == q ? ctx->bcnt_prev : ctx->bcnt[st], ctx->bk,
                                            ctx->offsets, (double *)flat, total[st], ctx->stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
      if (e == cudaSuccess) e = d2h(flat, 6 * ctx->rs * (size_t)total[st]);
      if (e != cudaSuccess) rs = fail(ctx, PIC_ECUDA, std::string("snapshot: ") + cudaGetErrorString(e));
      ctx->launches += 1;
    }
    if (flat) {
      cudaStreamSynchronize(ctx->stream);
      cfree(ctx, flat);
    }
    if (rs) return rs;
  }
  *bytes = need;
  return PIC_OK;
}

pic_status pic_restore(pic_ctx *ctx, const void *host, size_t bytes) {
  if (!ctx || !host) return PIC_EINVAL;
  if (ctx->c3) {
    CK(cudaSetDevice(ctx->cfg.device));
    return c3_restore(ctx->c3, host, bytes);
  }
  SnapHeader h;
  if (bytes < sizeof h) return fail(ctx, PIC_EINVAL, "snapshot too small");
  memcpy(&h, host, sizeof h);
  const Geom &g = ctx->g;
  if (memcmp(h.magic, "PICSNAP4", 8) || h.nx != g.nx || h.ny != g.ny || h.P != g.P || h.Q != g.Q ||
      h.fp32 != (int)ctx->fp32)
    return fail(ctx, PIC_EINVAL, "snapshot does not match this configuration");
  if (h.cap < 0 || (h.cap % 32)) return fail(ctx, PIC_EINVAL, "snapshot capacity is invalid");
  if (h.cap != ctx->cap && ctx->cap)
    return fail(ctx, PIC_EINVAL, "snapshot capacity differs from this context's");
  // walk the layout on the host first: sizes and counts are checked before
  // anything of the context changes
  const size_t head = sizeof h + field_bytes(g, ctx->rs) + sizeof(double) * g.cs + sizeof(DevState);
  if (bytes < head) return fail(ctx, PIC_EINVAL, "snapshot truncated");
  const Buckets bk = bucket_layout(h.cap);
  const char *sets[2] = {nullptr, nullptr};
  std::vector<long long> off[2];
  long long total[2] = {0, 0};
  size_t pos = head;
  if (h.cap) {
    for (int st = 0; st < 2; ++st) {
      const size_t cb = sizeof(int) * (size_t)g.nslots * 9;
      if (bytes < pos + cb) return fail(ctx, PIC_EINVAL, "snapshot truncated");
      sets[st] = (const char *)host + pos;
      const int *c = reinterpret_cast<const int *>(sets[st]);
      for (size_t k = 0; k < (size_t)g.nslots * 9; ++k) {
        const int lim = k < (size_t)g.nslots ? h.cap : bk.cap[(k - g.nslots) % 8];
        if (c[k] < 0 || c[k] > lim) return fail(ctx, PIC_EINVAL, "snapshot counts are invalid");
      }
      total[st] = pack_offsets(g, h.cap, bk, c, c + g.nslots, off[st]);
      pos += cb + 6 * ctx->rs * (size_t)total[st];
      if (bytes < pos) return fail(ctx, PIC_EINVAL, "snapshot truncated");
    }
  }
  CK(cudaSetDevice(ctx->cfg.device));
  CK(cudaStreamSynchronize(ctx->stream));
  if (h.cap != ctx->cap) {  // a context without particle storage takes the snapshot's
    free_graphs(ctx);
    if (h.cap) {
      const pic_status s = ctx->fp32 ? alloc_particles<float>(ctx, h.cap) : alloc_particles<double>(ctx, h.cap);
      if (s) return s;
    }
  }
  ctx->cap = h.cap;
  if (h.wmax != ctx->wmax) free_graphs(ctx);  // the current scales are baked into the graphs
  ctx->wmax = h.wmax;
  ctx->bk = bk;
  const char *p = (const char *)host + sizeof h;
  auto h2d = [&](void *dst, size_t n) -> cudaError_t {
    cudaError_t e = cudaMemcpy(dst, p, n, cudaMemcpyHostToDevice);
    p += n;
    return e;
  };
  CK(h2d(ctx->F, field_bytes(g, ctx->rs)));
  CK(h2d(ctx->rho_bg, sizeof(double) * g.cs));
  DevState ds;
  memcpy(&ds, p, sizeof ds);
  p += sizeof ds;
  ds.err = 0;
  CK(cudaMemcpy(ctx->st, &ds, sizeof ds, cudaMemcpyHostToDevice));
  if (h.cap) {
    void *flat = nullptr;
    const long long most = std::max(total[0], total[1]);
    if (most > 0) CK(cmalloc(ctx, &flat, 6 * ctx->rs * (size_t)most));
    pic_status rs = PIC_OK;
    for (int st = 0; st < 2 && rs == PIC_OK; ++st) {
      const char *c = sets[st];
      cudaError_t e = cudaMemcpy(ctx->cnt[st], c, sizeof(int) * g.nslots, cudaMemcpyHostToDevice);
      if (e == cudaSuccess)
        e = cudaMemcpy(ctx->bcnt[st], c + sizeof(int) * g.nslots, sizeof(int) * g.nslots * 8,
                       cudaMemcpyHostToDevice);
      if (e == cudaSuccess && total[st] > 0) {
        e = cudaMemcpy(flat, c + sizeof(int) * (size_t)g.nslots * 9,
                       6 * ctx->rs * (size_t)total[st], cudaMemcpyHostToDevice);
        if (e == cudaSuccess)
          e = cudaMemcpy(ctx->offsets, off[st].data(), sizeof(long long) * off[st].size(),
                         cudaMemcpyHostToDevice);
        if (e == cudaSuccess)
          e = ctx->fp32 ? launch_unpack<float>(g, (const float *)flat, total[st], ctx->offsets,
                                               soa<float>(ctx->seg[st]), ctx->cnt[st], ctx->cap,
                                               soa<float>(ctx->bkt[st]), ctx->bcnt[st], ctx->bk,
                                               ctx->stream)
                        : launch_unpack<double>(g, (const double *)flat, total[st], ctx->offsets,
                                                soa<double>(ctx->seg[st]), ctx->cnt[st], ctx->cap,
                                                soa<double>(ctx->bkt[st]), ctx->bcnt[st], ctx->bk,
                                                ctx->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
        ctx->launches += 1;
      }
      if (e != cudaSuccess) rs = fail(ctx, PIC_ECUDA, std::string("restore: ") + cudaGetErrorString(e));
    }
    if (flat) {
      cudaStreamSynchronize(ctx->stream);
      cfree(ctx, flat);
    }
    if (rs) return rs;
    const int q = (int)(h.step & 1);
    CK(cudaMemcpy(ctx->cnt_prev, ctx->cnt[1 - q], sizeof(int) * g.nslots, cudaMemcpyDeviceToDevice));
    CK(cudaMemcpy(ctx->bcnt_prev, ctx->bcnt[q], sizeof(int) * g.nslots * 8, cudaMemcpyDeviceToDevice));
  }
  ctx->step = h.step;
  ctx->t = h.t;
  ctx->nshift = h.nshift;
  ctx->col0 = h.col0;
  ctx->prev_valid = h.prev_valid != 0;
  ctx->plan_ready = false;
  ctx->calm_ok = false;
  ctx->sticky = PIC_OK;
  ctx->err.clear();
  return PIC_OK;
}

// ---------------------------------------------------------------- batches

pic_status pic_batch_create(const pic_batch_config *cfg, pic_batch **out) {
  if (!out || !cfg) return PIC_EINVAL;
  *out = nullptr;
  if (cfg->task_chunk < 0 || cfg->task_chunk > 4096) return PIC_EINVAL;
  pic_batch *b = new (std::nothrow) pic_batch();
  if (!b) return PIC_ENOMEM;
  b->device = cfg->device;
  b->use_graph = cfg->use_graph;
  b->task_chunk = cfg->task_chunk;
  auto bail = [&](pic_status s) {
    pic_batch_destroy(b);
    return s;
  };
  if (cudaSetDevice(cfg->device) != cudaSuccess) return bail(PIC_ECUDA);
  if (cfg->stream) {
    b->stream = (cudaStream_t)cfg->stream;
  } else {
    if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess)
      return bail(PIC_ECUDA);
    b->own_stream = true;
  }
  if (cudaEventCreateWithFlags(&b->ev, cudaEventDisableTiming) != cudaSuccess) return bail(PIC_ECUDA);
  const size_t sa = std::max(sizeof(StepArgs<double>), sizeof(StepArgs<float>));
  const size_t fa = std::max(sizeof(FieldArgs<double>), sizeof(FieldArgs<float>));
  for (int k = 0; k < 2; ++k) {
    if (cudaMalloc(&b->sargs[k], sa * kBatchMax) != cudaSuccess) return bail(PIC_ENOMEM);
    if (cudaMalloc(&b->fargs[k], fa * kBatchMax) != cudaSuccess) return bail(PIC_ENOMEM);
  }
  if (cudaMalloc(&b->plan.n_items, sizeof(int) * 2) != cudaSuccess) return bail(PIC_ENOMEM);
  b->plan.next = b->plan.n_items + 1;
  b->tm = new (std::nothrow) TmapSet<kBatchMax>();
  if (!b->tm) return bail(PIC_ENOMEM);
  *out = b;
  return PIC_OK;
}

pic_status pic_batch_set(pic_batch *b, pic_ctx *const *runs, int n) {
  if (!b) return PIC_EINVAL;
  if (n < 0 || n > kBatchMax || (n && !runs)) return bfail(b, PIC_EINVAL, "bad run count");
  for (int r = 0; r < n; ++r) {
    const pic_ctx *c = runs[r];
    if (!c) return bfail(b, PIC_EINVAL, "null run");
    for (int q = 0; q < r; ++q)
      if (runs[q] == c) return bfail(b, PIC_EINVAL, "a run appears twice");
    if (c->sticky != PIC_OK) return bfail(b, PIC_ESTATE, "a run holds a device fault");
    if (c->c3) return bfail(b, PIC_EINVAL, "3D runs are not batched");
    if (!c->cap) return bfail(b, PIC_ESTATE, "a run has no particles loaded");
    if (c->cfg.device != b->device) return bfail(b, PIC_EINVAL, "a run lives on another device");
    if (c->fp32 != runs[0]->fp32) return bfail(b, PIC_EINVAL, "runs of one batch share a precision");
    if ((c->cfg.deterministic != 0) != (runs[0]->cfg.deterministic != 0))
      return bfail(b, PIC_EINVAL, "runs of one batch share the deterministic setting");
  }
  b->runs.assign(runs, runs + n);
  b->fp32 = n ? runs[0]->fp32 : false;
  b->dirty = true;
  return PIC_OK;
}

pic_status pic_batch_step(pic_batch *b, int nsteps) {
  NvtxRange range("pic_batch_step");
  if (!b) return PIC_EINVAL;
  if (nsteps < 0) return bfail(b, PIC_EINVAL, "negative step count");
  if (nsteps == 0 || b->runs.empty()) return PIC_OK;
  for (pic_ctx *c : b->runs)
    if (c->sticky != PIC_OK || !c->cap)
      return bfail(b, PIC_ESTATE, "a run holds a device fault or lost its particles");
  BCK(cudaSetDevice(b->device));
  return b->fp32 ? batch_step<float>(b, nsteps) : batch_step<double>(b, nsteps);
}

int pic_batch_size(const pic_batch *b) { return b ? (int)b->runs.size() : 0; }

pic_status pic_batch_get_diag(const pic_batch *b, pic_batch_diag_t *out) {
  if (!b || !out) return PIC_EINVAL;
  out->steps = b->steps;
  out->launches = b->launches;
  out->builds = b->builds;
  out->nruns = (int)b->runs.size();
  out->grid = b->grid;
  return PIC_OK;
}

const char *pic_batch_last_error(const pic_batch *b) { return b ? b->err.c_str() : "no batch"; }

void pic_batch_destroy(pic_batch *b) {
  if (!b) return;
  if (b->stream) cudaStreamSynchronize(b->stream);
  batch_free_graphs(b);
  for (int k = 0; k < 2; ++k) {
    cudaFree(b->sargs[k]);
    cudaFree(b->fargs[k]);
  }
  cudaFree(b->plan.n_items);
  cudaFree(b->plan.item_slot);
  cudaFree(b->plan.item_first);
  cudaFree(b->plan.units);
  cudaFree(b->item_run);
  if (b->ev) cudaEventDestroy(b->ev);
  if (b->own_stream) cudaStreamDestroy(b->stream);
  delete b->tm;
  delete b;
}

}  // extern "C"
