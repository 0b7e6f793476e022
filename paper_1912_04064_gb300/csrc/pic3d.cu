// 3D3V path: the same SDMD step as the 2D path (Section 2.2 steps (i) and
// (ii), Section 3.2 operators) on a Yee lattice with E and J on cell edges
// and B on cell faces.
//
// Per step (context stream, optionally one CUDA graph per step parity):
//   k3_plan          work items (patch slot, first particle), heaviest first
//   k3_particle_step persistent blocks over the items: gather E, Bm at x^n
//                    (27-point quadratic stencils from a tile staged by one
//                    4D TMA box where it fits beside the current tile, e.g.
//                    8^3 or 16x8x8 patches; otherwise through the L1 /
//                    read-only path, as for 16^3, whose FP32 tile would need
//                    208 KB), Boris push, move, Esirkepov current on the
//                    4-node window per axis into the shared-memory current
//                    tile (halo 2: at most 144 atomics per particle; FP32 in
//                    32-bit fixed point), boundary conditions,
//                    compaction of stayers and 26 direction buckets for
//                    leavers; SDMD step (i): the tile is added into the
//                    region current with global atomics
//   k3_update_E      E^{n+1} = E^n + dt (curl_h B^{n+1/2} - J^{n+1/2})
//   k3_update_B      B^{n+3/2}, Bm^{n+1} = average, next J set cleared
//   k3_silver_mueller ghost B of every open face (laser at x_min)
//   moving-window shift when due (row shift of every stored value, ring of
//   slot columns, in-flight migration, plasma injection)
//
// Esirkepov in 3D with DS = S1 - S0 per axis:
//   W_x = DSx (S0y S0z + DSy S0z / 2 + S0y DSz / 2 + DSy DSz / 3)
// and cyclically; J_a = -q w (d_a / dt) x prefix sum of W_a along axis a.
// The prefix sums along the 4-node window are DS0, DS0 + DS1 and -DS3 (the
// sum of DS is zero).
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <type_traits>
#include <vector>

#include "common.cuh"
#include "alloc.h"
#include "pic3d.h"
#include "poisson.h"
#include "shape.cuh"

namespace pic {

namespace {

constexpr int G3 = 4;   // ghost cells per side of every axis
constexpr int NB3 = 26; // direction buckets per slot

struct Geom3 {
  int n[3];              // cells
  int p[3];              // patch size
  int np[3];             // patches per axis
  int pshift[3];         // log2 of the patch size when a power of two, else -1
  int nslots;
  int sx, sy, sz;        // stored extents (sx: row stride, multiple of 32)
  long long cs;          // elements per component
  double d[3], dt;
  int fbc[3];
  int pbc[3][2];
  double q, m;
};

__host__ __device__ __forceinline__ long long fidx3(const Geom3 &g, int i, int j, int k) {
  return ((long long)(k + G3) * g.sy + (j + G3)) * g.sx + (i + G3);
}

template <typename R>
struct SoA7 {
  R *x, *y, *z, *ux, *uy, *uz, *w;
};

struct Buckets26 {
  int cap[NB3];
  int off[NB3];
  int stride;
};

__host__ __device__ __forceinline__ int dir26(int dx, int dy, int dz) {
  const int i = (dz + 1) * 9 + (dy + 1) * 3 + (dx + 1);
  return i < 13 ? i : i - 1;
}
__host__ __device__ __forceinline__ void delta26(int d, int &dx, int &dy, int &dz) {
  const int i = d < 13 ? d : d + 1;
  dx = i % 3 - 1;
  dy = (i / 3) % 3 - 1;
  dz = i / 9 - 1;
}

// Physical patch coordinates of a slot (slot columns form a ring along x,
// rotated by the moving window: slot column (col0 + px) mod npx holds
// physical column px).
__host__ __device__ __forceinline__ void slot_patch(const Geom3 &g, int col0, int s, int &px,
                                                    int &py, int &pz) {
  const int sc = s % g.np[0], rest = s / g.np[0];
  px = sc - col0;
  if (px < 0) px += g.np[0];
  py = rest % g.np[1];
  pz = rest / g.np[1];
}
__host__ __device__ __forceinline__ int slot_of(const Geom3 &g, int col0, int px, int py,
                                                int pz) {
  return (pz * g.np[1] + py) * g.np[0] + (px + col0) % g.np[0];
}
// Neighbour of slot s in direction (dx, dy, dz); -1 outside a non-periodic
// face.
__host__ __device__ __forceinline__ int neighbour3(const Geom3 &g, int col0, int s, int dx, int dy,
                                                   int dz) {
  int p[3];
  slot_patch(g, col0, s, p[0], p[1], p[2]);
  const int dd[3] = {dx, dy, dz};
  for (int a = 0; a < 3; ++a) {
    p[a] += dd[a];
    if (p[a] < 0 || p[a] >= g.np[a]) {
      if (g.fbc[a] != FBC_PERIODIC) return -1;
      p[a] = (p[a] + g.np[a]) % g.np[a];
    }
  }
  return slot_of(g, col0, p[0], p[1], p[2]);
}

// Store v at the periodic ghost images of cell (i, j, k) in the stored range
// (one image per periodic axis: every periodic axis has n >= 2 G3 cells).
template <typename R>
__device__ __forceinline__ void mirror3(const Geom3 &g, R *a, int i, int j, int k, R v) {
  int m[3] = {0, 0, 0};
  const int c[3] = {i, j, k};
  for (int ax = 0; ax < 3; ++ax)
    if (g.fbc[ax] == FBC_PERIODIC)
      m[ax] = c[ax] < G3 ? g.n[ax] : (c[ax] >= g.n[ax] - G3 ? -g.n[ax] : 0);
  if (!(m[0] | m[1] | m[2])) return;  // no image: interior cell or no periodic axis
  for (int cz = 0; cz < 2; ++cz)
    for (int cy = 0; cy < 2; ++cy)
      for (int cx = 0; cx < 2; ++cx) {
        if (!(cx | cy | cz)) continue;
        if ((cx && !m[0]) || (cy && !m[1]) || (cz && !m[2])) continue;
        a[fidx3(g, i + cx * m[0], j + cy * m[1], k + cz * m[2])] = v;
      }
}

// ------------------------------------------------------------ step args --

template <typename R>
struct Step3 {
  Geom3 g;
  const R *F;
  R *Jdst;
  SoA7<R> pin, pout, bin, bout;
  const int *cnt_in, *bcnt_in;
  int *cnt_out, *bcnt_out;
  int cap;
  Buckets26 bk;
  int parity;
  DevState *st;
  R rd[3];   // dt / d (cells per unit velocity)
  R eps;     // q dt / (2 m)
  R cj[3];   // -q d / dt
  R RP[3];   // patch size as reals
  // FP32: the shared current tile accumulates in 32-bit fixed point (see
  // StepArgs::jscale): a contribution v adds round(v jscale), the tile's
  // integer times junit is the current
  R jscale, junit;
  int jfloat;  // FP32: accumulate the tile with float atomics instead
  Plan plan;
  const int *active;  // per physical patch: E or Bm nonzero on one of its cells
  long long wait_polls;  // bound on polls of a tile-staging wait
};

template <typename R>
struct Field3 {
  Geom3 g;
  R *F;
  int parity;
  DevState *st;
  R dt, id[3];                          // dt, 1 / d
  R inv1pr[3], omr[3], dtd[3];          // 1/(1+r), 1-r, dt/d per axis (r = dt/d)
  int laser_on;
  const double *laser_g;                // [nz + 1][ny]: a0 exp(-r^2 / w^2) at Ey's nodes
  double tau, t_peak;
  int *active;                          // per physical patch, set by k3_update_B
};

__device__ __forceinline__ int patch_coord(const Geom3 &g, int ax, int c) {
  return g.pshift[ax] >= 0 ? c >> g.pshift[ax] : c / g.p[ax];
}

// Mark the physical patch of cell (i, j, k) (inside the domain) active when
// v is nonzero.  Called by every lane of the active mask; the lanes that
// mark the same patch elect one, which reads the flag and sets it with an
// atomic only if it is still clear.
__device__ __forceinline__ void mark_active(const Geom3 &g, int *active, int i, int j, int k,
                                            bool v) {
  const bool in = v && i >= 0 && j >= 0 && k >= 0 && i < g.n[0] && j < g.n[1] && k < g.n[2];
  const unsigned mask = __ballot_sync(__activemask(), in);
  if (!in) return;
  const int p = (patch_coord(g, 2, k) * g.np[1] + patch_coord(g, 1, j)) * g.np[0] +
                patch_coord(g, 0, i);
  const unsigned same = __match_any_sync(mask, p);
  unsigned lane;
  asm("mov.u32 %0, %%laneid;" : "=r"(lane));
  if ((unsigned)(__ffs(same) - 1) != lane) return;
  if (!*(volatile int *)&active[p]) atomicOr(&active[p], 1);
}

// A patch is quiet when neither it nor any of its 26 neighbours holds a
// nonzero E or Bm on its cells and it touches no open face (whose ghost
// values its stencils also read): every interpolation stencil of the patch
// then reads only zeros.
__device__ __forceinline__ bool patch_quiet(const Geom3 &g, const int *active, const int pc[3]) {
  for (int ax = 0; ax < 3; ++ax)
    if (g.fbc[ax] != FBC_PERIODIC && (pc[ax] == 0 || pc[ax] == g.np[ax] - 1)) return false;
  for (int dz = -1; dz <= 1; ++dz)
    for (int dy = -1; dy <= 1; ++dy)
      for (int dx = -1; dx <= 1; ++dx) {
        const int q[3] = {(pc[0] + dx + g.np[0]) % g.np[0], (pc[1] + dy + g.np[1]) % g.np[1],
                          (pc[2] + dz + g.np[2]) % g.np[2]};
        if (active[(q[2] * g.np[1] + q[1]) * g.np[0] + q[0]]) return false;
      }
  return true;
}

// --------------------------------------------------------------- plan ----

constexpr int PLAN3_CLASSES = 64;

// Work plan in two grid-wide passes (a 3D grid has up to 10^5 patch slots).
// Pass 1: units per slot (segment plus the 26 incoming buckets, clamped to
// the capacities), items per slot, a histogram of item counts per class;
// the step's output counts are cleared.
template <typename R>
__global__ void __launch_bounds__(256) k3_plan_count(const Step3<R> a, int *hist) {
  __shared__ int h[PLAN3_CLASSES];
  const Geom3 &g = a.g;
  const Plan &plan = a.plan;
  const int tid = threadIdx.x;
  const int col0 = a.st->col0;
  for (int c = tid; c < PLAN3_CLASSES; c += blockDim.x) h[c] = 0;
  __syncthreads();
  for (int s = blockIdx.x * blockDim.x + tid; s < g.nslots; s += gridDim.x * blockDim.x) {
    int units = min(a.cnt_in[s], a.cap);
    for (int d = 0; d < NB3; ++d) {
      int dx, dy, dz;
      delta26(d, dx, dy, dz);
      const int src = neighbour3(g, col0, s, -dx, -dy, -dz);
      if (src >= 0) units += min(a.bcnt_in[(long long)src * NB3 + d], a.bk.cap[d]);
    }
    plan.units[s] = units;
    a.cnt_out[s] = 0;
    for (int d = 0; d < NB3; ++d) a.bcnt_out[(long long)s * NB3 + d] = 0;
    const int items = (units + plan.chunk - 1) / plan.chunk;
    if (items) atomicAdd(&h[min(items, PLAN3_CLASSES) - 1], items);
  }
  __syncthreads();
  for (int c = tid; c < PLAN3_CLASSES; c += blockDim.x)
    if (h[c]) atomicAdd(&hist[c], h[c]);
}

// Pass 2: items laid out by class, heaviest first (class offsets from the
// histogram, positions within a class from a per-class cursor).
template <typename R>
__global__ void __launch_bounds__(256) k3_plan_place(const Step3<R> a, const int *hist,
                                                     int *cursor) {
  __shared__ int off[PLAN3_CLASSES];
  const Geom3 &g = a.g;
  const Plan &plan = a.plan;
  const int tid = threadIdx.x;
  if (tid == 0) {
    int run = 0;
    for (int c = PLAN3_CLASSES - 1; c >= 0; --c) {
      off[c] = run;
      run += hist[c];
    }
    if (blockIdx.x == 0) {
      *plan.n_items = min(run, plan.max_items);
      *plan.next = 0;
    }
  }
  __syncthreads();
  for (int s = blockIdx.x * blockDim.x + tid; s < g.nslots; s += gridDim.x * blockDim.x) {
    const int items = (plan.units[s] + plan.chunk - 1) / plan.chunk;
    if (!items) continue;
    const int c = min(items, PLAN3_CLASSES) - 1;
    const int base = off[c] + atomicAdd(&cursor[c], items);
    for (int k = 0; k < items && base + k < plan.max_items; ++k) {
      plan.item_slot[base + k] = s;
      plan.item_first[base + k] = k * plan.chunk;
    }
  }
}

// ------------------------------------------------------ particle step ----

// 27-point interpolation from the region array F (component base) with the
// stencil starting at global node (i0, j0, k0).
template <typename R>
__device__ __forceinline__ R gather27(const R *__restrict__ F, const Geom3 &g, int i0, int j0,
                                      int k0, const R Sx[3], const R Sy[3], const R Sz[3]) {
  const R *p = F + fidx3(g, i0, j0, k0);
  R acc = R(0);
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    R pl = R(0);
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      const R *r = p + ((long long)c * g.sy + b) * g.sx;
      pl += Sy[b] * (Sx[0] * __ldg(r) + Sx[1] * __ldg(r + 1) + Sx[2] * __ldg(r + 2));
    }
    acc += Sz[c] * pl;
  }
  return acc;
}

// 27-point interpolation from a staged tile (row stride BX, plane stride
// BX * BY); (i0, j0, k0) is the stencil's first node in tile indices.
template <typename R>
__device__ __forceinline__ R gather27t(const R *T, int BX, int BY, int i0, int j0, int k0,
                                       const R Sx[3], const R Sy[3], const R Sz[3]) {
  const R *p = T + (k0 * BY + j0) * BX + i0;
  R acc = R(0);
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    R pl = R(0);
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      const R *r = p + (c * BY + b) * BX;
      pl += Sy[b] * (Sx[0] * r[0] + Sx[1] * r[1] + Sx[2] * r[2]);
    }
    acc += Sz[c] * pl;
  }
  return acc;
}

// Blocks per SM that the shared memory of a patch shape allows (at most 3),
// used as the launch bound of the compile-time-shaped kernels: it caps the
// registers so that the occupancy shared memory permits is also reached.
template <typename R, bool STAGED, int PX, int PY, int PZ>
constexpr int k3_min_blocks() {
  if (PX == 0) return sizeof(R) == 4 ? 2 : 1;
  const int smem = (STAGED ? 6 * (PX + 8) * (PY + 3) * (PZ + 3) * (int)sizeof(R) : 0) +
                   3 * (PX + 5) * (PY + 5) * (PZ + 5) * (int)sizeof(R) + 1024 + 128;
  const int n = (228 * 1024) / smem;
  return n >= 3 ? 3 : (n >= 1 ? n : 1);
}

// PX, PY, PZ: the patch shape when fixed at compile time (0: read from the
// geometry), so that tile strides become immediates.  JF (FP32): the current
// tile accumulates with float atomics instead of 32-bit fixed point.
template <typename R, bool STAGED, int PX = 0, int PY = 0, int PZ = 0, bool JF = false>
__global__ void __launch_bounds__(256, (k3_min_blocks<R, STAGED, PX, PY, PZ>()))
    k3_particle_step(const __grid_constant__ CUtensorMap tmap, const Step3<R> a) {
  // STAGED: the patch's E and Bm (nodes -4..P+3 along x, -1..Q+1, -1..R+1)
  // are staged into shared memory by one 4D TMA box (SDMD step (ii)) and
  // gathered there; otherwise gathered from the region in HBM.
  extern __shared__ unsigned char dsm3[];
  __shared__ uint64_t mbar;
  __shared__ int s_qoff[NB3 + 2];
  __shared__ int s_cnt[NB3 + 1];
  __shared__ long long s_base[NB3 + 1];
  __shared__ int s_item;
  __shared__ int s_ok;
  const Geom3 &g = a.g;
  const int tid = threadIdx.x, nth = blockDim.x, lane = tid & 31;
  const int P = PX ? PX : g.p[0], Q = PY ? PY : g.p[1], Rz = PZ ? PZ : g.p[2];
  const int JW = P + 5, JH = Q + 5, JD = Rz + 5, JT = JW * JH * JD;
  const int BX = P + 8, BY = Q + 3, BZ = Rz + 3, FT = BX * BY * BZ;
  const uint32_t pad = (128u - (smem_u32(dsm3) & 127u)) & 127u;
  R *Ft = reinterpret_cast<R *>(dsm3 + pad);
  R *Jt = STAGED ? Ft + 6 * FT : Ft;
  const int n_items = *a.plan.n_items;
  const R eps = a.eps;
  unsigned err = 0;
  uint32_t phase = 0;
  if (STAGED && tid == 0) {
    mbar_init(&mbar, 1);
    fence_mbar_init();
  }
  // STAGED: the next item is fetched, and its field tile load issued, as
  // soon as the particles of the current one are done with the field tile,
  // so that the load overlaps the current tile's flush to the domain.
  auto issue_tile = [&](int it) {
    int q[3];
    slot_patch(g, a.st->col0, a.plan.item_slot[it], q[0], q[1], q[2]);
    mbar_arrive_expect_tx(&mbar, (uint32_t)(6 * FT * sizeof(R)));
    tma_load_4d(Ft, &tmap, &mbar, q[0] * P - 4 + G3, q[1] * Q - 1 + G3, q[2] * Rz - 1 + G3, 0);
  };
  if (STAGED && tid == 0) {
    const int first = atomicAdd(a.plan.next, 1);
    s_item = first;
    if (first < n_items) issue_tile(first);
  }
  for (;;) {
    __syncthreads();
    if (!STAGED) {
      if (tid == 0) s_item = atomicAdd(a.plan.next, 1);
      __syncthreads();
    }
    const int item = s_item;
    if (item >= n_items) break;
    const int s = a.plan.item_slot[item];
    const int ufirst = a.plan.item_first[item];
    const int col0 = a.st->col0;
    int pc[3];
    slot_patch(g, col0, s, pc[0], pc[1], pc[2]);
    const int X0 = pc[0] * P, Y0 = pc[1] * Q, Z0 = pc[2] * Rz;
    for (int e = tid; e < 3 * JT; e += nth) Jt[e] = R(0);
    if (tid < NB3 + 1) {
      int cnt = 0;
      long long base = 0;
      if (tid == 0) {
        cnt = min(a.cnt_in[s], a.cap);
        base = (long long)s * a.cap;
      } else {
        const int d = tid - 1;
        int dx, dy, dz;
        delta26(d, dx, dy, dz);
        const int src = neighbour3(g, col0, s, -dx, -dy, -dz);
        if (src >= 0) {
          cnt = min(a.bcnt_in[(long long)src * NB3 + d], a.bk.cap[d]);
          base = (long long)src * a.bk.stride + a.bk.off[d];
        }
      }
      s_cnt[tid] = cnt;
      s_base[tid] = base;
    }
    __syncthreads();
    if (tid == 0) {
      s_qoff[0] = 0;
      for (int i = 0; i <= NB3; ++i) s_qoff[i + 1] = s_qoff[i] + s_cnt[i];
      int ok = 1;
      if (STAGED) {
        ok = 0;
        for (long long it = 0; it < a.wait_polls; ++it)
          if (mbar_try_wait(&mbar, phase)) { ok = 1; break; }
        if (!ok) {
          atomicOr(&a.st->err, ERR_TIMEOUT);
          for (long long it = 0; it < DRAIN_POLLS; ++it)
            if (mbar_try_wait(&mbar, phase)) break;
        }
      }
      s_ok = ok;
    }
    phase ^= 1u;
    __syncthreads();
    if (!s_ok) break;
    const int total = min(ufirst + a.plan.chunk, s_qoff[NB3 + 1]);
    // particles at rest in a quiet patch stay at rest, in place, and deposit
    // nothing: exactly what the full step computes
    const bool quiet = patch_quiet(g, a.active, pc);
    for (int qb = ufirst; qb < total; qb += nth) {
      const int qi = qb + tid;
      int dir = -2;  // -1 stay, -2 none, 0..25 bucket
      R x1[3] = {R(0), R(0), R(0)}, nu[3] = {R(0), R(0), R(0)}, w = R(0);
      if (qi < total) {
        int lo = 0, hi = NB3 + 1;  // source: last i with s_qoff[i] <= qi
        while (hi - lo > 1) {
          const int mid = (lo + hi) >> 1;
          if (s_qoff[mid] <= qi) lo = mid; else hi = mid;
        }
        const SoA7<R> &A = lo == 0 ? a.pin : a.bin;
        const long long b = s_base[lo] + (qi - s_qoff[lo]);
        const R x0[3] = {A.x[b], A.y[b], A.z[b]};
        R u[3] = {A.ux[b], A.uy[b], A.uz[b]};
        w = A.w[b];
        if (quiet && u[0] == R(0) && u[1] == R(0) && u[2] == R(0)) {
          x1[0] = x0[0];
          x1[1] = x0[1];
          x1[2] = x0[2];
          dir = -1;
        } else {
        // interpolation: primal and dual stencils per axis
        int ip[3], id[3];
        R Sp[3][3], Sd[3][3];
#pragma unroll
        for (int ax = 0; ax < 3; ++ax) shapes(x0[ax], ip[ax], Sp[ax], id[ax], Sd[ax]);
        const int gp[3] = {X0 + ip[0] - 1, Y0 + ip[1] - 1, Z0 + ip[2] - 1};
        const int gd[3] = {X0 + id[0] - 1, Y0 + id[1] - 1, Z0 + id[2] - 1};
        R Ex, Ey, Ez, Bx, By, Bz;
        // checked build: every 3 x 3 x 3 stencil inside the staged tile, or
        // inside the stored region when gathered from HBM
        const bool gok = STAGED
            ? PIC_IN(err, min(id[0] + 3, ip[0] + 3) >= 0 && max(id[0], ip[0]) + 3 + 2 < BX &&
                              min(min(id[1], ip[1]), min(id[2], ip[2])) >= 0 &&
                              max(id[1], ip[1]) + 2 < BY && max(id[2], ip[2]) + 2 < BZ)
            : PIC_IN(err, min(gd[0], gp[0]) >= -G3 && max(gd[0], gp[0]) + 2 < g.n[0] + G3 &&
                              min(gd[1], gp[1]) >= -G3 && max(gd[1], gp[1]) + 2 < g.n[1] + G3 &&
                              min(gd[2], gp[2]) >= -G3 && max(gd[2], gp[2]) + 2 < g.n[2] + G3);
        if (!gok) {
          Ex = Ey = Ez = Bx = By = Bz = R(0);
        } else if (STAGED) {
          // tile index of patch-relative node (x, y, z): x + 4, y + 1, z + 1
          const int tp[3] = {ip[0] + 3, ip[1], ip[2]}, td[3] = {id[0] + 3, id[1], id[2]};
          Ex = gather27t(Ft, BX, BY, td[0], tp[1], tp[2], Sd[0], Sp[1], Sp[2]);
          Ey = gather27t(Ft + FT, BX, BY, tp[0], td[1], tp[2], Sp[0], Sd[1], Sp[2]);
          Ez = gather27t(Ft + 2 * FT, BX, BY, tp[0], tp[1], td[2], Sp[0], Sp[1], Sd[2]);
          Bx = gather27t(Ft + 3 * FT, BX, BY, tp[0], td[1], td[2], Sp[0], Sd[1], Sd[2]);
          By = gather27t(Ft + 4 * FT, BX, BY, td[0], tp[1], td[2], Sd[0], Sp[1], Sd[2]);
          Bz = gather27t(Ft + 5 * FT, BX, BY, td[0], td[1], tp[2], Sd[0], Sd[1], Sp[2]);
        } else {
          const R *F = a.F;
          const long long cs = g.cs;
          Ex = gather27(F + C_EX * cs, g, gd[0], gp[1], gp[2], Sd[0], Sp[1], Sp[2]);
          Ey = gather27(F + C_EY * cs, g, gp[0], gd[1], gp[2], Sp[0], Sd[1], Sp[2]);
          Ez = gather27(F + C_EZ * cs, g, gp[0], gp[1], gd[2], Sp[0], Sp[1], Sd[2]);
          Bx = gather27(F + C_BMX * cs, g, gp[0], gd[1], gd[2], Sp[0], Sd[1], Sd[2]);
          By = gather27(F + C_BMY * cs, g, gd[0], gp[1], gd[2], Sd[0], Sp[1], Sd[2]);
          Bz = gather27(F + C_BMZ * cs, g, gd[0], gd[1], gp[2], Sd[0], Sd[1], Sp[2]);
        }
        // Boris push u^{n-1/2} -> u^{n+1/2}
        const R umx = u[0] + eps * Ex, umy = u[1] + eps * Ey, umz = u[2] + eps * Ez;
        const R ig = eps * rsq(R(1) + umx * umx + umy * umy + umz * umz);
        const R tx = ig * Bx, ty = ig * By, tz = ig * Bz;
        const R f = quot(R(2), R(1) + tx * tx + ty * ty + tz * tz);
        const R upx = umx + (umy * tz - umz * ty);
        const R upy = umy + (umz * tx - umx * tz);
        const R upz = umz + (umx * ty - umy * tx);
        nu[0] = umx + f * (upy * tz - upz * ty) + eps * Ex;
        nu[1] = umy + f * (upz * tx - upx * tz) + eps * Ey;
        nu[2] = umz + f * (upx * ty - upy * tx) + eps * Ez;
        const R inv = rsq(R(1) + nu[0] * nu[0] + nu[1] * nu[1] + nu[2] * nu[2]);
        bool finite = true, slow = true;
        R S0[3][4], DS[3][4];
        int org[3];
        bool x4[3];  // the window spans all four nodes along the axis
#pragma unroll
        for (int ax = 0; ax < 3; ++ax) {
          x1[ax] = x0[ax] + a.rd[ax] * nu[ax] * inv;
          R S13[3];
          const int i1 = shape_primal(x1[ax], S13);
          const int di = i1 - ip[ax];
          finite = finite && isfinite(x1[ax]) && isfinite(nu[ax]);
          slow = slow && di >= -1 && di <= 1;
          const bool sh = di < 0;
          R S1[4];
          window4(Sp[ax], sh, S0[ax]);
          window4(S13, di + (sh ? 1 : 0) != 0, S1);
#pragma unroll
          for (int c = 0; c < 4; ++c) DS[ax][c] = S1[c] - S0[ax][c];
          org[ax] = ip[ax] - 1 - (sh ? 1 : 0) + 2;  // window origin in the tile
          x4[ax] = di != 0;
        }
        if (!finite) err |= ERR_NONFINITE;
        else if (!slow) err |= ERR_FAST;
        if (finite && slow) {
          // Esirkepov: component c, prefix along c, A over the other two.
          // Along an axis where the particle kept its nearest node the
          // window's node 3 carries no shape (S0 = DS = 0 there) and the
          // prefix -DS[3] vanishes: those entries are skipped, as is a
          // whole component when the particle did not move along it.
          const int st3[3] = {1, JW, JW * JH};
          const int base = (org[2] * JH + org[1]) * JW + org[0];
          // checked build: the 4 x 4 x 4 window inside the current tile
          const bool wok = PIC_IN(err, base >= 0 && base + 3 * (1 + JW + JW * JH) < JT);
          constexpr bool fixed = sizeof(R) == 4 && !JF;
          // fixed point: the tile scale folded into the prefix factors, each
          // contribution formed and rounded by one FMA (red_fixed)
          const R jsc = fixed ? a.jscale : R(1);
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            const int b1 = (c + 1) % 3, b2 = (c + 2) % 3;
            const R cw = a.cj[c] * w * jsc;
            const R P0 = cw * DS[c][0], P1 = cw * (DS[c][0] + DS[c][1]), P2 = -cw * DS[c][3];
            if (!wok || (P0 == R(0) && P1 == R(0) && P2 == R(0))) continue;
            R *J = Jt + c * JT + base;
            const int sc = st3[c], s1 = st3[b1], s2 = st3[b2];
            const bool w1 = x4[b1], w2 = x4[b2], wc = x4[c];
            // the (m1, m2) entries of the component, issued in groups: the
            // window's node 3 along b1 (b2) only when w1 (w2), the third
            // prefix entry only when wc
            auto groups = [&](auto WC) {
              constexpr bool kWC = decltype(WC)::value;
              auto put = [&](int m1, int m2) {
                const R A = S0[b1][m1] * (S0[b2][m2] + R(0.5) * DS[b2][m2]) +
                            DS[b1][m1] * (R(0.5) * S0[b2][m2] + R(1.0 / 3.0) * DS[b2][m2]);
                R *row = J + m1 * s1 + m2 * s2;
                if constexpr (fixed) {
                  const uint32_t ad = smem_u32(row);
                  red_fixed(ad, fmaf(P0, A, kRoundMagic));
                  red_fixed(ad + 4u * sc, fmaf(P1, A, kRoundMagic));
                  if constexpr (kWC) red_fixed(ad + 8u * sc, fmaf(P2, A, kRoundMagic));
                } else {
                  atomicAdd(row, P0 * A);
                  atomicAdd(row + sc, P1 * A);
                  if constexpr (kWC) atomicAdd(row + 2 * sc, P2 * A);
                }
              };
#pragma unroll
              for (int m2 = 0; m2 < 3; ++m2)
#pragma unroll
                for (int m1 = 0; m1 < 3; ++m1) put(m1, m2);
              if (w1) {
#pragma unroll
                for (int m2 = 0; m2 < 3; ++m2) put(3, m2);
              }
              if (w2) {
#pragma unroll
                for (int m1 = 0; m1 < 3; ++m1) put(m1, 3);
                if (w1) put(3, 3);
              }
            };
            if (wc) groups(std::true_type{});
            else groups(std::false_type{});
          }
          // boundary conditions, destination patch
          int dd[3];
          bool gone = false;
#pragma unroll
          for (int ax = 0; ax < 3; ++ax) {
            dd[ax] = x1[ax] < R(0) ? -1 : (x1[ax] >= a.RP[ax] ? 1 : 0);
            if (dd[ax] != 0 && (pc[ax] + dd[ax] < 0 || pc[ax] + dd[ax] >= g.np[ax])) {
              const int bc = g.pbc[ax][dd[ax] > 0];
              if (bc == PBC_REFLECT) {
                x1[ax] = dd[ax] < 0 ? -x1[ax] : R(2 * g.p[ax]) - x1[ax];
                if (x1[ax] >= a.RP[ax]) x1[ax] = below(a.RP[ax]);
                nu[ax] = -nu[ax];
                dd[ax] = 0;
              } else if (bc == PBC_REMOVE) {
                gone = true;
              }
            }
          }
          if (!gone) {
#pragma unroll
            for (int ax = 0; ax < 3; ++ax) {
              if (dd[ax] < 0) {
                x1[ax] += a.RP[ax];
                if (x1[ax] >= a.RP[ax]) x1[ax] = below(a.RP[ax]);
              } else if (dd[ax] > 0) {
                x1[ax] -= a.RP[ax];
              }
            }
            dir = (dd[0] == 0 && dd[1] == 0 && dd[2] == 0) ? -1 : dir26(dd[0], dd[1], dd[2]);
          }
        }
        }
      }
      const bool stay = dir == -1;
      const unsigned bal = __ballot_sync(0xffffffffu, stay);
      int wbase = 0;
      if (lane == 0 && bal) wbase = atomicAdd(&a.cnt_out[s], __popc(bal));
      wbase = __shfl_sync(0xffffffffu, wbase, 0);
      if (stay) {
        const int pos = wbase + __popc(bal & ((1u << lane) - 1u));
        if (pos < a.cap) {
          const long long i = (long long)s * a.cap + pos;
          a.pout.x[i] = x1[0]; a.pout.y[i] = x1[1]; a.pout.z[i] = x1[2];
          a.pout.ux[i] = nu[0]; a.pout.uy[i] = nu[1]; a.pout.uz[i] = nu[2];
          a.pout.w[i] = w;
        } else {
          err |= ERR_OVERFLOW_SEG;
        }
      } else if (dir >= 0) {
        const int bp = atomicAdd(&a.bcnt_out[(long long)s * NB3 + dir], 1);
        if (bp < a.bk.cap[dir]) {
          const long long i = (long long)s * a.bk.stride + a.bk.off[dir] + bp;
          a.bout.x[i] = x1[0]; a.bout.y[i] = x1[1]; a.bout.z[i] = x1[2];
          a.bout.ux[i] = nu[0]; a.bout.uy[i] = nu[1]; a.bout.uz[i] = nu[2];
          a.bout.w[i] = w;
        } else {
          err |= ERR_OVERFLOW_BKT;
        }
      }
    }
    __syncthreads();
    // the field tile is free: fetch the next item and start its tile load
    if (STAGED && tid == 0) {
      const int nxt = atomicAdd(a.plan.next, 1);
      s_item = nxt;
      if (nxt < n_items) issue_tile(nxt);
    }
    // SDMD step (i): patch current tile -> region current
    for (int e = tid; e < 3 * JT; e += nth) {
      R v;
      if (sizeof(R) == 4 && !JF) {
        const int iv = reinterpret_cast<const int *>(Jt)[e];
        v = iv ? R(iv) * a.junit : R(0);
      } else {
        v = Jt[e];
      }
      if (v == R(0)) continue;
      const int c = e / JT, r = e - c * JT;
      const int l = r / (JW * JH), r2 = r - l * (JW * JH), m = r2 / JW, q = r2 - m * JW;
      int gi = X0 - 2 + q, gj = Y0 - 2 + m, gk = Z0 - 2 + l;
      if (g.fbc[0] == FBC_PERIODIC) gi = gi < 0 ? gi + g.n[0] : (gi >= g.n[0] ? gi - g.n[0] : gi);
      if (g.fbc[1] == FBC_PERIODIC) gj = gj < 0 ? gj + g.n[1] : (gj >= g.n[1] ? gj - g.n[1] : gj);
      if (g.fbc[2] == FBC_PERIODIC) gk = gk < 0 ? gk + g.n[2] : (gk >= g.n[2] ? gk - g.n[2] : gk);
      // checked build: the node inside the stored region
      if (PIC_IN(err, gi >= -G3 && gi < g.n[0] + G3 && gj >= -G3 && gj < g.n[1] + G3 &&
                          gk >= -G3 && gk < g.n[2] + G3))
        atomicAdd(&a.Jdst[c * g.cs + fidx3(g, gi, gj, gk)], v);
    }
    if (tid == 0) atomicMax(&a.st->maxcnt[a.parity], atomicAdd(&a.cnt_out[s], 0));
  }
  if (err) atomicOr(&a.st->err, err);
}

// -------------------------------------------------------------- fields ----

// E^{n+1} = E^n + dt (curl_h B^{n+1/2} - J^{n+1/2}): one cell per thread;
// periodic axes update [0, n), open axes primal nodes [0, n], dual [0, n).
template <typename R>
__global__ void __launch_bounds__(256) k3_update_E(const Field3<R> a) {
  const Geom3 &g = a.g;
  if (blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0 && threadIdx.x == 0 &&
      threadIdx.y == 0) {
    // laser temporal factor at t_{n+3/2} for the Silver-Mueller kernel
    double h = 0.0;
    if (a.laser_on) {
      const double t = a.st->t[a.parity] + 1.5 * g.dt;
      const double tr = t - (double)(a.st->nshift * g.p[0]) * g.d[0] - a.t_peak;
      h = exp(-2.0 * log(2.0) * tr * tr / (a.tau * a.tau)) * sin(tr);
    }
    a.st->laser_h = h;
  }
  const int i = blockIdx.x * 32 + threadIdx.x, j = blockIdx.y * 8 + threadIdx.y, k = blockIdx.z;
  int np_[3];
  for (int ax = 0; ax < 3; ++ax) np_[ax] = g.n[ax] + (g.fbc[ax] == FBC_SM);
  if (i >= np_[0] || j >= np_[1] || k >= np_[2]) return;
  const long long cs = g.cs, o = fidx3(g, i, j, k);
  const long long sy = g.sx, sz = (long long)g.sx * g.sy;
  R *F = a.F;
  R *Ex = F + C_EX * cs, *Ey = F + C_EY * cs, *Ez = F + C_EZ * cs;
  const R *Bx = F + C_BX * cs, *By = F + C_BY * cs, *Bz = F + C_BZ * cs;
  const R *J = F + (C_JA + 3 * a.parity) * cs;
  const R dt = a.dt, idx = a.id[0], idy = a.id[1], idz = a.id[2];
  const R bx = Bx[o], by = By[o], bz = Bz[o];
  if (i < g.n[0]) {
    const R v = Ex[o] + dt * ((bz - Bz[o - sy]) * idy - (by - By[o - sz]) * idz - J[o]);
    Ex[o] = v;
    mirror3(g, Ex, i, j, k, v);
  }
  if (j < g.n[1]) {
    const R v = Ey[o] + dt * ((bx - Bx[o - sz]) * idz - (bz - Bz[o - 1]) * idx - J[cs + o]);
    Ey[o] = v;
    mirror3(g, Ey, i, j, k, v);
  }
  if (k < g.n[2]) {
    const R v = Ez[o] + dt * ((by - By[o - 1]) * idx - (bx - Bx[o - sy]) * idy - J[2 * cs + o]);
    Ez[o] = v;
    mirror3(g, Ez, i, j, k, v);
  }
}

// B^{n+3/2} = B^{n+1/2} - dt curl_h E^{n+1}, Bm^{n+1} = (B^{n+1/2} +
// B^{n+3/2}) / 2 (= B where not updated), next J set cleared; covers every
// stored cell.
template <typename R>
__global__ void __launch_bounds__(256) k3_update_B(const Field3<R> a) {
  const Geom3 &g = a.g;
  if (blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0 && threadIdx.x == 0 &&
      threadIdx.y == 0) {
    const int p = a.parity;
    a.st->t[1 - p] = a.st->t[p] + g.dt;
    a.st->step[1 - p] = a.st->step[p] + 1;
    a.st->maxcnt[1 - p] = 0;
  }
  const int i = (int)(blockIdx.x * 32 + threadIdx.x) - G3;
  const int j = (int)(blockIdx.y * 8 + threadIdx.y) - G3;
  const int k = (int)blockIdx.z - G3;
  if (i >= g.n[0] + G3 || j >= g.n[1] + G3 || k >= g.n[2] + G3) return;
  const long long cs = g.cs, o = fidx3(g, i, j, k);
  const long long sy = g.sx, sz = (long long)g.sx * g.sy;
  R *F = a.F;
  R *Jn = F + (C_JA + 3 * (1 - a.parity)) * cs;
  Jn[o] = R(0);
  Jn[cs + o] = R(0);
  Jn[2 * cs + o] = R(0);
  const int c[3] = {i, j, k};
  for (int ax = 0; ax < 3; ++ax)
    if (g.fbc[ax] == FBC_PERIODIC && (c[ax] < 0 || c[ax] >= g.n[ax])) return;  // mirror cell
  const R *Ex = F + C_EX * cs, *Ey = F + C_EY * cs, *Ez = F + C_EZ * cs;
  R *Bx = F + C_BX * cs, *By = F + C_BY * cs, *Bz = F + C_BZ * cs;
  R *Bmx = F + C_BMX * cs, *Bmy = F + C_BMY * cs, *Bmz = F + C_BMZ * cs;
  const R dt = a.dt, idx = a.id[0], idy = a.id[1], idz = a.id[2];
  bool in = i >= 0 && j >= 0 && k >= 0;
  bool pr[3], du[3];  // inside the primal / dual update range per axis
  for (int ax = 0; ax < 3; ++ax) {
    pr[ax] = c[ax] < g.n[ax] + (g.fbc[ax] == FBC_SM);
    du[ax] = c[ax] < g.n[ax];
  }
  const bool ux = in && pr[0] && du[1] && du[2];
  const bool uy = in && du[0] && pr[1] && du[2];
  const bool uz = in && du[0] && du[1] && pr[2];
  const R bx0 = Bx[o], by0 = By[o], bz0 = Bz[o];
  const R ex = Ex[o], ey = Ey[o], ez = Ez[o];
  R bx1 = bx0, by1 = by0, bz1 = bz0;
  if (ux) bx1 = bx0 - dt * ((Ez[o + sy] - ez) * idy - (Ey[o + sz] - ey) * idz);
  if (uy) by1 = by0 - dt * ((Ex[o + sz] - ex) * idz - (Ez[o + 1] - ez) * idx);
  if (uz) bz1 = bz0 - dt * ((Ey[o + 1] - ey) * idx - (Ex[o + sy] - ex) * idy);
  if (ux) { Bx[o] = bx1; mirror3(g, Bx, i, j, k, bx1); }
  if (uy) { By[o] = by1; mirror3(g, By, i, j, k, by1); }
  if (uz) { Bz[o] = bz1; mirror3(g, Bz, i, j, k, bz1); }
  const R mx = R(0.5) * (bx0 + bx1), my = R(0.5) * (by0 + by1), mz = R(0.5) * (bz0 + bz1);
  Bmx[o] = mx;
  Bmy[o] = my;
  Bmz[o] = mz;
  mirror3(g, Bmx, i, j, k, mx);
  mirror3(g, Bmy, i, j, k, my);
  mirror3(g, Bmz, i, j, k, mz);
  const bool nz = mx != R(0) || my != R(0) || mz != R(0) || ex != R(0) || ey != R(0) ||
                  ez != R(0);
  if (__any_sync(__activemask(), nz)) mark_active(g, a.active, i, j, k, nz);
}

// Active flags from the stored fields (after any change outside a step:
// loading, setting fields, a window shift).
template <typename R>
__global__ void k3_scan_active(const Geom3 g, const R *F, int *active) {
  const long long nc = (long long)g.n[0] * g.n[1] * g.n[2];
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < nc;
       e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e % g.n[0]), j = (int)((e / g.n[0]) % g.n[1]);
    const int k = (int)(e / ((long long)g.n[0] * g.n[1]));
    const long long o = fidx3(g, i, j, k);
    bool nz = false;
    for (int c = 0; c < 6; ++c) nz = nz || F[(long long)c * g.cs + o] != R(0);
    mark_active(g, active, i, j, k, nz);
  }
}

template <typename R>
__device__ __forceinline__ void set_ghost3(const Geom3 &g, R *B, R *Bm, int i, int j, int k, R v) {
  const long long o = fidx3(g, i, j, k);
  const R old = Bm[o];  // = B^{n+1/2} at this ghost after k3_update_B
  B[o] = v;
  mirror3(g, B, i, j, k, v);
  const R m = R(0.5) * (old + v);
  Bm[o] = m;
  mirror3(g, Bm, i, j, k, m);
}

// Ghost B of the open faces from the first-order Silver-Mueller condition
// taken half a step ahead of E^{n+1} with Ampere's law on the boundary node.
// Face of axis a, pair (E_c, B_d) with d the third axis; s = +1 when
// (curl B)_c holds +d_a B_d, -1 when it holds -d_a B_d; T = -s d_d B_a the
// transverse part (zero where it needs a ghost of another open axis):
//   lower: G = [2 e + dt T - s (1 - r) I - 4 e_inc] / (s (1 + r))
//   upper: G = -[2 e + dt T + s (1 - r) I] / (s (1 + r))
// blockIdx.y = face (2 axis + upper); threads over the face's points.
template <typename R>
__global__ void k3_silver_mueller(const Field3<R> a) {
  const Geom3 &g = a.g;
  const int face = blockIdx.y, ax = face >> 1, upper = face & 1;
  if (g.fbc[ax] != FBC_SM) return;
  const double s_h = (ax == 0 && !upper) ? a.st->laser_h : 0.0;  // set by k3_update_E
  const int b1 = ax == 0 ? 1 : 0, b2 = ax == 2 ? 1 : 2;  // transverse axes, increasing
  const int n1 = g.n[b1] + 1, n2 = g.n[b2] + 1;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n1 * n2) return;
  const int u1 = t % n1, u2 = t / n1;
  R *F = a.F;
  const long long cs = g.cs;
  const R r1 = a.omr[ax], ia = a.inv1pr[ax];
  for (int c = 0; c < 3; ++c) {
    if (c == ax) continue;
    int s, d;
    if ((c + 1) % 3 == ax) { s = 1; d = (c + 2) % 3; }
    else { s = -1; d = (c + 1) % 3; }
    // transverse range of the ghost B_d: primal along d, dual elsewhere
    const int lim1 = (b1 == d && g.fbc[b1] == FBC_SM) ? g.n[b1] + 1 : g.n[b1];
    const int lim2 = (b2 == d && g.fbc[b2] == FBC_SM) ? g.n[b2] + 1 : g.n[b2];
    if (u1 >= lim1 || u2 >= lim2) continue;
    int node[3];
    node[ax] = upper ? g.n[ax] : 0;
    node[b1] = u1;
    node[b2] = u2;
    int gh[3] = {node[0], node[1], node[2]}, in[3] = {node[0], node[1], node[2]};
    gh[ax] = upper ? g.n[ax] : -1;
    in[ax] = upper ? g.n[ax] - 1 : 0;
    const R *E = F + (C_EX + c) * cs;
    R *Bd = F + (C_BX + d) * cs, *Bmd = F + (C_BMX + d) * cs;
    const R *Ba = F + (C_BX + ax) * cs;
    R T = R(0);
    const int nd = node[d];
    if (g.fbc[d] == FBC_PERIODIC || (nd >= 1 && nd <= g.n[d] - 1)) {
      int m[3] = {node[0], node[1], node[2]};
      m[d] -= 1;
      const R diff = Ba[fidx3(g, node[0], node[1], node[2])] - Ba[fidx3(g, m[0], m[1], m[2])];
      T = (s > 0 ? -diff : diff);  // times dt / d_d below
    }
    const R dtT = a.dtd[d] * T;
    const R e = E[fidx3(g, node[0], node[1], node[2])];
    const R I = Bd[fidx3(g, in[0], in[1], in[2])];
    R v;
    if (!upper) {
      R einc = R(0);
      if (a.laser_on && ax == 0 && c == 1) einc = R(a.laser_g[(long long)node[2] * g.n[1] + node[1]] * s_h);
      v = s > 0 ? (R(2) * e + dtT - r1 * I - R(4) * einc) * ia
                : -(R(2) * e + dtT + r1 * I - R(4) * einc) * ia;
    } else {
      v = s > 0 ? -(R(2) * e + dtT + r1 * I) * ia : (R(2) * e + dtT - r1 * I) * ia;
    }
    set_ghost3(g, Bd, Bmd, gh[0], gh[1], gh[2], v);
  }
}

// ------------------------------------------------------ field transfer ----

__host__ __device__ inline void out_dims3(const Geom3 &g, int lo[3], int cnt[3]) {
  for (int ax = 0; ax < 3; ++ax) {
    lo[ax] = g.fbc[ax] == FBC_PERIODIC ? 0 : -1;
    cnt[ax] = g.fbc[ax] == FBC_PERIODIC ? g.n[ax] : g.n[ax] + 2;
  }
}

template <typename R, typename S>
__global__ void k3_set_field(const Geom3 g, R *arr, const S *src, int mirror) {
  int lo[3], cnt[3];
  out_dims3(g, lo, cnt);
  const long long tot = (long long)cnt[0] * cnt[1] * cnt[2];
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
       e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e % cnt[0]), j = (int)((e / cnt[0]) % cnt[1]), k = (int)(e / ((long long)cnt[0] * cnt[1]));
    const R v = R(src[e]);
    arr[fidx3(g, lo[0] + i, lo[1] + j, lo[2] + k)] = v;
    if (mirror) mirror3(g, arr, lo[0] + i, lo[1] + j, lo[2] + k, v);
  }
}

template <typename R>
__global__ void k3_get_field(const Geom3 g, const R *arr, double *dst) {
  int lo[3], cnt[3];
  out_dims3(g, lo, cnt);
  const long long tot = (long long)cnt[0] * cnt[1] * cnt[2];
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
       e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e % cnt[0]), j = (int)((e / cnt[0]) % cnt[1]), k = (int)(e / ((long long)cnt[0] * cnt[1]));
    dst[e] = (double)arr[fidx3(g, lo[0] + i, lo[1] + j, lo[2] + k)];
  }
}

// Moving window: every stored row (along x) of `ncomp` components moves P
// cells down; indices with no source become vacuum.
template <typename R>
__global__ void k3_shift_rows(const Geom3 g, R *base, long long comp_stride) {
  extern __shared__ unsigned char row3_raw[];
  R *row = reinterpret_cast<R *>(row3_raw);
  R *a = base + blockIdx.y * comp_stride + (long long)blockIdx.x * g.sx;
  const int n = g.n[0] + 2 * G3, P = g.p[0];
  for (int e = threadIdx.x; e < n; e += blockDim.x) row[e] = a[e];
  __syncthreads();
  for (int e = threadIdx.x; e < n; e += blockDim.x) {
    const int i = e - G3;
    a[e] = (i + P < g.n[0] + G3) ? row[e + P] : R(0);
  }
}

// ----------------------------------------------------------- particles ----

__device__ __forceinline__ bool locate3(const Geom3 &g, int col0, const double *x, int &slot,
                                        int pc[3]) {
  for (int ax = 0; ax < 3; ++ax) {
    const double c = x[ax] / g.d[ax];
    if (!(c >= 0.0 && c < (double)g.n[ax])) return false;
    pc[ax] = min((int)floor(c) / g.p[ax], g.np[ax] - 1);
  }
  slot = slot_of(g, col0, pc[0], pc[1], pc[2]);
  return true;
}

template <typename R>
__device__ __forceinline__ R rel3(double c, int origin, int P) {
  R r = R(c - (double)origin);
  if (r < R(0)) r = R(0);
  if (r >= R(P)) r = nextafter(R(P), R(0));
  return r;
}

__global__ void k3_bin_count(const Geom3 g, int col0, const double *x, const double *y,
                             const double *z, size_t n, int *counts, unsigned *err) {
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n;
       k += (size_t)gridDim.x * blockDim.x) {
    int slot, pc[3];
    const double p[3] = {x[k], y[k], z[k]};
    if (!locate3(g, col0, p, slot, pc)) {
      atomicOr(err, ERR_LOAD_RANGE);
      continue;
    }
    atomicAdd(&counts[slot], 1);
  }
}

template <typename R>
__global__ void k3_bin_place(const Geom3 g, int col0, const double *x, const double *y,
                             const double *z, const double *ux, const double *uy,
                             const double *uz, const double *w, size_t n, SoA7<R> seg,
                             int *counts, int cap, unsigned *err) {
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n;
       k += (size_t)gridDim.x * blockDim.x) {
    int slot, pc[3];
    const double p[3] = {x[k], y[k], z[k]};
    if (!locate3(g, col0, p, slot, pc)) continue;
    const int pos = atomicAdd(&counts[slot], 1);
    if (pos >= cap) {
      atomicOr(err, ERR_OVERFLOW_LOAD);
      continue;
    }
    const long long i = (long long)slot * cap + pos;
    seg.x[i] = rel3<R>(x[k] / g.d[0], pc[0] * g.p[0], g.p[0]);
    seg.y[i] = rel3<R>(y[k] / g.d[1], pc[1] * g.p[1], g.p[1]);
    seg.z[i] = rel3<R>(z[k] / g.d[2], pc[2] * g.p[2], g.p[2]);
    seg.ux[i] = R(ux[k]);
    seg.uy[i] = R(uy[k]);
    seg.uz[i] = R(uz[k]);
    seg.w[i] = R(w[k]);
  }
}

// Live particles of a view: segments of one set plus the buckets of the
// other, bucket particles in the frame of their destination patch.
template <typename R>
struct View3 {
  SoA7<R> seg, bkt;
  const int *cnt, *bcnt;
  int cap;
  Buckets26 bk;
};

template <typename R, typename Fn>
__device__ void for_each3(const Geom3 &g, int col0, const View3<R> &v, Fn fn) {
  for (int slot = blockIdx.x; slot < g.nslots; slot += gridDim.x) {
    int pc[3];
    slot_patch(g, col0, slot, pc[0], pc[1], pc[2]);
    const int n = min(v.cnt[slot], v.cap);
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
      const long long i = (long long)slot * v.cap + k;
      fn(pc, v.seg, i);
    }
    for (int d = 0; d < NB3; ++d) {
      const int nb = min(v.bcnt[(long long)slot * NB3 + d], v.bk.cap[d]);
      if (nb == 0) continue;
      int dx, dy, dz;
      delta26(d, dx, dy, dz);
      const int dest = neighbour3(g, col0, slot, dx, dy, dz);
      if (dest < 0) continue;
      int qc[3];
      slot_patch(g, col0, dest, qc[0], qc[1], qc[2]);
      for (int k = threadIdx.x; k < nb; k += blockDim.x)
        fn(qc, v.bkt, (long long)slot * v.bk.stride + v.bk.off[d] + k);
    }
  }
}

__device__ __forceinline__ void shape_d3(double xi, int &i0, double S[3]) {
  const double fl = floor(xi + 0.5);
  const double d = xi - fl;
  S[0] = 0.5 * (0.5 - d) * (0.5 - d);
  S[1] = 0.75 - d * d;
  S[2] = 0.5 * (0.5 + d) * (0.5 + d);
  i0 = (int)fl;
}

// rho += qw S(x) S(y) S(z) at nodes (periodic axes wrapped to canonical
// nodes); position in cells relative to the patch origin O.
__device__ __forceinline__ void deposit_node3(const Geom3 &g, double *rho, const int O[3],
                                              const double xr[3], double qw) {
  int i0[3];
  double S[3][3];
  for (int ax = 0; ax < 3; ++ax) shape_d3(xr[ax], i0[ax], S[ax]);
  for (int c = 0; c < 3; ++c)
    for (int b = 0; b < 3; ++b)
      for (int a = 0; a < 3; ++a) {
        int gi = O[0] + i0[0] - 1 + a, gj = O[1] + i0[1] - 1 + b, gk = O[2] + i0[2] - 1 + c;
        if (g.fbc[0] == FBC_PERIODIC) gi = (gi + g.n[0]) % g.n[0];
        if (g.fbc[1] == FBC_PERIODIC) gj = (gj + g.n[1]) % g.n[1];
        if (g.fbc[2] == FBC_PERIODIC) gk = (gk + g.n[2]) % g.n[2];
        atomicAdd(&rho[fidx3(g, gi, gj, gk)], qw * S[0][a] * S[1][b] * S[2][c]);
      }
}

template <typename R>
__global__ void k3_deposit_rho(const Geom3 g, int col0, const View3<R> v, double *rho, double sign) {
  const double qs = sign * g.q;
  for_each3<R>(g, col0, v, [&](const int pc[3], const SoA7<R> &A, long long i) {
    const int O[3] = {pc[0] * g.p[0], pc[1] * g.p[1], pc[2] * g.p[2]};
    const double xr[3] = {(double)A.x[i], (double)A.y[i], (double)A.z[i]};
    deposit_node3(g, rho, O, xr, qs * (double)A.w[i]);
  });
}

template <typename R>
__global__ void k3_particle_diag(const Geom3 g, int col0, const View3<R> v, double *partials) {
  __shared__ double sh[3][256];
  double ek = 0.0, ws = 0.0, cnt = 0.0;
  for_each3<R>(g, col0, v, [&](const int *, const SoA7<R> &A, long long i) {
    const double a = A.ux[i], b = A.uy[i], c = A.uz[i];
    ek += (double)A.w[i] * (sqrt(1.0 + a * a + b * b + c * c) - 1.0);
    ws += (double)A.w[i];
    cnt += 1.0;
  });
  sh[0][threadIdx.x] = ek;
  sh[1][threadIdx.x] = ws;
  sh[2][threadIdx.x] = cnt;
  __syncthreads();
  for (int st = blockDim.x / 2; st > 0; st >>= 1) {
    if (threadIdx.x < st)
      for (int q = 0; q < 3; ++q) sh[q][threadIdx.x] += sh[q][threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int q = 0; q < 3; ++q) partials[3 * blockIdx.x + q] = sh[q][0];
}

// offsets: [physical-order segment offsets (nslots)] [bucket offsets
// (nslots * 26)]; rows x, y, z, ux, uy, uz, w of length `stride`.
template <typename R>
__global__ void k3_get_particles(const Geom3 g, int col0, const View3<R> v,
                                 const long long *offsets, double *out, size_t stride) {
  const int pp = blockIdx.x;  // physical patch index (x fastest)
  if (pp >= g.nslots) return;
  const int ppx = pp % g.np[0], ppy = (pp / g.np[0]) % g.np[1], ppz = pp / (g.np[0] * g.np[1]);
  const int slot = slot_of(g, col0, ppx, ppy, ppz);
  auto emit = [&](long long o, const int pc[3], const SoA7<R> &A, long long i) {
    out[o] = ((double)(pc[0] * g.p[0]) + (double)A.x[i]) * g.d[0];
    out[stride + o] = ((double)(pc[1] * g.p[1]) + (double)A.y[i]) * g.d[1];
    out[2 * stride + o] = ((double)(pc[2] * g.p[2]) + (double)A.z[i]) * g.d[2];
    out[3 * stride + o] = (double)A.ux[i];
    out[4 * stride + o] = (double)A.uy[i];
    out[5 * stride + o] = (double)A.uz[i];
    out[6 * stride + o] = (double)A.w[i];
  };
  const int pc[3] = {ppx, ppy, ppz};
  const int n = min(v.cnt[slot], v.cap);
  const long long base = offsets[pp];
  for (int k = threadIdx.x; k < n; k += blockDim.x) emit(base + k, pc, v.seg, (long long)slot * v.cap + k);
  for (int d = 0; d < NB3; ++d) {
    int dx, dy, dz;
    delta26(d, dx, dy, dz);
    const int dest = neighbour3(g, col0, slot, dx, dy, dz);
    if (dest < 0) continue;
    const int nb = min(v.bcnt[(long long)slot * NB3 + d], v.bk.cap[d]);
    int qc[3];
    slot_patch(g, col0, dest, qc[0], qc[1], qc[2]);
    const long long b = offsets[g.nslots + (long long)pp * NB3 + d];
    for (int k = threadIdx.x; k < nb; k += blockDim.x)
      emit(b + k, qc, v.bkt, (long long)slot * v.bk.stride + v.bk.off[d] + k);
  }
}

// Moving window, part 1 (old ring): particles that crossed from the leaving
// column during the last step are in the leaving slots' +x buckets; append
// them to their destination segments, then clear every bucket that points
// into or out of the leaving column.  One block per (py, pz).
template <typename R>
__global__ void k3_window_migrate(const Geom3 g, int col0, SoA7<R> seg, int *cnt, SoA7<R> bkt,
                                  int *bcnt, int cap, Buckets26 bk, unsigned *err) {
  const int py = blockIdx.x % g.np[1], pz = blockIdx.x / g.np[1];
  const int sdrop = slot_of(g, col0, 0, py, pz);
  const int snext = slot_of(g, col0, 1, py, pz);
  __shared__ int base;
  for (int e = 0; e < 9; ++e) {
    const int dy = e % 3 - 1, dz = e / 3 - 1;
    const int d = dir26(1, dy, dz);
    const int dest = neighbour3(g, col0, sdrop, 1, dy, dz);
    const int nb = min(bcnt[(long long)sdrop * NB3 + d], bk.cap[d]);
    if (dest < 0 || nb == 0) continue;
    if (threadIdx.x == 0) base = atomicAdd(&cnt[dest], nb);
    __syncthreads();
    for (int k = threadIdx.x; k < nb; k += blockDim.x) {
      const int pos = base + k;
      if (pos >= cap) {
        atomicOr(err, ERR_OVERFLOW_SEG);
        continue;
      }
      const long long i = (long long)sdrop * bk.stride + bk.off[d] + k;
      const long long o = (long long)dest * cap + pos;
      seg.x[o] = bkt.x[i]; seg.y[o] = bkt.y[i]; seg.z[o] = bkt.z[i];
      seg.ux[o] = bkt.ux[i]; seg.uy[o] = bkt.uy[i]; seg.uz[o] = bkt.uz[i];
      seg.w[o] = bkt.w[i];
    }
    __syncthreads();
  }
  if (threadIdx.x < NB3) {
    bcnt[(long long)sdrop * NB3 + threadIdx.x] = 0;
    int dx, dy, dz;
    delta26(threadIdx.x, dx, dy, dz);
    if (dx == -1) bcnt[(long long)snext * NB3 + threadIdx.x] = 0;
  }
}

// Plasma at rest, regularly placed (ppc per axis), weight = density(x_lab)
// / ppc, in the cells of the patch whose centre has y >= ymin, with the
// co-located immobile ions added to the background charge.  Block
// (py + npy pz, c) fills physical column phys0 + c, held by slot column
// (slot_col0 + c) mod npx.
template <typename R>
__global__ void k3_inject(const Geom3 g, int slot_col0, int phys0, int nshift, SoA7<R> seg,
                          int *cnt, int cap, double n0, double x0, double ramp, double ymin,
                          int ppcx, int ppcy, int ppcz, double *rho_bg, unsigned *err) {
  const int py = blockIdx.x % g.np[1], pz = blockIdx.x / g.np[1];
  const int phys = phys0 + (int)blockIdx.y;
  const int slot = (pz * g.np[1] + py) * g.np[0] + (slot_col0 + (int)blockIdx.y) % g.np[0];
  const int P = g.p[0], Q = g.p[1], Rz = g.p[2];
  const int X0 = phys * P, Y0 = py * Q, Z0 = pz * Rz;
  int jf = 0;  // first row of the patch with plasma (rows above it are all in)
  while (jf < Q && !(((double)(Y0 + jf) + 0.5) * g.d[1] >= ymin)) ++jf;
  const int rows = Q - jf;
  const int ppc = ppcx * ppcy * ppcz;
  const int total = P * rows * Rz * ppc;
  if (total > cap) {
    if (threadIdx.x == 0) atomicOr(err, ERR_OVERFLOW_SEG);
    return;
  }
  const double shift = __dmul_rn((double)nshift * P, g.d[0]);
  const int O[3] = {X0, Y0, Z0};
  for (int k = threadIdx.x; k < total; k += blockDim.x) {
    const int a = k % ppcx, b = (k / ppcx) % ppcy, c = (k / (ppcx * ppcy)) % ppcz;
    const int cell = k / ppc;
    const int ci = cell % P, cj = jf + (cell / P) % rows, ck = cell / (P * rows);
    const double fx = (a + 0.5) / ppcx, fy = (b + 0.5) / ppcy, fz = (c + 0.5) / ppcz;
    const double xl = ((double)(X0 + ci) + fx) * g.d[0];
    const double xphys = __dadd_rn(xl, shift);
    double n;
    if (ramp <= 0.0) {
      n = xphys >= x0 ? n0 : 0.0;
    } else {
      double f = (xphys - x0) / ramp;
      f = f < 0.0 ? 0.0 : (f > 1.0 ? 1.0 : f);
      n = n0 * f;
    }
    const double w = n / ppc;
    const long long o = (long long)slot * cap + k;
    seg.x[o] = R((double)ci + fx);
    seg.y[o] = R((double)cj + fy);
    seg.z[o] = R((double)ck + fz);
    seg.ux[o] = R(0);
    seg.uy[o] = R(0);
    seg.uz[o] = R(0);
    seg.w[o] = R(w);
    if (rho_bg) {
      const double xr[3] = {(double)ci + fx, (double)cj + fy, (double)ck + fz};
      deposit_node3(g, rho_bg, O, xr, -g.q * (double)R(w));
    }
  }
  if (threadIdx.x == 0) cnt[slot] = total;
}

// ---------------------------------------------------------- diagnostics ----

template <typename R>
__global__ void k3_field_energy(const Geom3 g, const R *F, double *partials) {
  __shared__ double sh[2][256];
  double ue = 0.0, ub = 0.0;
  const long long nc = (long long)g.n[0] * g.n[1] * g.n[2];
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < nc;
       e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e % g.n[0]), j = (int)((e / g.n[0]) % g.n[1]), k = (int)(e / ((long long)g.n[0] * g.n[1]));
    const long long o = fidx3(g, i, j, k);
    for (int c = 0; c < 3; ++c) {
      const double ev = (double)F[(C_EX + c) * g.cs + o], bv = (double)F[(C_BMX + c) * g.cs + o];
      ue += ev * ev;
      ub += bv * bv;
    }
  }
  sh[0][threadIdx.x] = ue;
  sh[1][threadIdx.x] = ub;
  __syncthreads();
  for (int st = blockDim.x / 2; st > 0; st >>= 1) {
    if (threadIdx.x < st) {
      sh[0][threadIdx.x] += sh[0][threadIdx.x + st];
      sh[1][threadIdx.x] += sh[1][threadIdx.x + st];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    partials[2 * blockIdx.x] = sh[0][0];
    partials[2 * blockIdx.x + 1] = sh[1][0];
  }
}

// max |div_h E - rho - rho_bg| and the continuity residual max |(rho -
// rho_prev)/dt + div_h J| over the cells 3 or more away from open faces.
template <typename R>
__global__ void k3_gauss(const Geom3 g, const R *F, int jset, const double *rho,
                         const double *rho_prev, const double *rho_bg, double *partials) {
  __shared__ double sh[2][256];
  int lo[3], w[3];
  for (int ax = 0; ax < 3; ++ax) {
    lo[ax] = g.fbc[ax] == FBC_PERIODIC ? 0 : 3;
    w[ax] = (g.fbc[ax] == FBC_PERIODIC ? g.n[ax] : g.n[ax] - 3) - lo[ax];
  }
  double gm = 0.0, cm = 0.0;
  const R *Ex = F + C_EX * g.cs, *Ey = F + C_EY * g.cs, *Ez = F + C_EZ * g.cs;
  const R *J = F + (C_JA + 3 * jset) * g.cs;
  const long long tot = (long long)max(w[0], 0) * max(w[1], 0) * max(w[2], 0);
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
       e += (long long)gridDim.x * blockDim.x) {
    const int i = lo[0] + (int)(e % w[0]), j = lo[1] + (int)((e / w[0]) % w[1]),
              k = lo[2] + (int)(e / ((long long)w[0] * w[1]));
    const long long o = fidx3(g, i, j, k);
    const double divE = ((double)Ex[o] - (double)Ex[fidx3(g, i - 1, j, k)]) / g.d[0] +
                        ((double)Ey[o] - (double)Ey[fidx3(g, i, j - 1, k)]) / g.d[1] +
                        ((double)Ez[o] - (double)Ez[fidx3(g, i, j, k - 1)]) / g.d[2];
    gm = fmax(gm, fabs(divE - rho[o] - rho_bg[o]));
    if (rho_prev) {
      // the current lives on canonical nodes: wrap the -1 neighbours
      const int im = (g.fbc[0] == FBC_PERIODIC && i == 0) ? g.n[0] - 1 : i - 1;
      const int jm = (g.fbc[1] == FBC_PERIODIC && j == 0) ? g.n[1] - 1 : j - 1;
      const int km = (g.fbc[2] == FBC_PERIODIC && k == 0) ? g.n[2] - 1 : k - 1;
      const double divJ = ((double)J[o] - (double)J[fidx3(g, im, j, k)]) / g.d[0] +
                          ((double)J[g.cs + o] - (double)J[g.cs + fidx3(g, i, jm, k)]) / g.d[1] +
                          ((double)J[2 * g.cs + o] - (double)J[2 * g.cs + fidx3(g, i, j, km)]) / g.d[2];
      cm = fmax(cm, fabs((rho[o] - rho_prev[o]) / g.dt + divJ));
    }
  }
  sh[0][threadIdx.x] = gm;
  sh[1][threadIdx.x] = cm;
  __syncthreads();
  for (int st = blockDim.x / 2; st > 0; st >>= 1) {
    if (threadIdx.x < st) {
      sh[0][threadIdx.x] = fmax(sh[0][threadIdx.x], sh[0][threadIdx.x + st]);
      sh[1][threadIdx.x] = fmax(sh[1][threadIdx.x], sh[1][threadIdx.x + st]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    partials[2 * blockIdx.x] = sh[0][0];
    partials[2 * blockIdx.x + 1] = sh[1][0];
  }
}

__global__ void k3_window_state(DevState *st, int col0, int nshift) {
  st->col0 = col0;
  st->nshift = nshift;
}

// Copy one particle set (patch segments of capacity cap_src and the 26
// direction buckets of layout bk_src) into storage of another capacity and
// bucket layout; counts beyond a destination capacity are cut to it.
template <typename R>
__global__ void k3_repack(int nslots, SoA7<R> src, const int *cnt_src, int cap_src, SoA7<R> bsrc,
                          const int *bcnt_src, Buckets26 bk_src, SoA7<R> dst, int *cnt_dst,
                          int cap_dst, SoA7<R> bdst, int *bcnt_dst, Buckets26 bk_dst) {
  auto copy = [](SoA7<R> &d, long long i, const SoA7<R> &s, long long j) {
    d.x[i] = s.x[j]; d.y[i] = s.y[j]; d.z[i] = s.z[j];
    d.ux[i] = s.ux[j]; d.uy[i] = s.uy[j]; d.uz[i] = s.uz[j]; d.w[i] = s.w[j];
  };
  for (int slot = blockIdx.x; slot < nslots; slot += gridDim.x) {
    const int n = min(min(cnt_src[slot], cap_src), cap_dst);
    const long long so = (long long)slot * cap_src, dof = (long long)slot * cap_dst;
    for (int k = threadIdx.x; k < n; k += blockDim.x) copy(dst, dof + k, src, so + k);
    for (int d = 0; d < NB3; ++d) {
      const int nb = min(min(bcnt_src[(long long)slot * NB3 + d], bk_src.cap[d]), bk_dst.cap[d]);
      const long long bs = (long long)slot * bk_src.stride + bk_src.off[d];
      const long long bd = (long long)slot * bk_dst.stride + bk_dst.off[d];
      for (int k = threadIdx.x; k < nb; k += blockDim.x) copy(bdst, bd + k, bsrc, bs + k);
      if (threadIdx.x == 0) bcnt_dst[(long long)slot * NB3 + d] = nb;
    }
    if (threadIdx.x == 0) cnt_dst[slot] = n;
  }
}

// Snapshot packing of one particle set: the live particles of every slot's
// segment and 26 buckets to or from seven contiguous arrays (x y z ux uy uz
// w), each `total` long; off[27 s] is slot s's segment offset, off[27 s + 1
// + d] its bucket d's (counts clamped to the capacities).
template <typename R, bool PACK>
__global__ void k3_pack(int nslots, SoA7<R> seg, const int *cnt, int cap, SoA7<R> bkt,
                        const int *bcnt, Buckets26 bk, const long long *off, R *flat,
                        long long total) {
  R *fa[7], *sa[7] = {seg.x, seg.y, seg.z, seg.ux, seg.uy, seg.uz, seg.w};
  R *ba[7] = {bkt.x, bkt.y, bkt.z, bkt.ux, bkt.uy, bkt.uz, bkt.w};
#pragma unroll
  for (int a = 0; a < 7; ++a) fa[a] = flat + a * total;
  for (int slot = blockIdx.x; slot < nslots; slot += gridDim.x) {
    const int n = min(cnt[slot], cap);
    const long long so = (long long)slot * cap, fo = off[27LL * slot];
    for (int k = threadIdx.x; k < n; k += blockDim.x)
#pragma unroll
      for (int a = 0; a < 7; ++a) {
        if (PACK) fa[a][fo + k] = sa[a][so + k];
        else sa[a][so + k] = fa[a][fo + k];
      }
    for (int d = 0; d < NB3; ++d) {
      const int nb = min(bcnt[(long long)slot * NB3 + d], bk.cap[d]);
      const long long bo = (long long)slot * bk.stride + bk.off[d], fb = off[27LL * slot + 1 + d];
      for (int k = threadIdx.x; k < nb; k += blockDim.x)
#pragma unroll
        for (int a = 0; a < 7; ++a) {
          if (PACK) fa[a][fb + k] = ba[a][bo + k];
          else ba[a][bo + k] = fa[a][fb + k];
        }
    }
  }
}

}  // namespace

// ================================================================ host ====

struct Ctx3 {
  pic_config cfg;
  Geom3 g;
  bool fp32;
  size_t rs;
  cudaStream_t stream;
  void *F = nullptr;
  double *rho_bg = nullptr, *rho_a = nullptr, *rho_b = nullptr, *laser_g = nullptr;
  void *seg[2][7] = {}, *bkt[2][7] = {};
  int *cnt[2] = {}, *bcnt[2] = {};
  int cap = 0;
  Buckets26 bk{};
  Plan plan{};
  int ps_grid = 0;
  size_t ps_smem = 0;
  const void *ps_kernel = nullptr;  // the particle-step instance for this patch shape
  bool staged = false;   // E and Bm tiles staged into shared memory by TMA
  CUtensorMap tmap{};
  DevState *st = nullptr;
  int *active = nullptr;       // per physical patch: nonzero E or Bm on its cells
  int *plan_hist = nullptr;    // class histogram and cursors of the work plan
  bool active_valid = false;   // the flags describe the stored fields
  double *partials = nullptr;
  int npartials = 1024;
  long long *offsets = nullptr;
  double *staging = nullptr;
  size_t staging_n = 0;
  long long step = 0;
  double t = 0.0;
  int nshift = 0, col0 = 0;
  double wmax = 0.0;  // largest |w| held or injected (FP32 current scale)
  bool prev_valid = false;
  cudaGraphExec_t gexec[2] = {nullptr, nullptr};
  double ms_particles = 0, ms_fields = 0, ms_window = 0;
  long long launches = 0, ps_launches = 0;
  int sticky = PIC_OK;
  std::string err;
  // state at the entry of pic_step (auto_grow): replayed after an overflow
  struct Backup {
    void *F = nullptr;
    double *rho_bg = nullptr;
    void *seg[7] = {}, *bkt[7] = {};
    int *cnt = nullptr, *bcnt = nullptr;
    DevState *st = nullptr;
    int cap = 0;
    Buckets26 bk{};
    long long step = 0;
    double t = 0.0;
    int nshift = 0, col0 = 0;
  } bak;
  int grows = 0;
};

// Device memory of a 3D context (the caller's allocator when configured).
template <typename T>
cudaError_t cmalloc3(Ctx3 *c, T **p, size_t bytes) {
  return dev_malloc(c->cfg, p, bytes);
}
void cfree3(Ctx3 *c, void *p) { dev_free(c->cfg, c->stream, p); }

namespace {

pic_status fail3(Ctx3 *c, pic_status s, const std::string &m) {
  if (c) c->err = m;
  return s;
}

#define CK3(call)                                                                        \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess)                                                               \
      return fail3(c, PIC_ECUDA, std::string(#call ": ") + cudaGetErrorString(e_));      \
  } while (0)

Geom3 make_geom3(const pic_config *cf) {
  Geom3 g{};
  for (int a = 0; a < 3; ++a) {
    g.n[a] = cf->n[a];
    g.p[a] = cf->patch[a];
    g.np[a] = g.n[a] / g.p[a];
    g.d[a] = cf->d[a];
    g.fbc[a] = cf->bc_field[a];
    g.pbc[a][0] = cf->bc_part[a][0];
    g.pbc[a][1] = cf->bc_part[a][1];
  }
  for (int a = 0; a < 3; ++a) {
    g.pshift[a] = -1;
    for (int b = 0; b < 16; ++b)
      if (g.p[a] == (1 << b)) g.pshift[a] = b;
  }
  g.nslots = g.np[0] * g.np[1] * g.np[2];
  g.sx = (g.n[0] + 2 * G3 + 31) / 32 * 32;
  g.sy = g.n[1] + 2 * G3;
  g.sz = g.n[2] + 2 * G3;
  g.cs = (long long)g.sx * g.sy * g.sz;
  g.dt = cf->dt;
  g.q = cf->q;
  g.m = cf->m;
  return g;
}

size_t tile_bytes(const pic_config *cf, size_t rs) {
  return (size_t)3 * (cf->patch[0] + 5) * (cf->patch[1] + 5) * (cf->patch[2] + 5) * rs + 128;
}

Buckets26 layout26(int cap) {
  Buckets26 b{};
  int off = 0;
  for (int d = 0; d < NB3; ++d) {
    int dx, dy, dz;
    delta26(d, dx, dy, dz);
    // a step crosses one face of a patch (at most one cell deep) far more
    // often than an edge or a corner; x faces take the laser-driven sheets
    const int m = (dx != 0) + (dy != 0) + (dz != 0);
    const int div = m == 1 ? (dx != 0 ? 2 : 4) : (m == 2 ? 16 : 32);
    b.cap[d] = std::max(32, (cap / div + 31) / 32 * 32);
    b.off[d] = off;
    off += b.cap[d];
  }
  b.stride = off;
  return b;
}

size_t particle_bytes3(const Geom3 &g, int cap, size_t rs) {
  const Buckets26 b = layout26(cap);
  return 2 * (7 * rs * ((size_t)g.nslots * cap + (size_t)g.nslots * b.stride) +
              sizeof(int) * ((size_t)g.nslots * (1 + NB3)));
}

template <typename R>
SoA7<R> soa7(void *const a[7]) {
  return SoA7<R>{(R *)a[0], (R *)a[1], (R *)a[2], (R *)a[3], (R *)a[4], (R *)a[5], (R *)a[6]};
}

template <typename R>
View3<R> view3(Ctx3 *c, int segset, int bktset) {
  View3<R> v;
  v.seg = soa7<R>(c->seg[segset]);
  v.bkt = soa7<R>(c->bkt[bktset]);
  v.cnt = c->cnt[segset];
  v.bcnt = c->bcnt[bktset];
  v.cap = c->cap;
  v.bk = c->bk;
  return v;
}

pic_status poll3(Ctx3 *c) {
  CK3(cudaStreamSynchronize(c->stream));
  DevState h;
  CK3(cudaMemcpy(&h, c->st, sizeof h, cudaMemcpyDeviceToHost));
  if (h.err) {
    pic_status s = PIC_ENONFINITE;
    std::string m = "device fault:";
    if (h.err & ERR_TIMEOUT) { s = PIC_ETIMEOUT; m += " wait ran out;"; }
    if (h.err & (ERR_OVERFLOW_SEG | ERR_OVERFLOW_BKT | ERR_OVERFLOW_LOAD)) {
      if (s != PIC_ETIMEOUT) s = PIC_EOVERFLOW;
      m += " patch capacity exceeded (raise capacity_factor);";
    }
    if (h.err & ERR_NONFINITE) m += " non-finite particle;";
    if (h.err & ERR_FAST) m += " particle moved more than one cell;";
    if (h.err & ERR_LOAD_RANGE) { s = PIC_EINVAL; m += " particle outside the domain;"; }
    if (h.err & ERR_BOUNDS) { s = PIC_ECUDA; m += " index out of bounds (checked build);"; }
    c->sticky = s;
    return fail3(c, s, m);
  }
  return PIC_OK;
}

void free_graphs3(Ctx3 *c) {
  for (int p = 0; p < 2; ++p)
    if (c->gexec[p]) {
      cudaGraphExecDestroy(c->gexec[p]);
      c->gexec[p] = nullptr;
    }
}

template <typename R>
pic_status alloc3(Ctx3 *c, int cap) {
  c->cap = cap;
  c->bk = layout26(cap);
  const Geom3 &g = c->g;
  for (int s = 0; s < 2; ++s) {
    for (int a = 0; a < 7; ++a) {
      CK3(cmalloc3(c, &c->seg[s][a], sizeof(R) * (size_t)g.nslots * cap));
      CK3(cmalloc3(c, &c->bkt[s][a], sizeof(R) * (size_t)g.nslots * c->bk.stride));
    }
    CK3(cmalloc3(c, &c->cnt[s], sizeof(int) * g.nslots));
    CK3(cmalloc3(c, &c->bcnt[s], sizeof(int) * (size_t)g.nslots * NB3));
    CK3(cudaMemsetAsync(c->cnt[s], 0, sizeof(int) * g.nslots, c->stream));
    CK3(cudaMemsetAsync(c->bcnt[s], 0, sizeof(int) * (size_t)g.nslots * NB3, c->stream));
  }
  CK3(cmalloc3(c, &c->offsets, sizeof(long long) * ((size_t)g.nslots * (1 + NB3) + 1)));
  Plan &pl = c->plan;
  pl.unit = 1;
  pl.chunk = c->cfg.task_chunk > 0 ? c->cfg.task_chunk : 2048;
  const long long units_max = (long long)cap + c->bk.stride;
  pl.max_items = (int)std::min<long long>((long long)g.nslots * ((units_max + pl.chunk - 1) / pl.chunk),
                                          1ll << 30);
  CK3(cmalloc3(c, &pl.item_slot, sizeof(int) * pl.max_items));
  CK3(cmalloc3(c, &pl.item_first, sizeof(int) * pl.max_items));
  CK3(cmalloc3(c, &pl.n_items, sizeof(int) * 2));
  pl.next = pl.n_items + 1;
  CK3(cmalloc3(c, &pl.units, sizeof(int) * g.nslots));
  return PIC_OK;
}

void free_particles3(Ctx3 *c) {
  for (int s = 0; s < 2; ++s) {
    for (int a = 0; a < 7; ++a) {
      cfree3(c, c->seg[s][a]);
      cfree3(c, c->bkt[s][a]);
      c->seg[s][a] = c->bkt[s][a] = nullptr;
    }
    cfree3(c, c->cnt[s]);
    cfree3(c, c->bcnt[s]);
    c->cnt[s] = c->bcnt[s] = nullptr;
  }
  cfree3(c, c->offsets);
  cfree3(c, c->plan.item_slot);
  cfree3(c, c->plan.item_first);
  cfree3(c, c->plan.n_items);
  cfree3(c, c->plan.units);
  c->offsets = nullptr;
  c->plan = Plan{};
}

template <typename R>
Step3<R> step_args3(Ctx3 *c, int p) {
  const Geom3 &g = c->g;
  Step3<R> a;
  a.g = g;
  a.wait_polls = wait_polls_of(c->cfg.staging_wait_polls);
  a.F = (const R *)c->F;
  a.Jdst = (R *)c->F + (C_JA + 3 * p) * g.cs;
  a.pin = soa7<R>(c->seg[p]);
  a.pout = soa7<R>(c->seg[1 - p]);
  a.bin = soa7<R>(c->bkt[1 - p]);
  a.bout = soa7<R>(c->bkt[p]);
  a.cnt_in = c->cnt[p];
  a.cnt_out = c->cnt[1 - p];
  a.bcnt_in = c->bcnt[1 - p];
  a.bcnt_out = c->bcnt[p];
  a.cap = c->cap;
  a.bk = c->bk;
  a.parity = p;
  a.st = c->st;
  for (int ax = 0; ax < 3; ++ax) {
    a.rd[ax] = R(g.dt / g.d[ax]);
    a.cj[ax] = R(-g.q * g.d[ax] / g.dt);
    a.RP[ax] = R(g.p[ax]);
  }
  a.eps = R(g.q * g.dt / (2.0 * g.m));
  a.plan = c->plan;
  a.active = c->active;
  // Every contribution is (q d/dt) w P A with |P| <= |displacement in
  // cells| < dt/d (the prefix sum of the quadratic shape weights changes at
  // most at rate 1) and the transverse weight A <= (3/4)^2: below (3/4)^2
  // |q| w_max.  The scale 2^K / ((3/4)^3 |q| w_max) keeps it below (4/3)
  // 2^K and an item's sums below (4/3) 2^30 < 2^31 (K = 30 - ceil(log2 of
  // the particles of an item)); K <= 20 keeps each contribution below
  // 2^22, the range in which the kernel rounds it by adding 1.5 * 2^23.
  const int per_item = c->plan.chunk > 0 ? c->plan.chunk : 2048;
  int lg = 0;
  while ((1 << lg) < per_item) ++lg;
  const double two_k = std::ldexp(1.0, std::min(30 - lg, 20));
  const double cm = 0.421875 * std::fabs(g.q);
  const double wm = cm > 0 ? std::max(c->wmax, two_k / (cm * 1e30)) : 0.0;
  const double sc = cm > 0 ? two_k / (cm * wm) : 0.0;
  a.jscale = R(sc);
  a.junit = sc > 0 ? R(1.0 / sc) : R(0);
  a.jfloat = c->cfg.current_float != 0;
  return a;
}

template <typename R>
Field3<R> field_args3(Ctx3 *c, int p) {
  const Geom3 &g = c->g;
  Field3<R> f;
  f.g = g;
  f.F = (R *)c->F;
  f.parity = p;
  f.st = c->st;
  f.dt = R(g.dt);
  for (int ax = 0; ax < 3; ++ax) {
    const double r = g.dt / g.d[ax];
    f.id[ax] = R(1.0 / g.d[ax]);
    f.inv1pr[ax] = R(1.0 / (1.0 + r));
    f.omr[ax] = R(1.0 - r);
    f.dtd[ax] = R(g.dt / g.d[ax]);
  }
  f.laser_on = c->cfg.laser_on;
  f.laser_g = c->laser_g;
  f.tau = c->cfg.laser_tau;
  f.t_peak = c->cfg.laser_t_peak;
  f.active = c->active;
  return f;
}

template <typename R>
pic_status enqueue_step3(Ctx3 *c, int p, cudaEvent_t mid = nullptr) {
  const Geom3 &g = c->g;
  const Step3<R> a = step_args3<R>(c, p);
  CK3(cudaMemsetAsync(c->plan_hist, 0, sizeof(int) * 2 * PLAN3_CLASSES, c->stream));
  const int pb = std::min(1024, (g.nslots + 255) / 256);
  k3_plan_count<R><<<pb, 256, 0, c->stream>>>(a, c->plan_hist);
  k3_plan_place<R><<<pb, 256, 0, c->stream>>>(a, c->plan_hist, c->plan_hist + PLAN3_CLASSES);
  {
    using K = void (*)(CUtensorMap, Step3<R>);
    const K k = reinterpret_cast<K>(const_cast<void *>(c->ps_kernel));
    k<<<c->ps_grid, 256, c->ps_smem, c->stream>>>(c->tmap, a);
  }
  CK3(cudaGetLastError());
  if (mid) CK3(cudaEventRecord(mid, c->stream));
  const Field3<R> f = field_args3<R>(c, p);
  int npn[3];
  for (int ax = 0; ax < 3; ++ax) npn[ax] = g.n[ax] + (g.fbc[ax] == FBC_SM);
  k3_update_E<R><<<dim3((npn[0] + 31) / 32, (npn[1] + 7) / 8, npn[2]), dim3(32, 8), 0, c->stream>>>(f);
  CK3(cudaMemsetAsync(c->active, 0, sizeof(int) * g.nslots, c->stream));  // marked again by B
  k3_update_B<R><<<dim3((g.n[0] + 2 * G3 + 31) / 32, (g.n[1] + 2 * G3 + 7) / 8, g.n[2] + 2 * G3),
                   dim3(32, 8), 0, c->stream>>>(f);
  if (g.fbc[0] == FBC_SM || g.fbc[1] == FBC_SM || g.fbc[2] == FBC_SM) {
    int mx = 0;
    for (int ax = 0; ax < 3; ++ax) {
      const int b1 = ax == 0 ? 1 : 0, b2 = ax == 2 ? 1 : 2;
      mx = std::max(mx, (g.n[b1] + 1) * (g.n[b2] + 1));
    }
    k3_silver_mueller<R><<<dim3((mx + 255) / 256, 6), 256, 0, c->stream>>>(f);
  }
  CK3(cudaGetLastError());
  return PIC_OK;
}

int kernels_per_step3(const Ctx3 *c) {
  const Geom3 &g = c->g;
  return 5 + ((g.fbc[0] == FBC_SM || g.fbc[1] == FBC_SM || g.fbc[2] == FBC_SM) ? 1 : 0);
}

template <typename R>
pic_status window_shift3(Ctx3 *c) {
  const Geom3 &g = c->g;
  const int q = (int)(c->step & 1), bset = 1 - q, last_j = 1 - q;
  R *F = (R *)c->F;
  const size_t smem = sizeof(R) * (g.n[0] + 2 * G3 + g.p[0]);
  k3_shift_rows<R><<<dim3(g.sy * g.sz, 9), 256, smem, c->stream>>>(g, F, g.cs);
  k3_shift_rows<R><<<dim3(g.sy * g.sz, 3), 256, smem, c->stream>>>(g, F + (C_JA + 3 * last_j) * g.cs, g.cs);
  k3_shift_rows<double><<<dim3(g.sy * g.sz, 1), 256, sizeof(double) * (g.n[0] + 2 * G3 + g.p[0]),
                          c->stream>>>(g, c->rho_bg, g.cs);
  const int old_col0 = c->col0;
  c->nshift += 1;
  c->col0 = (old_col0 + 1) % g.np[0];
  k3_window_migrate<R><<<g.np[1] * g.np[2], 256, 0, c->stream>>>(
      g, old_col0, soa7<R>(c->seg[q]), c->cnt[q], soa7<R>(c->bkt[bset]), c->bcnt[bset], c->cap, c->bk,
      &c->st->err);
  k3_inject<R><<<dim3(g.np[1] * g.np[2], 1), 256, 0, c->stream>>>(
      g, old_col0, g.np[0] - 1, c->nshift, soa7<R>(c->seg[q]), c->cnt[q], c->cap, c->cfg.inj_n0,
      c->cfg.inj_x0, c->cfg.inj_ramp, c->cfg.inj_ymin, c->cfg.inj_ppc[0], c->cfg.inj_ppc[1],
      c->cfg.inj_ppc[2], c->rho_bg, &c->st->err);
  k3_window_state<<<1, 1, 0, c->stream>>>(c->st, c->col0, c->nshift);
  CK3(cudaGetLastError());
  c->launches += 6;
  c->prev_valid = false;
  c->active_valid = false;  // the fields moved
  return PIC_OK;
}

int window_columns3(const pic_config &c) {
  return c.window_cells > 0 ? c.window_cells / c.patch[0] : 1;
}

bool window_due3(const Ctx3 *c) {
  const int m = window_columns3(c->cfg);
  return c->cfg.moving_window && c->t > c->cfg.mw_t0 &&
         c->t - c->cfg.mw_t0 >= (c->nshift / m + 1) * (double)m * c->g.p[0] * c->g.d[0];
}

PFN_cuTensorMapEncodeTiled_v12000 encode3() {
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

// The particle-step instance for a patch shape: FP32 patches of 16x8x8,
// 8x8x8 and 16x16x16 cells get compile-time-shaped kernels, every other
// shape (and FP64, bound by its FP64 rate, and the FP32 float-atomic
// current tile) the runtime-shaped one.
template <typename R>
const void *pick_particle_step3(const int p[3], bool staged, bool jfloat) {
  if constexpr (sizeof(R) == 4) {
    // float-atomic current tile: the runtime-shaped instances
    if (jfloat)
      return staged ? (const void *)k3_particle_step<R, true, 0, 0, 0, true>
                    : (const void *)k3_particle_step<R, false, 0, 0, 0, true>;
    if (p[0] == 16 && p[1] == 8 && p[2] == 8)
      return staged ? (const void *)k3_particle_step<R, true, 16, 8, 8>
                    : (const void *)k3_particle_step<R, false, 16, 8, 8>;
    if (p[0] == 8 && p[1] == 8 && p[2] == 8)
      return staged ? (const void *)k3_particle_step<R, true, 8, 8, 8>
                    : (const void *)k3_particle_step<R, false, 8, 8, 8>;
    if (p[0] == 16 && p[1] == 16 && p[2] == 16 && !staged)
      return (const void *)k3_particle_step<R, false, 16, 16, 16>;
  }
  return staged ? (const void *)k3_particle_step<R, true> : (const void *)k3_particle_step<R, false>;
}

template <typename R>
pic_status prepare3(Ctx3 *c) {
  if (c->ps_grid) return PIC_OK;
  const Geom3 &g = c->g;
  const size_t field_tile = (size_t)6 * (g.p[0] + 8) * (g.p[1] + 3) * (g.p[2] + 3) * sizeof(R);
  const size_t staged_smem = field_tile + tile_bytes(&c->cfg, sizeof(R));
  auto enc = encode3();
  c->staged = c->cfg.tma != 0 && enc && staged_smem <= 227 * 1024;
  if (c->staged) {
    // 4D box (x, y, z, component) over E and Bm, components 0..5
    cuuint64_t dims[4] = {(cuuint64_t)g.sx, (cuuint64_t)g.sy, (cuuint64_t)g.sz, 6};
    cuuint64_t strides[3] = {(cuuint64_t)g.sx * sizeof(R), (cuuint64_t)g.sx * g.sy * sizeof(R),
                             (cuuint64_t)g.cs * sizeof(R)};
    cuuint32_t box[4] = {(cuuint32_t)(g.p[0] + 8), (cuuint32_t)(g.p[1] + 3),
                         (cuuint32_t)(g.p[2] + 3), 6};
    cuuint32_t es[4] = {1, 1, 1, 1};
    const CUresult r = enc(&c->tmap,
                           sizeof(R) == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                          : CU_TENSOR_MAP_DATA_TYPE_FLOAT64,
                           4, c->F, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                           CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) c->staged = false;
  }
  c->ps_smem = c->staged ? staged_smem : tile_bytes(&c->cfg, sizeof(R));
  const void *k = pick_particle_step3<R>(g.p, c->staged, c->cfg.current_float != 0);
  c->ps_kernel = k;
  CK3(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)c->ps_smem));
  int per_sm = 0, dev = 0, nsm = 0;
  CK3(cudaGetDevice(&dev));
  CK3(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  CK3(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, 256, c->ps_smem));
  if (per_sm <= 0) return fail3(c, PIC_EINVAL, "the patch current tile does not fit in shared memory");
  c->ps_grid = per_sm * nsm;
  return PIC_OK;
}

template <typename R>
pic_status capture3(Ctx3 *c) {
  for (int p = 0; p < 2; ++p) {
    cudaGraph_t gr;
    CK3(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
    pic_status s = enqueue_step3<R>(c, p);
    cudaError_t e = cudaStreamEndCapture(c->stream, &gr);
    if (s != PIC_OK) return s;
    CK3(e);
    e = cudaGraphInstantiate(&c->gexec[p], gr, 0);
    cudaGraphDestroy(gr);
    CK3(e);
  }
  return PIC_OK;
}

template <typename R>
pic_status run3(Ctx3 *c, int nsteps) {
  pic_status s = prepare3<R>(c);
  if (s) return s;
  const bool timing = c->cfg.timing != 0;
  const bool use_graph = c->cfg.use_graph && !timing;
  if (use_graph && !c->gexec[0]) {
    s = capture3<R>(c);
    if (s) return s;
  }
  std::vector<cudaEvent_t> ev;
  std::vector<int> kind;
  pic_status rs = PIC_OK;
  for (int n = 0; n < nsteps && rs == PIC_OK; ++n) {
    const int p = (int)(c->step & 1);
    if (!c->active_valid) {
      CK3(cudaMemsetAsync(c->active, 0, sizeof(int) * c->g.nslots, c->stream));
      k3_scan_active<R><<<1024, 256, 0, c->stream>>>(c->g, (const R *)c->F, c->active);
      CK3(cudaGetLastError());
      c->launches += 1;
      c->active_valid = true;
    }
    if (use_graph) {
      CK3(cudaGraphLaunch(c->gexec[p], c->stream));
    } else if (timing) {
      cudaEvent_t e[3];
      for (int k = 0; k < 3; ++k) CK3(cudaEventCreate(&e[k]));
      CK3(cudaEventRecord(e[0], c->stream));
      rs = enqueue_step3<R>(c, p, e[1]);
      CK3(cudaEventRecord(e[2], c->stream));
      for (int k = 0; k < 3; ++k) ev.push_back(e[k]);
      kind.push_back(0);
    } else {
      rs = enqueue_step3<R>(c, p);
    }
    c->launches += kernels_per_step3(c);
    c->ps_launches += 1;
    c->step += 1;
    c->t += c->g.dt;
    c->prev_valid = true;
    if (rs == PIC_OK && window_due3(c)) {
      cudaEvent_t e[2];
      if (timing) {
        for (int k = 0; k < 2; ++k) CK3(cudaEventCreate(&e[k]));
        CK3(cudaEventRecord(e[0], c->stream));
      }
      for (int k = 0; k < window_columns3(c->cfg) && rs == PIC_OK; ++k) rs = window_shift3<R>(c);
      if (timing) {
        CK3(cudaEventRecord(e[1], c->stream));
        ev.push_back(e[0]);
        ev.push_back(e[1]);
        kind.push_back(1);
      }
    }
  }
  if (!ev.empty()) {
    CK3(cudaStreamSynchronize(c->stream));
    size_t k = 0;
    for (int t : kind) {
      float a = 0, b = 0;
      if (t == 0) {
        CK3(cudaEventElapsedTime(&a, ev[k], ev[k + 1]));
        CK3(cudaEventElapsedTime(&b, ev[k + 1], ev[k + 2]));
        c->ms_particles += a;
        c->ms_fields += b;
        k += 3;
      } else {
        CK3(cudaEventElapsedTime(&a, ev[k], ev[k + 1]));
        c->ms_window += a;
        k += 2;
      }
    }
    for (cudaEvent_t e : ev) cudaEventDestroy(e);
  }
  if (rs) return rs;
  return poll3(c);
}

int capacity_for(const Ctx3 *c, int fullest) {
  const double cf = c->cfg.capacity_factor > 0 ? c->cfg.capacity_factor : 2.0;
  const int cmin = c->cfg.capacity_min > 0 ? c->cfg.capacity_min : 256;
  int cap = std::max(cmin, (int)std::ceil(cf * fullest));
  return (cap + 31) / 32 * 32;
}

template <typename R>
pic_status load3(Ctx3 *c, const double *const src[7], size_t n, int where) {
  const Geom3 &g = c->g;
  const double *d[7];
  double *tmp = nullptr;
  if (where == PIC_HOST) {
    CK3(cmalloc3(c, &tmp, sizeof(double) * 7 * std::max<size_t>(n, 1)));
    for (int a = 0; a < 7; ++a) {
      CK3(cudaMemcpyAsync(tmp + a * n, src[a], sizeof(double) * n, cudaMemcpyHostToDevice, c->stream));
      d[a] = tmp + a * n;
    }
  } else {
    for (int a = 0; a < 7; ++a) d[a] = src[a];
  }
  int *cnt = nullptr;
  CK3(cmalloc3(c, &cnt, sizeof(int) * g.nslots));
  CK3(cudaMemsetAsync(cnt, 0, sizeof(int) * g.nslots, c->stream));
  const int blocks = (int)std::min<size_t>((n + 255) / 256 + 1, 4096);
  k3_bin_count<<<blocks, 256, 0, c->stream>>>(g, c->col0, d[0], d[1], d[2], n, cnt, &c->st->err);
  unsigned long long *wbits = reinterpret_cast<unsigned long long *>(c->partials);
  CK3(cudaMemsetAsync(wbits, 0, sizeof *wbits, c->stream));
  CK3(launch_absmax_f64(d[6], n, wbits, c->stream));
  unsigned long long hw = 0;
  CK3(cudaMemcpyAsync(&hw, wbits, sizeof hw, cudaMemcpyDeviceToHost, c->stream));
  std::vector<int> h(g.nslots);
  CK3(cudaMemcpyAsync(h.data(), cnt, sizeof(int) * g.nslots, cudaMemcpyDeviceToHost, c->stream));
  DevState hs;
  CK3(cudaMemcpyAsync(&hs, c->st, sizeof hs, cudaMemcpyDeviceToHost, c->stream));
  CK3(cudaStreamSynchronize(c->stream));
  cfree3(c, cnt);
  c->launches += 1;
  if (hs.err & ERR_LOAD_RANGE) {
    const unsigned keep = hs.err & ~ERR_LOAD_RANGE;
    CK3(cudaMemcpy(&c->st->err, &keep, sizeof keep, cudaMemcpyHostToDevice));
    if (tmp) cfree3(c, tmp);
    return fail3(c, PIC_EINVAL, "particle position outside the domain");
  }
  double wl = 0.0;
  memcpy(&wl, &hw, sizeof wl);
  if (!std::isfinite(wl)) {
    if (tmp) cfree3(c, tmp);
    return fail3(c, PIC_EINVAL, "non-finite particle weight");
  }
  if (wl > c->wmax) {
    c->wmax = wl;
    free_graphs3(c);  // the current scale is baked into captured steps
  }
  if (!c->cap) {
    int mx = *std::max_element(h.begin(), h.end());
    if (c->cfg.moving_window)
      mx = std::max(mx, g.p[0] * g.p[1] * g.p[2] * c->cfg.inj_ppc[0] * c->cfg.inj_ppc[1] * c->cfg.inj_ppc[2]);
    pic_status s = alloc3<R>(c, capacity_for(c, mx));
    if (s) return s;
  }
  const int q = (int)(c->step & 1);
  k3_bin_place<R><<<blocks, 256, 0, c->stream>>>(g, c->col0, d[0], d[1], d[2], d[3], d[4], d[5],
                                                 d[6], n, soa7<R>(c->seg[q]), c->cnt[q], c->cap,
                                                 &c->st->err);
  CK3(cudaGetLastError());
  CK3(launch_clamp_counts(c->cnt[q], g.nslots, c->cap, c->stream));
  c->launches += 2;
  if (tmp) {
    CK3(cudaStreamSynchronize(c->stream));
    cfree3(c, tmp);
  }
  c->prev_valid = false;
  free_graphs3(c);
  return poll3(c);
}

template <typename R>
pic_status fill3(Ctx3 *c) {
  const Geom3 &g = c->g;
  const pic_config &cf = c->cfg;
  const int full = g.p[0] * g.p[1] * g.p[2] * cf.inj_ppc[0] * cf.inj_ppc[1] * cf.inj_ppc[2];
  pic_status s = alloc3<R>(c, capacity_for(c, full));
  if (s) return s;
  const int q = (int)(c->step & 1);
  k3_inject<R><<<dim3(g.np[1] * g.np[2], g.np[0]), 256, 0, c->stream>>>(
      g, c->col0, 0, c->nshift, soa7<R>(c->seg[q]), c->cnt[q], c->cap, cf.inj_n0, cf.inj_x0,
      cf.inj_ramp, cf.inj_ymin, cf.inj_ppc[0], cf.inj_ppc[1], cf.inj_ppc[2], c->rho_bg,
      &c->st->err);
  CK3(cudaGetLastError());
  c->launches += 1;
  c->prev_valid = false;
  free_graphs3(c);
  return poll3(c);
}

pic_status ensure_staging3(Ctx3 *c, size_t n) {
  if (c->staging_n >= n) return PIC_OK;
  cfree3(c, c->staging);
  c->staging = nullptr;
  CK3(cmalloc3(c, &c->staging, sizeof(double) * n));
  c->staging_n = n;
  return PIC_OK;
}

size_t out_count3(const Geom3 &g) {
  int lo[3], cnt[3];
  out_dims3(g, lo, cnt);
  return (size_t)cnt[0] * cnt[1] * cnt[2];
}

int comp_of3(int which) {
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
pic_status deposit_rho3(Ctx3 *c, double *rho, bool previous) {
  const Geom3 &g = c->g;
  CK3(cudaMemsetAsync(rho, 0, sizeof(double) * g.cs, c->stream));
  if (!c->cap) return PIC_OK;
  const int q = (int)(c->step & 1);
  const int segset = previous ? 1 - q : q, bktset = previous ? q : 1 - q;
  k3_deposit_rho<R><<<g.nslots, 256, 0, c->stream>>>(g, c->col0, view3<R>(c, segset, bktset), rho, 1.0);
  CK3(cudaGetLastError());
  c->launches += 1;
  return PIC_OK;
}

template <typename R>
pic_status get_field3(Ctx3 *c, int which, double *dst, int where) {
  const Geom3 &g = c->g;
  const size_t n = out_count3(g);
  double *d = dst;
  if (where == PIC_HOST) {
    pic_status s = ensure_staging3(c, n);
    if (s) return s;
    d = c->staging;
  }
  const int blocks = (int)std::min<size_t>((n + 255) / 256, 8192);
  if (which == PIC_RHO || which == PIC_RHO_BG) {
    const double *src = c->rho_bg;
    if (which == PIC_RHO) {
      pic_status s = deposit_rho3<R>(c, c->rho_a, false);
      if (s) return s;
      src = c->rho_a;
    }
    k3_get_field<double><<<blocks, 256, 0, c->stream>>>(g, src, d);
  } else {
    int comp = comp_of3(which);
    if (which >= PIC_JX && which <= PIC_JZ)
      comp = C_JA + 3 * (int)((c->step + 1) & 1) + (which - PIC_JX);
    if (comp < 0) return fail3(c, PIC_EINVAL, "bad field id");
    k3_get_field<R><<<blocks, 256, 0, c->stream>>>(g, (const R *)c->F + comp * g.cs, d);
  }
  CK3(cudaGetLastError());
  c->launches += 1;
  if (where == PIC_HOST)
    CK3(cudaMemcpyAsync(dst, d, sizeof(double) * n, cudaMemcpyDeviceToHost, c->stream));
  return poll3(c);
}

template <typename R>
pic_status set_field3(Ctx3 *c, int which, const double *src, int where) {
  const Geom3 &g = c->g;
  const size_t n = out_count3(g);
  const double *d = src;
  if (where == PIC_HOST) {
    pic_status s = ensure_staging3(c, n);
    if (s) return s;
    CK3(cudaMemcpyAsync(c->staging, src, sizeof(double) * n, cudaMemcpyHostToDevice, c->stream));
    d = c->staging;
  }
  const int blocks = (int)std::min<size_t>((n + 255) / 256, 8192);
  if (which == PIC_RHO_BG) {
    k3_set_field<double, double><<<blocks, 256, 0, c->stream>>>(g, c->rho_bg, d, 0);
  } else {
    const int comp = comp_of3(which);
    if (comp < 0) return fail3(c, PIC_EINVAL, "field not settable");
    k3_set_field<R, double><<<blocks, 256, 0, c->stream>>>(g, (R *)c->F + comp * g.cs, d, 1);
  }
  CK3(cudaGetLastError());
  c->launches += 1;
  c->prev_valid = false;
  c->active_valid = false;
  return poll3(c);
}

template <typename R>
pic_status get_particles3(Ctx3 *c, double *out, size_t cap, size_t *n, int where) {
  const Geom3 &g = c->g;
  if (!c->cap) {
    *n = 0;
    return PIC_OK;
  }
  const int q = (int)(c->step & 1);
  std::vector<int> cn(g.nslots), b((size_t)g.nslots * NB3);
  CK3(cudaMemcpyAsync(cn.data(), c->cnt[q], sizeof(int) * g.nslots, cudaMemcpyDeviceToHost, c->stream));
  CK3(cudaMemcpyAsync(b.data(), c->bcnt[1 - q], sizeof(int) * b.size(), cudaMemcpyDeviceToHost, c->stream));
  CK3(cudaStreamSynchronize(c->stream));
  std::vector<long long> off((size_t)g.nslots * (1 + NB3) + 1, 0);
  long long tot = 0;
  for (int pp = 0; pp < g.nslots; ++pp) {
    const int px = pp % g.np[0], py = (pp / g.np[0]) % g.np[1], pz = pp / (g.np[0] * g.np[1]);
    const int slot = slot_of(g, c->col0, px, py, pz);
    off[pp] = tot;
    tot += std::min(cn[slot], c->cap);
  }
  for (int pp = 0; pp < g.nslots; ++pp) {
    const int px = pp % g.np[0], py = (pp / g.np[0]) % g.np[1], pz = pp / (g.np[0] * g.np[1]);
    const int slot = slot_of(g, c->col0, px, py, pz);
    for (int d = 0; d < NB3; ++d) {
      int dx, dy, dz;
      delta26(d, dx, dy, dz);
      off[g.nslots + (size_t)pp * NB3 + d] = tot;
      if (neighbour3(g, c->col0, slot, dx, dy, dz) >= 0)
        tot += std::min(b[(size_t)slot * NB3 + d], c->bk.cap[d]);
    }
  }
  *n = (size_t)tot;
  if (!out) return PIC_OK;
  if ((size_t)tot > cap) return fail3(c, PIC_EINVAL, "output capacity too small");
  CK3(cudaMemcpyAsync(c->offsets, off.data(), sizeof(long long) * off.size(), cudaMemcpyHostToDevice,
                      c->stream));
  double *dst = out, *tmp = nullptr;
  if (where == PIC_HOST) {
    CK3(cmalloc3(c, &tmp, sizeof(double) * 7 * std::max<size_t>(cap, 1)));
    dst = tmp;
  }
  k3_get_particles<R><<<g.nslots, 256, 0, c->stream>>>(g, c->col0, view3<R>(c, q, 1 - q), c->offsets,
                                                       dst, cap);
  CK3(cudaGetLastError());
  c->launches += 1;
  if (tmp) {
    CK3(cudaMemcpyAsync(out, tmp, sizeof(double) * 7 * cap, cudaMemcpyDeviceToHost, c->stream));
    CK3(cudaStreamSynchronize(c->stream));
    cfree3(c, tmp);
  }
  return poll3(c);
}

template <typename R>
pic_status diag3(Ctx3 *c, pic_diag_t *out) {
  const Geom3 &g = c->g;
  memset(out, 0, sizeof *out);
  const int nb = c->npartials;
  std::vector<double> h(3 * nb);
  const double dV = g.d[0] * g.d[1] * g.d[2];
  k3_field_energy<R><<<nb, 256, 0, c->stream>>>(g, (const R *)c->F, c->partials);
  CK3(cudaGetLastError());
  CK3(cudaMemcpyAsync(h.data(), c->partials, sizeof(double) * 2 * nb, cudaMemcpyDeviceToHost, c->stream));
  CK3(cudaStreamSynchronize(c->stream));
  double ue = 0, ub = 0;
  for (int b = 0; b < nb; ++b) {
    ue += h[2 * b];
    ub += h[2 * b + 1];
  }
  out->U_E = 0.5 * ue * dV;
  out->U_B = 0.5 * ub * dV;
  double ek = 0, ws = 0, cnt = 0;
  if (c->cap) {
    const int q = (int)(c->step & 1);
    k3_particle_diag<R><<<nb, 256, 0, c->stream>>>(g, c->col0, view3<R>(c, q, 1 - q), c->partials);
    CK3(cudaGetLastError());
    CK3(cudaMemcpyAsync(h.data(), c->partials, sizeof(double) * 3 * nb, cudaMemcpyDeviceToHost, c->stream));
    CK3(cudaStreamSynchronize(c->stream));
    for (int b = 0; b < nb; ++b) {
      ek += h[3 * b];
      ws += h[3 * b + 1];
      cnt += h[3 * b + 2];
    }
  }
  out->U_K = ek * g.m * dV;
  out->charge = g.q * ws * dV;
  out->np = (long long)llround(cnt);
  pic_status s = deposit_rho3<R>(c, c->rho_a, false);
  if (s) return s;
  const bool cont = c->prev_valid && c->cap;
  if (cont) {
    s = deposit_rho3<R>(c, c->rho_b, true);
    if (s) return s;
  }
  const int jset = (int)((c->step + 1) & 1);
  k3_gauss<R><<<nb, 256, 0, c->stream>>>(g, (const R *)c->F, jset, c->rho_a, cont ? c->rho_b : nullptr,
                                         c->rho_bg, c->partials);
  CK3(cudaGetLastError());
  CK3(cudaMemcpyAsync(h.data(), c->partials, sizeof(double) * 2 * nb, cudaMemcpyDeviceToHost, c->stream));
  DevState hs;
  CK3(cudaMemcpyAsync(&hs, c->st, sizeof hs, cudaMemcpyDeviceToHost, c->stream));
  CK3(cudaStreamSynchronize(c->stream));
  double gm = 0, cm = 0;
  for (int b = 0; b < nb; ++b) {
    gm = std::max(gm, h[2 * b]);
    cm = std::max(cm, h[2 * b + 1]);
  }
  out->gauss = gm;
  out->continuity = cont ? cm : NAN;
  out->step = c->step;
  out->t = c->t;
  out->shifts = c->nshift / window_columns3(c->cfg);
  out->max_patch_count = hs.maxcnt[(c->step + 1) & 1];
  out->capacity = c->cap;
  out->ms_particles = c->ms_particles;
  out->ms_fields = c->ms_fields;
  out->ms_window = c->ms_window;
  c->launches += 5 + (cont ? 1 : 0);
  out->launches = c->launches;
  out->particle_step_launches = c->ps_launches;
  out->grows = c->grows;
  out->calm_particle_steps = 0;  // the 3D step has no calm-slot skip
  return poll3(c);
}

// -------------------------------------- auto-grow replay and snapshots ----

void free_backup3(Ctx3 *c) {
  auto &b = c->bak;
  cfree3(c, b.F);
  cfree3(c, b.rho_bg);
  for (int a = 0; a < 7; ++a) {
    cfree3(c, b.seg[a]);
    cfree3(c, b.bkt[a]);
  }
  cfree3(c, b.cnt);
  cfree3(c, b.bcnt);
  cfree3(c, b.st);
  b = Ctx3::Backup{};
}

// Copy the live state (current particle set and its in-flight buckets, E,
// B, Bm, background charge, device scalars) into the backup; particles are
// copied patch by patch, only the slots each count covers.
template <typename R>
pic_status take_backup3(Ctx3 *c) {
  auto &b = c->bak;
  const Geom3 &g = c->g;
  if (b.cap != c->cap) free_backup3(c);
  if (!b.F) {
    b.cap = c->cap;
    b.bk = c->bk;
    CK3(cmalloc3(c, &b.F, 9 * g.cs * sizeof(R)));
    CK3(cmalloc3(c, &b.rho_bg, g.cs * sizeof(double)));
    for (int a = 0; a < 7; ++a) {
      CK3(cmalloc3(c, &b.seg[a], sizeof(R) * (size_t)g.nslots * b.cap));
      CK3(cmalloc3(c, &b.bkt[a], sizeof(R) * (size_t)g.nslots * b.bk.stride));
    }
    CK3(cmalloc3(c, &b.cnt, sizeof(int) * g.nslots));
    CK3(cmalloc3(c, &b.bcnt, sizeof(int) * (size_t)g.nslots * NB3));
    CK3(cmalloc3(c, &b.st, sizeof(DevState)));
  }
  const int q = (int)(c->step & 1);
  CK3(cudaMemcpyAsync(b.F, c->F, 9 * g.cs * sizeof(R), cudaMemcpyDeviceToDevice, c->stream));
  CK3(cudaMemcpyAsync(b.rho_bg, c->rho_bg, g.cs * sizeof(double), cudaMemcpyDeviceToDevice,
                      c->stream));
  const int blocks = std::min(g.nslots, 65535);
  k3_repack<R><<<blocks, 256, 0, c->stream>>>(g.nslots, soa7<R>(c->seg[q]), c->cnt[q], c->cap,
                                              soa7<R>(c->bkt[1 - q]), c->bcnt[1 - q], c->bk,
                                              soa7<R>(b.seg), b.cnt, b.cap, soa7<R>(b.bkt), b.bcnt,
                                              b.bk);
  CK3(cudaGetLastError());
  CK3(cudaMemcpyAsync(b.st, c->st, sizeof(DevState), cudaMemcpyDeviceToDevice, c->stream));
  b.step = c->step;
  b.t = c->t;
  b.nshift = c->nshift;
  b.col0 = c->col0;
  c->launches += 1;
  return PIC_OK;
}

// Return to the backup with a patch capacity of new_cap (particle storage
// reallocated, bucket layout recomputed, particles repacked); clears the
// device fault.  The current sets restart at zero, as after a load.
template <typename R>
pic_status restore_backup3(Ctx3 *c, int new_cap) {
  auto &b = c->bak;
  const Geom3 &g = c->g;
  CK3(cudaStreamSynchronize(c->stream));
  if (new_cap != c->cap) {
    free_graphs3(c);
    free_particles3(c);
    pic_status s = alloc3<R>(c, new_cap);
    if (s) return s;
  }
  const int q = (int)(b.step & 1);
  CK3(cudaMemcpyAsync(c->F, b.F, 9 * g.cs * sizeof(R), cudaMemcpyDeviceToDevice, c->stream));
  CK3(cudaMemsetAsync((R *)c->F + C_JA * g.cs, 0, 6 * g.cs * sizeof(R), c->stream));
  CK3(cudaMemcpyAsync(c->rho_bg, b.rho_bg, g.cs * sizeof(double), cudaMemcpyDeviceToDevice,
                      c->stream));
  CK3(cudaMemsetAsync(c->cnt[1 - q], 0, sizeof(int) * g.nslots, c->stream));
  CK3(cudaMemsetAsync(c->bcnt[q], 0, sizeof(int) * (size_t)g.nslots * NB3, c->stream));
  const int blocks = std::min(g.nslots, 65535);
  k3_repack<R><<<blocks, 256, 0, c->stream>>>(g.nslots, soa7<R>(b.seg), b.cnt, b.cap,
                                              soa7<R>(b.bkt), b.bcnt, b.bk, soa7<R>(c->seg[q]),
                                              c->cnt[q], c->cap, soa7<R>(c->bkt[1 - q]),
                                              c->bcnt[1 - q], c->bk);
  CK3(cudaGetLastError());
  DevState ds;
  CK3(cudaMemcpyAsync(&ds, b.st, sizeof ds, cudaMemcpyDeviceToHost, c->stream));
  CK3(cudaStreamSynchronize(c->stream));
  ds.err = 0;
  CK3(cudaMemcpy(c->st, &ds, sizeof ds, cudaMemcpyHostToDevice));
  c->step = b.step;
  c->t = b.t;
  c->nshift = b.nshift;
  c->col0 = b.col0;
  c->prev_valid = false;
  c->active_valid = false;
  c->sticky = PIC_OK;
  c->launches += 1;
  return PIC_OK;
}

// Advance nsteps; with auto_grow, an overflow of a patch or bucket capacity
// grows the capacity and replays the steps from the state at entry.
template <typename R>
pic_status step3(Ctx3 *c, int nsteps) {
  if (!c->cfg.auto_grow) return run3<R>(c, nsteps);
  pic_status s = take_backup3<R>(c);
  if (s) return s;
  for (int attempt = 0;; ++attempt) {
    s = run3<R>(c, nsteps);
    if (s != PIC_EOVERFLOW || attempt >= 4) return s;
    DevState h;
    CK3(cudaMemcpy(&h, c->st, sizeof h, cudaMemcpyDeviceToHost));
    const int seen = std::max(h.maxcnt[0], h.maxcnt[1]);
    int cap = std::max((int)(1.5 * c->cap), (int)(1.25 * seen));
    cap = (cap + 31) / 32 * 32;
    s = restore_backup3<R>(c, cap);
    if (s) return s;
    c->grows += 1;
    c->err.clear();
  }
}

// Host snapshot: header, the 15 field components, the background charge,
// both particle sets with their buckets and counts, the device scalars.
struct Snap3Header {
  char magic[8];
  int n[3], p[3];
  int fp32, cap, nshift, col0;
  long long step;
  double t;
  int prev_valid, pad;
  double wmax;
};

// Offsets of one set's packed arrays from its counts (nslots segment counts
// then 26 nslots bucket counts); returns the total.
long long pack_offsets3(const Geom3 &g, int cap, const Buckets26 &bk, const int *cnt,
                        const int *bcnt, std::vector<long long> &off) {
  off.assign((size_t)g.nslots * 27 + 1, 0);
  long long o = 0;
  for (int s = 0; s < g.nslots; ++s) {
    off[27 * (size_t)s] = o;
    o += std::min(std::max(cnt[s], 0), cap);
    for (int d = 0; d < NB3; ++d) {
      off[27 * (size_t)s + 1 + d] = o;
      o += std::min(std::max(bcnt[(size_t)s * NB3 + d], 0), bk.cap[d]);
    }
  }
  off.back() = o;
  return o;
}

template <typename R>
cudaError_t launch_pack3(const Ctx3 *c, int st, bool pack, void *flat, long long total) {
  const int blocks = std::min(c->g.nslots, 65535);
  if (pack)
    k3_pack<R, true><<<blocks, 256, 0, c->stream>>>(c->g.nslots, soa7<R>(c->seg[st]), c->cnt[st],
                                                    c->cap, soa7<R>(c->bkt[st]), c->bcnt[st],
                                                    c->bk, c->offsets, (R *)flat, total);
  else
    k3_pack<R, false><<<blocks, 256, 0, c->stream>>>(c->g.nslots, soa7<R>(c->seg[st]), c->cnt[st],
                                                     c->cap, soa7<R>(c->bkt[st]), c->bcnt[st],
                                                     c->bk, c->offsets, (R *)flat, total);
  return cudaGetLastError();
}

}  // namespace

// --------------------------------------------------------- entry points ----

bool valid_config3(const pic_config *cf, std::string &why) {
  for (int a = 0; a < 3; ++a) {
    if (cf->n[a] <= 0 || cf->patch[a] <= 0) { why = "cells and patch sizes must be positive"; return false; }
    if (cf->patch[a] % 4 || cf->patch[a] > 32) { why = "3D patch sizes must be multiples of 4 up to 32"; return false; }
    if (cf->n[a] % cf->patch[a]) { why = "cells must be a multiple of the patch size"; return false; }
    if (!(cf->d[a] > 0)) { why = "cell sizes must be positive"; return false; }
    if (cf->bc_field[a] != PIC_BC_PERIODIC && cf->bc_field[a] != PIC_BC_SILVER_MULLER) { why = "bad field boundary"; return false; }
    if (cf->bc_field[a] == PIC_BC_PERIODIC && cf->n[a] < 2 * G3) { why = "periodic axes need at least 8 cells"; return false; }
    for (int f = 0; f < 2; ++f) {
      const int b = cf->bc_part[a][f];
      if (b < 0 || b > 2) { why = "bad particle boundary"; return false; }
      if ((b == PIC_PBC_PERIODIC) != (cf->bc_field[a] == PIC_BC_PERIODIC)) { why = "periodic particle and field boundaries must pair"; return false; }
    }
  }
  double s = 0.0;
  for (int a = 0; a < 3; ++a) s += 1.0 / (cf->d[a] * cf->d[a]);
  if (!(cf->dt > 0) || !(cf->dt * std::sqrt(s) < 1.0)) { why = "dt must satisfy the 3D Courant condition"; return false; }
  if (cf->filter_passes != 0) { why = "the current filter is a 2D option"; return false; }
  if (cf->moving_window && cf->inj_ppc[2] < 1) { why = "injected particles per cell must be >= 1"; return false; }
  const size_t rs = cf->prec == PIC_FP32 ? 4 : 8;
  if (tile_bytes(cf, rs) > 227 * 1024) { why = "patch current tile exceeds shared memory"; return false; }
  return true;
}

size_t footprint3(const pic_config *cf, size_t np_max) {
  const Geom3 g = make_geom3(cf);
  const size_t rs = cf->prec == PIC_FP32 ? 4 : 8;
  const double cfac = cf->capacity_factor > 0 ? cf->capacity_factor : 2.0;
  const int cmin = cf->capacity_min > 0 ? cf->capacity_min : 256;
  size_t per = (np_max + g.nslots - 1) / g.nslots;
  if (cf->moving_window)
    per = std::max(per, (size_t)g.p[0] * g.p[1] * g.p[2] * cf->inj_ppc[0] * cf->inj_ppc[1] * cf->inj_ppc[2]);
  int cap = std::max(cmin, (int)std::ceil(cfac * (double)per));
  cap = (cap + 31) / 32 * 32;
  return (size_t)NCOMP * g.cs * rs + 3 * sizeof(double) * g.cs + particle_bytes3(g, cap, rs) +
         sizeof(long long) * ((size_t)g.nslots * (1 + NB3) + 1) + sizeof(double) * 3 * 1024 +
         sizeof(DevState);
}

pic_status c3_create(const pic_config *cfg, cudaStream_t stream, Ctx3 **out, std::string &err) {
  *out = nullptr;
  Ctx3 *c = new (std::nothrow) Ctx3();
  if (!c) return PIC_ENOMEM;
  c->cfg = *cfg;
  c->g = make_geom3(cfg);
  {
    // weights the injection (window, pic_load_plasma) can create
    const int ppc = cfg->inj_ppc[0] * cfg->inj_ppc[1] * cfg->inj_ppc[2];
    if (ppc > 0 && std::isfinite(cfg->inj_n0)) c->wmax = std::fabs(cfg->inj_n0) / ppc;
  }
  c->fp32 = cfg->prec == PIC_FP32;
  c->rs = c->fp32 ? 4 : 8;
  c->stream = stream;
  const Geom3 &g = c->g;
  auto bail = [&](pic_status s) {
    err = c->err.empty() ? "device allocation failed" : c->err;
    c3_destroy(c);
    return s;
  };
  if (cmalloc3(c, &c->F, (size_t)NCOMP * g.cs * c->rs) != cudaSuccess) return bail(PIC_ENOMEM);
  for (double **p : {&c->rho_bg, &c->rho_a, &c->rho_b})
    if (cmalloc3(c, p, sizeof(double) * g.cs) != cudaSuccess) return bail(PIC_ENOMEM);
  if (cmalloc3(c, &c->st, sizeof(DevState)) != cudaSuccess) return bail(PIC_ENOMEM);
  if (cmalloc3(c, &c->active, sizeof(int) * g.nslots) != cudaSuccess) return bail(PIC_ENOMEM);
  if (cmalloc3(c, &c->plan_hist, sizeof(int) * 2 * PLAN3_CLASSES) != cudaSuccess) return bail(PIC_ENOMEM);
  if (cmalloc3(c, &c->partials, sizeof(double) * 3 * c->npartials) != cudaSuccess) return bail(PIC_ENOMEM);
  if (cfg->laser_on) {
    std::vector<double> prof((size_t)(g.n[2] + 1) * g.n[1]);
    for (int k = 0; k <= g.n[2]; ++k)
      for (int j = 0; j < g.n[1]; ++j) {
        const double ry = ((j + 0.5) * g.d[1] - cfg->laser_y_center) / cfg->laser_waist;
        const double rz = (k * g.d[2] - cfg->laser_z_center) / cfg->laser_waist;
        prof[(size_t)k * g.n[1] + j] = cfg->laser_a0 * std::exp(-(ry * ry + rz * rz));
      }
    if (cmalloc3(c, &c->laser_g, sizeof(double) * prof.size()) != cudaSuccess) return bail(PIC_ENOMEM);
    if (cudaMemcpy(c->laser_g, prof.data(), sizeof(double) * prof.size(), cudaMemcpyHostToDevice) !=
        cudaSuccess)
      return bail(PIC_ECUDA);
  }
  if (cudaMemsetAsync(c->F, 0, (size_t)NCOMP * g.cs * c->rs, stream) != cudaSuccess ||
      cudaMemsetAsync(c->rho_bg, 0, sizeof(double) * g.cs, stream) != cudaSuccess ||
      cudaMemsetAsync(c->st, 0, sizeof(DevState), stream) != cudaSuccess ||
      cudaStreamSynchronize(stream) != cudaSuccess)
    return bail(PIC_ECUDA);
  *out = c;
  return PIC_OK;
}

void c3_destroy(Ctx3 *c) {
  if (!c) return;
  if (c->stream) cudaStreamSynchronize(c->stream);
  free_graphs3(c);
  cfree3(c, c->F);
  cfree3(c, c->rho_bg);
  cfree3(c, c->rho_a);
  cfree3(c, c->rho_b);
  cfree3(c, c->laser_g);
  cfree3(c, c->st);
  cfree3(c, c->active);
  cfree3(c, c->plan_hist);
  cfree3(c, c->partials);
  cfree3(c, c->staging);
  free_backup3(c);
  free_particles3(c);
  delete c;
}

const char *c3_error(const Ctx3 *c) { return c ? c->err.c_str() : "no context"; }

static pic_status usable3(Ctx3 *c) {
  if (c->sticky != PIC_OK) return fail3(c, PIC_ESTATE, "context holds a device fault");
  return PIC_OK;
}

pic_status c3_load(Ctx3 *c, const double *x, const double *y, const double *z, const double *ux,
                   const double *uy, const double *uz, const double *w, size_t n, int where) {
  pic_status s = usable3(c);
  if (s) return s;
  const double *src[7] = {x, y, z, ux, uy, uz, w};
  return c->fp32 ? load3<float>(c, src, n, where) : load3<double>(c, src, n, where);
}

pic_status c3_fill_plasma(Ctx3 *c) {
  pic_status s = usable3(c);
  if (s) return s;
  if (c->cap) return fail3(c, PIC_ESTATE, "particles are already loaded");
  for (int a = 0; a < 3; ++a)
    if (c->cfg.inj_ppc[a] < 1) return fail3(c, PIC_EINVAL, "plasma needs inj_ppc >= 1 on every axis");
  return c->fp32 ? fill3<float>(c) : fill3<double>(c);
}

pic_status c3_set_field(Ctx3 *c, int which, const double *src, int where) {
  pic_status s = usable3(c);
  if (s) return s;
  return c->fp32 ? set_field3<float>(c, which, src, where) : set_field3<double>(c, which, src, where);
}

pic_status c3_get_field(Ctx3 *c, int which, double *dst, int where) {
  pic_status s = usable3(c);
  if (s) return s;
  return c->fp32 ? get_field3<float>(c, which, dst, where) : get_field3<double>(c, which, dst, where);
}

pic_status c3_set_background(Ctx3 *c, int mode, double value) {
  pic_status s = usable3(c);
  if (s) return s;
  const Geom3 &g = c->g;
  if (mode == PIC_BG_NONE) {
    CK3(cudaMemsetAsync(c->rho_bg, 0, sizeof(double) * g.cs, c->stream));
  } else if (mode == PIC_BG_UNIFORM) {
    std::vector<double> h((size_t)g.cs, value);
    CK3(cudaMemcpyAsync(c->rho_bg, h.data(), sizeof(double) * g.cs, cudaMemcpyHostToDevice, c->stream));
    CK3(cudaStreamSynchronize(c->stream));
  } else if (mode == PIC_BG_NEUTRALISING) {
    CK3(cudaMemsetAsync(c->rho_bg, 0, sizeof(double) * g.cs, c->stream));
    if (c->cap) {
      const int q = (int)(c->step & 1);
      if (c->fp32)
        k3_deposit_rho<float><<<g.nslots, 256, 0, c->stream>>>(g, c->col0, view3<float>(c, q, 1 - q), c->rho_bg, -1.0);
      else
        k3_deposit_rho<double><<<g.nslots, 256, 0, c->stream>>>(g, c->col0, view3<double>(c, q, 1 - q), c->rho_bg, -1.0);
      CK3(cudaGetLastError());
      c->launches += 1;
    }
  } else {
    return fail3(c, PIC_EINVAL, "bad background mode");
  }
  return poll3(c);
}

pic_status c3_init_fields(Ctx3 *c, int mode) {
  pic_status s = usable3(c);
  if (s) return s;
  const Geom3 &g = c->g;
  CK3(cudaStreamSynchronize(c->stream));
  CK3(cudaMemsetAsync(c->F, 0, 9 * g.cs * c->rs, c->stream));  // E, Bm, B
  c->prev_valid = false;
  c->active_valid = false;
  if (mode == PIC_INIT_ZERO) return poll3(c);
  for (int a = 0; a < 3; ++a)
    if (g.fbc[a] != FBC_PERIODIC) return fail3(c, PIC_EINVAL, "the Poisson start needs periodic axes");
  const size_t n = (size_t)g.n[0] * g.n[1] * g.n[2];
  double *buf = nullptr;
  CK3(cmalloc3(c, &buf, sizeof(double) * 5 * n));
  double *rho = buf, *bg = buf + n, *ex = buf + 2 * n, *ey = buf + 3 * n, *ez = buf + 4 * n;
  s = c->fp32 ? deposit_rho3<float>(c, c->rho_a, false) : deposit_rho3<double>(c, c->rho_a, false);
  if (s) { cfree3(c, buf); return s; }
  const int blocks = (int)std::min<size_t>((n + 255) / 256, 8192);
  k3_get_field<double><<<blocks, 256, 0, c->stream>>>(g, c->rho_a, rho);
  k3_get_field<double><<<blocks, 256, 0, c->stream>>>(g, c->rho_bg, bg);
  CK3(cudaGetLastError());
  CK3(launch_axpy_f64(rho, bg, n, c->stream));
  const double dd[3] = {g.d[0], g.d[1], g.d[2]};
  s = poisson_fields(c->cfg, 3, g.n, dd, rho, ex, ey, ez, c->stream, c->err);
  if (!s) {
    const double *src[3] = {ex, ey, ez};
    for (int k = 0; k < 3 && !s; ++k)
      s = c->fp32 ? set_field3<float>(c, PIC_EX + k, src[k], PIC_DEVICE)
                  : set_field3<double>(c, PIC_EX + k, src[k], PIC_DEVICE);
  }
  cudaStreamSynchronize(c->stream);
  cfree3(c, buf);
  c->launches += 6;
  if (s) return s;
  return poll3(c);
}

pic_status c3_step(Ctx3 *c, int nsteps) {
  pic_status s = usable3(c);
  if (s) return s;
  if (!c->cap) return fail3(c, PIC_ESTATE, "no particles loaded");
  return c->fp32 ? step3<float>(c, nsteps) : step3<double>(c, nsteps);
}

pic_status c3_get_particles(Ctx3 *c, double *out, size_t cap, size_t *n, int where) {
  pic_status s = usable3(c);
  if (s) return s;
  return c->fp32 ? get_particles3<float>(c, out, cap, n, where)
                 : get_particles3<double>(c, out, cap, n, where);
}

pic_status c3_diag(Ctx3 *c, pic_diag_t *out) {
  pic_status s = usable3(c);
  if (s) return s;
  return c->fp32 ? diag3<float>(c, out) : diag3<double>(c, out);
}

pic_status c3_sync(Ctx3 *c) {
  pic_status s = usable3(c);
  if (s) return s;
  return poll3(c);
}

// Snapshot layout (3D): Snap3Header, the 15 field components, the
// background charge, the device scalars, then for each particle set st = 0,
// 1 (segments seg[st] with buckets bkt[st], counts cnt[st], bcnt[st]): its
// 27 nslots counts and its live particles packed into seven arrays, slot by
// slot (capacity slack not stored).
pic_status c3_snapshot(Ctx3 *c, void *host, size_t *bytes) {
  CK3(cudaStreamSynchronize(c->stream));
  const Geom3 &g = c->g;
  std::vector<int> counts[2];
  std::vector<long long> off[2];
  long long total[2] = {0, 0};
  size_t need = sizeof(Snap3Header) + (size_t)NCOMP * g.cs * c->rs + sizeof(double) * g.cs +
                sizeof(DevState);
  if (c->cap) {
    for (int st = 0; st < 2; ++st) {
      counts[st].resize((size_t)g.nslots * 27);
      CK3(cudaMemcpy(counts[st].data(), c->cnt[st], sizeof(int) * g.nslots, cudaMemcpyDeviceToHost));
      CK3(cudaMemcpy(counts[st].data() + g.nslots, c->bcnt[st], sizeof(int) * (size_t)g.nslots * NB3,
                     cudaMemcpyDeviceToHost));
      total[st] = pack_offsets3(g, c->cap, c->bk, counts[st].data(), counts[st].data() + g.nslots,
                                off[st]);
      need += sizeof(int) * (size_t)g.nslots * 27 + 7 * c->rs * (size_t)total[st];
    }
  }
  if (!host) {
    *bytes = need;
    return PIC_OK;
  }
  if (*bytes < need) return fail3(c, PIC_EINVAL, "snapshot buffer too small");
  char *p = (char *)host;
  Snap3Header h{};
  memcpy(h.magic, "PICSNAP5", 8);
  for (int a = 0; a < 3; ++a) {
    h.n[a] = g.n[a];
    h.p[a] = g.p[a];
  }
  h.fp32 = c->fp32; h.cap = c->cap; h.nshift = c->nshift; h.col0 = c->col0;
  h.step = c->step; h.t = c->t; h.prev_valid = c->prev_valid; h.wmax = c->wmax;
  memcpy(p, &h, sizeof h);
  p += sizeof h;
  auto d2h = [&](const void *src, size_t n) -> cudaError_t {
    cudaError_t e = cudaMemcpy(p, src, n, cudaMemcpyDeviceToHost);
    p += n;
    return e;
  };
  CK3(d2h(c->F, (size_t)NCOMP * g.cs * c->rs));
  CK3(d2h(c->rho_bg, sizeof(double) * g.cs));
  CK3(d2h(c->st, sizeof(DevState)));
  if (c->cap) {
    void *flat = nullptr;
    const long long most = std::max(total[0], total[1]);
    if (most > 0) CK3(cmalloc3(c, &flat, 7 * c->rs * (size_t)most));
    cudaError_t e = cudaSuccess;
    for (int st = 0; st < 2 && e == cudaSuccess; ++st) {
      memcpy(p, counts[st].data(), sizeof(int) * counts[st].size());
      p += sizeof(int) * counts[st].size();
      if (total[st] == 0) continue;
      e = cudaMemcpy(c->offsets, off[st].data(), sizeof(long long) * off[st].size(),
                     cudaMemcpyHostToDevice);
      if (e == cudaSuccess)
        e = c->fp32 ? launch_pack3<float>(c, st, true, flat, total[st])
                    : launch_pack3<double>(c, st, true, flat, total[st]);
      if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
      if (e == cudaSuccess) e = d2h(flat, 7 * c->rs * (size_t)total[st]);
      c->launches += 1;
    }
    if (flat) {
      cudaStreamSynchronize(c->stream);
      cfree3(c, flat);
    }
    if (e != cudaSuccess) return fail3(c, PIC_ECUDA, std::string("snapshot: ") + cudaGetErrorString(e));
  }
  *bytes = need;
  return PIC_OK;
}

pic_status c3_restore(Ctx3 *c, const void *host, size_t bytes) {
  Snap3Header h;
  if (bytes < sizeof h) return fail3(c, PIC_EINVAL, "snapshot too small");
  memcpy(&h, host, sizeof h);
  const Geom3 &g = c->g;
  bool same = !memcmp(h.magic, "PICSNAP5", 8) && h.fp32 == (int)c->fp32;
  for (int a = 0; a < 3; ++a) same = same && h.n[a] == g.n[a] && h.p[a] == g.p[a];
  if (!same) return fail3(c, PIC_EINVAL, "snapshot does not match this configuration");
  if (h.cap < 0 || (h.cap % 32)) return fail3(c, PIC_EINVAL, "snapshot capacity is invalid");
  if (h.cap != c->cap && c->cap)
    return fail3(c, PIC_EINVAL, "snapshot capacity differs from this context's");
  // walk the layout on the host first: sizes and counts are checked before
  // anything of the context changes
  const size_t head = sizeof h + (size_t)NCOMP * g.cs * c->rs + sizeof(double) * g.cs +
                      sizeof(DevState);
  if (bytes < head) return fail3(c, PIC_EINVAL, "snapshot truncated");
  const Buckets26 bk = layout26(h.cap);
  const char *sets[2] = {nullptr, nullptr};
  std::vector<long long> off[2];
  long long total[2] = {0, 0};
  size_t pos = head;
  if (h.cap) {
    for (int st = 0; st < 2; ++st) {
      const size_t cb = sizeof(int) * (size_t)g.nslots * 27;
      if (bytes < pos + cb) return fail3(c, PIC_EINVAL, "snapshot truncated");
      sets[st] = (const char *)host + pos;
      const int *cn = reinterpret_cast<const int *>(sets[st]);
      for (size_t k = 0; k < (size_t)g.nslots * 27; ++k) {
        const int lim = k < (size_t)g.nslots ? h.cap : bk.cap[(k - g.nslots) % NB3];
        if (cn[k] < 0 || cn[k] > lim) return fail3(c, PIC_EINVAL, "snapshot counts are invalid");
      }
      total[st] = pack_offsets3(g, h.cap, bk, cn, cn + g.nslots, off[st]);
      pos += cb + 7 * c->rs * (size_t)total[st];
      if (bytes < pos) return fail3(c, PIC_EINVAL, "snapshot truncated");
    }
  }
  CK3(cudaStreamSynchronize(c->stream));
  if (h.cap != c->cap) {  // a context without particle storage takes the snapshot's
    free_graphs3(c);
    if (h.cap) {
      const pic_status s = c->fp32 ? alloc3<float>(c, h.cap) : alloc3<double>(c, h.cap);
      if (s) return s;
    }
  }
  if (h.wmax != c->wmax) free_graphs3(c);  // the current scale is baked into captured steps
  c->wmax = h.wmax;
  const char *p = (const char *)host + sizeof h;
  auto h2d = [&](void *dst, size_t n) -> cudaError_t {
    cudaError_t e = cudaMemcpy(dst, p, n, cudaMemcpyHostToDevice);
    p += n;
    return e;
  };
  CK3(h2d(c->F, (size_t)NCOMP * g.cs * c->rs));
  CK3(h2d(c->rho_bg, sizeof(double) * g.cs));
  DevState ds;
  memcpy(&ds, p, sizeof ds);
  ds.err = 0;
  CK3(cudaMemcpy(c->st, &ds, sizeof ds, cudaMemcpyHostToDevice));
  if (h.cap) {
    void *flat = nullptr;
    const long long most = std::max(total[0], total[1]);
    if (most > 0) CK3(cmalloc3(c, &flat, 7 * c->rs * (size_t)most));
    cudaError_t e = cudaSuccess;
    for (int st = 0; st < 2 && e == cudaSuccess; ++st) {
      const char *cn = sets[st];
      e = cudaMemcpy(c->cnt[st], cn, sizeof(int) * g.nslots, cudaMemcpyHostToDevice);
      if (e == cudaSuccess)
        e = cudaMemcpy(c->bcnt[st], cn + sizeof(int) * g.nslots, sizeof(int) * (size_t)g.nslots * NB3,
                       cudaMemcpyHostToDevice);
      if (e == cudaSuccess && total[st] > 0) {
        e = cudaMemcpy(flat, cn + sizeof(int) * (size_t)g.nslots * 27, 7 * c->rs * (size_t)total[st],
                       cudaMemcpyHostToDevice);
        if (e == cudaSuccess)
          e = cudaMemcpy(c->offsets, off[st].data(), sizeof(long long) * off[st].size(),
                         cudaMemcpyHostToDevice);
        if (e == cudaSuccess)
          e = c->fp32 ? launch_pack3<float>(c, st, false, flat, total[st])
                      : launch_pack3<double>(c, st, false, flat, total[st]);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        c->launches += 1;
      }
    }
    if (flat) {
      cudaStreamSynchronize(c->stream);
      cfree3(c, flat);
    }
    if (e != cudaSuccess) return fail3(c, PIC_ECUDA, std::string("restore: ") + cudaGetErrorString(e));
  }
  c->step = h.step;
  c->t = h.t;
  c->nshift = h.nshift;
  c->col0 = h.col0;
  c->prev_valid = h.prev_valid != 0;
  c->active_valid = false;
  c->sticky = PIC_OK;
  c->err.clear();
  return PIC_OK;
}

}  // namespace pic
