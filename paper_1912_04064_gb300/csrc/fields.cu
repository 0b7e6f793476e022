// Region (coarse decomposition) field kernels: the Yee FDTD update of the
// single domain (Section 3.2), the Silver-Mueller open boundaries with laser
// injection, the moving-window shift and field I/O / diagnostics.
//
//   E^{n+1}   = E^n + dt (curl_h B^{n+1/2} - J^{n+1/2})        k_update_E
//   B^{n+3/2} = B^{n+1/2} - dt curl_h E^{n+1},
//   Bm^{n+1}  = (B^{n+1/2} + B^{n+3/2}) / 2, clear next J      k_update_B
//   ghost B on open faces from the discrete Silver-Mueller condition
//   (E_t -/+ n x B_t = 2 E_inc, centred at the half step and combined with
//   Ampere's law on the boundary node)                          k_silver_mueller
//
// Update ranges per axis: periodic axes update [0, n); open axes update the
// primal nodes [0, n] and the dual points [0, n-1].
#include "common.cuh"

namespace pic {

namespace {

struct Ranges {
  int nxp, nxd, nyp, nyd;
};
__device__ __forceinline__ Ranges ranges(const Geom &g) {
  Ranges r;
  r.nxd = g.nx;
  r.nyd = g.ny;
  r.nxp = g.nx + (g.fbc_x == FBC_SM);
  r.nyp = g.ny + (g.fbc_y == FBC_SM);
  return r;
}

constexpr int YBX = 32, YBY = 8;  // Yee block: 32 x 8 cells, one cell per thread

// True when any cell of the block's tile lies in a periodic mirror band.
__device__ __forceinline__ bool block_mirrors(const Geom &g, int i0, int i1, int j0, int j1) {
  return (g.fbc_x == FBC_PERIODIC && (i0 < GX || i1 > g.nx - GX)) ||
         (g.fbc_y == FBC_PERIODIC && (j0 < GY || j1 > g.ny - GY));
}

// E^{n+1} = E^n + dt (curl_h B^{n+1/2} - J^{n+1/2}); one cell per thread so
// that every thread issues its loads at once.
// Laser temporal factor envelope(t) carrier(t) at t_{n+3/2}, retarded by the
// window's displacement; evaluated once per step by one thread of the E
// update (FP64, off the Silver-Mueller kernel's path) into the device state.
template <typename R>
__device__ __forceinline__ void laser_factor(const FieldArgs<R> &a) {
  const Geom &g = a.g;
  double h = 0.0;
  if (a.laser_on) {
    const double t = a.st->t[a.parity] + 1.5 * g.dt;
    const double tr = t - (double)(a.st->nshift * g.P) * g.dx - a.t_peak;
    h = exp(-2.0 * log(2.0) * tr * tr / (a.tau * a.tau)) * sin(tr);
  }
  a.st->laser_h = h;
}

template <typename R>
__device__ __forceinline__ void update_E(const FieldArgs<R> &a, int blk_x, int blk_y) {
  const Geom &g = a.g;
  if (blk_x == 0 && blk_y == 0 && threadIdx.x == 0 && threadIdx.y == 0) laser_factor(a);
  const Ranges rg = ranges(g);
  const int i0 = blk_x * YBX, j0 = blk_y * YBY;
  const int i = i0 + threadIdx.x, j = j0 + threadIdx.y;
  const bool mir = block_mirrors(g, i0, i0 + YBX, j0, j0 + YBY);
  if (i >= rg.nxp || j >= rg.nyp) return;
  const long long cs = g.cs;
  const int sx = g.sx;
  R *F = a.F;
  R *Ex = F + C_EX * cs, *Ey = F + C_EY * cs, *Ez = F + C_EZ * cs;
  const R *Bx = F + C_BX * cs, *By = F + C_BY * cs, *Bz = F + C_BZ * cs;
  const R *J = F + (C_JA + 3 * (a.filter_passes > 0 ? 1 - a.parity : a.parity)) * cs;
  const R dt = a.dt, idx = a.idx, idy = a.idy;
  const long long o = (long long)(j + GY) * sx + (i + GX);
  {
    // checked build: the cell and its lower neighbours inside the arrays
    unsigned err = 0;
    if (!PIC_IN(err, o >= sx && o < cs)) {
      atomicOr(&a.st->err, err);
      return;
    }
  }
  const R bz = Bz[o], bzl = Bz[o - 1], bzd = Bz[o - sx];
  const R by = By[o], byl = By[o - 1];
  const R bx = Bx[o], bxd = Bx[o - sx];
  const R jx = J[o], jy = J[cs + o], jz = J[2 * cs + o];
  const R ex = Ex[o], ey = Ey[o], ez = Ez[o];
  if (i < rg.nxd) {
    const R v = ex + dt * ((bz - bzd) * idy - jx);
    Ex[o] = v;
    if (mir) mirror(g, Ex, o, i, j, v);
  }
  if (j < rg.nyd) {
    const R v = ey + dt * (-(bz - bzl) * idx - jy);
    Ey[o] = v;
    if (mir) mirror(g, Ey, o, i, j, v);
  }
  {
    const R v = ez + dt * ((by - byl) * idx - (bx - bxd) * idy - jz);
    Ez[o] = v;
    if (mir) mirror(g, Ez, o, i, j, v);
  }
}

// B^{n+3/2} = B^{n+1/2} - dt curl_h E^{n+1}, Bm^{n+1} = (B^{n+1/2} +
// B^{n+3/2}) / 2 (= B at stored cells that are not updated), and the
// current set of the next step cleared.  Covers every stored column and row.
template <typename R>
__device__ __forceinline__ void update_B(const FieldArgs<R> &a, int blk_x, int blk_y) {
  const Geom &g = a.g;
  if (blk_x == 0 && blk_y == 0 && threadIdx.x == 0 && threadIdx.y == 0) {
    const int p = a.parity;
    a.st->t[1 - p] = a.st->t[p] + g.dt;
    a.st->step[1 - p] = a.st->step[p] + 1;
    a.st->maxcnt[1 - p] = 0;  // the next particle step starts a new maximum
  }
  const Ranges rg = ranges(g);
  const int i0 = blk_x * YBX - GX, j0 = blk_y * YBY - GY;
  const int i = i0 + threadIdx.x, j = j0 + threadIdx.y;
  const bool mir = block_mirrors(g, i0, i0 + YBX, j0, j0 + YBY);
  if (i >= g.nx + GX || j >= g.ny + GY) return;
  const long long cs = g.cs;
  const int sx = g.sx;
  R *F = a.F;
  const long long o = (long long)(j + GY) * sx + (i + GX);
  R *Jn = F + (C_JA + 3 * (1 - a.parity)) * cs;
  Jn[o] = R(0);
  Jn[cs + o] = R(0);
  Jn[2 * cs + o] = R(0);
  if ((g.fbc_x == FBC_PERIODIC && (i < 0 || i >= g.nx)) ||
      (g.fbc_y == FBC_PERIODIC && (j < 0 || j >= g.ny)))
    return;  // mirror cell: written by its owner
  const R *Ex = F + C_EX * cs, *Ey = F + C_EY * cs, *Ez = F + C_EZ * cs;
  R *Bx = F + C_BX * cs, *By = F + C_BY * cs, *Bz = F + C_BZ * cs;
  R *Bmx = F + C_BMX * cs, *Bmy = F + C_BMY * cs, *Bmz = F + C_BMZ * cs;
  const R dt = a.dt, idx = a.idx, idy = a.idy;
  const bool in = i >= 0 && j >= 0;
  const bool ux = in && i < rg.nxp && j < rg.nyd;
  const bool uy = in && i < rg.nxd && j < rg.nyp;
  const bool uz = in && i < rg.nxd && j < rg.nyd;
  {
    // checked build: the cell, and its upper neighbours where read, inside
    // the arrays
    unsigned err = 0;
    if (!PIC_IN(err, o >= 0 && o < cs && (!(ux || uy || uz) || o + sx + 1 < cs))) {
      atomicOr(&a.st->err, err);
      return;
    }
  }
  const R bx0 = Bx[o], by0 = By[o], bz0 = Bz[o];
  R ez = R(0), ezu = R(0), ezr = R(0), ey = R(0), eyr = R(0), ex = R(0), exu = R(0);
  if (ux || uy) ez = Ez[o];
  if (ux) ezu = Ez[o + sx];
  if (uy) ezr = Ez[o + 1];
  if (uz) {
    ey = Ey[o];
    eyr = Ey[o + 1];
    ex = Ex[o];
    exu = Ex[o + sx];
  }
  {
    R b1 = bx0;
    if (ux) {
      b1 = bx0 - dt * (ezu - ez) * idy;
      Bx[o] = b1;
      if (mir) mirror(g, Bx, o, i, j, b1);
    }
    const R m = R(0.5) * (bx0 + b1);
    Bmx[o] = m;
    if (mir) mirror(g, Bmx, o, i, j, m);
  }
  {
    R b1 = by0;
    if (uy) {
      b1 = by0 + dt * (ezr - ez) * idx;
      By[o] = b1;
      if (mir) mirror(g, By, o, i, j, b1);
    }
    const R m = R(0.5) * (by0 + b1);
    Bmy[o] = m;
    if (mir) mirror(g, Bmy, o, i, j, m);
  }
  {
    R b1 = bz0;
    if (uz) {
      b1 = bz0 - dt * ((eyr - ey) * idx - (exu - ex) * idy);
      Bz[o] = b1;
      if (mir) mirror(g, Bz, o, i, j, b1);
    }
    const R m = R(0.5) * (bz0 + b1);
    Bmz[o] = m;
    if (mir) mirror(g, Bmz, o, i, j, m);
  }
}

// Ghost B on open faces from the discrete Silver-Mueller condition; the
// coefficients 1/(1+r), 1-r and the transverse dt/d are precomputed.  The
// laser Ey_inc(y, t) = profile(y) * envelope(t) carrier(t): the transverse
// profile is a precomputed array, the temporal factor comes from the device
// state (set by the E update of this step).  One thread
// per face point, faces in parallel (face = 0 x_min, 1 x_max, 2 y_min,
// 3 y_max): no face reads a value another face writes, and every load is
// issued before the ghost stores.
template <typename R>
__device__ __forceinline__ void silver_mueller(const FieldArgs<R> &a, int bx, int face) {
  const Geom &g = a.g;
  const bool xface = face < 2, upper = (face & 1) != 0;
  if (xface ? g.fbc_x != FBC_SM : g.fbc_y != FBC_SM) return;
  const double s_h = face == 0 ? a.st->laser_h : 0.0;
  const int t = bx * blockDim.x + threadIdx.x;
  R *F = a.F;
  const long long cs = g.cs;
  const R *Ex = F + C_EX * cs, *Ey = F + C_EY * cs, *Ez = F + C_EZ * cs;
  R *Bx = F + C_BX * cs, *By = F + C_BY * cs, *Bz = F + C_BZ * cs;
  R *Bmx = F + C_BMX * cs, *Bmy = F + C_BMY * cs, *Bmz = F + C_BMZ * cs;
  const Ranges rg = ranges(g);
  if (xface) {
    if (t >= rg.nyp) return;
    const int j = t, nx = g.nx;
    const int ib = upper ? nx : 0, in = upper ? nx - 1 : 0, gh = upper ? nx : -1;
    const R ia = a.smx_inv1pr, b = a.smx_1mr, c = a.smx_dtt;
    const bool inter = g.fbc_y == FBC_PERIODIC || (j >= 1 && j <= g.ny - 1);
    const bool hasz = j < rg.nyd;
    const R dBx = inter ? Bx[fidx(g, ib, j)] - Bx[fidx(g, ib, j - 1)] : R(0);
    const R ez = Ez[fidx(g, ib, j)], byi = By[fidx(g, in, j)];
    const R ey = hasz ? Ey[fidx(g, ib, j)] : R(0), bzi = hasz ? Bz[fidx(g, in, j)] : R(0);
    const long long og = fidx(g, gh, j);
    {
      unsigned err = 0;  // checked build: ghost and boundary nodes inside the arrays
      if (!PIC_IN(err, og >= 0 && og < cs && fidx(g, ib, j) < cs && fidx(g, ib, j - 1) >= 0)) {
        atomicOr(&a.st->err, err);
        return;
      }
    }
    const R by_old = Bmy[og], bz_old = hasz ? Bmz[og] : R(0);
    R by, bz;
    if (!upper) {
      const R eyinc = (a.laser_on && hasz) ? R(a.laser_g[j] * s_h) : R(0);
      by = (R(2) * ez - b * byi - c * dBx) * ia;
      bz = (R(4) * eyinc - R(2) * ey - b * bzi) * ia;
    } else {
      by = (R(-2) * ez - b * byi + c * dBx) * ia;
      bz = (R(2) * ey - b * bzi) * ia;
    }
    By[og] = by;
    mirror(g, By, og, gh, j, by);
    const R mby = R(0.5) * (by_old + by);
    Bmy[og] = mby;
    mirror(g, Bmy, og, gh, j, mby);
    if (hasz) {
      Bz[og] = bz;
      mirror(g, Bz, og, gh, j, bz);
      const R mbz = R(0.5) * (bz_old + bz);
      Bmz[og] = mbz;
      mirror(g, Bmz, og, gh, j, mbz);
    }
  } else {
    if (t >= rg.nxp) return;
    const int i = t, ny = g.ny;
    const int jb = upper ? ny : 0, jn = upper ? ny - 1 : 0, gh = upper ? ny : -1;
    const R ia = a.smy_inv1pr, b = a.smy_1mr, c = a.smy_dtt;
    const bool inter = g.fbc_x == FBC_PERIODIC || (i >= 1 && i <= g.nx - 1);
    const bool hasz = i < rg.nxd;
    const R dBy = inter ? By[fidx(g, i, jb)] - By[fidx(g, i - 1, jb)] : R(0);
    const R ez = Ez[fidx(g, i, jb)], bxi = Bx[fidx(g, i, jn)];
    const R ex = hasz ? Ex[fidx(g, i, jb)] : R(0), bzi = hasz ? Bz[fidx(g, i, jn)] : R(0);
    const long long og = fidx(g, i, gh);
    {
      unsigned err = 0;  // checked build: ghost and boundary nodes inside the arrays
      if (!PIC_IN(err, og >= 0 && og < cs && fidx(g, i, jb) < cs && fidx(g, i - 1, jb) >= 0)) {
        atomicOr(&a.st->err, err);
        return;
      }
    }
    const R bx_old = Bmx[og], bz_old = hasz ? Bmz[og] : R(0);
    R bx, bz;
    if (!upper) {
      bx = (R(-2) * ez - b * bxi - c * dBy) * ia;
      bz = (R(2) * ex - b * bzi) * ia;
    } else {
      bx = (R(2) * ez - b * bxi + c * dBy) * ia;
      bz = (R(-2) * ex - b * bzi) * ia;
    }
    Bx[og] = bx;
    mirror(g, Bx, og, i, gh, bx);
    const R mbx = R(0.5) * (bx_old + bx);
    Bmx[og] = mbx;
    mirror(g, Bmx, og, i, gh, mbx);
    if (hasz) {
      Bz[og] = bz;
      mirror(g, Bz, og, i, gh, bz);
      const R mbz = R(0.5) * (bz_old + bz);
      Bmz[og] = mbz;
      mirror(g, Bmz, og, i, gh, mbz);
    }
  }
}

// Binomial current filter (Section 3.2): NP passes of (1,2,1)/4 along x then
// y, applied as the separable stencil (1,2,1)/4 (NP = 1) or (1,4,6,4,1)/16
// (NP = 2) per axis, from the deposited set into the other current set.
// Periodic axes wrap; open axes read zero outside the stored range (the
// deposit never reaches the outer two stored layers, so this equals the
// pass-by-pass definition).
template <typename R, int NP>
__device__ __forceinline__ void filter_current(const FieldArgs<R> &a, int src, int dst, int bx,
                                               int by) {
  const Geom &g = a.g;
  const bool px = g.fbc_x == FBC_PERIODIC, py = g.fbc_y == FBC_PERIODIC;
  const int ilo = px ? 0 : -GX, jlo = py ? 0 : -GY;
  const int ihi = px ? g.nx : g.nx + GX, jhi = py ? g.ny : g.ny + GY;
  const int i = ilo + bx * YBX + (int)threadIdx.x;
  const int j = jlo + by * YBY + (int)threadIdx.y;
  if (i >= ihi || j >= jhi) return;
  constexpr int W = 2 * NP + 1;
  const R c1[3] = {R(0.25), R(0.5), R(0.25)};
  const R c2[5] = {R(1.0 / 16), R(4.0 / 16), R(6.0 / 16), R(4.0 / 16), R(1.0 / 16)};
  const R *cw = NP == 1 ? c1 : c2;
  int ii[W], jj[W];
  bool okx[W], oky[W];
#pragma unroll
  for (int k = 0; k < W; ++k) {
    int u = i + k - NP, v = j + k - NP;
    okx[k] = true;
    oky[k] = true;
    if (px) u = u < 0 ? u + g.nx : (u >= g.nx ? u - g.nx : u);
    else okx[k] = u >= -GX && u < g.nx + GX;
    if (py) v = v < 0 ? v + g.ny : (v >= g.ny ? v - g.ny : v);
    else oky[k] = v >= -GY && v < g.ny + GY;
    ii[k] = u;
    jj[k] = v;
  }
  const long long o = fidx(g, i, j);
  for (int c = 0; c < 3; ++c) {
    const R *J = a.F + (C_JA + 3 * src + c) * g.cs;
    R acc = R(0);
#pragma unroll
    for (int b = 0; b < W; ++b) {
      if (!oky[b]) continue;
      R row = R(0);
#pragma unroll
      for (int k = 0; k < W; ++k)
        if (okx[k]) row += cw[k] * J[fidx(g, ii[k], jj[b])];
      acc += cw[b] * row;
    }
    a.F[(C_JA + 3 * dst + c) * g.cs + o] = acc;
  }
}

// Single-run kernels: one 2D grid per kernel.
template <typename R>
__global__ void __launch_bounds__(YBX * YBY) k_update_E(const FieldArgs<R> a) {
  update_E(a, blockIdx.x, blockIdx.y);
}
template <typename R>
__global__ void __launch_bounds__(YBX * YBY) k_update_B(const FieldArgs<R> a) {
  update_B(a, blockIdx.x, blockIdx.y);
}
template <typename R>
__global__ void k_silver_mueller(const FieldArgs<R> a) {
  silver_mueller(a, blockIdx.x, blockIdx.y);
}
template <typename R, int NP>
__global__ void __launch_bounds__(YBX * YBY) k_filter_current(const FieldArgs<R> a, int src,
                                                              int dst) {
  filter_current<R, NP>(a, src, dst, blockIdx.x, blockIdx.y);
}

// Batched kernels: a 1D grid over the blocks of every run (BatchGrid); each
// block reads its run's arguments and works as the block (bx, by) of that
// run's own grid.
__device__ __forceinline__ int batch_block(const BatchGrid &bg, int &bx, int &by) {
  const int b = blockIdx.x;
  const int r = batch_run(bg.off, bg.n, b);
  const int k = b - bg.off[r];
  by = k / bg.gx[r];
  bx = k - by * bg.gx[r];
  return r;
}
template <typename R>
__global__ void __launch_bounds__(YBX * YBY) k_update_E_batch(const FieldArgs<R> *fa,
                                                              const BatchGrid bg) {
  int bx, by;
  const FieldArgs<R> a = fa[batch_block(bg, bx, by)];
  update_E(a, bx, by);
}
template <typename R>
__global__ void __launch_bounds__(YBX * YBY) k_update_B_batch(const FieldArgs<R> *fa,
                                                              const BatchGrid bg) {
  int bx, by;
  const FieldArgs<R> a = fa[batch_block(bg, bx, by)];
  update_B(a, bx, by);
}
template <typename R>
__global__ void k_silver_mueller_batch(const FieldArgs<R> *fa, const BatchGrid bg) {
  int bx, by;
  const FieldArgs<R> a = fa[batch_block(bg, bx, by)];
  silver_mueller(a, bx, by);
}
template <typename R>
__global__ void __launch_bounds__(YBX * YBY) k_filter_current_batch(const FieldArgs<R> *fa,
                                                                    const BatchGrid bg) {
  int bx, by;
  const FieldArgs<R> a = fa[batch_block(bg, bx, by)];
  if (a.filter_passes == 1) filter_current<R, 1>(a, a.parity, 1 - a.parity, bx, by);
  else filter_current<R, 2>(a, a.parity, 1 - a.parity, bx, by);
}

// ---------------------------------------------------------------- I/O ----
__host__ __device__ inline void out_layout(const Geom &g, int &lx, int &nxo, int &ly, int &nyo) {
  lx = g.fbc_x == FBC_PERIODIC ? 0 : -1;
  nxo = g.fbc_x == FBC_PERIODIC ? g.nx : g.nx + 2;
  ly = g.fbc_y == FBC_PERIODIC ? 0 : -1;
  nyo = g.fbc_y == FBC_PERIODIC ? g.ny : g.ny + 2;
}

template <typename R>
__global__ void k_set_field(const Geom g, R *arr, const double *src) {
  int lx, nxo, ly, nyo;
  out_layout(g, lx, nxo, ly, nyo);
  const int a = blockIdx.x * blockDim.x + threadIdx.x, b = blockIdx.y;
  if (a >= nxo || b >= nyo) return;
  store_mirrored(g, arr, lx + a, ly + b, R(src[(long long)b * nxo + a]));
}

template <typename R>
__global__ void k_get_field(const Geom g, const R *arr, double *dst) {
  int lx, nxo, ly, nyo;
  out_layout(g, lx, nxo, ly, nyo);
  const int a = blockIdx.x * blockDim.x + threadIdx.x, b = blockIdx.y;
  if (a >= nxo || b >= nyo) return;
  dst[(long long)b * nxo + a] = (double)arr[fidx(g, lx + a, ly + b)];
}

// Moving-window shift of whole rows: the value at stored index i takes the
// value at i + P when that index is stored (boundary and ghost nodes
// included), else 0 (vacuum), for every stored row.
template <typename R>
__global__ void k_shift_rows(const Geom g, R *base, long long comp_stride) {
  extern __shared__ unsigned char row_raw[];
  R *row = reinterpret_cast<R *>(row_raw);
  R *a = base + blockIdx.y * comp_stride + (long long)blockIdx.x * g.sx;
  const int n = g.nx + 2 * GX;
  for (int e = threadIdx.x; e < n; e += blockDim.x) row[e] = a[e];
  __syncthreads();
  for (int e = threadIdx.x; e < n; e += blockDim.x) {
    const int i = e - GX;
    a[e] = (i + g.P < g.nx + GX) ? row[e + g.P] : R(0);
  }
}

// ----------------------------------------------------------- diagnostics ----
template <typename R>
__global__ void k_field_energy(const Geom g, const R *F, double *partials) {
  __shared__ double sh[2][256];
  double ue = 0.0, ub = 0.0;
  const long long ncell = (long long)g.nx * g.ny;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < ncell;
       c += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(c % g.nx), j = (int)(c / g.nx);
    const long long o = fidx(g, i, j);
    for (int k = 0; k < 3; ++k) {
      const double e = (double)F[(C_EX + k) * g.cs + o];
      const double b = (double)F[(C_BMX + k) * g.cs + o];
      ue += e * e;
      ub += b * b;
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

template <typename R>
__global__ void k_gauss(const Geom g, const R *F, int jset, const double *rho,
                        const double *rho_prev, const double *rho_bg, double *partials) {
  __shared__ double sh[2][256];
  const int xl = g.fbc_x == FBC_PERIODIC ? 0 : 3, xh = g.fbc_x == FBC_PERIODIC ? g.nx : g.nx - 3;
  const int yl = g.fbc_y == FBC_PERIODIC ? 0 : 3, yh = g.fbc_y == FBC_PERIODIC ? g.ny : g.ny - 3;
  const int wx = xh - xl, wy = yh - yl;
  double gm = 0.0, cm = 0.0;
  const R *Ex = F + C_EX * g.cs, *Ey = F + C_EY * g.cs;
  const R *Jx = F + (C_JA + 3 * jset) * g.cs, *Jy = Jx + g.cs;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < (long long)wx * wy;
       c += (long long)gridDim.x * blockDim.x) {
    const int i = xl + (int)(c % wx), j = yl + (int)(c / wx);
    const long long o = fidx(g, i, j);
    // index i-1 / j-1 of a periodic axis at i = 0 reads the mirror ghost
    const double divE = ((double)Ex[o] - (double)Ex[o - 1]) / g.dx +
                        ((double)Ey[o] - (double)Ey[o - g.sx]) / g.dy;
    const double r = rho[o] + rho_bg[o];
    gm = fmax(gm, fabs(divE - r));
    if (rho_prev) {
      // the current is stored on canonical nodes only: wrap the -1 neighbour
      long long oxm = o - 1, oym = o - g.sx;
      if (g.fbc_x == FBC_PERIODIC && i == 0) oxm = fidx(g, g.nx - 1, j);
      if (g.fbc_y == FBC_PERIODIC && j == 0) oym = fidx(g, i, g.ny - 1);
      const double divJ = ((double)Jx[o] - (double)Jx[oxm]) / g.dx +
                          ((double)Jy[o] - (double)Jy[oym]) / g.dy;
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

}  // namespace

template <typename R>
cudaError_t launch_filter(const FieldArgs<R> &a, int src, int dst, cudaStream_t s) {
  const Geom &g = a.g;
  const dim3 blk(YBX, YBY);
  const int fw = g.fbc_x == FBC_PERIODIC ? g.nx : g.nx + 2 * GX;
  const int fh = g.fbc_y == FBC_PERIODIC ? g.ny : g.ny + 2 * GY;
  const dim3 fgrid((fw + YBX - 1) / YBX, (fh + YBY - 1) / YBY);
  if (a.filter_passes == 1)
    k_filter_current<R, 1><<<fgrid, blk, 0, s>>>(a, src, dst);
  else if (a.filter_passes == 2)
    k_filter_current<R, 2><<<fgrid, blk, 0, s>>>(a, src, dst);
  return cudaGetLastError();
}
template cudaError_t launch_filter<float>(const FieldArgs<float> &, int, int, cudaStream_t);
template cudaError_t launch_filter<double>(const FieldArgs<double> &, int, int, cudaStream_t);

template <typename R>
cudaError_t launch_fields(const FieldArgs<R> &a, cudaStream_t s) {
  const Geom &g = a.g;
  const int nxp = g.nx + (g.fbc_x == FBC_SM), nyp = g.ny + (g.fbc_y == FBC_SM);
  const dim3 blk(YBX, YBY);
  if (a.filter_passes > 0) {
    const cudaError_t e = launch_filter(a, a.parity, 1 - a.parity, s);
    if (e != cudaSuccess) return e;
  }
  k_update_E<R><<<dim3((nxp + YBX - 1) / YBX, (nyp + YBY - 1) / YBY), blk, 0, s>>>(a);
  const int ncol = g.nx + 2 * GX, nrow = g.ny + 2 * GY;
  k_update_B<R><<<dim3((ncol + YBX - 1) / YBX, (nrow + YBY - 1) / YBY), blk, 0, s>>>(a);
  if (g.fbc_x == FBC_SM || g.fbc_y == FBC_SM) {
    const int n = (g.nx > g.ny ? g.nx : g.ny) + 1;
    k_silver_mueller<R><<<dim3((n + 63) / 64, 4), 64, 0, s>>>(a);
  }
  return cudaGetLastError();
}

void field_batch_blocks(const Geom &g, int filter_passes, int gx[4], int gy[4]) {
  const int nxp = g.nx + (g.fbc_x == FBC_SM), nyp = g.ny + (g.fbc_y == FBC_SM);
  gx[0] = gy[0] = 0;
  if (filter_passes > 0) {
    const int fw = g.fbc_x == FBC_PERIODIC ? g.nx : g.nx + 2 * GX;
    const int fh = g.fbc_y == FBC_PERIODIC ? g.ny : g.ny + 2 * GY;
    gx[0] = (fw + YBX - 1) / YBX;
    gy[0] = (fh + YBY - 1) / YBY;
  }
  gx[1] = (nxp + YBX - 1) / YBX;
  gy[1] = (nyp + YBY - 1) / YBY;
  gx[2] = (g.nx + 2 * GX + YBX - 1) / YBX;
  gy[2] = (g.ny + 2 * GY + YBY - 1) / YBY;
  gx[3] = gy[3] = 0;
  if (g.fbc_x == FBC_SM || g.fbc_y == FBC_SM) {
    gx[3] = ((g.nx > g.ny ? g.nx : g.ny) + 1 + 63) / 64;
    gy[3] = 4;  // one row of blocks per face
  }
}

template <typename R>
cudaError_t launch_fields_batch(const FieldArgs<R> *fa, const BatchGrid grid[4], cudaStream_t s) {
  const dim3 blk(YBX, YBY);
  if (grid[0].off[grid[0].n] > 0)
    k_filter_current_batch<R><<<grid[0].off[grid[0].n], blk, 0, s>>>(fa, grid[0]);
  k_update_E_batch<R><<<grid[1].off[grid[1].n], blk, 0, s>>>(fa, grid[1]);
  k_update_B_batch<R><<<grid[2].off[grid[2].n], blk, 0, s>>>(fa, grid[2]);
  if (grid[3].off[grid[3].n] > 0)
    k_silver_mueller_batch<R><<<grid[3].off[grid[3].n], 64, 0, s>>>(fa, grid[3]);
  return cudaGetLastError();
}
template cudaError_t launch_fields_batch<float>(const FieldArgs<float> *, const BatchGrid[4],
                                                cudaStream_t);
template cudaError_t launch_fields_batch<double>(const FieldArgs<double> *, const BatchGrid[4],
                                                 cudaStream_t);

template <typename R>
cudaError_t launch_set_field(const Geom &g, R *arr, const double *src, cudaStream_t s) {
  int lx, nxo, ly, nyo;
  out_layout(g, lx, nxo, ly, nyo);
  k_set_field<R><<<dim3((nxo + 255) / 256, nyo), 256, 0, s>>>(g, arr, src);
  return cudaGetLastError();
}
template <typename R>
cudaError_t launch_get_field(const Geom &g, const R *arr, double *dst, cudaStream_t s) {
  int lx, nxo, ly, nyo;
  out_layout(g, lx, nxo, ly, nyo);
  k_get_field<R><<<dim3((nxo + 255) / 256, nyo), 256, 0, s>>>(g, arr, dst);
  return cudaGetLastError();
}
cudaError_t launch_get_field_f64(const Geom &g, const double *arr, double *dst, cudaStream_t s) {
  return launch_get_field<double>(g, arr, dst, s);
}
namespace {
__global__ void k_axpy_f64(double *y, const double *x, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x)
    y[i] += x[i];
}
}  // namespace

namespace {
__global__ void k_absmax_f64(const double *w, size_t n, unsigned long long *out) {
  unsigned long long m = 0ull;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x) {
    const double a = fabs(w[i]);
    // bits of a non-negative double order as the values; NaN counts as inf
    const unsigned long long b =
        isfinite(a) ? (unsigned long long)__double_as_longlong(a) : 0x7ff0000000000000ull;
    m = b > m ? b : m;
  }
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long v = __shfl_down_sync(0xffffffffu, m, o);
    m = v > m ? v : m;
  }
  if ((threadIdx.x & 31) == 0 && m) atomicMax(out, m);
}
}  // namespace

cudaError_t launch_absmax_f64(const double *w, size_t n, unsigned long long *out, cudaStream_t s) {
  const int blocks = (int)((n + 255) / 256 < 2048 ? (n + 255) / 256 : 2048);
  k_absmax_f64<<<blocks > 0 ? blocks : 1, 256, 0, s>>>(w, n, out);
  return cudaGetLastError();
}

cudaError_t launch_axpy_f64(double *y, const double *x, size_t n, cudaStream_t s) {
  const int blocks = (int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096);
  k_axpy_f64<<<blocks > 0 ? blocks : 1, 256, 0, s>>>(y, x, n);
  return cudaGetLastError();
}

cudaError_t launch_set_field_f64(const Geom &g, double *arr, const double *src, cudaStream_t s) {
  return launch_set_field<double>(g, arr, src, s);
}

template <typename R>
cudaError_t launch_shift_fields(const Geom &g, R *F, int ncomp, cudaStream_t s) {
  const size_t smem = (size_t)(g.nx + 2 * GX) * sizeof(R);
  k_shift_rows<R><<<dim3(g.nys, ncomp), 256, smem, s>>>(g, F, g.cs);
  return cudaGetLastError();
}
cudaError_t launch_shift_f64(const Geom &g, double *a, cudaStream_t s) {
  return launch_shift_fields<double>(g, a, 1, s);
}

template <typename R>
cudaError_t launch_field_diag(const Geom &g, const R *F, double *partials, int nblocks,
                              cudaStream_t s) {
  k_field_energy<R><<<nblocks, 256, 0, s>>>(g, F, partials);
  return cudaGetLastError();
}
template <typename R>
cudaError_t launch_gauss_diag(const Geom &g, const R *F, int jset, const double *rho,
                              const double *rho_prev, const double *rho_bg, double *partials,
                              int nblocks, cudaStream_t s) {
  k_gauss<R><<<nblocks, 256, 0, s>>>(g, F, jset, rho, rho_prev, rho_bg, partials);
  return cudaGetLastError();
}

#define PIC_INST(R)                                                                          \
  template cudaError_t launch_fields<R>(const FieldArgs<R> &, cudaStream_t);                 \
  template cudaError_t launch_set_field<R>(const Geom &, R *, const double *, cudaStream_t); \
  template cudaError_t launch_get_field<R>(const Geom &, const R *, double *, cudaStream_t); \
  template cudaError_t launch_shift_fields<R>(const Geom &, R *, int, cudaStream_t);         \
  template cudaError_t launch_field_diag<R>(const Geom &, const R *, double *, int,          \
                                            cudaStream_t);                                   \
  template cudaError_t launch_gauss_diag<R>(const Geom &, const R *, int, const double *,    \
                                            const double *, const double *, double *, int,   \
                                            cudaStream_t);
PIC_INST(float)
PIC_INST(double)
#undef PIC_INST

}  // namespace pic
