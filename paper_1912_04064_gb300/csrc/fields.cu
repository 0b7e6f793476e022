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

constexpr int RY = 8;      // rows per thread in the Yee kernels
constexpr int YEE_BX = 128;

// True when any cell of the block's tile lies in a periodic mirror band.
__device__ __forceinline__ bool block_mirrors(const Geom &g, int i0, int i1, int j0, int j1) {
  return (g.fbc_x == FBC_PERIODIC && (i0 < GX || i1 > g.nx - GX)) ||
         (g.fbc_y == FBC_PERIODIC && (j0 < GY || j1 > g.ny - GY));
}

// E^{n+1} = E^n + dt (curl_h B^{n+1/2} - J^{n+1/2}); one thread per column
// segment of RY rows, the previous row's B carried in registers.
template <typename R>
__global__ void __launch_bounds__(YEE_BX) k_update_E(const FieldArgs<R> a) {
  const Geom &g = a.g;
  const Ranges rg = ranges(g);
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j0 = blockIdx.y * RY;
  const int j1 = min(j0 + RY, rg.nyp);
  const int ib0 = blockIdx.x * blockDim.x;
  const bool mir = block_mirrors(g, ib0, ib0 + blockDim.x, j0, j1);
  if (i >= rg.nxp) return;
  const long long cs = g.cs;
  const int sx = g.sx;
  R *F = a.F;
  R *Ex = F + C_EX * cs, *Ey = F + C_EY * cs, *Ez = F + C_EZ * cs;
  const R *Bx = F + C_BX * cs, *By = F + C_BY * cs, *Bz = F + C_BZ * cs;
  const R *J = F + (C_JA + 3 * a.parity) * cs;
  const R dt = R(g.dt), idx = R(1.0 / g.dx), idy = R(1.0 / g.dy);
  long long o = fidx(g, i, j0);
  R bzp = Bz[o - sx], bxp = Bx[o - sx];
  for (int j = j0; j < j1; ++j, o += sx) {
    const R bz = Bz[o], bx = Bx[o], by = By[o];
    const R bzl = Bz[o - 1], byl = By[o - 1];
    if (i < rg.nxd) {
      const R v = Ex[o] + dt * ((bz - bzp) * idy - J[o]);
      Ex[o] = v;
      if (mir) mirror(g, Ex, o, i, j, v);
    }
    if (j < rg.nyd) {
      const R v = Ey[o] + dt * (-(bz - bzl) * idx - J[cs + o]);
      Ey[o] = v;
      if (mir) mirror(g, Ey, o, i, j, v);
    }
    {
      const R v = Ez[o] + dt * ((by - byl) * idx - (bx - bxp) * idy - J[2 * cs + o]);
      Ez[o] = v;
      if (mir) mirror(g, Ez, o, i, j, v);
    }
    bzp = bz;
    bxp = bx;
  }
}

// B^{n+3/2} = B^{n+1/2} - dt curl_h E^{n+1}, Bm^{n+1} = (B^{n+1/2} +
// B^{n+3/2}) / 2 (= B at stored cells that are not updated), and the
// current set of the next step cleared.  Covers every stored column and row.
template <typename R>
__global__ void __launch_bounds__(YEE_BX) k_update_B(const FieldArgs<R> a) {
  const Geom &g = a.g;
  if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) {
    const int p = a.parity;
    a.st->t[1 - p] = a.st->t[p] + g.dt;
    a.st->step[1 - p] = a.st->step[p] + 1;
    a.st->maxcnt[1 - p] = 0;  // the next particle step starts a new maximum
  }
  const Ranges rg = ranges(g);
  const int i = (int)(blockIdx.x * blockDim.x + threadIdx.x) - GX;
  const int j0 = (int)(blockIdx.y * RY) - GY;
  const int j1 = min(j0 + RY, g.ny + GY);
  const int ib0 = (int)(blockIdx.x * blockDim.x) - GX;
  const bool mir = block_mirrors(g, ib0, ib0 + blockDim.x, j0, j1);
  if (i >= g.nx + GX) return;
  const bool perx = g.fbc_x == FBC_PERIODIC, pery = g.fbc_y == FBC_PERIODIC;
  const bool ghost_x = i < 0 || i >= g.nx;
  const long long cs = g.cs;
  const int sx = g.sx;
  R *F = a.F;
  const R *Ex = F + C_EX * cs, *Ey = F + C_EY * cs, *Ez = F + C_EZ * cs;
  R *Bx = F + C_BX * cs, *By = F + C_BY * cs, *Bz = F + C_BZ * cs;
  R *Bmx = F + C_BMX * cs, *Bmy = F + C_BMY * cs, *Bmz = F + C_BMZ * cs;
  R *Jn = F + (C_JA + 3 * (1 - a.parity)) * cs;
  const R dt = R(g.dt), idx = R(1.0 / g.dx), idy = R(1.0 / g.dy);
  long long o = fidx(g, i, j0);
  for (int j = j0; j < j1; ++j, o += sx) {
    Jn[o] = R(0);
    Jn[cs + o] = R(0);
    Jn[2 * cs + o] = R(0);
    if ((perx && ghost_x) || (pery && (j < 0 || j >= g.ny))) continue;  // mirror cells
    const bool in = i >= 0 && j >= 0;
    {
      const R b0 = Bx[o];
      R b1 = b0;
      if (in && i < rg.nxp && j < rg.nyd) {
        b1 = b0 - dt * (Ez[o + sx] - Ez[o]) * idy;
        Bx[o] = b1;
        if (mir) mirror(g, Bx, o, i, j, b1);
      }
      const R m = R(0.5) * (b0 + b1);
      Bmx[o] = m;
      if (mir) mirror(g, Bmx, o, i, j, m);
    }
    {
      const R b0 = By[o];
      R b1 = b0;
      if (in && i < rg.nxd && j < rg.nyp) {
        b1 = b0 + dt * (Ez[o + 1] - Ez[o]) * idx;
        By[o] = b1;
        if (mir) mirror(g, By, o, i, j, b1);
      }
      const R m = R(0.5) * (b0 + b1);
      Bmy[o] = m;
      if (mir) mirror(g, Bmy, o, i, j, m);
    }
    {
      const R b0 = Bz[o];
      R b1 = b0;
      if (in && i < rg.nxd && j < rg.nyd) {
        b1 = b0 - dt * ((Ey[o + 1] - Ey[o]) * idx - (Ex[o + sx] - Ex[o]) * idy);
        Bz[o] = b1;
        if (mir) mirror(g, Bz, o, i, j, b1);
      }
      const R m = R(0.5) * (b0 + b1);
      Bmz[o] = m;
      if (mir) mirror(g, Bmz, o, i, j, m);
    }
  }
}

template <typename R>
__device__ __forceinline__ double laser_field(const FieldArgs<R> &a, double y, double t,
                                              int nshift) {
  const double tr = t - (double)(nshift * a.g.P) * a.g.dx - a.t_peak;
  const double r = (y - a.yc) / a.waist;
  return a.a0 * exp(-r * r) * exp(-2.0 * log(2.0) * tr * tr / (a.tau * a.tau)) * sin(tr);
}

template <typename R>
__device__ __forceinline__ void set_ghost(const Geom &g, R *B, R *Bm, int i, int j, R v) {
  const long long o = fidx(g, i, j);
  const R old = Bm[o];  // = B^{n+1/2} at this ghost after k_update_B
  store_mirrored(g, B, i, j, v);
  store_mirrored(g, Bm, i, j, R(0.5) * (old + v));
}

template <typename R>
__global__ void k_silver_mueller(const FieldArgs<R> a) {
  const Geom &g = a.g;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  R *F = a.F;
  const long long cs = g.cs;
  const R *Ex = F + C_EX * cs, *Ey = F + C_EY * cs, *Ez = F + C_EZ * cs;
  R *Bx = F + C_BX * cs, *By = F + C_BY * cs, *Bz = F + C_BZ * cs;
  R *Bmx = F + C_BMX * cs, *Bmy = F + C_BMY * cs, *Bmz = F + C_BMZ * cs;
  const Ranges rg = ranges(g);
  const double dt = g.dt;
  if (g.fbc_x == FBC_SM && t < rg.nyp) {
    const int j = t, nx = g.nx;
    const double r = dt / g.dx;
    const bool inter = g.fbc_y == FBC_PERIODIC || (j >= 1 && j <= g.ny - 1);
    double dBx0 = 0.0, dBxn = 0.0;
    if (inter) {
      dBx0 = (double)Bx[fidx(g, 0, j)] - (double)Bx[fidx(g, 0, j - 1)];
      dBxn = (double)Bx[fidx(g, nx, j)] - (double)Bx[fidx(g, nx, j - 1)];
    }
    const double by_lo = (2.0 * Ez[fidx(g, 0, j)] - (1.0 - r) * By[fidx(g, 0, j)] -
                          (dt / g.dy) * dBx0) / (1.0 + r);
    const double by_hi = (-2.0 * Ez[fidx(g, nx, j)] - (1.0 - r) * By[fidx(g, nx - 1, j)] +
                          (dt / g.dy) * dBxn) / (1.0 + r);
    set_ghost(g, By, Bmy, -1, j, R(by_lo));
    set_ghost(g, By, Bmy, nx, j, R(by_hi));
    if (j < rg.nyd) {
      double eyinc = 0.0;
      if (a.laser_on)
        eyinc = laser_field(a, (j + 0.5) * g.dy, a.st->t[a.parity] + 1.5 * dt, a.st->nshift);
      const double bz_lo =
          (4.0 * eyinc - 2.0 * Ey[fidx(g, 0, j)] - (1.0 - r) * Bz[fidx(g, 0, j)]) / (1.0 + r);
      const double bz_hi =
          (2.0 * Ey[fidx(g, nx, j)] - (1.0 - r) * Bz[fidx(g, nx - 1, j)]) / (1.0 + r);
      set_ghost(g, Bz, Bmz, -1, j, R(bz_lo));
      set_ghost(g, Bz, Bmz, nx, j, R(bz_hi));
    }
  }
  if (g.fbc_y == FBC_SM && t < rg.nxp) {
    const int i = t, ny = g.ny;
    const double r = dt / g.dy;
    const bool inter = g.fbc_x == FBC_PERIODIC || (i >= 1 && i <= g.nx - 1);
    double dBy0 = 0.0, dByn = 0.0;
    if (inter) {
      dBy0 = (double)By[fidx(g, i, 0)] - (double)By[fidx(g, i - 1, 0)];
      dByn = (double)By[fidx(g, i, ny)] - (double)By[fidx(g, i - 1, ny)];
    }
    const double bx_lo = (-2.0 * Ez[fidx(g, i, 0)] - (1.0 - r) * Bx[fidx(g, i, 0)] -
                          (dt / g.dx) * dBy0) / (1.0 + r);
    const double bx_hi = (2.0 * Ez[fidx(g, i, ny)] - (1.0 - r) * Bx[fidx(g, i, ny - 1)] +
                          (dt / g.dx) * dByn) / (1.0 + r);
    set_ghost(g, Bx, Bmx, i, -1, R(bx_lo));
    set_ghost(g, Bx, Bmx, i, ny, R(bx_hi));
    if (i < rg.nxd) {
      const double bz_lo = (2.0 * Ex[fidx(g, i, 0)] - (1.0 - r) * Bz[fidx(g, i, 0)]) / (1.0 + r);
      const double bz_hi =
          (-2.0 * Ex[fidx(g, i, ny)] - (1.0 - r) * Bz[fidx(g, i, ny - 1)]) / (1.0 + r);
      set_ghost(g, Bz, Bmz, i, -1, R(bz_lo));
      set_ghost(g, Bz, Bmz, i, ny, R(bz_hi));
    }
  }
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
cudaError_t launch_fields(const FieldArgs<R> &a, cudaStream_t s) {
  const Geom &g = a.g;
  const int nxp = g.nx + (g.fbc_x == FBC_SM), nyp = g.ny + (g.fbc_y == FBC_SM);
  k_update_E<R><<<dim3((nxp + YEE_BX - 1) / YEE_BX, (nyp + RY - 1) / RY), YEE_BX, 0, s>>>(a);
  const int ncol = g.nx + 2 * GX, nrow = g.ny + 2 * GY;
  k_update_B<R><<<dim3((ncol + YEE_BX - 1) / YEE_BX, (nrow + RY - 1) / RY), YEE_BX, 0, s>>>(a);
  if (g.fbc_x == FBC_SM || g.fbc_y == FBC_SM) {
    const int n = (g.nx > g.ny ? g.nx : g.ny) + 1;
    k_silver_mueller<R><<<(n + 127) / 128, 128, 0, s>>>(a);
  }
  return cudaGetLastError();
}

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
