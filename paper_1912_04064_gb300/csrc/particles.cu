// Particle storage kernels: binning of loaded particles into patch segments,
// the float64 charge deposit used by diagnostics, particle reductions,
// read-back in global coordinates and the moving-window bookkeeping
// (migration of in-flight particles, removal of the leaving column and
// injection of plasma in the new one).
#include "common.cuh"
#include "pack.h"

namespace pic {

namespace {

__device__ __forceinline__ bool locate(const Geom &g, int col0, double x, double y, int &slot,
                                       int &px, int &py) {
  const double cx = x / g.dx, cy = y / g.dy;
  if (!(cx >= 0.0 && cx < (double)g.nx && cy >= 0.0 && cy < (double)g.ny)) return false;
  px = (int)floor(cx) / g.P;
  py = (int)floor(cy) / g.Q;
  if (px >= g.npx) px = g.npx - 1;
  if (py >= g.npy) py = g.npy - 1;
  slot = py * g.npx + (px + col0) % g.npx;
  return true;
}

template <typename R>
__device__ __forceinline__ R rel(double c, int origin, int P) {
  double v = c - (double)origin;
  R r = R(v);
  if (r < R(0)) r = R(0);
  if (r >= R(P)) r = nextafter(R(P), R(0));
  return r;
}

template <typename R>
__global__ void k_bin_count(const Geom g, int col0, const double *x, const double *y, size_t n,
                            int *counts, unsigned *err) {
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n;
       k += (size_t)gridDim.x * blockDim.x) {
    int slot, px, py;
    const bool ok = locate(g, col0, x[k], y[k], slot, px, py);
    if (!ok) atomicOr(err, ERR_LOAD_RANGE);
    // neighbouring particles mostly share a slot: one atomic per slot and warp
    const unsigned same = __match_any_sync(__activemask(), ok ? slot : -1);
    if (ok && (unsigned)(__ffs(same) - 1) == (threadIdx.x & 31u)) atomicAdd(&counts[slot], __popc(same));
  }
}

template <typename R>
__global__ void k_bin_place(const Geom g, int col0, const double *x, const double *y,
                            const double *ux, const double *uy, const double *uz,
                            const double *w, size_t n, SoA<R> seg, int *counts, int cap,
                            unsigned *err) {
  const unsigned lane = threadIdx.x & 31u;
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n;
       k += (size_t)gridDim.x * blockDim.x) {
    int slot, px, py;
    const bool ok = locate(g, col0, x[k], y[k], slot, px, py);
    // positions within a slot: one atomic per slot and warp, lanes in order
    const unsigned same = __match_any_sync(__activemask(), ok ? slot : -1);
    const int leader = __ffs(same) - 1;
    int base = 0;
    if (ok && (int)lane == leader) base = atomicAdd(&counts[slot], __popc(same));
    base = __shfl_sync(same, base, leader);
    if (!ok) continue;
    const int pos = base + __popc(same & ((1u << lane) - 1u));
    if (pos >= cap) {
      atomicOr(err, ERR_OVERFLOW_LOAD);
      continue;
    }
    const long long i = (long long)slot * cap + pos;
    seg.x[i] = rel<R>(x[k] / g.dx, px * g.P, g.P);
    seg.y[i] = rel<R>(y[k] / g.dy, py * g.Q, g.Q);
    seg.ux[i] = R(ux[k]);
    seg.uy[i] = R(uy[k]);
    seg.uz[i] = R(uz[k]);
    seg.w[i] = R(w[k]);
  }
}

__global__ void k_clamp_counts(int *cnt, int n, int cap) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && cnt[i] > cap) cnt[i] = cap;
}

// Origin (in cells) of the physical patch held by a slot.
__device__ __forceinline__ void slot_origin(const Geom &g, int col0, int slot, int &X0, int &Y0) {
  int px = slot % g.npx - col0;
  if (px < 0) px += g.npx;
  X0 = px * g.P;
  Y0 = (slot / g.npx) * g.Q;
}

// Visit every particle of a view: blocks walk slots; each slot's segment and
// its 8 outgoing buckets (bucket particles are expressed in the frame of the
// destination patch).
template <typename R, typename Fn>
__device__ void for_each_particle(const Geom &g, int col0, const PartView<R> &v, Fn fn) {
  for (int slot = blockIdx.x; slot < g.nslots; slot += gridDim.x) {
    int X0, Y0;
    slot_origin(g, col0, slot, X0, Y0);
    const int n = min(v.cnt[slot], v.cap);
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
      const long long i = (long long)slot * v.cap + k;
      fn(X0, Y0, v.seg.x[i], v.seg.y[i], v.seg.ux[i], v.seg.uy[i], v.seg.uz[i], v.seg.w[i]);
    }
    for (int d = 0; d < 8; ++d) {
      const int nb = min(v.bcnt[(long long)slot * 8 + d], v.bk.cap[d]);
      if (nb == 0) continue;
      int ddx, ddy;
      dir_delta(d, ddx, ddy);
      const int dest = neighbour_slot(g, col0, slot, ddx, ddy);
      if (dest < 0) continue;
      int DX0, DY0;
      slot_origin(g, col0, dest, DX0, DY0);
      for (int k = threadIdx.x; k < nb; k += blockDim.x) {
        const long long i = (long long)slot * v.bk.stride + v.bk.off[d] + k;
        fn(DX0, DY0, v.bkt.x[i], v.bkt.y[i], v.bkt.ux[i], v.bkt.uy[i], v.bkt.uz[i], v.bkt.w[i]);
      }
    }
  }
}

__device__ __forceinline__ void shape_d(double xi, int &i0, double S[3]) {
  const double fl = floor(xi + 0.5);
  const double d = xi - fl;
  S[0] = 0.5 * (0.5 - d) * (0.5 - d);
  S[1] = 0.75 - d * d;
  S[2] = 0.5 * (0.5 + d) * (0.5 + d);
  i0 = (int)fl;
}

__device__ __forceinline__ void deposit_node(const Geom &g, double *rho, int X0, int Y0, double xr,
                                             double yr, double qw) {
  int i0, j0;
  double Sx[3], Sy[3];
  shape_d(xr, i0, Sx);
  shape_d(yr, j0, Sy);
  for (int b = 0; b < 3; ++b)
    for (int a = 0; a < 3; ++a) {
      int gi = X0 + i0 - 1 + a, gj = Y0 + j0 - 1 + b;
      if (g.fbc_x == FBC_PERIODIC) gi = (gi + g.nx) % g.nx;
      if (g.fbc_y == FBC_PERIODIC) gj = (gj + g.ny) % g.ny;
      atomicAdd(&rho[fidx(g, gi, gj)], qw * Sx[a] * Sy[b]);
    }
}

template <typename R>
__global__ void k_deposit_rho(const Geom g, int col0, const PartView<R> v, double *rho,
                              double sign) {
  const double qs = sign * g.q;
  for_each_particle<R>(g, col0, v, [&](int X0, int Y0, R x, R y, R, R, R, R w) {
    deposit_node(g, rho, X0, Y0, (double)x, (double)y, qs * (double)w);
  });
}

template <typename R>
__global__ void k_particle_diag(const Geom g, int col0, const PartView<R> v, double *partials) {
  __shared__ double sh[3][256];
  double ek = 0.0, ws = 0.0, cnt = 0.0;
  for_each_particle<R>(g, col0, v, [&](int, int, R, R, R ux, R uy, R uz, R w) {
    const double a = ux, b = uy, c = uz;
    ek += (double)w * (sqrt(1.0 + a * a + b * b + c * c) - 1.0);
    ws += (double)w;
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

// offsets: [phys-order segment offsets (nslots)] [bucket offsets (nslots*8)]
template <typename R>
__global__ void k_get_particles(const Geom g, int col0, const PartView<R> v,
                                const long long *offsets, double *out, size_t stride) {
  const int pp = blockIdx.x;  // physical patch index
  if (pp >= g.nslots) return;
  const int ppx = pp % g.npx, ppy = pp / g.npx;
  const int slot = ppy * g.npx + (ppx + col0) % g.npx;
  auto emit = [&](long long o, int X0, int Y0, R x, R y, R ux, R uy, R uz, R w) {
    out[o] = ((double)X0 + (double)x) * g.dx;
    out[stride + o] = ((double)Y0 + (double)y) * g.dy;
    out[2 * stride + o] = (double)ux;
    out[3 * stride + o] = (double)uy;
    out[4 * stride + o] = (double)uz;
    out[5 * stride + o] = (double)w;
  };
  const int X0 = ppx * g.P, Y0 = ppy * g.Q;
  const int n = min(v.cnt[slot], v.cap);
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    const long long i = (long long)slot * v.cap + k;
    emit(offsets[pp] + k, X0, Y0, v.seg.x[i], v.seg.y[i], v.seg.ux[i], v.seg.uy[i], v.seg.uz[i],
         v.seg.w[i]);
  }
  for (int d = 0; d < 8; ++d) {
    const int nb = min(v.bcnt[(long long)slot * 8 + d], v.bk.cap[d]);
    if (nb == 0) continue;
    int ddx, ddy;
    dir_delta(d, ddx, ddy);
    const int dest = neighbour_slot(g, col0, slot, ddx, ddy);
    if (dest < 0) continue;
    int DX0, DY0;
    slot_origin(g, col0, dest, DX0, DY0);
    const long long base = offsets[g.nslots + (long long)pp * 8 + d];
    for (int k = threadIdx.x; k < nb; k += blockDim.x) {
      const long long i = (long long)slot * v.bk.stride + v.bk.off[d] + k;
      emit(base + k, DX0, DY0, v.bkt.x[i], v.bkt.y[i], v.bkt.ux[i], v.bkt.uy[i], v.bkt.uz[i],
           v.bkt.w[i]);
    }
  }
}

// Moving window, part 1 (old ring, col0 = old): particles that crossed from
// the leaving column into the next one during the last step are still in the
// leaving slots' +x buckets; append them to their destination segments, then
// clear every bucket that points into or out of the leaving column.
template <typename R>
__global__ void k_window_migrate(const Geom g, int col0, SoA<R> seg, int *cnt, SoA<R> bkt,
                                 int *bcnt, int cap, Buckets bk, unsigned *err) {
  const int py = blockIdx.x;
  const int sdrop = py * g.npx + col0;
  const int snext = py * g.npx + (col0 + 1) % g.npx;
  for (int ddy = -1; ddy <= 1; ++ddy) {
    const int d = dir_index(1, ddy);
    const int dest = neighbour_slot(g, col0, sdrop, 1, ddy);
    const int nb = min(bcnt[(long long)sdrop * 8 + d], bk.cap[d]);
    if (dest < 0) continue;
    __shared__ int base;
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
      seg.x[o] = bkt.x[i]; seg.y[o] = bkt.y[i];
      seg.ux[o] = bkt.ux[i]; seg.uy[o] = bkt.uy[i]; seg.uz[o] = bkt.uz[i]; seg.w[o] = bkt.w[i];
    }
    __syncthreads();
    if (threadIdx.x == 0 && cnt[dest] > cap) cnt[dest] = cap;
    __syncthreads();
  }
  if (threadIdx.x < 8) {
    bcnt[(long long)sdrop * 8 + threadIdx.x] = 0;
    int ddx, ddy;
    dir_delta(threadIdx.x, ddx, ddy);
    if (ddx == -1) bcnt[(long long)snext * 8 + threadIdx.x] = 0;
  }
}

// Plasma at rest, regularly placed (ppcx x ppcy per cell), weight =
// density / ppc at the particle's x in the laboratory frame, with the
// co-located immobile ions added to the background charge.  Blocks (py, c,
// *) fill physical patch column phys0 + c, held by slot column
// (slot_col0 + c) mod npx; the z index splits a patch's particles among
// gridDim.z blocks (each particle's slot index k is fixed by its cell and
// sub-cell, whichever block writes it).  Moving window, part 2: after the
// ring advanced, the leaving slots (slot_col0 = old col0) hold the new
// column (phys0 = npx - 1); loading a run's initial plasma fills every
// column.
template <typename R>
__global__ void k_window_inject(const Geom g, int slot_col0, int phys0, int nshift, SoA<R> seg,
                                int *cnt, int cap, double n0, double x0, double ramp, int ppcx,
                                int ppcy, double *rho_bg, unsigned *err) {
  const int py = blockIdx.x;
  const int slot_col = (slot_col0 + (int)blockIdx.y) % g.npx;
  const int slot = py * g.npx + slot_col;
  const int ppc = ppcx * ppcy;
  const int total = g.P * g.Q * ppc;
  if (total > cap) {
    if (threadIdx.x == 0 && blockIdx.z == 0) atomicOr(err, ERR_OVERFLOW_SEG);
    return;
  }
  const int X0 = (phys0 + (int)blockIdx.y) * g.P, Y0 = py * g.Q;
  const double shift = __dmul_rn((double)nshift * g.P, g.dx);
  for (int k = blockIdx.z * blockDim.x + threadIdx.x; k < total; k += gridDim.z * blockDim.x) {
    // order: cell row, cell column, sub-row, sub-column
    const int a = k % ppcx, b = (k / ppcx) % ppcy, cell = k / ppc;
    const int ci = cell % g.P, cj = cell / g.P;
    const double fx = (a + 0.5) / ppcx, fy = (b + 0.5) / ppcy;
    const double xl = ((double)(X0 + ci) + fx) * g.dx;
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
    seg.ux[o] = R(0);
    seg.uy[o] = R(0);
    seg.uz[o] = R(0);
    seg.w[o] = R(w);
    if (rho_bg) deposit_node(g, rho_bg, X0, Y0, (double)ci + fx, (double)cj + fy, -g.q * (double)R(w));
  }
  if (threadIdx.x == 0 && blockIdx.z == 0) cnt[slot] = total;
}

// Blocks per patch of the plasma fill: one per 256 particles, at most 16.
inline unsigned inject_split(const Geom &g, int ppcx, int ppcy) {
  const int blocks = (g.P * g.Q * ppcx * ppcy + 255) / 256;
  return (unsigned)(blocks < 1 ? 1 : (blocks > 16 ? 16 : blocks));
}

template <typename R>
__global__ void k_repack(const Geom g, SoA<R> src, const int *cnt_src, int cap_src, SoA<R> bsrc,
                         const int *bcnt_src, Buckets bk_src, SoA<R> dst, int *cnt_dst,
                         int cap_dst, SoA<R> bdst, int *bcnt_dst, Buckets bk_dst) {
  const int slot = blockIdx.x;
  const int n = min(min(cnt_src[slot], cap_src), cap_dst);
  const long long so = (long long)slot * cap_src, dof = (long long)slot * cap_dst;
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    dst.x[dof + k] = src.x[so + k]; dst.y[dof + k] = src.y[so + k];
    dst.ux[dof + k] = src.ux[so + k]; dst.uy[dof + k] = src.uy[so + k];
    dst.uz[dof + k] = src.uz[so + k]; dst.w[dof + k] = src.w[so + k];
  }
  for (int d = 0; d < 8; ++d) {
    const int nb = min(min(bcnt_src[(long long)slot * 8 + d], bk_src.cap[d]), bk_dst.cap[d]);
    const long long bs = (long long)slot * bk_src.stride + bk_src.off[d];
    const long long bd = (long long)slot * bk_dst.stride + bk_dst.off[d];
    for (int k = threadIdx.x; k < nb; k += blockDim.x) {
      bdst.x[bd + k] = bsrc.x[bs + k]; bdst.y[bd + k] = bsrc.y[bs + k];
      bdst.ux[bd + k] = bsrc.ux[bs + k]; bdst.uy[bd + k] = bsrc.uy[bs + k];
      bdst.uz[bd + k] = bsrc.uz[bs + k]; bdst.w[bd + k] = bsrc.w[bs + k];
    }
    if (threadIdx.x == 0) bcnt_dst[(long long)slot * 8 + d] = nb;
  }
  if (threadIdx.x == 0) cnt_dst[slot] = n;
}

// Interleaved cell order of one patch.  Each row of cells is cut into
// segments of at most 32 cells; inside a segment particles are laid out rank
// slice by rank slice: slice r holds, in column order, the r-th particle of
// every cell of the segment that has more than r particles.  A warp then
// processes 32 particles in 32 distinct neighbouring cells.  Ranks >= SORT_R
// (dense cells) go to a tail after all segments.  Incoming bucket particles
// are absorbed (their counts cleared by the one reader).
constexpr int SORT_R = 64;

template <typename R>
__global__ void k_sort_cells(const Geom g, int col0, SoA<R> src, const int *cnt_src, int cap,
                             SoA<R> bsrc, int *bcnt, Buckets bk, SoA<R> dst, int *cnt_dst,
                             unsigned *err) {
  extern __shared__ int sm[];
  const int P = g.P, Q = g.Q;
  const int spr = (P + 31) / 32;      // segments per row
  const int nseg = Q * spr;
  int *hist = sm;                     // P*Q
  int *rank = hist + P * Q;           // P*Q
  int *segoff = rank + P * Q;         // nseg + 1
  int *sliceoff = segoff + nseg + 1;  // nseg * SORT_R
  unsigned *mask = (unsigned *)(sliceoff + nseg * SORT_R);  // nseg * SORT_R
  __shared__ int s_cnt[9];
  __shared__ long long s_base[9];
  __shared__ int s_off[10];
  __shared__ int s_tail;
  const int slot = blockIdx.x, tid = threadIdx.x, nth = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5, nwarp = nth >> 5;
  for (int e = tid; e < 2 * P * Q; e += nth) sm[e] = 0;
  if (tid < 9) {
    int cnt = 0;
    long long base = 0;
    if (tid == 0) {
      cnt = min(cnt_src[slot], cap);
      base = (long long)slot * cap;
    } else {
      int k = tid - 1, ddx, ddy;
      dir_delta(k, ddx, ddy);
      const int sv = neighbour_slot(g, col0, slot, -ddx, -ddy);
      if (sv >= 0) {
        cnt = min(bcnt[(long long)sv * 8 + k], bk.cap[k]);
        base = (long long)sv * bk.stride + bk.off[k];
      }
    }
    s_cnt[tid] = cnt;
    s_base[tid] = base;
  }
  if (tid == 0) s_tail = 0;
  __syncthreads();
  if (tid == 0) {
    s_off[0] = 0;
    for (int i = 0; i < 9; ++i) s_off[i + 1] = s_off[i] + s_cnt[i];
  }
  __syncthreads();
  const int total = s_off[9];
  auto cell_of = [&](int k, long long &idx, const SoA<R> *&A) {
    int sidx = 0;
    while (sidx < 8 && k >= s_off[sidx + 1]) ++sidx;
    idx = s_base[sidx] + (k - s_off[sidx]);
    A = sidx == 0 ? &src : &bsrc;
    int cx = (int)A->x[idx], cy = (int)A->y[idx];
    cx = cx < 0 ? 0 : (cx >= P ? P - 1 : cx);
    cy = cy < 0 ? 0 : (cy >= Q ? Q - 1 : cy);
    return cy * P + cx;
  };
  for (int k = tid; k < total; k += nth) {
    long long idx;
    const SoA<R> *A;
    atomicAdd(&hist[cell_of(k, idx, A)], 1);
  }
  __syncthreads();
  // per segment: rank slices (warp ballots over the segment's columns)
  for (int sg = warp; sg < nseg; sg += nwarp) {
    const int row = sg / spr, c = (sg % spr) * 32 + lane;
    const int cnt = c < P ? hist[row * P + c] : 0;
    int mx = cnt;
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    int run = 0;
    for (int r = 0; r < SORT_R; ++r) {
      const unsigned m = __ballot_sync(0xffffffffu, cnt > r);
      if (lane == 0) {
        mask[sg * SORT_R + r] = m;
        sliceoff[sg * SORT_R + r] = run;
      }
      run += __popc(m);
      if (r + 1 >= mx) {
        for (int rr = r + 1 + lane; rr < SORT_R; rr += 32) mask[sg * SORT_R + rr] = 0u;
        break;
      }
    }
    if (lane == 0) segoff[sg + 1] = run;
  }
  __syncthreads();
  if (tid == 0) {
    segoff[0] = 0;
    for (int sg = 0; sg < nseg; ++sg) segoff[sg + 1] += segoff[sg];
  }
  __syncthreads();
  const int tail0 = segoff[nseg];
  for (int k = tid; k < total; k += nth) {
    long long idx;
    const SoA<R> *A;
    const int c = cell_of(k, idx, A);
    const int r = atomicAdd(&rank[c], 1);
    const int row = c / P, col = c - row * P;
    const int sg = row * spr + col / 32, bit = col % 32;
    int pos;
    if (r < SORT_R)
      pos = segoff[sg] + sliceoff[sg * SORT_R + r] +
            __popc(mask[sg * SORT_R + r] & ((1u << bit) - 1u));
    else
      pos = tail0 + atomicAdd(&s_tail, 1);
    if (pos >= cap) {
      atomicOr(err, ERR_OVERFLOW_SEG);
      continue;
    }
    const long long o = (long long)slot * cap + pos;
    dst.x[o] = A->x[idx]; dst.y[o] = A->y[idx];
    dst.ux[o] = A->ux[idx]; dst.uy[o] = A->uy[idx]; dst.uz[o] = A->uz[idx]; dst.w[o] = A->w[idx];
  }
  __syncthreads();
  if (tid == 0) cnt_dst[slot] = min(total, cap);
  // the incoming buckets have been absorbed: this block is their one reader
  if (tid >= 1 && tid < 9) {
    int k = tid - 1, ddx, ddy;
    dir_delta(k, ddx, ddy);
    const int sv = neighbour_slot(g, col0, slot, -ddx, -ddy);
    if (sv >= 0) bcnt[(long long)sv * 8 + k] = 0;
  }
}

template <typename R>
__global__ void k_copy_segments(const Geom g, SoA<R> src, const int *cnt_src, SoA<R> dst,
                                int *cnt_dst, int cap) {
  const int slot = blockIdx.x;
  const int n = min(cnt_src[slot], cap);
  const long long o = (long long)slot * cap;
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    dst.x[o + k] = src.x[o + k]; dst.y[o + k] = src.y[o + k];
    dst.ux[o + k] = src.ux[o + k]; dst.uy[o + k] = src.uy[o + k];
    dst.uz[o + k] = src.uz[o + k]; dst.w[o + k] = src.w[o + k];
  }
  if (threadIdx.x == 0) cnt_dst[slot] = n;
}

}  // namespace

size_t sort_smem(int P, int Q) {
  const int nseg = Q * ((P + 31) / 32);
  return sizeof(int) * (2 * (size_t)P * Q + nseg + 1 + 2 * (size_t)nseg * SORT_R);
}

template <typename R>
cudaError_t launch_sort_cells(const Geom &g, int col0, SoA<R> seg, int *cnt, SoA<R> scratch,
                              int *cnt_scratch, int cap, SoA<R> bkt, int *bcnt, Buckets bk,
                              unsigned *err, cudaStream_t s) {
  const size_t smem = sort_smem(g.P, g.Q);
  cudaError_t e = cudaFuncSetAttribute(k_sort_cells<R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  k_sort_cells<R><<<g.nslots, 256, smem, s>>>(g, col0, seg, cnt, cap, bkt, bcnt, bk, scratch,
                                              cnt_scratch, err);
  k_copy_segments<R><<<g.nslots, 256, 0, s>>>(g, scratch, cnt_scratch, seg, cnt, cap);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_repack(const Geom &g, SoA<R> src, const int *cnt_src, int cap_src,
                          SoA<R> bsrc, const int *bcnt_src, Buckets bk_src, SoA<R> dst,
                          int *cnt_dst, int cap_dst, SoA<R> bdst, int *bcnt_dst, Buckets bk_dst,
                          cudaStream_t s) {
  k_repack<R><<<g.nslots, 256, 0, s>>>(g, src, cnt_src, cap_src, bsrc, bcnt_src, bk_src, dst,
                                        cnt_dst, cap_dst, bdst, bcnt_dst, bk_dst);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_bin_count(const Geom &g, int col0, const double *x, const double *y, size_t n,
                             int *counts, unsigned *err, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  const int blocks = (int)((n + 255) / 256 < 65535 ? (n + 255) / 256 : 65535);
  k_bin_count<R><<<blocks, 256, 0, s>>>(g, col0, x, y, n, counts, err);
  return cudaGetLastError();
}

cudaError_t launch_clamp_counts(int *cnt, int n, int cap, cudaStream_t s) {
  k_clamp_counts<<<(n + 255) / 256, 256, 0, s>>>(cnt, n, cap);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_bin_place(const Geom &g, int col0, const double *x, const double *y,
                             const double *ux, const double *uy, const double *uz,
                             const double *w, size_t n, SoA<R> seg, int *counts, int cap,
                             unsigned *err, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  const int blocks = (int)((n + 255) / 256 < 65535 ? (n + 255) / 256 : 65535);
  k_bin_place<R><<<blocks, 256, 0, s>>>(g, col0, x, y, ux, uy, uz, w, n, seg, counts, cap, err);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_deposit_rho(const Geom &g, int col0, const PartView<R> &v, double *rho,
                               double sign, cudaStream_t s) {
  k_deposit_rho<R><<<g.nslots, 256, 0, s>>>(g, col0, v, rho, sign);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_particle_diag(const Geom &g, int col0, const PartView<R> &v, double *partials,
                                 int nblocks, cudaStream_t s) {
  k_particle_diag<R><<<nblocks, 256, 0, s>>>(g, col0, v, partials);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_get_particles(const Geom &g, int col0, const PartView<R> &v,
                                 const long long *offsets, double *out, size_t stride,
                                 cudaStream_t s) {
  k_get_particles<R><<<g.nslots, 256, 0, s>>>(g, col0, v, offsets, out, stride);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_window_particles(const Geom &g, int old_col0, int nshift, SoA<R> seg,
                                    int *cnt, SoA<R> bkt, int *bcnt, int cap, Buckets bk,
                                    double n0, double x0, double ramp, int ppcx, int ppcy,
                                    double *rho_bg, unsigned *err, cudaStream_t s) {
  k_window_migrate<R><<<g.npy, 256, 0, s>>>(g, old_col0, seg, cnt, bkt, bcnt, cap, bk, err);
  k_window_inject<R><<<dim3(g.npy, 1, inject_split(g, ppcx, ppcy)), 256, 0, s>>>(
      g, old_col0, g.npx - 1, nshift, seg, cnt, cap, n0, x0, ramp, ppcx, ppcy, rho_bg, err);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_fill_plasma(const Geom &g, int col0, int nshift, SoA<R> seg, int *cnt, int cap,
                               double n0, double x0, double ramp, int ppcx, int ppcy,
                               double *rho_bg, unsigned *err, cudaStream_t s) {
  k_window_inject<R><<<dim3(g.npy, g.npx, inject_split(g, ppcx, ppcy)), 256, 0, s>>>(
      g, col0, 0, nshift, seg, cnt, cap, n0, x0, ramp, ppcx, ppcy, rho_bg, err);
  return cudaGetLastError();
}

// Snapshot packing (pack.h): block per slot, grid-stride over the slots.
template <typename R, bool PACK>
__global__ void k_pack(const Geom g, SoA<R> seg, const int *cnt, int cap, SoA<R> bkt,
                       const int *bcnt, Buckets bk, const long long *off, R *flat,
                       long long total) {
  R *fa[6] = {flat, flat + total, flat + 2 * total, flat + 3 * total, flat + 4 * total,
              flat + 5 * total};
  R *sa[6] = {seg.x, seg.y, seg.ux, seg.uy, seg.uz, seg.w};
  R *ba[6] = {bkt.x, bkt.y, bkt.ux, bkt.uy, bkt.uz, bkt.w};
  for (int slot = blockIdx.x; slot < g.nslots; slot += gridDim.x) {
    const int n = min(cnt[slot], cap);
    const long long so = (long long)slot * cap, fo = off[9LL * slot];
    for (int k = threadIdx.x; k < n; k += blockDim.x)
#pragma unroll
      for (int a = 0; a < 6; ++a) {
        if (PACK) fa[a][fo + k] = sa[a][so + k];
        else sa[a][so + k] = fa[a][fo + k];
      }
    for (int d = 0; d < 8; ++d) {
      const int nb = min(bcnt[(long long)slot * 8 + d], bk.cap[d]);
      const long long bo = (long long)slot * bk.stride + bk.off[d], fb = off[9LL * slot + 1 + d];
      for (int k = threadIdx.x; k < nb; k += blockDim.x)
#pragma unroll
        for (int a = 0; a < 6; ++a) {
          if (PACK) fa[a][fb + k] = ba[a][bo + k];
          else ba[a][bo + k] = fa[a][fb + k];
        }
    }
  }
}

template <typename R>
cudaError_t launch_pack(const Geom &g, SoA<R> seg, const int *cnt, int cap, SoA<R> bkt,
                        const int *bcnt, Buckets bk, const long long *off, R *dst,
                        long long total, cudaStream_t s) {
  const int blocks = g.nslots < 65535 ? g.nslots : 65535;
  k_pack<R, true><<<blocks, 256, 0, s>>>(g, seg, cnt, cap, bkt, bcnt, bk, off, dst, total);
  return cudaGetLastError();
}
template <typename R>
cudaError_t launch_unpack(const Geom &g, const R *src, long long total, const long long *off,
                          SoA<R> seg, const int *cnt, int cap, SoA<R> bkt, const int *bcnt,
                          Buckets bk, cudaStream_t s) {
  const int blocks = g.nslots < 65535 ? g.nslots : 65535;
  k_pack<R, false><<<blocks, 256, 0, s>>>(g, seg, cnt, cap, bkt, bcnt, bk, off,
                                          const_cast<R *>(src), total);
  return cudaGetLastError();
}
template cudaError_t launch_pack<float>(const Geom &, SoA<float>, const int *, int, SoA<float>,
                                        const int *, Buckets, const long long *, float *,
                                        long long, cudaStream_t);
template cudaError_t launch_pack<double>(const Geom &, SoA<double>, const int *, int, SoA<double>,
                                         const int *, Buckets, const long long *, double *,
                                         long long, cudaStream_t);
template cudaError_t launch_unpack<float>(const Geom &, const float *, long long,
                                          const long long *, SoA<float>, const int *, int,
                                          SoA<float>, const int *, Buckets, cudaStream_t);
template cudaError_t launch_unpack<double>(const Geom &, const double *, long long,
                                           const long long *, SoA<double>, const int *, int,
                                           SoA<double>, const int *, Buckets, cudaStream_t);

#define PIC_INST(R)                                                                           \
  template cudaError_t launch_sort_cells<R>(const Geom &, int, SoA<R>, int *, SoA<R>, int *,   \
                                            int, SoA<R>, int *, Buckets, unsigned *,           \
                                            cudaStream_t);                                     \
  template cudaError_t launch_repack<R>(const Geom &, SoA<R>, const int *, int, SoA<R>,        \
                                        const int *, Buckets, SoA<R>, int *, int, SoA<R>,      \
                                        int *, Buckets, cudaStream_t);                         \
  template cudaError_t launch_bin_count<R>(const Geom &, int, const double *, const double *, \
                                           size_t, int *, unsigned *, cudaStream_t);          \
  template cudaError_t launch_bin_place<R>(const Geom &, int, const double *, const double *, \
                                           const double *, const double *, const double *,    \
                                           const double *, size_t, SoA<R>, int *, int,        \
                                           unsigned *, cudaStream_t);                         \
  template cudaError_t launch_deposit_rho<R>(const Geom &, int, const PartView<R> &, double *, \
                                             double, cudaStream_t);                           \
  template cudaError_t launch_particle_diag<R>(const Geom &, int, const PartView<R> &,        \
                                               double *, int, cudaStream_t);                  \
  template cudaError_t launch_get_particles<R>(const Geom &, int, const PartView<R> &,        \
                                               const long long *, double *, size_t,           \
                                               cudaStream_t);                                 \
  template cudaError_t launch_window_particles<R>(const Geom &, int, int, SoA<R>, int *,      \
                                                  SoA<R>, int *, int, Buckets, double, double, \
                                                  double, int, int, double *, unsigned *,     \
                                                  cudaStream_t);                              \
  template cudaError_t launch_fill_plasma<R>(const Geom &, int, int, SoA<R>, int *, int, double, \
                                             double, double, int, int, double *, unsigned *,  \
                                             cudaStream_t);
PIC_INST(float)
PIC_INST(double)
#undef PIC_INST

}  // namespace pic
