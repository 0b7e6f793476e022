// Patch particle step (the fine decomposition of SDMD, Section 2.2): a
// persistent grid whose blocks pull work items (a patch slot, or a chunk of
// a heavy one) from a per-step plan.  Per item:
//   1. SDMD step (ii): the patch's E and Bm tile (nodes -4..P+3 in x,
//      -1..Q+1 in y, six components) is staged into shared memory with one
//      3D TMA box copy (or plain coalesced loads); single runs issue the
//      next item's copy while the current tile is flushed;
//   2. every particle of the patch (its segment plus the particles that
//      entered from the 8 neighbours during the previous step) is
//      interpolated with the quadratic shape, pushed with the Boris scheme
//      and moved;
//   3. Esirkepov deposition (second-order shape, Section 3.2) into a shared
//      memory current tile with a 2-node halo, on the 4-node window that
//      covers both shapes (at most 40 shared atomics per particle, exact
//      zeros skipped); FP32 accumulates in 32-bit fixed point (integer
//      shared atomics), FP64 in float64;
//   4. SDMD step (i): the tile is added into the region current;
//   5. re-binning: particles that stay are compacted into the output
//      segment, particles that left are appended to the direction bucket
//      read by the destination patch at the next step (positions already
//      rebased to it), boundary conditions applied at the domain faces.
//
// The Esirkepov weights are evaluated as outer products of 1D factors:
// with DS = S1 - S0 and A = S0 + DS/2 on each axis,
//   W_x = DSx (x) A_y,  W_y = A_x (x) DSy,  W_z = A_x (x) A_y + DSx (x) DSy / 12
// (the last identity: S0xS0y + DSxS0y/2 + S0xDSy/2 + DSxDSy/3 =
// (S0x + DSx/2)(S0y + DSy/2) + DSxDSy/12), and the prefix sums of DS along
// the window end at exactly zero (sum DS = 0), written as -DS[3].
#include <cstring>

#include "common.cuh"
#include "shape.cuh"

namespace pic {

namespace {

template <typename R>
struct Vec;
template <>
struct Vec<float> {
  using T = float4;
};
template <>
struct Vec<double> {
  using T = double2;
};

// Sum of a 3 x 3 stencil at tile offset o (row stride BX).
template <typename R, int BXc>
__device__ __forceinline__ R gather(const R *T, int BXr, int o, const R Sx[3], const R Sy[3]) {
  const int BX = BXc ? BXc : BXr;
  const R *r = T + o;
  return Sy[0] * (Sx[0] * r[0] + Sx[1] * r[1] + Sx[2] * r[2]) +
         Sy[1] * (Sx[0] * r[BX] + Sx[1] * r[BX + 1] + Sx[2] * r[BX + 2]) +
         Sy[2] * (Sx[0] * r[2 * BX] + Sx[1] * r[2 * BX + 1] + Sx[2] * r[2 * BX + 2]);
}

// The 40 current contributions of one window: Jx rows l (4) x dual columns
// q (3); Jy columns q (4) x dual rows l (3); Jz 4 x 4.
template <typename R>
struct Win {
  R x[4][3], y[4][3], z[4][4];
};

// FP64 deposit: the same groups as the fixed-point FP32 deposit below
// (entries that are zero by construction skipped a group at a time: the
// window's last column (row) when the particle kept its nearest node along
// x (y), x4 / y4 false, and a whole component whose weight is zero), each
// entry an unconditional float64 shared reduction.  Volatile, without a
// memory clobber: the tile is read only after the block barrier that
// follows the particle loop, which the compiler does not move these
// statements across.
__device__ __forceinline__ void red_f64(uint32_t addr, double v) {
  asm volatile("red.shared.add.f64 [%0], %1;" ::"r"(addr), "d"(v));
}
// FIX64 (deterministic mode): the tile holds 64-bit integers, a contribution
// v adding round(v dsc) (integer sums do not depend on their order)
template <bool FIX64>
__device__ __forceinline__ void red_d(uint32_t addr, double v, double dsc) {
  if constexpr (FIX64)
    asm volatile("red.shared.add.u64 [%0], %1;" ::"r"(addr), "l"(__double2ll_rn(v * dsc)));
  else
    red_f64(addr, v);
}
template <int JWc, bool FIX64 = false>
__device__ __forceinline__ void deposit_f64(const double *Jt, int JWr, int JHW, int o,
                                            const double Px[3], const double Py[3],
                                            const double Ax[4], const double Ay[4],
                                            const double zA[4], const double zD[4],
                                            const double DSy[4], bool x4, bool y4, bool jx,
                                            bool jy, bool jz, double dsc = 0.0) {
  const int JW = JWc ? JWc : JWr;
  const uint32_t bx = smem_u32(Jt + o), by = bx + 8u * JHW, bz = by + 8u * JHW;
  auto ax = [&](int l, int q) { red_d<FIX64>(bx + 8u * (l * JW + q), Px[q] * Ay[l], dsc); };
  auto ay = [&](int q, int l) { red_d<FIX64>(by + 8u * (l * JW + q), Py[l] * Ax[q], dsc); };
  auto az = [&](int l, int q) {
    red_d<FIX64>(bz + 8u * (l * JW + q), zA[q] * Ay[l] + zD[q] * DSy[l], dsc);
  };
  if (jx) {
#pragma unroll
    for (int l = 0; l < 3; ++l) {
      ax(l, 0);
      ax(l, 1);
    }
    if (x4) {
#pragma unroll
      for (int l = 0; l < 3; ++l) ax(l, 2);
    }
    if (y4) {
      ax(3, 0);
      ax(3, 1);
      if (x4) ax(3, 2);
    }
  }
  if (jy) {
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      ay(q, 0);
      ay(q, 1);
    }
    if (y4) {
#pragma unroll
      for (int q = 0; q < 3; ++q) ay(q, 2);
    }
    if (x4) {
      ay(3, 0);
      ay(3, 1);
      if (y4) ay(3, 2);
    }
  }
  if (jz) {
#pragma unroll
    for (int l = 0; l < 3; ++l)
#pragma unroll
      for (int q = 0; q < 3; ++q) az(l, q);
    if (x4) {
#pragma unroll
      for (int l = 0; l < 3; ++l) az(l, 3);
    }
    if (y4) {
#pragma unroll
      for (int q = 0; q < 3; ++q) az(3, q);
      if (x4) az(3, 3);
    }
  }
}

// FP32 window flush into the 32-bit fixed-point current tile: each
// contribution becomes round(v scale) (native integer shared atomics; a
// contribution that rounds to zero is skipped).
template <int JWc>
__device__ __forceinline__ void flush_fixed(float *Jt, int JWr, int JHW, int o, const Win<float> &w,
                                            const float sc[3]) {
  const int JW = JWc ? JWc : JWr;
  int *Jx = reinterpret_cast<int *>(Jt) + o, *Jy = Jx + JHW, *Jz = Jx + 2 * JHW;
#pragma unroll
  for (int l = 0; l < 4; ++l)
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      const int v = __float2int_rn(w.x[l][q] * sc[0]);
      if (v != 0) atomicAdd(&Jx[l * JW + q], v);
    }
#pragma unroll
  for (int q = 0; q < 4; ++q)
#pragma unroll
    for (int l = 0; l < 3; ++l) {
      const int v = __float2int_rn(w.y[q][l] * sc[1]);
      if (v != 0) atomicAdd(&Jy[l * JW + q], v);
    }
#pragma unroll
  for (int l = 0; l < 4; ++l)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int v = __float2int_rn(w.z[l][q] * sc[2]);
      if (v != 0) atomicAdd(&Jz[l * JW + q], v);
    }
}

// A float not below v (statistics bounding the fixed-point scales).
__device__ __forceinline__ float to_float_up(float v) { return v; }
__device__ __forceinline__ float to_float_up(double v) { return __double2float_ru(v); }

// FP32 fixed-point deposit with the scale folded into the 1D factors (one
// FMA forms and rounds each contribution, see red_fixed).
// Jx[l][q] = Px[q] Ay[l], Jy[q][l] = Py[l] Ax[q], Jz[l][q] = zA[q] Ay[l] +
// zD[q] DSy[l], all already in units of the tile (scale folded into Px, Py,
// zA, zD).  Entries are issued in groups, skipping those that are zero by
// construction: the window's last column (row) when the particle kept its
// nearest node along x (y) (x4, y4 false), and a whole component whose
// weight is zero (jx, jy: no displacement along it; jz: u_z = 0).  Inside a
// group every entry is issued unconditionally (no per-entry test, so no
// branch per entry).
template <int JWc>
__device__ __forceinline__ void deposit_fixed(const float *Jt, int JWr, int JHW, int o,
                                              const float Px[3], const float Py[3],
                                              const float Ax[4], const float Ay[4],
                                              const float zA[4], const float zD[4],
                                              const float DSy[4], bool x4, bool y4, bool jx,
                                              bool jy, bool jz) {
  const int JW = JWc ? JWc : JWr;
  const uint32_t bx = smem_u32(Jt + o), by = bx + 4u * JHW, bz = by + 4u * JHW;
  auto ax = [&](int l, int q) { red_fixed(bx + 4u * (l * JW + q), fmaf(Px[q], Ay[l], kRoundMagic)); };
  auto ay = [&](int q, int l) { red_fixed(by + 4u * (l * JW + q), fmaf(Py[l], Ax[q], kRoundMagic)); };
  auto az = [&](int l, int q) {
    red_fixed(bz + 4u * (l * JW + q), fmaf(zA[q], Ay[l], zD[q] * DSy[l]) + kRoundMagic);
  };
  if (jx) {
#pragma unroll
    for (int l = 0; l < 3; ++l) {
      ax(l, 0);
      ax(l, 1);
    }
    if (x4) {
#pragma unroll
      for (int l = 0; l < 3; ++l) ax(l, 2);
    }
    if (y4) {
      ax(3, 0);
      ax(3, 1);
      if (x4) ax(3, 2);
    }
  }
  if (jy) {
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      ay(q, 0);
      ay(q, 1);
    }
    if (y4) {
#pragma unroll
      for (int q = 0; q < 3; ++q) ay(q, 2);
    }
    if (x4) {
      ay(3, 0);
      ay(3, 1);
      if (y4) ay(3, 2);
    }
  }
  if (jz) {
#pragma unroll
    for (int l = 0; l < 3; ++l)
#pragma unroll
      for (int q = 0; q < 3; ++q) az(l, q);
    if (x4) {
#pragma unroll
      for (int l = 0; l < 3; ++l) az(l, 3);
    }
    if (y4) {
#pragma unroll
      for (int q = 0; q < 3; ++q) az(3, q);
      if (x4) az(3, 3);
    }
  }
}

// The window's contributions into the current tile: FP32 in fixed point
// (or, jfloat, by value-tested float atomics), FP64 by value-tested float64
// atomics (the MERGE path's sums).
template <typename R, int JWc>
__device__ __forceinline__ void flush(R *Jt, int JWr, int JHW, int o, const Win<R> &w,
                                      const R sc[3], bool jfloat) {
  if (sizeof(R) == 4 && !jfloat) {
    flush_fixed<JWc>(reinterpret_cast<float *>(Jt), JWr, JHW, o,
                     reinterpret_cast<const Win<float> &>(w), reinterpret_cast<const float *>(sc));
  } else {
    const int JW = JWc ? JWc : JWr;
    R *Jx = Jt + o, *Jy = Jt + JHW + o, *Jz = Jt + 2 * JHW + o;
#pragma unroll
    for (int l = 0; l < 4; ++l)
#pragma unroll
      for (int q = 0; q < 3; ++q)
        if (w.x[l][q] != R(0)) atomicAdd(&Jx[l * JW + q], w.x[l][q]);
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int l = 0; l < 3; ++l)
        if (w.y[q][l] != R(0)) atomicAdd(&Jy[l * JW + q], w.y[q][l]);
#pragma unroll
    for (int l = 0; l < 4; ++l)
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (w.z[l][q] != R(0)) atomicAdd(&Jz[l * JW + q], w.z[l][q]);
  }
}

// Particle step kernel.  PT, QT: patch size known at compile time (0 =
// runtime).  MERGE: consecutive particles of a thread that share a window
// are summed in registers before one set of shared atomics.  BATCH: the
// work items of several independent runs in one launch; each item names its
// run, whose arguments and tensor map are read from device arrays.  JF
// (FP32): the current tile accumulates with float atomics instead of 32-bit
// fixed point.
template <typename R, int PT, int QT, bool TMA, bool MERGE, bool BATCH, bool JF = false>
__global__ void __launch_bounds__(256, (sizeof(R) == 4 ? (MERGE ? 2 : (JF ? 3 : 4)) : 1))
    k_particle_step(const __grid_constant__ TmapSet<BATCH ? kBatchMax : 1> tm,
                    const StepArgs<R> a0, const BatchRef<R> br) {
  // MERGE: M = 16 / sizeof(R) consecutive particles per thread, one 128-bit
  // load per array; otherwise one particle per thread per slice, lanes on
  // consecutive particles (coalesced 32/64-bit loads), which keeps the 32
  // lanes of a warp on 32 distinct, neighbouring cells for particles stored
  // in the interleaved cell order (conflict-free gathers and atomics).
  constexpr int M = MERGE ? 16 / sizeof(R) : 1;
  // FP32 fixed point with the tile scale chosen per work item (single
  // particles; the merge variant keeps the run-wide scale)
  constexpr bool FIXA = sizeof(R) == 4 && !JF && !MERGE;
  constexpr int BXc = PT ? PT + 8 : 0, BYc = QT ? QT + 3 : 0;
  constexpr int JWc = PT ? PT + 5 : 0, JHc = QT ? QT + 5 : 0;
  using V = typename Vec<R>::T;
  extern __shared__ unsigned char dsm_raw[];
  __shared__ uint64_t mbar;
  __shared__ int s_qoff[10];
  __shared__ int s_cnt[9];
  __shared__ long long s_base[9];
  __shared__ int s_item;
  __shared__ int s_ok;
  __shared__ int s_calm;
  __shared__ unsigned s_cmask;  // staged components that hold a nonzero value
  // FP32 fixed point (StepArgs::stat_in): the item's source slots' largest
  // (w |u|)^2 and w, the tile's largest |E_x|, |E_y|, |E_z|, and the
  // item's own largest (w |u|)^2 and w (float bits, non-negative)
  __shared__ unsigned s_src[2], s_emax[3], s_stat[2];
  __shared__ float s_isc;   // the item's fixed-point scale (FP32)
  __shared__ double s_dsc;  // the item's 64-bit fixed-point scale (FP64, deterministic)
  // BATCH: the current item's run arguments, copied from the device array
  __shared__ __align__(16) StepArgs<R> s_args[1];

  const int tid = threadIdx.x, nth = blockDim.x;
  const uint32_t pad = (128u - (smem_u32(dsm_raw) & 127u)) & 127u;
  if (tid < 2) s_src[tid] = s_stat[tid] = 0u;
  if (tid < 3) s_emax[tid] = 0u;
  const int lane = tid & 31;
  const Plan &plan = BATCH ? br.plan : a0.plan;
  const int n_items = *plan.n_items;
  uint32_t phase = 0;
  if (TMA && tid == 0) {
    mbar_init(&mbar, 1);
    fence_mbar_init();
  }

  // PF: the next item is fetched, and its field tile load issued, as soon
  // as the particles of the current one are done with the field tile, so
  // that the load overlaps the current tile's flush to the domain (single
  // runs; a batch's next item may belong to another run).
  constexpr bool PF = TMA && !BATCH;
  auto issue_tile = [&](int it) {
    const Geom &g0 = a0.g;
    const int P0 = PT ? PT : g0.P, Q0 = QT ? QT : g0.Q;
    const int FT0 = (BYc ? BYc : Q0 + 3) * (BXc ? BXc : P0 + 8);
    const int ss = plan.item_slot[it];
    int pxx = ss % g0.npx - a0.st->col0;
    if (pxx < 0) pxx += g0.npx;
    const int pyy = ss / g0.npx;
    R *F0 = reinterpret_cast<R *>(dsm_raw + pad);
    mbar_arrive_expect_tx(&mbar, (uint32_t)(6 * FT0 * sizeof(R)));
    tma_load_3d(F0, &tm.m[0], &mbar, pxx * P0 - 4 + GX, pyy * Q0 - 1 + GY, 0);
  };
  if (PF && tid == 0) {
    const int first = atomicAdd(plan.next, 1);
    s_item = first;
    if (first < n_items) issue_tile(first);
  }

  // Persistent loop over work items: (run, patch slot, chunk of its
  // particles), heaviest patches first, fetched from a global counter.
  for (;;) {
    __syncthreads();  // the previous item is done with the tiles
    if (!PF) {
      if (tid == 0) s_item = atomicAdd(plan.next, 1);
      __syncthreads();
    }
    const int item = s_item;
    if (item >= n_items) break;
    const int run = BATCH ? br.item_run[item] : 0;
    if (BATCH) {
      constexpr int NW = sizeof(StepArgs<R>) / 4;
      const int *src = reinterpret_cast<const int *>(br.args + run);
      int *dst = reinterpret_cast<int *>(s_args);
      for (int e = tid; e < NW; e += nth) dst[e] = src[e];
      __syncthreads();
    }
    const StepArgs<R> &a = BATCH ? s_args[0] : a0;
    // the item's fixed-point tile scale follows a bound on its contributions
    // (FP32 by default; FP64 in deterministic mode)
    const bool adapt = FIXA || (sizeof(R) == 8 && a.det != 0);
    const CUtensorMap *tmap = &tm.m[BATCH ? run : 0];
    const Geom &g = a.g;
    const int P = PT ? PT : g.P, Q = QT ? QT : g.Q;
    const int BX = BXc ? BXc : P + 8, BY = BYc ? BYc : Q + 3;  // field tile
    const int JW = JWc ? JWc : P + 5, JH = JHc ? JHc : Q + 5;  // current tile
    const int FT = BY * BX, JT = JH * JW;
    R *Ft = reinterpret_cast<R *>(dsm_raw + pad);
    R *Jt = Ft + 6 * FT;
    const R rdx = a.rdx, rdy = a.rdy, eps = a.eps;
    const R cjx = a.cjx, cjy = a.cjy, cjz = a.cjz;
    const R jsc[3] = {a.jscale[0], a.jscale[1], a.jscale[2]};
    const R ju0 = a.junit[0], ju1 = a.junit[1], ju2 = a.junit[2];
    constexpr bool jfloat = JF;
    const R RP = PT ? R(PT) : a.RP, RQ = QT ? R(QT) : a.RQ;
    const int col0 = a.st->col0;
    unsigned err = 0;
    const int s = plan.item_slot[item];
    const int ufirst = plan.item_first[item];
    const int sxs = s % g.npx, sy = s / g.npx;
    int px = sxs - col0;
    if (px < 0) px += g.npx;
    const int py = sy;
    const int X0 = px * P, Y0 = py * Q;

    // ---- 1. region -> patch field staging (SDMD step ii)
    if (TMA && !PF) {
      if (tid == 0) {
        mbar_arrive_expect_tx(&mbar, (uint32_t)(6 * FT * sizeof(R)));
        tma_load_3d(Ft, tmap, &mbar, X0 - 4 + GX, Y0 - 1 + GY, 0);
      }
    } else if (!TMA) {
      for (int e = tid; e < 6 * FT; e += nth) {
        int c = e / FT, r = e - c * FT, yy = r / BX, xx = r - yy * BX;
        Ft[e] = a.F[c * g.cs + fidx(g, X0 - 4 + xx, Y0 - 1 + yy)];
      }
    }
    {
      // current tile cleared with 16-byte stores (it starts 16-byte aligned:
      // 6 FT s bytes after the aligned field tile)
      uint4 *J4 = reinterpret_cast<uint4 *>(Jt);
      const int n4 = (int)(3 * JT * sizeof(R) / 16);
      for (int e = tid; e < n4; e += nth) J4[e] = make_uint4(0u, 0u, 0u, 0u);
      for (int e = n4 * (int)(16 / sizeof(R)) + tid; e < 3 * JT; e += nth) Jt[e] = R(0);
    }
    if (tid < 9) {
      int cnt = 0;
      long long base = 0;
      int src = s;
      if (tid == 0) {
        cnt = min(a.cnt_in[s], a.cap);
        base = (long long)s * a.cap;
        s_calm = a.calm_in[s];
      } else {
        int k = tid - 1, ddx, ddy;
        dir_delta(k, ddx, ddy);
        src = neighbour_slot(g, col0, s, -ddx, -ddy);
        if (src >= 0) {
          cnt = min(a.bcnt_in[(long long)src * 8 + k], a.bk.cap[k]);
          base = (long long)src * a.bk.stride + a.bk.off[k];
        }
      }
      if (adapt && src >= 0) {
        atomicMax(&s_src[0], a.stat_in[2 * src]);
        atomicMax(&s_src[1], a.stat_in[2 * src + 1]);
      }
      s_cnt[tid] = cnt;
      s_base[tid] = base;
    }
    __syncthreads();
    if (tid == 0) {
      s_cmask = 0u;
      s_qoff[0] = 0;
      for (int i = 0; i < 9; ++i) s_qoff[i + 1] = s_qoff[i] + (s_cnt[i] + M - 1) / M;
      int ok = 1;
      if (TMA) {
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
    const int totalq = min(ufirst + plan.chunk, s_qoff[9]);
    // A patch whose staged E and Bm are exactly zero (plasma the laser has
    // not reached yet): a particle at rest there stays at rest, in place,
    // and deposits nothing (exactly what the full step computes), so it is
    // copied through without the interpolation, push and deposit.
    // (16-byte words of the tile, sign bits masked: -0 counts as zero; the
    // tile holds a multiple of 16 bytes since P is a multiple of 16 / s)
    // (also per component: a component that is zero over the whole tile,
    // e.g. E_z, B_x, B_y of a field polarised in the plane, is not gathered)
    {
      unsigned cmask = 0;
      const uint4 *F4 = reinterpret_cast<const uint4 *>(Ft);
      const int wc = (int)(FT * sizeof(R) / 16);  // 16-byte words per component
      unsigned em[3] = {0u, 0u, 0u};  // FIXA: largest |E_c| bits seen
#pragma unroll
      for (int c = 0; c < 6; ++c) {
        unsigned any = 0u, mx = 0u;
        for (int e = tid; e < wc; e += nth) {
          const uint4 v = F4[c * wc + e];
          if (sizeof(R) == 4) {
            const unsigned ax = v.x & 0x7fffffffu, ay = v.y & 0x7fffffffu,
                           az = v.z & 0x7fffffffu, aw = v.w & 0x7fffffffu;
            any |= ax | ay | az | aw;
            if (FIXA && c < 3) mx = max(mx, max(max(ax, ay), max(az, aw)));
          } else {
            any |= v.x | v.z | ((v.y | v.w) & 0x7fffffffu);
            // FP64: the high words (sign masked) of the two values; their
            // largest + 1, shifted up, bounds the largest |value|
            if (adapt && c < 3) mx = max(mx, max(v.y & 0x7fffffffu, v.w & 0x7fffffffu));
          }
        }
        if (any) cmask |= 1u << c;
        if (c < 3) em[c] = mx;
      }
      cmask = __reduce_or_sync(0xffffffffu, cmask);
      if (lane == 0 && cmask) atomicOr(&s_cmask, cmask);
      if (adapt) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const unsigned m = __reduce_max_sync(0xffffffffu, em[c]);
          if (lane == 0 && m) atomicMax(&s_emax[c], m);
        }
      }
    }
    __syncthreads();
    const unsigned cmask = s_cmask;
    const bool quiet = cmask == 0u;
    // A calm slot (the previous step found its particles at rest in a zero
    // tile with nothing arriving, so both segment sets hold the same
    // particles) that is still calm is skipped: its output set already
    // holds its particles, unchanged.  Only the count is carried over.
    const bool arrivals = (s_cnt[1] | s_cnt[2] | s_cnt[3] | s_cnt[4] | s_cnt[5] | s_cnt[6] |
                           s_cnt[7] | s_cnt[8]) != 0;
    const bool skip = quiet && !arrivals && s_calm;
    if (skip && tid == 0 && ufirst == 0) {
      a.cnt_out[s] = s_cnt[0];
      atomicAdd(&a.st->calm_particles, (unsigned long long)s_cnt[0]);
    }
    bool moving = false;  // a particle of this item had u != 0
    float st_wu2 = 0.0f, st_w = 0.0f;  // this thread's largest (w |u|)^2, w
    // this item's tile scale, formed once by thread 0
    if (adapt && !skip) {
      if (tid == 0) {
        auto emax_of = [&](unsigned m) -> float {
          if (sizeof(R) == 4) return __uint_as_float(m);
          return m ? __double2float_ru(__longlong_as_double((long long)(m + 1u) << 32)) : 0.0f;
        };
        const float ex = emax_of(s_emax[0]), ey = emax_of(s_emax[1]), ez = emax_of(s_emax[2]);
        const float m1 = sqrtf(__uint_as_float(s_src[0])), m2 = __uint_as_float(s_src[1]);
        const float emax = sqrtf(ex * ex + ey * ey + ez * ez);
        // bound on w |v| after the push, with a margin for rounding
        float B = fminf(fminf(fmaf(2.0f * fabsf((float)eps) * emax, m2, m1), m2), (float)a.wglob);
        B = fmaxf(B * 1.001f, 1e-30f);
        const int n = totalq - ufirst;
        const int lg = n > 1 ? 32 - __clz(n - 1) : 0;
        if (sizeof(R) == 4) {
          const int K = min(30 - lg, 20);
          s_isc = __int_as_float((127 + K) << 23) * (float)a.jk / B;
        } else {
          // FP64 deterministic mode: 64-bit fixed point, K = 62 - ceil(log2
          // n): every contribution below (4/3) 2^K, an item's sums below
          // (4/3) 2^62
          s_dsc = ldexp((double)a.jk, 62 - lg) / (double)B;
        }
      }
      __syncthreads();
    }
    const R isc = FIXA ? R(s_isc) : R(0);
    const R dsc = (sizeof(R) == 8 && a.det) ? R(s_dsc) : R(1);  // read only in deterministic FP64

  // particles of work item qi (M consecutive of one source) -> registers
  auto load = [&](int qi, R(&x)[M], R(&y)[M], R(&ux)[M], R(&uy)[M], R(&uz)[M], R(&w)[M]) {
    int nval = 0;
#pragma unroll
    for (int m = 0; m < M; ++m) x[m] = y[m] = ux[m] = uy[m] = uz[m] = w[m] = R(0);
    if (qi < totalq) {
      int src = 0;
      while (src < 8 && qi >= s_qoff[src + 1]) ++src;
      const int k0 = (qi - s_qoff[src]) * M;
      nval = min(M, s_cnt[src] - k0);
      // checked build: the source's elements stay inside its segment or bucket
      if (!PIC_IN(err, k0 >= 0 && k0 + nval <= (src == 0 ? a.cap : a.bk.cap[src - 1]))) return 0;
      const SoA<R> &A = src == 0 ? a.pin : a.bin;
      const long long b = s_base[src] + k0;
      if (M > 1 && nval == M) {
        const V vx = *reinterpret_cast<const V *>(A.x + b);
        const V vy = *reinterpret_cast<const V *>(A.y + b);
        const V vux = *reinterpret_cast<const V *>(A.ux + b);
        const V vuy = *reinterpret_cast<const V *>(A.uy + b);
        const V vuz = *reinterpret_cast<const V *>(A.uz + b);
        const V vw = *reinterpret_cast<const V *>(A.w + b);
        memcpy(x, &vx, sizeof vx);
        memcpy(y, &vy, sizeof vy);
        memcpy(ux, &vux, sizeof vux);
        memcpy(uy, &vuy, sizeof vuy);
        memcpy(uz, &vuz, sizeof vuz);
        memcpy(w, &vw, sizeof vw);
      } else {
#pragma unroll
        for (int m = 0; m < M; ++m)
          if (m < nval) {
            x[m] = A.x[b + m]; y[m] = A.y[b + m];
            ux[m] = A.ux[b + m]; uy[m] = A.uy[b + m]; uz[m] = A.uz[b + m]; w[m] = A.w[b + m];
          }
      }
    }
    return nval;
  };
  R x[M], y[M], ux[M], uy[M], uz[M], w[M];
  int nval = skip ? 0 : load(ufirst + tid, x, y, ux, uy, uz, w);
  for (int qb = ufirst; qb < (skip ? ufirst : totalq); qb += nth) {
    // prefetch the next work item so its global loads overlap this one
    R nx_[M], ny_[M], nux_[M], nuy_[M], nuz_[M], nw_[M];
    const int nnval = load(qb + nth + tid, nx_, ny_, nux_, nuy_, nuz_, nw_);
    Win<R> acc;
    int key = -1;
#pragma unroll
    for (int m = 0; m < M; ++m) {
      int dir = -2;  // -1 stay, -2 gone / invalid, 0..7 bucket
      R x1 = R(0), y1 = R(0), nux = R(0), nuy = R(0), nuz = R(0);
      moving |= m < nval && (ux[m] != R(0) || uy[m] != R(0) || uz[m] != R(0));
      if (adapt && m < nval) st_w = fmaxf(st_w, to_float_up(w[m]));
      if (m < nval && quiet && ux[m] == R(0) && uy[m] == R(0) && uz[m] == R(0)) {
        x1 = x[m];
        y1 = y[m];
        dir = -1;
      } else if (m < nval) {
        // interpolation at x^n with the shape of each component's stagger
        int ip, id, jp, jd;
        R Sxp[3], Sxd[3], Syp[3], Syd[3];
        shapes(x[m], ip, Sxp, id, Sxd);
        shapes(y[m], jp, Syp, jd, Syd);
        // tile offsets: column node n -> n + 3 (tile starts at node -4,
        // stencil at n - 1); row node n -> n (tile starts at node -1)
        const int opp = jp * BX + ip + 3, opd = jd * BX + ip + 3;
        const int odp = jp * BX + id + 3, odd = jd * BX + id + 3;
        // checked build: every 3 x 3 stencil inside its component's tile
        const unsigned gm =
            PIC_IN(err, min(min(opp, opd), min(odp, odd)) >= 0 &&
                            max(max(opp, opd), max(odp, odd)) + 2 * BX + 2 < FT)
                ? cmask
                : 0u;
        const R Ex = (gm & 1u) ? gather<R, BXc>(Ft, BX, odp, Sxd, Syp) : R(0);
        const R Ey = (gm & 2u) ? gather<R, BXc>(Ft + FT, BX, opd, Sxp, Syd) : R(0);
        const R Ez = (gm & 4u) ? gather<R, BXc>(Ft + 2 * FT, BX, opp, Sxp, Syp) : R(0);
        const R Bx = (gm & 8u) ? gather<R, BXc>(Ft + 3 * FT, BX, opd, Sxp, Syd) : R(0);
        const R By = (gm & 16u) ? gather<R, BXc>(Ft + 4 * FT, BX, odp, Sxd, Syp) : R(0);
        const R Bz = (gm & 32u) ? gather<R, BXc>(Ft + 5 * FT, BX, odd, Sxd, Syd) : R(0);
        // Boris push u^{n-1/2} -> u^{n+1/2}
        const R umx = ux[m] + eps * Ex, umy = uy[m] + eps * Ey, umz = uz[m] + eps * Ez;
        const R ig = eps * rsq(R(1) + umx * umx + umy * umy + umz * umz);
        const R tx = ig * Bx, ty = ig * By, tz = ig * Bz;
        const R f = quot(R(2), R(1) + tx * tx + ty * ty + tz * tz);
        const R upx = umx + (umy * tz - umz * ty);
        const R upy = umy + (umz * tx - umx * tz);
        const R upz = umz + (umx * ty - umy * tx);
        nux = umx + f * (upy * tz - upz * ty) + eps * Ex;
        nuy = umy + f * (upz * tx - upx * tz) + eps * Ey;
        nuz = umz + f * (upx * ty - upy * tx) + eps * Ez;
        const R usq = nux * nux + nuy * nuy + nuz * nuz;
        const R inv = rsq(R(1) + usq);
        if (adapt) st_wu2 = fmaxf(st_wu2, to_float_up(w[m] * w[m] * usq));
        x1 = x[m] + rdx * nux * inv;
        y1 = y[m] + rdy * nuy * inv;
        R S1x3[3], S1y3[3];
        const int i1 = shape_primal(x1, S1x3);
        const int j1 = shape_primal(y1, S1y3);
        const int di = i1 - ip, dj = j1 - jp;
        const bool finite = isfinite(x1) && isfinite(y1) && isfinite(nux) && isfinite(nuy) &&
                            isfinite(nuz);
        const bool slow = di >= -1 && di <= 1 && dj >= -1 && dj <= 1;
        if (!finite) err |= ERR_NONFINITE;
        else if (!slow) err |= ERR_FAST;
        if (finite && slow) {
          // Esirkepov weights on the 4-node window covering S(x^n), S(x^{n+1})
          const bool shx = di < 0, shy = dj < 0;
          R S0x[4], S1x[4], S0y[4], S1y[4], DSx[4], DSy[4], Ax[4], Ay[4];
          window4(Sxp, shx, S0x);
          window4(S1x3, di + (shx ? 1 : 0) != 0, S1x);
          window4(Syp, shy, S0y);
          window4(S1y3, dj + (shy ? 1 : 0) != 0, S1y);
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            DSx[c] = S1x[c] - S0x[c];
            DSy[c] = S1y[c] - S0y[c];
            Ax[c] = S0x[c] + R(0.5) * DSx[c];
            Ay[c] = S0y[c] + R(0.5) * DSy[c];
          }
          // FP32 fixed point (single particles): the tile scale folded into
          // the per-particle factors
          constexpr bool FIX = sizeof(R) == 4 && !JF && !MERGE;
          const R wx = (FIX ? cjx * isc : cjx) * w[m];
          const R wy = (FIX ? cjy * isc : cjy) * w[m];
          const R wz = (FIX ? cjz * isc : cjz) * w[m] * nuz * inv;
          const R Px[3] = {wx * DSx[0], wx * (DSx[0] + DSx[1]), -wx * DSx[3]};
          const R Py[3] = {wy * DSy[0], wy * (DSy[0] + DSy[1]), -wy * DSy[3]};
          R zA[4], zD[4];
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            zA[c] = wz * Ax[c];
            zD[c] = (wz * R(1.0 / 12.0)) * DSx[c];
          }
          Win<R> cur;
          if constexpr (MERGE || (sizeof(R) == 4 && JF)) {
#pragma unroll
            for (int l = 0; l < 4; ++l)
#pragma unroll
              for (int q = 0; q < 3; ++q) cur.x[l][q] = Px[q] * Ay[l];
#pragma unroll
            for (int q = 0; q < 4; ++q)
#pragma unroll
              for (int l = 0; l < 3; ++l) cur.y[q][l] = Py[l] * Ax[q];
#pragma unroll
            for (int l = 0; l < 4; ++l)
#pragma unroll
              for (int q = 0; q < 4; ++q) cur.z[l][q] = zA[q] * Ay[l] + zD[q] * DSy[l];
          }
          // window origin in the current tile (tile starts at node -2)
          const int o = (jp - 1 - (shy ? 1 : 0) + 2) * JW + ip - 1 - (shx ? 1 : 0) + 2;
          if (MERGE) {
            if (o == key) {
#pragma unroll
              for (int l = 0; l < 4; ++l)
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                  acc.x[l][q] += cur.x[l][q];
                  acc.y[l][q] += cur.y[l][q];
                }
#pragma unroll
              for (int l = 0; l < 4; ++l)
#pragma unroll
                for (int q = 0; q < 4; ++q) acc.z[l][q] += cur.z[l][q];
            } else {
              if (key >= 0) flush<R, JWc>(Jt, JW, JT, key, acc, jsc, jfloat);
              acc = cur;
              key = o;
            }
          } else if ((x1 != x[m] || y1 != y[m] || nuz != R(0)) &&
                     PIC_IN(err, o >= 0 && o + 3 * JW + 3 < JT)) {  // window in the tile
            // (a particle that did not move deposits nothing).  FP64 skips
            // the structural zeros by integer flags (an FP64 compare per
            // entry costs FP64-pipe slots, the path's bound); FP32 converts
            // each entry to fixed point and skips the zeros.
            if constexpr (sizeof(R) == 8) {
              const double *dPx = reinterpret_cast<const double *>(Px);
              const double *dPy = reinterpret_cast<const double *>(Py);
              const double *dAx = reinterpret_cast<const double *>(Ax);
              const double *dAy = reinterpret_cast<const double *>(Ay);
              const double *dzA = reinterpret_cast<const double *>(zA);
              const double *dzD = reinterpret_cast<const double *>(zD);
              const double *dDSy = reinterpret_cast<const double *>(DSy);
              const bool fx = wx != R(0) && x1 != x[m], fy = wy != R(0) && y1 != y[m];
              if (a.det)
                deposit_f64<JWc, true>(reinterpret_cast<const double *>(Jt), JW, JT, o, dPx, dPy,
                                       dAx, dAy, dzA, dzD, dDSy, di != 0, dj != 0, fx, fy,
                                       wz != R(0), (double)dsc);
              else
                deposit_f64<JWc>(reinterpret_cast<const double *>(Jt), JW, JT, o, dPx, dPy, dAx,
                                 dAy, dzA, dzD, dDSy, di != 0, dj != 0, fx, fy, wz != R(0));
            }
            else if constexpr (FIX)
              deposit_fixed<JWc>(reinterpret_cast<const float *>(Jt), JW, JT, o,
                                 reinterpret_cast<const float *>(Px),
                                 reinterpret_cast<const float *>(Py),
                                 reinterpret_cast<const float *>(Ax),
                                 reinterpret_cast<const float *>(Ay),
                                 reinterpret_cast<const float *>(zA),
                                 reinterpret_cast<const float *>(zD),
                                 reinterpret_cast<const float *>(DSy), di != 0, dj != 0,
                                 x1 != x[m], y1 != y[m], nuz != R(0));
            else
              flush<R, JWc>(Jt, JW, JT, o, cur, jsc, jfloat);
          }
          // boundary conditions at domain faces, then destination patch
          int ddx = 0, ddy = 0;
          if (x1 < R(0)) ddx = -1; else if (x1 >= RP) ddx = 1;
          if (y1 < R(0)) ddy = -1; else if (y1 >= RQ) ddy = 1;
          bool gone = false;
          if (ddx != 0 && (px + ddx < 0 || px + ddx >= g.npx)) {
            const int bc = g.pbc[0][ddx > 0];
            if (bc == PBC_REFLECT) {
              x1 = ddx < 0 ? -x1 : R(2 * P) - x1;
              if (x1 >= RP) x1 = below(RP);
              nux = -nux;
              ddx = 0;
            } else if (bc == PBC_REMOVE) {
              gone = true;
            }
          }
          if (ddy != 0 && (py + ddy < 0 || py + ddy >= g.npy)) {
            const int bc = g.pbc[1][ddy > 0];
            if (bc == PBC_REFLECT) {
              y1 = ddy < 0 ? -y1 : R(2 * Q) - y1;
              if (y1 >= RQ) y1 = below(RQ);
              nuy = -nuy;
              ddy = 0;
            } else if (bc == PBC_REMOVE) {
              gone = true;
            }
          }
          if (!gone) {
            if (ddx < 0) { x1 += RP; if (x1 >= RP) x1 = below(RP); }
            else if (ddx > 0) x1 -= RP;
            if (ddy < 0) { y1 += RQ; if (y1 >= RQ) y1 = below(RQ); }
            else if (ddy > 0) y1 -= RQ;
            dir = (ddx == 0 && ddy == 0) ? -1 : dir_index(ddx, ddy);
          }
        }
      }
      // compaction of the particles that stay (warp ballot, one shared
      // atomic per warp), exits appended to their direction bucket
      const bool stay = dir == -1;
      const unsigned bal = __ballot_sync(0xffffffffu, stay);
      int wbase = 0;
      if (lane == 0 && bal) wbase = atomicAdd(&a.cnt_out[s], __popc(bal));
      wbase = __shfl_sync(0xffffffffu, wbase, 0);
      if (stay) {
        const int pos = wbase + __popc(bal & ((1u << lane) - 1u));
        if (pos < a.cap) {
          const long long i = (long long)s * a.cap + pos;
          a.pout.x[i] = x1; a.pout.y[i] = y1;
          a.pout.ux[i] = nux; a.pout.uy[i] = nuy; a.pout.uz[i] = nuz; a.pout.w[i] = w[m];
        } else {
          err |= ERR_OVERFLOW_SEG;
        }
      } else if (dir >= 0) {
        const int bp = atomicAdd(&a.bcnt_out[(long long)s * 8 + dir], 1);
        if (bp < a.bk.cap[dir]) {
          const long long i = (long long)s * a.bk.stride + a.bk.off[dir] + bp;
          a.bout.x[i] = x1; a.bout.y[i] = y1;
          a.bout.ux[i] = nux; a.bout.uy[i] = nuy; a.bout.uz[i] = nuz; a.bout.w[i] = w[m];
        } else {
          err |= ERR_OVERFLOW_BKT;
        }
      }
    }
    if (MERGE && key >= 0) flush<R, JWc>(Jt, JW, JT, key, acc, jsc, jfloat);
#pragma unroll
    for (int m = 0; m < M; ++m) {
      x[m] = nx_[m]; y[m] = ny_[m]; ux[m] = nux_[m]; uy[m] = nuy_[m]; uz[m] = nuz_[m];
      w[m] = nw_[m];
    }
    nval = nnval;
  }
    if (adapt) {
      const unsigned m1 = __reduce_max_sync(0xffffffffu, __float_as_uint(st_wu2));
      const unsigned m2 = __reduce_max_sync(0xffffffffu, __float_as_uint(st_w));
      if (lane == 0 && m1) atomicMax(&s_stat[0], m1);
      if (lane == 0 && m2) atomicMax(&s_stat[1], m2);
    }
    // the slot stays calm only if every item of it was calm (its output is
    // then a copy of its input)
    const bool moved = __syncthreads_or(moving) != 0;
    if (tid == 0 && !skip && (!quiet || arrivals || moved)) a.calm_out[s] = 0;
    if (adapt && tid == 0) {
      // a skipped slot keeps its particles, hence its maxima
      const unsigned m1 = skip ? a.stat_in[2 * s] : s_stat[0];
      const unsigned m2 = skip ? a.stat_in[2 * s + 1] : s_stat[1];
      if (m1) atomicMax(&a.stat_out[2 * s], m1);
      if (m2) atomicMax(&a.stat_out[2 * s + 1], m2);
      s_stat[0] = s_stat[1] = 0u;
      s_src[0] = s_src[1] = 0u;
      s_emax[0] = s_emax[1] = s_emax[2] = 0u;
    }
    // the field tile is free: fetch the next item and start its tile load
    if (PF && tid == 0) {
      const int nxt = atomicAdd(plan.next, 1);
      s_item = nxt;
      if (nxt < n_items) issue_tile(nxt);
    }
    // ---- SDMD step (i): patch current tile -> region current (deterministic
    // mode: the whole tile stored for the fixed-order reduction)
    const R iju = FIXA && !skip ? R(1) / isc : R(0);
    const bool det = a.det != 0;
    if (det && !skip && tid == 0) a.jflag[s] = 1;
    for (int e = skip ? 3 * JT : tid; e < 3 * JT; e += nth) {
      R v;
      if (sizeof(R) == 4 && !jfloat) {
        const int iv = reinterpret_cast<const int *>(Jt)[e];
        const int c = e / JT;
        v = iv ? R(iv) * (FIXA ? iju : (c == 0 ? ju0 : (c == 1 ? ju1 : ju2))) : R(0);
      } else if (sizeof(R) == 8 && det) {
        const long long iv = reinterpret_cast<const long long *>(Jt)[e];
        v = iv ? R((double)iv / (double)dsc) : R(0);
      } else {
        v = Jt[e];
      }
      if (det) {
        a.jbuf[(long long)s * 3 * JT + e] = v;
      } else if (v != R(0)) {
        const int c = e / JT, r = e - c * JT, l = r / JW, q = r - l * JW;
        int gi = X0 - 2 + q, gj = Y0 - 2 + l;
        if (g.fbc_x == FBC_PERIODIC) gi = gi < 0 ? gi + g.nx : (gi >= g.nx ? gi - g.nx : gi);
        if (g.fbc_y == FBC_PERIODIC) gj = gj < 0 ? gj + g.ny : (gj >= g.ny ? gj - g.ny : gj);
        // checked build: the node inside the stored region
        if (PIC_IN(err, gi >= -GX && gi < g.nx + GX && gj >= -GY && gj < g.ny + GY))
          atomicAdd(&a.Jdst[c * g.cs + fidx(g, gi, gj)], v);
      }
    }
    if (tid == 0) atomicMax(&a.st->maxcnt[a.parity], atomicAdd(&a.cnt_out[s], 0));
    if (err) atomicOr(&a.st->err, err);
  }
}

// Plan of one step: units per slot (segment plus incoming buckets, counts
// clamped to the capacities), items per slot, items ordered by decreasing
// item count of their slot (classes of one item count, heaviest first);
// the output counts of the step are cleared here (zero_out) and its calm
// flags set, after the previous state's counts are copied aside: those of
// the step's inputs, or (prev_from_out: a plan built ahead, while the step
// before is still the most recent one) the ones its outputs hold.  BATCH: the slots of all
// runs, flattened (run r owns flat slots [br.slots.off[r], off[r + 1])).
constexpr int PLAN_CLASSES = 64;
// Class of a slot with `items` work items: slots that were calm at the
// previous step (likely skipped again, so cheap) form the last class;
// the others go heaviest first.
__device__ __forceinline__ int plan_class(int items, unsigned char calm) {
  return calm ? 0 : min(items, PLAN_CLASSES - 1);
}

template <typename R, bool BATCH>
__global__ void __launch_bounds__(1024) k_plan(const StepArgs<R> a0, const BatchRef<R> br,
                                               bool zero_out, bool prev_from_out) {
  __shared__ int hist[PLAN_CLASSES], off[PLAN_CLASSES];
  const int tid = threadIdx.x, nth = blockDim.x;
  const Plan &plan = BATCH ? br.plan : a0.plan;
  const int u = plan.unit;
  const int nflat = BATCH ? br.slots.off[br.slots.n] : a0.g.nslots;
  for (int c = tid; c < PLAN_CLASSES; c += nth) hist[c] = 0;
  __syncthreads();
  for (int f = tid; f < nflat; f += nth) {
    const int run = BATCH ? batch_run(br.slots.off, br.slots.n, f) : 0;
    const StepArgs<R> &a = BATCH ? br.args[run] : a0;
    const int s = BATCH ? f - br.slots.off[run] : f;
    const int col0 = a.st->col0;
    int units = (min(a.cnt_in[s], a.cap) + u - 1) / u;
    for (int d = 0; d < 8; ++d) {
      int ddx, ddy;
      dir_delta(d, ddx, ddy);
      const int src = neighbour_slot(a.g, col0, s, -ddx, -ddy);
      if (src >= 0) units += (min(a.bcnt_in[(long long)src * 8 + d], a.bk.cap[d]) + u - 1) / u;
    }
    plan.units[f] = units;
    if (zero_out && a.cnt_prev) {
      a.cnt_prev[s] = prev_from_out ? a.cnt_out[s] : a.cnt_in[s];
      for (int d = 0; d < 8; ++d)
        a.bcnt_prev[(long long)s * 8 + d] =
            prev_from_out ? a.bcnt_out[(long long)s * 8 + d] : a.bcnt_in[(long long)s * 8 + d];
    }
    if (zero_out) {
      a.cnt_out[s] = 0;
      for (int d = 0; d < 8; ++d) a.bcnt_out[(long long)s * 8 + d] = 0;
      a.calm_out[s] = 1;
      if (a.stat_out) a.stat_out[2 * s] = a.stat_out[2 * s + 1] = 0u;
      if (a.det) a.jflag[s] = 0;
    }
    const int items = (units + plan.chunk - 1) / plan.chunk;
    if (items) atomicAdd(&hist[plan_class(items, a.calm_in[s])], items);
  }
  __syncthreads();
  if (tid == 0) {
    int run = 0;
    for (int c = PLAN_CLASSES - 1; c >= 0; --c) {
      off[c] = run;
      run += hist[c];
    }
    *plan.n_items = min(run, plan.max_items);
    *plan.next = 0;
  }
  __syncthreads();
  for (int f = tid; f < nflat; f += nth) {
    const int items = (plan.units[f] + plan.chunk - 1) / plan.chunk;
    if (!items) continue;
    const int run = BATCH ? batch_run(br.slots.off, br.slots.n, f) : 0;
    const int s = BATCH ? f - br.slots.off[run] : f;
    const StepArgs<R> &a = BATCH ? br.args[run] : a0;
    const int base = atomicAdd(&off[plan_class(items, a.calm_in[s])], items);
    for (int k = 0; k < items && base + k < plan.max_items; ++k) {
      plan.item_slot[base + k] = s;
      plan.item_first[base + k] = k * plan.chunk;
      if (BATCH) br.item_run[base + k] = run;
    }
  }
}

// Deterministic mode: the region current of every stored node (periodic
// axes: [0, n); open axes: the ghost band included) is the sum, in a fixed
// order (patch rows ascending, then columns), of the entries of the stored
// tiles that cover it (a tile spans nodes -2 .. P+2 of its patch; periodic
// images wrap).  BATCH: block b works on run batch_run(bg, b).
__device__ __forceinline__ int floor_div(int a, int b) { return a >= 0 ? a / b : -((-a + b - 1) / b); }

template <typename R, bool BATCH>
__global__ void __launch_bounds__(256) k_gather_current(const StepArgs<R> a0, const BatchRef<R> br,
                                                        const BatchGrid bg) {
  const int run = BATCH ? batch_run(bg.off, bg.n, blockIdx.x) : 0;
  const StepArgs<R> &a = BATCH ? br.args[run] : a0;
  const Geom &g = a.g;
  const int b = BATCH ? blockIdx.x - bg.off[run] : blockIdx.x;
  const bool px_per = g.fbc_x == FBC_PERIODIC, py_per = g.fbc_y == FBC_PERIODIC;
  const int i0 = px_per ? 0 : -GX, j0 = py_per ? 0 : -GY;
  const int ni = px_per ? g.nx : g.nx + 2 * GX, nj = py_per ? g.ny : g.ny + 2 * GY;
  const int e = b * blockDim.x + threadIdx.x;
  if (e >= ni * nj) return;
  const int i = i0 + e % ni, j = j0 + e / ni;
  const int JW = g.P + 5, JH = g.Q + 5, JT = JW * JH;
  const int col0 = a.st->col0;
  R acc[3] = {R(0), R(0), R(0)};
  for (int pyu = floor_div(j + 2 - JH + 1, g.Q); pyu <= floor_div(j + 2, g.Q); ++pyu) {
    const int l = j + 2 - pyu * g.Q;
    if (l < 0 || l >= JH) continue;
    int py = pyu;
    if (py < 0 || py >= g.npy) {
      if (!py_per) continue;
      py = ((py % g.npy) + g.npy) % g.npy;
    }
    for (int pxu = floor_div(i + 2 - JW + 1, g.P); pxu <= floor_div(i + 2, g.P); ++pxu) {
      const int q = i + 2 - pxu * g.P;
      if (q < 0 || q >= JW) continue;
      int px = pxu;
      if (px < 0 || px >= g.npx) {
        if (!px_per) continue;
        px = ((px % g.npx) + g.npx) % g.npx;
      }
      const int slot = py * g.npx + (px + col0) % g.npx;
      if (!a.jflag[slot]) continue;
      const R *t = a.jbuf + (long long)slot * 3 * JT + l * JW + q;
      acc[0] += t[0];
      acc[1] += t[JT];
      acc[2] += t[2 * JT];
    }
  }
  const long long o = fidx(g, i, j);
  for (int c = 0; c < 3; ++c) a.Jdst[c * g.cs + o] = acc[c];
}

template <typename R, int PT, int QT, bool TMA, bool MERGE, bool BATCH, bool JF>
const void *kernel_ptr() {
  return (const void *)k_particle_step<R, PT, QT, TMA, MERGE, BATCH, JF>;
}

// Kernel for a patch shape: compile-time tile sizes for the common square
// patches, a runtime-size kernel otherwise; plain loads always runtime-size.
// Batched launches (runs may differ in patch size) use runtime sizes unless
// every run shares the patch shape.
template <typename R, bool MERGE, bool BATCH, bool JF = false>
const void *pick(int P, int Q, bool tma) {
  if (!tma) return kernel_ptr<R, 0, 0, false, MERGE, BATCH, JF>();
  if (P == 32 && Q == 32) return kernel_ptr<R, 32, 32, true, MERGE, BATCH, JF>();
  if (P == 16 && Q == 16) return kernel_ptr<R, 16, 16, true, MERGE, BATCH, JF>();
  if (P == 8 && Q == 8) return kernel_ptr<R, 8, 8, true, MERGE, BATCH, JF>();
  return kernel_ptr<R, 0, 0, true, MERGE, BATCH, JF>();
}

// jfloat (FP32 float-atomic current tile) has its own single-run kernels;
// batches and the merge variant accumulate in fixed point.
template <typename R>
const void *pick_kernel(int P, int Q, bool tma, bool merge, bool batch = false,
                        bool jfloat = false) {
  if (batch) return pick<R, false, true>(P, Q, tma);  // batches: one particle per thread
  if (merge) return pick<R, true, false>(P, Q, tma);
  if constexpr (sizeof(R) == 4) {
    if (jfloat) return pick<R, false, false, true>(P, Q, tma);
  }
  return pick<R, false, false>(P, Q, tma);
}

}  // namespace

size_t particle_step_smem(int P, int Q, size_t rsize) {
  return (size_t)(6 * (Q + 3) * (P + 8) + 3 * (Q + 5) * (P + 5)) * rsize + 128;
}

template <typename R>
cudaError_t prepare_particle_step(int P, int Q) {
  const int smem = (int)particle_step_smem(P, Q, sizeof(R));
  for (int t = 0; t < 2; ++t)
    for (int mg = 0; mg < 3; ++mg) {
      cudaError_t e = cudaFuncSetAttribute(pick_kernel<R>(P, Q, t != 0, mg == 1, false, mg == 2),
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
      if (e != cudaSuccess) return e;
    }
  return cudaSuccess;
}

template <typename R>
cudaError_t prepare_particle_step_batch(int P, int Q, size_t smem) {
  for (int t = 0; t < 2; ++t) {
    cudaError_t e = cudaFuncSetAttribute(pick_kernel<R>(P, Q, t != 0, false, true),
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

namespace {
int resident_grid(const void *k, int block, size_t smem) {
  int per_sm = 0, dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, block, smem) != cudaSuccess)
    return 0;
  return per_sm * nsm;
}
}  // namespace

template <typename R>
int particle_step_grid(int P, int Q, bool tma, bool merge, int block, bool jfloat) {
  return resident_grid(pick_kernel<R>(P, Q, tma, merge, false, jfloat), block,
                       particle_step_smem(P, Q, sizeof(R)));
}

template <typename R>
int particle_step_batch_grid(int P, int Q, bool tma, int block, size_t smem) {
  return resident_grid(pick_kernel<R>(P, Q, tma, false, true), block, smem);
}

template <typename R>
cudaError_t launch_plan(const StepArgs<R> &a, bool ahead, cudaStream_t s) {
  BatchRef<R> none{};
  k_plan<R, false><<<1, 1024, 0, s>>>(a, none, true, ahead);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_particle_step(const StepArgs<R> &a, const CUtensorMap *tmap, bool tma,
                                 bool merge, int block, int grid, bool plan, cudaStream_t s) {
  BatchRef<R> none{};
  if (plan) {
    k_plan<R, false><<<1, 1024, 0, s>>>(a, none, true, false);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  const size_t smem = particle_step_smem(a.g.P, a.g.Q, sizeof(R));
  const void *k = pick_kernel<R>(a.g.P, a.g.Q, tma, merge, false, a.jfloat != 0);
  TmapSet<1> tm;
  tm.m[0] = *tmap;
  void *args[] = {(void *)&tm, (void *)&a, (void *)&none};
  return cudaLaunchKernel(k, dim3(grid), dim3(block), args, smem, s);
}

// P, Q: the runs' common patch shape (0 when they differ: runtime sizes);
// smem: the largest tile footprint of the runs.
template <typename R>
cudaError_t launch_particle_step_batch(const BatchRef<R> &b, const TmapSet<kBatchMax> *tm,
                                       int P, int Q, bool tma, int block, int grid,
                                       size_t smem, cudaStream_t s) {
  StepArgs<R> none{};
  k_plan<R, true><<<1, 1024, 0, s>>>(none, b, true, false);
  const void *k = pick_kernel<R>(P, Q, tma, false, true);
  void *args[] = {(void *)tm, (void *)&none, (void *)&b};
  return cudaLaunchKernel(k, dim3(grid), dim3(block), args, smem, s);
}

template <typename R>
cudaError_t launch_gather_current(const StepArgs<R> &a, cudaStream_t s) {
  const Geom &g = a.g;
  const int ni = g.fbc_x == FBC_PERIODIC ? g.nx : g.nx + 2 * GX;
  const int nj = g.fbc_y == FBC_PERIODIC ? g.ny : g.ny + 2 * GY;
  BatchRef<R> none{};
  BatchGrid bg{};
  k_gather_current<R, false><<<(ni * nj + 255) / 256, 256, 0, s>>>(a, none, bg);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_gather_current_batch(const BatchRef<R> &b, const BatchGrid &bg, cudaStream_t s) {
  StepArgs<R> none{};
  if (bg.off[bg.n] == 0) return cudaSuccess;
  k_gather_current<R, true><<<bg.off[bg.n], 256, 0, s>>>(none, b, bg);
  return cudaGetLastError();
}

template int particle_step_grid<float>(int, int, bool, bool, int, bool);
template int particle_step_grid<double>(int, int, bool, bool, int, bool);
template int particle_step_batch_grid<float>(int, int, bool, int, size_t);
template int particle_step_batch_grid<double>(int, int, bool, int, size_t);
template cudaError_t prepare_particle_step<float>(int, int);
template cudaError_t prepare_particle_step<double>(int, int);
template cudaError_t prepare_particle_step_batch<float>(int, int, size_t);
template cudaError_t prepare_particle_step_batch<double>(int, int, size_t);
template cudaError_t launch_particle_step<float>(const StepArgs<float> &, const CUtensorMap *,
                                                 bool, bool, int, int, bool, cudaStream_t);
template cudaError_t launch_particle_step<double>(const StepArgs<double> &,
                                                  const CUtensorMap *, bool, bool, int, int, bool,
                                                  cudaStream_t);
template cudaError_t launch_gather_current<float>(const StepArgs<float> &, cudaStream_t);
template cudaError_t launch_gather_current<double>(const StepArgs<double> &, cudaStream_t);
template cudaError_t launch_gather_current_batch<float>(const BatchRef<float> &, const BatchGrid &,
                                                        cudaStream_t);
template cudaError_t launch_gather_current_batch<double>(const BatchRef<double> &,
                                                         const BatchGrid &, cudaStream_t);
template cudaError_t launch_plan<float>(const StepArgs<float> &, bool, cudaStream_t);
template cudaError_t launch_plan<double>(const StepArgs<double> &, bool, cudaStream_t);
template cudaError_t launch_particle_step_batch<float>(const BatchRef<float> &,
                                                       const TmapSet<kBatchMax> *, int, int,
                                                       bool, int, int, size_t, cudaStream_t);
template cudaError_t launch_particle_step_batch<double>(const BatchRef<double> &,
                                                        const TmapSet<kBatchMax> *, int, int,
                                                        bool, int, int, size_t, cudaStream_t);

}  // namespace pic
