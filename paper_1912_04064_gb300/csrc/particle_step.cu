// Patch particle step: one thread block per patch slot (the fine
// decomposition of SDMD, Section 2.2).  Per block:
//   1. SDMD step (ii): the patch's E and Bm tile (nodes -4..P+3 in x,
//      -1..Q+1 in y, six components) is staged into shared memory with one
//      3D TMA box copy (or plain coalesced loads);
//   2. every particle of the patch (its segment plus the particles that
//      entered from the 8 neighbours during the previous step) is
//      interpolated with the quadratic shape, pushed with the Boris scheme
//      and moved;
//   3. Esirkepov deposition (second-order shape, Section 3.2) into a shared
//      memory current tile with a 2-node halo, 40 shared atomics per
//      particle on the 4-node window that covers both shapes;
//   4. SDMD step (i): the tile is added into the region current;
//   5. re-binning: particles that stay are compacted into the output
//      segment, particles that left are appended to the direction bucket
//      read by the destination patch at the next step (positions already
//      rebased to it), boundary conditions applied at the domain faces.
#include "common.cuh"

namespace pic {

namespace {

template <typename R>
__device__ __forceinline__ R below(R v);
template <>
__device__ __forceinline__ float below<float>(float v) {
  return __int_as_float(__float_as_int(v) - 1);
}
template <>
__device__ __forceinline__ double below<double>(double v) {
  return __longlong_as_double(__double_as_longlong(v) - 1);
}

template <typename R>
__device__ __forceinline__ R gather(const R *T, int BX, int cx, const R Sx[3], int ry,
                                    const R Sy[3]) {
  const R *r0 = T + ry * BX + cx;
  R v = R(0);
#pragma unroll
  for (int b = 0; b < 3; ++b) {
    const R *r = r0 + b * BX;
    v += Sy[b] * (Sx[0] * r[0] + Sx[1] * r[1] + Sx[2] * r[2]);
  }
  return v;
}

// Place the three shape weights into a 4-node window: shifted by one node
// when `sh` is set.
template <typename R>
__device__ __forceinline__ void window4(const R S3[3], int sh, R S[4]) {
  S[0] = sh ? R(0) : S3[0];
  S[1] = sh ? S3[0] : S3[1];
  S[2] = sh ? S3[1] : S3[2];
  S[3] = sh ? S3[2] : R(0);
}

template <typename R, bool TMA>
__global__ void __launch_bounds__(256) k_particle_step(const __grid_constant__ CUtensorMap tmap,
                                                       const StepArgs<R> a) {
  extern __shared__ unsigned char dsm_raw[];
  __shared__ uint64_t mbar;
  __shared__ int s_off[10];
  __shared__ int s_cnt[9];
  __shared__ int s_src[9];
  __shared__ int s_out;
  __shared__ int s_bcnt[8];
  __shared__ int s_ok;

  const Geom &g = a.g;
  const int tid = threadIdx.x, nth = blockDim.x;
  const int s = blockIdx.x;
  const int P = g.P, Q = g.Q;
  const int BX = P + 8, BY = Q + 3;   // field tile
  const int JW = P + 5, JH = Q + 5;   // current tile
  const uint32_t pad = (128u - (smem_u32(dsm_raw) & 127u)) & 127u;
  R *Ft = reinterpret_cast<R *>(dsm_raw + pad);
  R *Jt = Ft + 6 * BY * BX;

  const int col0 = a.st->col0;
  const int sxs = s % g.npx, sy = s / g.npx;
  int px = sxs - col0;
  if (px < 0) px += g.npx;
  const int py = sy;
  const int X0 = px * P, Y0 = py * Q;

  // ---- 1. region -> patch field staging (SDMD step ii)
  if (TMA) {
    if (tid == 0) {
      mbar_init(&mbar, 1);
      fence_mbar_init();
    }
    __syncthreads();
    if (tid == 0) {
      mbar_arrive_expect_tx(&mbar, (uint32_t)(6 * BY * BX * sizeof(R)));
      tma_load_3d(Ft, &tmap, &mbar, X0 - 4 + GX, Y0 - 1 + GY, 0);
    }
  } else {
    for (int e = tid; e < 6 * BY * BX; e += nth) {
      int c = e / (BY * BX), r = e - c * (BY * BX), yy = r / BX, xx = r - yy * BX;
      Ft[e] = a.F[c * g.cs + fidx(g, X0 - 4 + xx, Y0 - 1 + yy)];
    }
  }
  for (int e = tid; e < 3 * JH * JW; e += nth) Jt[e] = R(0);
  if (tid < 9) {
    int cnt = 0, src = s;
    if (tid == 0) {
      cnt = a.cnt_in[s];
    } else {
      int k = tid - 1, ddx, ddy;
      dir_delta(k, ddx, ddy);
      src = neighbour_slot(g, col0, s, -ddx, -ddy);
      cnt = src >= 0 ? a.bcnt_in[(long long)src * 8 + k] : 0;
    }
    s_src[tid] = src;
    s_cnt[tid] = cnt;
  }
  if (tid < 8) s_bcnt[tid] = 0;
  if (tid == 0) s_out = 0;
  __syncthreads();
  if (tid == 0) {
    s_off[0] = 0;
    for (int i = 0; i < 9; ++i) s_off[i + 1] = s_off[i] + s_cnt[i];
    int ok = 1;
    if (TMA) {
      ok = 0;
      for (long long it = 0; it < WAIT_POLLS; ++it)
        if (mbar_try_wait(&mbar, 0)) { ok = 1; break; }
      if (!ok) {
        atomicOr(&a.st->err, ERR_TIMEOUT);
        for (long long it = 0; it < DRAIN_POLLS; ++it)
          if (mbar_try_wait(&mbar, 0)) break;
      }
    }
    s_ok = ok;
  }
  __syncthreads();
  if (!s_ok) return;

  // ---- 2..5. particles
  const int total = s_off[9];
  const R rdx = R(g.dt / g.dx), rdy = R(g.dt / g.dy);
  const R eps = R(g.q * g.dt / (2.0 * g.m));
  const R cjx = R(-g.q * g.dx / g.dt), cjy = R(-g.q * g.dy / g.dt), cjz = R(g.q);
  const R RP = R(P), RQ = R(Q);
  const int lane = tid & 31;
  R *Jx = Jt, *Jy = Jt + JH * JW, *Jz = Jt + 2 * JH * JW;
  const R *TEx = Ft, *TEy = Ft + BY * BX, *TEz = Ft + 2 * BY * BX;
  const R *TBx = Ft + 3 * BY * BX, *TBy = Ft + 4 * BY * BX, *TBz = Ft + 5 * BY * BX;
  unsigned err = 0;

  for (int b0 = 0; b0 < total; b0 += nth) {
    const int k = b0 + tid;
    bool alive = k < total;
    R x = 0, y = 0, ux = 0, uy = 0, uz = 0, w = 0;
    if (alive) {
      int src = 0;
      while (src < 8 && k >= s_off[src + 1]) ++src;
      const int kk = k - s_off[src];
      if (src == 0) {
        const long long i = (long long)s * a.cap + kk;
        x = a.pin.x[i]; y = a.pin.y[i];
        ux = a.pin.ux[i]; uy = a.pin.uy[i]; uz = a.pin.uz[i]; w = a.pin.w[i];
      } else {
        const long long i = (long long)s_src[src] * a.bk.stride + a.bk.off[src - 1] + kk;
        x = a.bin.x[i]; y = a.bin.y[i];
        ux = a.bin.ux[i]; uy = a.bin.uy[i]; uz = a.bin.uz[i]; w = a.bin.w[i];
      }
    }
    int ddx = 0, ddy = 0;
    if (alive) {
      // interpolation at x^n with the shape of each component's stagger
      R Sxp[3], Sxd[3], Syp[3], Syd[3];
      const int ip = shape2(x, Sxp);
      const int id = shape2(x - R(0.5), Sxd);
      const int jp = shape2(y, Syp);
      const int jd = shape2(y - R(0.5), Syd);
      const R Ex = gather(TEx, BX, id + 3, Sxd, jp, Syp);
      const R Ey = gather(TEy, BX, ip + 3, Sxp, jd, Syd);
      const R Ez = gather(TEz, BX, ip + 3, Sxp, jp, Syp);
      const R Bx = gather(TBx, BX, ip + 3, Sxp, jd, Syd);
      const R By = gather(TBy, BX, id + 3, Sxd, jp, Syp);
      const R Bz = gather(TBz, BX, id + 3, Sxd, jd, Syd);
      // Boris push u^{n-1/2} -> u^{n+1/2}
      const R umx = ux + eps * Ex, umy = uy + eps * Ey, umz = uz + eps * Ez;
      const R gm = sqrt(R(1) + umx * umx + umy * umy + umz * umz);
      const R ig = eps / gm;
      const R tx = ig * Bx, ty = ig * By, tz = ig * Bz;
      const R f = R(2) / (R(1) + tx * tx + ty * ty + tz * tz);
      const R sx_ = f * tx, sy_ = f * ty, sz_ = f * tz;
      const R upx = umx + (umy * tz - umz * ty);
      const R upy = umy + (umz * tx - umx * tz);
      const R upz = umz + (umx * ty - umy * tx);
      ux = umx + (upy * sz_ - upz * sy_) + eps * Ex;
      uy = umy + (upz * sx_ - upx * sz_) + eps * Ey;
      uz = umz + (upx * sy_ - upy * sx_) + eps * Ez;
      const R gam = sqrt(R(1) + ux * ux + uy * uy + uz * uz);
      const R inv = R(1) / gam;
      R x1 = x + rdx * ux * inv;
      R y1 = y + rdy * uy * inv;
      // Esirkepov deposition on the 4-node window covering S(x^n), S(x^{n+1})
      R S1x3[3], S1y3[3];
      const int i1 = shape2(x1, S1x3);
      const int j1 = shape2(y1, S1y3);
      const int di = i1 - ip, dj = j1 - jp;
      if (!(isfinite(x1) && isfinite(y1) && isfinite(ux) && isfinite(uy) && isfinite(uz))) {
        err |= ERR_NONFINITE;
        alive = false;
      } else if (di < -1 || di > 1 || dj < -1 || dj > 1) {
        err |= ERR_FAST;
        alive = false;
      } else {
        const int shx = di < 0, shy = dj < 0;
        R S0x[4], S1x[4], S0y[4], S1y[4], DSx[4], DSy[4];
        window4(Sxp, shx, S0x);
        window4(S1x3, di + shx, S1x);
        window4(Syp, shy, S0y);
        window4(S1y3, dj + shy, S1y);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          DSx[q] = S1x[q] - S0x[q];
          DSy[q] = S1y[q] - S0y[q];
        }
        const int cx = ip - 1 - shx + 2, cy = jp - 1 - shy + 2;  // tile coords
        const R wjx = cjx * w, wjy = cjy * w, wjz = cjz * w * uz * inv;
#pragma unroll
        for (int l = 0; l < 4; ++l) {
          const R Ay = S0y[l] + R(0.5) * DSy[l];
          R acc = R(0);
#pragma unroll
          for (int q = 0; q < 3; ++q) {
            acc += DSx[q] * Ay;
            atomicAdd(&Jx[(cy + l) * JW + cx + q], wjx * acc);
          }
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const R Ax = S0x[q] + R(0.5) * DSx[q];
          R acc = R(0);
#pragma unroll
          for (int l = 0; l < 3; ++l) {
            acc += DSy[l] * Ax;
            atomicAdd(&Jy[(cy + l) * JW + cx + q], wjy * acc);
          }
        }
#pragma unroll
        for (int l = 0; l < 4; ++l)
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const R Wz = S0x[q] * S0y[l] + R(0.5) * DSx[q] * S0y[l] +
                         R(0.5) * S0x[q] * DSy[l] + R(1.0 / 3.0) * DSx[q] * DSy[l];
            atomicAdd(&Jz[(cy + l) * JW + cx + q], wjz * Wz);
          }
        // boundary conditions at domain faces, then destination patch
        if (x1 < R(0)) ddx = -1; else if (x1 >= RP) ddx = 1;
        if (y1 < R(0)) ddy = -1; else if (y1 >= RQ) ddy = 1;
        if (ddx != 0 && (px + ddx < 0 || px + ddx >= g.npx)) {
          const int bc = g.pbc[0][ddx > 0];
          if (bc == PBC_REFLECT) {
            x1 = ddx < 0 ? -x1 : R(2 * P) - x1;
            if (x1 >= RP) x1 = below(RP);
            ux = -ux;
            ddx = 0;
          } else if (bc == PBC_REMOVE) {
            alive = false;
          }
        }
        if (ddy != 0 && (py + ddy < 0 || py + ddy >= g.npy)) {
          const int bc = g.pbc[1][ddy > 0];
          if (bc == PBC_REFLECT) {
            y1 = ddy < 0 ? -y1 : R(2 * Q) - y1;
            if (y1 >= RQ) y1 = below(RQ);
            uy = -uy;
            ddy = 0;
          } else if (bc == PBC_REMOVE) {
            alive = false;
          }
        }
        if (ddx < 0) { x1 += RP; if (x1 >= RP) x1 = below(RP); }
        else if (ddx > 0) x1 -= RP;
        if (ddy < 0) { y1 += RQ; if (y1 >= RQ) y1 = below(RQ); }
        else if (ddy > 0) y1 -= RQ;
        x = x1;
        y = y1;
      }
    }
    // compaction of the particles that stay
    const bool stay = alive && ddx == 0 && ddy == 0;
    const unsigned m = __ballot_sync(0xffffffffu, stay);
    int wbase = 0;
    if (lane == 0 && m) wbase = atomicAdd(&s_out, __popc(m));
    wbase = __shfl_sync(0xffffffffu, wbase, 0);
    if (stay) {
      const int pos = wbase + __popc(m & ((1u << lane) - 1u));
      if (pos < a.cap) {
        const long long i = (long long)s * a.cap + pos;
        a.pout.x[i] = x; a.pout.y[i] = y;
        a.pout.ux[i] = ux; a.pout.uy[i] = uy; a.pout.uz[i] = uz; a.pout.w[i] = w;
      } else {
        err |= ERR_OVERFLOW_SEG;
      }
    } else if (alive) {
      const int dir = dir_index(ddx, ddy);
      const int pos = atomicAdd(&s_bcnt[dir], 1);
      if (pos < a.bk.cap[dir]) {
        const long long i = (long long)s * a.bk.stride + a.bk.off[dir] + pos;
        a.bout.x[i] = x; a.bout.y[i] = y;
        a.bout.ux[i] = ux; a.bout.uy[i] = uy; a.bout.uz[i] = uz; a.bout.w[i] = w;
      } else {
        err |= ERR_OVERFLOW_BKT;
      }
    }
  }
  if (err) atomicOr(&a.st->err, err);
  __syncthreads();

  // ---- SDMD step (i): patch current tile -> region current
  for (int e = tid; e < 3 * JH * JW; e += nth) {
    const R v = Jt[e];
    if (v != R(0)) {
      const int c = e / (JH * JW), r = e - c * (JH * JW), l = r / JW, q = r - l * JW;
      int gi = X0 - 2 + q, gj = Y0 - 2 + l;
      if (g.fbc_x == FBC_PERIODIC) gi = gi < 0 ? gi + g.nx : (gi >= g.nx ? gi - g.nx : gi);
      if (g.fbc_y == FBC_PERIODIC) gj = gj < 0 ? gj + g.ny : (gj >= g.ny ? gj - g.ny : gj);
      atomicAdd(&a.Jdst[c * g.cs + fidx(g, gi, gj)], v);
    }
  }
  if (tid == 0) {
    const int n = s_out < a.cap ? s_out : a.cap;
    a.cnt_out[s] = n;
    atomicMax(&a.st->maxcnt[a.parity], s_out);
  }
  if (tid < 8)
    a.bcnt_out[(long long)s * 8 + tid] = s_bcnt[tid] < a.bk.cap[tid] ? s_bcnt[tid] : a.bk.cap[tid];
}

}  // namespace

size_t particle_step_smem(int P, int Q, size_t rsize) {
  return (size_t)(6 * (Q + 3) * (P + 8) + 3 * (Q + 5) * (P + 5)) * rsize + 128;
}

template <typename R>
cudaError_t prepare_particle_step(int P, int Q) {
  const int smem = (int)particle_step_smem(P, Q, sizeof(R));
  cudaError_t e = cudaFuncSetAttribute(k_particle_step<R, true>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_particle_step<R, false>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
}

template <typename R>
cudaError_t launch_particle_step(const StepArgs<R> &a, const CUtensorMap *tmap, bool tma,
                                 int block, cudaStream_t s) {
  const size_t smem = particle_step_smem(a.g.P, a.g.Q, sizeof(R));
  auto kern = tma ? k_particle_step<R, true> : k_particle_step<R, false>;
  kern<<<a.g.nslots, block, smem, s>>>(*tmap, a);
  return cudaGetLastError();
}

template cudaError_t prepare_particle_step<float>(int, int);
template cudaError_t prepare_particle_step<double>(int, int);
template cudaError_t launch_particle_step<float>(const StepArgs<float> &, const CUtensorMap *,
                                                 bool, int, cudaStream_t);
template cudaError_t launch_particle_step<double>(const StepArgs<double> &,
                                                  const CUtensorMap *, bool, int, cudaStream_t);

}  // namespace pic
