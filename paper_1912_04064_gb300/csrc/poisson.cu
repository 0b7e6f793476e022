// Initial electric field of a periodic run from Gauss's law (FP64): the
// discrete Poisson problem div_h E = rho - <rho>, E = -grad_h phi on the Yee
// lattice, solved spectrally.  A Fourier mode exp(i k.x) of phi has the
// discrete Laplacian -sum_a (2 / d_a)^2 sin^2(k_a d_a / 2); the k = 0 mode
// (the mean charge) is dropped.  The transforms are cuFFT's (an
// initialisation step off the time-stepping path); everything else runs in
// the kernels below.
#include <cufft.h>

#include <string>

#include "alloc.h"
#include "common.cuh"
#include "poisson.h"

namespace pic {

namespace {

// phi_hat = rho_hat / k_h^2 / N (the 1 / N of the unnormalised inverse
// transform folded in); k = 0 dropped.  Half-spectrum layout of a real
// transform: the fastest axis holds n0 / 2 + 1 entries.
__global__ void k_poisson_scale(cufftDoubleComplex *h, int dims, int n0, int n1, int n2,
                                double d0, double d1, double d2) {
  const int h0 = n0 / 2 + 1;
  const long long tot = (long long)h0 * n1 * (dims == 3 ? n2 : 1);
  const double N = (double)n0 * n1 * (dims == 3 ? n2 : 1);
  const double PI = 3.14159265358979323846;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
       e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e % h0);
    const int j = (int)((e / h0) % n1);
    const int k = dims == 3 ? (int)(e / ((long long)h0 * n1)) : 0;
    // signed wave numbers
    const int mi = i, mj = j <= n1 / 2 ? j : j - n1, mk = k <= n2 / 2 ? k : k - n2;
    const double s0 = (2.0 / d0) * sin(PI * mi / n0);
    const double s1 = (2.0 / d1) * sin(PI * mj / n1);
    const double s2 = dims == 3 ? (2.0 / d2) * sin(PI * mk / n2) : 0.0;
    const double k2 = s0 * s0 + s1 * s1 + s2 * s2;
    if (i == 0 && j == 0 && k == 0) {
      h[e].x = 0.0;
      h[e].y = 0.0;
    } else {
      const double f = 1.0 / (k2 * N);
      h[e].x *= f;
      h[e].y *= f;
    }
  }
}

// E_a = -(phi(x + d_a) - phi(x)) / d_a on the periodic grid (E_a sits half a
// cell along a from the node of phi).
__global__ void k_poisson_gradient(const double *phi, int dims, int n0, int n1, int n2, double d0,
                                   double d1, double d2, double *Ex, double *Ey, double *Ez) {
  const long long tot = (long long)n0 * n1 * (dims == 3 ? n2 : 1);
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
       e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e % n0), j = (int)((e / n0) % n1);
    const int k = dims == 3 ? (int)(e / ((long long)n0 * n1)) : 0;
    const long long row = (long long)k * n1 * n0 + (long long)j * n0;
    const double p = phi[e];
    Ex[e] = -(phi[row + (i + 1) % n0] - p) / d0;
    Ey[e] = -(phi[(long long)k * n1 * n0 + (long long)((j + 1) % n1) * n0 + i] - p) / d1;
    if (dims == 3)
      Ez[e] = -(phi[(long long)((k + 1) % n2) * n1 * n0 + (long long)j * n0 + i] - p) / d2;
  }
}

}  // namespace

pic_status poisson_fields(const pic_config &cf, int dims, const int n[3], const double d[3],
                          double *rho, double *Ex, double *Ey, double *Ez, cudaStream_t s,
                          std::string &err) {
  const long long cells = (long long)n[0] * n[1] * (dims == 3 ? n[2] : 1);
  const long long half = (long long)(n[0] / 2 + 1) * n[1] * (dims == 3 ? n[2] : 1);
  cufftDoubleComplex *h = nullptr;
  if (dev_malloc(cf, &h, sizeof(cufftDoubleComplex) * half) != cudaSuccess) {
    err = "cannot allocate the Poisson spectrum";
    return PIC_ENOMEM;
  }
  // plans without their own work areas: one shared area from the context's
  // allocator
  cufftHandle fwd = 0, inv = 0;
  size_t ws_f = 0, ws_i = 0;
  void *work = nullptr;
  bool ok = cufftCreate(&fwd) == CUFFT_SUCCESS && cufftCreate(&inv) == CUFFT_SUCCESS &&
            cufftSetAutoAllocation(fwd, 0) == CUFFT_SUCCESS &&
            cufftSetAutoAllocation(inv, 0) == CUFFT_SUCCESS;
  if (ok && dims == 3) {
    ok = cufftMakePlan3d(fwd, n[2], n[1], n[0], CUFFT_D2Z, &ws_f) == CUFFT_SUCCESS &&
         cufftMakePlan3d(inv, n[2], n[1], n[0], CUFFT_Z2D, &ws_i) == CUFFT_SUCCESS;
  } else if (ok) {
    ok = cufftMakePlan2d(fwd, n[1], n[0], CUFFT_D2Z, &ws_f) == CUFFT_SUCCESS &&
         cufftMakePlan2d(inv, n[1], n[0], CUFFT_Z2D, &ws_i) == CUFFT_SUCCESS;
  }
  const size_t ws = ws_f > ws_i ? ws_f : ws_i;
  ok = ok && (ws == 0 || dev_malloc(cf, &work, ws) == cudaSuccess);
  ok = ok && cufftSetWorkArea(fwd, work) == CUFFT_SUCCESS &&
       cufftSetWorkArea(inv, work) == CUFFT_SUCCESS;
  ok = ok && cufftSetStream(fwd, s) == CUFFT_SUCCESS && cufftSetStream(inv, s) == CUFFT_SUCCESS;
  ok = ok && cufftExecD2Z(fwd, rho, h) == CUFFT_SUCCESS;
  if (ok) {
    const int blocks = (int)std::min<long long>((half + 255) / 256, 4096);
    k_poisson_scale<<<blocks, 256, 0, s>>>(h, dims, n[0], n[1], dims == 3 ? n[2] : 1, d[0], d[1],
                                           dims == 3 ? d[2] : 1.0);
    ok = cudaGetLastError() == cudaSuccess;
  }
  ok = ok && cufftExecZ2D(inv, h, rho) == CUFFT_SUCCESS;  // rho now holds phi
  if (ok) {
    const int blocks = (int)std::min<long long>((cells + 255) / 256, 4096);
    k_poisson_gradient<<<blocks, 256, 0, s>>>(rho, dims, n[0], n[1], dims == 3 ? n[2] : 1, d[0],
                                              d[1], dims == 3 ? d[2] : 1.0, Ex, Ey, Ez);
    ok = cudaGetLastError() == cudaSuccess;
  }
  ok = ok && cudaStreamSynchronize(s) == cudaSuccess;
  if (fwd) cufftDestroy(fwd);
  if (inv) cufftDestroy(inv);
  dev_free(cf, s, work);
  dev_free(cf, s, h);
  if (!ok) {
    err = "the Poisson solve failed";
    return PIC_ECUDA;
  }
  return PIC_OK;
}

}  // namespace pic
