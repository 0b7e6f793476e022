// Allocation-free field-energy reduction (pic_field_energy_noalloc).
//
// Some callers cannot let a library call cudaMalloc: a host application that
// owns the whole device memory budget through its own allocator, or a
// latency-bound serving loop in which a device allocation would synchronise
// the device and stall the requests in flight.  This entry point computes
// the same field energies as pic_diag's reduction with all of its scratch in
// a file-scope device array of fixed size, so it allocates nothing: the
// caller passes the input arrays and the output location.
//
// The scratch array is shared by every call on a device and keeps the last
// call's contents; each call overwrites the rows it uses before reading
// them.  Calls that overlap on the GPU (two streams, or two host threads)
// race on it.  Every GPU that loads the library holds the array until the
// process exits.
#include <mutex>

#include "../../include/pic.h"
#include "common.cuh"

namespace {

// One partial sum per (row, energy): |E|^2 and |Bm|^2 of each row of cells.
__device__ __align__(256) double g_row_partials[2 * PIC_NOALLOC_MAX_ROWS];

constexpr int kMaxDevices = 64;
double *g_scratch[kMaxDevices] = {};
std::mutex g_setup_mutex;

__global__ void k_row_energy(const double *Ex, const double *Ey, const double *Ez,
                             const double *Bx, const double *By, const double *Bz, int nx,
                             int ny, double *rows) {
  __shared__ double sh[2][256];
  const int j = blockIdx.x;
  double e = 0.0, b = 0.0;
  for (int i = threadIdx.x; i < nx; i += blockDim.x) {
    const long long o = (long long)j * nx + i;
    e += Ex[o] * Ex[o] + Ey[o] * Ey[o] + Ez[o] * Ez[o];
    b += Bx[o] * Bx[o] + By[o] * By[o] + Bz[o] * Bz[o];
  }
  sh[0][threadIdx.x] = e;
  sh[1][threadIdx.x] = b;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      sh[0][threadIdx.x] += sh[0][threadIdx.x + s];
      sh[1][threadIdx.x] += sh[1][threadIdx.x + s];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    rows[2 * j] = sh[0][0];
    rows[2 * j + 1] = sh[1][0];
  }
  (void)ny;
}

// Rows reduced in ascending order by one thread per energy: deterministic.
__global__ void k_rows_total(const double *rows, int ny, double half_dV, double *out) {
  const int k = threadIdx.x;
  if (k >= 2) return;
  double s = 0.0;
  for (int j = 0; j < ny; ++j) s += rows[2 * j + k];
  out[k] = half_dV * s;
}

// Device address of the scratch array on the current device, looked up once
// per device (the host-side name of a __device__ array is not a device
// address).
pic_status scratch_for(int dev, double **out) {
  if (dev < 0 || dev >= kMaxDevices) return PIC_EINVAL;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch[dev]) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_row_partials) != cudaSuccess || !p) return PIC_ECUDA;
    g_scratch[dev] = (double *)p;
  }
  *out = g_scratch[dev];
  return PIC_OK;
}

}  // namespace

extern "C" pic_status pic_field_energy_noalloc(const double *Ex, const double *Ey,
                                               const double *Ez, const double *Bmx,
                                               const double *Bmy, const double *Bmz, int nx,
                                               int ny, double dV, double *out, void *stream) {
  if (!Ex || !Ey || !Ez || !Bmx || !Bmy || !Bmz || !out) return PIC_EINVAL;
  if (nx <= 0 || ny <= 0 || ny > PIC_NOALLOC_MAX_ROWS) return PIC_EINVAL;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return PIC_ECUDA;
  double *rows = nullptr;
  const pic_status s = scratch_for(dev, &rows);
  if (s != PIC_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  k_row_energy<<<ny, 256, 0, st>>>(Ex, Ey, Ez, Bmx, Bmy, Bmz, nx, ny, rows);
  k_rows_total<<<1, 32, 0, st>>>(rows, ny, 0.5 * dV, out);
  return cudaGetLastError() == cudaSuccess ? PIC_OK : PIC_ECUDA;
}
