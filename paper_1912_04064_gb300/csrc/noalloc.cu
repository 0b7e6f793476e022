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
//
// Set-up (once per device and CUDA context, on the first call or by
// pic_create on that device): the module is loaded and the array's device
// address looked up, with the kernels' code loaded too, so that later calls
// make no allocation at all.  The address is cached together with the
// context it belongs to: after a device reset (a new primary context) the
// next call looks it up again instead of using a stale address.
#include <cudaTypedefs.h>

#include <mutex>

#include "../../include/pic.h"
#include "common.cuh"
#include "noalloc.h"

namespace {

// One partial sum per (row, energy): |E|^2 and |Bm|^2 of each row of cells.
__device__ __align__(256) double g_row_partials[2 * PIC_NOALLOC_MAX_ROWS];

constexpr int kMaxDevices = 64;
double *g_scratch[kMaxDevices] = {};
CUcontext g_scratch_ctx[kMaxDevices] = {};  // context the cached address belongs to
std::mutex g_setup_mutex;

// The current CUDA context (driver entry point; null if unavailable).
CUcontext current_context() {
  static PFN_cuCtxGetCurrent_v4000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 4000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuCtxGetCurrent_v4000)p;
  });
  CUcontext c = nullptr;
  if (fn) fn(&c);
  return c;
}

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

// Rows reduced by one block of 256 threads in a fixed order (each thread
// its rows t, t + 256, ... in turn, then a fixed tree): deterministic.
__global__ void __launch_bounds__(256) k_rows_total(const double *rows, int ny, double half_dV,
                                                   double *out) {
  __shared__ double sh[2][256];
  double e = 0.0, b = 0.0;
  for (int j = threadIdx.x; j < ny; j += 256) {
    e += rows[2 * j];
    b += rows[2 * j + 1];
  }
  sh[0][threadIdx.x] = e;
  sh[1][threadIdx.x] = b;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      sh[0][threadIdx.x] += sh[0][threadIdx.x + s];
      sh[1][threadIdx.x] += sh[1][threadIdx.x + s];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[0] = half_dV * sh[0][0];
    out[1] = half_dV * sh[1][0];
  }
}

// Device address of the scratch array on the current device (the host-side
// name of a __device__ array is not a device address), looked up once per
// device and context; the look-up loads the module, and querying the
// kernels' attributes loads their code.
pic_status scratch_for(int dev, double **out) {
  if (dev < 0 || dev >= kMaxDevices) return PIC_EINVAL;
  const CUcontext ctx = current_context();
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch[dev] || g_scratch_ctx[dev] != ctx) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_row_partials) != cudaSuccess || !p) return PIC_ECUDA;
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, k_row_energy) != cudaSuccess ||
        cudaFuncGetAttributes(&fa, k_rows_total) != cudaSuccess)
      return PIC_ECUDA;
    g_scratch[dev] = (double *)p;
    g_scratch_ctx[dev] = ctx;
  }
  *out = g_scratch[dev];
  return PIC_OK;
}

}  // namespace

namespace pic {
pic_status noalloc_setup(int dev) {
  double *p = nullptr;
  return scratch_for(dev, &p);
}
}  // namespace pic

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
  k_rows_total<<<1, 256, 0, st>>>(rows, ny, 0.5 * dV, out);
  return cudaGetLastError() == cudaSuccess ? PIC_OK : PIC_ECUDA;
}
