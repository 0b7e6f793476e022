// Device memory of a context: the caller's allocator when pic_config names
// one (dev_alloc / dev_free / alloc_user), else cudaMalloc / cudaFree; and
// NVTX ranges for the host API calls.
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "../../include/pic.h"

namespace pic {

inline cudaError_t dev_malloc(const pic_config &cf, void **p, size_t bytes) {
  if (!cf.dev_alloc) return cudaMalloc(p, bytes);
  *p = bytes ? cf.dev_alloc(bytes, cf.alloc_user) : nullptr;
  return (*p || !bytes) ? cudaSuccess : cudaErrorMemoryAllocation;
}

template <typename T>
inline cudaError_t dev_malloc(const pic_config &cf, T **p, size_t bytes) {
  void *q = nullptr;
  const cudaError_t e = dev_malloc(cf, &q, bytes);
  *p = static_cast<T *>(q);
  return e;
}

// Release p.  cudaFree waits for the device; a caller's allocator may hand
// the memory out again at once, so the context's stream is drained first.
inline void dev_free(const pic_config &cf, cudaStream_t s, void *p) {
  if (!p) return;
  if (!cf.dev_free) {
    cudaFree(p);
    return;
  }
  cudaStreamSynchronize(s);
  cf.dev_free(p, cf.alloc_user);
}

// NVTX range around a host API call (visible in a profiler's timeline; no
// cost without one attached).
struct NvtxRange {
  explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange &) = delete;
  NvtxRange &operator=(const NvtxRange &) = delete;
};

}  // namespace pic
