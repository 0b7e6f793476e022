// Periodic Poisson solve for the initial electric field (poisson.cu).
#pragma once

#include <cuda_runtime.h>

#include <string>

#include "../../include/pic.h"

namespace pic {

// rho: charge density on the canonical nodes of a periodic grid, contiguous
// (x fastest; n[0] x n[1] (x n[2] when dims = 3)), overwritten with phi.
// Ex, Ey (, Ez): the field on the same index grid, E_a at the node + d_a / 2.
// Scratch (the half spectrum and the FFT work area) comes from cf's
// allocator.
pic_status poisson_fields(const pic_config &cf, int dims, const int n[3], const double d[3],
                          double *rho, double *Ex, double *Ey, double *Ez, cudaStream_t s,
                          std::string &err);

}  // namespace pic
