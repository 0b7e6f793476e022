// 3D3V contexts (dims = 3): the host side of the 3D path in pic3d.cu, called
// by the C-ABI entry points of api.cu for a context created with dims = 3.
#pragma once

#include <cuda_runtime.h>

#include <string>

#include "../../include/pic.h"

namespace pic {

struct Ctx3;

// Configuration checks of the 3D path (after the dimension-free ones).
bool valid_config3(const pic_config *c, std::string &why);
size_t footprint3(const pic_config *c, size_t np_max);

pic_status c3_create(const pic_config *cfg, cudaStream_t stream, Ctx3 **out, std::string &err);
void c3_destroy(Ctx3 *c);
pic_status c3_load(Ctx3 *c, const double *x, const double *y, const double *z, const double *ux,
                   const double *uy, const double *uz, const double *w, size_t n, int where);
pic_status c3_fill_plasma(Ctx3 *c);
pic_status c3_set_field(Ctx3 *c, int which, const double *src, int where);
pic_status c3_get_field(Ctx3 *c, int which, double *dst, int where);
pic_status c3_set_background(Ctx3 *c, int mode, double value);
pic_status c3_init_fields(Ctx3 *c, int mode);
pic_status c3_step(Ctx3 *c, int nsteps);
pic_status c3_get_particles(Ctx3 *c, double *out, size_t cap, size_t *n, int where);
pic_status c3_diag(Ctx3 *c, pic_diag_t *out);
pic_status c3_sync(Ctx3 *c);
// Host snapshot of the whole 3D state (host == nullptr: *bytes = size) and
// its restore into a context of the same geometry and precision.
pic_status c3_snapshot(Ctx3 *c, void *host, size_t *bytes);
pic_status c3_restore(Ctx3 *c, const void *host, size_t bytes);
const char *c3_error(const Ctx3 *c);

}  // namespace pic
