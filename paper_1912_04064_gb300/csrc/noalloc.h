// Set-up of the allocation-free field-energy entry point on a device.
#pragma once

#include "../../include/pic.h"

namespace pic {
// Load the allocation-free entry point's module and kernels on device dev
// (current) and look up its scratch array, so that later calls of
// pic_field_energy_noalloc on that device allocate nothing.
pic_status noalloc_setup(int dev);
}  // namespace pic
