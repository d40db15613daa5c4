// trid_internal.h -- host-side helpers shared by the library's translation
// units (not part of the public ABI).
#pragma once
#include <cstddef>
#include <cstdint>

#include "../../include/trid.h"

namespace trid {

inline bool is_aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// Library-owned scratch pool of the current device: returns a buffer of at
// least `bytes` bytes, growing it (device sync + cudaFree + cudaMalloc) when
// too small.  Shared by all calls on that device.
trid_status pool_reserve(size_t bytes, void **out);

// Device address of the status word of the current device (see
// trid_get_device_status); kernels that run bounded waits record failures there.
int *device_status_word();

}  // namespace trid
