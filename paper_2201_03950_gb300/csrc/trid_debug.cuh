// trid_debug.cuh -- device-side index checks of the debug build.
//
// Built with -DTRID_DEBUG_BOUNDS (build(debug_bounds=True) ->
// _lib/libtrid_dbg.so), the hot kernels check the global element ranges they
// are about to read or write against the extents of their arrays; a failed
// check skips the access and records TRID_ERR_INVALID_ARG in a device word of
// its translation unit, which trid_get_device_status reports (and clears)
// like the status word of the bounded waits.  Nothing traps.  In the release
// build TRID_BOUNDS(cond) is the constant true and costs nothing.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/trid.h"

namespace trid {
// Registry of the debug-word readers of the translation units (host side;
// each reader returns and clears its word).  Defined in trid_api.cu.
int register_dbg_reader(int (*reader)());
}  // namespace trid

namespace trid {
// [off, off + count) lies inside an array of `total` elements.
__host__ __device__ __forceinline__ bool in_span(int64_t off, int64_t count, int64_t total) {
    return off >= 0 && count >= 0 && off + count <= total;
}
}  // namespace trid

#ifdef TRID_DEBUG_BOUNDS
namespace trid {
namespace {
__device__ int g_dbg_word;  // one per translation unit

__device__ __forceinline__ bool dbg_check(bool ok) {
    if (!ok) atomicCAS(&g_dbg_word, 0, int(TRID_ERR_INVALID_ARG));
    return ok;
}

int dbg_take() {
    int v = 0;
    if (cudaMemcpyFromSymbol(&v, g_dbg_word, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    if (v != 0) {
        const int zero = 0;
        cudaMemcpyToSymbol(g_dbg_word, &zero, sizeof(int));
    }
    return v;
}

const int dbg_registered = register_dbg_reader(&dbg_take);
}  // namespace
}  // namespace trid
#define TRID_BOUNDS(cond) (trid::dbg_check(cond))
#else
#define TRID_BOUNDS(cond) (true)
#endif
