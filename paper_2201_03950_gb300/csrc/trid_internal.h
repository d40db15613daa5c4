// trid_internal.h -- host-side helpers shared by the library's translation
// units (not part of the public ABI).
#pragma once
#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

#include "../../include/trid.h"

namespace trid {

inline bool is_aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// Library-owned scratch pool of the current device: returns a buffer of at
// least `bytes` bytes, growing it (device sync + cudaFree + cudaMalloc) when
// too small.  Shared by all calls on that device.
trid_status pool_reserve(size_t bytes, void **out);

// As trid_solve_batch_ws, but the solution is stored into `out` (which must
// not overlap a, b, c or d) rather than into d or added into u; d is only
// read.  Used by the differentiable ADI, whose adjoint solves would otherwise
// accumulate into buffers zeroed every step.
trid_status solve_into_ws(const void *a, const void *b, const void *c, const void *d, void *out,
                          const int64_t *dims, int ndim, int solve_dim, trid_dtype dtype,
                          void *workspace, size_t workspace_bytes, cudaStream_t st);

// Cached attributes of the current device (queried on first use per device).
struct DeviceInfo {
    int sm_count;
    int max_smem_optin;   // dynamic shared memory a block may opt in to
    int smem_per_sm;
};
const DeviceInfo *device_info();

// 3D tensor map over a strided line set viewed as (inner, n, outer) with the
// box (box_x, box_rows, 1) (box_rows = 0: all n rows, n <= 256); false if the
// TMA constraints do not hold.
bool encode_lines_map(void *map /* CUtensorMap */, const void *base, int esz, int64_t inner,
                      int64_t n, int64_t outer, int box_x, int box_rows = 0);

// 2D tensor map over `nrows` rows of `row_elems` contiguous elements (row
// pitch = row_elems), box (row_elems, box_rows), shared-memory swizzle of
// 32, 64 or 128 bytes (row_elems * esz <= swizzle); false if the TMA
// constraints do not hold.
bool encode_rows_map(void *map /* CUtensorMap */, const void *base, int esz, int64_t row_elems,
                     int64_t nrows, int box_rows, int swizzle);

// Clusters of `csize` CTAs of `kernel` that can be resident at once (0 if
// none or the query fails); sizes above 8 are enabled on the function first.
int cluster_capacity(const void *kernel, int csize, int threads, size_t smem);

// Blocks of `kernel` resident per SM for (threads, dynamic smem) on the
// current device, after raising the kernel's dynamic shared-memory limit to
// `smem`.  Both results are cached per (kernel, device, threads, smem), so a
// launch in a time-stepping loop costs no extra driver calls.  0 on failure.
int kernel_blocks_per_sm(const void *kernel, int threads, size_t smem);

// Batched solve with caller-chosen scratch (checks arguments on the host;
// TRID_ERR_ALLOC without launching when scratch_bytes < need).
trid_status solve_with_scratch(const void *a, const void *b, const void *c, void *d, void *u,
                               const int64_t *dims, int ndim, int solve_dim, trid_dtype dtype,
                               void *scratch, size_t scratch_bytes, size_t &need,
                               cudaStream_t st);

// Device address of the status word of the current device (see
// trid_get_device_status); kernels that run bounded waits record failures there.
int *device_status_word();

// 3D ADI on a batch of meshes stacked along z (two-pass schedule).
bool adi3_batch_eligible(const int64_t *n3, int ndim);
size_t adi3_batch_ws_bytes(const int64_t *n3, size_t esz, int64_t nb);
trid_status adi3_batch_run(void *u, int64_t nb, const int64_t *n3, double lam, int nsteps,
                           trid_dtype dtype, void *ws, size_t ws_bytes, cudaStream_t st);

// Allocation-free entry point's fixed array: looks its device address up on
// the current device (true on success), and forgets the cached address of
// device `dev` (trid_finalize).
bool noalloc_scratch_ready();
void noalloc_forget_device(int dev);

// Optional NVTX ranges around the compute entry points, for timeline tools
// (Nsight Systems): on when the environment has TRID_NVTX=1 (read once per
// process), otherwise the scope costs one branch.
struct NvtxScope {
    bool on;
    explicit NvtxScope(const char *name);
    ~NvtxScope();
};

// A library-owned non-blocking stream of the current device (created on first
// use and by trid_init, destroyed by trid_finalize; nullptr if it cannot be
// created, e.g. inside a stream capture before it exists).  Calls that use it
// order it against the caller's stream with events only.
cudaStream_t aux_stream();

// Record a failed CUDA runtime call (read back by trid_last_cuda_error).
void note_cuda_error(cudaError_t e);
// cudaGetLastError() == cudaSuccess after a launch; a failure is recorded.
bool launch_ok();
// Whether a launch on `st` may carry the programmatic-dependent-launch
// attribute: not while the stream is being captured (for the kernels that use
// this, the captured graph's plain edges measured faster than programmatic
// ones: 1024^2 differentiable ADI, forward and backward 3.88 ms against
// 4.02 ms), and not when the capture state cannot be read.
bool pdl_launch_allowed(cudaStream_t st);

}  // namespace trid
