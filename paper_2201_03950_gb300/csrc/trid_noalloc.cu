// trid_noalloc.cu -- the allocation-free variant of the batched solve.
//
// Some callers cannot let a library call cudaMalloc: a framework whose own
// memory pool has reserved the device memory (a library allocation can fail
// or fragment that pool), or a latency-critical loop that must not pay the
// device-wide synchronisation that growing a pool (cudaFree + cudaMalloc)
// implies.  For them the scratch of the long-system path (the reduced systems
// of the tiled Thomas-PCR passes) lives in one fixed, file-scope device array
// instead of the library pool.
#include <cuda_runtime.h>

#include <mutex>

#include "trid_internal.h"

namespace {

// Fixed scratch shared by every call of trid_solve_batch_noalloc on a device.
static __device__ __align__(256) unsigned char g_noalloc_scratch[TRID_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device, looked up once
// per device (with that device current) and cached; nullptr on failure.
void *scratch_address() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return nullptr;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    if (g_addr[dev] == nullptr) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || p == nullptr) {
            cudaGetLastError();
            return nullptr;
        }
        g_addr[dev] = p;
    }
    return g_addr[dev];
}

}  // namespace

namespace trid {
bool noalloc_scratch_ready() { return scratch_address() != nullptr; }
void noalloc_forget_device(int dev) {
    if (dev < 0 || dev >= kMaxDevices) return;
    std::lock_guard<std::mutex> lk(g_mu);
    g_addr[dev] = nullptr;
}
}  // namespace trid

extern "C" trid_status trid_solve_batch_noalloc(const void *a, const void *b, const void *c,
                                                void *d, void *u, const int64_t *dims, int ndim,
                                                int solve_dim, trid_dtype dtype,
                                                trid_stream_t stream) {
    trid::NvtxScope nvtx_scope("trid_solve_batch_noalloc");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    // size and argument check first, without touching the device
    size_t need = 0;
    trid_status s = trid::solve_with_scratch(a, b, c, d, u, dims, ndim, solve_dim, dtype, nullptr,
                                             0, need, st);
    if (s != TRID_ERR_ALLOC) return s;  // invalid, empty, or done without scratch
    if (need > TRID_NOALLOC_SCRATCH_BYTES) return TRID_ERR_ALLOC;  // beyond the fixed maximum
    void *scratch = scratch_address();
    if (!scratch) return TRID_ERR_CUDA;
    return trid::solve_with_scratch(a, b, c, d, u, dims, ndim, solve_dim, dtype, scratch,
                                    TRID_NOALLOC_SCRATCH_BYTES, need, st);
}
