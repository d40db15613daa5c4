// trid_waitcheck.cu -- a bounded wait on a device flag, recorded in the device
// status word on expiry.  The TMA-fed kernels wait on mbarriers the same way
// (give up after a time limit, record TRID_ERR_TIMEOUT, return); this entry
// point lets a caller exercise that path on demand without any kernel of the
// solver hanging or faulting.
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/trid.h"
#include "trid_internal.h"

namespace trid {

__global__ void k_wait_flag(const int *flag, int expect, unsigned long long timeout_ns,
                            int *status) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const volatile int *f = flag;
    uint64_t t0;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
    unsigned ns = 32;
    while (*f != expect) {
        __nanosleep(ns);
        if (ns < 1024) ns <<= 1;
        uint64_t t;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
        if (t - t0 > timeout_ns) {
            atomicCAS(status, 0, int(TRID_ERR_TIMEOUT));
            return;
        }
    }
}

}  // namespace trid

extern "C" trid_status trid_wait_flag(const int *flag, int expect, double timeout_s,
                                      trid_stream_t stream) {
    if (!flag || !(timeout_s > 0.0) || timeout_s > 1.0) return TRID_ERR_INVALID_ARG;
    if ((reinterpret_cast<uintptr_t>(flag) % alignof(int)) != 0) return TRID_ERR_MISALIGNED;
    int *status = trid::device_status_word();
    if (!status) return TRID_ERR_CUDA;
    trid::k_wait_flag<<<1, 32, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
        flag, expect, (unsigned long long)(timeout_s * 1e9), status);
    return trid::launch_ok() ? TRID_OK : TRID_ERR_CUDA;
}
