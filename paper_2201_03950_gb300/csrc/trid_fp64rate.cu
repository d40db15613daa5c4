// trid_fp64rate.cu -- measured FP64 arithmetic rates of the current device.
//
// On GB300 the FP64 pipe runs at a small fraction of the FP32 rate, so the
// FP64 solves are bound by FP64 arithmetic, not by HBM.  Their roofline needs
// the device's own FP64 rates: this entry point times, with CUDA events, a
// grid of independent fused multiply-add chains and one of IEEE divisions
// (eight independent chains per thread, enough threads to fill every SM).
#include <cuda_runtime.h>

#include "../../include/trid.h"
#include "trid_internal.h"

namespace trid {

constexpr int FR_ITERS = 2048;
__device__ double g_fp64_sink;  // written only if a chain ends at -1 (never)

template <bool DIV>
__global__ void k_fp64_rate(double s) {
    double v[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = 1.0 + 1e-3 * threadIdx.x + 0.1 * k;
#pragma unroll 4
    for (int i = 0; i < FR_ITERS; ++i) {
#pragma unroll
        for (int k = 0; k < 8; ++k) v[k] = DIV ? 1.0 / v[k] : fma(v[k], s, 1e-9);
    }
    double acc = 0.0;
#pragma unroll
    for (int k = 0; k < 8; ++k) acc += v[k];
    if (acc == -1.0) g_fp64_sink = acc;  // never true; keeps the chains live
}

}  // namespace trid

extern "C" trid_status trid_fp64_rates(double *fma_gops, double *div_gops, trid_stream_t stream) {
    if (!fma_gops || !div_gops) return TRID_ERR_INVALID_ARG;
    const trid::DeviceInfo *di = trid::device_info();
    if (!di) return TRID_ERR_CUDA;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const int threads = 256, blocks = di->sm_count * 8;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    trid_status rs = TRID_OK;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        cudaGetLastError();
        rs = TRID_ERR_CUDA;
    }
    for (int op = 0; op < 2 && rs == TRID_OK; ++op) {
        float best = 0.0f;
        for (int rep = 0; rep < 3; ++rep) {  // first run warms up; best of the other two
            cudaEventRecord(e0, st);
            if (op == 0) trid::k_fp64_rate<false><<<blocks, threads, 0, st>>>(0.999999);
            else trid::k_fp64_rate<true><<<blocks, threads, 0, st>>>(0.999999);
            cudaEventRecord(e1, st);
            float ms = 0.0f;
            if (!trid::launch_ok() || cudaEventSynchronize(e1) != cudaSuccess ||
                cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
                rs = TRID_ERR_CUDA;
                break;
            }
            if (rep > 0 && (best == 0.0f || ms < best)) best = ms;
        }
        const double n = double(blocks) * threads * trid::FR_ITERS * 8;
        (op == 0 ? *fma_gops : *div_gops) = best > 0.0f ? n / (double(best) * 1e6) : 0.0;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (rs == TRID_OK && cudaStreamSynchronize(st) != cudaSuccess) rs = TRID_ERR_CUDA;
    return rs;
}
