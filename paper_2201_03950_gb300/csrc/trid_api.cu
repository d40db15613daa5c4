// trid_api.cu -- status strings, version, device status word and the
// library-owned scratch pool behind trid_solve_batch.
#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <atomic>
#include <cstdlib>
#include <cstring>
#include <mutex>

#include <nvtx3/nvToolsExt.h>

#include "trid_internal.h"

namespace trid {

__device__ int g_status_word;  // 0 = OK, else a trid_status recorded by a kernel

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_pool_mu;
void *g_pool_ptr[kMaxDevices] = {};
size_t g_pool_size[kMaxDevices] = {};
int *g_status_ptr[kMaxDevices] = {};
DeviceInfo g_info[kMaxDevices];
bool g_info_ok[kMaxDevices] = {};
cudaStream_t g_aux_stream[kMaxDevices] = {};
PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
bool g_encode_tried = false;
}  // namespace

const DeviceInfo *device_info() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return nullptr;
    std::lock_guard<std::mutex> lk(g_pool_mu);
    if (!g_info_ok[dev]) {
        DeviceInfo d{};
        if (cudaDeviceGetAttribute(&d.sm_count, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&d.max_smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) !=
                cudaSuccess ||
            cudaDeviceGetAttribute(&d.smem_per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) !=
                cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        g_info[dev] = d;
        g_info_ok[dev] = true;
    }
    return &g_info[dev];
}

namespace {
struct OccEntry {
    const void *kernel;
    int dev, threads;
    size_t smem;
    int blocks;
};
constexpr int kOccCache = 256;
OccEntry g_occ[kOccCache];
int g_nocc = 0;
}  // namespace

namespace {
struct ClusterEntry {
    const void *kernel;
    int dev, csize, threads;
    size_t smem;
    int clusters;
};
constexpr int kClusterCache = 64;
ClusterEntry g_ccache[kClusterCache];
int g_ncc = 0;
}  // namespace

int cluster_capacity(const void *kernel, int csize, int threads, size_t smem) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    std::lock_guard<std::mutex> lk(g_pool_mu);
    for (int i = 0; i < g_ncc; ++i) {
        const ClusterEntry &e = g_ccache[i];
        if (e.kernel == kernel && e.dev == dev && e.csize == csize && e.threads == threads &&
            e.smem == smem)
            return e.clusters;
    }
    if (csize > 8) {
        const cudaError_t ae =
            cudaFuncSetAttribute(kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (ae != cudaSuccess) {
            cudaGetLastError();
            note_cuda_error(ae);
            return 0;
        }
    }
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = unsigned(csize);
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(unsigned(csize));
    cfg.blockDim = dim3(unsigned(threads));
    cfg.dynamicSmemBytes = smem;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    const cudaError_t oe = cudaOccupancyMaxActiveClusters(&n, kernel, &cfg);
    if (oe != cudaSuccess) {
        cudaGetLastError();
        n = 0;
    }
    if (g_ncc < kClusterCache)
        g_ccache[g_ncc++] = ClusterEntry{kernel, dev, csize, threads, smem, n};
    return n;
}

int kernel_blocks_per_sm(const void *kernel, int threads, size_t smem) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    std::lock_guard<std::mutex> lk(g_pool_mu);
    for (int i = 0; i < g_nocc; ++i) {
        const OccEntry &e = g_occ[i];
        if (e.kernel == kernel && e.dev == dev && e.threads == threads && e.smem == smem)
            return e.blocks;
    }
    // The attribute is per function: raise it to the largest size this
    // function is ever queried with, never lower it (a cached smaller query
    // must not shrink the limit a larger launch relies on).
    int need = int(smem);
    for (int i = 0; i < g_nocc; ++i)
        if (g_occ[i].kernel == kernel && g_occ[i].dev == dev && int(g_occ[i].smem) > need)
            need = int(g_occ[i].smem);
    const cudaError_t ae =
        cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, need);
    if (ae != cudaSuccess) {
        cudaGetLastError();
        note_cuda_error(ae);
        return 0;
    }
    int blocks = 0;
    const cudaError_t oe = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, kernel, threads, smem);
    if (oe != cudaSuccess) {
        cudaGetLastError();
        note_cuda_error(oe);
        return 0;
    }
    if (g_nocc < kOccCache) g_occ[g_nocc++] = OccEntry{kernel, dev, threads, smem, blocks};
    return blocks;
}

// Looks up cuTensorMapEncodeTiled once; false if the driver lacks it.
static bool encode_lines_map_ready() {
    std::lock_guard<std::mutex> lk(g_pool_mu);
    if (!g_encode_tried) {
        g_encode_tried = true;
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                             cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
        else
            cudaGetLastError();
    }
    return g_encode != nullptr;
}

bool encode_lines_map(void *map, const void *base, int esz, int64_t inner, int64_t n,
                      int64_t outer, int box_x, int box_rows) {
    if (!encode_lines_map_ready()) return false;
    if ((reinterpret_cast<uintptr_t>(base) & 15u) != 0) return false;
    const int64_t rows = box_rows > 0 ? box_rows : n;
    if ((inner * esz) % 16 != 0 || n < 1 || rows > 256 || inner < 1 || outer < 1) return false;
    if (inner >= (int64_t(1) << 32) || outer >= (int64_t(1) << 31) || n >= (int64_t(1) << 32))
        return false;
    const cuuint64_t dims[3] = {cuuint64_t(inner), cuuint64_t(n), cuuint64_t(outer)};
    const cuuint64_t strides[2] = {cuuint64_t(inner * esz), cuuint64_t(inner * n * esz)};
    if (strides[1] >= (cuuint64_t(1) << 40)) return false;
    const cuuint32_t box[3] = {cuuint32_t(box_x), cuuint32_t(rows), 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    const CUresult r = g_encode(
        static_cast<CUtensorMap *>(map),
        esz == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 3,
        const_cast<void *>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
        CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

bool encode_rows_map(void *map, const void *base, int esz, int64_t row_elems, int64_t nrows,
                     int box_rows, int swizzle) {
    if (!encode_lines_map_ready()) return false;
    if ((reinterpret_cast<uintptr_t>(base) & 15u) != 0) return false;
    const int64_t row_bytes = row_elems * esz;
    if (row_bytes % 16 != 0 || row_bytes > swizzle || nrows < 1 || box_rows < 1 ||
        box_rows > 256 || nrows >= (int64_t(1) << 32))
        return false;
    CUtensorMapSwizzle sw;
    if (swizzle == 32) sw = CU_TENSOR_MAP_SWIZZLE_32B;
    else if (swizzle == 64) sw = CU_TENSOR_MAP_SWIZZLE_64B;
    else if (swizzle == 128) sw = CU_TENSOR_MAP_SWIZZLE_128B;
    else return false;
    const cuuint64_t dims[2] = {cuuint64_t(row_elems), cuuint64_t(nrows)};
    const cuuint64_t strides[1] = {cuuint64_t(row_bytes)};
    const cuuint32_t box[2] = {cuuint32_t(row_elems), cuuint32_t(box_rows)};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult r = g_encode(
        static_cast<CUtensorMap *>(map),
        esz == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2,
        const_cast<void *>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, sw,
        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

trid_status pool_reserve(size_t bytes, void **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return TRID_ERR_CUDA;
    std::lock_guard<std::mutex> lk(g_pool_mu);
    if (g_pool_size[dev] < bytes) {
        if (g_pool_ptr[dev]) {
            // in-flight work may still use the old buffer
            if (cudaDeviceSynchronize() != cudaSuccess) return TRID_ERR_CUDA;
            cudaFree(g_pool_ptr[dev]);
            g_pool_ptr[dev] = nullptr;
            g_pool_size[dev] = 0;
        }
        void *p = nullptr;
        if (cudaMalloc(&p, bytes) != cudaSuccess) {
            cudaGetLastError();
            return TRID_ERR_ALLOC;
        }
        g_pool_ptr[dev] = p;
        g_pool_size[dev] = bytes;
    }
    *out = g_pool_ptr[dev];
    return TRID_OK;
}

// Drops every cached per-device state of device `dev` and frees its pool
// (the caller has synchronised the device).  Used by trid_finalize.
static void forget_device(int dev) {
    std::lock_guard<std::mutex> lk(g_pool_mu);
    if (g_pool_ptr[dev]) cudaFree(g_pool_ptr[dev]);
    g_pool_ptr[dev] = nullptr;
    g_pool_size[dev] = 0;
    g_status_ptr[dev] = nullptr;
    g_info_ok[dev] = false;
    if (g_aux_stream[dev]) cudaStreamDestroy(g_aux_stream[dev]);
    g_aux_stream[dev] = nullptr;
    int k = 0;
    for (int i = 0; i < g_nocc; ++i)
        if (g_occ[i].dev != dev) g_occ[k++] = g_occ[i];
    g_nocc = k;
    k = 0;
    for (int i = 0; i < g_ncc; ++i)
        if (g_ccache[i].dev != dev) g_ccache[k++] = g_ccache[i];
    g_ncc = k;
}

cudaStream_t aux_stream() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return nullptr;
    std::lock_guard<std::mutex> lk(g_pool_mu);
    if (!g_aux_stream[dev]) {
        cudaStream_t s = nullptr;
        if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        g_aux_stream[dev] = s;
    }
    return g_aux_stream[dev];
}

int *device_status_word() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return nullptr;
    std::lock_guard<std::mutex> lk(g_pool_mu);
    if (!g_status_ptr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_status_word) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        g_status_ptr[dev] = static_cast<int *>(p);
    }
    return g_status_ptr[dev];
}

}  // namespace trid

extern "C" const char *trid_status_string(trid_status s) {
    switch (s) {
        case TRID_OK: return "TRID_OK";
        case TRID_ERR_INVALID_ARG: return "TRID_ERR_INVALID_ARG";
        case TRID_ERR_UNSUPPORTED: return "TRID_ERR_UNSUPPORTED";
        case TRID_ERR_MISALIGNED: return "TRID_ERR_MISALIGNED";
        case TRID_ERR_CUDA: return "TRID_ERR_CUDA";
        case TRID_ERR_ALLOC: return "TRID_ERR_ALLOC";
        case TRID_ERR_TIMEOUT: return "TRID_ERR_TIMEOUT";
    }
    return "TRID_ERR_UNKNOWN";
}

namespace trid {
static std::atomic<int> g_last_cuda_error{0};
void note_cuda_error(cudaError_t e) {
    if (e != cudaSuccess) g_last_cuda_error.store(int(e));
}
bool launch_ok() {
    const cudaError_t e = cudaGetLastError();
    note_cuda_error(e);
    return e == cudaSuccess;
}
bool pdl_launch_allowed(cudaStream_t st) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return cs == cudaStreamCaptureStatusNone;
}
static bool nvtx_enabled() {
    static const bool on = [] {
        const char *v = std::getenv("TRID_NVTX");
        return v != nullptr && std::strcmp(v, "1") == 0;
    }();
    return on;
}

NvtxScope::NvtxScope(const char *name) : on(nvtx_enabled()) {
    if (on) nvtxRangePushA(name);
}

NvtxScope::~NvtxScope() {
    if (on) nvtxRangePop();
}
}  // namespace trid

extern "C" const char *trid_last_cuda_error(void) {
    const int e = trid::g_last_cuda_error.load();
    return e == 0 ? "none" : cudaGetErrorString(cudaError_t(e));
}

extern "C" const char *trid_version(void) { return "gb300-trid 0.2 (sm_103a)"; }

extern "C" trid_status trid_init(size_t pool_bytes) {
    if (!trid::device_info()) return TRID_ERR_CUDA;
    if (!trid::device_status_word()) return TRID_ERR_CUDA;
    if (!trid::noalloc_scratch_ready()) return TRID_ERR_CUDA;
    if (!trid::encode_lines_map_ready()) return TRID_ERR_UNSUPPORTED;
    if (!trid::aux_stream()) return TRID_ERR_CUDA;
    if (pool_bytes > 0) {
        void *p = nullptr;
        const trid_status s = trid::pool_reserve(pool_bytes, &p);
        if (s != TRID_OK) return s;
    }
    return TRID_OK;
}

extern "C" trid_status trid_finalize(void) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= trid::kMaxDevices) {
        cudaGetLastError();
        return TRID_ERR_CUDA;
    }
    // work in flight on any stream may still use the pool
    const cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        trid::note_cuda_error(e);
        return TRID_ERR_CUDA;
    }
    trid::forget_device(dev);
    trid::noalloc_forget_device(dev);
    return TRID_OK;
}

namespace trid {
namespace {
constexpr int kMaxDbgReaders = 32;
int (*g_dbg_readers[kMaxDbgReaders])() = {};
int g_ndbg = 0;
}  // namespace

// Called from static initialisers of the debug build's translation units.
int register_dbg_reader(int (*reader)()) {
    if (g_ndbg < kMaxDbgReaders) g_dbg_readers[g_ndbg++] = reader;
    return g_ndbg;
}
}  // namespace trid

extern "C" trid_status trid_get_device_status(trid_stream_t stream) {
    int *w = trid::device_status_word();
    if (!w) return TRID_ERR_CUDA;
    int h = 0;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (cudaMemcpyAsync(&h, w, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return TRID_ERR_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return TRID_ERR_CUDA;
    if (h != 0) {
        const int zero = 0;
        if (cudaMemcpyAsync(w, &zero, sizeof(int), cudaMemcpyHostToDevice, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return TRID_ERR_CUDA;
    }
    // debug build: failed index checks of the kernels (none registered otherwise)
    for (int i = 0; i < trid::g_ndbg; ++i) {
        const int v = trid::g_dbg_readers[i]();
        if (h == 0 && v != 0) h = v;
    }
    return static_cast<trid_status>(h);
}
