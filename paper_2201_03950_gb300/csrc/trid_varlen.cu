// trid_varlen.cu -- a batch of independent systems of different lengths in one
// persistent launch (the batching of Section 4, with the tiled Thomas-PCR
// hybrid of Section 3.1 for the long systems).
//
// System k occupies rows [offsets[k], offsets[k+1]) of a, b, c, d (and u);
// a at its first row and c at its last row are not read.
//
// On the caller's stream, no host synchronisation:
//   plan            a memset of the work struct, k_varlen_hist (length
//                   histogram, ceil log2 buckets) and k_varlen_scatter (order[],
//                   longest bucket first; systems longer than 248 rows first).
//   k_varlen_solve  persistent: every block first pulls long systems from one
//                   atomic counter and solves each with all its threads --
//                   pass 1 reads the system once and writes the two reduced
//                   rows of every 8-row tile to shared memory; the reduced
//                   system (a quarter of the length) is reduced again in
//                   shared memory until it fits one warp, solved with the warp
//                   shuffles, and substituted back level by level; pass 2
//                   re-reads the system (now L2-resident), repeats the tile
//                   pass and writes x.  Then the block pulls batches of short
//                   systems (one per warp, lane tiles in registers).
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/trid.h"
#include "trid_device.cuh"
#include "trid_internal.h"

namespace trid {

constexpr int VL_M = 8;               // tile height
constexpr int VL_SHORT = 32 * VL_M;   // most rows (with alignment padding) one warp solves
constexpr int VL_SHORT_N = VL_SHORT - VL_M;  // systems up to this length go to one warp
constexpr int VL_THREADS = 512;       // threads per block of the persistent kernel
constexpr int VL_BUCKETS = 40;
constexpr int VL_PLAN_THREADS = 256;

struct VarlenWork {
    unsigned long long next_long;   // work counters
    unsigned long long next_short;
    unsigned long long hist[VL_BUCKETS];    // systems per length bucket
    unsigned long long cursor[VL_BUCKETS];  // scatter cursors (relative to the bucket base)
};

// Workspace layout: VarlenWork, then order[nsys] (int64).
inline size_t varlen_ws_bytes(int64_t nsys) {
    return (sizeof(VarlenWork) + 255) / 256 * 256 + size_t(nsys) * sizeof(int64_t);
}

// ceil(log2 n) (0 for n <= 1), with every system longer than VL_SHORT_N in a
// bucket >= 9 and every shorter one in a bucket <= 8: the descending order puts
// the long systems (one block each) before the short ones (one warp each).
__device__ __forceinline__ int len_bucket(int64_t n) {
    if (n <= 1) return 0;
    int b = 64 - __clzll((unsigned long long)(n - 1));
    if (n > VL_SHORT_N && b < 9) b = 9;
    return b < VL_BUCKETS ? b : VL_BUCKETS - 1;
}

// Bucket base (start position in the descending order) of bucket b.
__device__ __forceinline__ unsigned long long bucket_base(const VarlenWork *w, int b) {
    unsigned long long base = 0;
    for (int q = VL_BUCKETS - 1; q > b; --q) base += w->hist[q];
    return base;
}

__device__ __forceinline__ unsigned long long n_long_of(const VarlenWork *w) {
    unsigned long long s = 0;
    for (int q = 9; q < VL_BUCKETS; ++q) s += w->hist[q];
    return s;
}

// A system is usable when its rows lie inside [0, total).
__device__ __forceinline__ bool sys_valid(int64_t s0, int64_t n, int64_t total) {
    return s0 >= 0 && n >= 0 && s0 + n <= total;
}

// Planning, two kernels after a memset of the work struct: per-block length
// histograms added into the global one, then every block reserves a range of
// each bucket with one atomic and scatters its systems into order[].
__device__ __forceinline__ int64_t plan_len(const int64_t *__restrict__ offsets, int64_t k,
                                            int64_t total, int *status, bool flag) {
    const int64_t s0 = offsets[k];
    const int64_t n = offsets[k + 1] - s0;
    if (!sys_valid(s0, n, total)) {  // skipped by the solve kernel
        if (flag && status) atomicCAS(status, 0, int(TRID_ERR_INVALID_ARG));
        return 0;
    }
    return n;
}

__global__ void __launch_bounds__(VL_PLAN_THREADS)
k_varlen_hist(const int64_t *__restrict__ offsets, int64_t nsys, int64_t total, VarlenWork *work,
              int *status) {
    __shared__ unsigned long long hist[VL_BUCKETS];
    const int tid = threadIdx.x;
    if (tid < VL_BUCKETS) hist[tid] = 0;
    __syncthreads();
    for (int64_t k = int64_t(blockIdx.x) * blockDim.x + tid; k < nsys;
         k += int64_t(gridDim.x) * blockDim.x)
        atomicAdd(&hist[len_bucket(plan_len(offsets, k, total, status, true))], 1ull);
    __syncthreads();
    if (tid < VL_BUCKETS && hist[tid]) atomicAdd(&work->hist[tid], hist[tid]);
}

__global__ void __launch_bounds__(VL_PLAN_THREADS)
k_varlen_scatter(const int64_t *__restrict__ offsets, int64_t nsys, int64_t total,
                 VarlenWork *work, int64_t *__restrict__ order) {
    __shared__ unsigned long long hist[VL_BUCKETS];
    __shared__ unsigned long long start[VL_BUCKETS];
    const int tid = threadIdx.x;
    for (int64_t k0 = int64_t(blockIdx.x) * blockDim.x; k0 < nsys;
         k0 += int64_t(gridDim.x) * blockDim.x) {
        if (tid < VL_BUCKETS) hist[tid] = 0;
        __syncthreads();
        const int64_t k = k0 + tid;
        int b = -1;
        unsigned long long local = 0;
        if (k < nsys) {
            b = len_bucket(plan_len(offsets, k, total, nullptr, false));
            local = atomicAdd(&hist[b], 1ull);
        }
        __syncthreads();
        if (tid < VL_BUCKETS && hist[tid])
            start[tid] = bucket_base(work, tid) + atomicAdd(&work->cursor[tid], hist[tid]);
        __syncthreads();
        if (b >= 0) order[start[b] + local] = k;
        __syncthreads();
    }
}

// ---- shared-memory reduced systems: a level holds R rows (unit diagonal) ---
template <typename T>
struct RLevel {
    T *a, *c, *d;
    int R;
};

// Tile pass of level `src` (tiles of 8 rows) into the reduced rows of `dst`.
template <typename T>
__device__ void level_reduce(const RLevel<T> &src, RLevel<T> &dst) {
    const int nt = (src.R + VL_M - 1) / VL_M;
    for (int t = threadIdx.x; t < nt; t += blockDim.x) {
        T ra[VL_M], rb[VL_M], rc[VL_M], rd[VL_M];
#pragma unroll
        for (int j = 0; j < VL_M; ++j) {
            const int i = t * VL_M + j;
            const bool in = i < src.R;
            ra[j] = (in && i > 0) ? src.a[i] : T(0);
            rb[j] = T(1);
            rc[j] = (in && i < src.R - 1) ? src.c[i] : T(0);
            rd[j] = in ? src.d[i] : T(0);
        }
        T as, cs, ds, ae, ce, de;
        tile_reduce<T, VL_M>(ra, rb, rc, rd, as, cs, ds, ae, ce, de);
        dst.a[2 * t] = as; dst.c[2 * t] = cs; dst.d[2 * t] = ds;
        dst.a[2 * t + 1] = ae; dst.c[2 * t + 1] = ce; dst.d[2 * t + 1] = de;
    }
}

// Substitute the solution of `dst` (held in dst.d) back into level `src`,
// writing src's solution into src.d.
template <typename T>
__device__ void level_substitute(RLevel<T> &src, const RLevel<T> &dst) {
    const int nt = (src.R + VL_M - 1) / VL_M;
    for (int t = threadIdx.x; t < nt; t += blockDim.x) {
        T ra[VL_M], rb[VL_M], rc[VL_M], rd[VL_M];
#pragma unroll
        for (int j = 0; j < VL_M; ++j) {
            const int i = t * VL_M + j;
            const bool in = i < src.R;
            ra[j] = (in && i > 0) ? src.a[i] : T(0);
            rb[j] = T(1);
            rc[j] = (in && i < src.R - 1) ? src.c[i] : T(0);
            rd[j] = in ? src.d[i] : T(0);
        }
        T as, cs, ds, ae, ce, de;
        tile_reduce<T, VL_M>(ra, rb, rc, rd, as, cs, ds, ae, ce, de);
        tile_substitute<T, VL_M>(ra, rc, rd, dst.d[2 * t], dst.d[2 * t + 1]);
#pragma unroll
        for (int j = 0; j < VL_M; ++j)
            if (t * VL_M + j < src.R) src.d[t * VL_M + j] = rd[j];
    }
}

// One warp solves a level of R <= 256 rows in place (lane tiles, shuffles).
template <typename T>
__device__ void level_warp_solve(RLevel<T> &lv) {
    const int lane = threadIdx.x & 31;
    T ra[VL_M], rb[VL_M], rc[VL_M], rd[VL_M];
#pragma unroll
    for (int j = 0; j < VL_M; ++j) {
        const int i = lane * VL_M + j;
        const bool in = i < lv.R;
        ra[j] = (in && i > 0) ? lv.a[i] : T(0);
        rb[j] = T(1);
        rc[j] = (in && i < lv.R - 1) ? lv.c[i] : T(0);
        rd[j] = in ? lv.d[i] : T(0);
    }
    T as, cs, ds, ae, ce, de, xs, xe;
    tile_reduce<T, VL_M>(ra, rb, rc, rd, as, cs, ds, ae, ce, de);
    group_solve<T, 32>(as, cs, ds, ae, ce, de, lane, xs, xe);
    tile_substitute<T, VL_M>(ra, rc, rd, xs, xe);
#pragma unroll
    for (int j = 0; j < VL_M; ++j)
        if (lane * VL_M + j < lv.R) lv.d[lane * VL_M + j] = rd[j];
}

// Tiles of a system are aligned to 16 bytes: the system starting at element
// s0 is read as if it began `pad` = s0 mod (16 / sizeof(T)) identity rows
// earlier (a = c = d = 0, b = 1: decoupled, x = 0), so every tile starts on a
// 16-byte boundary and is loaded with vector loads when it lies inside the
// arrays.  Row j of tile t is system row 8t + j - pad.
template <typename T>
__device__ __forceinline__ int sys_pad(int64_t s0) {
    return int(s0 % (16 / int(sizeof(T))));
}

template <typename T>
__device__ __forceinline__ void load_sys_tile(const T *__restrict__ a, const T *__restrict__ b,
                                              const T *__restrict__ c, const T *d, int64_t s0,
                                              int64_t n, int pad, int64_t total, int64_t t,
                                              T (&ra)[VL_M], T (&rb)[VL_M], T (&rc)[VL_M],
                                              T (&rd)[VL_M]) {
    const int64_t p0 = s0 - pad + t * VL_M;  // element of tile row 0 (16-byte aligned)
    const int64_t i0 = t * VL_M - pad;       // system row of tile row 0
    if (p0 + VL_M <= total) {
        load_contig_vec<T, VL_M>(a + p0, ra);
        load_contig_vec<T, VL_M>(b + p0, rb);
        load_contig_vec<T, VL_M>(c + p0, rc);
        load_contig_vec<T, VL_M>(d + p0, rd);
    } else {
#pragma unroll
        for (int j = 0; j < VL_M; ++j) {
            const bool in = p0 + j < total;
            ra[j] = in ? a[p0 + j] : T(0);
            rb[j] = in ? b[p0 + j] : T(1);
            rc[j] = in ? c[p0 + j] : T(0);
            rd[j] = in ? d[p0 + j] : T(0);
        }
    }
#pragma unroll
    for (int j = 0; j < VL_M; ++j) {
        const int64_t i = i0 + j;
        if (i < 0 || i >= n) { ra[j] = T(0); rb[j] = T(1); rc[j] = T(0); rd[j] = T(0); }
        if (i == 0) ra[j] = T(0);
        if (i == n - 1) rc[j] = T(0);
    }
}

template <typename T>
__device__ __forceinline__ void store_sys_tile(T *out, int accumulate, int64_t s0, int64_t n,
                                               int pad, int64_t total, int64_t t,
                                               const T (&rd)[VL_M]) {
    const int64_t p0 = s0 - pad + t * VL_M;
    const int64_t i0 = t * VL_M - pad;
    if (i0 >= 0 && i0 + VL_M <= n && !accumulate) {
        store_contig_vec<T, VL_M>(out + p0, rd);
        return;
    }
#pragma unroll
    for (int j = 0; j < VL_M; ++j) {
        const int64_t i = i0 + j;
        if (i >= 0 && i < n) {
            if (accumulate) out[p0 + j] += rd[j];
            else out[p0 + j] = rd[j];
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(VL_THREADS, sizeof(T) == 4 ? 2 : 1)
k_varlen_solve(const T *__restrict__ a, const T *__restrict__ b, const T *__restrict__ c, const T *d,
               T *out, int accumulate, const int64_t *__restrict__ offsets, int64_t nsys,
               int64_t total, int64_t max_len, VarlenWork *work,
               const int64_t *__restrict__ order, int nlevels, int *status) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ long long s_item;
    // level sizes for the longest admissible system
    RLevel<T> lv[8];
    {
        T *p = reinterpret_cast<T *>(smem_raw);
        int64_t R = 2 * ((max_len + 2 * VL_M - 1) / VL_M);  // includes alignment padding
        for (int l = 0; l < nlevels; ++l) {
            lv[l].a = p; lv[l].c = p + R; lv[l].d = p + 2 * R;
            p += 3 * R;
            R = 2 * ((R + VL_M - 1) / VL_M);
        }
    }
    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    const int64_t n_long = int64_t(n_long_of(work));

    // ---- long systems: one per block
    for (;;) {
        if (tid == 0) s_item = (long long)atomicAdd(&work->next_long, 1ull);
        __syncthreads();
        const int64_t item = s_item;
        __syncthreads();
        if (item >= n_long) break;
        const int64_t k = order[item];
        const int64_t s0 = offsets[k];
        const int64_t n = offsets[k + 1] - s0;
        if (!sys_valid(s0, n, total) || n > max_len) {
            if (tid == 0 && status) atomicCAS(status, 0, int(TRID_ERR_INVALID_ARG));
            continue;
        }
        const int pad = sys_pad<T>(s0);
        const int64_t ntiles = (n + pad + VL_M - 1) / VL_M;
        // pass 1: tile reduction of the system into level 0
        lv[0].R = int(2 * ntiles);
        for (int64_t t = tid; t < ntiles; t += blockDim.x) {
            T ra[VL_M], rb[VL_M], rc[VL_M], rd[VL_M];
            load_sys_tile<T>(a, b, c, d, s0, n, pad, total, t, ra, rb, rc, rd);
            T as, cs, ds, ae, ce, de;
            tile_reduce<T, VL_M>(ra, rb, rc, rd, as, cs, ds, ae, ce, de);
            lv[0].a[2 * t] = as; lv[0].c[2 * t] = cs; lv[0].d[2 * t] = ds;
            lv[0].a[2 * t + 1] = ae; lv[0].c[2 * t + 1] = ce; lv[0].d[2 * t + 1] = de;
        }
        __syncthreads();
        // reduce in shared memory until one warp can solve the top level
        int top = 0;
        while (lv[top].R > VL_SHORT && top + 1 < nlevels) {
            lv[top + 1].R = 2 * ((lv[top].R + VL_M - 1) / VL_M);
            level_reduce<T>(lv[top], lv[top + 1]);
            __syncthreads();
            ++top;
        }
        if (warp == 0) level_warp_solve<T>(lv[top]);
        __syncthreads();
        for (int l = top - 1; l >= 0; --l) {
            level_substitute<T>(lv[l], lv[l + 1]);
            __syncthreads();
        }
        // pass 2: recompute every tile and substitute its end values
        for (int64_t t = tid; t < ntiles; t += blockDim.x) {
            T ra[VL_M], rb[VL_M], rc[VL_M], rd[VL_M];
            load_sys_tile<T>(a, b, c, d, s0, n, pad, total, t, ra, rb, rc, rd);
            T as, cs, ds, ae, ce, de;
            tile_reduce<T, VL_M>(ra, rb, rc, rd, as, cs, ds, ae, ce, de);
            tile_substitute<T, VL_M>(ra, rc, rd, lv[0].d[2 * t], lv[0].d[2 * t + 1]);
            store_sys_tile<T>(out, accumulate, s0, n, pad, total, t, rd);
        }
        __syncthreads();  // level 0 is rewritten by the next system
    }

    // ---- short systems: one per warp
    const int64_t n_short = nsys - n_long;
    for (;;) {
        long long item = 0;
        if (lane == 0) item = (long long)atomicAdd(&work->next_short, 1ull);
        item = __shfl_sync(0xffffffffu, item, 0);
        if (item >= n_short) break;
        const int64_t k = order[n_long + item];
        const int64_t s0 = offsets[k];
        const int64_t n = offsets[k + 1] - s0;
        if (n <= 0 || n > VL_SHORT_N || !sys_valid(s0, n, total)) continue;
        const int pad = sys_pad<T>(s0);
        T ra[VL_M], rb[VL_M], rc[VL_M], rd[VL_M];
        load_sys_tile<T>(a, b, c, d, s0, n, pad, total, lane, ra, rb, rc, rd);
        T as, cs, ds, ae, ce, de, xs, xe;
        tile_reduce<T, VL_M>(ra, rb, rc, rd, as, cs, ds, ae, ce, de);
        group_solve<T, 32>(as, cs, ds, ae, ce, de, lane, xs, xe);
        tile_substitute<T, VL_M>(ra, rc, rd, xs, xe);
        store_sys_tile<T>(out, accumulate, s0, n, pad, total, lane, rd);
    }
}

// Levels and shared-memory bytes for systems up to max_len rows.
template <typename T>
static bool varlen_levels(int64_t max_len, int &nlevels, size_t &smem) {
    int64_t R = 2 * ((max_len + 2 * VL_M - 1) / VL_M);
    nlevels = 0;
    size_t rows = 0;
    for (;;) {
        rows += 3 * size_t(R);
        ++nlevels;
        if (R <= VL_SHORT) break;
        if (nlevels >= 8) return false;
        R = 2 * ((R + VL_M - 1) / VL_M);
    }
    smem = rows * sizeof(T);
    return true;
}

template <typename T>
static trid_status varlen_run(const T *a, const T *b, const T *c, const T *d, T *out, int acc,
                              const int64_t *offsets, int64_t nsys, int64_t total, int64_t max_len,
                              void *ws, cudaStream_t st) {
    int nlevels = 0;
    size_t smem = 0;
    if (!varlen_levels<T>(max_len, nlevels, smem)) return TRID_ERR_UNSUPPORTED;
    const DeviceInfo *di = device_info();
    if (!di) return TRID_ERR_CUDA;
    if (smem > size_t(di->max_smem_optin) - 512) return TRID_ERR_UNSUPPORTED;
    VarlenWork *work = static_cast<VarlenWork *>(ws);
    int64_t *order =
        reinterpret_cast<int64_t *>(static_cast<char *>(ws) + (sizeof(VarlenWork) + 255) / 256 * 256);
    int64_t pblocks = (nsys + VL_PLAN_THREADS - 1) / VL_PLAN_THREADS;
    if (pblocks > 4 * int64_t(di->sm_count)) pblocks = 4 * int64_t(di->sm_count);
    if (cudaMemsetAsync(work, 0, sizeof(VarlenWork), st) != cudaSuccess) return TRID_ERR_CUDA;
    k_varlen_hist<<<dim3(unsigned(pblocks)), VL_PLAN_THREADS, 0, st>>>(offsets, nsys, total, work,
                                                                      device_status_word());
    k_varlen_scatter<<<dim3(unsigned(pblocks)), VL_PLAN_THREADS, 0, st>>>(offsets, nsys, total,
                                                                         work, order);
    if (cudaGetLastError() != cudaSuccess) return TRID_ERR_CUDA;
    auto kern = k_varlen_solve<T>;
    const int per_sm = kernel_blocks_per_sm(reinterpret_cast<const void *>(kern), VL_THREADS, smem);
    if (per_sm < 1) return TRID_ERR_UNSUPPORTED;
    int64_t grid = int64_t(di->sm_count) * per_sm;
    kern<<<dim3(unsigned(grid)), VL_THREADS, smem, st>>>(a, b, c, d, out, acc, offsets, nsys,
                                                         total, max_len, work, order, nlevels,
                                                         device_status_word());
    return cudaGetLastError() == cudaSuccess ? TRID_OK : TRID_ERR_CUDA;
}

}  // namespace trid

using namespace trid;

extern "C" size_t trid_solve_varlen_workspace_bytes(int64_t nsys) {
    if (nsys < 0) return 0;
    return varlen_ws_bytes(nsys);
}

extern "C" trid_status trid_solve_batch_varlen(const void *a, const void *b, const void *c,
                                               void *d, void *u, const int64_t *offsets,
                                               int64_t nsys, int64_t total, int64_t max_len,
                                               trid_dtype dtype, void *workspace,
                                               size_t workspace_bytes, trid_stream_t stream) {
    if (dtype != TRID_F32 && dtype != TRID_F64) return TRID_ERR_INVALID_ARG;
    if (nsys < 0 || total < 0 || max_len < 0) return TRID_ERR_INVALID_ARG;
    if (nsys == 0 || total == 0) return TRID_OK;
    if (!a || !b || !c || !d || !offsets) return TRID_ERR_INVALID_ARG;
    const size_t esz = dtype == TRID_F32 ? 4 : 8;
    const void *ptrs[5] = {a, b, c, d, u};
    for (int k = 0; k < 5; ++k)
        if (ptrs[k] && (reinterpret_cast<uintptr_t>(ptrs[k]) % esz) != 0) return TRID_ERR_MISALIGNED;
    if (reinterpret_cast<uintptr_t>(offsets) % 8 != 0) return TRID_ERR_MISALIGNED;
    if (u) {
        const char *pu = static_cast<const char *>(u);
        const size_t bytes = size_t(total) * esz;
        for (int k = 0; k < 4; ++k) {
            const char *q = static_cast<const char *>(ptrs[k]);
            if (pu < q + bytes && q < pu + bytes) return TRID_ERR_INVALID_ARG;
        }
    }
    if (!workspace || workspace_bytes < varlen_ws_bytes(nsys)) return TRID_ERR_ALLOC;
    if ((reinterpret_cast<uintptr_t>(workspace) % 256) != 0) return TRID_ERR_MISALIGNED;
    if (max_len == 0) max_len = 1;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const int acc = u ? 1 : 0;
    if (dtype == TRID_F32)
        return varlen_run<float>(static_cast<const float *>(a), static_cast<const float *>(b),
                                 static_cast<const float *>(c), static_cast<const float *>(d),
                                 static_cast<float *>(u ? u : d), acc, offsets, nsys, total,
                                 max_len, workspace, st);
    return varlen_run<double>(static_cast<const double *>(a), static_cast<const double *>(b),
                              static_cast<const double *>(c), static_cast<const double *>(d),
                              static_cast<double *>(u ? u : d), acc, offsets, nsys, total,
                              max_len, workspace, st);
}
