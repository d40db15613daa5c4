// trid_varlen.cu -- a batch of independent systems of different lengths in one
// persistent launch (the batching of Section 4, with the tiled Thomas-PCR
// hybrid of Section 3.1 for the long systems).
//
// System k occupies rows [offsets[k], offsets[k+1]) of a, b, c, d (and u);
// a at its first row and c at its last row are not read.
//
// On the caller's stream, no host synchronisation:
//   plan            a memset of the work struct, k_varlen_hist (length
//                   histogram, ceil log2 buckets with the class boundaries
//                   below forced onto bucket edges) and k_varlen_scatter
//                   (meta[]: first row and length, longest bucket first).
//   k_varlen_solve  persistent; every block takes the classes in turn, each
//                   from its own atomic counter, longest first (row limits
//                   for tiles of M = 8 rows; tile_rows 16 doubles them):
//     L   (> 4088 rows)  one system per block, two passes: pass 1 reads the
//                        system and writes the two reduced rows of every
//                        M-row tile to shared memory; the reduced system is
//                        reduced again in shared memory until it has at most
//                        two rows per thread, solved there by block-wide PCR
//                        (stopping once the couplings are below 1/16 ulp) and
//                        substituted back level by level; pass 2 re-reads the
//                        system (L2-resident), repeats the tile pass and
//                        writes x.
//     M2  (<= 4088)      one system per block, one pass: every thread keeps
//                        its tile in registers through the reduced solve.
//     M1  (<= 1016)      one system per team of 4 warps (4 teams per block,
//                        named barriers), one pass, the reduced system (<= 256
//                        rows) solved by the team's first warp.
//     S   (<= 248)       one system per warp, lane tiles and shuffles.
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/trid.h"
#include "trid_device.cuh"
#include "trid_internal.h"

namespace trid {

// Tile height M (rows per thread) is a template parameter: 8 (any dtype) or
// 16 (FP32).  The class limits follow from it.
constexpr int VL_THREADS = 512;       // threads per block of the persistent kernel
constexpr int VL_TEAM = 128;          // threads of an M1 team (default; 64 is the other choice)
constexpr int VL_TEAM_MIN = 64;
constexpr int VL_BUCKETS = 40;
constexpr int VL_PLAN_THREADS = 256;
__host__ __device__ constexpr int vl_log2(int m) { return m == 16 ? 4 : 3; }
__host__ __device__ constexpr int vl_short_n(int m) { return 32 * m - m; }   // one warp
__host__ __device__ constexpr int vl_m1_n(int m) { return VL_TEAM * m - m; }  // one team
__host__ __device__ constexpr int vl_m2_n(int m) { return VL_THREADS * m - m; }  // one block
// Buckets are ceil log2 of the length, raised to the class edges for lengths
// above the smaller class's limit.  The first M1 bucket is fixed; the first M2
// and L buckets (e1, e2) are run-time choices (trid_varlen_config, picked by
// trid_varlen_autotune): a class spanning buckets [lo, hi) holds lengths up to
// 2^(hi-1) - M, the padding of a 16-byte-aligned tile start included.
__host__ __device__ constexpr int vl_b_m1(int m) { return 6 + vl_log2(m); }
__host__ __device__ constexpr int vl_e1_default(int m) { return 8 + vl_log2(m); }  // M1 <= 128 M - M
__host__ __device__ constexpr int vl_e2_default(int m) { return 10 + vl_log2(m); }  // M2 <= 512 M - M

__host__ __device__ __forceinline__ int64_t vl_class_max(int edge, int m) {
    return (int64_t(1) << (edge - 1)) - m;
}

struct VarlenWork {
    unsigned long long next_long;   // work counters: class L
    unsigned long long next_short;  // class S
    unsigned long long next_m2;     // class M2
    unsigned long long next_m1;     // class M1
    unsigned long long hist[VL_BUCKETS];    // systems per length bucket
    unsigned long long cursor[VL_BUCKETS];  // scatter cursors (relative to the bucket base)
};

// Workspace layout: VarlenWork, then meta[nsys]: (first row, length) of the
// systems in solve order (int64 pairs).
inline size_t varlen_ws_bytes(int64_t nsys) {
    return (sizeof(VarlenWork) + 255) / 256 * 256 + size_t(nsys) * sizeof(longlong2);
}

// ceil(log2 n) (0 for n <= 1), raised so that each class occupies whole
// buckets (for M = 8: S <= 8, M1 9..10, M2 11..12, L >= 13; every length fits
// its class: 2^8 = 256 > 248, 2^10 = 1024 > 1016, 2^12 = 4096 > 4088).
__device__ __forceinline__ int len_bucket(int64_t n, int e1, int e2, int m) {
    if (n <= 1) return 0;
    int b = 64 - __clzll((unsigned long long)(n - 1));
    if (n > vl_short_n(m) && b < vl_b_m1(m)) b = vl_b_m1(m);
    if (e1 > vl_b_m1(m) && n > vl_class_max(e1, m) && b < e1) b = e1;
    if (n > vl_class_max(e2, m) && b < e2) b = e2;
    return b < VL_BUCKETS ? b : VL_BUCKETS - 1;
}

// Bucket base (start position in the descending order) of bucket b.
__device__ __forceinline__ unsigned long long bucket_base(const VarlenWork *w, int b) {
    unsigned long long base = 0;
    for (int q = VL_BUCKETS - 1; q > b; --q) base += w->hist[q];
    return base;
}

// Systems in buckets [lo, hi).
__device__ __forceinline__ unsigned long long n_in_buckets(const VarlenWork *w, int lo, int hi) {
    unsigned long long s = 0;
    for (int q = lo; q < hi; ++q) s += w->hist[q];
    return s;
}

// A system is usable when its rows lie inside [0, total).
__device__ __forceinline__ bool sys_valid(int64_t s0, int64_t n, int64_t total) {
    return s0 >= 0 && n >= 0 && s0 + n <= total;
}

// Planning, two kernels after a memset of the work struct: per-block length
// histograms added into the global one, then every block reserves a range of
// each bucket with one atomic and scatters its systems into meta[].
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
              int *status, int e1, int e2, int m) {
    __shared__ unsigned long long hist[VL_BUCKETS];
    const int tid = threadIdx.x;
    if (tid < VL_BUCKETS) hist[tid] = 0;
    __syncthreads();
    for (int64_t k = int64_t(blockIdx.x) * blockDim.x + tid; k < nsys;
         k += int64_t(gridDim.x) * blockDim.x)
        atomicAdd(&hist[len_bucket(plan_len(offsets, k, total, status, true), e1, e2, m)], 1ull);
    __syncthreads();
    if (tid < VL_BUCKETS && hist[tid]) atomicAdd(&work->hist[tid], hist[tid]);
}

__global__ void __launch_bounds__(VL_PLAN_THREADS)
k_varlen_scatter(const int64_t *__restrict__ offsets, int64_t nsys, int64_t total,
                 VarlenWork *work, longlong2 *__restrict__ meta, int e1, int e2, int m) {
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
            b = len_bucket(plan_len(offsets, k, total, nullptr, false), e1, e2, m);
            local = atomicAdd(&hist[b], 1ull);
        }
        __syncthreads();
        if (tid < VL_BUCKETS && hist[tid])
            start[tid] = bucket_base(work, tid) + atomicAdd(&work->cursor[tid], hist[tid]);
        __syncthreads();
        if (b >= 0) {
            const int64_t s0 = offsets[k];
            meta[start[b] + local] = make_longlong2(s0, offsets[k + 1] - s0);
        }
        __syncthreads();
    }
}

__device__ __forceinline__ void named_barrier_sync(int id, int nthreads) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

// ---- shared-memory reduced systems: a level holds R rows (unit diagonal) ---
// Rows are padded by one element per 128 bytes (row i at i + i / 32 in FP32,
// i + i / 16 in FP64): a warp whose threads each walk M consecutive rows (a
// stride of M elements) then hits 32 different banks, where the unpadded
// rows put the whole warp on M-fold shared banks.
template <typename T>
__host__ __device__ constexpr int vpad_shift() { return sizeof(T) == 4 ? 5 : 4; }
template <typename T>
__host__ __device__ constexpr int64_t vpad_len(int64_t R) {  // elements for R padded rows
    return R + (R >> vpad_shift<T>()) + 1;
}
template <typename T>
struct RLevel {
    T *a, *c, *d;  // padded arrays: use A, C, D
    int R;
    __device__ __forceinline__ T &A(int i) const { return a[i + (i >> vpad_shift<T>())]; }
    __device__ __forceinline__ T &C(int i) const { return c[i + (i >> vpad_shift<T>())]; }
    __device__ __forceinline__ T &D(int i) const { return d[i + (i >> vpad_shift<T>())]; }
};

// Tile pass of level `src` (tiles of M rows) into the reduced rows of `dst`.
template <typename T, int VL_M>
__device__ __forceinline__ void level_reduce(const RLevel<T> &src, RLevel<T> &dst) {
    const int nt = (src.R + VL_M - 1) / VL_M;
    for (int t = threadIdx.x; t < nt; t += blockDim.x) {
        T ra[VL_M], rb[VL_M], rc[VL_M], rd[VL_M];
#pragma unroll
        for (int j = 0; j < VL_M; ++j) {
            const int i = t * VL_M + j;
            const bool in = i < src.R;
            ra[j] = (in && i > 0) ? src.A(i) : T(0);
            rb[j] = T(1);
            rc[j] = (in && i < src.R - 1) ? src.C(i) : T(0);
            rd[j] = in ? src.D(i) : T(0);
        }
        T as, cs, ds, ae, ce, de;
        tile_reduce<T, VL_M>(ra, rb, rc, rd, as, cs, ds, ae, ce, de);
        dst.A(2 * t) = as; dst.C(2 * t) = cs; dst.D(2 * t) = ds;
        dst.A(2 * t + 1) = ae; dst.C(2 * t + 1) = ce; dst.D(2 * t + 1) = de;
    }
}

// Substitute the solution of `dst` (held in dst.d) back into level `src`,
// writing src's solution into src.d.
template <typename T, int VL_M>
__device__ __forceinline__ void level_substitute(RLevel<T> &src, const RLevel<T> &dst) {
    const int nt = (src.R + VL_M - 1) / VL_M;
    for (int t = threadIdx.x; t < nt; t += blockDim.x) {
        T ra[VL_M], rb[VL_M], rc[VL_M], rd[VL_M];
#pragma unroll
        for (int j = 0; j < VL_M; ++j) {
            const int i = t * VL_M + j;
            const bool in = i < src.R;
            ra[j] = (in && i > 0) ? src.A(i) : T(0);
            rb[j] = T(1);
            rc[j] = (in && i < src.R - 1) ? src.C(i) : T(0);
            rd[j] = in ? src.D(i) : T(0);
        }
        T as, cs, ds, ae, ce, de;
        tile_reduce<T, VL_M>(ra, rb, rc, rd, as, cs, ds, ae, ce, de);
        tile_substitute<T, VL_M>(ra, rc, rd, dst.D(2 * t), dst.D(2 * t + 1));
#pragma unroll
        for (int j = 0; j < VL_M; ++j)
            if (t * VL_M + j < src.R) src.D(t * VL_M + j) = rd[j];
    }
}

// One warp solves a level of R <= 32 M rows in place (lane tiles, shuffles).
template <typename T, int VL_M>
__device__ __forceinline__ void level_warp_solve(RLevel<T> &lv) {
    const int lane = threadIdx.x & 31;
    T ra[VL_M], rb[VL_M], rc[VL_M], rd[VL_M];
#pragma unroll
    for (int j = 0; j < VL_M; ++j) {
        const int i = lane * VL_M + j;
        const bool in = i < lv.R;
        ra[j] = (in && i > 0) ? lv.A(i) : T(0);
        rb[j] = T(1);
        rc[j] = (in && i < lv.R - 1) ? lv.C(i) : T(0);
        rd[j] = in ? lv.D(i) : T(0);
    }
    T as, cs, ds, ae, ce, de, xs, xe;
    tile_reduce<T, VL_M>(ra, rb, rc, rd, as, cs, ds, ae, ce, de);
    group_solve<T, 32>(as, cs, ds, ae, ce, de, lane, xs, xe);
    tile_substitute<T, VL_M>(ra, rc, rd, xs, xe);
#pragma unroll
    for (int j = 0; j < VL_M; ++j)
        if (lane * VL_M + j < lv.R) lv.D(lane * VL_M + j) = rd[j];
}

// Tiles of a system are aligned to 16 bytes: the system starting at element
// s0 is read as if it began `pad` = s0 mod (16 / sizeof(T)) identity rows
// earlier (a = c = d = 0, b = 1: decoupled, x = 0), so every tile starts on a
// 16-byte boundary and is loaded with vector loads when it lies inside the
// arrays.  Row j of tile t is system row M t + j - pad.
template <typename T>
__device__ __forceinline__ int sys_pad(int64_t s0) {
    return int(s0 % (16 / int(sizeof(T))));
}

template <typename T, int VL_M>
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

template <typename T, int VL_M>
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

// Parallel cyclic reduction (Algorithm "pcr") of one unit-diagonal level held
// in shared memory, by the whole block: the calling thread owns rows tid and
// tid + blockDim.x (R <= 2 blockDim.x).  Each round reads the neighbours it
// needs into registers, waits for the block, then writes.  On a diagonally
// dominant system every round squares the coupling coefficients; once all of
// them are below 2^-(p+4) (p the significand bits) the remaining rounds change
// no value by more than 1/16 ulp, and the level's d holds the solution.
template <typename T>
__device__ __forceinline__ void block_pcr(RLevel<T> &lv) {
    constexpr float negligible = sizeof(T) == 4 ? 3.7252903e-09f : 6.9388939e-18f;
    const int R = lv.R, nth = blockDim.x, tid = threadIdx.x;
    float cpl = 0.0f;
    for (int i = tid; i < R; i += nth)
        cpl = fmaxf(cpl, float(fmax(fabs(lv.A(i)), fabs(lv.C(i)))));
    if (!__syncthreads_or(cpl >= negligible)) return;
    for (int s = 1; s < R; s <<= 1) {
        T na[2], nc[2], nd[2];
        float cmax = 0.0f;
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int i = tid + q * nth;
            na[q] = nc[q] = nd[q] = T(0);
            if (i < R) {
                const T ai = lv.A(i), ci = lv.C(i), di = lv.D(i);
                T am = T(0), cm = T(0), dm = T(0), ap = T(0), cp = T(0), dp = T(0);
                if (i - s >= 0) { am = lv.A(i - s); cm = lv.C(i - s); dm = lv.D(i - s); }
                if (i + s < R) { ap = lv.A(i + s); cp = lv.C(i + s); dp = lv.D(i + s); }
                const T r = rcp(T(1) - ai * cm - ci * ap);
                na[q] = -r * (ai * am);
                nc[q] = -r * (ci * cp);
                nd[q] = r * (di - ai * dm - ci * dp);
                cmax = fmaxf(cmax, float(fmax(fabs(na[q]), fabs(nc[q]))));
            }
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int i = tid + q * nth;
            if (i < R) { lv.A(i) = na[q]; lv.C(i) = nc[q]; lv.D(i) = nd[q]; }
        }
        if (!__syncthreads_or(cmax >= negligible)) break;
    }
}

// Level l of the shared-memory hierarchy (R rows of data): its arrays sit
// after the padded arrays of the levels above it, each sized for the longest
// admissible system (level 0 holds rmax0 rows).  The pointers are formed from
// the shared-memory base at every use (never kept in an indexed array, which
// would put them in local memory), so the accesses compile to shared-memory
// loads and stores rather than generic ones.
template <typename T, int VL_M>
__device__ __forceinline__ RLevel<T> level_at(T *sbase, int rmax0, int l, int R) {
    int64_t off = 0, rm = rmax0;
    for (int k = 0; k < l; ++k) {
        off += 3 * vpad_len<T>(rm);
        rm = 2 * ((rm + VL_M - 1) / VL_M);
    }
    const int64_t P = vpad_len<T>(rm);
    RLevel<T> v;
    v.a = sbase + off;
    v.c = v.a + P;
    v.d = v.a + 2 * P;
    v.R = R;
    return v;
}

// Rows of level l of a system whose level 0 holds R0 rows.
template <int VL_M>
__device__ __forceinline__ int level_rows(int R0, int l) {
    int R = R0;
    for (int k = 0; k < l; ++k) R = 2 * ((R + VL_M - 1) / VL_M);
    return R;
}

// Solve the reduced system held in level 0 (R0 rows already written, block
// synchronised): tile passes in shared memory while it is longer than two rows
// per thread, the block PCR on the top level, then substitution back down to
// level 0 (whose solution is then in its d).  All threads of the block call it.
template <typename T, int VL_M>
__device__ __forceinline__ void block_reduced_solve(T *sbase, int rmax0, int R0, int nlevels) {
    int top = 0, R = R0;
    while (R > 2 * int(blockDim.x) && top + 1 < nlevels) {
        const int Rn = 2 * ((R + VL_M - 1) / VL_M);
        RLevel<T> dst = level_at<T, VL_M>(sbase, rmax0, top + 1, Rn);
        level_reduce<T, VL_M>(level_at<T, VL_M>(sbase, rmax0, top, R), dst);
        __syncthreads();
        ++top;
        R = Rn;
    }
    {
        RLevel<T> t = level_at<T, VL_M>(sbase, rmax0, top, R);
        block_pcr<T>(t);
    }
    __syncthreads();
    for (int l = top - 1; l >= 0; --l) {
        const int Rl = level_rows<VL_M>(R0, l);
        RLevel<T> src = level_at<T, VL_M>(sbase, rmax0, l, Rl);
        level_substitute<T, VL_M>(src, level_at<T, VL_M>(sbase, rmax0, l + 1,
                                                         2 * ((Rl + VL_M - 1) / VL_M)));
        __syncthreads();
    }
}

// Work items of a class come from one atomic counter.  One helper thread per
// group (block, team or warp) runs ahead: it takes the next item at the start
// of the current system, loads its (first row, length) after the first
// phase, and publishes it before the last, so the counter and meta[] round
// trips overlap the current system's solve.
struct VItem {
    long long item, s0, n;
};

__device__ __forceinline__ VItem vitem_fetch(unsigned long long *ctr, int64_t limit, int64_t base,
                                             const longlong2 *__restrict__ meta) {
    VItem v;
    v.item = (long long)atomicAdd(ctr, 1ull);
    v.s0 = 0;
    v.n = 0;
    if (v.item < limit) {
        const longlong2 m = meta[base + v.item];
        v.s0 = m.x;
        v.n = m.y;
    }
    return v;
}

template <typename T, int VL_M>
__global__ void __launch_bounds__(VL_THREADS, (sizeof(T) == 4 && VL_M == 8) ? 2 : 1)
k_varlen_solve(const T *__restrict__ a, const T *__restrict__ b, const T *__restrict__ c, const T *d,
               T *out, int accumulate, int64_t nsys, int64_t total, int64_t max_len,
               VarlenWork *work, const longlong2 *__restrict__ meta, int nlevels, int *status,
               int e1, int e2, int team_threads) {
    constexpr int VL_M2_N = vl_m2_n(VL_M), VL_SHORT_N = vl_short_n(VL_M);
    const int64_t m1_max = vl_class_max(e1, VL_M), m2_max = vl_class_max(e2, VL_M);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ VItem s_it[2];
    __shared__ VItem s_team_it[VL_THREADS / VL_TEAM_MIN][2];
    // level sizes for the longest admissible system (at least an M2 system)
    T *const sbase = reinterpret_cast<T *>(smem_raw);
    const int rmax0 = int(2 * (((max_len > VL_M2_N ? max_len : int64_t(VL_M2_N)) + 2 * VL_M - 1) /
                               VL_M));  // includes alignment padding
    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int helper = blockDim.x - 1;
    const int64_t n_l = int64_t(n_in_buckets(work, e2, VL_BUCKETS));
    const int64_t n_m2 = int64_t(n_in_buckets(work, e1, e2));
    const int64_t n_m1 = int64_t(n_in_buckets(work, vl_b_m1(VL_M), e1));
    const int64_t n_s = nsys - n_l - n_m2 - n_m1;

    // ---- class L: one system per block, two passes
    if (tid == helper) s_it[0] = vitem_fetch(&work->next_long, n_l, 0, meta);
    __syncthreads();
    for (int cur = 0;; cur ^= 1) {
        const VItem it = s_it[cur];
        if (it.item >= n_l) break;
        unsigned long long nx_item = 0;
        if (tid == helper) nx_item = atomicAdd(&work->next_long, 1ull);
        const int64_t s0 = it.s0, n = it.n;
        const bool ok = sys_valid(s0, n, total) && n <= max_len;
        if (!ok && tid == 0 && status) atomicCAS(status, 0, int(TRID_ERR_INVALID_ARG));
        const int pad = sys_pad<T>(s0);
        const int64_t ntiles = ok ? (n + pad + VL_M - 1) / VL_M : 0;
        // pass 1: tile reduction of the system into level 0
        const RLevel<T> l0 = level_at<T, VL_M>(sbase, rmax0, 0, int(2 * ntiles));
        for (int64_t t = tid; t < ntiles; t += blockDim.x) {
            T ra[VL_M], rb[VL_M], rc[VL_M], rd[VL_M];
            load_sys_tile<T, VL_M>(a, b, c, d, s0, n, pad, total, t, ra, rb, rc, rd);
            T as, cs, ds, ae, ce, de;
            tile_reduce<T, VL_M>(ra, rb, rc, rd, as, cs, ds, ae, ce, de);
            l0.A(2 * t) = as; l0.C(2 * t) = cs; l0.D(2 * t) = ds;
            l0.A(2 * t + 1) = ae; l0.C(2 * t + 1) = ce; l0.D(2 * t + 1) = de;
        }
        longlong2 nx_meta = make_longlong2(0, 0);
        if (tid == helper && (long long)nx_item < n_l) nx_meta = meta[nx_item];
        __syncthreads();
        if (ok) block_reduced_solve<T, VL_M>(sbase, rmax0, l0.R, nlevels);
        if (tid == helper) s_it[cur ^ 1] = VItem{(long long)nx_item, nx_meta.x, nx_meta.y};
        // pass 2: recompute every tile and substitute its end values
        for (int64_t t = tid; t < ntiles; t += blockDim.x) {
            T ra[VL_M], rb[VL_M], rc[VL_M], rd[VL_M];
            load_sys_tile<T, VL_M>(a, b, c, d, s0, n, pad, total, t, ra, rb, rc, rd);
            T as, cs, ds, ae, ce, de;
            tile_reduce<T, VL_M>(ra, rb, rc, rd, as, cs, ds, ae, ce, de);
            tile_substitute<T, VL_M>(ra, rc, rd, l0.D(2 * t), l0.D(2 * t + 1));
            store_sys_tile<T, VL_M>(out, accumulate, s0, n, pad, total, t, rd);
        }
        __syncthreads();  // level 0 is rewritten by the next system
    }

    // ---- class M2: one system per block, the tiles stay in registers
    // every thread has read the L class's final item (whose slot may be s_it[0])
    // before the helper reuses the slot: without this barrier a late warp could
    // take the first M2 item for an L item and meet the other warps' barriers
    // on a different path
    __syncthreads();
    if (tid == helper) s_it[0] = vitem_fetch(&work->next_m2, n_m2, n_l, meta);
    __syncthreads();
    for (int cur = 0;; cur ^= 1) {
        const VItem it = s_it[cur];
        if (it.item >= n_m2) break;
        unsigned long long nx_item = 0;
        if (tid == helper) nx_item = atomicAdd(&work->next_m2, 1ull);
        const int64_t s0 = it.s0, n = it.n;
        const bool ok = sys_valid(s0, n, total) && n <= m2_max;
        if (!ok && tid == 0 && status) atomicCAS(status, 0, int(TRID_ERR_INVALID_ARG));
        const int pad = sys_pad<T>(s0);
        const int ntiles = ok ? int((n + pad + VL_M - 1) / VL_M) : 0;  // <= blockDim.x
        const bool mine = tid < ntiles;
        T ra[VL_M], rb[VL_M], rc[VL_M], rd[VL_M];
        const RLevel<T> l0 = level_at<T, VL_M>(sbase, rmax0, 0, 2 * ntiles);
        if (mine) {
            load_sys_tile<T, VL_M>(a, b, c, d, s0, n, pad, total, tid, ra, rb, rc, rd);
            T as, cs, ds, ae, ce, de;
            tile_reduce<T, VL_M>(ra, rb, rc, rd, as, cs, ds, ae, ce, de);
            l0.A(2 * tid) = as; l0.C(2 * tid) = cs; l0.D(2 * tid) = ds;
            l0.A(2 * tid + 1) = ae; l0.C(2 * tid + 1) = ce; l0.D(2 * tid + 1) = de;
        }
        longlong2 nx_meta = make_longlong2(0, 0);
        if (tid == helper && (long long)nx_item < n_m2) nx_meta = meta[n_l + nx_item];
        __syncthreads();
        if (ok) block_reduced_solve<T, VL_M>(sbase, rmax0, l0.R, nlevels);
        if (tid == helper) s_it[cur ^ 1] = VItem{(long long)nx_item, nx_meta.x, nx_meta.y};
        if (mine) {
            tile_substitute<T, VL_M>(ra, rc, rd, l0.D(2 * tid), l0.D(2 * tid + 1));
            store_sys_tile<T, VL_M>(out, accumulate, s0, n, pad, total, tid, rd);
        }
        __syncthreads();
    }

    // ---- class M1: one system per team of 4 warps, tiles in registers
    {
        const int tsz = team_threads;  // 64 or 128: 8 or 4 systems in flight per block
        const int team = tid / tsz, tt = tid % tsz;
        const int bar = 1 + team;  // named barrier of the team (0 is __syncthreads)
        const int thelper = tsz - 1;
        const int64_t base1 = n_l + n_m2;
        // the team's reduced rows: R <= 2 * tsz (padded; the host sizes the
        // shared memory for every team's arrays)
        const int64_t tp = vpad_len<T>(2 * tsz);
        T *tbase = reinterpret_cast<T *>(smem_raw) + size_t(team) * 3 * tp;
        RLevel<T> tl;
        tl.a = tbase; tl.c = tbase + tp; tl.d = tbase + 2 * tp;
        if (tt == thelper) s_team_it[team][0] = vitem_fetch(&work->next_m1, n_m1, base1, meta);
        named_barrier_sync(bar, tsz);
        for (int cur = 0;; cur ^= 1) {
            const VItem it = s_team_it[team][cur];
            if (it.item >= n_m1) break;
            unsigned long long nx_item = 0;
            if (tt == thelper) nx_item = atomicAdd(&work->next_m1, 1ull);
            const int64_t s0 = it.s0, n = it.n;
            const bool ok = sys_valid(s0, n, total) && n <= m1_max;
            if (!ok && tt == 0 && status) atomicCAS(status, 0, int(TRID_ERR_INVALID_ARG));
            const int pad = sys_pad<T>(s0);
            const int ntiles = ok ? int((n + pad + VL_M - 1) / VL_M) : 0;  // <= tsz
            const bool mine = tt < ntiles;
            T ra[VL_M], rb[VL_M], rc[VL_M], rd[VL_M];
            tl.R = 2 * ntiles;
            if (mine) {
                load_sys_tile<T, VL_M>(a, b, c, d, s0, n, pad, total, tt, ra, rb, rc, rd);
                T as, cs, ds, ae, ce, de;
                tile_reduce<T, VL_M>(ra, rb, rc, rd, as, cs, ds, ae, ce, de);
                tl.A(2 * tt) = as; tl.C(2 * tt) = cs; tl.D(2 * tt) = ds;
                tl.A(2 * tt + 1) = ae; tl.C(2 * tt + 1) = ce; tl.D(2 * tt + 1) = de;
            }
            longlong2 nx_meta = make_longlong2(0, 0);
            if (tt == thelper && (long long)nx_item < n_m1) nx_meta = meta[base1 + nx_item];
            named_barrier_sync(bar, tsz);
            if (ok && tt < 32) level_warp_solve<T, VL_M>(tl);
            if (tt == thelper)
                s_team_it[team][cur ^ 1] = VItem{(long long)nx_item, nx_meta.x, nx_meta.y};
            named_barrier_sync(bar, tsz);
            if (mine) {
                tile_substitute<T, VL_M>(ra, rc, rd, tl.D(2 * tt), tl.D(2 * tt + 1));
                store_sys_tile<T, VL_M>(out, accumulate, s0, n, pad, total, tt, rd);
            }
            named_barrier_sync(bar, tsz);  // the team's rows are rewritten next
        }
    }

    // ---- class S: one system per warp; lane 31 runs ahead
    {
        const int64_t base0 = n_l + n_m2 + n_m1;
        VItem it{0, 0, 0};
        if (lane == 31) it = vitem_fetch(&work->next_short, n_s, base0, meta);
        for (;;) {
            const long long item = __shfl_sync(0xffffffffu, it.item, 31);
            if (item >= n_s) break;
            const int64_t s0 = __shfl_sync(0xffffffffu, it.s0, 31);
            const int64_t n = __shfl_sync(0xffffffffu, it.n, 31);
            unsigned long long nx_item = 0;
            if (lane == 31) nx_item = atomicAdd(&work->next_short, 1ull);
            const bool ok = n > 0 && n <= VL_SHORT_N && sys_valid(s0, n, total);
            const int pad = sys_pad<T>(s0);
            T ra[VL_M], rb[VL_M], rc[VL_M], rd[VL_M];
            if (ok) load_sys_tile<T, VL_M>(a, b, c, d, s0, n, pad, total, lane, ra, rb, rc, rd);
            if (lane == 31) {
                it.item = (long long)nx_item;
                it.s0 = 0;
                it.n = 0;
                if ((long long)nx_item < n_s) {
                    const longlong2 m = meta[base0 + nx_item];
                    it.s0 = m.x;
                    it.n = m.y;
                }
            }
            if (!ok) continue;
            T as, cs, ds, ae, ce, de, xs, xe;
            tile_reduce<T, VL_M>(ra, rb, rc, rd, as, cs, ds, ae, ce, de);
            group_solve<T, 32>(as, cs, ds, ae, ce, de, lane, xs, xe);
            tile_substitute<T, VL_M>(ra, rc, rd, xs, xe);
            store_sys_tile<T, VL_M>(out, accumulate, s0, n, pad, total, lane, rd);
        }
    }
}

// Levels and shared-memory bytes for systems up to max_len rows.
template <typename T, int VL_M>
static bool varlen_levels(int64_t max_len, int &nlevels, size_t &smem) {
    constexpr int VL_M2_N = vl_m2_n(VL_M), VL_SHORT = 32 * VL_M;
    if (max_len < VL_M2_N) max_len = VL_M2_N;  // the M2 class uses the same levels
    int64_t R = 2 * ((max_len + 2 * VL_M - 1) / VL_M);
    nlevels = 0;
    size_t rows = 0;
    for (;;) {
        rows += 3 * size_t(vpad_len<T>(R));
        ++nlevels;
        if (R <= VL_SHORT) break;
        if (nlevels >= 8) return false;
        R = 2 * ((R + VL_M - 1) / VL_M);
    }
    smem = rows * sizeof(T);
    // the M1 teams' padded rows (either team size) share the same memory
    for (int tsz = VL_TEAM_MIN; tsz <= VL_TEAM; tsz *= 2) {
        const size_t teams = size_t(VL_THREADS / tsz) * 3 * size_t(vpad_len<T>(2 * tsz)) * sizeof(T);
        if (smem < teams) smem = teams;
    }
    return true;
}

template <typename T, int VL_M>
static trid_status varlen_run(const T *a, const T *b, const T *c, const T *d, T *out, int acc,
                              const int64_t *offsets, int64_t nsys, int64_t total, int64_t max_len,
                              void *ws, cudaStream_t st, int e1, int e2, int team_threads) {
    int nlevels = 0;
    size_t smem = 0;
    if (!varlen_levels<T, VL_M>(max_len, nlevels, smem)) return TRID_ERR_UNSUPPORTED;
    const DeviceInfo *di = device_info();
    if (!di) return TRID_ERR_CUDA;
    if (smem > size_t(di->max_smem_optin) - 512) return TRID_ERR_UNSUPPORTED;
    VarlenWork *work = static_cast<VarlenWork *>(ws);
    longlong2 *meta = reinterpret_cast<longlong2 *>(static_cast<char *>(ws) +
                                                    (sizeof(VarlenWork) + 255) / 256 * 256);
    int64_t pblocks = (nsys + VL_PLAN_THREADS - 1) / VL_PLAN_THREADS;
    if (pblocks > 4 * int64_t(di->sm_count)) pblocks = 4 * int64_t(di->sm_count);
    if (cudaMemsetAsync(work, 0, sizeof(VarlenWork), st) != cudaSuccess) return TRID_ERR_CUDA;
    k_varlen_hist<<<dim3(unsigned(pblocks)), VL_PLAN_THREADS, 0, st>>>(offsets, nsys, total, work,
                                                                      device_status_word(), e1, e2,
                                                                      VL_M);
    k_varlen_scatter<<<dim3(unsigned(pblocks)), VL_PLAN_THREADS, 0, st>>>(offsets, nsys, total,
                                                                         work, meta, e1, e2, VL_M);
    if (cudaGetLastError() != cudaSuccess) return TRID_ERR_CUDA;
    auto kern = k_varlen_solve<T, VL_M>;
    const int per_sm = kernel_blocks_per_sm(reinterpret_cast<const void *>(kern), VL_THREADS, smem);
    if (per_sm < 1) return TRID_ERR_UNSUPPORTED;
    int64_t grid = int64_t(di->sm_count) * per_sm;
    kern<<<dim3(unsigned(grid)), VL_THREADS, smem, st>>>(a, b, c, d, out, acc, nsys, total,
                                                         max_len, work, meta, nlevels,
                                                         device_status_word(), e1, e2,
                                                         team_threads);
    return cudaGetLastError() == cudaSuccess ? TRID_OK : TRID_ERR_CUDA;
}

}  // namespace trid

using namespace trid;

extern "C" size_t trid_solve_varlen_workspace_bytes(int64_t nsys) {
    if (nsys < 0) return 0;
    return varlen_ws_bytes(nsys);
}

// Tile height and class edges of a configuration (see trid_varlen_config in
// include/trid.h); false for a configuration outside the admissible list.
static bool vl_edges(const trid_varlen_config *cfg, trid_dtype dtype, int &m, int &e1, int &e2,
                     int &team_threads) {
    m = 8;
    team_threads = VL_TEAM;
    if (cfg && cfg->tile_rows != 0 && cfg->tile_rows != 8) {
        if (cfg->tile_rows != 16 || dtype != TRID_F32) return false;
        m = 16;
    }
    if (!cfg) { e1 = vl_e1_default(m); e2 = vl_e2_default(m); return true; }
    const int lo = vl_b_m1(m), e1max = vl_e1_default(m), e2max = vl_e2_default(m);
    auto edge_of = [&](int32_t len, int &e) {
        for (int k = lo; k <= e2max; ++k)
            if (vl_class_max(k, m) == len) { e = k; return true; }
        return false;
    };
    if (cfg->team_max == vl_short_n(m)) e1 = lo;
    else if (!edge_of(cfg->team_max, e1) || e1 > e1max) return false;
    if (cfg->block_max == cfg->team_max) e2 = e1;
    else if (!edge_of(cfg->block_max, e2) || e2 > e2max || e2 < e1) return false;
    if (cfg->team_warps != 0 && cfg->team_warps != 4) {
        // teams of 2 warps: only for a team class that fits them
        if (cfg->team_warps != 2 || e1 != lo + 1) return false;
        team_threads = VL_TEAM_MIN;
    }
    return true;
}

static trid_status varlen_entry(const void *a, const void *b, const void *c, void *d, void *u,
                                const int64_t *offsets, int64_t nsys, int64_t total,
                                int64_t max_len, trid_dtype dtype, void *workspace,
                                size_t workspace_bytes, trid_stream_t stream,
                                const trid_varlen_config *cfg) {
    if (dtype != TRID_F32 && dtype != TRID_F64) return TRID_ERR_INVALID_ARG;
    if (nsys < 0 || total < 0 || max_len < 0) return TRID_ERR_INVALID_ARG;
    int m, e1, e2, tt;
    if (!vl_edges(cfg, dtype, m, e1, e2, tt)) return TRID_ERR_INVALID_ARG;
    if (nsys == 0 || total == 0) return TRID_OK;
    if (!a || !b || !c || !d || !offsets) return TRID_ERR_INVALID_ARG;
    const size_t esz = dtype == TRID_F32 ? 4 : 8;
    const void *ptrs[5] = {a, b, c, d, u};
    // the kernels read 16-byte tiles aligned to the arrays' bases
    for (int k = 0; k < 5; ++k)
        if (ptrs[k] && (reinterpret_cast<uintptr_t>(ptrs[k]) % 16) != 0) return TRID_ERR_MISALIGNED;
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
    if (dtype == TRID_F32) {
        const float *fa = static_cast<const float *>(a), *fb = static_cast<const float *>(b);
        const float *fc = static_cast<const float *>(c), *fd = static_cast<const float *>(d);
        float *fo = static_cast<float *>(u ? u : d);
        if (m == 16)
            return varlen_run<float, 16>(fa, fb, fc, fd, fo, acc, offsets, nsys, total, max_len,
                                         workspace, st, e1, e2, tt);
        return varlen_run<float, 8>(fa, fb, fc, fd, fo, acc, offsets, nsys, total, max_len,
                                    workspace, st, e1, e2, tt);
    }
    return varlen_run<double, 8>(static_cast<const double *>(a), static_cast<const double *>(b),
                              static_cast<const double *>(c), static_cast<const double *>(d),
                              static_cast<double *>(u ? u : d), acc, offsets, nsys, total,
                              max_len, workspace, st, e1, e2, tt);
}

extern "C" trid_status trid_solve_batch_varlen(const void *a, const void *b, const void *c,
                                               void *d, void *u, const int64_t *offsets,
                                               int64_t nsys, int64_t total, int64_t max_len,
                                               trid_dtype dtype, void *workspace,
                                               size_t workspace_bytes, trid_stream_t stream) {
    trid::NvtxScope nvtx_scope("trid_solve_batch_varlen");
    return varlen_entry(a, b, c, d, u, offsets, nsys, total, max_len, dtype, workspace,
                        workspace_bytes, stream, nullptr);
}

extern "C" trid_status trid_solve_batch_varlen_cfg(const void *a, const void *b, const void *c,
                                                   void *d, void *u, const int64_t *offsets,
                                                   int64_t nsys, int64_t total, int64_t max_len,
                                                   trid_dtype dtype, void *workspace,
                                                   size_t workspace_bytes, trid_stream_t stream,
                                                   const trid_varlen_config *cfg) {
    trid::NvtxScope nvtx_scope("trid_solve_batch_varlen_cfg");
    return varlen_entry(a, b, c, d, u, offsets, nsys, total, max_len, dtype, workspace,
                        workspace_bytes, stream, cfg);
}

extern "C" size_t trid_varlen_autotune_workspace_bytes(int64_t nsys, int64_t total,
                                                       trid_dtype dtype) {
    if (nsys < 0 || total < 0 || (dtype != TRID_F32 && dtype != TRID_F64)) return 0;
    const size_t esz = dtype == TRID_F32 ? 4 : 8;
    return (varlen_ws_bytes(nsys) + 255) / 256 * 256 + size_t(total) * esz;
}

// Time every admissible configuration on the caller's batch (on a scratch
// copy of d, so d is not modified) and return the fastest.
extern "C" trid_status trid_varlen_autotune(const void *a, const void *b, const void *c,
                                            const void *d, const int64_t *offsets, int64_t nsys,
                                            int64_t total, int64_t max_len, trid_dtype dtype,
                                            void *workspace, size_t workspace_bytes,
                                            trid_stream_t stream, trid_varlen_config *best,
                                            float *best_ms) {
    trid::NvtxScope nvtx_scope("trid_varlen_autotune");
    if (!best) return TRID_ERR_INVALID_ARG;
    best->team_max = int32_t(vl_class_max(vl_e1_default(8), 8));
    best->block_max = int32_t(vl_class_max(vl_e2_default(8), 8));
    best->tile_rows = 8;
    best->team_warps = 4;
    if (best_ms) *best_ms = 0.0f;
    if (dtype != TRID_F32 && dtype != TRID_F64) return TRID_ERR_INVALID_ARG;
    if (nsys < 0 || total < 0 || max_len < 0) return TRID_ERR_INVALID_ARG;
    if (nsys == 0 || total == 0) return TRID_OK;
    if (!a || !b || !c || !d || !offsets) return TRID_ERR_INVALID_ARG;
    if (!workspace || workspace_bytes < trid_varlen_autotune_workspace_bytes(nsys, total, dtype))
        return TRID_ERR_ALLOC;
    if ((reinterpret_cast<uintptr_t>(workspace) % 256) != 0) return TRID_ERR_MISALIGNED;
    const size_t esz = dtype == TRID_F32 ? 4 : 8;
    const size_t wsb = (varlen_ws_bytes(nsys) + 255) / 256 * 256;
    void *scratch = static_cast<char *>(workspace) + wsb;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        cudaGetLastError();
        return TRID_ERR_CUDA;
    }
    float best_t = -1.0f;
    trid_status rs = TRID_OK;
    const int nm = dtype == TRID_F32 ? 2 : 1;  // tile heights 8 (and 16 in FP32)
    for (int mi = 0; mi < nm && rs == TRID_OK; ++mi) {
    const int m = mi == 0 ? 8 : 16;
    const int32_t teams[3] = {vl_short_n(m), int32_t(vl_class_max(vl_b_m1(m) + 1, m)),
                              int32_t(vl_class_max(vl_b_m1(m) + 2, m))};
    const int32_t blocks[4] = {int32_t(vl_class_max(vl_b_m1(m) + 2, m)),
                               int32_t(vl_class_max(vl_b_m1(m) + 3, m)),
                               int32_t(vl_class_max(vl_b_m1(m) + 4, m)), 0};
    for (int ti = 0; ti < 3 && rs == TRID_OK; ++ti) {
        for (int bi = 0; bi < 4 && rs == TRID_OK; ++bi) {
        for (int tw = 4; tw >= 2 && rs == TRID_OK; tw -= 2) {  // warps per team
            if (bi < 3 && blocks[bi] == teams[ti]) continue;  // same as bi == 3
            trid_varlen_config cfg{teams[ti], bi == 3 ? teams[ti] : blocks[bi], m, tw};
            int mm, ea, eb, tt;
            if (!vl_edges(&cfg, dtype, mm, ea, eb, tt)) continue;
            float t_best = -1.0f;
            for (int rep = 0; rep < 4 && rs == TRID_OK; ++rep) {  // first run warms up
                if (cudaMemcpyAsync(scratch, d, size_t(total) * esz, cudaMemcpyDeviceToDevice,
                                    st) != cudaSuccess) { rs = TRID_ERR_CUDA; break; }
                cudaEventRecord(e0, st);
                rs = varlen_entry(a, b, c, scratch, nullptr, offsets, nsys, total, max_len, dtype,
                                  workspace, wsb, stream, &cfg);
                cudaEventRecord(e1, st);
                if (rs != TRID_OK) break;
                if (cudaEventSynchronize(e1) != cudaSuccess) { rs = TRID_ERR_CUDA; break; }
                float ms = 0.0f;
                cudaEventElapsedTime(&ms, e0, e1);
                if (rep > 0 && (t_best < 0.0f || ms < t_best)) t_best = ms;
            }
            if (rs == TRID_OK && t_best >= 0.0f && (best_t < 0.0f || t_best < best_t)) {
                best_t = t_best;
                *best = cfg;
            }
        }
        }
    }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rs != TRID_OK) { launch_ok(); return rs; }
    if (best_ms) *best_ms = best_t;
    return launch_ok() ? TRID_OK : TRID_ERR_CUDA;
}
