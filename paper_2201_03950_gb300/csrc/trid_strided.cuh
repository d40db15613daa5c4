// trid_strided.cuh -- the strided-systems kernel (systems along y or z of a
// column-major mesh, Section 2.1), shared by the batched solve and the ADI
// step through a coefficient policy.
//
// A block holds SG systems that are memory neighbours (consecutive x) times
// NT tiles of M rows.  Thread (tile, lane) loads rows [tile*M, tile*M + M) of
// system `lane`: for every row, the SG lanes read SG consecutive elements, one
// coalesced segment, so no transpose is needed (the FPGA design buffers XY/XZ
// planes for the same reason, Section 3).  The two reduced rows per tile go through shared memory
// to a warp-shuffle solve (NT lanes per system), and the tile-end unknowns
// come back the same way.
#pragma once
#include "trid_device.cuh"
#include "trid_tma.cuh"
#include "trid_internal.h"

namespace trid {

// Systems per block of the strided kernel: 16 neighbours (a 64-byte FP32 /
// 128-byte FP64 segment per row), so that two 512-thread blocks share an SM
// and one block loads while the other computes.
template <typename T> struct SysCfg;
template <> struct SysCfg<float> { static constexpr int SG = 16; };
template <> struct SysCfg<double> { static constexpr int SG = 16; };

// Coefficients read from arrays; a of row 0 and c of row n-1 are not read.
// b == nullptr means unit diagonal (the reduced systems of the long path).
template <typename T>
struct ArrayCoef {
    const T *__restrict__ a;
    const T *__restrict__ b;
    const T *__restrict__ c;
    __device__ __forceinline__ ArrayCoef shifted(int64_t base) const {
        return ArrayCoef{a + base, b ? b + base : nullptr, c + base};
    }
    // off: element offset from the shifted base; i: row index in the system
    __device__ __forceinline__ void get(int off, int i, int n, T &ra, T &rb, T &rc) const {
        ra = (i == 0) ? T(0) : a[off];
        rb = b ? b[off] : T(1);
        rc = (i == n - 1) ? T(0) : c[off];
    }
    // TMA path: a, b, c staged in shared memory slots 0..2
    static constexpr int NCOEF = 3;
    __device__ __forceinline__ void get_smem(const T *sa, const T *sb, const T *sc, int k, int i,
                                             int n, T &ra, T &rb, T &rc) const {
        ra = (i == 0) ? T(0) : sa[k];
        rb = sb[k];
        rc = (i == n - 1) ? T(0) : sc[k];
    }
};

// The ADI operator of Section 4.1 generated in the kernel:
// tridiag(-lambda, 1 + 2 lambda, -lambda) on interior rows, identity at the two
// Dirichlet boundary nodes.
template <typename T>
struct AdiCoef {
    T lam;
    __device__ __forceinline__ AdiCoef shifted(int64_t) const { return *this; }
    __device__ __forceinline__ void get(int, int i, int n, T &ra, T &rb, T &rc) const {
        const bool bnd = (i == 0) || (i == n - 1);
        ra = bnd ? T(0) : -lam;
        rb = bnd ? T(1) : T(1) + T(2) * lam;
        rc = bnd ? T(0) : -lam;
    }
    static constexpr int NCOEF = 0;
    __device__ __forceinline__ void get_smem(const T *, const T *, const T *, int, int i, int n,
                                             T &ra, T &rb, T &rc) const {
        get(0, i, n, ra, rb, rc);
    }
};

// Grid: blockIdx.x walks groups of SG consecutive systems inside one block of
// `inner` neighbours; (blockIdx.z, blockIdx.y) walk the outer index.  Element
// i of system (x, o) sits at x + o*inner*n + i*stride; offsets inside one
// system are 32-bit (the host checks (n-1)*stride < 2^31).
template <typename T, int M, int NT, int SG, bool ACC, typename Coef>
__global__ void __launch_bounds__(NT * SG)
k_strided(Coef coef, const T *d, T *out, Lines L, int64_t outer) {
    constexpr int P = SG + 1;  // padded row pitch of the shared tables
    __shared__ T s_as[NT * P], s_cs[NT * P], s_ds[NT * P];
    __shared__ T s_ae[NT * P], s_ce[NT * P], s_de[NT * P];
    __shared__ T s_xs[NT * P], s_xe[NT * P];

    const int tid = threadIdx.x;
    const int sl = tid % SG;    // system within block
    const int tile = tid / SG;  // tile within system
    const int64_t x = int64_t(blockIdx.x) * SG + sl;
    const int n = int(L.n);
    const int stride = int(L.stride);
    const int i0 = tile * M;
    const bool full = (i0 + M <= n);
    const int w = tile * P + sl;

    const int64_t o = int64_t(blockIdx.z) * gridDim.y + blockIdx.y;
    if (o >= outer) return;  // whole block: no barrier is skipped by part of it
    {
        const bool active = x < L.inner;
        const int64_t base = active ? x + o * L.inner * L.n : 0;
        const Coef cf = coef.shifted(base);
        const T *db = d + base;
        T ra[M], rb[M], rc[M], rd[M];
        if (active && full &&
            TRID_BOUNDS(base + int64_t(i0 + M - 1) * stride < L.nsys * L.n)) {
#pragma unroll
            for (int j = 0; j < M; ++j) {
                const int off = (i0 + j) * stride;
                cf.get(off, i0 + j, n, ra[j], rb[j], rc[j]);
                rd[j] = db[off];
            }
        } else {
#pragma unroll
            for (int j = 0; j < M; ++j) {
                const int i = i0 + j;
                if (active && i < n && TRID_BOUNDS(base + int64_t(i) * stride < L.nsys * L.n)) {
                    const int off = i * stride;
                    cf.get(off, i, n, ra[j], rb[j], rc[j]);
                    rd[j] = db[off];
                } else {
                    ra[j] = T(0); rb[j] = T(1); rc[j] = T(0); rd[j] = T(0);
                }
            }
        }
        T as, cs, ds, ae, ce, de;
        tile_reduce<T, M>(ra, rb, rc, rd, as, cs, ds, ae, ce, de);
        // the accumulate target is loaded now, behind the reduced solve
        T *ob = out + base;
        T ru[M];
        if (ACC) {
#pragma unroll
            for (int j = 0; j < M; ++j)
                ru[j] = (active && i0 + j < n) ? ob[(i0 + j) * stride] : T(0);
        }
        s_as[w] = as; s_cs[w] = cs; s_ds[w] = ds;
        s_ae[w] = ae; s_ce[w] = ce; s_de[w] = de;
        __syncthreads();
        {
            // reduced layout: NT consecutive threads hold the NT tiles of a system
            const int rs = tid / NT, rt = tid % NT;
            const int q = rt * P + rs;
            T xs, xe;
            group_solve<T, NT>(s_as[q], s_cs[q], s_ds[q], s_ae[q], s_ce[q], s_de[q], rt, xs, xe);
            s_xs[q] = xs;
            s_xe[q] = xe;
        }
        __syncthreads();
        tile_substitute<T, M>(ra, rc, rd, s_xs[w], s_xe[w]);
        if (active) {
#pragma unroll
            for (int j = 0; j < M; ++j) {
                if ((full || i0 + j < n) &&
                    TRID_BOUNDS(base + int64_t(i0 + j) * stride < L.nsys * L.n))
                    ob[(i0 + j) * stride] = ACC ? rd[j] + ru[j] : rd[j];
            }
        }
    }
}


// ---------------------------------------------------------------------------
// TMA-fed variant (Blackwell): one producer warp streams boxes of
// [SG systems x n rows] of every input array through a ring of `stages`
// shared-memory buffers (3D tensor map over (inner, n, outer), box
// (SG, n, 1)); NT*SG consumer threads take their tile rows from shared memory
// and solve exactly as k_strided.  The loads of the next batches are in flight
// while the current batch is solved, and the consumers issue no global loads.
// Persistent: the grid walks the batches (x-chunk, outer index).
// Shared memory: stages x slots x [n][SG] staging, 8 reduced tables, mbarriers.
// ---------------------------------------------------------------------------
template <typename T, int NT, int SG>
struct TmaLayout {
    static constexpr int P = SG + 1;
    __host__ __device__ static size_t slot_bytes(int n) { return (size_t(n) * SG * sizeof(T) + 127) / 128 * 128; }
    __host__ __device__ static size_t table_bytes() { return (8 * NT * P * sizeof(T) + 127) / 128 * 128; }
    __host__ __device__ static size_t bytes(int n, int nslots, int stages) {
        return size_t(stages) * nslots * slot_bytes(n) + table_bytes() + 2 * 8 * size_t(stages);
    }
};

template <typename T, int M, int NT, int SG, bool ACC, typename Coef>
__global__ void __launch_bounds__(NT * SG + 32, 2)
k_strided_tma(const __grid_constant__ TmaSet maps, Coef coef, T *out, Lines L, int64_t nbatch,
              int stages, int *status) {
    using LY = TmaLayout<T, NT, SG>;
    constexpr int P = LY::P;
    constexpr int NCONS = NT * SG;
    static_assert(NCONS % 32 == 0, "consumers must be whole warps");
    constexpr int NSLOT = Coef::NCOEF + 1 + (ACC ? 1 : 0);
    extern __shared__ __align__(128) unsigned char smem[];
    const int n = int(L.n);
    const size_t slot_bytes = LY::slot_bytes(n);
    const size_t stage_bytes = NSLOT * slot_bytes;
    T *tab = reinterpret_cast<T *>(smem + stages * stage_bytes);
    T *s_as = tab, *s_cs = tab + NT * P, *s_ds = tab + 2 * NT * P;
    T *s_ae = tab + 3 * NT * P, *s_ce = tab + 4 * NT * P, *s_de = tab + 5 * NT * P;
    T *s_xs = tab + 6 * NT * P, *s_xe = tab + 7 * NT * P;
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + stages * stage_bytes + LY::table_bytes());
    uint64_t *empty = full + stages;

    __shared__ int abort_flag;  // set once a bounded wait gave up: later waits are skipped
    const int tid = threadIdx.x;
    if (tid == 0) {
        abort_flag = 0;
        for (int s = 0; s < stages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], NCONS / 32);
        }
        fence_mbar_init();
    }
    __syncthreads();
    const int64_t nxc = (L.inner + SG - 1) / SG;

    if (tid >= NCONS) {
        // producer warp: one elected lane issues the copies
        if (tid == NCONS) {
            const uint32_t tx = uint32_t(NSLOT) * uint32_t(n) * SG * sizeof(T);
            int k = 0;
            for (int64_t bt = blockIdx.x; bt < nbatch; bt += gridDim.x, ++k) {
                const int s = k % stages;
                if (k >= stages && !mbar_wait(&empty[s], uint32_t((k / stages) - 1) & 1u, status)) {
                    *(volatile int *)&abort_flag = 1;
                    break;
                }
                mbar_expect_tx(&full[s], tx);
                const int b32 = int(bt), n32 = int(nxc);  // nbatch < 2^31 (host)
                const int o = b32 / n32;
                const int x0 = (b32 - o * n32) * SG;
                unsigned char *dst = smem + s * stage_bytes;
#pragma unroll
                for (int q = 0; q < NSLOT; ++q)
                    tma_load_3d(dst + q * slot_bytes, &maps.map[q], x0, 0, o, &full[s]);
            }
        }
        return;
    }

    const int lane = tid & 31;
    const int sl = tid % SG;
    const int tile = tid / SG;
    const int i0 = tile * M;
    const bool full_tile = (i0 + M <= n);
    const int w = tile * P + sl;
    const int stride = int(L.stride);
    const int inner32 = int(L.inner);
    const size_t inner_n = size_t(L.inner) * size_t(L.n);
    int k = 0;
    for (int64_t bt = blockIdx.x; bt < nbatch; bt += gridDim.x, ++k) {
        const int s = k % stages;
        bool ok = false;
        if (!*(volatile int *)&abort_flag) {
            ok = mbar_wait(&full[s], uint32_t(k / stages) & 1u, status);
            if (!ok) *(volatile int *)&abort_flag = 1;
        }
        const unsigned char *stg = smem + s * stage_bytes;
        const T *sa = reinterpret_cast<const T *>(stg);
        const T *sb = reinterpret_cast<const T *>(stg + slot_bytes);
        const T *sc = reinterpret_cast<const T *>(stg + 2 * slot_bytes);
        const T *sd = reinterpret_cast<const T *>(stg + Coef::NCOEF * slot_bytes);
        const T *su = reinterpret_cast<const T *>(stg + (Coef::NCOEF + 1) * slot_bytes);
        const int b32 = int(bt), n32 = int(nxc);  // nbatch < 2^31 (host)
        const int o = b32 / n32;
        const int x = (b32 - o * n32) * SG + sl;
        const bool active = ok && x < inner32;
        T ra[M], rb[M], rc[M], rd[M], ru[M];
#pragma unroll
        for (int j = 0; j < M; ++j) {
            const int i = i0 + j;
            if (active && (full_tile || i < n)) {
                const int q = i * SG + sl;
                coef.get_smem(sa, sb, sc, q, i, n, ra[j], rb[j], rc[j]);
                rd[j] = sd[q];
                if (ACC) ru[j] = su[q];
            } else {
                ra[j] = T(0); rb[j] = T(1); rc[j] = T(0); rd[j] = T(0);
                if (ACC) ru[j] = T(0);
            }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[s]);  // this warp is done with the stage

        T as, cs, ds, ae, ce, de;
        tile_reduce<T, M>(ra, rb, rc, rd, as, cs, ds, ae, ce, de);
        s_as[w] = as; s_cs[w] = cs; s_ds[w] = ds;
        s_ae[w] = ae; s_ce[w] = ce; s_de[w] = de;
        named_barrier(1, NCONS);
        {
            const int rs = tid / NT, rt = tid % NT;
            const int q = rt * P + rs;
            T xs, xe;
            group_solve<T, NT>(s_as[q], s_cs[q], s_ds[q], s_ae[q], s_ce[q], s_de[q], rt, xs, xe);
            s_xs[q] = xs;
            s_xe[q] = xe;
        }
        named_barrier(1, NCONS);
        tile_substitute<T, M>(ra, rc, rd, s_xs[w], s_xe[w]);
        if (active) {
            const size_t base = size_t(o) * inner_n + x;
            T *ob = out + base;
#pragma unroll
            for (int j = 0; j < M; ++j)
                if ((full_tile || i0 + j < n) &&
                    TRID_BOUNDS(base + size_t(i0 + j) * stride < size_t(L.nsys) * size_t(L.n)))
                    ob[(i0 + j) * stride] = ACC ? rd[j] + ru[j] : rd[j];
        }
    }
}
}  // namespace trid

namespace trid {
// Launch grid of k_strided: x over groups of SG neighbouring systems, (z, y)
// over the outer index.
inline dim3 strided_grid(const Lines &L, int SG) {
    const int64_t gx = (L.inner + SG - 1) / SG;
    const int64_t outer = L.nsys / L.inner;
    const int64_t gy = outer < 65535 ? outer : 65535;
    const int64_t gz = (outer + gy - 1) / gy;
    return dim3(unsigned(gx), unsigned(gy), unsigned(gz));
}
// k_strided indexes inside a system with 32-bit offsets.
inline bool strided_offsets_fit(const Lines &L) {
    return (L.n - 1) * L.stride < (int64_t(1) << 31) && L.n < (int64_t(1) << 31);
}

// Host launcher of k_strided_tma.  `arrs` = the Coef::NCOEF coefficient
// arrays, then d, then (ACC) u.  Returns false, having launched nothing, when
// the TMA constraints do not hold (the caller then uses k_strided).
template <typename T, int M, int NT, int SG, bool ACC, typename Coef>
inline bool launch_strided_tma(const void *const *arrs, Coef coef, T *out, const Lines &L,
                               cudaStream_t st) {
    // the consumer group must be whole warps (named barrier, per-warp arrivals)
    if constexpr ((NT * SG) % 32 != 0 || NT * SG + 32 > 1024) {
        return false;
    } else {
    constexpr int NSLOT = Coef::NCOEF + 1 + (ACC ? 1 : 0);
    const DeviceInfo *di = device_info();
    if (!di || L.n > NT * M || L.inner < 1) return false;
    const int64_t outer = L.nsys / L.inner;
    TmaSet maps;
    for (int q = 0; q < NSLOT; ++q)
        if (!encode_lines_map(&maps.map[q], arrs[q], int(sizeof(T)), L.inner, L.n, outer, SG))
            return false;
    using LY = TmaLayout<T, NT, SG>;
    // Prefer two blocks per SM (two consumer groups hide each other's barrier
    // and recurrence latency), each with as many stages (<= 4) as then fit.
    const size_t per_block = size_t(di->smem_per_sm) / 2 - 1024;
    const size_t cap = per_block < size_t(di->max_smem_optin) ? per_block
                                                                : size_t(di->max_smem_optin);
    int stages = 4;
    while (stages > 1 && LY::bytes(int(L.n), NSLOT, stages) > cap) --stages;
    if (LY::bytes(int(L.n), NSLOT, stages) > cap) {
        // one block per SM: deepen the pipeline instead
        stages = 4;
        while (stages > 1 && LY::bytes(int(L.n), NSLOT, stages) > size_t(di->max_smem_optin))
            --stages;
    }
    const size_t smem = LY::bytes(int(L.n), NSLOT, stages);
    if (smem > size_t(di->max_smem_optin)) return false;
    auto kern = k_strided_tma<T, M, NT, SG, ACC, Coef>;
    const int per_sm = kernel_blocks_per_sm(reinterpret_cast<const void *>(kern), NT * SG + 32, smem);
    if (per_sm < 1) return false;
    const int64_t nbatch = (L.inner + SG - 1) / SG * outer;
    // the kernel indexes batches and lines with 32-bit integers
    if (nbatch >= (int64_t(1) << 31) || L.inner >= (int64_t(1) << 31)) return false;
    const int64_t slots = int64_t(di->sm_count) * per_sm;
    const int64_t grid = nbatch < slots ? nbatch : slots;
    kern<<<dim3(unsigned(grid)), NT * SG + 32, smem, st>>>(maps, coef, out, L, nbatch, stages,
                                                           device_status_word());
    return cudaGetLastError() == cudaSuccess;
    }
}

}  // namespace trid
