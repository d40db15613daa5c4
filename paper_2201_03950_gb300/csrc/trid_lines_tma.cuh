// trid_lines_tma.cuh -- contiguous systems of 256 < N <= 4096 rows (FP32) in
// one pass (arXiv 2201.03950, Section 3.1, tiled Thomas-PCR).
//
// A persistent block (one per SM) of 16 consumer warps and one producer warp.
// The producer streams batches of consecutive systems into a ring of
// shared-memory stages with 1D bulk copies (cp.async.bulk, one per array and
// batch: a batch is one contiguous range of every array), completion counted
// on mbarriers; it runs up to `stages` batches ahead, so HBM keeps streaming
// while the consumers solve.  The consumers form teams of TW warps, one system
// per team: every thread owns M = 8 (16 for N > 2048) consecutive rows
// (tile_reduce in registers), the team's 2 * ntiles reduced rows go to shared memory and are
// solved there by parallel cyclic reduction (Algorithm "pcr") with named
// barriers, stopping as soon as every coupling coefficient is below 1/16 ulp
// (the later rounds would change no value by more than that), and every
// thread substitutes its tile and stores it with 16-byte vector stores.
// Every byte of a, b, c, d is read from HBM once and x written once.
#pragma once
#include "trid_device.cuh"
#include "trid_tma.cuh"

namespace trid {

constexpr int LT_CONS = 512;      // consumer threads (16 warps)
constexpr int LT_MAX_N = 4096;    // longest system (8 warps x 32 lanes x 16 rows)

// 1D bulk copy global -> shared, completion counted on `bar` (both addresses
// and the size multiples of 16 bytes).
__device__ __forceinline__ void bulk_load_1d(void *dst, const void *src, uint32_t bytes,
                                             uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
            "r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// Named barrier over `nthreads` threads that also returns whether any of
// them passed v = true.
__device__ __forceinline__ bool named_barrier_or(int id, int nthreads, bool v) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 q, %1, 0;\n\t"
        "bar.red.or.pred p, %2, %3, q;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(r)
        : "r"(uint32_t(v)), "r"(id), "r"(nthreads)
        : "memory");
    return r != 0;
}

// Parallel cyclic reduction of R <= 2 * nth unit-diagonal rows (A, C, D in
// shared memory, already written and synchronised) by the nth threads of a
// team; the caller owns rows t and t + nth.  Returns with the solution in D,
// visible to the team.  Rounds stop once every |a|, |c| < 2^-(p+4).
template <typename T>
__device__ __forceinline__ void team_pcr(T *A, T *C, T *D, int R, int t, int nth, int bar) {
    constexpr float negligible = sizeof(T) == 4 ? 3.7252903e-09f : 6.9388939e-18f;
    float cpl = 0.0f;
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        const int i = t + q * nth;
        if (i < R) cpl = fmaxf(cpl, float(fmax(fabs(A[i]), fabs(C[i]))));
    }
    if (!named_barrier_or(bar, nth, cpl >= negligible)) return;
    for (int s = 1; s < R; s <<= 1) {
        T na[2], nc[2], nd[2];
        float cmax = 0.0f;
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int i = t + q * nth;
            na[q] = nc[q] = nd[q] = T(0);
            if (i < R) {
                const T ai = A[i], ci = C[i], di = D[i];
                T am = T(0), cm = T(0), dm = T(0), ap = T(0), cp = T(0), dp = T(0);
                if (i - s >= 0) { am = A[i - s]; cm = C[i - s]; dm = D[i - s]; }
                if (i + s < R) { ap = A[i + s]; cp = C[i + s]; dp = D[i + s]; }
                const T r = rcp(T(1) - ai * cm - ci * ap);
                na[q] = -r * (ai * am);
                nc[q] = -r * (ci * cp);
                nd[q] = r * (di - ai * dm - ci * dp);
                cmax = fmaxf(cmax, float(fmax(fabs(na[q]), fabs(nc[q]))));
            }
        }
        named_barrier(bar, nth);
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int i = t + q * nth;
            if (i < R) { A[i] = na[q]; C[i] = nc[q]; D[i] = nd[q]; }
        }
        if (!named_barrier_or(bar, nth, cmax >= negligible)) break;
    }
}

// Shared-memory layout of k_lines_tma: `stages` stages of narr slots (one per
// array), each slot SPS * n elements (SPS systems per stage); then two
// buffers of reduced rows (A, C, D per team); then the full/empty mbarriers.
template <typename T, int TW, int SPS>
struct LinesTmaLayout {
    static constexpr int TT = 32 * TW;               // threads per team
    static constexpr int NTEAM = LT_CONS / TT;       // teams per block
    static_assert(NTEAM % SPS == 0, "teams split evenly over the systems of a stage");
    // slots on 1024-byte boundaries (the swizzled boxes' pattern repeats every 512 bytes)
    __host__ __device__ static size_t slot_bytes(int n) {
        return (size_t(SPS) * n * sizeof(T) + 1023) / 1024 * 1024;
    }
    __host__ __device__ static size_t red_bytes() {
        return 2 * size_t(NTEAM) * 3 * 2 * TT * sizeof(T);
    }
    // + 1 KB so that the stages can start on a 1024-byte boundary (swizzled copies)
    __host__ __device__ static size_t bytes(int n, int narr, int stages) {
        return size_t(stages) * narr * slot_bytes(n) + red_bytes() + 2 * stages * sizeof(uint64_t) +
               1024;
    }
};

// nsys systems of n rows, system s at [s * n, s * n + n) of every array;
// b == nullptr means a unit diagonal.  M rows per thread; a stage holds SPS
// systems, and the NG = NTEAM / SPS groups of SPS teams take the batches in
// turn (batch k: stage k % stages, group k % NG).  The host keeps stages a
// multiple of NG, so every stage always serves the same group and no group
// ever waits on a stage's full barrier more than one phase ahead.
// Requirements (host): every pointer 16-byte aligned, n % 4 == 0 (FP32),
// n <= M * 32 * TW.
// SWZ (rows of M * sizeof(T) = 32 or 64 bytes, n % M == 0, every system's
// region 1024-byte aligned): each array of a system arrives as one 2D TMA
// box of n / M rows with the 32- or 64-byte shared-memory swizzle (maps: a,
// c, d, b), which puts the 16-byte chunk q of a row at chunk q ^ (address
// bits 7.. of the row) -- bit 7 for 32-byte rows, bits 7-8 for 64-byte rows;
// a warp reading chunk q of 32 consecutive rows then touches 32 different
// banks (the plain layout gives a 2- or 4-way conflict at that lane stride).
template <typename T, int TW, int M, int SPS, bool SWZ>
__global__ void __launch_bounds__(LT_CONS + 32, 1)
k_lines_tma(const __grid_constant__ TmaSet maps, const T *a, const T *b, const T *c, const T *d,
            T *out, int accumulate, int nsys, int n, int nbatch, int stages, int *status) {
    // launched with programmatic dependent launch: one wave of persistent
    // blocks, so the next kernel may be scheduled at once; nothing is read or
    // written before the previous kernel has completed
    pdl_trigger();
    pdl_wait();
    static_assert(!SWZ || M * sizeof(T) == 32 || M * sizeof(T) == 64,
                  "swizzled rows are 32 or 64 bytes");
    using LY = LinesTmaLayout<T, TW, SPS>;
    constexpr int TT = LY::TT;
    constexpr int NTEAM = LY::NTEAM;
    constexpr int NG = NTEAM / SPS;  // team groups, taking stages in turn
    extern __shared__ __align__(128) unsigned char smem_raw[];
    // stages on a 1024-byte boundary (the swizzle pattern follows address bits)
    unsigned char *smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    const int narr = b ? 4 : 3;
    const size_t slot = LY::slot_bytes(n);
    const size_t stage_bytes = size_t(narr) * slot;
    T *red = reinterpret_cast<T *>(smem + stages * stage_bytes);
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + stages * stage_bytes + LY::red_bytes());
    uint64_t *empty = full + stages;

    __shared__ int abort_flag;  // set once a bounded wait gave up: later waits are skipped
    const int tid = threadIdx.x;
    if (tid == 0) {
        abort_flag = 0;
        for (int s = 0; s < stages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], SPS * TW);  // the warps of one team group
        }
        fence_mbar_init();
    }
    __syncthreads();

    if (tid >= LT_CONS) {
        // producer warp: one lane issues the copies of each batch
        if (tid == LT_CONS) {
            const T *src[4] = {a, c, d, b};
            int k = 0;
            for (int bt = blockIdx.x; bt < nbatch; bt += gridDim.x, ++k) {
                const int s = k % stages;
                if (k >= stages &&
                    !mbar_wait(&empty[s], uint32_t((k / stages) - 1) & 1u, status)) {
                    *(volatile int *)&abort_flag = 1;
                    break;
                }
                const int sys0 = bt * SPS;
                const int cnt = nsys - sys0 < SPS ? nsys - sys0 : SPS;
                const uint32_t bytes = uint32_t(cnt) * uint32_t(n) * uint32_t(sizeof(T));
                mbar_expect_tx(&full[s], uint32_t(narr) * bytes);
                unsigned char *dst = smem + s * stage_bytes;
                if (SWZ) {
                    const int rows = n / M;
                    const size_t sb = size_t(n) * sizeof(T);
                    for (int q = 0; q < narr; ++q)
                        for (int j = 0; j < cnt; ++j)
                            tma_load_2d(dst + q * slot + j * sb, &maps.map[q], 0,
                                        (sys0 + j) * rows, &full[s]);
                } else {
                    const size_t off = size_t(sys0) * size_t(n);
                    for (int q = 0; q < narr; ++q)
                        bulk_load_1d(dst + q * slot, src[q] + off, bytes, &full[s]);
                }
            }
        }
        return;
    }

    const int lane = tid & 31;
    const int team = tid / TT, t = tid % TT;
    const int tg = team / SPS, ts = team % SPS;  // team group, system of the stage
    const int bar = 1 + team;  // named barrier of the team (0 is __syncthreads)
    const int i0 = t * M;
    const int ntiles = (n + M - 1) / M;
    const bool mine = t < ntiles;
    const bool full_tile = i0 + M <= n;
    int kk = 0;  // this team's own batch count
    for (int k = tg, bt = blockIdx.x + tg * gridDim.x; bt < nbatch;
         k += NG, bt += NG * gridDim.x, ++kk) {
        const int s = k % stages;
        bool ok = false;
        if (!*(volatile int *)&abort_flag) {
            ok = mbar_wait(&full[s], uint32_t(k / stages) & 1u, status);
            if (!ok) *(volatile int *)&abort_flag = 1;
        }
        const int sys = bt * SPS + ts;
        const bool active = ok && sys < nsys;  // uniform over the team
        const unsigned char *stg = smem + s * stage_bytes;
        const size_t row0 = size_t(ts) * n + i0;
        const T *sa = reinterpret_cast<const T *>(stg) + row0;
        const T *sc = reinterpret_cast<const T *>(stg + slot) + row0;
        const T *sd = reinterpret_cast<const T *>(stg + 2 * slot) + row0;
        const T *sb = reinterpret_cast<const T *>(stg + 3 * slot) + row0;
        T ra[M], rb[M], rc[M], rd[M];
        if (SWZ) {
            // row t of the box: chunk q at chunk q ^ x of the row (x from the
            // row's shared-memory address bits 7-8)
            using V = typename Vec16<T>::type;
            constexpr int W = Vec16<T>::n;
            const size_t r = row0 / W;  // 16-byte chunk of the row's start
            const V *va = reinterpret_cast<const V *>(stg) + r;
            const V *vc = reinterpret_cast<const V *>(stg + slot) + r;
            const V *vd = reinterpret_cast<const V *>(stg + 2 * slot) + r;
            const V *vb = reinterpret_cast<const V *>(stg + 3 * slot) + r;
            const int x = int((smem_u32(va) >> 7) & unsigned(M / W - 1));
#pragma unroll
            for (int q = 0; q < M / W; ++q) {
                const int pq = q ^ x;
                V w;
                if (active && mine) {
                    w = va[pq];
#pragma unroll
                    for (int j = 0; j < W; ++j) ra[q * W + j] = reinterpret_cast<const T *>(&w)[j];
                    w = vc[pq];
#pragma unroll
                    for (int j = 0; j < W; ++j) rc[q * W + j] = reinterpret_cast<const T *>(&w)[j];
                    w = vd[pq];
#pragma unroll
                    for (int j = 0; j < W; ++j) rd[q * W + j] = reinterpret_cast<const T *>(&w)[j];
                    if (b) {
                        w = vb[pq];
#pragma unroll
                        for (int j = 0; j < W; ++j)
                            rb[q * W + j] = reinterpret_cast<const T *>(&w)[j];
                    } else {
#pragma unroll
                        for (int j = 0; j < W; ++j) rb[q * W + j] = T(1);
                    }
                } else {
#pragma unroll
                    for (int j = 0; j < W; ++j) {
                        ra[q * W + j] = T(0); rb[q * W + j] = T(1);
                        rc[q * W + j] = T(0); rd[q * W + j] = T(0);
                    }
                }
            }
        } else if (active && mine && full_tile) {
            load_contig_vec<T, M>(sa, ra);
            load_contig_vec<T, M>(sc, rc);
            load_contig_vec<T, M>(sd, rd);
            if (b) load_contig_vec<T, M>(sb, rb);
            else {
#pragma unroll
                for (int j = 0; j < M; ++j) rb[j] = T(1);
            }
        } else {
#pragma unroll
            for (int j = 0; j < M; ++j) {
                if (active && mine && i0 + j < n) {
                    ra[j] = sa[j]; rc[j] = sc[j]; rd[j] = sd[j];
                    rb[j] = b ? sb[j] : T(1);
                } else {
                    ra[j] = T(0); rb[j] = T(1); rc[j] = T(0); rd[j] = T(0);
                }
            }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[s]);  // this warp is done with the stage
        if (!active) continue;
#pragma unroll
        for (int j = 0; j < M; ++j) {
            if (i0 + j == 0) ra[j] = T(0);
            if (i0 + j == n - 1) rc[j] = T(0);
        }
        T as, cs, ds, ae, ce, de;
        tile_reduce<T, M>(ra, rb, rc, rd, as, cs, ds, ae, ce, de);
        // reduced rows: buffer kk & 1 (the previous system's stays readable)
        T *RA = red + (size_t((kk & 1) * NTEAM + team) * 3) * (2 * TT);
        T *RC = RA + 2 * TT, *RD = RA + 4 * TT;
        if (mine) {
            RA[2 * t] = as; RC[2 * t] = cs; RD[2 * t] = ds;
            RA[2 * t + 1] = ae; RC[2 * t + 1] = ce; RD[2 * t + 1] = de;
        }
        named_barrier(bar, TT);
        team_pcr<T>(RA, RC, RD, 2 * ntiles, t, TT, bar);
        if (!mine) continue;
        tile_substitute<T, M>(ra, rc, rd, RD[2 * t], RD[2 * t + 1]);
        T *o = out + size_t(sys) * n + i0;
        if (full_tile) {
            if (accumulate) {
                T ru[M];
                load_contig_vec<T, M>(o, ru);
#pragma unroll
                for (int j = 0; j < M; ++j) rd[j] += ru[j];
            }
            store_contig_vec<T, M>(o, rd);
        } else {
#pragma unroll
            for (int j = 0; j < M; ++j)
                if (i0 + j < n) o[j] = accumulate ? o[j] + rd[j] : rd[j];
        }
    }
}

}  // namespace trid
