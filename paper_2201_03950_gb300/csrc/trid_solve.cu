// trid_solve.cu -- batched tridiagonal solve along one mesh axis
// (arXiv 2201.03950, Section 2 / 2.1 / 3.1) and its C-ABI entry points.
//
// Kernel families (all FP32 and FP64, tile of M = 8 rows per thread):
//
//  k_lines    systems contiguous in memory (x axis, stride 1).  G = 1..32
//             lanes of a warp share one system, lane g owning rows
//             [g*M, g*M + M) loaded with 16-byte vector loads; the reduced
//             system lives in registers and is solved with warp shuffles.
//             No shared memory, no block-wide barrier: every warp runs
//             independently.  Serves N <= 32*M.
//  k_strided  systems strided in memory (y/z axes, and the reduced systems
//             of the long path).  A block holds SG systems that are
//             neighbours in memory (lane = system, so each row of the tile is
//             one coalesced 128/256-byte segment) times NT tiles (thread
//             group = tile); the reduced rows go through shared memory to a
//             warp-shuffle solve with G = NT lanes per system.  N <= 32*M.
//  k_long_*   longer systems: tiled Thomas-PCR in passes.  k_long_reduce
//             writes the two reduced rows of each tile to scratch, the reduced
//             systems (2 rows per tile) are solved by a recursive call, and
//             k_long_subst recomputes each tile and substitutes the tile-end
//             unknowns back.
//  k_lines_tma  contiguous FP32 systems of 256 < N <= 4096 in one pass:
//             whole systems staged in shared memory by bulk copies, one team
//             of warps per system (trid_lines_tma.cuh).
//  k_chunk_cluster  strided FP32 systems of 256 < N <= 4096 in one pass:
//             chunks of 256 or 512 rows, one CTA each, joined by a chunk-level
//             solve across a thread-block cluster (trid_chunked.cuh).
#include "trid_device.cuh"
#include "trid_strided.cuh"
#include "trid_lines_tma.cuh"
#include "trid_chunked.cuh"
#include "../../include/trid.h"
#include "trid_internal.h"

#include <cstdio>
#include <type_traits>

namespace trid {

constexpr int TILE_M = 8;
constexpr int MAX_SINGLE_PASS = 32 * TILE_M;  // longest system served in one pass


// ---------------------------------------------------------------------------
// Contiguous systems: one group of G lanes per system.
// ---------------------------------------------------------------------------
template <typename T, int M, int G>
__global__ void __launch_bounds__(256)
k_lines(const T *__restrict__ a, const T *__restrict__ b, const T *__restrict__ c, const T *d,
        T *out, int accumulate, int64_t nsys, int64_t n, int vec_ok) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int g = lane % G;
    const int64_t sys = warp * (32 / G) + lane / G;
    const bool active = sys < nsys;
    const int64_t i0 = int64_t(g) * M;
    const int64_t base = sys * n;

    T ra[M], rb[M], rc[M], rd[M];
    if (active && vec_ok && i0 + M <= n && TRID_BOUNDS(base + i0 + M <= nsys * n)) {
        load_contig_vec<T, M>(a + base + i0, ra);
        if (b) load_contig_vec<T, M>(b + base + i0, rb);
        else {
#pragma unroll
            for (int j = 0; j < M; ++j) rb[j] = T(1);
        }
        load_contig_vec<T, M>(c + base + i0, rc);
        load_contig_vec<T, M>(d + base + i0, rd);
    } else {
#pragma unroll
        for (int j = 0; j < M; ++j) {
            const int64_t i = i0 + j;
            if (active && i < n && TRID_BOUNDS(base + i < nsys * n)) {
                ra[j] = a[base + i];
                rb[j] = b ? b[base + i] : T(1);
                rc[j] = c[base + i];
                rd[j] = d[base + i];
            } else {
                ra[j] = T(0); rb[j] = T(1); rc[j] = T(0); rd[j] = T(0);
            }
        }
    }
#pragma unroll
    for (int j = 0; j < M; ++j) {
        if (i0 + j == 0) ra[j] = T(0);
        if (i0 + j == n - 1) rc[j] = T(0);
    }
    T as, cs, ds, ae, ce, de, xs, xe;
    tile_reduce<T, M>(ra, rb, rc, rd, as, cs, ds, ae, ce, de);
    group_solve<T, G>(as, cs, ds, ae, ce, de, g, xs, xe);
    tile_substitute<T, M>(ra, rc, rd, xs, xe);
    if (!active) return;
    if (vec_ok && i0 + M <= n && TRID_BOUNDS(base + i0 + M <= nsys * n)) {
        if (accumulate) {
            T ru[M];
            load_contig_vec<T, M>(out + base + i0, ru);
#pragma unroll
            for (int j = 0; j < M; ++j) rd[j] += ru[j];
        }
        store_contig_vec<T, M>(out + base + i0, rd);
    } else {
#pragma unroll
        for (int j = 0; j < M; ++j) {
            const int64_t i = i0 + j;
            if (i < n && TRID_BOUNDS(base + i < nsys * n)) {
                if (accumulate) out[base + i] += rd[j];
                else out[base + i] = rd[j];
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Long systems, pass 1: reduced rows of every tile.  Thread = (system, tile);
// STRIDED: systems are memory neighbours (lane = system) and the reduced
// system is stored row-major over systems (row r of system s at r*nsys + s);
// otherwise lane = tile and the reduced system is contiguous per system.
// ---------------------------------------------------------------------------
template <typename T, int M>
__device__ __forceinline__ void long_load(const T *__restrict__ a, const T *__restrict__ b,
                                          const T *__restrict__ c, const T *d, const Lines &L,
                                          int64_t base, int64_t i0, bool vec_ok, T (&ra)[M],
                                          T (&rb)[M], T (&rc)[M], T (&rd)[M]) {
    if (vec_ok && L.stride == 1 && i0 + M <= L.n) {
        load_contig_vec<T, M>(a + base + i0, ra);
        if (b) load_contig_vec<T, M>(b + base + i0, rb);
        else {
#pragma unroll
            for (int j = 0; j < M; ++j) rb[j] = T(1);
        }
        load_contig_vec<T, M>(c + base + i0, rc);
        load_contig_vec<T, M>(d + base + i0, rd);
    } else {
#pragma unroll
        for (int j = 0; j < M; ++j) {
            const int64_t i = i0 + j;
            if (i < L.n) {
                const int64_t p = base + i * L.stride;
                ra[j] = a[p];
                rb[j] = b ? b[p] : T(1);
                rc[j] = c[p];
                rd[j] = d[p];
            } else {
                ra[j] = T(0); rb[j] = T(1); rc[j] = T(0); rd[j] = T(0);
            }
        }
    }
#pragma unroll
    for (int j = 0; j < M; ++j) {
        if (i0 + j == 0) ra[j] = T(0);
        if (i0 + j == L.n - 1) rc[j] = T(0);
    }
}

// Thread -> (system, tile).  With every index below 2^31 (checked on the
// host: nsys * ntiles and the line geometry) the divisions run in 32 bits.
template <bool STRIDED>
__device__ __forceinline__ void long_index(const Lines &L, int64_t ntiles, int64_t &sys,
                                           int64_t &tile) {
    if (STRIDED) {
        sys = int64_t(blockIdx.x) * 32 + (threadIdx.x & 31);
        tile = int64_t(blockIdx.y) * (blockDim.x >> 5) + (threadIdx.x >> 5);
    } else {
        const int g32 = int(blockIdx.x * blockDim.x + threadIdx.x);
        const int nt = int(ntiles);
        const int q = g32 / nt;
        sys = q;
        tile = g32 - q * nt;
    }
}

// First element of line `sys` (32-bit division, as above).
__device__ __forceinline__ int64_t line_base32(const Lines &L, int64_t sys) {
    if (L.inner == 1) return sys * L.n;
    const int s32 = int(sys), in32 = int(L.inner);
    const int q = s32 / in32;
    return int64_t(s32 - q * in32) + int64_t(q) * L.inner * L.n;
}

template <typename T, int M, bool STRIDED>
__global__ void __launch_bounds__(256)
k_long_reduce(const T *__restrict__ a, const T *__restrict__ b, const T *__restrict__ c,
              const T *__restrict__ d, Lines L, int64_t ntiles, int vec_ok,
              T *__restrict__ ra_out, T *__restrict__ rc_out, T *__restrict__ rd_out) {
    int64_t sys, tile;
    long_index<STRIDED>(L, ntiles, sys, tile);
    if (sys >= L.nsys || tile >= ntiles) return;
    const int64_t base = line_base32(L, sys);
    const int64_t i0 = tile * M;
    T ra[M], rb[M], rc[M], rd[M];
    long_load<T, M>(a, b, c, d, L, base, i0, vec_ok, ra, rb, rc, rd);
    T as, cs, ds, ae, ce, de;
    tile_reduce<T, M>(ra, rb, rc, rd, as, cs, ds, ae, ce, de);
    const int64_t R = 2 * ntiles;
    int64_t ps, pe;
    if (STRIDED) { ps = (2 * tile) * L.nsys + sys; pe = ps + L.nsys; }
    else { ps = sys * R + 2 * tile; pe = ps + 1; }
    ra_out[ps] = as; rc_out[ps] = cs; rd_out[ps] = ds;
    ra_out[pe] = ae; rc_out[pe] = ce; rd_out[pe] = de;
}

template <typename T, int M, bool STRIDED>
__global__ void __launch_bounds__(256)
k_long_subst(const T *__restrict__ a, const T *__restrict__ b, const T *__restrict__ c,
             const T *d, T *out, int accumulate, Lines L, int64_t ntiles, int vec_ok,
             const T *__restrict__ rx) {
    int64_t sys, tile;
    long_index<STRIDED>(L, ntiles, sys, tile);
    if (sys >= L.nsys || tile >= ntiles) return;
    const int64_t base = line_base32(L, sys);
    const int64_t i0 = tile * M;
    T ra[M], rb[M], rc[M], rd[M];
    long_load<T, M>(a, b, c, d, L, base, i0, vec_ok, ra, rb, rc, rd);
    T as, cs, ds, ae, ce, de;
    tile_reduce<T, M>(ra, rb, rc, rd, as, cs, ds, ae, ce, de);
    const int64_t R = 2 * ntiles;
    int64_t ps, pe;
    if (STRIDED) { ps = (2 * tile) * L.nsys + sys; pe = ps + L.nsys; }
    else { ps = sys * R + 2 * tile; pe = ps + 1; }
    tile_substitute<T, M>(ra, rc, rd, rx[ps], rx[pe]);
    if (vec_ok && L.stride == 1 && i0 + M <= L.n) {
        if (accumulate) {
            T ru[M];
            load_contig_vec<T, M>(out + base + i0, ru);
#pragma unroll
            for (int j = 0; j < M; ++j) rd[j] += ru[j];
        }
        store_contig_vec<T, M>(out + base + i0, rd);
    } else {
#pragma unroll
        for (int j = 0; j < M; ++j) {
            const int64_t i = i0 + j;
            if (i < L.n) {
                const int64_t p = base + i * L.stride;
                if (accumulate) out[p] += rd[j];
                else out[p] = rd[j];
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Host dispatch
// ---------------------------------------------------------------------------
static int pow2_at_least(int64_t v) {
    int p = 1;
    while (p < v) p <<= 1;
    return p;
}

static inline size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Scratch bytes of the long-system path for systems of length n.
template <typename T>
static size_t long_ws_bytes(int64_t nsys, int64_t n) {
    if (n <= MAX_SINGLE_PASS) return 0;
    const int64_t ntiles = (n + TILE_M - 1) / TILE_M;
    const int64_t R = 2 * ntiles;
    const size_t one = align_up(size_t(nsys) * size_t(R) * sizeof(T), 256);
    return 3 * one + long_ws_bytes<T>(nsys, R);
}

template <typename T, int G>
static void launch_lines(const T *a, const T *b, const T *c, const T *d, T *out, int acc,
                         const Lines &L, int vec_ok, cudaStream_t st) {
    const int64_t warps = (L.nsys + (32 / G) - 1) / (32 / G);
    const int64_t blocks = (warps + 7) / 8;
    k_lines<T, TILE_M, G><<<dim3(unsigned(blocks)), 256, 0, st>>>(a, b, c, d, out, acc, L.nsys,
                                                                   L.n, vec_ok);
}

template <typename T, int NT>
static void launch_strided(const T *a, const T *b, const T *c, const T *d, T *out, int acc,
                           const Lines &L, cudaStream_t st) {
    // at least one full warp per block: the reduced solve shuffles over all 32 lanes
    constexpr int SG = (NT * SysCfg<T>::SG < 32) ? 32 / NT : SysCfg<T>::SG;
    ArrayCoef<T> coef{a, b, c};
    if constexpr (std::is_same<T, float>::value) {
      if (b != nullptr) {
        // Blackwell path: TMA-staged tiles (16 systems x n rows per box)
        const void *arrs[5] = {a, b, c, d, out};
        const bool ok = acc ? launch_strided_tma<T, TILE_M, NT, 16, true>(arrs, coef, out, L, st)
                            : launch_strided_tma<T, TILE_M, NT, 16, false>(arrs, coef, out, L, st);
        if (ok) return;
      }
    }
    if (acc)
        k_strided<T, TILE_M, NT, SG, true, ArrayCoef<T>>
            <<<strided_grid(L, SG), NT * SG, 0, st>>>(coef, d, out, L, L.nsys / L.inner);
    else
        k_strided<T, TILE_M, NT, SG, false, ArrayCoef<T>>
            <<<strided_grid(L, SG), NT * SG, 0, st>>>(coef, d, out, L, L.nsys / L.inner);
}

// Contiguous FP32 systems of 256 < n <= 4096 through k_lines_tma with teams
// of TW warps, M rows per thread (n <= 32 * TW * M).  False, having launched nothing, when the
// shared memory does not fit.
template <int TW, int M, int SPS, bool SWZ = false>
static bool launch_lines_tma_tw(const float *a, const float *b, const float *c, const float *d,
                                float *out, int acc, const Lines &L, cudaStream_t st) {
    using LY = LinesTmaLayout<float, TW, SPS>;
    const DeviceInfo *di = device_info();
    if (!di) return false;
    const int n = int(L.n);
    const int narr = b ? 4 : 3;
    // With NG > 1 team groups taking batches in turn, every stage must always
    // serve the same group (stages a multiple of NG, batch k in stage k %
    // stages, group k % NG): a group that could wait on a stage another group
    // uses might wait two phases ahead of the stage's barrier, which the
    // parity wait reports as complete, and read another batch's data.
    constexpr int NG = LY::NTEAM / SPS;
    int stages = 6;
    while (stages > NG && LY::bytes(n, narr, stages) > size_t(di->max_smem_optin)) --stages;
    stages -= stages % NG;
    if (stages < NG) return false;
    const size_t smem = LY::bytes(n, narr, stages);
    if (smem > size_t(di->max_smem_optin)) return false;
    TmaSet maps{};  // used by the swizzled variant only
    if constexpr (SWZ) {
        // one 2D box of n / M rows of M elements per array and system, swizzled
        // by the row size; several systems per stage need 1024-byte regions
        if (n % M != 0 || (SPS > 1 && n % 256 != 0) ||
            L.nsys * (L.n / M) >= (int64_t(1) << 31))
            return false;
        const float *arr[4] = {a, c, d, b};
        for (int q = 0; q < narr; ++q)
            if (!encode_rows_map(&maps.map[q], arr[q], 4, M, L.nsys * (L.n / M), n / M, M * 4))
                return false;
    }
    auto kern = k_lines_tma<float, TW, M, SPS, SWZ>;
    const int per_sm = kernel_blocks_per_sm(reinterpret_cast<const void *>(kern), LT_CONS + 32, smem);
    if (per_sm < 1) return false;
    const int64_t nbatch = (L.nsys + SPS - 1) / SPS;
    const int64_t slots = int64_t(di->sm_count) * per_sm;
    const int64_t grid = nbatch < slots ? nbatch : slots;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.gridDim = dim3(unsigned(grid));
    cfg.blockDim = dim3(LT_CONS + 32);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cfg.attrs = attr;
    cfg.numAttrs = pdl_launch_allowed(st) ? 1 : 0;
    const cudaError_t e = cudaLaunchKernelEx(&cfg, kern, maps, a, b, c, d, out, acc, int(L.nsys),
                                             n, int(nbatch), stages, device_status_word());
    if (e != cudaSuccess) {
        note_cuda_error(e);
        cudaGetLastError();
        return false;
    }
    return true;
}

template <typename T>
static bool launch_lines_tma(const T *a, const T *b, const T *c, const T *d, T *out, int acc,
                             const Lines &L, cudaStream_t st) {
    if constexpr (!std::is_same<T, float>::value) {
        return false;
    } else {
        const bool aligned = is_aligned16(a) && is_aligned16(c) && is_aligned16(d) &&
                             is_aligned16(out) && (!b || is_aligned16(b));
        if (L.stride != 1 || !aligned || L.n % 4 != 0 || L.n <= MAX_SINGLE_PASS ||
            L.n > LT_MAX_N || L.nsys >= (int64_t(1) << 31) || L.nsys * L.n >= (int64_t(1) << 40))
            return false;
        // 8 rows per thread: one contiguous bulk copy per array and stage
        // (per-system swizzled 32-byte-row boxes measured slower at 1024 and
        // 2048 rows)
        if (L.n <= 512) return launch_lines_tma_tw<2, 8, 8>(a, b, c, d, out, acc, L, st);
        if (L.n <= 1024) return launch_lines_tma_tw<4, 8, 4>(a, b, c, d, out, acc, L, st);
        if (L.n <= 2048) return launch_lines_tma_tw<8, 8, 2>(a, b, c, d, out, acc, L, st);
        // two teams of 8 warps, 16 rows per thread, taking one-system stages
        // in turn: two systems in flight; swizzled 64-byte-row boxes when
        // n % 16 == 0
        return launch_lines_tma_tw<8, 16, 1, true>(a, b, c, d, out, acc, L, st) ||
               launch_lines_tma_tw<8, 16, 1>(a, b, c, d, out, acc, L, st);
    }
}

// Strided FP32 systems of 256 < n <= 4096 rows through k_chunk_cluster: one
// cluster of C = ceil(n / (32 CM)) CTAs per strip of 16 systems, as many
// clusters as can be resident.  CM = 8 rows per thread (256-row chunks, two
// CTAs per SM) up to 2048 rows, CM = 16 (512-row chunks, one CTA per SM:
// half the per-chunk barriers and exchanges per byte) above.  False, having
// launched nothing, when a constraint (TMA alignment, 32-bit indexing,
// cluster scheduling) does not hold.
template <typename T, int CM>
static bool launch_chunk_cluster_cm(const T *a, const T *b, const T *c, const T *d, T *out,
                                    int acc, const Lines &L, cudaStream_t st) {
    using LY = ChunkLayout<T, CM>;
    const int C = int((L.n + LY::ROWS - 1) / LY::ROWS);
    if (C > CK_MAX_CHUNKS) return false;
    const int64_t outer = L.nsys / L.inner;
    const int64_t nxc = (L.inner + CK_SG - 1) / CK_SG;
    const int64_t nstrips = nxc * outer;
    if (nstrips >= (int64_t(1) << 31) || L.inner >= (int64_t(1) << 31)) return false;
    TmaSet maps{};
    const void *arrs[4] = {a, b, c, d};
    for (int q = 0; q < 4; ++q)
        if (!encode_lines_map(&maps.map[q], arrs[q], int(sizeof(T)), L.inner, L.n, outer, CK_SG,
                              CK_BOX))
            return false;
    // x through TMA stores unless accumulating (or out is not TMA-addressable)
    const int tma_store =
        !acc && encode_lines_map(&maps.map[4], out, int(sizeof(T)), L.inner, L.n, outer, CK_SG,
                                 CK_BOX);
    const size_t smem = LY::bytes(C);
    auto kern = k_chunk_cluster<T, CM>;
    const void *kp = reinterpret_cast<const void *>(kern);
    if (kernel_blocks_per_sm(kp, CK_THREADS, smem) < 1) return false;
    const int ncl_max = cluster_capacity(kp, C, CK_THREADS, smem);
    if (ncl_max < 1) return false;
    const int64_t ncl = nstrips < ncl_max ? nstrips : ncl_max;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = unsigned(C);
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[1].val.programmaticStreamSerializationAllowed = 1;
    cfg.gridDim = dim3(unsigned(C * ncl));
    cfg.blockDim = dim3(CK_THREADS);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cfg.attrs = attr;
    cfg.numAttrs = pdl_launch_allowed(st) ? 2 : 1;
    const cudaError_t e = cudaLaunchKernelEx(&cfg, kern, maps, out, acc, L, int(nstrips),
                                             tma_store, device_status_word());
    if (e != cudaSuccess) {
        note_cuda_error(e);
        cudaGetLastError();
        return false;
    }
    return true;
}

template <typename T>
static bool launch_chunk_cluster(const T *a, const T *b, const T *c, const T *d, T *out, int acc,
                                 const Lines &L, cudaStream_t st) {
    if constexpr (!std::is_same<T, float>::value) {
        return false;
    } else {
        if (L.stride == 1 || !b || L.n <= MAX_SINGLE_PASS || L.n > 4096 ||
            !strided_offsets_fit(L))
            return false;
        if (L.n <= 2048) return launch_chunk_cluster_cm<T, 8>(a, b, c, d, out, acc, L, st);
        return launch_chunk_cluster_cm<T, 16>(a, b, c, d, out, acc, L, st);
    }
}

template <typename T>
static trid_status solve_lines(const T *a, const T *b, const T *c, const T *d, T *out, int acc,
                               const Lines &L, char *ws, size_t ws_bytes, cudaStream_t st) {
    if (L.nsys == 0 || L.n == 0) return TRID_OK;
    const bool contig = (L.stride == 1);
    if (L.n <= MAX_SINGLE_PASS) {
        const int G = pow2_at_least((L.n + TILE_M - 1) / TILE_M);
        if (contig) {
            const int vec_ok = is_aligned16(a) && is_aligned16(c) && is_aligned16(d) &&
                               is_aligned16(out) && (!b || is_aligned16(b)) &&
                               (L.n * int64_t(sizeof(T))) % 16 == 0;
            switch (G) {
                case 1: launch_lines<T, 1>(a, b, c, d, out, acc, L, vec_ok, st); break;
                case 2: launch_lines<T, 2>(a, b, c, d, out, acc, L, vec_ok, st); break;
                case 4: launch_lines<T, 4>(a, b, c, d, out, acc, L, vec_ok, st); break;
                case 8: launch_lines<T, 8>(a, b, c, d, out, acc, L, vec_ok, st); break;
                case 16: launch_lines<T, 16>(a, b, c, d, out, acc, L, vec_ok, st); break;
                default: launch_lines<T, 32>(a, b, c, d, out, acc, L, vec_ok, st); break;
            }
        } else {
            if (!strided_offsets_fit(L)) return TRID_ERR_UNSUPPORTED;
            switch (G) {
                case 1: launch_strided<T, 1>(a, b, c, d, out, acc, L, st); break;
                case 2: launch_strided<T, 2>(a, b, c, d, out, acc, L, st); break;
                case 4: launch_strided<T, 4>(a, b, c, d, out, acc, L, st); break;
                case 8: launch_strided<T, 8>(a, b, c, d, out, acc, L, st); break;
                case 16: launch_strided<T, 16>(a, b, c, d, out, acc, L, st); break;
                default: launch_strided<T, 32>(a, b, c, d, out, acc, L, st); break;
            }
        }
        return cudaGetLastError() == cudaSuccess ? TRID_OK : TRID_ERR_CUDA;
    }
    // up to 4096 contiguous FP32 rows: one pass, systems staged by bulk copies
    if (launch_lines_tma<T>(a, b, c, d, out, acc, L, st)) return TRID_OK;
    // strided FP32 up to 4096 rows: one cluster per strip of systems
    if (launch_chunk_cluster<T>(a, b, c, d, out, acc, L, st)) return TRID_OK;
    // long systems: tiled Thomas-PCR in passes
    const int64_t ntiles = (L.n + TILE_M - 1) / TILE_M;
    const int64_t R = 2 * ntiles;
    const size_t one = align_up(size_t(L.nsys) * size_t(R) * sizeof(T), 256);
    // limits of the multi-pass path first, so that a problem no path serves
    // reports TRID_ERR_UNSUPPORTED whether or not scratch was given
    if (!contig && (ntiles + 7) / 8 > 65535) return TRID_ERR_UNSUPPORTED;  // grid.y limit
    // the kernels' 32-bit thread and line indices
    if (L.nsys * ntiles >= (int64_t(1) << 31) || L.nsys >= (int64_t(1) << 31))
        return TRID_ERR_UNSUPPORTED;
    if (ws_bytes < long_ws_bytes<T>(L.nsys, L.n) || ws == nullptr) return TRID_ERR_ALLOC;
    T *ra = reinterpret_cast<T *>(ws);
    T *rc = reinterpret_cast<T *>(ws + one);
    T *rd = reinterpret_cast<T *>(ws + 2 * one);
    const int vec_ok = contig && is_aligned16(a) && is_aligned16(c) && is_aligned16(d) &&
                       is_aligned16(out) && (!b || is_aligned16(b)) &&
                       (L.n * int64_t(sizeof(T))) % 16 == 0;
    Lines LR;
    LR.nsys = L.nsys;
    LR.n = R;
    if (contig) {
        LR.inner = 1; LR.stride = 1;
        const int64_t total = L.nsys * ntiles;
        const int64_t blocks = (total + 255) / 256;
        k_long_reduce<T, TILE_M, false><<<dim3(unsigned(blocks)), 256, 0, st>>>(
            a, b, c, d, L, ntiles, vec_ok, ra, rc, rd);
    } else {
        LR.inner = L.nsys; LR.stride = L.nsys;
        dim3 grid(unsigned((L.nsys + 31) / 32), unsigned((ntiles + 7) / 8));
        k_long_reduce<T, TILE_M, true><<<grid, 256, 0, st>>>(a, b, c, d, L, ntiles, 0, ra, rc,
                                                             rd);
    }
    if (cudaGetLastError() != cudaSuccess) return TRID_ERR_CUDA;
    trid_status s = solve_lines<T>(ra, nullptr, rc, rd, rd, 0, LR, ws + 3 * one,
                                   ws_bytes - 3 * one, st);
    if (s != TRID_OK) return s;
    if (contig) {
        const int64_t total = L.nsys * ntiles;
        const int64_t blocks = (total + 255) / 256;
        k_long_subst<T, TILE_M, false><<<dim3(unsigned(blocks)), 256, 0, st>>>(
            a, b, c, d, out, acc, L, ntiles, vec_ok, rd);
    } else {
        dim3 grid(unsigned((L.nsys + 31) / 32), unsigned((ntiles + 7) / 8));
        k_long_subst<T, TILE_M, true><<<grid, 256, 0, st>>>(a, b, c, d, out, acc, L, ntiles, 0,
                                                            rd);
    }
    return cudaGetLastError() == cudaSuccess ? TRID_OK : TRID_ERR_CUDA;
}

// ---------------------------------------------------------------------------
// Argument checks and entry points
// ---------------------------------------------------------------------------
static trid_status mesh_lines(const int64_t *dims, int ndim, int solve_dim, Lines &L,
                              int64_t &total) {
    if (!dims || ndim < 1 || ndim > 3 || solve_dim < 0 || solve_dim >= ndim)
        return TRID_ERR_INVALID_ARG;
    int64_t n3[3] = {1, 1, 1};
    total = 1;
    for (int k = 0; k < ndim; ++k) {
        if (dims[k] < 0) return TRID_ERR_INVALID_ARG;
        n3[k] = dims[k];
    }
    // guard against overflow of the element count
    for (int k = 0; k < 3; ++k) {
        if (n3[k] != 0 && total > (int64_t(1) << 62) / n3[k]) return TRID_ERR_INVALID_ARG;
        total *= n3[k];
    }
    int64_t inner = 1;
    for (int k = 0; k < solve_dim; ++k) inner *= n3[k];
    L.n = n3[solve_dim];
    L.inner = inner;
    L.stride = inner;
    L.nsys = (L.n == 0) ? 0 : total / L.n;
    if (L.n > (int64_t(1) << 31)) return TRID_ERR_UNSUPPORTED;
    return TRID_OK;
}

static bool overlaps(const void *p, const void *q, size_t bytes) {
    const char *a = static_cast<const char *>(p), *b = static_cast<const char *>(q);
    return a < b + bytes && b < a + bytes;
}

static trid_status check_solve_args(const void *a, const void *b, const void *c, void *d,
                                    void *u, const int64_t *dims, int ndim, int solve_dim,
                                    trid_dtype dtype, Lines &L, size_t &esz) {
    if (dtype != TRID_F32 && dtype != TRID_F64) return TRID_ERR_INVALID_ARG;
    esz = dtype == TRID_F32 ? 4 : 8;
    int64_t total = 0;
    trid_status s = mesh_lines(dims, ndim, solve_dim, L, total);
    if (s != TRID_OK) return s;
    if (total == 0) return TRID_OK;
    if (!a || !b || !c || !d) return TRID_ERR_INVALID_ARG;
    const void *ptrs[5] = {a, b, c, d, u};
    for (int k = 0; k < 5; ++k)
        if (ptrs[k] && (reinterpret_cast<uintptr_t>(ptrs[k]) % esz) != 0) return TRID_ERR_MISALIGNED;
    if (u) {
        const size_t bytes = size_t(total) * esz;
        for (int k = 0; k < 4; ++k)
            if (overlaps(u, ptrs[k], bytes)) return TRID_ERR_INVALID_ARG;
    }
    return TRID_OK;
}

// x into `out`: stored (acc = 0) or added (acc = 1); every path reads d only.
static trid_status solve_dispatch_out(const void *a, const void *b, const void *c, const void *d,
                                      void *out, int acc, const Lines &L, trid_dtype dtype,
                                      char *ws, size_t ws_bytes, cudaStream_t st) {
    if (dtype == TRID_F32)
        return solve_lines<float>(static_cast<const float *>(a), static_cast<const float *>(b),
                                  static_cast<const float *>(c), static_cast<const float *>(d),
                                  static_cast<float *>(out), acc, L, ws, ws_bytes, st);
    return solve_lines<double>(static_cast<const double *>(a), static_cast<const double *>(b),
                               static_cast<const double *>(c), static_cast<const double *>(d),
                               static_cast<double *>(out), acc, L, ws, ws_bytes, st);
}

static trid_status solve_dispatch(const void *a, const void *b, const void *c, void *d, void *u,
                                  const Lines &L, trid_dtype dtype, char *ws, size_t ws_bytes,
                                  cudaStream_t st) {
    return solve_dispatch_out(a, b, c, d, u ? u : d, u ? 1 : 0, L, dtype, ws, ws_bytes, st);
}

// Argument check, scratch size and dispatch for a caller that supplies its own
// scratch (used by the allocation-free entry point).  `need` receives the
// scratch bytes the multi-pass path would require.  With less scratch than
// that the problem is still solved when the one-pass long-system kernels take
// it (they need none); otherwise TRID_ERR_ALLOC is returned and nothing is
// launched.
trid_status solve_with_scratch(const void *a, const void *b, const void *c, void *d, void *u,
                               const int64_t *dims, int ndim, int solve_dim, trid_dtype dtype,
                               void *scratch, size_t scratch_bytes, size_t &need,
                               cudaStream_t st);

size_t solve_ws_bytes(const Lines &L, trid_dtype dtype) {
    return dtype == TRID_F32 ? long_ws_bytes<float>(L.nsys, L.n)
                             : long_ws_bytes<double>(L.nsys, L.n);
}

trid_status solve_with_scratch(const void *a, const void *b, const void *c, void *d, void *u,
                               const int64_t *dims, int ndim, int solve_dim, trid_dtype dtype,
                               void *scratch, size_t scratch_bytes, size_t &need,
                               cudaStream_t st) {
    Lines L;
    size_t esz;
    need = 0;
    trid_status s = check_solve_args(a, b, c, d, u, dims, ndim, solve_dim, dtype, L, esz);
    if (s != TRID_OK || L.nsys == 0 || L.n == 0) return s;
    need = solve_ws_bytes(L, dtype);
    if (need > scratch_bytes)  // OK if a one-pass kernel took it, else ALLOC with nothing launched
        return solve_dispatch(a, b, c, d, u, L, dtype, nullptr, 0, st);
    return solve_dispatch(a, b, c, d, u, L, dtype, static_cast<char *>(scratch), scratch_bytes, st);
}

trid_status solve_into_ws(const void *a, const void *b, const void *c, const void *d, void *out,
                          const int64_t *dims, int ndim, int solve_dim, trid_dtype dtype,
                          void *workspace, size_t workspace_bytes, cudaStream_t st) {
    Lines L;
    size_t esz;
    if (!out) return TRID_ERR_INVALID_ARG;
    trid_status s = check_solve_args(a, b, c, const_cast<void *>(d), out, dims, ndim, solve_dim,
                                     dtype, L, esz);
    if (s != TRID_OK || L.nsys == 0 || L.n == 0) return s;
    const size_t need = solve_ws_bytes(L, dtype);
    if (need > 0 && (workspace == nullptr || workspace_bytes < need)) return TRID_ERR_ALLOC;
    if (need > 0 && (reinterpret_cast<uintptr_t>(workspace) % 256) != 0) return TRID_ERR_MISALIGNED;
    return solve_dispatch_out(a, b, c, d, out, 0, L, dtype, static_cast<char *>(workspace),
                              workspace_bytes, st);
}

}  // namespace trid

using namespace trid;

extern "C" size_t trid_solve_workspace_bytes(const int64_t *dims, int ndim, int solve_dim,
                                             trid_dtype dtype) {
    Lines L;
    int64_t total;
    if (dtype != TRID_F32 && dtype != TRID_F64) return 0;
    if (mesh_lines(dims, ndim, solve_dim, L, total) != TRID_OK) return 0;
    return solve_ws_bytes(L, dtype);
}

extern "C" trid_status trid_solve_batch_ws(const void *a, const void *b, const void *c, void *d,
                                           void *u, const int64_t *dims, int ndim,
                                           int solve_dim, trid_dtype dtype, void *workspace,
                                           size_t workspace_bytes, trid_stream_t stream) {
    trid::NvtxScope nvtx_scope("trid_solve_batch_ws");
    Lines L;
    size_t esz;
    trid_status s = check_solve_args(a, b, c, d, u, dims, ndim, solve_dim, dtype, L, esz);
    if (s != TRID_OK || L.nsys == 0 || L.n == 0) return s;
    const size_t need = solve_ws_bytes(L, dtype);
    if (need > 0 && (workspace == nullptr || workspace_bytes < need)) return TRID_ERR_ALLOC;
    if (need > 0 && (reinterpret_cast<uintptr_t>(workspace) % 256) != 0) return TRID_ERR_MISALIGNED;
    return solve_dispatch(a, b, c, d, u, L, dtype, static_cast<char *>(workspace),
                          workspace_bytes, reinterpret_cast<cudaStream_t>(stream));
}

extern "C" trid_status trid_solve_batch(const void *a, const void *b, const void *c, void *d,
                                        void *u, const int64_t *dims, int ndim, int solve_dim,
                                        trid_dtype dtype, trid_stream_t stream) {
    trid::NvtxScope nvtx_scope("trid_solve_batch");
    Lines L;
    size_t esz;
    trid_status s = check_solve_args(a, b, c, d, u, dims, ndim, solve_dim, dtype, L, esz);
    if (s != TRID_OK || L.nsys == 0 || L.n == 0) return s;
    const size_t need = solve_ws_bytes(L, dtype);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    void *ws = nullptr;
    if (need > 0) {
        // the one-pass long-system kernels need no scratch: only when they
        // decline (nothing launched, TRID_ERR_ALLOC) is the pool grown
        s = solve_dispatch(a, b, c, d, u, L, dtype, nullptr, 0, st);
        if (s != TRID_ERR_ALLOC) return s;
        s = pool_reserve(need, &ws);
        if (s != TRID_OK) return s;
    }
    return solve_dispatch(a, b, c, d, u, L, dtype, static_cast<char *>(ws), need, st);
}
