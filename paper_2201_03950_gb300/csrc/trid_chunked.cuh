// trid_chunked.cuh -- strided FP32 systems of 256 < N <= 4096 rows (y/z axes
// of large meshes) in one pass, one thread-block cluster per strip of 16
// neighbouring systems (arXiv 2201.03950, Section 3.1: the tiled hybrid
// applied once more, one level up).
//
// A system is cut into C <= 8 chunks of CH rows (CH = 256 for N <= 2048, with
// 8 rows per thread and two CTAs per SM; CH = 512 above, with 16 rows per
// thread and one CTA per SM, which halves the per-chunk barriers and
// exchanges per byte); CTA `rank` of a
// cluster of C CTAs owns chunk `rank` of the strip.  By linearity the
// solution restricted to a chunk is
//     x = p + q * x_L + r * x_R
// where x_L, x_R are the unknowns just outside the chunk, p solves the chunk
// with x_L = x_R = 0 and q, r are its responses to x_L = 1 and x_R = 1.
//
//  1. TMA loads the chunk's [16 systems x CH rows] of a, b, c, d (boxes of
//     256 rows); each of the 512 threads takes one tile (CH / 32 rows) of one
//     system into registers, and the next strip's boxes are requested at once.
//  2. tile_reduce, then one warp per system solves the chunk's reduced
//     system (PCR over 32 tiles, as group_solve) for p, q and r at once:
//     every tile end's p, q, r value stays in the solving lane's registers.
//  3. The values at the chunk's first row (F) and last row (E) are sent to
//     every CTA of the cluster (st.async into its shared memory, counted on
//     an mbarrier there, one per strip parity: no cluster barrier per strip);
//     once all C chunks' values have landed, every CTA solves the chunk-level
//     system
//         F_k = P0_k + Q0_k E_{k-1} + R0_k F_{k+1}
//         E_k = P1_k + Q1_k E_{k-1} + R1_k F_{k+1}
//     (2x2 block elimination, one thread per system) for its own x_L and x_R.
//  4. Tile ends x = p + q x_L + r x_R, then tile_substitute, and the chunk's
//     rows of x are stored.
// a, b, c, d are read from HBM once and x written once; the chunk never
// leaves the chip.
#pragma once
#include <cooperative_groups.h>

#include "trid_device.cuh"
#include "trid_tma.cuh"

namespace trid {

constexpr int CK_NT = 32;            // tiles per chunk (one warp per system)
constexpr int CK_SG = 16;            // neighbouring systems per strip
constexpr int CK_BOX = 256;          // rows per TMA box
constexpr int CK_THREADS = CK_NT * CK_SG;
constexpr int CK_MAX_CHUNKS = 8;     // cluster size (portable)

// Shared memory: the chunk's box of 4 arrays, the reduced tables (6 rows + 2
// solutions per tile, row pitch SG + 1), the received values of all chunks
// per strip parity (2 x C x 6 x SG), x_L and x_R, and the mbarriers (box
// landed; values of parity 0 and 1 landed).
// CM rows per thread: chunks of CK_NT * CM rows (256 or 512).
template <typename T, int CM>
struct ChunkLayout {
    static constexpr int P = CK_SG + 1;
    static constexpr int ROWS = CK_NT * CM;
    __host__ __device__ static size_t slot_bytes() { return size_t(ROWS) * CK_SG * sizeof(T); }
    __host__ __device__ static size_t tab_off() { return 4 * slot_bytes(); }
    __host__ __device__ static size_t gat_off() { return tab_off() + 8 * CK_NT * P * sizeof(T); }
    __host__ __device__ static size_t bar_off(int C) {
        return (gat_off() + 2 * size_t(C) * 6 * CK_SG * sizeof(T) + 2 * 2 * CK_SG * sizeof(T) +
                15) / 16 * 16;
    }
    // x staging for the TMA store of the chunk (same [row][SG] layout)
    __host__ __device__ static size_t xst_off(int C) { return (bar_off(C) + 32 + 127) / 128 * 128; }
    __host__ __device__ static size_t bytes(int C) { return xst_off(C) + slot_bytes(); }
};

// group_solve (full warp, G = 32 tiles) for three right-hand sides that
// share one reduced matrix: p with the tiles' own (ds, de); q, the response
// to x_L = 1 (-as on lane 0's S row); r, the response to x_R = 1 (-ce on the
// last lane's E row).  The fold and every PCR round compute the matrix
// factors once and carry the three right-hand sides.
template <typename T>
__device__ __forceinline__ void group_solve_spikes(T as, T cs, T ds, T ae, T ce, T de, int g,
                                                   T &ps, T &pe, T &qs, T &qe, T &us, T &ue) {
    constexpr unsigned FULL = 0xffffffffu;
    constexpr int G = 32;
    T nas = __shfl_down_sync(FULL, as, 1);
    T ncs = __shfl_down_sync(FULL, cs, 1);
    T nds = __shfl_down_sync(FULL, ds, 1);
    if (g + 1 >= G) { nas = T(0); ncs = T(0); nds = T(0); }
    T ra = -(ae * as);
    T rc = -(ce * ncs);
    T dp = de - ae * ds - ce * nds;
    T dq = g == 0 ? ae * as : T(0);       // -ae * (-as): lane 0's folded row
    T du = g == G - 1 ? -ce : T(0);
    {
        const T r = rcp(T(1) - ae * cs - ce * nas);
        ra *= r; rc *= r; dp *= r; dq *= r; du *= r;
    }
    constexpr float negligible = sizeof(T) == 4 ? 3.7252903e-09f : 6.9388939e-18f;
#pragma unroll
    for (int s = 1; s < G; s <<= 1) {
        const float cpl = float(fmax(fabs(ra), fabs(rc)));
        const unsigned top = __reduce_max_sync(FULL, __float_as_uint(cpl));
        if (__uint_as_float(top) < negligible) break;
        T am = __shfl_up_sync(FULL, ra, s), cm = __shfl_up_sync(FULL, rc, s);
        T ap = __shfl_down_sync(FULL, ra, s), cp = __shfl_down_sync(FULL, rc, s);
        T pm = __shfl_up_sync(FULL, dp, s), pp = __shfl_down_sync(FULL, dp, s);
        T qm = __shfl_up_sync(FULL, dq, s), qp = __shfl_down_sync(FULL, dq, s);
        T um = __shfl_up_sync(FULL, du, s), up = __shfl_down_sync(FULL, du, s);
        if (g < s) { am = T(0); cm = T(0); pm = T(0); qm = T(0); um = T(0); }
        if (g + s >= G) { ap = T(0); cp = T(0); pp = T(0); qp = T(0); up = T(0); }
        const T r = rcp(T(1) - ra * cm - rc * ap);
        const T na = -r * (ra * am), nc = -r * (rc * cp);
        dp = r * (dp - ra * pm - rc * pp);
        dq = r * (dq - ra * qm - rc * qp);
        du = r * (du - ra * um - rc * up);
        ra = na;
        rc = nc;
    }
    pe = dp; qe = dq; ue = du;
    T xp = __shfl_up_sync(FULL, pe, 1), xq = __shfl_up_sync(FULL, qe, 1);
    T xu = __shfl_up_sync(FULL, ue, 1);
    if (g == 0) { xp = T(0); xq = T(0); xu = T(0); }
    ps = ds - as * xp - cs * pe;
    qs = (g == 0 ? -as : T(0)) - as * xq - cs * qe;
    us = -as * xu - cs * ue;
}

// Strip s -> (outer o, x-group xg); the cluster walks strips with stride
// nclusters.  TMA map over (inner, n, outer), box (SG, 256, 1).
template <typename T, int CM>
__global__ void __launch_bounds__(CK_THREADS, CM == 8 ? 2 : 1)
k_chunk_cluster(const __grid_constant__ TmaSet maps, T *out, int accumulate, Lines L,
                int nstrips, int tma_store, int *status) {
    namespace cg = cooperative_groups;
    constexpr int NT = CK_NT, SG = CK_SG, M = CM, CH = CK_NT * CM;
    static_assert(CH % CK_BOX == 0, "a chunk is whole TMA boxes");
    // programmatic dependent launch (one wave of clusters): see k_lines_tma
    pdl_trigger();
    pdl_wait();
    using LY = ChunkLayout<T, CM>;
    constexpr int P = LY::P;
    extern __shared__ __align__(128) unsigned char smem[];
    cg::cluster_group cluster = cg::this_cluster();
    const int C = int(cluster.num_blocks());
    const int rank = int(cluster.block_rank());
    const int cid = int(blockIdx.x) / C;
    const int ncl = int(gridDim.x) / C;
    const T *sa = reinterpret_cast<const T *>(smem);
    const T *sb = reinterpret_cast<const T *>(smem + LY::slot_bytes());
    const T *sc = reinterpret_cast<const T *>(smem + 2 * LY::slot_bytes());
    const T *sd = reinterpret_cast<const T *>(smem + 3 * LY::slot_bytes());
    T *tab = reinterpret_cast<T *>(smem + LY::tab_off());
    T *s_as = tab, *s_cs = tab + NT * P, *s_ds = tab + 2 * NT * P;
    T *s_ae = tab + 3 * NT * P, *s_ce = tab + 4 * NT * P, *s_de = tab + 5 * NT * P;
    T *s_xs = tab + 6 * NT * P, *s_xe = tab + 7 * NT * P;
    T *gat = reinterpret_cast<T *>(smem + LY::gat_off());     // [2][C][6][SG]
    T *xlr = gat + 2 * size_t(C) * 6 * SG;                    // [2][SG]: x_L, x_R
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + LY::bar_off(C));
    uint64_t *gbar = full + 1;  // [2]: all chunks' values of a strip parity landed
    T *xst = reinterpret_cast<T *>(smem + LY::xst_off(C));

    __shared__ int abort_flag;
    const int tid = threadIdx.x;
    const int nxc = int((L.inner + SG - 1) / SG);  // < 2^31 (host)
    const int n = int(L.n);
    if (tid == 0) {
        abort_flag = 0;
        mbar_init(full, 1);
        mbar_init(&gbar[0], 1);
        mbar_init(&gbar[1], 1);
        fence_mbar_init();
    }
    __syncthreads();
    cluster.sync();  // every peer's mbarriers are initialised before values are sent to it

    const uint32_t tx = 4u * uint32_t(CH) * SG * sizeof(T);
    auto issue = [&](int strip) {
        const int o = strip / nxc, xg = strip - (strip / nxc) * nxc;
        mbar_expect_tx(full, tx);
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
            for (int h = 0; h < CH / CK_BOX; ++h)
                tma_load_3d(smem + q * LY::slot_bytes() + size_t(h) * CK_BOX * SG * sizeof(T),
                            &maps.map[q], xg * SG, rank * CH + h * CK_BOX, o, full);
    };
    if (tid == 0 && cid < nstrips) issue(cid);

    const int sl = tid % SG, tile = tid / SG;   // tile layout
    const int i0 = tile * M;
    const int w = tile * P + sl;
    const int rs = tid / NT, rt = tid % NT;     // solve layout: warp rs = system rs
    const int q = rt * P + rs;
    const int g0 = rank * CH;
    const int stride = int(L.stride);
    int j = 0;
    for (int strip = cid; strip < nstrips; strip += ncl, ++j) {
        T *gj = gat + size_t(j & 1) * C * 6 * SG;  // this strip's received values
        // this CTA's arrival on the parity's mbarrier, with the bytes that the C
        // chunks (itself included) will send
        if (tid == 0) mbar_expect_tx(&gbar[j & 1], uint32_t(C) * 6 * SG * uint32_t(sizeof(T)));
        bool ok = false;
        if (!*(volatile int *)&abort_flag) {
            ok = mbar_wait(full, uint32_t(j) & 1u, status);
            if (!ok) *(volatile int *)&abort_flag = 1;
        }
        const int o = strip / nxc, xg = strip - (strip / nxc) * nxc;
        const int x = xg * SG + sl;
        const bool active = ok && x < int(L.inner);
        T ra[M], rb[M], rc[M], rd[M];
#pragma unroll
        for (int k = 0; k < M; ++k) {
            const int gi = g0 + i0 + k;
            if (active && gi < n) {
                const int e = (i0 + k) * SG + sl;
                ra[k] = gi == 0 ? T(0) : sa[e];
                rb[k] = sb[e];
                rc[k] = gi == n - 1 ? T(0) : sc[e];
                rd[k] = sd[e];
            } else {
                ra[k] = T(0); rb[k] = T(1); rc[k] = T(0); rd[k] = T(0);
            }
        }
        __syncthreads();  // the box is free: fetch the next strip's behind this one
        if (tid == 0 && ok && strip + ncl < nstrips) issue(strip + ncl);

        T as, cs, ds, ae, ce, de;
        tile_reduce<T, M>(ra, rb, rc, rd, as, cs, ds, ae, ce, de);
        s_as[w] = as; s_cs[w] = cs; s_ds[w] = ds;
        s_ae[w] = ae; s_ce[w] = ce; s_de[w] = de;
        __syncthreads();
        T ps, pe, us, ue, vs, ve;
        {
            const T qas = s_as[q], qcs = s_cs[q], qae = s_ae[q], qce = s_ce[q];
            group_solve_spikes<T>(qas, qcs, s_ds[q], qae, qce, s_de[q], rt, ps, pe, us, ue, vs,
                                  ve);
        }
        // send this chunk's F (first tile) and E (last tile) values to slot
        // `rank` of every CTA of the cluster
        if (rt == 0 || rt == NT - 1) {
            const int row = rt == 0 ? 0 : 1;
            const T v0 = rt == 0 ? ps : pe, v1 = rt == 0 ? us : ue, v2 = rt == 0 ? vs : ve;
            const uint32_t loc = smem_u32(gj + size_t(rank) * 6 * SG + row * SG + rs);
            const uint32_t lbar = smem_u32(&gbar[j & 1]);
            for (int r = 0; r < C; ++r) {
                const uint32_t dst = cluster_map(loc, uint32_t(r));
                const uint32_t bar = cluster_map(lbar, uint32_t(r));
                st_async_f32(dst, v0, bar);
                st_async_f32(dst + 2u * SG * uint32_t(sizeof(T)), v1, bar);
                st_async_f32(dst + 4u * SG * uint32_t(sizeof(T)), v2, bar);
            }
        }
        // every chunk's values of this strip have landed (bounded wait)
        if (!mbar_wait(&gbar[j & 1], uint32_t(j >> 1) & 1u, status)) *(volatile int *)&abort_flag = 1;
        if (tid < SG) {
            // chunk-level system of system `tid`: forward elimination
            // E_k = al_k + be_k F_{k+1}, F_k = ga_k + de_k F_{k+1}
            T al = T(0), be = T(0);
            for (int k = 0; k < C; ++k) {
                T *g = gj + size_t(k) * 6 * SG + tid;
                const T p0 = g[0], p1 = g[SG], q0 = g[2 * SG], q1 = g[3 * SG];
                const T r0 = g[4 * SG], r1 = g[5 * SG];
                const T inv = rcp(T(1) - q0 * be);
                const T ga = (p0 + q0 * al) * inv, dl = r0 * inv;
                const T nal = p1 + q1 * (al + be * ga);
                const T nbe = r1 + q1 * be * dl;
                g[0] = ga; g[4 * SG] = dl; g[SG] = nal; g[5 * SG] = nbe;
                al = nal;
                be = nbe;
            }
            // back substitution from F_C = 0 down to this chunk
            T fnext = T(0), xl = T(0), xr = T(0);
            for (int k = C - 1; k >= rank - 1 && k >= 0; --k) {
                const T *g = gj + size_t(k) * 6 * SG + tid;
                if (k == rank) xr = fnext;
                if (k == rank - 1) xl = g[SG] + g[5 * SG] * fnext;  // E_{rank-1}
                fnext = g[0] + g[4 * SG] * fnext;                   // F_k
            }
            xlr[tid] = xl;
            xlr[SG + tid] = xr;
        }
        __syncthreads();
        {
            const T xl = xlr[rs], xr = xlr[SG + rs];
            s_xs[q] = ps + us * xl + vs * xr;
            s_xe[q] = pe + ue * xl + ve * xr;
        }
        __syncthreads();
        tile_substitute<T, M>(ra, rc, rd, s_xs[w], s_xe[w]);
        if (tma_store) {
            // x leaves through the shared-memory box and one TMA store per
            // 256 rows: the async stores stay out of every thread's release
            // fence at the next cluster barrier (global stores issued by the
            // threads would have to complete there first)
            if (tid == 0) bulk_wait_read_all();  // the previous strip's store has read xst
            __syncthreads();
            if (active) {
#pragma unroll
                for (int k = 0; k < M; ++k) xst[(i0 + k) * SG + sl] = rd[k];
            }
            fence_proxy_async_smem();
            __syncthreads();
            if (tid == 0 && ok) {
#pragma unroll
                for (int h = 0; h < CH / CK_BOX; ++h)
                    if (g0 + h * CK_BOX < n)  // rows past n (and x past inner) are clipped
                        tma_store_3d(&maps.map[4], xg * SG, g0 + h * CK_BOX, o,
                                     xst + size_t(h) * CK_BOX * SG);
                bulk_commit();
            }
        } else if (active) {
            T *ob = out + (int64_t(o) * L.inner * L.n + x);
#pragma unroll
            for (int k = 0; k < M; ++k) {
                const int gi = g0 + i0 + k;
                if (gi < n) {
                    T *p = ob + int64_t(gi) * stride;
                    *p = accumulate ? *p + rd[k] : rd[k];
                }
            }
        }
    }
    if (tma_store && tid == 0) bulk_wait_all();  // every store of this CTA has landed
    cluster.sync();  // no CTA leaves while values it sent may still be in flight
}

}  // namespace trid
