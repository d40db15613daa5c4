// trid_adi_2pass.cuh -- two-pass schedule of the 3D ADI step (Section 4.1)
// with the constant operator's precomputed tables.
//
// One step is  u <- u + Z^{-1} Y^{-1} X^{-1} d  with d the explicit 7-point
// right-hand side.  Since Z^{-1}(Z u + w) = u + Z^{-1} w, it is computed as
//   pass A (k_adi_xy):   per (16-row y tile, z plane): stencil RHS, x solve
//                        (lane tiles + shuffled PCR), then the Section 3.1
//                        tile pass of the y solve on the tile's columns.  It
//                        writes  e = (hatted y-tile values) + Z u  for every
//                        point and the two reduced right-hand sides of each
//                        (column, tile).  The last block to finish a plane
//                        solves that plane's reduced y systems (2 unknowns per
//                        tile, unit diagonal, Thomas with host-factored
//                        pivots) in place.
//   pass B (k_adi_z_ysub): per [16 x, nz] box at fixed y: finishes the y
//                        solve by substitution, q = e + alpha_r x_s + beta_r
//                        x_e, then solves Z u_new = q along z (identity rows
//                        at z = 0, nz - 1 carry q through) and stores u_new.
// DRAM per point: A reads u, writes e; B reads e, writes u; plus the reduced
// values (2 per 16 points, written by A and read by B).
#pragma once
#include "trid_adi_static.cuh"

namespace trid {

// Reduced y system of one plane column: 2T unknowns (s_0, e_0, s_1, e_1, ...)
// with unit diagonal; Thomas factors computed on the host in double.
template <typename T>
struct YReduced {
    T sub[32], w[32], cst[32];
    int n2;
};

// y substitution weights of row r of a tile, and lambda for the z boundary rows.
template <typename T>
struct YSubst {
    T alpha[ADI_YM], beta[ADI_YM];
    T lam;
};

template <typename T, int G>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 4 : 1)
k_adi_xy(const T *__restrict__ u, T *__restrict__ e, T *__restrict__ rs, T *__restrict__ re,
         unsigned *__restrict__ cnt, const T *__restrict__ gtab, int nx, int ny, int nz, T lam,
         const __grid_constant__ AdiStatics<T, ADI_XM> sx,
         const __grid_constant__ AdiStatics<T, ADI_YM> sy,
         const __grid_constant__ YReduced<T> ry) {
    constexpr int M = ADI_XM;
    constexpr int YM = ADI_YM;
    constexpr unsigned FULL = 0xffffffffu;
    extern __shared__ __align__(16) unsigned char smem_xy[];
    T *sd = reinterpret_cast<T *>(smem_xy);  // [YM][nx] x-solved right-hand side
    T *sz = sd + YM * nx;                     // [YM][nx] Z u
    __shared__ T lane_tab[AS_NLANE][32];
    __shared__ int s_last;
    const int tid = threadIdx.x;
    // per-lane reduced-solve factors: a coalesced copy of the table that
    // k_adi_setup wrote (a lane-indexed read of the kernel parameters would
    // serialise on the constant cache in every block)
    for (int q = tid; q < AS_NLANE * 32; q += blockDim.x) (&lane_tab[0][0])[q] = gtab[q];
    __syncthreads();
    const int lane = tid & 31, warp = tid >> 5;
    const int g = lane % G;
    const bool firstx = (g == 0), lastx = (g == sx.real_tiles - 1);
    const int x0 = g * M;
    const int ntile = ny / YM;
    const int plane = nx * ny;
    const T c6 = T(6) * lam, bz = T(1) + T(2) * lam;
    constexpr int RPW = 32 / G;  // rows per warp pass
    constexpr int PASSES = (YM * G + 255) / 256;
    const int c = tid;  // column of the y tile pass
    {
        // z: plane over the whole batch (meshes stacked along z); the
        // boundary test uses the plane's index inside its own mesh
        const int t = int(blockIdx.x), z = int(blockIdx.y);
        const int zl = z % nz;
        const bool zint = zl > 0 && zl < nz - 1;
        const T *ut = u + size_t(z) * size_t(plane) + size_t(t) * YM * nx;

        // x solve of the tile's rows; G lanes per row
#pragma unroll 1
        for (int p = 0; p < PASSES; ++p) {
            const int r = p * 8 * RPW + warp * RPW + lane / G;
            const bool act = r < YM && x0 < nx;
            const int y = t * YM + r;
            const bool rowint = act && zint && y > 0 && y < ny - 1;
            const T *row = ut + r * nx;
            T uc[M], zs[M], d[M], zu[M], ym[M], yp[M];
            // all five lines' loads in flight together (one round trip): the
            // y neighbours of a boundary row are read from the row itself and
            // not used
            load_line_tile<T, M>(row, x0, nx, act, uc);
            load_line_tile<T, M>(rowint ? row - nx : row, x0, nx, act, ym);
            load_line_tile<T, M>(rowint ? row + nx : row, x0, nx, act, yp);
            {
                T zm[M], zp[M];
                load_line_tile<T, M>(row - plane, x0, nx, act && zint, zm);
                load_line_tile<T, M>(row + plane, x0, nx, act && zint, zp);
#pragma unroll
                for (int j = 0; j < M; ++j) zs[j] = zm[j] + zp[j];
            }
#pragma unroll
            for (int j = 0; j < M; ++j) zu[j] = zint ? fma(-lam, zs[j], bz * uc[j]) : uc[j];
            const T left = __shfl_up_sync(FULL, uc[M - 1], 1, G);
            const T right = __shfl_down_sync(FULL, uc[0], 1, G);
            if (rowint) {
#pragma unroll
                for (int j = 0; j < M; ++j) {
                    const T xm = (j == 0) ? left : uc[j - 1];
                    const T xp = (j == M - 1) ? right : uc[j + 1];
                    const T s = ((xm + xp) + (ym[j] + yp[j])) + zs[j];
                    d[j] = fma(lam, s, -c6 * uc[j]);
                }
                if (firstx) d[0] = T(0);
                if (lastx) d[M - 1] = T(0);
            } else {
#pragma unroll
                for (int j = 0; j < M; ++j) d[j] = T(0);
            }
            T ds, de, xs, xe;
            static_tile_reduce<T, M>(sx, d, firstx, lastx, ds, de);
            static_group_solve_tab<T, G>(lane_tab, ds, de, g, xs, xe, sx.rounds);
            static_tile_substitute<T, M>(sx, d, xs, xe);
            if (act) {
                store_contig_vec<T, M>(sd + r * nx + x0, d);
                store_contig_vec<T, M>(sz + r * nx + x0, zu);
            }
        }
        __syncthreads();

        // tile pass of the y solve, one thread per column
        const size_t rbase = size_t(z) * ntile * nx + c;
        if (c < nx) {
            T v[YM];
#pragma unroll
            for (int r = 0; r < YM; ++r) v[r] = sd[r * nx + c];
            T ds, de;
            static_tile_reduce<T, YM>(sy, v, t == 0, t == ntile - 1, ds, de);
            T *ecol = e + (size_t(z) * plane + size_t(t) * YM * nx + c);
#pragma unroll
            for (int r = 0; r < YM; ++r) {
                const T zr = sz[r * nx + c];
                ecol[r * nx] = (r == 0 || r == YM - 1) ? zr : v[r] + zr;
            }
            rs[rbase + size_t(t) * nx] = ds;
            re[rbase + size_t(t) * nx] = de;
        }

        // the last block to finish a plane solves its reduced y systems
        __syncthreads();
        if (tid == 0) {
            __threadfence();
            s_last = (atomicAdd(&cnt[z], 1u) == unsigned(ntile - 1));
            __threadfence();
        }
        __syncthreads();
        if (s_last) {
            if (c < nx) {
                // the column's reduced system, in registers: all loads in
                // flight at once (one L2 round trip), then the Thomas sweeps
                const int n2 = ry.n2;
                T y[32];
#pragma unroll
                for (int k = 0; k < 32; ++k) {
                    const T *src = (k & 1) ? re : rs;
                    y[k] = (k < n2) ? __ldcg(src + rbase + size_t(k >> 1) * nx) : T(0);
                }
                T prev = T(0);
#pragma unroll
                for (int k = 0; k < 32; ++k) {
                    if (k < n2) {
                        prev = (y[k] - ry.sub[k] * prev) * ry.w[k];
                        y[k] = prev;
                    }
                }
                T xn = T(0);
#pragma unroll
                for (int k = 31; k >= 0; --k) {
                    if (k < n2) {
                        xn = fma(-ry.cst[k], xn, y[k]);
                        T *dst = (k & 1) ? re : rs;
                        dst[rbase + size_t(k >> 1) * nx] = xn;
                    }
                }
            }
            if (tid == 0) cnt[z] = 0u;  // ready for the next step
        }
    }
}

// Once per call: the per-lane factor table of the x solve into device memory,
// and the per-plane completion counters to zero.
template <typename T>
__global__ void k_adi_setup(const __grid_constant__ AdiStatics<T, ADI_XM> sx, T *gtab,
                            unsigned *cnt, int nz) {
    __shared__ T tab[AS_NLANE][32];
    stage_lane_statics<T>(sx, tab, threadIdx.x, blockDim.x);
    __syncthreads();
    for (int q = threadIdx.x; q < AS_NLANE * 32; q += blockDim.x) gtab[q] = (&tab[0][0])[q];
    for (int q = threadIdx.x; q < nz; q += blockDim.x) cnt[q] = 0u;
}

// ---------------------------------------------------------------------------
// Pass B: y substitution + z solve, TMA-fed like k_adi_strided_static.  Each
// stage holds three [SG x nz] boxes: e, and the x_s / x_e of the y tile of
// the box's row (the reduced arrays are laid out [z][tile][x]).  Reading the
// last two through the consumers' own loads instead cost more issue slots
// and latency than the extra shared memory does.
// ---------------------------------------------------------------------------
template <typename T, int NT, int SG>
__global__ void __launch_bounds__(NT * SG + 32, 2)
k_adi_z_ysub(const __grid_constant__ TmaSet maps,
             const __grid_constant__ AdiStatics<T, ADI_YM> st,
             const __grid_constant__ YSubst<T> ys, T *out, int nx, int nplane, int n,
             int64_t nbatch, int stages, int *status) {
    // batches: nbox boxes of SG columns per z line set of one mesh, meshes
    // stacked (nbatch = nbox * number of meshes)
    const int64_t nbox = nplane / SG;
    constexpr int M = ADI_YM;
    constexpr int P = SG + 1;
    constexpr int NCONS = NT * SG;
    static_assert(NCONS % 32 == 0, "consumers must be whole warps");
    constexpr int NSLOT = 3;
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ int abort_flag;
    __shared__ T lane_tab[AS_NLANE][32];
    const size_t slot_bytes = (size_t(n) * SG * sizeof(T) + 127) / 128 * 128;
    const size_t stage_bytes = NSLOT * slot_bytes;
    T *s_ds = reinterpret_cast<T *>(smem + stages * stage_bytes);
    T *s_de = s_ds + NT * P;
    T *s_xs = s_de + NT * P;
    T *s_xe = s_xs + NT * P;
    uint64_t *full = reinterpret_cast<uint64_t *>(
        smem + stages * stage_bytes + (4 * NT * P * sizeof(T) + 127) / 128 * 128);
    uint64_t *empty = full + stages;

    const int tid = threadIdx.x;
    stage_lane_statics<T>(st, lane_tab, tid, blockDim.x);
    if (tid == 0) {
        abort_flag = 0;
        for (int s = 0; s < stages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], NCONS / 32);
        }
        fence_mbar_init();
    }
    __syncthreads();

    if (tid >= NCONS) {
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
                const int mesh = int(bt / nbox);
                const int f0 = int(bt - int64_t(mesh) * nbox) * SG;
                const int y = f0 / nx;
                const int rx = (y / M) * nx + (f0 - y * nx);
                unsigned char *dst = smem + s * stage_bytes;
                tma_load_3d(dst, &maps.map[0], f0, 0, mesh, &full[s]);
                tma_load_3d(dst + slot_bytes, &maps.map[1], rx, 0, mesh, &full[s]);
                tma_load_3d(dst + 2 * slot_bytes, &maps.map[2], rx, 0, mesh, &full[s]);
            }
        }
        return;
    }

    const int lane = tid & 31;
    const int sl = tid % SG;
    const int tile = tid / SG;
    const int i0 = tile * M;
    const int w = tile * P + sl;
    const bool first = (tile == 0);
    const bool last = (tile == st.real_tiles - 1);
    const int rsn = tid / NT, rt = tid % NT;
    const int q = rt * P + rsn;
    LaneStatics<T> LS;
    LS.load(lane_tab, rt);
    const T lam = ys.lam;
    int k = 0;
    for (int64_t bt = blockIdx.x; bt < nbatch; bt += gridDim.x, ++k) {
        const int s = k % stages;
        bool ok = false;
        if (!*(volatile int *)&abort_flag) {
            ok = mbar_wait(&full[s], uint32_t(k / stages) & 1u, status);
            if (!ok) *(volatile int *)&abort_flag = 1;
        }
        const T *se = reinterpret_cast<const T *>(smem + s * stage_bytes);
        const T *sxs = reinterpret_cast<const T *>(smem + s * stage_bytes + slot_bytes);
        const T *sxe = reinterpret_cast<const T *>(smem + s * stage_bytes + 2 * slot_bytes);
        const int b32 = int(bt), nb32 = int(nbox);
        const int mesh = b32 / nb32;
        const int f0 = (b32 - mesh * nb32) * SG;
        const int r = (f0 / nx) % M;
        const T al = ys.alpha[r], be = ys.beta[r];
        // n is a multiple of M: a tile is entirely inside the line or padding
        const bool tin = ok && i0 < n;
        T d[M];
#pragma unroll
        for (int j = 0; j < M; ++j) {
            const int o = (i0 + j) * SG + sl;
            d[j] = tin ? fma(be, sxe[o], fma(al, sxs[o], se[o])) : T(0);
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[s]);
        // identity rows at z = 0 and z = n - 1: their value is q itself and
        // enters the neighbouring interior row's right-hand side
        const T b0 = d[0], b1 = d[M - 1];
        if (first) d[1] = fma(lam, b0, d[1]);
        if (last) d[M - 2] = fma(lam, b1, d[M - 2]);
        T ds, de;
        static_tile_reduce<T, M>(st, d, first, last, ds, de);
        s_ds[w] = ds;
        s_de[w] = de;
        named_barrier(1, NCONS);
        {
            T xs, xe;
            static_group_solve<T, NT>(LS, s_ds[q], s_de[q], rt, xs, xe, st.rounds);
            s_xs[q] = xs;
            s_xe[q] = xe;
        }
        named_barrier(1, NCONS);
        static_tile_substitute<T, M>(st, d, s_xs[w], s_xe[w]);
        if (first) d[0] = b0;
        if (last) d[M - 1] = b1;
        if (tin) {
            T *ob = out + (size_t(mesh) * n + i0) * nplane + f0 + sl;
#pragma unroll
            for (int j = 0; j < M; ++j, ob += nplane) *ob = d[j];
        }
    }
}

}  // namespace trid
