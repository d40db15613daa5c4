// trid_adi_window.cuh -- 3D ADI step (Section 4.1, Algorithm "adi") with the
// y and z solves computed over windows of the constant operator.
//
// The inverse of the ADI operator tridiag(-lambda, 1 + 2 lambda, -lambda)
// decays geometrically away from its diagonal: Thomas' forward multipliers
// and back-substitution factors converge to rho = |c*| of the infinite line
// (0.084 for lambda = 0.1).  A right-hand-side value k rows away from row i
// moves x_i by about rho^k relative, so when rho^(H+1) is below 2^-28 (1/16
// of an FP32 ulp; H = 8 for lambda = 0.1) the rows of a tile need only the
// right-hand side within H rows of the tile: Thomas on the window [tile - H,
// tile + H] -- physical boundary rows kept exactly, the couplings across the
// window's two ends dropped -- returns the tile's rows to within that bound.
// The host computes the bound from the operator and precision (as it does for
// the early stop of the PCR rounds) and takes this path only when it holds.
//
// One step is u <- u + Z^{-1} Y^{-1} X^{-1} d with d the explicit 7-point
// right-hand side, computed as u <- Z^{-1}(Z u + Y^{-1} X^{-1} d):
//   pass A (k_adi_xyw): one CTA per (32-row y tile, z plane), the tiles of a
//     plane forming a thread-block cluster.  Warps compute the stencil and
//     Z u of the tile's rows (the z neighbours staged in shared memory by
//     cp.async) and solve x (lane tiles of 8 points, one cyclic-reduction fold
//     through warp shuffles, Section 3.1 form), leaving X^{-1} d in shared
//     memory.  The y window solve is split by linearity (WinSplit): each CTA
//     sends its two neighbours one scalar per column summarising the rows
//     they need (st.async into their shared memory, counted on an mbarrier),
//     solves its own rows with zero halos meanwhile, adds the received
//     summaries' responses and writes e = Y^{-1} X^{-1} d + Z u.
//   pass B (k_adi_zw): a producer warp streams [32 x, nz] boxes of e into a
//     ring of shared-memory stages (TMA, mbarrier completion); one consumer
//     warp per 16-row z tile solves the tile's z window for the box's 32 lines
//     and stores u.  Identity rows at z = 0 and nz - 1 carry e through.
// DRAM per point: A reads u and writes e; B reads e and writes u (4 words).
#pragma once
#include "trid_adi_static.cuh"

namespace trid {

constexpr int WIN_H = 8;                  // window rows on each side of a tile
constexpr int WA_YT = 32;                 // y rows per CTA of pass A
constexpr int WA_W = WA_YT + 2 * WIN_H;   // y window rows
constexpr int WB_ZT = 16;                 // z rows per consumer warp of pass B
constexpr int WB_W = WB_ZT + 2 * WIN_H;   // z window rows
constexpr int WB_SG = 32;                 // x lines per box of pass B

// Thomas factors of a tile's window, per tile kind (0 first, 1 interior,
// 2 last, 3 the only tile): forward f_j = F_j d_j + FA_j f_{j-1}, backward
// x_j = f_j - C_j x_{j+1}.  Window rows outside the line have F = FA = C = 0.
template <typename T, int W>
struct WinTab {
    T F[4][W], FA[4][W], C[4][W];
};

// The tile-pass multipliers of the x solve (the part of AdiStatics that the
// fold-only solve reads; a small kernel parameter keeps the launch cheap).
template <typename T, int AS_M>
struct XTile {
    T F[AS_M], G[AS_M], B[AS_M], SA[AS_M], SC[AS_M];
    T DS0, DS1;
    int real_tiles;
};

// The y window solve of a 32-row tile split by linearity (window rows 0..7
// the halo above, 8..39 the tile, 40..47 the halo below; x = X^{-1} d per
// column):
//   x_tile = x0 + T h + B b,
// where x0 is the window solve with both halos zero (Thomas over the tile's
// rows, the rows below entering only through x_40 = R f_39), h = sum_k Wt_k
// v_k the forward value that the halo above leaves at window row 7, b = sum_k
// Wb_k v_{40+k} the value x_40 that the halo below alone produces, T the
// tile's response to a unit forward value at row 7 and B its response to a
// unit x_40.  A CTA computes h and b for its neighbours from its own rows and
// sends them one scalar per column, so no CTA reads another's rows.  Per tile
// kind (0 first, 1 interior, 2 last, 3 only); halves that do not exist are 0.
struct WinSplit {
    float F[4][WA_YT], FA[4][WA_YT], C[4][WA_YT];  // window rows 8..39
    float R[4];
    float T[4][WA_YT], B[4][WA_YT];
    float Wt[4][WIN_H], Wb[4][WIN_H];
};

// Fold factors of the x solve per lane kind (0 first tile of the line,
// 1 interior tile, 2 last tile, 3 lane beyond the line); the reduced rows of
// the constant operator are the same for every interior tile.
template <typename T>
struct XFold {
    T fr[4], fae[4], fce[4], xas[4], xcs[4];
};

__device__ __forceinline__ void cluster_wait_acquire() {
    asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

__device__ __forceinline__ void cluster_arrive_relaxed() {
    asm volatile("barrier.cluster.arrive.relaxed.aligned;" ::: "memory");
}

template <typename T>
__device__ __forceinline__ T pick4(int k, const T (&v)[4]) {
    return k == 0 ? v[0] : (k == 1 ? v[1] : (k == 2 ? v[2] : v[3]));
}

// Thomas over a window held in registers, with the factors of tile kind K
// (a compile-time index, so every factor is an immediate constant operand):
// forward over all W rows, backward down to row `lo`.
template <int K, int W, int lo>
__device__ __forceinline__ void win_solve_k(float (&v)[W], const WinTab<float, W> &tab) {
    float f = 0.0f;
#pragma unroll
    for (int j = 0; j < W; ++j) {
        f = fmaf(tab.FA[K][j], f, tab.F[K][j] * v[j]);
        v[j] = f;
    }
    float xv = v[W - 1];
#pragma unroll
    for (int j = W - 2; j >= lo; --j) {
        xv = fmaf(-tab.C[K][j], xv, v[j]);
        v[j] = xv;
    }
}


// The tile's part of the split window solve for kind K: Thomas over the 32
// tile rows with zero halos (x_40 = R f_39).
template <int K>
__device__ __forceinline__ void tile_own_solve(float (&v)[WA_YT], const WinSplit &ys) {
    float f = 0.0f;
#pragma unroll
    for (int j = 0; j < WA_YT; ++j) {
        f = fmaf(ys.FA[K][j], f, ys.F[K][j] * v[j]);
        v[j] = f;
    }
    float xv = ys.R[K] * f;
#pragma unroll
    for (int j = WA_YT - 1; j >= 0; --j) {
        xv = fmaf(-ys.C[K][j], xv, v[j]);
        v[j] = xv;
    }
}
template <int K>
__device__ __forceinline__ void tile_halo_add(float (&v)[WA_YT], const WinSplit &ys, float h,
                                              float b) {
#pragma unroll
    for (int j = 0; j < WA_YT; ++j) {
        if (K == 1 || K == 2) v[j] = fmaf(ys.T[K][j], h, v[j]);
        if (K == 0 || K == 1) v[j] = fmaf(ys.B[K][j], b, v[j]);
    }
}

// Shared-memory rows of pass A are swizzled: 16-byte chunk q of a row sits at
// chunk q ^ ((q >> 3) & 1), so that the eight lanes of a quarter warp, each
// reading its own 32-byte piece (chunks 2g, 2g + 1), and the 32 threads of a
// warp reading one column each, both hit 32 different banks.
__device__ __forceinline__ int swz_chunk(int q) { return q ^ ((q >> 3) & 1); }
__device__ __forceinline__ int swz_elem(int x) { return (swz_chunk(x >> 2) << 2) | (x & 3); }

__device__ __forceinline__ void lds8_swz(const float *row, int x0, float (&r)[8]) {
    const float4 a = *reinterpret_cast<const float4 *>(row + (swz_chunk(x0 >> 2) << 2));
    const float4 b = *reinterpret_cast<const float4 *>(row + (swz_chunk((x0 >> 2) + 1) << 2));
    r[0] = a.x; r[1] = a.y; r[2] = a.z; r[3] = a.w;
    r[4] = b.x; r[5] = b.y; r[6] = b.z; r[7] = b.w;
}
__device__ __forceinline__ void sts8_swz(float *row, int x0, const float (&r)[8]) {
    *reinterpret_cast<float4 *>(row + (swz_chunk(x0 >> 2) << 2)) = make_float4(r[0], r[1], r[2], r[3]);
    *reinterpret_cast<float4 *>(row + (swz_chunk((x0 >> 2) + 1) << 2)) =
        make_float4(r[4], r[5], r[6], r[7]);
}

// 16-byte asynchronous global -> shared copies (Ampere-style cp.async), one
// commit group per row of a lane group.
__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
    asm volatile("cp.async.commit_group;" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// ---------------------------------------------------------------------------
// Pass A.  Grid (ny / 32, nz * nbatch) in clusters of (ny / 32, 1, 1): the
// cluster is one z plane (meshes stacked along z), CTA t its rows
// [32 t, 32 t + 32).  256 threads.  In the x phase a group of G lanes (lane g
// owning x in [8 g, 8 g + 8)) walks a run of consecutive rows with the rows
// y - 1, y, y + 1 in registers, loading the rows ahead.  In the y phase thread
// c handles column c: the halo summaries for the neighbours, its own rows'
// window solve, the received summaries' responses, the store of e.
// ---------------------------------------------------------------------------
// PPC planes per CTA (1, or 32 / G when a plane is one 32-row tile: then the
// planes' rows fill the lane groups and their columns the threads of the y
// phase); the planes of a CTA are consecutive in the stacked z order.
template <int G, int NXC, int PPC>  // NXC: nx as a compile-time constant (0: run-time nx)
__global__ void __launch_bounds__(256, 3)
k_adi_xyw(const float *u, float *e, int nx_arg, int ny, int nz, float lam,
          float c6, float bz, const __grid_constant__ XTile<float, ADI_XM> sx,
          const __grid_constant__ XFold<float> xf, const __grid_constant__ WinSplit ys,
          int *status) {
    constexpr int M = ADI_XM;
    constexpr unsigned FULL = 0xffffffffu;
    const int nx = NXC ? NXC : nx_arg;  // constant row strides when NXC is given
    constexpr int NGROUP = 8 * (32 / G);                      // lane groups per CTA
    constexpr int ROWS = PPC * WA_YT;                         // rows of the CTA's planes
    constexpr int RG = NGROUP >= ROWS ? 1 : ROWS / NGROUP;    // rows per group
    static_assert(PPC == 1 || RG * NGROUP == ROWS, "several planes fill every lane group");
    extern __shared__ __align__(16) unsigned char smem_xyw[];
    float *sd = reinterpret_cast<float *>(smem_xyw);  // [PPC * 32][nx] X^{-1} d
    float *sz = sd + ROWS * nx;                        // [PPC * 32][nx] Z u
    float *rh = sz + ROWS * nx;   // [nx] h from the tile above
    float *rb = rh + nx;          // [nx] b from the tile below
    uint64_t *rbar = reinterpret_cast<uint64_t *>(rb + nx);  // both have landed
    const int tid = threadIdx.x, lane = tid & 31;
    const int g = lane % G;
    // the group's first row: row rl of plane pl of the CTA; rows r0 .. r0 + RG - 1
    // of the CTA's shared-memory tiles
    const int r0 = ((tid >> 5) * (32 / G) + lane / G) * RG;
    const int pl = PPC == 1 ? 0 : r0 / WA_YT, rl = PPC == 1 ? r0 : r0 % WA_YT;
    const bool gact = r0 < ROWS && g * M < nx;
    const int x0 = g * M;
    const int t = int(blockIdx.x), ntile = int(gridDim.x);
    const int z = int(blockIdx.y) * PPC + pl;  // the group's plane (stacked z)
    const int zl = z % nz;
    const bool zint = zl > 0 && zl < nz - 1;
    const int plane = nx * ny;
    const int y0 = t * WA_YT;
    const float *ut = u + size_t(z) * size_t(plane) + size_t(y0) * nx + x0;
    // elements of u and e (all planes of all meshes): the debug build's bounds
    [[maybe_unused]] const int64_t total = int64_t(gridDim.y) * PPC * plane;
    auto ld = [&](int dy, int dz, bool ok, float (&v)[M]) {  // row y0 + dy of plane z + dz
        if (ok && TRID_BOUNDS(in_span(ut + (dz * ny + dy) * nx - u, M, total))) {
            load_contig_vec<float, M>(ut + (dz * ny + dy) * nx, v);
        } else {
#pragma unroll
            for (int j = 0; j < M; ++j) v[j] = 0.0f;
        }
    };
    if (tid == 0) {
        mbar_init(rbar, 1);
        fence_mbar_init();
    }
    // every CTA's mbarrier is initialised before any neighbour sends to it
    cluster_arrive_relaxed();
    pdl_trigger();
    pdl_wait();  // u is written by the previous kernel on the stream
    // the rows y - 1 .. y + 1 of the group's first row first, then the z
    // neighbours of every row of the group (all in flight at once; plane
    // z - 1 lands where X^{-1} d of the row will go, plane z + 1 where its
    // Z u will go, each lane copying, and later reading, only its own chunks),
    // then the row y + 2
    const bool yok0 = y0 + rl - 1 >= 0;
    float ym[M], uc[M], yp[M], yq[M];  // rows y - 1 .. y + 2 of the group's first row
    ld(rl - 1, 0, gact && yok0, ym);
    ld(rl, 0, gact, uc);
    ld(rl + 1, 0, gact && y0 + rl + 1 < ny, yp);
#pragma unroll
    for (int i = 0; i < RG; ++i) {
        const int r = rl + i;  // row of the plane; r0 + i: row of the tiles
        if (gact && zint && TRID_BOUNDS(in_span(ut + r * nx - ny * nx - u, M, total) &&
                                        in_span(ut + r * nx + ny * nx - u, M, total))) {
            const float *src = ut + r * nx;
            float *dm = sd + (r0 + i) * nx, *dp = sz + (r0 + i) * nx;
            const int q0 = x0 >> 2;
            cp_async16(dm + (swz_chunk(q0) << 2), src - ny * nx);
            cp_async16(dm + (swz_chunk(q0 + 1) << 2), src - ny * nx + 4);
            cp_async16(dp + (swz_chunk(q0) << 2), src + ny * nx);
            cp_async16(dp + (swz_chunk(q0 + 1) << 2), src + ny * nx + 4);
        }
        cp_async_commit();
    }
    ld(rl + 2, 0, gact && RG > 1 && y0 + rl + 2 < ny, yq);
    const int rt = sx.real_tiles;
    const bool firstx = (g == 0), lastx = (g == rt - 1);
    const int kd = g == 0 ? 0 : (g < rt - 1 ? 1 : (g == rt - 1 ? 2 : 3));
    const float fr = pick4(kd, xf.fr), fae = pick4(kd, xf.fae), fce = pick4(kd, xf.fce);
    const float xas = pick4(kd, xf.xas), xcs = pick4(kd, xf.xcs);

#pragma unroll
    for (int i = 0; i < RG; ++i) {
        const int r = rl + i;   // row of the plane
        const int rs = r0 + i;  // row of the shared-memory tiles
        const int y = y0 + r;
        // the rows two and three ahead stay in flight while this row is solved
        float ny3[M];
        ld(r + 3, 0, gact && i + 2 < RG && y + 3 < ny, ny3);
        const bool rowint = gact && zint && y > 0 && y < ny - 1;
        // this row's z neighbours have landed (this lane's own copies)
        if (i == 0) cp_async_wait<RG - 1>();
        if (i == 1) cp_async_wait<(RG > 1 ? RG - 2 : 0)>();
        if (i == 2) cp_async_wait<(RG > 2 ? RG - 3 : 0)>();
        if (i == 3) cp_async_wait<0>();
        float zs[M];
        if (gact && zint) {
            float zp[M];
            lds8_swz(sd + rs * nx, x0, zs);
            lds8_swz(sz + rs * nx, x0, zp);
#pragma unroll
            for (int j = 0; j < M; ++j) zs[j] += zp[j];
        } else {
#pragma unroll
            for (int j = 0; j < M; ++j) zs[j] = 0.0f;
        }
        float d[M];
        {
            float zu[M];
#pragma unroll
            for (int j = 0; j < M; ++j) zu[j] = zint ? fmaf(-lam, zs[j], bz * uc[j]) : uc[j];
            if (gact) sts8_swz(sz + rs * nx, x0, zu);
        }
        const float left = __shfl_up_sync(FULL, uc[M - 1], 1, G);
        const float right = __shfl_down_sync(FULL, uc[0], 1, G);
        if (rowint) {
#pragma unroll
            for (int j = 0; j < M; ++j) {
                const float xm = (j == 0) ? left : uc[j - 1];
                const float xp = (j == M - 1) ? right : uc[j + 1];
                const float sm = ((xm + xp) + (ym[j] + yp[j])) + zs[j];
                d[j] = fmaf(lam, sm, -c6 * uc[j]);
            }
            if (firstx) d[0] = 0.0f;
            if (lastx) d[M - 1] = 0.0f;
        } else {
#pragma unroll
            for (int j = 0; j < M; ++j) d[j] = 0.0f;
        }
        float ds, de;
        static_tile_reduce<float, M>(sx, d, firstx, lastx, ds, de);
        {
            // reduced system of the line's tiles: one fold (its coupling is
            // below the bound the host checked, so no PCR round follows)
            float nds = __shfl_down_sync(FULL, ds, 1, G);
            if (g + 1 >= G) nds = 0.0f;
            const float xe = fmaf(-fce, nds, fmaf(-fae, ds, fr * de));
            float xprev = __shfl_up_sync(FULL, xe, 1, G);
            if (g == 0) xprev = 0.0f;
            const float xs = fmaf(-xcs, xe, fmaf(-xas, xprev, ds));
            static_tile_substitute<float, M>(sx, d, xs, xe);
        }
        if (gact) sts8_swz(sd + rs * nx, x0, d);
#pragma unroll
        for (int j = 0; j < M; ++j) {
            ym[j] = uc[j];
            uc[j] = yp[j];
            yp[j] = yq[j];
            yq[j] = ny3[j];
        }
    }
    __syncthreads();  // this CTA's X^{-1} d rows are complete
    const bool has_up = t > 0, has_dn = t < ntile - 1;
    if (tid == 0) mbar_expect_tx(rbar, uint32_t((has_up ? nx : 0) + (has_dn ? nx : 0)) * 4u);
    // thread (yp, c): column c of the CTA's plane yp
    const int c = PPC == 1 ? tid : tid % nx, ypl = PPC == 1 ? 0 : tid / nx;
    const bool col = PPC == 1 ? c < nx : ypl < PPC;
    const int cs = swz_elem(c);
    float *sdc = sd + ypl * WA_YT * nx;  // the plane's tiles
    const float *szc = sz + ypl * WA_YT * nx;
    const int zy = int(blockIdx.y) * PPC + ypl;  // its plane (stacked z)
    const int kind = ntile == 1 ? 3 : (t == 0 ? 0 : (t == ntile - 1 ? 2 : 1));
    cluster_wait_acquire();  // the neighbours' mbarriers are initialised
    if (col) {
        // the halo summaries this tile's rows give its neighbours
        if (has_dn) {  // h of the tile below (kind 2 if it is the last, else 1)
            const bool last = t + 1 == ntile - 1;
            float h = 0.0f;
#pragma unroll
            for (int k = 0; k < WIN_H; ++k)
                h = fmaf(last ? ys.Wt[2][k] : ys.Wt[1][k], sdc[(WA_YT - WIN_H + k) * nx + cs], h);
            st_async_f32(cluster_map(smem_u32(rh + c), t + 1), h,
                         cluster_map(smem_u32(rbar), t + 1));
        }
        if (has_up) {  // b of the tile above (kind 0 if it is the first, else 1)
            const bool first = t - 1 == 0;
            float b = 0.0f;
#pragma unroll
            for (int k = 0; k < WIN_H; ++k)
                b = fmaf(first ? ys.Wb[0][k] : ys.Wb[1][k], sdc[k * nx + cs], b);
            st_async_f32(cluster_map(smem_u32(rb + c), t - 1), b,
                         cluster_map(smem_u32(rbar), t - 1));
        }
    }
    float v[WA_YT];
    if (col) {
#pragma unroll
        for (int j = 0; j < WA_YT; ++j) v[j] = sdc[j * nx + cs];
        switch (kind) {  // uniform across the CTA
            case 0: tile_own_solve<0>(v, ys); break;
            case 1: tile_own_solve<1>(v, ys); break;
            case 2: tile_own_solve<2>(v, ys); break;
            default: tile_own_solve<3>(v, ys); break;
        }
    }
    // the neighbours' summaries have landed (bounded wait)
    const bool got = mbar_wait(rbar, 0u, status);
    if (col) {
        const float h = (has_up && got) ? rh[c] : 0.0f;
        const float b = (has_dn && got) ? rb[c] : 0.0f;
        switch (kind) {
            case 0: tile_halo_add<0>(v, ys, h, b); break;
            case 1: tile_halo_add<1>(v, ys, h, b); break;
            case 2: tile_halo_add<2>(v, ys, h, b); break;
            default: break;
        }
    }
    if (col && TRID_BOUNDS(in_span(int64_t(zy) * plane + int64_t(y0) * nx + c,
                                   int64_t(WA_YT - 1) * nx + 1, total))) {
        float *ecol = e + size_t(zy) * size_t(plane) + size_t(y0) * nx + c;
#pragma unroll
        for (int j = 0; j < WA_YT; ++j) ecol[j * nx] = v[j] + szc[j * nx + cs];
    }
    // No cluster barrier before leaving: the only accesses to another CTA's
    // shared memory are the st.async summaries, and their receiver does not
    // leave before its mbarrier has counted every byte sent to it, so no CTA
    // leaves while a write into it may still land (the sender keeps no shared
    // memory that a neighbour reads).  Without that barrier a CTA's slot is
    // free as soon as its own stores are issued (pass A 41.8 -> 39.3 us).
}

// Window of a z tile of kind K from the box in shared memory (sb points at
// the window's first row, column of this lane), then the window solve.  Rows
// outside the line (before the first tile, after the last) are zero.
template <int K>
__device__ __forceinline__ void zw_load_solve(float (&v)[WB_W], const float *col, int r0,
                                              const WinTab<float, WB_W> &zw) {
#pragma unroll
    for (int j = 0; j < WB_W; ++j) {
        const bool exists = !((K == 0 || K == 3) && j < WIN_H) &&
                            !((K == 2 || K == 3) && j >= WIN_H + WB_ZT);
        v[j] = exists ? col[(r0 + j) * WB_SG] : 0.0f;
    }
    win_solve_k<K, WB_W, WIN_H>(v, zw);
}

// ---------------------------------------------------------------------------
// Pass B.  Persistent blocks of 32 * (nz / 16) consumer threads (one warp per
// z tile, one lane per x line of the box) + one producer warp.  Boxes are
// [32 x, nz] of e at (x0, mesh), mesh-major; the output u has the same layout.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(WB_SG * 16 + 32, 2)
k_adi_zw(const __grid_constant__ TmaSet maps, const __grid_constant__ WinTab<float, WB_W> zw,
         float *__restrict__ out, int nplane, int n, int64_t nbatch, int stages, int *status) {
    extern __shared__ __align__(128) unsigned char smem_zw[];
    __shared__ int abort_flag;
    const int ntz = n / WB_ZT;
    const int ncons = 32 * ntz;
    const size_t stage_bytes = (size_t(n) * WB_SG * sizeof(float) + 127) / 128 * 128;
    uint64_t *full = reinterpret_cast<uint64_t *>(smem_zw + stages * stage_bytes);
    uint64_t *empty = full + stages;
    const int64_t nbox = nplane / WB_SG;
    const int tid = threadIdx.x;
    if (tid == 0) {
        abort_flag = 0;
        for (int s = 0; s < stages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], ntz);
        }
        fence_mbar_init();
    }
    pdl_trigger();
    pdl_wait();  // e is written, and u read, by the previous kernel on the stream
    __syncthreads();

    if (tid >= ncons) {
        if (tid == ncons) {
            const uint32_t tx = uint32_t(n) * WB_SG * sizeof(float);
            int k = 0;
            for (int64_t bt = blockIdx.x; bt < nbatch; bt += gridDim.x, ++k) {
                const int s = k % stages;
                if (k >= stages && !mbar_wait(&empty[s], uint32_t((k / stages) - 1) & 1u, status)) {
                    *(volatile int *)&abort_flag = 1;
                    break;
                }
                mbar_expect_tx(&full[s], tx);
                const int mesh = int(bt / nbox);
                const int x0 = int(bt - int64_t(mesh) * nbox) * WB_SG;
                tma_load_3d(smem_zw + s * stage_bytes, &maps.map[0], x0, 0, mesh, &full[s]);
            }
        }
        return;
    }

    const int lane = tid & 31;
    const int tz = tid >> 5;  // z tile of this warp
    const int kind = ntz == 1 ? 3 : (tz == 0 ? 0 : (tz == ntz - 1 ? 2 : 1));
    const int r0 = tz * WB_ZT - WIN_H;  // first window row (negative for the first tile)
    int k = 0;
    for (int64_t bt = blockIdx.x; bt < nbatch; bt += gridDim.x, ++k) {
        const int s = k % stages;
        bool ok = false;
        if (!*(volatile int *)&abort_flag) {
            ok = mbar_wait(&full[s], uint32_t(k / stages) & 1u, status);
            if (!ok) *(volatile int *)&abort_flag = 1;
        }
        const float *col = reinterpret_cast<const float *>(smem_zw + s * stage_bytes) + lane;
        float v[WB_W];
        switch (ok ? kind : -1) {  // uniform across the warp
            case 0: zw_load_solve<0>(v, col, r0, zw); break;
            case 1: zw_load_solve<1>(v, col, r0, zw); break;
            case 2: zw_load_solve<2>(v, col, r0, zw); break;
            case 3: zw_load_solve<3>(v, col, r0, zw); break;
            default: break;
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[s]);
        if (!ok) continue;
        const int mesh = int(bt / nbox);
        const int x0 = int(bt - int64_t(mesh) * nbox) * WB_SG;
        const int64_t obase = (int64_t(mesh) * n + int64_t(tz) * WB_ZT) * nplane + x0 + lane;
        if (!TRID_BOUNDS(in_span(obase, int64_t(WB_ZT - 1) * nplane + 1,
                                 nbatch / nbox * n * int64_t(nplane))))
            continue;
        float *ob = out + obase;
#pragma unroll
        for (int j = 0; j < WB_ZT; ++j) ob[size_t(j) * nplane] = v[WIN_H + j];
    }
}

// ---------------------------------------------------------------------------
// Host: window tables and the truncation bound.
// ---------------------------------------------------------------------------

// Thomas factors of the window of `tile` (rows tile * tile_rows - H + j,
// j < W) of a line of n nodes: identity rows at nodes 0 and n - 1,
// tridiag(-lam, 1 + 2 lam, -lam) inside, the couplings across the window's
// ends dropped.  `trunc` receives the largest factor by which a dropped
// coupling can reach a tile row: (lam F_0) * prod FA_1..H at the start and
// prod of the back-substitution factors over the H + 1 rows after the tile
// at the end (0 where the window reaches the line's end).
template <int W>
inline void win_fill_one(double (&F)[W], double (&FA)[W], double (&C)[W], int n, int tile,
                         int tile_rows, double lam, double &trunc) {
    const int y0 = tile * tile_rows - WIN_H;
    double cprev = 0.0, cfull[W];
    bool prev = false;
    for (int j = 0; j < W; ++j) {
        const int y = y0 + j;
        if (y < 0 || y >= n) {
            F[j] = FA[j] = C[j] = cfull[j] = 0.0;
            cprev = 0.0;
            prev = false;
            continue;
        }
        const bool ident = (y == 0 || y == n - 1);
        const double a = (ident || !prev) ? 0.0 : -lam;
        const double b = ident ? 1.0 : 1.0 + 2.0 * lam;
        const double c_in = (ident || y + 1 >= n) ? 0.0 : -lam;  // the operator's coupling
        const double c = (j == W - 1) ? 0.0 : c_in;               // dropped at the window end
        const double den = b - a * cprev;
        F[j] = 1.0 / den;
        FA[j] = -a / den;
        C[j] = c / den;
        cfull[j] = c_in / den;
        cprev = C[j];
        prev = true;
    }
    trunc = 0.0;
    if (y0 > 0) {  // rows before the window exist: its first row lost a coupling
        double p = lam * F[0];
        for (int j = 1; j <= WIN_H; ++j) p *= fabs(FA[j]);
        trunc = fmax(trunc, p);
    }
    if (y0 + W < n) {  // rows after the window exist
        double p = 1.0;
        for (int j = W - 1 - WIN_H; j < W; ++j) p *= fabs(cfull[j]);
        trunc = fmax(trunc, p);
    }
}

// Tables of the four tile kinds of a line of n = ntile * tile_rows nodes;
// returns the largest truncation factor over the kinds that occur.
template <typename T, int W>
inline double win_fill(WinTab<T, W> &tab, int n, int tile_rows, double lam) {
    const int ntile = n / tile_rows;
    // representative tiles: first, interior, last, only
    const int rep[4] = {0, ntile >= 3 ? 1 : 0, ntile - 1, 0};
    const bool occurs[4] = {ntile >= 2, ntile >= 3, ntile >= 2, ntile == 1};
    double worst = 0.0;
    for (int k = 0; k < 4; ++k) {
        double F[W], FA[W], C[W], tr = 0.0;
        win_fill_one<W>(F, FA, C, n, rep[k], tile_rows, lam, tr);
        for (int j = 0; j < W; ++j) {
            tab.F[k][j] = T(F[j]);
            tab.FA[k][j] = T(FA[j]);
            tab.C[k][j] = T(C[j]);
        }
        if (occurs[k]) worst = fmax(worst, tr);
    }
    return worst;
}

// Tables of the split y window solve (see WinSplit) for a line of n nodes in
// 32-row tiles, from the window factors in double; returns the largest
// truncation factor over the kinds that occur (as win_fill).
inline double winsplit_fill(WinSplit &ys, int n, double lam) {
    constexpr int W = WA_W, H = WIN_H, Y = WA_YT;
    const int ntile = n / Y;
    const int rep[4] = {0, ntile >= 3 ? 1 : 0, ntile - 1, 0};
    const bool occurs[4] = {ntile >= 2, ntile >= 3, ntile >= 2, ntile == 1};
    double worst = 0.0;
    for (int k = 0; k < 4; ++k) {
        double F[W], FA[W], C[W], tr = 0.0;
        win_fill_one<W>(F, FA, C, n, rep[k], Y, lam, tr);
        if (occurs[k]) worst = fmax(worst, tr);
        const bool top = rep[k] > 0, bot = (rep[k] + 1) * Y < n;
        for (int j = 0; j < Y; ++j) {
            ys.F[k][j] = float(F[H + j]);
            ys.FA[k][j] = float(FA[H + j]);
            ys.C[k][j] = float(C[H + j]);
        }
        // x_40 per unit f_39 with the halo below zero
        double f[W], x[W];
        f[H + Y - 1] = 1.0;
        for (int j = H + Y; j < W; ++j) f[j] = FA[j] * f[j - 1];
        double xv = f[W - 1];
        for (int j = W - 2; j >= H + Y; --j) xv = f[j] - C[j] * xv;
        ys.R[k] = float(bot ? xv : 0.0);
        // response of the tile rows to a unit forward value at row 7
        f[H - 1] = 1.0;
        for (int j = H; j < W; ++j) f[j] = FA[j] * f[j - 1];
        x[W - 1] = f[W - 1];
        for (int j = W - 2; j >= H; --j) x[j] = f[j] - C[j] * x[j + 1];
        for (int j = 0; j < Y; ++j) ys.T[k][j] = float(top ? x[H + j] : 0.0);
        // response of the tile rows to a unit x_40
        xv = 1.0;
        for (int j = H + Y - 1; j >= H; --j) {
            xv = -C[j] * xv;
            ys.B[k][j - H] = float(bot ? xv : 0.0);
        }
        // h per value of each row above: F_k prod_{i > k} FA_i up to row 7
        for (int m = 0; m < H; ++m) {
            double w = F[m];
            for (int i = m + 1; i < H; ++i) w *= FA[i];
            ys.Wt[k][m] = float(top ? w : 0.0);
        }
        // b per value of each row below: the window solve of rows 40..47 alone
        for (int m = 0; m < H; ++m) {
            double g[W];
            for (int j = 0; j < W; ++j) g[j] = 0.0;
            for (int j = H + Y; j < W; ++j) {
                const double vj = (j == H + Y + m) ? 1.0 : 0.0;
                g[j] = F[j] * vj + FA[j] * g[j - 1];
            }
            double xb = g[W - 1];
            for (int j = W - 2; j >= H + Y; --j) xb = g[j] - C[j] * xb;
            ys.Wb[k][m] = float(bot ? xb : 0.0);
        }
    }
    return worst;
}

template <typename T>
inline void xtile_fill(XTile<T, ADI_XM> &xt, const AdiStatics<T, ADI_XM> &sx) {
    for (int j = 0; j < ADI_XM; ++j) {
        xt.F[j] = sx.F[j]; xt.G[j] = sx.G[j]; xt.B[j] = sx.B[j];
        xt.SA[j] = sx.SA[j]; xt.SC[j] = sx.SC[j];
    }
    xt.DS0 = sx.DS0;
    xt.DS1 = sx.DS1;
    xt.real_tiles = sx.real_tiles;
}

// Fold factors of the x solve per lane kind, taken from the per-lane tables.
template <typename T>
inline void xfold_fill(XFold<T> &xf, const AdiStatics<T, ADI_XM> &sx) {
    const int rt = sx.real_tiles;
    const int rep[4] = {0, rt > 2 ? 1 : 0, rt - 1, rt < 32 ? rt : 31};
    for (int k = 0; k < 4; ++k) {
        const int g = rep[k];
        xf.fr[k] = sx.FR[g];
        xf.fae[k] = sx.FAE[g];
        xf.fce[k] = sx.FCE[g];
        xf.xas[k] = sx.XAS[g];
        xf.xcs[k] = sx.XCS[g];
    }
}

}  // namespace trid
