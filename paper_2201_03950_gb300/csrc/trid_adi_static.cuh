// trid_adi_static.cuh -- the lane-tile Thomas-PCR solve specialised to the
// constant ADI operator of Section 4.1, with every coefficient-only quantity
// precomputed.
//
// On a line of n nodes (n a multiple of the tile height M = 8) the operator
// is the identity on rows 0 and n-1 and tridiag(-lambda, 1 + 2 lambda,
// -lambda) inside, and the right-hand side is 0 on the two boundary rows.
// Cut into tiles of 8 rows, every tile's modified Thomas pass (Section 3.1)
// then has the same coefficient recurrences: the first tile differs only in
// its start row (identity, d = 0) and the last tile only in its end row.  So
// the per-row multipliers are one table shared by all tiles, and only the
// right-hand side flows through the recurrences:
//   forward   d'_0 = F_0 d_0, d'_1 = F_1 d_1, d'_j = F_j d_j + G_j d'_{j-1}
//   backward  d'_j -= B_j d'_{j+1}                     (j = 5 .. 1)
//   reduced   ds = DS0 d'_0 + DS1 d'_1 (0 on the first tile), de = d'_7
//   substitute x_j = d'_j - SA_j x_s - SC_j x_e        (j = 1 .. 6)
// The reduced system over the G tiles of a line is solved exactly as in
// group_solve (one fold + log2 G PCR rounds), its coefficient updates again
// precomputed per lane position:
//   fold      rd = FR de - FAE ds - FCE ds_next
//   round k   rd = PR_k rd - PA_k rd_{g-s} - PC_k rd_{g+s}
//   x_s       = ds - XAS x_e,prev - XCS x_e.
// The tables are computed once per call in double precision (adi_static_fill)
// and passed to the kernels as a grid constant.
#pragma once
#include "trid_device.cuh"

namespace trid {

constexpr int AS_ROUNDS = 5; // PCR rounds for up to 32 tiles

template <typename T, int AS_M>
struct AdiStatics {
    T F[AS_M], G[AS_M], B[AS_M], SA[AS_M], SC[AS_M];
    T DS0, DS1;
    T FR[32], FAE[32], FCE[32];
    T PR[AS_ROUNDS][32], PA[AS_ROUNDS][32], PC[AS_ROUNDS][32];
    T XAS[32], XCS[32];
    int ntiles;      // G = tiles per line (power of two <= 32)
    int real_tiles;  // n / 8; tiles beyond are zero padding
    int rounds;      // PCR rounds executed (see adi_static_fill)
};

// Host: fill the tables for a line of n nodes (n % M == 0, M <= n <= 32 M).
// If red4 is given it receives the interior tiles' reduced-row coefficients
// (as, cs of the start row; ae, ce of the end row) in double precision.
template <typename T, int AS_M>
inline bool adi_static_fill(AdiStatics<T, AS_M> &s, int n, double lam, double *red4 = nullptr) {
    if (n % AS_M != 0 || n < AS_M || n > 32 * AS_M) return false;
    int Gt = 1;
    while (Gt * AS_M < n) Gt <<= 1;
    const int real_tiles = n / AS_M;
    s.ntiles = Gt;
    s.real_tiles = real_tiles;
    const double a = -lam, b = 1.0 + 2.0 * lam, c = -lam;
    // interior tile: rows 0..7 all interior
    double ah[AS_M], ch[AS_M], F[AS_M], G[AS_M], B[AS_M];
    F[0] = 1.0 / b; G[0] = 0.0;
    const double a0 = a * F[0], c0 = c * F[0];
    F[1] = 1.0 / b; G[1] = 0.0;
    ah[1] = a * F[1]; ch[1] = c * F[1];
    for (int j = 2; j < AS_M; ++j) {
        const double r = 1.0 / (b - a * ch[j - 1]);
        F[j] = r;
        G[j] = -r * a;
        ah[j] = -r * a * ah[j - 1];
        ch[j] = r * c;
    }
    for (int j = 0; j < AS_M; ++j) B[j] = 0.0;
    for (int j = AS_M - 3; j >= 1; --j) {
        B[j] = ch[j];
        ah[j] = ah[j] - ch[j] * ah[j + 1];
        ch[j] = -(ch[j] * ch[j + 1]);
    }
    const double rb = 1.0 / (1.0 - c0 * ah[1]);
    const double as_in = a0 * rb, cs_in = -(c0 * ch[1]) * rb;
    const double ae_in = ah[AS_M - 1], ce_in = ch[AS_M - 1];
    if (red4) {
        red4[0] = as_in; red4[1] = cs_in; red4[2] = ae_in; red4[3] = ce_in;
    }
    for (int j = 0; j < AS_M; ++j) {
        s.F[j] = T(F[j]); s.G[j] = T(G[j]); s.B[j] = T(B[j]);
        s.SA[j] = T(j >= 1 && j <= AS_M - 2 ? ah[j] : 0.0);
        s.SC[j] = T(j >= 1 && j <= AS_M - 2 ? ch[j] : 0.0);
    }
    s.DS0 = T(rb);
    s.DS1 = T(-c0 * rb);
    // reduced rows per tile position (tiles >= real_tiles are padding: zero rows)
    double as_g[32], cs_g[32], ae_g[32], ce_g[32];
    for (int g = 0; g < 32; ++g) {
        const bool real = g < real_tiles;
        as_g[g] = (real && g > 0) ? as_in : 0.0;
        cs_g[g] = (real && g > 0) ? cs_in : 0.0;
        ae_g[g] = (real && g < real_tiles - 1) ? ae_in : 0.0;
        ce_g[g] = (real && g < real_tiles - 1) ? ce_in : 0.0;
    }
    double ra[32], rc[32];
    for (int g = 0; g < 32; ++g) {
        const double nas = (g + 1 < Gt) ? as_g[g + 1] : 0.0;
        const double ncs = (g + 1 < Gt) ? cs_g[g + 1] : 0.0;
        const double fr = 1.0 / (1.0 - ae_g[g] * cs_g[g] - ce_g[g] * nas);
        ra[g] = -(ae_g[g] * as_g[g]) * fr;
        rc[g] = -(ce_g[g] * ncs) * fr;
        s.FR[g] = T(fr);
        s.FAE[g] = T(fr * ae_g[g]);
        s.FCE[g] = T(fr * ce_g[g]);
        s.XAS[g] = T(as_g[g]);
        s.XCS[g] = T(cs_g[g]);
    }
    // A PCR round whose coupling coefficients are all below 2^-(p+4) (p the
    // significand bits of T) changes no result by more than 1/16 ulp; for a
    // diagonally dominant constant operator the coupling falls geometrically
    // from round to round (each round squares it), so the rounds from the
    // first such one on are not executed.
    const double negligible = sizeof(T) == 4 ? 1.0 / double(1 << 28) : 1.0 / 144115188075855872.0;
    s.rounds = AS_ROUNDS;
    for (int k = 0; k < AS_ROUNDS; ++k) {
        const int st = 1 << k;
        double na[32], nc[32];
        double coup = 0.0;
        for (int g = 0; g < 32; ++g) {
            if (st >= Gt) {  // unused round: identity
                s.PR[k][g] = T(1); s.PA[k][g] = T(0); s.PC[k][g] = T(0);
                na[g] = ra[g]; nc[g] = rc[g];
                continue;
            }
            const double cm = (g - st >= 0) ? rc[g - st] : 0.0, am = (g - st >= 0) ? ra[g - st] : 0.0;
            const double ap = (g + st < Gt) ? ra[g + st] : 0.0, cp = (g + st < Gt) ? rc[g + st] : 0.0;
            const double r = 1.0 / (1.0 - ra[g] * cm - rc[g] * ap);
            s.PR[k][g] = T(r);
            s.PA[k][g] = T(r * ra[g]);
            s.PC[k][g] = T(r * rc[g]);
            coup = fmax(coup, fmax(fabs(r * ra[g]), fabs(r * rc[g])));
            coup = fmax(coup, fabs(r - 1.0));
            na[g] = -r * (ra[g] * am);
            nc[g] = -r * (rc[g] * cp);
        }
        for (int g = 0; g < 32; ++g) { ra[g] = na[g]; rc[g] = nc[g]; }
        if (s.rounds == AS_ROUNDS && st < Gt && coup < negligible) s.rounds = k;
    }
    return true;
}

// Per-lane reduced-solve factors.  Blocks stage them in shared memory once
// (stage_lane_statics: a per-lane index into kernel parameters would be a
// divergent constant-cache access) and every thread then keeps its own set in
// registers.
constexpr int AS_NLANE = 5 + 3 * AS_ROUNDS;

template <typename T>
struct LaneStatics {
    T fr, fae, fce, xas, xcs;
    T pr[AS_ROUNDS], pa[AS_ROUNDS], pc[AS_ROUNDS];
    __device__ __forceinline__ void load(const T (*tab)[32], int g) {
        fr = tab[0][g]; fae = tab[1][g]; fce = tab[2][g]; xas = tab[3][g]; xcs = tab[4][g];
#pragma unroll
        for (int k = 0; k < AS_ROUNDS; ++k) {
            pr[k] = tab[5 + 3 * k][g];
            pa[k] = tab[6 + 3 * k][g];
            pc[k] = tab[7 + 3 * k][g];
        }
    }
};

template <typename T, int AS_M>
__device__ __forceinline__ void stage_lane_statics(const AdiStatics<T, AS_M> &st, T (*tab)[32],
                                                   int tid, int nthreads) {
    for (int q = tid; q < AS_NLANE * 32; q += nthreads) {
        const int e = q / 32, g = q % 32;
        T v;
        if (e == 0) v = st.FR[g];
        else if (e == 1) v = st.FAE[g];
        else if (e == 2) v = st.FCE[g];
        else if (e == 3) v = st.XAS[g];
        else if (e == 4) v = st.XCS[g];
        else {
            const int k = (e - 5) / 3, m = (e - 5) % 3;
            v = (m == 0) ? st.PR[k][g] : (m == 1) ? st.PA[k][g] : st.PC[k][g];
        }
        tab[e][g] = v;
    }
}

// Tile pass on the right-hand side only: d (8 rows) -> hatted d, returns the
// dynamic parts ds, de of the tile's reduced rows.
template <typename T, int AS_M, typename S>
__device__ __forceinline__ void static_tile_reduce(const S &s, T (&d)[AS_M],
                                                   bool first, bool last, T &ds, T &de) {
    d[0] = s.F[0] * d[0];
    d[1] = s.F[1] * d[1];
#pragma unroll
    for (int j = 2; j < AS_M; ++j) d[j] = fma(s.G[j], d[j - 1], s.F[j] * d[j]);
    if (last) d[AS_M - 1] = T(0);  // identity end row with zero right-hand side
#pragma unroll
    for (int j = AS_M - 3; j >= 1; --j) d[j] = fma(-s.B[j], d[j + 1], d[j]);
    ds = first ? T(0) : fma(s.DS1, d[1], s.DS0 * d[0]);
    de = d[AS_M - 1];
}

template <typename T, int AS_M, typename S>
__device__ __forceinline__ void static_tile_substitute(const S &s, T (&d)[AS_M],
                                                       T xs, T xe) {
#pragma unroll
    for (int j = 1; j < AS_M - 1; ++j) d[j] = fma(-s.SC[j], xe, fma(-s.SA[j], xs, d[j]));
    d[0] = xs;
    d[AS_M - 1] = xe;
}

// Reduced solve over G consecutive lanes with precomputed factors; every lane
// of the warp must call it.
template <typename T, int G>
__device__ __forceinline__ void static_group_solve(const LaneStatics<T> &L, T ds, T de, int g,
                                                   T &xs, T &xe, int rounds = AS_ROUNDS) {
    constexpr unsigned FULL = 0xffffffffu;
    T nds = __shfl_down_sync(FULL, ds, 1, G);
    if (g + 1 >= G) nds = T(0);
    T rd = fma(-L.fce, nds, fma(-L.fae, ds, L.fr * de));
#pragma unroll
    for (int k = 0; k < AS_ROUNDS; ++k) {
        const int st = 1 << k;
        if (st >= G || k >= rounds) break;
        T dm = __shfl_up_sync(FULL, rd, st, G);
        T dp = __shfl_down_sync(FULL, rd, st, G);
        if (g < st) dm = T(0);
        if (g + st >= G) dp = T(0);
        rd = fma(-L.pc[k], dp, fma(-L.pa[k], dm, L.pr[k] * rd));
    }
    xe = rd;
    T xprev = __shfl_up_sync(FULL, xe, 1, G);
    if (g == 0) xprev = T(0);
    xs = fma(-L.xcs, xe, fma(-L.xas, xprev, ds));
}

// As static_group_solve, reading the per-lane factors from the staged table
// (lane g reads column g: conflict-free) instead of holding them in registers.
template <typename T, int G>
__device__ __forceinline__ void static_group_solve_tab(const T (*tab)[32], T ds, T de, int g,
                                                       T &xs, T &xe, int rounds = AS_ROUNDS) {
    constexpr unsigned FULL = 0xffffffffu;
    T nds = __shfl_down_sync(FULL, ds, 1, G);
    if (g + 1 >= G) nds = T(0);
    T rd = fma(-tab[2][g], nds, fma(-tab[1][g], ds, tab[0][g] * de));
#pragma unroll
    for (int k = 0; k < AS_ROUNDS; ++k) {
        const int st = 1 << k;
        if (st >= G || k >= rounds) break;
        T dm = __shfl_up_sync(FULL, rd, st, G);
        T dp = __shfl_down_sync(FULL, rd, st, G);
        if (g < st) dm = T(0);
        if (g + st >= G) dp = T(0);
        rd = fma(-tab[7 + 3 * k][g], dp, fma(-tab[6 + 3 * k][g], dm, tab[5 + 3 * k][g] * rd));
    }
    xe = rd;
    T xprev = __shfl_up_sync(FULL, xe, 1, G);
    if (g == 0) xprev = T(0);
    xs = fma(-tab[4][g], xe, fma(-tab[3][g], xprev, ds));
}

}  // namespace trid

#include "trid_tma.cuh"
#include "trid_internal.h"

namespace trid {

constexpr int ADI_XM = 8;   // tile height of the x solve (lane tiles of a warp)
constexpr int ADI_YM = 16;  // tile height of the y / z solves

// Load one line tile of M values (vector path when the whole tile is inside).
template <typename T, int M>
__device__ __forceinline__ void load_line_tile(const T *__restrict__ p, int x0, int nx, bool act,
                                               T (&r)[M]) {
    if (act && x0 + M <= nx) {
        load_contig_vec<T, M>(p + x0, r);
    } else {
#pragma unroll
        for (int j = 0; j < M; ++j) r[j] = (act && x0 + j < nx) ? p[x0 + j] : T(0);
    }
}

// ---------------------------------------------------------------------------
// RHS stencil + x solve.  A group of G lanes owns a line, lane g holding x in
// [8g, 8g + 8).  With G = 32 each warp walks LPW consecutive lines of one
// plane and keeps a sliding window of u(y - 1), u(y), u(y + 1), so per line
// it loads one new in-plane line and the two z neighbours.  The per-lane
// reduced-solve factors are staged in shared memory once per block.
// ---------------------------------------------------------------------------
template <typename T, int G, int LPW>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 3 : 1)
k_adi_x_static(const T *__restrict__ u, T *__restrict__ w, int nx, int ny, int nz, int ndim, T lam,
               const __grid_constant__ AdiStatics<T, ADI_XM> st) {
    constexpr int M = ADI_XM;
    __shared__ T lane_tab[AS_NLANE][32];
    stage_lane_statics<T>(st, lane_tab, threadIdx.x, blockDim.x);
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int g = lane % G;
    LaneStatics<T> L;
    L.load(lane_tab, g);
    const bool first = (g == 0);
    const bool last = (g == st.real_tiles - 1);
    const int x0 = g * M;
    const int z = int(blockIdx.y);
    const bool zin = (ndim == 2) || (z > 0 && z < nz - 1);
    const int64_t plane = int64_t(nx) * ny;
    const T *uz = u + int64_t(z) * plane;
    T *wz = w + int64_t(z) * plane;
    constexpr int GPW = 32 / G;  // lines per warp pass
    const int warp_global = int((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const T centre = T(2 * ndim);
    constexpr unsigned FULLM = 0xffffffffu;
    const int ybase = warp_global * LPW * GPW;

    T prev[M], cur[M];
    if constexpr (G == 32) {
        load_line_tile<T, M>(uz + int64_t(ybase - 1) * nx, x0, nx, ybase >= 1 && ybase - 1 < ny, prev);
        load_line_tile<T, M>(uz + int64_t(ybase) * nx, x0, nx, ybase < ny, cur);
    }
    for (int pass = 0; pass < LPW; ++pass) {
        const int y = ybase + pass * GPW + lane / G;
        const bool act = y < ny;
        const bool interior = act && zin && y > 0 && y < ny - 1;
        const bool zok = interior && ndim == 3;
        T uc[M], ym[M], yp[M], zm[M], zp[M];
        if constexpr (G == 32) {
#pragma unroll
            for (int j = 0; j < M; ++j) { uc[j] = cur[j]; ym[j] = prev[j]; }
            load_line_tile<T, M>(uz + int64_t(y + 1) * nx, x0, nx, y + 1 < ny, yp);
        } else {
            load_line_tile<T, M>(uz + int64_t(y) * nx, x0, nx, act, uc);
            load_line_tile<T, M>(uz + int64_t(y - 1) * nx, x0, nx, interior, ym);
            load_line_tile<T, M>(uz + int64_t(y + 1) * nx, x0, nx, interior, yp);
        }
        load_line_tile<T, M>(uz - plane + int64_t(y) * nx, x0, nx, zok, zm);
        load_line_tile<T, M>(uz + plane + int64_t(y) * nx, x0, nx, zok, zp);
        const T left = __shfl_up_sync(FULLM, uc[M - 1], 1, G);
        const T right = __shfl_down_sync(FULLM, uc[0], 1, G);
        T d[M];
#pragma unroll
        for (int j = 0; j < M; ++j) {
            const int i = x0 + j;
            const T xm = (j == 0) ? left : uc[j - 1];
            const T xp = (j == M - 1) ? right : uc[j + 1];
            const T sum = (xm + xp) + (ym[j] + yp[j]) + (zm[j] + zp[j]);
            d[j] = (interior && i > 0 && i < nx - 1) ? lam * (sum - centre * uc[j]) : T(0);
        }
        if constexpr (G == 32) {
#pragma unroll
            for (int j = 0; j < M; ++j) { prev[j] = uc[j]; cur[j] = yp[j]; }
        }
        T ds, de, xs, xe;
        static_tile_reduce<T, M>(st, d, first, last, ds, de);
        static_group_solve<T, G>(L, ds, de, g, xs, xe, st.rounds);
        static_tile_substitute<T, M>(st, d, xs, xe);
        if (act) {
            if (x0 + M <= nx) {
                store_contig_vec<T, M>(wz + int64_t(y) * nx + x0, d);
            } else {
#pragma unroll
                for (int j = 0; j < M; ++j)
                    if (x0 + j < nx) wz[int64_t(y) * nx + x0 + j] = d[j];
            }
        }
    }
}

// ---------------------------------------------------------------------------
// y or z solve (optionally u += result), TMA-fed: one producer warp streams
// [SG lines x n rows] boxes of d (and u) into a ring of shared-memory stages;
// NT*SG = 256 consumer threads (tile of 16 rows, line) run the static tile
// pass, exchange the two dynamic reduced values through shared memory, solve
// the reduced systems with the per-lane factors and substitute.  Small blocks
// (288 threads) so that three share an SM and one block's barrier phase
// overlaps the others' streaming.
// ---------------------------------------------------------------------------
template <typename T, int NT, int SG, bool ACC>
__global__ void __launch_bounds__(NT * SG + 32, sizeof(T) == 4 ? 3 : 1)
k_adi_strided_static(const __grid_constant__ TmaSet maps,
                     const __grid_constant__ AdiStatics<T, ADI_YM> st, T *out, Lines L,
                     int64_t nbatch, int stages, int *status) {
    constexpr int M = ADI_YM;
    constexpr int P = SG + 1;
    constexpr int NCONS = NT * SG;
    static_assert(NCONS % 32 == 0, "consumers must be whole warps");
    constexpr int NSLOT = ACC ? 2 : 1;
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ int abort_flag;
    __shared__ T lane_tab[AS_NLANE][32];
    const int n = int(L.n);
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
    const int64_t nxc = (L.inner + SG - 1) / SG;

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
                const int x0 = int((bt % nxc) * SG);
                const int o = int(bt / nxc);
                unsigned char *dst = smem + s * stage_bytes;
                tma_load_3d(dst, &maps.map[0], x0, 0, o, &full[s]);
                if (ACC) tma_load_3d(dst + slot_bytes, &maps.map[1], x0, 0, o, &full[s]);
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
    const int rs = tid / NT, rt = tid % NT;
    const int q = rt * P + rs;
    LaneStatics<T> LS;
    LS.load(lane_tab, rt);
    const int stride = int(L.stride);
    int k = 0;
    for (int64_t bt = blockIdx.x; bt < nbatch; bt += gridDim.x, ++k) {
        const int s = k % stages;
        bool ok = false;
        if (!*(volatile int *)&abort_flag) {
            ok = mbar_wait(&full[s], uint32_t(k / stages) & 1u, status);
            if (!ok) *(volatile int *)&abort_flag = 1;
        }
        const T *sd = reinterpret_cast<const T *>(smem + s * stage_bytes);
        const T *su = reinterpret_cast<const T *>(smem + s * stage_bytes + slot_bytes);
        const int64_t x = (bt % nxc) * SG + sl;
        const int64_t o = bt / nxc;
        const bool active = ok && x < L.inner;
        T d[M], uu[M];
#pragma unroll
        for (int j = 0; j < M; ++j) {
            const int i = i0 + j;
            const bool in = active && i < n;
            d[j] = in ? sd[i * SG + sl] : T(0);
            if (ACC) uu[j] = in ? su[i * SG + sl] : T(0);
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[s]);
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
        if (active) {
            T *ob = out + (x + o * L.inner * L.n);
#pragma unroll
            for (int j = 0; j < M; ++j)
                if (i0 + j < n) ob[(i0 + j) * stride] = ACC ? d[j] + uu[j] : d[j];
        }
    }
}

}  // namespace trid
