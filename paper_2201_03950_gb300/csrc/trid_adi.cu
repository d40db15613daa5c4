// trid_adi.cu -- ADI heat-diffusion step (arXiv 2201.03950, Section 4.1,
// Algorithm "adi") with the coefficients generated inside the kernels.
//
// One step, delta form, Dirichlet boundary (boundary nodes never change):
//   d = lambda * (sum of axis neighbours - 2*ndim*u)   (interior; 0 on boundary)
//   d <- X^{-1} d ; d <- Y^{-1} d ; [d <- Z^{-1} d] ; u <- u + d
// with X, Y, Z = tridiag(-lambda, 1 + 2 lambda, -lambda) on interior rows and
// identity rows at the boundary nodes.
//
// Schedules of a 3D step, tried in this order:
//   windowed (trid_adi_window.cuh, FP32, when the operator's inverse decays
//     below 1/16 ulp within 8 rows): k_adi_xyw (stencil + x solve + windowed
//     y solve per plane cluster, writes e = Z u + Y^{-1} X^{-1} d) and k_adi_zw
//     (windowed z solve, u = Z^{-1} e); 4 mesh words per point.
//   two-pass (trid_adi_2pass.cuh, extents multiples of 16): k_adi_xy and
//     k_adi_z_ysub, the y solve split by the Section 3.1 tiling across them.
//   general (any extents <= 256): stencil + x solve (k_adi_x_static or
//     k_adi_x_rhs), then y and z solves (k_adi_strided_static / k_strided),
//     the last one accumulating into u.
// 2D steps use the general schedule without z.
#include "trid_device.cuh"
#include "trid_strided.cuh"
#include "trid_adi_static.cuh"
#include "trid_adi_2pass.cuh"
#include "trid_adi_window.cuh"
#include "../../include/trid.h"
#include "trid_internal.h"

#include <type_traits>

namespace trid {

constexpr int ADI_M = 8;
constexpr int ADI_MAX_N = 32 * ADI_M;

static int pow2_at_least(int64_t v) {
    int p = 1;
    while (p < v) p <<= 1;
    return p;
}

template <typename T, int M>
__device__ __forceinline__ void adi_load_tile(const T *__restrict__ p, int64_t i0, int64_t n,
                                              bool vec, T (&r)[M]) {
    if (vec && i0 + M <= n) {
        load_contig_vec<T, M>(p + i0, r);
    } else {
#pragma unroll
        for (int j = 0; j < M; ++j) r[j] = (i0 + j < n) ? p[i0 + j] : T(0);
    }
}

// RHS stencil fused with the x solve.  Lines along x are contiguous; G lanes
// of a warp share a line, lane g owning x in [g*M, g*M + M).
template <typename T, int M, int G>
__global__ void __launch_bounds__(256)
k_adi_x_rhs(const T *__restrict__ u, T *__restrict__ w, int64_t nx, int64_t ny, int64_t nz,
            int ndim, T lam, int vec_ok) {
    // grid: x over groups of lines of one plane, y over planes (no division)
    const int lane = threadIdx.x & 31;
    const int g = lane % G;
    const int y = int((blockIdx.x * blockDim.x + threadIdx.x) >> 5) * (32 / G) + lane / G;
    const int z = int(blockIdx.y);
    const bool active = y < ny;
    const bool interior = active && y > 0 && y < ny - 1 && (ndim == 2 || (z > 0 && z < nz - 1));
    const int64_t base = (int64_t(z) * ny + y) * nx;
    const int64_t i0 = int64_t(g) * M;
    const bool vec = vec_ok != 0;

    T uc[M];
    if (active) adi_load_tile<T, M>(u + base, i0, nx, vec, uc);
    else {
#pragma unroll
        for (int j = 0; j < M; ++j) uc[j] = T(0);
    }
    constexpr unsigned FULL = 0xffffffffu;
    const T left = __shfl_up_sync(FULL, uc[M - 1], 1, G);
    const T right = __shfl_down_sync(FULL, uc[0], 1, G);

    T ra[M], rb[M], rc[M], rd[M];
#pragma unroll
    for (int j = 0; j < M; ++j) {
        const int64_t i = i0 + j;
        const bool in_x = i > 0 && i < nx - 1;
        ra[j] = in_x ? -lam : T(0);
        rb[j] = (i < nx && in_x) ? T(1) + T(2) * lam : T(1);
        rc[j] = in_x ? -lam : T(0);
        rd[j] = T(0);
    }
    if (interior) {
        T s[M];
#pragma unroll
        for (int j = 0; j < M; ++j) {
            const T xm = (j == 0) ? left : uc[j - 1];
            const T xp = (j == M - 1) ? right : uc[j + 1];
            s[j] = xm + xp;
        }
        T nb[M];
        adi_load_tile<T, M>(u + base - nx, i0, nx, vec, nb);
#pragma unroll
        for (int j = 0; j < M; ++j) s[j] += nb[j];
        adi_load_tile<T, M>(u + base + nx, i0, nx, vec, nb);
#pragma unroll
        for (int j = 0; j < M; ++j) s[j] += nb[j];
        if (ndim == 3) {
            adi_load_tile<T, M>(u + base - nx * ny, i0, nx, vec, nb);
#pragma unroll
            for (int j = 0; j < M; ++j) s[j] += nb[j];
            adi_load_tile<T, M>(u + base + nx * ny, i0, nx, vec, nb);
#pragma unroll
            for (int j = 0; j < M; ++j) s[j] += nb[j];
        }
        const T centre = T(2 * ndim);
#pragma unroll
        for (int j = 0; j < M; ++j) {
            const int64_t i = i0 + j;
            rd[j] = (i > 0 && i < nx - 1) ? lam * (s[j] - centre * uc[j]) : T(0);
        }
    }
    T as, cs, ds, ae, ce, de, xs, xe;
    tile_reduce<T, M>(ra, rb, rc, rd, as, cs, ds, ae, ce, de);
    group_solve<T, G>(as, cs, ds, ae, ce, de, g, xs, xe);
    tile_substitute<T, M>(ra, rc, rd, xs, xe);
    if (!active) return;
    if (vec && i0 + M <= nx) {
        store_contig_vec<T, M>(w + base + i0, rd);
    } else {
#pragma unroll
        for (int j = 0; j < M; ++j)
            if (i0 + j < nx) w[base + i0 + j] = rd[j];
    }
}


template <typename T, int G>
static void launch_x_rhs(const T *u, T *w, const int64_t *n3, int ndim, T lam, int vec,
                         cudaStream_t st) {
    const int64_t warps = (n3[1] + (32 / G) - 1) / (32 / G);  // per plane
    const int64_t blocks = (warps + 7) / 8;
    k_adi_x_rhs<T, ADI_M, G><<<dim3(unsigned(blocks), unsigned(n3[2])), 256, 0, st>>>(
        u, w, n3[0], n3[1], n3[2], ndim, lam, vec);
}

template <typename T, int NT>
static void launch_adi_strided(T lam, const T *d, T *out, int acc, const Lines &L,
                               cudaStream_t st) {
    // at least one full warp per block: the reduced solve shuffles over all 32 lanes
    constexpr int SG = (NT * SysCfg<T>::SG < 32) ? 32 / NT : SysCfg<T>::SG;
    AdiCoef<T> coef{lam};
    if constexpr (std::is_same<T, float>::value) {
        const void *arrs[2] = {d, out};
        const bool ok = acc ? launch_strided_tma<T, ADI_M, NT, 16, true>(arrs, coef, out, L, st)
                            : launch_strided_tma<T, ADI_M, NT, 16, false>(arrs, coef, out, L, st);
        if (ok) return;
    }
    if (acc)
        k_strided<T, ADI_M, NT, SG, true, AdiCoef<T>>
            <<<strided_grid(L, SG), NT * SG, 0, st>>>(coef, d, out, L, L.nsys / L.inner);
    else
        k_strided<T, ADI_M, NT, SG, false, AdiCoef<T>>
            <<<strided_grid(L, SG), NT * SG, 0, st>>>(coef, d, out, L, L.nsys / L.inner);
}

// ---- kernels specialised to the constant operator (axis length % 8 == 0)
template <typename T, int G>
static bool launch_x_static_g(const T *u, T *w, const int64_t *n3, int ndim, T lam,
                              const AdiStatics<T, ADI_XM> &st, cudaStream_t st_) {
    constexpr int LPW = 4;            // line passes per warp
    constexpr int GPW = 32 / G;       // lines per warp pass
    const int64_t lines_per_block = int64_t(8) * GPW * LPW;
    const int64_t gx = (n3[1] + lines_per_block - 1) / lines_per_block;
    k_adi_x_static<T, G, LPW><<<dim3(unsigned(gx), unsigned(n3[2])), 256, 0, st_>>>(
        u, w, int(n3[0]), int(n3[1]), int(n3[2]), ndim, lam, st);
    return cudaGetLastError() == cudaSuccess;
}

template <typename T>
static bool launch_x_static(const T *u, T *w, const int64_t *n3, int ndim, T lam,
                            cudaStream_t st_) {
    AdiStatics<T, ADI_XM> st;
    if (!adi_static_fill<T, ADI_XM>(st, int(n3[0]), double(lam))) return false;
    if (!is_aligned16(u) || !is_aligned16(w) || (n3[0] * int64_t(sizeof(T))) % 16 != 0)
        return false;
    switch (st.ntiles) {
        case 1: return launch_x_static_g<T, 1>(u, w, n3, ndim, lam, st, st_);
        case 2: return launch_x_static_g<T, 2>(u, w, n3, ndim, lam, st, st_);
        case 4: return launch_x_static_g<T, 4>(u, w, n3, ndim, lam, st, st_);
        case 8: return launch_x_static_g<T, 8>(u, w, n3, ndim, lam, st, st_);
        case 16: return launch_x_static_g<T, 16>(u, w, n3, ndim, lam, st, st_);
        default: return launch_x_static_g<T, 32>(u, w, n3, ndim, lam, st, st_);
    }
}

template <typename T, int NT, bool ACC>
static bool launch_strided_static_nt(const T *d, T *out, const Lines &L,
                                     const AdiStatics<T, ADI_YM> &st, cudaStream_t st_) {
    constexpr int SG = 16;
    if constexpr ((NT * SG) % 32 != 0) {
        return false;
    } else {
        const DeviceInfo *di = device_info();
        if (!di || L.inner < 1) return false;
        const int64_t outer = L.nsys / L.inner;
        TmaSet maps;
        if (!encode_lines_map(&maps.map[0], d, int(sizeof(T)), L.inner, L.n, outer, SG))
            return false;
        if (ACC && !encode_lines_map(&maps.map[1], out, int(sizeof(T)), L.inner, L.n, outer, SG))
            return false;
        const size_t slot = (size_t(L.n) * SG * sizeof(T) + 127) / 128 * 128;
        const size_t stage = (ACC ? 2 : 1) * slot;
        const size_t fixed = (4 * NT * (SG + 1) * sizeof(T) + 127) / 128 * 128;
        auto bytes = [&](int stages) { return size_t(stages) * (stage + 16) + fixed; };
        // three blocks per SM when possible, as many stages (<= 4) as then fit
        const size_t cap2 = size_t(di->smem_per_sm) / 3 - 1024 - 1024;
        size_t cap = cap2 < size_t(di->max_smem_optin) - 256 ? cap2 : size_t(di->max_smem_optin) - 256;
        int stages = 4;
        while (stages > 1 && bytes(stages) > cap) --stages;
        if (bytes(stages) > cap) {
            cap = size_t(di->max_smem_optin) - 256;
            stages = 4;
            while (stages > 1 && bytes(stages) > cap) --stages;
            if (bytes(stages) > cap) return false;
        }
        const size_t smem = bytes(stages);
        auto kern = k_adi_strided_static<T, NT, SG, ACC>;
        const int per_sm =
            kernel_blocks_per_sm(reinterpret_cast<const void *>(kern), NT * SG + 32, smem);
        if (per_sm < 1) return false;
        const int64_t nbatch = (L.inner + SG - 1) / SG * outer;
        const int64_t slots = int64_t(di->sm_count) * per_sm;
        const int64_t grid = nbatch < slots ? nbatch : slots;
        kern<<<dim3(unsigned(grid)), NT * SG + 32, smem, st_>>>(maps, st, out, L, nbatch, stages,
                                                               device_status_word());
        return cudaGetLastError() == cudaSuccess;
    }
}

template <typename T, bool ACC>
static bool launch_strided_static(T lam, const T *d, T *out, const Lines &L, cudaStream_t st_) {
    AdiStatics<T, ADI_YM> st;
    if (!adi_static_fill<T, ADI_YM>(st, int(L.n), double(lam))) return false;
    if (!strided_offsets_fit(L)) return false;
    switch (st.ntiles) {
        case 1: return launch_strided_static_nt<T, 1, ACC>(d, out, L, st, st_);
        case 2: return launch_strided_static_nt<T, 2, ACC>(d, out, L, st, st_);
        case 4: return launch_strided_static_nt<T, 4, ACC>(d, out, L, st, st_);
        case 8: return launch_strided_static_nt<T, 8, ACC>(d, out, L, st, st_);
        case 16: return launch_strided_static_nt<T, 16, ACC>(d, out, L, st, st_);
        case 32: return launch_strided_static_nt<T, 32, ACC>(d, out, L, st, st_);
        default: return false;
    }
}

template <typename T>
static void adi_strided(T lam, const T *d, T *out, int acc, const Lines &L, cudaStream_t st) {
    if (acc ? launch_strided_static<T, true>(lam, d, out, L, st)
            : launch_strided_static<T, false>(lam, d, out, L, st))
        return;
    switch (pow2_at_least((L.n + ADI_M - 1) / ADI_M)) {
        case 1: launch_adi_strided<T, 1>(lam, d, out, acc, L, st); break;
        case 2: launch_adi_strided<T, 2>(lam, d, out, acc, L, st); break;
        case 4: launch_adi_strided<T, 4>(lam, d, out, acc, L, st); break;
        case 8: launch_adi_strided<T, 8>(lam, d, out, acc, L, st); break;
        case 16: launch_adi_strided<T, 16>(lam, d, out, acc, L, st); break;
        default: launch_adi_strided<T, 32>(lam, d, out, acc, L, st); break;
    }
}

// ---------------------------------------------------------------------------
// Two-pass 3D schedule (trid_adi_2pass.cuh).  Workspace: e (mesh-sized), the
// reduced y arrays rs / re ([z][tile][x]) and one counter per plane.
// ---------------------------------------------------------------------------
struct Adi2Layout {
    size_t e, red, cnt, tab, total;
};

static Adi2Layout adi2_layout(const int64_t *n3, size_t esz, int64_t nb = 1) {
    auto up = [](size_t v) { return (v + 255) / 256 * 256; };
    Adi2Layout l;
    l.e = up(size_t(n3[0] * n3[1] * n3[2]) * esz * size_t(nb));
    l.red = up(size_t(n3[0] * ((n3[1] + ADI_YM - 1) / ADI_YM) * n3[2]) * esz * size_t(nb));
    l.cnt = up(size_t(n3[2]) * sizeof(unsigned) * size_t(nb));
    l.tab = up(size_t(AS_NLANE) * 32 * esz);
    l.total = l.e + 2 * l.red + l.cnt + l.tab;
    return l;
}

static bool adi2_eligible(const int64_t *n3, int ndim) {
    if (ndim != 3) return false;
    for (int k = 0; k < 3; ++k)
        if (n3[k] % 16 != 0 || n3[k] < 16 || n3[k] > ADI_MAX_N) return false;
    if (n3[2] < 32) return false;  // the z pass needs whole warps of consumers
    return true;
}

template <typename T>
static bool adi2_tables(const int64_t *n3, T lam, AdiStatics<T, ADI_XM> &sx,
                        AdiStatics<T, ADI_YM> &sy, AdiStatics<T, ADI_YM> &sz, YReduced<T> &ry,
                        YSubst<T> &ys) {
    double red[4];
    if (!adi_static_fill<T, ADI_XM>(sx, int(n3[0]), double(lam))) return false;
    if (!adi_static_fill<T, ADI_YM>(sy, int(n3[1]), double(lam), red)) return false;
    if (!adi_static_fill<T, ADI_YM>(sz, int(n3[2]), double(lam))) return false;
    // reduced y system: unknowns (s_0, e_0, s_1, e_1, ...); row s_k couples
    // e_{k-1} (as) and e_k (cs), row e_k couples s_k (ae) and s_{k+1} (ce);
    // the first tile's start row and the last tile's end row are identities
    const int nt = int(n3[1] / ADI_YM);
    const int n2 = 2 * nt;
    double sub[32] = {0}, sup[32] = {0};
    for (int k = 0; k < nt; ++k) {
        sub[2 * k] = (k > 0) ? red[0] : 0.0;
        sup[2 * k] = (k > 0) ? red[1] : 0.0;
        sub[2 * k + 1] = (k < nt - 1) ? red[2] : 0.0;
        sup[2 * k + 1] = (k < nt - 1) ? red[3] : 0.0;
    }
    double cst = 0.0;
    for (int i = 0; i < 32; ++i) {
        if (i < n2) {
            const double wv = 1.0 / (1.0 - sub[i] * cst);
            cst = sup[i] * wv;
            ry.sub[i] = T(sub[i]);
            ry.w[i] = T(wv);
            ry.cst[i] = T(cst);
        } else {
            ry.sub[i] = T(0); ry.w[i] = T(1); ry.cst[i] = T(0);
        }
    }
    ry.n2 = n2;
    for (int r = 0; r < ADI_YM; ++r) {
        ys.alpha[r] = (r == 0) ? T(1) : (r == ADI_YM - 1) ? T(0) : -sy.SA[r];
        ys.beta[r] = (r == 0) ? T(0) : (r == ADI_YM - 1) ? T(1) : -sy.SC[r];
    }
    ys.lam = lam;
    return true;
}

template <typename T, int G>
static bool launch_xy(const T *u, T *e, T *rs, T *re, unsigned *cnt, const T *gtab,
                      const int64_t *n3, int64_t nb, T lam, const AdiStatics<T, ADI_XM> &sx,
                      const AdiStatics<T, ADI_YM> &sy, const YReduced<T> &ry, cudaStream_t st) {
    const size_t smem = 2 * size_t(ADI_YM) * size_t(n3[0]) * sizeof(T);
    auto kern = k_adi_xy<T, G>;
    if (kernel_blocks_per_sm(reinterpret_cast<const void *>(kern), 256, smem) < 1) return false;
    if (n3[2] * nb > 65535) return false;
    kern<<<dim3(unsigned(n3[1] / ADI_YM), unsigned(n3[2] * nb)), 256, smem, st>>>(
        u, e, rs, re, cnt, gtab, int(n3[0]), int(n3[1]), int(n3[2]), lam, sx, sy, ry);
    return launch_ok();
}

template <typename T, int NT>
static bool launch_z_ysub(const T *e, const T *rs, const T *re, T *u, const int64_t *n3,
                          int64_t nb, const AdiStatics<T, ADI_YM> &sz, const YSubst<T> &ys,
                          cudaStream_t st) {
    constexpr int SG = 16;
    if constexpr ((NT * SG) % 32 != 0) {
        return false;
    } else {
        const DeviceInfo *di = device_info();
        if (!di) return false;
        const int64_t nplane = n3[0] * n3[1];
        const int64_t nred = n3[0] * (n3[1] / ADI_YM);
        TmaSet maps;
        if (!encode_lines_map(&maps.map[0], e, int(sizeof(T)), nplane, n3[2], nb, SG) ||
            !encode_lines_map(&maps.map[1], rs, int(sizeof(T)), nred, n3[2], nb, SG) ||
            !encode_lines_map(&maps.map[2], re, int(sizeof(T)), nred, n3[2], nb, SG))
            return false;
        const size_t slot = (size_t(n3[2]) * SG * sizeof(T) + 127) / 128 * 128;
        const size_t stage = 3 * slot;
        const size_t fixed = (4 * NT * (SG + 1) * sizeof(T) + 127) / 128 * 128;
        auto bytes = [&](int stages) { return size_t(stages) * (stage + 16) + fixed; };
        const size_t optin = size_t(di->max_smem_optin) - 256;
        // two blocks per SM with two or more stages (<= 4), else fewer blocks
        int stages = 0;
        for (int per = 2; per >= 1 && stages == 0; --per) {
            size_t cap = size_t(di->smem_per_sm) / per - 4096;
            if (cap > optin) cap = optin;
            for (int sg = 4; sg >= 2; --sg)
                if (bytes(sg) <= cap) { stages = sg; break; }
        }
        if (stages == 0) return false;
        const size_t smem = bytes(stages);
        auto kern = k_adi_z_ysub<T, NT, SG>;
        const int per_sm =
            kernel_blocks_per_sm(reinterpret_cast<const void *>(kern), NT * SG + 32, smem);
        if (per_sm < 1) return false;
        const int64_t nbatch = nplane / SG * nb;
        const int64_t slots = int64_t(di->sm_count) * per_sm;
        const int64_t grid = nbatch < slots ? nbatch : slots;
        kern<<<dim3(unsigned(grid)), NT * SG + 32, smem, st>>>(
            maps, sz, ys, u, int(n3[0]), int(nplane), int(n3[2]), nbatch, stages,
            device_status_word());
        return launch_ok();
    }
}

template <typename T>
static trid_status adi_run_2pass(T *u, const int64_t *n3, T lam, int nsteps, char *ws,
                                 cudaStream_t st, int64_t nb = 1) {
    AdiStatics<T, ADI_XM> sx;
    AdiStatics<T, ADI_YM> sy, sz;
    YReduced<T> ry;
    YSubst<T> ys;
    if (!adi2_tables<T>(n3, lam, sx, sy, sz, ry, ys)) return TRID_ERR_UNSUPPORTED;
    const Adi2Layout l = adi2_layout(n3, sizeof(T), nb);
    T *e = reinterpret_cast<T *>(ws);
    T *rs = reinterpret_cast<T *>(ws + l.e);
    T *re = reinterpret_cast<T *>(ws + l.e + l.red);
    unsigned *cnt = reinterpret_cast<unsigned *>(ws + l.e + 2 * l.red);
    T *gtab = reinterpret_cast<T *>(ws + l.e + 2 * l.red + l.cnt);
    k_adi_setup<T><<<1, 256, 0, st>>>(sx, gtab, cnt, int(n3[2] * nb));
    if (!launch_ok()) return TRID_ERR_CUDA;
    for (int step = 0; step < nsteps; ++step) {
        bool ok;
        switch (sx.ntiles) {
            case 2: ok = launch_xy<T, 2>(u, e, rs, re, cnt, gtab, n3, nb, lam, sx, sy, ry, st); break;
            case 4: ok = launch_xy<T, 4>(u, e, rs, re, cnt, gtab, n3, nb, lam, sx, sy, ry, st); break;
            case 8: ok = launch_xy<T, 8>(u, e, rs, re, cnt, gtab, n3, nb, lam, sx, sy, ry, st); break;
            case 16: ok = launch_xy<T, 16>(u, e, rs, re, cnt, gtab, n3, nb, lam, sx, sy, ry, st); break;
            case 32: ok = launch_xy<T, 32>(u, e, rs, re, cnt, gtab, n3, nb, lam, sx, sy, ry, st); break;
            default: ok = false;
        }
        if (!ok) return TRID_ERR_CUDA;
        switch (sz.ntiles) {
            case 1: ok = launch_z_ysub<T, 1>(e, rs, re, u, n3, nb, sz, ys, st); break;
            case 2: ok = launch_z_ysub<T, 2>(e, rs, re, u, n3, nb, sz, ys, st); break;
            case 4: ok = launch_z_ysub<T, 4>(e, rs, re, u, n3, nb, sz, ys, st); break;
            case 8: ok = launch_z_ysub<T, 8>(e, rs, re, u, n3, nb, sz, ys, st); break;
            case 16: ok = launch_z_ysub<T, 16>(e, rs, re, u, n3, nb, sz, ys, st); break;
            default: ok = false;
        }
        if (!ok) return TRID_ERR_CUDA;
    }
    return TRID_OK;
}

// ---------------------------------------------------------------------------
// Windowed 3D schedule (trid_adi_window.cuh): FP32, extents nx % 8 == 0,
// ny % 32 == 0 (one cluster of ny / 32 CTAs per plane, at most 8), nz % 16 ==
// 0, all <= 256, and an operator whose window truncation stays below 1/16 ulp.
// Workspace: e (mesh-sized).
// ---------------------------------------------------------------------------
struct AdiWPlan {
    AdiStatics<float, ADI_XM> sx;
    XTile<float, ADI_XM> xt;
    XFold<float> xf;
    WinSplit ys;
    WinTab<float, WB_W> zw;
    int G;
};

static bool adiw_plan(const int64_t *n3, int64_t nb, double lam, AdiWPlan &p) {
    const int64_t nx = n3[0], ny = n3[1], nz = n3[2];
    if (nx % 8 != 0 || nx < 8 || nx > 256) return false;
    if (ny % WA_YT != 0 || ny < WA_YT || ny > 8 * WA_YT) return false;
    if (nz % WB_ZT != 0 || nz < WB_ZT || nz > 256) return false;
    if (nz * nb > 65535) return false;
    if (!adi_static_fill<float, ADI_XM>(p.sx, int(nx), lam)) return false;
    if (p.sx.rounds != 0) return false;  // the x solve runs the fold alone
    const double negligible = 1.0 / double(1 << 28);
    if (winsplit_fill(p.ys, int(ny), lam) > negligible) return false;
    if (win_fill<float, WB_W>(p.zw, int(nz), WB_ZT, lam) > negligible) return false;
    xfold_fill<float>(p.xf, p.sx);
    xtile_fill<float>(p.xt, p.sx);
    p.G = pow2_at_least((nx + ADI_XM - 1) / ADI_XM);
    return true;
}

// Planes per CTA of pass A: 32 / G (at most 16, dividing the stacked plane
// count) when a plane is one 32-row tile, else 1.
template <int G>
static int xyw_ppc(const int64_t *n3, int64_t nb) {
    if (n3[1] != WA_YT) return 1;
    int ppc = 32 / G < 16 ? 32 / G : 16;
    while (ppc > 1 && (n3[2] * nb) % ppc != 0) ppc /= 2;
    return ppc;
}

template <int G, int NXC = 0, int PPC = 1>
static bool launch_xyw(const float *u, float *e, const int64_t *n3, int64_t nb, float lam,
                       const AdiWPlan &p, cudaStream_t st, bool check_only) {
    const int C = int(n3[1] / WA_YT);
    // X^{-1} d and Z u rows of the CTA's planes, the two received summaries, the mbarrier
    const size_t smem = (2 * size_t(WA_YT) * PPC + 2) * size_t(n3[0]) * sizeof(float) + 16;
    auto kern = k_adi_xyw<G, NXC, PPC>;
    const void *kp = reinterpret_cast<const void *>(kern);
    if (kernel_blocks_per_sm(kp, 256, smem) < 1) return false;
    if (cluster_capacity(kp, C, 256, smem) < 1) return false;
    if (check_only) return true;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = unsigned(C);
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[1].val.programmaticStreamSerializationAllowed = 1;
    cfg.gridDim = dim3(unsigned(C), unsigned(n3[2] * nb / PPC));
    cfg.blockDim = dim3(256);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cfg.attrs = attr;
    cfg.numAttrs = 2;
    const cudaError_t err =
        cudaLaunchKernelEx(&cfg, kern, u, e, int(n3[0]), int(n3[1]), int(n3[2]), lam, 6.0f * lam,
                           1.0f + 2.0f * lam, p.xt, p.xf, p.ys, device_status_word());
    if (err != cudaSuccess) {
        cudaGetLastError();
        note_cuda_error(err);
        return false;
    }
    return true;
}

// Pass A with G lanes per row: several planes per CTA when the planes are one
// tile high, else one.
template <int G>
static bool launch_xyw_ppc(const float *u, float *e, const int64_t *n3, int64_t nb, float lam,
                           const AdiWPlan &p, cudaStream_t st, bool check_only) {
    constexpr int PMAX = 32 / G < 16 ? 32 / G : 16;
    switch (xyw_ppc<G>(n3, nb)) {
        case PMAX: return launch_xyw<G, 0, PMAX>(u, e, n3, nb, lam, p, st, check_only);
        default: return launch_xyw<G, 0, 1>(u, e, n3, nb, lam, p, st, check_only);
    }
}

static bool launch_xyw_g(const float *u, float *e, const int64_t *n3, int64_t nb, float lam,
                         const AdiWPlan &p, cudaStream_t st, bool check_only) {
    switch (p.G) {
        case 1: return launch_xyw_ppc<1>(u, e, n3, nb, lam, p, st, check_only);
        case 2: return launch_xyw_ppc<2>(u, e, n3, nb, lam, p, st, check_only);
        case 4: return launch_xyw_ppc<4>(u, e, n3, nb, lam, p, st, check_only);
        case 8: return launch_xyw_ppc<8>(u, e, n3, nb, lam, p, st, check_only);
        case 16: return launch_xyw_ppc<16>(u, e, n3, nb, lam, p, st, check_only);
        case 32:
            return n3[0] == 256 ? launch_xyw<32, 256>(u, e, n3, nb, lam, p, st, check_only)
                                : launch_xyw<32>(u, e, n3, nb, lam, p, st, check_only);
        default: return false;
    }
}

// Pass B launch shape: stages and blocks per SM (two blocks with two to four
// stages when they fit, else one).
struct ZwShape {
    int threads, stages, per_sm;
    size_t smem;
};

static bool zw_shape(const int64_t *n3, ZwShape &z) {
    const DeviceInfo *di = device_info();
    if (!di) return false;
    const int n = int(n3[2]);
    z.threads = 32 * (n / WB_ZT) + 32;
    const size_t stage = (size_t(n) * WB_SG * sizeof(float) + 127) / 128 * 128;
    auto bytes = [&](int s) { return size_t(s) * (stage + 16); };
    const size_t optin = size_t(di->max_smem_optin) - 256;
    z.stages = 0;
    for (int per = 2; per >= 1 && z.stages == 0; --per) {
        size_t cap = size_t(di->smem_per_sm) / per - 4096;
        if (cap > optin) cap = optin;
        for (int sg = 4; sg >= 2; --sg)
            if (bytes(sg) <= cap) { z.stages = sg; break; }
    }
    if (z.stages == 0) return false;
    z.smem = bytes(z.stages);
    z.per_sm = kernel_blocks_per_sm(reinterpret_cast<const void *>(k_adi_zw), z.threads, z.smem);
    return z.per_sm >= 1;
}

static bool launch_zw(const float *e, float *u, const int64_t *n3, int64_t nb, const AdiWPlan &p,
                      const ZwShape &z, cudaStream_t st) {
    const DeviceInfo *di = device_info();
    if (!di) return false;
    const int64_t nplane = n3[0] * n3[1];
    TmaSet maps{};
    if (!encode_lines_map(&maps.map[0], e, int(sizeof(float)), nplane, n3[2], nb, WB_SG))
        return false;
    const int64_t nbatch = nplane / WB_SG * nb;
    const int64_t slots = int64_t(di->sm_count) * z.per_sm;
    const int64_t grid = nbatch < slots ? nbatch : slots;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.gridDim = dim3(unsigned(grid));
    cfg.blockDim = dim3(unsigned(z.threads));
    cfg.dynamicSmemBytes = z.smem;
    cfg.stream = st;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const cudaError_t err = cudaLaunchKernelEx(&cfg, k_adi_zw, maps, p.zw, u, int(nplane),
                                               int(n3[2]), nbatch, z.stages, device_status_word());
    if (err != cudaSuccess) {
        cudaGetLastError();
        note_cuda_error(err);
        return false;
    }
    return true;
}

// Runs nsteps windowed steps; `taken` is false (nothing launched) when the
// problem does not suit the windowed schedule.
static trid_status adi_run_window(float *u, const int64_t *n3, double lam, int nsteps, char *ws,
                                  cudaStream_t st, int64_t nb, bool &taken) {
    taken = false;
    static thread_local AdiWPlan p;  // large tables: kept off the stack
    if (!adiw_plan(n3, nb, lam, p)) return TRID_OK;
    if (!is_aligned16(u) || !is_aligned16(ws)) return TRID_OK;
    ZwShape z;
    if (!zw_shape(n3, z)) return TRID_OK;
    float *e = reinterpret_cast<float *>(ws);
    if (!launch_xyw_g(u, e, n3, nb, float(lam), p, st, true)) return TRID_OK;
    taken = true;
    for (int step = 0; step < nsteps; ++step) {
        if (!launch_xyw_g(u, e, n3, nb, float(lam), p, st, false)) return TRID_ERR_CUDA;
        if (!launch_zw(e, u, n3, nb, p, z, st)) return TRID_ERR_CUDA;
    }
    return TRID_OK;
}

template <typename T>
static trid_status adi_run(T *u, const int64_t *n3, int ndim, T lam, int nsteps, T *w,
                           cudaStream_t st) {
    const int vec = is_aligned16(u) && is_aligned16(w) && (n3[0] * int64_t(sizeof(T))) % 16 == 0;
    const int G = pow2_at_least((n3[0] + ADI_M - 1) / ADI_M);
    Lines Ly{n3[0] * n3[2], n3[1], n3[0], n3[0]};
    Lines Lz{n3[0] * n3[1], n3[2], n3[0] * n3[1], n3[0] * n3[1]};
    for (int step = 0; step < nsteps; ++step) {
        if (launch_x_static<T>(u, w, n3, ndim, lam, st)) {
            if (ndim == 3) {
                adi_strided<T>(lam, w, w, 0, Ly, st);
                adi_strided<T>(lam, w, u, 1, Lz, st);
            } else {
                adi_strided<T>(lam, w, u, 1, Ly, st);
            }
            if (cudaGetLastError() != cudaSuccess) return TRID_ERR_CUDA;
            continue;
        }
        switch (G) {
            case 1: launch_x_rhs<T, 1>(u, w, n3, ndim, lam, vec, st); break;
            case 2: launch_x_rhs<T, 2>(u, w, n3, ndim, lam, vec, st); break;
            case 4: launch_x_rhs<T, 4>(u, w, n3, ndim, lam, vec, st); break;
            case 8: launch_x_rhs<T, 8>(u, w, n3, ndim, lam, vec, st); break;
            case 16: launch_x_rhs<T, 16>(u, w, n3, ndim, lam, vec, st); break;
            default: launch_x_rhs<T, 32>(u, w, n3, ndim, lam, vec, st); break;
        }
        if (ndim == 3) {
            adi_strided<T>(lam, w, w, 0, Ly, st);
            adi_strided<T>(lam, w, u, 1, Lz, st);
        } else {
            adi_strided<T>(lam, w, u, 1, Ly, st);
        }
        if (cudaGetLastError() != cudaSuccess) return TRID_ERR_CUDA;
    }
    return TRID_OK;
}

static trid_status adi_dims(const int64_t *dims, int ndim, int64_t (&n3)[3], int64_t &total) {
    if (!dims || ndim < 2 || ndim > 3) return TRID_ERR_INVALID_ARG;
    n3[0] = n3[1] = n3[2] = 1;
    total = 1;
    for (int k = 0; k < ndim; ++k) {
        if (dims[k] < 3) return TRID_ERR_INVALID_ARG;
        if (dims[k] > ADI_MAX_N) return TRID_ERR_UNSUPPORTED;
        n3[k] = dims[k];
        total *= dims[k];
    }
    return TRID_OK;
}

// Batches of 3D meshes stacked along z (each mesh keeps its own boundary
// planes), through the two-pass schedule; used by adi_step_batched.
bool adi3_batch_eligible(const int64_t *n3, int ndim) { return adi2_eligible(n3, ndim); }

size_t adi3_batch_ws_bytes(const int64_t *n3, size_t esz, int64_t nb) {
    return adi2_layout(n3, esz, nb).total;
}

trid_status adi3_batch_run(void *u, int64_t nb, const int64_t *n3, double lam, int nsteps,
                           trid_dtype dtype, void *ws, size_t ws_bytes, cudaStream_t st) {
    const size_t esz = dtype == TRID_F32 ? 4 : 8;
    if (!ws || ws_bytes < adi3_batch_ws_bytes(n3, esz, nb)) return TRID_ERR_ALLOC;
    if ((reinterpret_cast<uintptr_t>(ws) % 256) != 0) return TRID_ERR_MISALIGNED;
    if (!is_aligned16(u)) return TRID_ERR_MISALIGNED;
    if (dtype == TRID_F32) {
        bool taken = false;
        const trid_status s = adi_run_window(static_cast<float *>(u), n3, lam, nsteps,
                                             static_cast<char *>(ws), st, nb, taken);
        if (taken || s != TRID_OK) return s;
    }
    if (dtype == TRID_F32)
        return adi_run_2pass<float>(static_cast<float *>(u), n3, float(lam), nsteps,
                                    static_cast<char *>(ws), st, nb);
    return adi_run_2pass<double>(static_cast<double *>(u), n3, lam, nsteps,
                                 static_cast<char *>(ws), st, nb);
}

}  // namespace trid

using namespace trid;

extern "C" size_t adi_workspace_bytes(const int64_t *dims, int ndim, trid_dtype dtype) {
    int64_t n3[3], total;
    if (dtype != TRID_F32 && dtype != TRID_F64) return 0;
    if (adi_dims(dims, ndim, n3, total) != TRID_OK) return 0;
    const size_t esz = dtype == TRID_F32 ? 4 : 8;
    if (ndim == 3) return adi2_layout(n3, esz).total;
    return (size_t(total) * esz + 255) / 256 * 256;
}

extern "C" trid_status adi_step(void *u, const int64_t *dims, int ndim, double lambda,
                                int nsteps, trid_dtype dtype, void *workspace,
                                size_t workspace_bytes, trid_stream_t stream) {
    trid::NvtxScope nvtx_scope("adi_step");
    int64_t n3[3], total;
    if (dtype != TRID_F32 && dtype != TRID_F64) return TRID_ERR_INVALID_ARG;
    trid_status s = adi_dims(dims, ndim, n3, total);
    if (s != TRID_OK) return s;
    if (!u || nsteps < 0 || !(lambda > 0.0) || lambda > 1e30) return TRID_ERR_INVALID_ARG;
    const size_t esz = dtype == TRID_F32 ? 4 : 8;
    if ((reinterpret_cast<uintptr_t>(u) % esz) != 0) return TRID_ERR_MISALIGNED;
    if (!workspace || workspace_bytes < adi_workspace_bytes(dims, ndim, dtype))
        return TRID_ERR_ALLOC;
    if ((reinterpret_cast<uintptr_t>(workspace) % 256) != 0) return TRID_ERR_MISALIGNED;
    {
        const char *pu = static_cast<const char *>(u), *pw = static_cast<const char *>(workspace);
        const size_t bytes = size_t(total) * esz;
        const size_t wbytes = adi_workspace_bytes(dims, ndim, dtype);
        if (pu < pw + wbytes && pw < pu + bytes) return TRID_ERR_INVALID_ARG;
    }
    if (nsteps == 0) return TRID_OK;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (ndim == 3 && dtype == TRID_F32) {
        bool taken = false;
        s = adi_run_window(static_cast<float *>(u), n3, lambda, nsteps,
                           static_cast<char *>(workspace), st, 1, taken);
        if (taken || s != TRID_OK) return s;
    }
    if (adi2_eligible(n3, ndim) && is_aligned16(u)) {
        char *ws = static_cast<char *>(workspace);
        if (dtype == TRID_F32)
            return adi_run_2pass<float>(static_cast<float *>(u), n3, float(lambda), nsteps, ws, st);
        return adi_run_2pass<double>(static_cast<double *>(u), n3, lambda, nsteps, ws, st);
    }
    if (dtype == TRID_F32)
        return adi_run<float>(static_cast<float *>(u), n3, ndim, float(lambda), nsteps,
                              static_cast<float *>(workspace), st);
    return adi_run<double>(static_cast<double *>(u), n3, ndim, lambda, nsteps,
                           static_cast<double *>(workspace), st);
}
