// trid_adjoint.cu -- adjoint of the batched solve, for reverse-mode
// differentiation through x = A^{-1} d.
//
// With g_x = dL/dx, the gradients are g_d = A^{-T} g_x and
//   g_a_i = -g_d_i x_{i-1},  g_b_i = -g_d_i x_i,  g_c_i = -g_d_i x_{i+1}
// (g_a of each system's first row and g_c of its last row are 0: those
// entries are not part of A).  A^T is tridiagonal with sub-diagonal c_{i-1},
// diagonal b_i and super-diagonal a_{i+1}, so the same tile / reduced-PCR
// machinery solves it; the kernels read the shifted coefficients directly and
// form the three coefficient gradients in the same pass.
//
//   k_adjoint_lines    contiguous systems (x axis), lane tiles of a warp; the
//                      neighbouring rows come from the adjacent lanes.
//   k_adjoint_strided  strided systems (y/z axes), as k_strided; neighbouring
//                      rows are loaded directly.
// Systems longer than 256 go through three steps: the transposed coefficients
// are written to scratch, the generic solve runs on them, and a gradient
// kernel forms g_a, g_b, g_c.
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/trid.h"
#include "trid_device.cuh"
#include "trid_internal.h"
#include "trid_strided.cuh"

namespace trid {

constexpr int ADJ_M = 8;

template <typename T>
__device__ __forceinline__ void adj_store(T *ga, T *gb, T *gc, T *gd, int64_t p, int64_t i,
                                          int64_t n, T g, T xm, T x0, T xp) {
    gd[p] = g;
    if (gb) gb[p] = -g * x0;
    if (ga) ga[p] = (i > 0) ? -g * xm : T(0);
    if (gc) gc[p] = (i < n - 1) ? -g * xp : T(0);
}

// ---------------------------------------------------------------------------
template <typename T, int M, int G>
__global__ void __launch_bounds__(256)
k_adjoint_lines(const T *__restrict__ a, const T *__restrict__ b, const T *__restrict__ c,
                const T *__restrict__ x, const T *__restrict__ gx, T *ga, T *gb, T *gc, T *gd,
                int64_t nsys, int64_t n, int vec_ok) {
    constexpr unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int64_t warp = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int g = lane % G;
    const int64_t sys = warp * (32 / G) + lane / G;
    const bool active = sys < nsys;
    const int64_t i0 = int64_t(g) * M;
    const int64_t base = sys * n;
    const bool vec = active && vec_ok && i0 + M <= n;

    T ra[M], rb[M], rc[M], rd[M], rx[M];
    if (vec) {
        load_contig_vec<T, M>(a + base + i0, ra);
        load_contig_vec<T, M>(b + base + i0, rb);
        load_contig_vec<T, M>(c + base + i0, rc);
        load_contig_vec<T, M>(gx + base + i0, rd);
    } else {
#pragma unroll
        for (int j = 0; j < M; ++j) {
            const int64_t i = i0 + j;
            const bool in = active && i < n;
            ra[j] = in ? a[base + i] : T(0);  // raw a, shifted below
            rb[j] = in ? b[base + i] : T(1);
            rc[j] = in ? c[base + i] : T(0);  // raw c, shifted below
            rd[j] = in ? gx[base + i] : T(0);
        }
    }
    // A^T: sub-diagonal at row i is c_{i-1}, super-diagonal is a_{i+1}
    const T c_prev = __shfl_up_sync(FULL, rc[M - 1], 1, G);
    const T a_next = __shfl_down_sync(FULL, ra[0], 1, G);
    T ta[M], tc[M];
#pragma unroll
    for (int j = 0; j < M; ++j) {
        const int64_t i = i0 + j;
        ta[j] = (i == 0 || i >= n) ? T(0) : ((j == 0) ? c_prev : rc[j - 1]);
        tc[j] = (i >= n - 1) ? T(0) : ((j == M - 1) ? a_next : ra[j + 1]);
    }
    T as, cs, ds, ae, ce, de, xs, xe;
    tile_reduce<T, M>(ta, rb, tc, rd, as, cs, ds, ae, ce, de);
    // x for the gradients, fetched behind the reduced solve
    if (vec) {
        load_contig_vec<T, M>(x + base + i0, rx);
    } else {
#pragma unroll
        for (int j = 0; j < M; ++j) {
            const int64_t i = i0 + j;
            rx[j] = (active && i < n) ? x[base + i] : T(0);
        }
    }
    group_solve<T, G>(as, cs, ds, ae, ce, de, g, xs, xe);
    const T x_prev = __shfl_up_sync(FULL, rx[M - 1], 1, G);
    const T x_next = __shfl_down_sync(FULL, rx[0], 1, G);
    tile_substitute<T, M>(ta, tc, rd, xs, xe);
    if (!active) return;
    if (vec) {
        T r[M];
        store_contig_vec<T, M>(gd + base + i0, rd);
        if (gb) {
#pragma unroll
            for (int j = 0; j < M; ++j) r[j] = -rd[j] * rx[j];
            store_contig_vec<T, M>(gb + base + i0, r);
        }
        if (ga) {
#pragma unroll
            for (int j = 0; j < M; ++j)
                r[j] = (i0 + j > 0) ? -rd[j] * ((j == 0) ? x_prev : rx[j - 1]) : T(0);
            store_contig_vec<T, M>(ga + base + i0, r);
        }
        if (gc) {
#pragma unroll
            for (int j = 0; j < M; ++j)
                r[j] = (i0 + j < n - 1) ? -rd[j] * ((j == M - 1) ? x_next : rx[j + 1]) : T(0);
            store_contig_vec<T, M>(gc + base + i0, r);
        }
        return;
    }
#pragma unroll
    for (int j = 0; j < M; ++j) {
        const int64_t i = i0 + j;
        if (i < n) {
            const T xm = (j == 0) ? x_prev : rx[j - 1];
            const T xp = (j == M - 1) ? x_next : rx[j + 1];
            adj_store<T>(ga, gb, gc, gd, base + i, i, n, rd[j], xm, rx[j], xp);
        }
    }
}

// ---------------------------------------------------------------------------
template <typename T, int M, int NT, int SG>
__global__ void __launch_bounds__(NT * SG)
k_adjoint_strided(const T *__restrict__ a, const T *__restrict__ b, const T *__restrict__ c,
                  const T *__restrict__ x, const T *__restrict__ gx, T *ga, T *gb, T *gc, T *gd,
                  Lines L, int64_t outer) {
    constexpr int P = SG + 1;
    __shared__ T s_as[NT * P], s_cs[NT * P], s_ds[NT * P];
    __shared__ T s_ae[NT * P], s_ce[NT * P], s_de[NT * P];
    __shared__ T s_xs[NT * P], s_xe[NT * P];
    const int tid = threadIdx.x;
    const int sl = tid % SG, tile = tid / SG;
    const int64_t xi = int64_t(blockIdx.x) * SG + sl;
    const int64_t o = int64_t(blockIdx.z) * gridDim.y + blockIdx.y;
    if (o >= outer) return;
    const int n = int(L.n);
    const int stride = int(L.stride);
    const int i0 = tile * M;
    const bool active = xi < L.inner;
    const int64_t base = active ? xi + o * L.inner * L.n : 0;
    const int w = tile * P + sl;

    T ta[M], rb[M], tc[M], rd[M];
#pragma unroll
    for (int j = 0; j < M; ++j) {
        const int i = i0 + j;
        if (active && i < n) {
            const int64_t p = base + int64_t(i) * stride;
            ta[j] = (i == 0) ? T(0) : c[p - stride];
            rb[j] = b[p];
            tc[j] = (i == n - 1) ? T(0) : a[p + stride];
            rd[j] = gx[p];
        } else {
            ta[j] = T(0); rb[j] = T(1); tc[j] = T(0); rd[j] = T(0);
        }
    }
    T as, cs, ds, ae, ce, de;
    tile_reduce<T, M>(ta, rb, tc, rd, as, cs, ds, ae, ce, de);
    // x for the gradients, fetched behind the reduced solve
    T rx[M + 2];
#pragma unroll
    for (int j = -1; j <= M; ++j) {
        const int i = i0 + j;
        rx[j + 1] = (active && i >= 0 && i < n) ? x[base + int64_t(i) * stride] : T(0);
    }
    s_as[w] = as; s_cs[w] = cs; s_ds[w] = ds;
    s_ae[w] = ae; s_ce[w] = ce; s_de[w] = de;
    __syncthreads();
    {
        const int rs = tid / NT, rt = tid % NT;
        const int q = rt * P + rs;
        T xs, xe;
        group_solve<T, NT>(s_as[q], s_cs[q], s_ds[q], s_ae[q], s_ce[q], s_de[q], rt, xs, xe);
        s_xs[q] = xs;
        s_xe[q] = xe;
    }
    __syncthreads();
    tile_substitute<T, M>(ta, tc, rd, s_xs[w], s_xe[w]);
    if (!active) return;
#pragma unroll
    for (int j = 0; j < M; ++j) {
        const int i = i0 + j;
        if (i < n)
            adj_store<T>(ga, gb, gc, gd, base + int64_t(i) * stride, i, n, rd[j], rx[j], rx[j + 1],
                         rx[j + 2]);
    }
}

// ---------------------------------------------------------------------------
// Long systems: transposed coefficients to scratch, then gradients.
template <typename T>
__global__ void k_adjoint_transpose(const T *__restrict__ a, const T *__restrict__ c,
                                    const T *__restrict__ gx, T *__restrict__ at,
                                    T *__restrict__ ct, T *__restrict__ gd, Lines L) {
    const int64_t total = L.nsys * L.n;
    for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < total;
         e += int64_t(gridDim.x) * blockDim.x) {
        // element e in memory order; its row index inside its system
        const int64_t i = (e / L.inner) % L.n;
        at[e] = (i == 0) ? T(0) : c[e - L.stride];
        ct[e] = (i == L.n - 1) ? T(0) : a[e + L.stride];
        gd[e] = gx[e];
    }
}

template <typename T>
__global__ void k_adjoint_grads(const T *__restrict__ x, const T *__restrict__ gd, T *ga, T *gb,
                                T *gc, Lines L) {
    const int64_t total = L.nsys * L.n;
    for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < total;
         e += int64_t(gridDim.x) * blockDim.x) {
        const int64_t i = (e / L.inner) % L.n;
        const T g = gd[e];
        if (gb) gb[e] = -g * x[e];
        if (ga) ga[e] = (i > 0) ? -g * x[e - L.stride] : T(0);
        if (gc) gc[e] = (i < L.n - 1) ? -g * x[e + L.stride] : T(0);
    }
}

static int pow2_at_least(int64_t v) {
    int p = 1;
    while (p < v) p <<= 1;
    return p;
}

template <typename T, int G>
static void launch_adj_lines(const T *a, const T *b, const T *c, const T *x, const T *gx, T *ga,
                             T *gb, T *gc, T *gd, const Lines &L, cudaStream_t st) {
    const int64_t warps = (L.nsys + (32 / G) - 1) / (32 / G);
    const int64_t blocks = (warps + 7) / 8;
    // 16-byte vector access needs every array 16-byte aligned and each
    // system's start on a 16-byte boundary (n a multiple of 16 / sizeof(T))
    const void *ptrs[9] = {a, b, c, x, gx, ga, gb, gc, gd};
    int vec_ok = (L.n * int64_t(sizeof(T))) % 16 == 0;
    for (const void *p : ptrs)
        if (p && !is_aligned16(p)) vec_ok = 0;
    k_adjoint_lines<T, ADJ_M, G><<<dim3(unsigned(blocks)), 256, 0, st>>>(
        a, b, c, x, gx, ga, gb, gc, gd, L.nsys, L.n, vec_ok);
}

template <typename T, int NT>
static void launch_adj_strided(const T *a, const T *b, const T *c, const T *x, const T *gx, T *ga,
                               T *gb, T *gc, T *gd, const Lines &L, cudaStream_t st) {
    constexpr int SG = (NT * SysCfg<T>::SG < 32) ? 32 / NT : SysCfg<T>::SG;
    k_adjoint_strided<T, ADJ_M, NT, SG><<<strided_grid(L, SG), NT * SG, 0, st>>>(
        a, b, c, x, gx, ga, gb, gc, gd, L, L.nsys / L.inner);
}

template <typename T>
static trid_status adjoint_run(const T *a, const T *b, const T *c, const T *x, const T *gx, T *ga,
                               T *gb, T *gc, T *gd, const Lines &L, char *ws, size_t ws_bytes,
                               cudaStream_t st) {
    if (L.n <= 32 * ADJ_M) {
        const int G = pow2_at_least((L.n + ADJ_M - 1) / ADJ_M);
        if (L.stride == 1) {
            switch (G) {
                case 1: launch_adj_lines<T, 1>(a, b, c, x, gx, ga, gb, gc, gd, L, st); break;
                case 2: launch_adj_lines<T, 2>(a, b, c, x, gx, ga, gb, gc, gd, L, st); break;
                case 4: launch_adj_lines<T, 4>(a, b, c, x, gx, ga, gb, gc, gd, L, st); break;
                case 8: launch_adj_lines<T, 8>(a, b, c, x, gx, ga, gb, gc, gd, L, st); break;
                case 16: launch_adj_lines<T, 16>(a, b, c, x, gx, ga, gb, gc, gd, L, st); break;
                default: launch_adj_lines<T, 32>(a, b, c, x, gx, ga, gb, gc, gd, L, st); break;
            }
        } else {
            if (!strided_offsets_fit(L)) return TRID_ERR_UNSUPPORTED;
            switch (G) {
                case 1: launch_adj_strided<T, 1>(a, b, c, x, gx, ga, gb, gc, gd, L, st); break;
                case 2: launch_adj_strided<T, 2>(a, b, c, x, gx, ga, gb, gc, gd, L, st); break;
                case 4: launch_adj_strided<T, 4>(a, b, c, x, gx, ga, gb, gc, gd, L, st); break;
                case 8: launch_adj_strided<T, 8>(a, b, c, x, gx, ga, gb, gc, gd, L, st); break;
                case 16: launch_adj_strided<T, 16>(a, b, c, x, gx, ga, gb, gc, gd, L, st); break;
                default: launch_adj_strided<T, 32>(a, b, c, x, gx, ga, gb, gc, gd, L, st); break;
            }
        }
        return cudaGetLastError() == cudaSuccess ? TRID_OK : TRID_ERR_CUDA;
    }
    // long systems: at, ct in scratch, solve A^T g_d = g_x in place in g_d
    const size_t arr = (size_t(L.nsys * L.n) * sizeof(T) + 255) / 256 * 256;
    if (ws_bytes < 2 * arr) return TRID_ERR_ALLOC;
    T *at = reinterpret_cast<T *>(ws);
    T *ct = reinterpret_cast<T *>(ws + arr);
    const DeviceInfo *di = device_info();
    if (!di) return TRID_ERR_CUDA;
    const int blocks = di->sm_count * 8;
    k_adjoint_transpose<T><<<blocks, 256, 0, st>>>(a, c, gx, at, ct, gd, L);
    if (cudaGetLastError() != cudaSuccess) return TRID_ERR_CUDA;
    const int64_t dims[3] = {L.inner, L.n, L.nsys / L.inner};
    size_t need = 0;
    const trid_status s = solve_with_scratch(at, b, ct, gd, nullptr, dims, 3, 1,
                                             sizeof(T) == 4 ? TRID_F32 : TRID_F64, ws + 2 * arr,
                                             ws_bytes - 2 * arr, need, st);
    if (s != TRID_OK) return s;
    k_adjoint_grads<T><<<blocks, 256, 0, st>>>(x, gd, ga, gb, gc, L);
    return cudaGetLastError() == cudaSuccess ? TRID_OK : TRID_ERR_CUDA;
}

}  // namespace trid

using namespace trid;

static trid_status adjoint_lines(const int64_t *dims, int ndim, int solve_dim, Lines &L,
                                 int64_t &total) {
    if (!dims || ndim < 1 || ndim > 3 || solve_dim < 0 || solve_dim >= ndim)
        return TRID_ERR_INVALID_ARG;
    int64_t n3[3] = {1, 1, 1};
    total = 1;
    for (int k = 0; k < ndim; ++k) {
        if (dims[k] < 0) return TRID_ERR_INVALID_ARG;
        n3[k] = dims[k];
    }
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
    return TRID_OK;
}

extern "C" size_t trid_adjoint_workspace_bytes(const int64_t *dims, int ndim, int solve_dim,
                                               trid_dtype dtype) {
    Lines L;
    int64_t total;
    if ((dtype != TRID_F32 && dtype != TRID_F64) ||
        adjoint_lines(dims, ndim, solve_dim, L, total) != TRID_OK)
        return 0;
    if (L.n <= 32 * ADJ_M) return 0;
    const size_t esz = dtype == TRID_F32 ? 4 : 8;
    const size_t arr = (size_t(total) * esz + 255) / 256 * 256;
    const int64_t d3[3] = {L.inner, L.n, L.nsys / L.inner};
    return 2 * arr + trid_solve_workspace_bytes(d3, 3, 1, dtype);
}

extern "C" trid_status trid_solve_batch_adjoint(const void *a, const void *b, const void *c,
                                                const void *x, const void *gx, void *ga, void *gb,
                                                void *gc, void *gd, const int64_t *dims, int ndim,
                                                int solve_dim, trid_dtype dtype, void *workspace,
                                                size_t workspace_bytes, trid_stream_t stream) {
    trid::NvtxScope nvtx_scope("trid_solve_batch_adjoint");
    if (dtype != TRID_F32 && dtype != TRID_F64) return TRID_ERR_INVALID_ARG;
    Lines L;
    int64_t total;
    trid_status s = adjoint_lines(dims, ndim, solve_dim, L, total);
    if (s != TRID_OK) return s;
    if (total == 0) return TRID_OK;
    if (!a || !b || !c || !x || !gx || !gd) return TRID_ERR_INVALID_ARG;
    const size_t esz = dtype == TRID_F32 ? 4 : 8;
    const void *ptrs[9] = {a, b, c, x, gx, ga, gb, gc, gd};
    for (int k = 0; k < 9; ++k)
        if (ptrs[k] && (reinterpret_cast<uintptr_t>(ptrs[k]) % esz) != 0) return TRID_ERR_MISALIGNED;
    // outputs must not alias each other or the inputs
    const size_t bytes = size_t(total) * esz;
    for (int o = 5; o < 9; ++o) {
        if (!ptrs[o]) continue;
        for (int q = 0; q < 9; ++q) {
            if (q == o || !ptrs[q]) continue;
            const char *p1 = static_cast<const char *>(ptrs[o]);
            const char *p2 = static_cast<const char *>(ptrs[q]);
            if (p1 < p2 + bytes && p2 < p1 + bytes) return TRID_ERR_INVALID_ARG;
        }
    }
    const size_t need = trid_adjoint_workspace_bytes(dims, ndim, solve_dim, dtype);
    if (need > 0 && (workspace == nullptr || workspace_bytes < need)) return TRID_ERR_ALLOC;
    if (need > 0 && (reinterpret_cast<uintptr_t>(workspace) % 256) != 0) return TRID_ERR_MISALIGNED;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    char *ws = static_cast<char *>(workspace);
    if (dtype == TRID_F32)
        return adjoint_run<float>(static_cast<const float *>(a), static_cast<const float *>(b),
                                  static_cast<const float *>(c), static_cast<const float *>(x),
                                  static_cast<const float *>(gx), static_cast<float *>(ga),
                                  static_cast<float *>(gb), static_cast<float *>(gc),
                                  static_cast<float *>(gd), L, ws, workspace_bytes, st);
    return adjoint_run<double>(static_cast<const double *>(a), static_cast<const double *>(b),
                               static_cast<const double *>(c), static_cast<const double *>(x),
                               static_cast<const double *>(gx), static_cast<double *>(ga),
                               static_cast<double *>(gb), static_cast<double *>(gc),
                               static_cast<double *>(gd), L, ws, workspace_bytes, st);
}
