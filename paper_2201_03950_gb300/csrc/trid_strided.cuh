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
        if (active && full) {
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
                if (active && i < n) {
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
                if (full || i0 + j < n) ob[(i0 + j) * stride] = ACC ? rd[j] + ru[j] : rd[j];
            }
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
}  // namespace trid
