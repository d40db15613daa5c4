// trid_strided.cuh -- the strided-systems kernel (systems along y or z of a
// column-major mesh, Section 2.1), shared by the batched solve and the ADI
// step through a coefficient policy.
//
// A block holds SG systems that are memory neighbours (consecutive x) times
// NT tiles of M rows.  Thread (tile, lane) loads rows [tile*M, tile*M + M) of
// system `lane`: for every row, the SG lanes read SG consecutive elements, one
// coalesced 128-byte segment (SG = 32 in FP32, 16 in FP64),
// so no transpose is needed (the FPGA design buffers XY/XZ planes for the same
// reason, Section 3).  The two reduced rows per tile go through shared memory
// to a warp-shuffle solve (NT lanes per system), and the tile-end unknowns
// come back the same way.
#pragma once
#include "trid_device.cuh"

namespace trid {

// Systems per block of the strided kernel: one 128-byte segment per row.
template <typename T> struct SysCfg;
template <> struct SysCfg<float> { static constexpr int SG = 32; };
template <> struct SysCfg<double> { static constexpr int SG = 16; };

// Coefficients read from arrays; a of row 0 and c of row n-1 are not read.
// b == nullptr means unit diagonal (the reduced systems of the long path).
template <typename T>
struct ArrayCoef {
    const T *__restrict__ a;
    const T *__restrict__ b;
    const T *__restrict__ c;
    __device__ __forceinline__ void get(int64_t p, int64_t i, int64_t n, T &ra, T &rb,
                                        T &rc) const {
        ra = (i == 0) ? T(0) : a[p];
        rb = b ? b[p] : T(1);
        rc = (i == n - 1) ? T(0) : c[p];
    }
};

// The ADI operator of Section 4.1 generated in the kernel:
// tridiag(-lambda, 1 + 2 lambda, -lambda) on interior rows, identity at the two
// Dirichlet boundary nodes.
template <typename T>
struct AdiCoef {
    T lam;
    __device__ __forceinline__ void get(int64_t, int64_t i, int64_t n, T &ra, T &rb,
                                        T &rc) const {
        const bool bnd = (i == 0) || (i == n - 1);
        ra = bnd ? T(0) : -lam;
        rb = bnd ? T(1) : T(1) + T(2) * lam;
        rc = bnd ? T(0) : -lam;
    }
};

template <typename T, int M, int NT, int SG, typename Coef>
__global__ void __launch_bounds__(NT * SG)
k_strided(Coef coef, const T *d, T *out, int accumulate, Lines L) {
    constexpr int P = SG + 1;  // padded row pitch of the shared tables
    __shared__ T s_as[NT * P], s_cs[NT * P], s_ds[NT * P];
    __shared__ T s_ae[NT * P], s_ce[NT * P], s_de[NT * P];
    __shared__ T s_xs[NT * P], s_xe[NT * P];

    const int tid = threadIdx.x;
    const int sl = tid % SG;    // system within block
    const int tile = tid / SG;  // tile within system
    const int64_t sys = int64_t(blockIdx.x) * SG + sl;
    const bool active = sys < L.nsys;
    const int64_t base = active ? L.base(sys) : 0;
    const int64_t i0 = int64_t(tile) * M;

    T ra[M], rb[M], rc[M], rd[M];
#pragma unroll
    for (int j = 0; j < M; ++j) {
        const int64_t i = i0 + j;
        if (active && i < L.n) {
            const int64_t p = base + i * L.stride;
            coef.get(p, i, L.n, ra[j], rb[j], rc[j]);
            rd[j] = d[p];
        } else {
            ra[j] = T(0); rb[j] = T(1); rc[j] = T(0); rd[j] = T(0);
        }
    }
    T as, cs, ds, ae, ce, de;
    tile_reduce<T, M>(ra, rb, rc, rd, as, cs, ds, ae, ce, de);
    const int w = tile * P + sl;
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
    if (!active) return;
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

}  // namespace trid
