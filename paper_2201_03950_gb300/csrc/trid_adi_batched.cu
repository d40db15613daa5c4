// trid_adi_batched.cu -- ADI steps on a batch of small meshes, several steps
// per kernel (Section 4.1, Algorithm "adi"; the batched 2D / 3D workloads of
// Section 4 and the chained-iteration (temporal) pipelining of the 2D ADI
// design).
//
// When one mesh and its right-hand side fit in one block's shared memory, a
// block loads the mesh once, runs all nsteps steps in shared memory and writes
// it back: per step the 5-point / 7-point RHS, then one thread per line runs
// the Thomas sweeps of each axis with the constant operator's pivots factored
// once on the host, the last axis adding its result into u.  Rows are padded
// to an odd stride, so the threads of a warp (one line each) hit distinct
// banks on every axis.  Larger 3D meshes whose extents suit the two-pass
// schedule run stacked along z through its kernels (each mesh keeps its own
// boundary planes); the rest go through adi_step one mesh at a time.
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/trid.h"
#include "trid_internal.h"

namespace trid {

constexpr int BA_MAXN = 256;

// Thomas factors of the line operator tridiag(-lam, 1 + 2 lam, -lam) with
// identity end rows:  y_i = (d_i - A_i y_{i-1}) M_i,  x_i = y_i - C_i x_{i+1}
// (the end rows' right-hand side is always 0 here: M of the last row is 0).
template <typename T>
struct BAxis {
    T A[BA_MAXN], M[BA_MAXN], C[BA_MAXN];
};

template <typename T>
struct BTabs {
    BAxis<T> ax[3];
};

template <typename T>
static void baxis_fill(BAxis<T> &t, int n, double lam) {
    double cprev = 0.0;
    for (int i = 0; i < BA_MAXN; ++i) {
        if (i >= n) { t.A[i] = T(0); t.M[i] = T(1); t.C[i] = T(0); continue; }
        const bool bnd = (i == 0 || i == n - 1);
        const double a = bnd ? 0.0 : -lam, b = bnd ? 1.0 : 1.0 + 2.0 * lam, c = bnd ? 0.0 : -lam;
        const double m = 1.0 / (b - a * cprev);
        cprev = c * m;
        t.A[i] = T(a); t.C[i] = T(cprev);
        // last row: identity with a zero right-hand side, so its value is 0
        t.M[i] = (i == n - 1) ? T(0) : T(m);
    }
}

// Lines of one axis: the calling thread solves d along one line in place, or
// (last axis) adds its solution into u.  tab: A, M, C rows of the axis in
// shared memory (every thread of a warp reads the same entry: a broadcast).
template <typename T>
__device__ __forceinline__ void ba_solve_line(const T *tab, T *d, T *u, int n, int step,
                                              bool acc, T lam) {
    // chunks of BA_C values: the chunk's loads are issued together, so the
    // shared-memory latency is paid once per chunk, not once per row.  The
    // sub-diagonal is -lam on every interior row; the end rows are identity
    // rows whose right-hand side is 0 in an ADI step (boundary nodes), so row
    // 0 starts the sweep with prev = 0 and the last row's factor M is 0.
    constexpr int BA_C = 8;
    const T *M = tab + BA_MAXN, *C = tab + 2 * BA_MAXN;
    const T *A = tab;
    T prev = T(0);
    const int nfull = (n / BA_C) * BA_C;
    T *p = d;
    for (int i0 = 0; i0 < nfull; i0 += BA_C, p += BA_C * step) {
        T v[BA_C];
#pragma unroll
        for (int j = 0; j < BA_C; ++j) v[j] = p[j * step];
#pragma unroll
        for (int j = 0; j < BA_C; ++j) {
            prev = fma(lam, prev, v[j]) * M[i0 + j];
            v[j] = prev;
        }
#pragma unroll
        for (int j = 0; j < BA_C; ++j) p[j * step] = v[j];
    }
    for (int i = nfull; i < n; ++i) {
        prev = (d[i * step] - A[i] * prev) * M[i];
        d[i * step] = prev;
    }
    T xn = T(0);
    for (int i = n - 1; i >= nfull; --i) {
        xn = fma(-C[i], xn, d[i * step]);
        if (acc) u[i * step] += xn;
        else d[i * step] = xn;
    }
    for (int i0 = nfull - BA_C; i0 >= 0; i0 -= BA_C) {
        T *q = d + i0 * step;
        T *r = u + i0 * step;
        T v[BA_C], w[BA_C];
#pragma unroll
        for (int j = 0; j < BA_C; ++j) {
            v[j] = q[j * step];
            if (acc) w[j] = r[j * step];
        }
#pragma unroll
        for (int j = BA_C - 1; j >= 0; --j) {
            xn = fma(-C[i0 + j], xn, v[j]);
            v[j] = xn;
        }
#pragma unroll
        for (int j = 0; j < BA_C; ++j) {
            if (acc) r[j * step] = w[j] + v[j];
            else q[j * step] = v[j];
        }
    }
}

template <typename T, int NDIM>
__global__ void __launch_bounds__(1024)
k_adi_fused(T *__restrict__ ug, int64_t nbatch, int nx, int ny, int nz, int p1, int p2, T lam,
            int nsteps, const __grid_constant__ BTabs<T> tabs) {
    extern __shared__ __align__(16) unsigned char smem_ba[];
    T *tab = reinterpret_cast<T *>(smem_ba);  // [3 axes][A, M, C][BA_MAXN]
    T *u = tab + 9 * BA_MAXN;
    T *d = u + size_t(p2) * nz;
    const int tid = threadIdx.x, nth = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5, nwarp = nth >> 5;
    const int nrow = ny * nz;  // x rows of the mesh
    const T centre = T(2 * NDIM);
    for (int q = tid; q < 9 * BA_MAXN; q += nth) {
        const int ax = q / (3 * BA_MAXN), r = q % (3 * BA_MAXN), k = r / BA_MAXN, i = r % BA_MAXN;
        tab[q] = (k == 0) ? tabs.ax[ax].A[i] : (k == 1) ? tabs.ax[ax].M[i] : tabs.ax[ax].C[i];
    }
    for (int64_t mb = blockIdx.x; mb < nbatch; mb += gridDim.x) {
        T *um = ug + mb * int64_t(nx) * nrow;
        for (int row = warp; row < nrow; row += nwarp) {
            const int y = row % ny, z = row / ny;
            for (int x = lane; x < nx; x += 32) u[z * p2 + y * p1 + x] = um[row * nx + x];
        }
        __syncthreads();
        for (int s = 0; s < nsteps; ++s) {
            // explicit part on the interior, 0 on the boundary
            for (int row = warp; row < nrow; row += nwarp) {
                const int y = row % ny, z = row / ny;
                bool rin = y > 0 && y < ny - 1;
                if (NDIM == 3) rin = rin && z > 0 && z < nz - 1;
                const int o0 = z * p2 + y * p1;
                for (int x = lane; x < nx; x += 32) {
                    const int o = o0 + x;
                    T v = T(0);
                    if (rin && x > 0 && x < nx - 1) {
                        T sum = (u[o - 1] + u[o + 1]) + (u[o - p1] + u[o + p1]);
                        if (NDIM == 3) sum += u[o - p2] + u[o + p2];
                        v = lam * (sum - centre * u[o]);
                    }
                    d[o] = v;
                }
            }
            __syncthreads();
            // x lines: one per (y, z)
            for (int l = tid; l < nrow; l += nth) {
                const int y = l % ny, z = l / ny;
                ba_solve_line<T>(tab, d + z * p2 + y * p1, nullptr, nx, 1, false, lam);
            }
            __syncthreads();
            // y lines: one per (x, z); the last axis in 2D adds into u
            for (int l = tid; l < nx * nz; l += nth) {
                const int x = l % nx, z = l / nx;
                const int o = z * p2 + x;
                ba_solve_line<T>(tab + 3 * BA_MAXN, d + o, u + o, ny, p1, NDIM == 2, lam);
            }
            __syncthreads();
            if (NDIM == 3) {
                for (int l = tid; l < nx * ny; l += nth) {
                    const int x = l % nx, y = l / nx;
                    const int o = y * p1 + x;
                    ba_solve_line<T>(tab + 6 * BA_MAXN, d + o, u + o, nz, p2, true, lam);
                }
                __syncthreads();
            }
        }
        for (int row = warp; row < nrow; row += nwarp) {
            const int y = row % ny, z = row / ny;
            for (int x = lane; x < nx; x += 32) um[row * nx + x] = u[z * p2 + y * p1 + x];
        }
        __syncthreads();
    }
}

struct BaPlan {
    int p1, p2, threads;
    size_t smem;
    bool fused;
};

static bool ba_plan(const int64_t *n3, int ndim, size_t esz, BaPlan &pl) {
    const DeviceInfo *di = device_info();
    if (!di) return false;
    pl.p1 = int(n3[0] | 1);  // odd row stride: one line per lane hits distinct banks
    pl.p2 = pl.p1 * int(n3[1]);
    if (ndim == 3 && (pl.p2 % 2) == 0) pl.p2 += 1;
    const size_t elems = size_t(pl.p2) * size_t(n3[2]);
    pl.smem = (2 * elems + 9 * BA_MAXN) * esz;
    int64_t lines = n3[1] * n3[2];
    if (n3[0] * n3[2] > lines) lines = n3[0] * n3[2];
    if (ndim == 3 && n3[0] * n3[1] > lines) lines = n3[0] * n3[1];
    pl.threads = int(((lines + 31) / 32) * 32);
    if (pl.threads > 1024) pl.threads = 1024;
    if (pl.threads < 128) pl.threads = 128;
    pl.fused = n3[0] <= BA_MAXN && n3[1] <= BA_MAXN && n3[2] <= BA_MAXN &&
               pl.smem <= size_t(di->max_smem_optin) - 256;
    return true;
}

template <typename T>
static trid_status ba_run(T *u, int64_t nbatch, const int64_t *n3, int ndim, double lam,
                          int nsteps, const BaPlan &pl, cudaStream_t st) {
    BTabs<T> tabs;
    for (int k = 0; k < 3; ++k) baxis_fill<T>(tabs.ax[k], int(n3[k]), lam);
    const void *kern = ndim == 2 ? reinterpret_cast<const void *>(k_adi_fused<T, 2>)
                                 : reinterpret_cast<const void *>(k_adi_fused<T, 3>);
    const int per_sm = kernel_blocks_per_sm(kern, pl.threads, pl.smem);
    const DeviceInfo *di = device_info();
    if (per_sm < 1 || !di) return TRID_ERR_UNSUPPORTED;
    int64_t grid = int64_t(di->sm_count) * per_sm;
    if (grid > nbatch) grid = nbatch;
    if (ndim == 2)
        k_adi_fused<T, 2><<<dim3(unsigned(grid)), pl.threads, pl.smem, st>>>(
            u, nbatch, int(n3[0]), int(n3[1]), 1, pl.p1, pl.p2, T(lam), nsteps, tabs);
    else
        k_adi_fused<T, 3><<<dim3(unsigned(grid)), pl.threads, pl.smem, st>>>(
            u, nbatch, int(n3[0]), int(n3[1]), int(n3[2]), pl.p1, pl.p2, T(lam), nsteps, tabs);
    return launch_ok() ? TRID_OK : TRID_ERR_CUDA;
}

}  // namespace trid

using namespace trid;

static trid_status ba_dims(const int64_t *dims, int ndim, int64_t (&n3)[3]) {
    if (!dims || ndim < 2 || ndim > 3) return TRID_ERR_INVALID_ARG;
    n3[0] = n3[1] = n3[2] = 1;
    for (int k = 0; k < ndim; ++k) {
        if (dims[k] < 3) return TRID_ERR_INVALID_ARG;
        if (dims[k] > 256) return TRID_ERR_UNSUPPORTED;
        n3[k] = dims[k];
    }
    return TRID_OK;
}

extern "C" size_t adi_batched_workspace_bytes(int64_t nbatch, const int64_t *dims, int ndim,
                                              trid_dtype dtype) {
    int64_t n3[3];
    if (nbatch < 0 || (dtype != TRID_F32 && dtype != TRID_F64) ||
        ba_dims(dims, ndim, n3) != TRID_OK)
        return 0;
    const size_t esz = dtype == TRID_F32 ? 4 : 8;
    BaPlan pl;
    if (!ba_plan(n3, ndim, esz, pl)) return 0;
    if (pl.fused || nbatch == 0) return 0;
    if (adi3_batch_eligible(n3, ndim)) return adi3_batch_ws_bytes(n3, esz, nbatch);
    return adi_workspace_bytes(dims, ndim, dtype);
}

extern "C" trid_status adi_step_batched(void *u, int64_t nbatch, const int64_t *dims, int ndim,
                                        double lambda, int nsteps, trid_dtype dtype,
                                        void *workspace, size_t workspace_bytes,
                                        trid_stream_t stream) {
    trid::NvtxScope nvtx_scope("adi_step_batched");
    int64_t n3[3];
    if (dtype != TRID_F32 && dtype != TRID_F64) return TRID_ERR_INVALID_ARG;
    trid_status s = ba_dims(dims, ndim, n3);
    if (s != TRID_OK) return s;
    if (nbatch < 0 || nsteps < 0 || !(lambda > 0.0) || lambda > 1e30) return TRID_ERR_INVALID_ARG;
    if (nbatch == 0 || nsteps == 0) return TRID_OK;
    if (!u) return TRID_ERR_INVALID_ARG;
    const size_t esz = dtype == TRID_F32 ? 4 : 8;
    if ((reinterpret_cast<uintptr_t>(u) % esz) != 0) return TRID_ERR_MISALIGNED;
    BaPlan pl;
    if (!ba_plan(n3, ndim, esz, pl)) return TRID_ERR_CUDA;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (pl.fused) {
        if (dtype == TRID_F32)
            return ba_run<float>(static_cast<float *>(u), nbatch, n3, ndim, lambda, nsteps, pl, st);
        return ba_run<double>(static_cast<double *>(u), nbatch, n3, ndim, lambda, nsteps, pl, st);
    }
    // 3D meshes stacked along z through the two-pass kernels (boundary planes
    // per mesh), when the extents allow it
    if (adi3_batch_eligible(n3, ndim) && n3[2] * nbatch <= 65535)
        return adi3_batch_run(u, nbatch, n3, lambda, nsteps, dtype, workspace, workspace_bytes, st);
    // otherwise one mesh at a time through the single-mesh path
    const size_t mesh = size_t(n3[0] * n3[1] * n3[2]) * esz;
    for (int64_t b = 0; b < nbatch; ++b) {
        s = adi_step(static_cast<char *>(u) + b * mesh, dims, ndim, lambda, nsteps, dtype,
                     workspace, workspace_bytes, stream);
        if (s != TRID_OK) return s;
    }
    return TRID_OK;
}
