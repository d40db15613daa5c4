// trid_adi2v.cu -- 2D ADI with a diffusivity field kappa, and its reverse
// mode with checkpointing (the ADI step of Section 4.1, Algorithm "adi", made
// differentiable; the paper has no variable-coefficient form).
//
// Reading of the operator: face diffusivities are node means,
//   kx_p = (kappa_p + kappa_{p+1}) / 2,   ky_p = (kappa_p + kappa_{p+nx}) / 2,
// and on rows 0 < i < nx-1 the x operator is
//   a_p = -lam kx_{p-1},  c_p = -lam kx_p,  b_p = 1 - a_p - c_p
// (identity rows at i = 0, nx-1; y alike with stride nx).  One step:
//   d_p = -c_p (u_{p+1} - u_p) + a_p (u_p - u_{p-1}) + (y terms)  (interior,
//         0 on the boundary),  w = X^{-1} d,  delta = Y^{-1} w,  u += delta.
// With kappa = 1 this is the constant-coefficient 2D step.
//
// Reverse mode of one step, g = dL/du_{t+1}:
//   g_w = Y^{-T} g and g_d = X^{-T} g_w, with the coefficient gradients of
//        the solves -g_w delta_{p-nx}, -g_w delta_p, -g_w delta_{p+nx} (Y) and
//        -g_d w_{p-1}, -g_d w_p, -g_d w_{p+1} (X),
//   g_d restricted to the interior, dL/du_t = g + (transposed stencil) g_d,
//   and the stencil adds g_d (u_p - u_{p-1}) to the gradient of a_p and
//   g_d (u_p - u_{p+1}) to that of c_p (y alike).
// The coefficient arrays do not change over the steps: the transposed
// operators (sub-diagonal c_{i-1}, super-diagonal a_{i+1}) are formed once
// per backward call, each step's two adjoint solves are plain solves of them
// stored into their own buffers (so g and g_w stay intact), and one kernel
// per step forms the stencil's reverse, every coefficient gradient of the step
// and their sums over the steps (taken to kappa once at the end).
//
// Checkpointing: the forward keeps u every `every` steps; the backward
// recomputes each segment forward from its checkpoint (keeping u_t, w_t and
// delta_t of the segment) and then runs the segment's steps in reverse.
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/trid.h"
#include "trid_device.cuh"
#include "trid_internal.h"
#include "trid_tma.cuh"

namespace trid {

template <typename T>
__global__ void k_v2_coef(const T *__restrict__ kap, T *ax, T *bx, T *cx, T *ay, T *by, T *cy,
                          int nx, int ny, T lam) {
    for (int j = blockIdx.y; j < ny; j += gridDim.y) {
        const int i = blockIdx.x * blockDim.x + threadIdx.x;
        if (i >= nx) continue;
        const size_t p = size_t(j) * nx + i;
        const T k0 = kap[p];
        if (i == 0 || i == nx - 1) {
            ax[p] = T(0); bx[p] = T(1); cx[p] = T(0);
        } else {
            const T a = -lam * (T(0.5) * (kap[p - 1] + k0));
            const T c = -lam * (T(0.5) * (k0 + kap[p + 1]));
            ax[p] = a; cx[p] = c; bx[p] = (T(1) - a) - c;
        }
        if (j == 0 || j == ny - 1) {
            ay[p] = T(0); by[p] = T(1); cy[p] = T(0);
        } else {
            const T a = -lam * (T(0.5) * (kap[p - nx] + k0));
            const T c = -lam * (T(0.5) * (k0 + kap[p + nx]));
            ay[p] = a; cy[p] = c; by[p] = (T(1) - a) - c;
        }
    }
}

// The per-step kernels are launched with programmatic dependent launch (the
// next kernel may be scheduled while the previous one drains); each waits
// for the previous kernel before touching memory, and their pointers are not
// __restrict__, so that no load is moved ahead of that wait.
//
// Explicit part: d = lam (Lx + Ly) u on the interior, 0 on the boundary.
template <typename T>
__global__ void k_v2_rhs(const T *u, const T *ax, const T *cx, const T *ay, const T *cy, T *d,
                         int nx, int ny) {
    pdl_wait();
    for (int j = blockIdx.y; j < ny; j += gridDim.y) {
        const int i = blockIdx.x * blockDim.x + threadIdx.x;
        if (i >= nx) continue;
        const size_t p = size_t(j) * nx + i;
        T v = T(0);
        if (i > 0 && i < nx - 1 && j > 0 && j < ny - 1) {
            const T uc = u[p];
            v = -cx[p] * (u[p + 1] - uc) + ax[p] * (uc - u[p - 1]);
            v += -cy[p] * (u[p + nx] - uc) + ay[p] * (uc - u[p - nx]);
        }
        d[p] = v;
    }
}

// The explicit part fused with the x solve, one block per x line (row j):
// w = X^{-1} d with d as k_v2_rhs.  KEEP (a recomputed step): u = up + dp is
// formed on the fly for rows j - 1 .. j + 1 and row j is written to u, as
// k_v2_rhs_keep; without KEEP, u is read.  Thread t owns columns [8 t, 8 t +
// 8) (nx % 8 == 0, nx <= 1024, so at most 128 threads): the RHS and the tile
// pass of Section 3.1 in registers, the 2 nx / 8 reduced rows in shared memory
// (padded by one element per 128 bytes: warp 0's lanes walk them in runs of
// 8) solved by warp 0 (tiles of 8 reduced rows, then the shuffled reduced
// solve of 32 lanes), then every tile substituted and stored.  d never goes
// to memory, and the step saves a launch.
constexpr int V2X_M = 8;
constexpr int V2X_MAXT = 128;  // threads (tiles) per line: nx <= 1024

template <typename T>
__device__ __forceinline__ int v2x_pad(int i) {
    return i + (i >> (sizeof(T) == 4 ? 5 : 4));
}

template <typename T, bool KEEP>
__global__ void __launch_bounds__(V2X_MAXT)
k_v2_rhs_x(const T *up, const T *dp, T *u, const T *ax, const T *bx, const T *cx, const T *ay,
           const T *cy, T *w, int nx, int ny, int vec_u) {
    constexpr int M = V2X_M;
    constexpr int RP = 2 * V2X_MAXT + (2 * V2X_MAXT) / (sizeof(T) == 4 ? 32 : 16) + 1;
    __shared__ T ra_s[RP], rc_s[RP], rd_s[RP];  // reduced rows (padded)
    __shared__ T edge_l[V2X_MAXT], edge_r[V2X_MAXT];  // u at each tile's first / last column
    pdl_wait();
    const int t = threadIdx.x, lane = t & 31;
    const int nt = nx / M;           // tiles of the line
    const int nthr = int(blockDim.x);  // >= nt, a multiple of 32
    const bool own = t < nt;
    const int x0 = t * M;
    for (int j = blockIdx.x; j < ny; j += gridDim.x) {
        const size_t rowp = size_t(j) * nx;
        auto ld = [&](const T *q, T (&r)[M]) {  // vector loads unless u is unaligned
            if (vec_u) {
                load_contig_vec<T, M>(q, r);
            } else {
#pragma unroll
                for (int k = 0; k < M; ++k) r[k] = q[k];
            }
        };
        auto ldrow = [&](int jj, T (&r)[M]) {  // u of row jj at the thread's columns
            if (KEEP && dp) {
                T e[M];
                ld(up + size_t(jj) * nx + x0, r);
                ld(dp + size_t(jj) * nx + x0, e);
#pragma unroll
                for (int k = 0; k < M; ++k) r[k] = r[k] + e[k];
            } else {
                ld(u + size_t(jj) * nx + x0, r);
            }
        };
        T uc[M], d[M], a[M], b[M], c[M];
        if (own) {
            ldrow(j, uc);
            edge_l[t] = uc[0];
            edge_r[t] = uc[M - 1];
        }
        __syncthreads();
        if (own) {
            const bool jin = j > 0 && j < ny - 1;
            T um[M], upn[M], axv[M], cxv[M], ayv[M], cyv[M];
            if (jin) {
                ldrow(j - 1, um);
                ldrow(j + 1, upn);
                load_contig_vec<T, M>(ay + rowp + x0, ayv);
                load_contig_vec<T, M>(cy + rowp + x0, cyv);
            }
            load_contig_vec<T, M>(ax + rowp + x0, axv);
            load_contig_vec<T, M>(cx + rowp + x0, cxv);
            load_contig_vec<T, M>(bx + rowp + x0, b);
            const T left = t > 0 ? edge_r[t - 1] : T(0);
            const T right = t + 1 < nt ? edge_l[t + 1] : T(0);
#pragma unroll
            for (int k = 0; k < M; ++k) {
                const int i = x0 + k;
                T v = T(0);
                if (jin && i > 0 && i < nx - 1) {
                    const T ul = k == 0 ? left : uc[k - 1];
                    const T ur = k == M - 1 ? right : uc[k + 1];
                    v = -cxv[k] * (ur - uc[k]) + axv[k] * (uc[k] - ul);
                    v += -cyv[k] * (upn[k] - uc[k]) + ayv[k] * (uc[k] - um[k]);
                }
                d[k] = v;
                a[k] = i == 0 ? T(0) : axv[k];
                c[k] = i == nx - 1 ? T(0) : cxv[k];
            }
            if (KEEP && dp) {
                if (vec_u) {
                    store_contig_vec<T, M>(u + rowp + x0, uc);
                } else {
#pragma unroll
                    for (int k = 0; k < M; ++k) u[rowp + x0 + k] = uc[k];
                }
            }
        } else {
#pragma unroll
            for (int k = 0; k < M; ++k) { a[k] = T(0); b[k] = T(1); c[k] = T(0); d[k] = T(0); }
        }
        T as, cs, ds, ae, ce, de;
        tile_reduce<T, M>(a, b, c, d, as, cs, ds, ae, ce, de);
        ra_s[v2x_pad<T>(2 * t)] = as; rc_s[v2x_pad<T>(2 * t)] = cs; rd_s[v2x_pad<T>(2 * t)] = ds;
        ra_s[v2x_pad<T>(2 * t + 1)] = ae; rc_s[v2x_pad<T>(2 * t + 1)] = ce;
        rd_s[v2x_pad<T>(2 * t + 1)] = de;
        __syncthreads();
        if (t < 32) {
            // the 2 nthr reduced rows: lane l takes rows [8 l, 8 l + 8)
            const int R = 2 * nthr;
            T qa[M], qb[M], qc[M], qd[M];
#pragma unroll
            for (int k = 0; k < M; ++k) {
                const int i = lane * M + k;
                const bool in = i < R;
                qa[k] = (in && i > 0) ? ra_s[v2x_pad<T>(i)] : T(0);
                qb[k] = T(1);
                qc[k] = (in && i < R - 1) ? rc_s[v2x_pad<T>(i)] : T(0);
                qd[k] = in ? rd_s[v2x_pad<T>(i)] : T(0);
            }
            T qas, qcs, qds, qae, qce, qde, xs, xe;
            tile_reduce<T, M>(qa, qb, qc, qd, qas, qcs, qds, qae, qce, qde);
            group_solve<T, 32>(qas, qcs, qds, qae, qce, qde, lane, xs, xe);
            tile_substitute<T, M>(qa, qc, qd, xs, xe);
#pragma unroll
            for (int k = 0; k < M; ++k)
                if (lane * M + k < R) rd_s[v2x_pad<T>(lane * M + k)] = qd[k];
        }
        __syncthreads();
        if (own) {
            tile_substitute<T, M>(a, c, d, rd_s[v2x_pad<T>(2 * t)], rd_s[v2x_pad<T>(2 * t + 1)]);
            store_contig_vec<T, M>(w + rowp + x0, d);
        }
        __syncthreads();  // the shared rows are rewritten for the next line
    }
}

// The fused explicit part + x solve takes lines of nx a multiple of 8 up to
// 1024.  The choice depends on nx alone, so that the forward and the
// backward's recomputation (separate calls) always run the same arithmetic;
// the workspace arrays are 256-byte aligned, and u (the caller's) is read
// with scalar loads when it is not on a 16-byte boundary.
static bool v2x_fits(int nx) {
    return nx % V2X_M == 0 && nx / V2X_M <= V2X_MAXT && nx >= 2 * V2X_M;
}


// The transposed operators: A^T has sub-diagonal c_{i-1} and super-diagonal
// a_{i+1} (the diagonal is b).
template <typename T>
__global__ void k_v2_transpose(const T *__restrict__ ax, const T *__restrict__ cx,
                               const T *__restrict__ ay, const T *__restrict__ cy, T *atx, T *ctx,
                               T *aty, T *cty, int nx, int ny) {
    for (int j = blockIdx.y; j < ny; j += gridDim.y) {
        const int i = blockIdx.x * blockDim.x + threadIdx.x;
        if (i >= nx) continue;
        const size_t p = size_t(j) * nx + i;
        atx[p] = i > 0 ? cx[p - 1] : T(0);
        ctx[p] = i < nx - 1 ? ax[p + 1] : T(0);
        aty[p] = j > 0 ? cy[p - nx] : T(0);
        cty[p] = j < ny - 1 ? ay[p + nx] : T(0);
    }
}

// The explicit part of a recomputed step, from the previous step's state and
// increment: u = up + dp (when dp is given; else u is read as is), written to
// u; d = lam (Lx + Ly) u as k_v2_rhs.
template <typename T>
__global__ void k_v2_rhs_keep(const T *up, const T *dp, T *u, const T *ax, const T *cx,
                              const T *ay, const T *cy, T *d, int nx, int ny) {
    pdl_wait();
    for (int j = blockIdx.y; j < ny; j += gridDim.y) {
        const int i = blockIdx.x * blockDim.x + threadIdx.x;
        if (i >= nx) continue;
        const size_t p = size_t(j) * nx + i;
        auto U = [&](size_t q) -> T { return dp ? up[q] + dp[q] : u[q]; };
        const T uc = U(p);
        T v = T(0);
        if (i > 0 && i < nx - 1 && j > 0 && j < ny - 1) {
            v = -cx[p] * (U(p + 1) - uc) + ax[p] * (uc - U(p - 1));
            v += -cy[p] * (U(p + nx) - uc) + ay[p] * (uc - U(p - nx));
        }
        d[p] = v;
        if (dp) u[p] = uc;
    }
}

// Reverse of the explicit part and of the identity path, plus the summed
// coefficient gradients:  gn = g + S^T gm  (gm = g_d on the interior).
// Gather form: point q collects the stencil rows p = q, q +- 1, q +- nx that
// read u_q.  w and dl are the step's X^{-1} d and delta.  Per point p the
// step's coefficient gradients are
//   a_x: -g_d,p w_{p-1} + gm_p (u_p - u_{p-1}),  b_x: -g_d,p w_p,
//   c_x: -g_d,p w_{p+1} + gm_p (u_p - u_{p+1})   (y alike with g_w, delta).
// COEF: G_k += each of the six (the caller wants them); otherwise only the
// face sums that the kappa gradient needs are kept: F_x[p] += (b_x - a_x) at
// p + 1 (if interior) + (b_x - c_x) at p (if interior), face (p, p + 1);
// F_y alike for face (p, p + nx).
//
// Each thread walks V2_ROWS consecutive rows of one column, keeping the
// column's values of the rows above and below in registers (the x
// neighbours are read directly and mostly hit L1).
constexpr int V2_ROWS = 8;

template <typename T, bool COEF>
__global__ void __launch_bounds__(256)
k_v2_rhs_adj(const T *g, const T *gd, const T *gw, const T *u, const T *w, const T *dl,
             const T *ax, const T *cx, const T *ay, const T *cy, T *G, T *gn, int nx, int ny,
             size_t n) {
    pdl_wait();
    // n: element stride between the arrays of G
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nx) return;
    const bool xin = i > 0 && i < nx - 1;
    for (int64_t jb = int64_t(blockIdx.y) * V2_ROWS; jb < ny; jb += int64_t(gridDim.y) * V2_ROWS) {
    const int j0 = int(jb);
    const int j1 = j0 + V2_ROWS < ny ? j0 + V2_ROWS : ny;
    auto col = [&](const T *a, int jj) -> T {  // a at (i, jj), 0 outside the mesh
        return (jj >= 0 && jj < ny) ? a[size_t(jj) * nx + i] : T(0);
    };
    auto mask = [&](int jj, T v) -> T { return (xin && jj > 0 && jj < ny - 1) ? v : T(0); };
    // column window: rows j - 1, j, j + 1 (u, delta, g_d), j, j + 1 (g_w, a_y),
    // j - 1, j (c_y)
    T u_m = col(u, j0 - 1), u_c = col(u, j0), u_p = col(u, j0 + 1);
    T d_m = col(dl, j0 - 1), d_c = col(dl, j0), d_p = col(dl, j0 + 1);
    T r_m = col(gd, j0 - 1), r_c = col(gd, j0), r_p = col(gd, j0 + 1);
    T gw_c = col(gw, j0), gw_p = col(gw, j0 + 1);
    T ay_c = col(ay, j0), ay_p = col(ay, j0 + 1);
    T cy_m = col(cy, j0 - 1), cy_c = col(cy, j0);
    for (int j = j0; j < j1; ++j) {
        const size_t p = size_t(j) * nx + i;
        auto gmx = [&](int ii) -> T {  // g_d on the interior at (ii, j)
            return (ii > 0 && ii < nx - 1 && j > 0 && j < ny - 1) ? gd[p + (ii - i)] : T(0);
        };
        const T g0 = mask(j, r_c);
        T acc = g[p] + (ax[p] + cx[p] + ay_c + cy_c) * g0;
        if (i > 0) acc -= cx[p - 1] * gmx(i - 1);
        if (i < nx - 1) acc -= ax[p + 1] * gmx(i + 1);
        if (j > 0) acc -= cy_m * mask(j - 1, r_m);
        if (j < ny - 1) acc -= ay_p * mask(j + 1, r_p);
        gn[p] = acc;
        // the step's coefficient gradients at p: x solve and stencil, y solve and stencil
        T sa = i > 0 ? -r_c * w[p - 1] : T(0);
        const T sb = -r_c * w[p];
        T sc = i < nx - 1 ? -r_c * w[p + 1] : T(0);
        T ta = j > 0 ? -gw_c * d_m : T(0);
        const T tb = -gw_c * d_c;
        T tc = j < ny - 1 ? -gw_c * d_p : T(0);
        if (g0 != T(0)) {
            sa += g0 * (u_c - u[p - 1]);
            sc += g0 * (u_c - u[p + 1]);
            ta += g0 * (u_c - u_m);
            tc += g0 * (u_c - u_p);
        }
        if (COEF) {
            G[p] += sa;
            G[n + p] += sb;
            G[2 * n + p] += sc;
            G[3 * n + p] += ta;
            G[4 * n + p] += tb;
            G[5 * n + p] += tc;
        } else {
            if (i < nx - 1) {  // face (p, p + 1): (b - c) at p, (b - a) at p + 1
                T f = (i > 0) ? sb - sc : T(0);
                if (i + 1 < nx - 1) {
                    const T r1 = gd[p + 1], g1 = gmx(i + 1), u1 = u[p + 1];
                    T a1 = -r1 * w[p];
                    const T b1 = -r1 * w[p + 1];
                    if (g1 != T(0)) a1 += g1 * (u1 - u_c);
                    f += b1 - a1;
                }
                G[p] += f;
            }
            if (j < ny - 1) {  // face (p, p + nx)
                T f = (j > 0) ? tb - tc : T(0);
                if (j + 1 < ny - 1) {
                    const T g1 = mask(j + 1, r_p);
                    T a1 = -gw_p * d_c;
                    const T b1 = -gw_p * d_p;
                    if (g1 != T(0)) a1 += g1 * (u_p - u_c);
                    f += b1 - a1;
                }
                G[n + p] += f;
            }
        }
        // slide the column window down one row
        u_m = u_c; u_c = u_p; u_p = col(u, j + 2);
        d_m = d_c; d_c = d_p; d_p = col(dl, j + 2);
        r_m = r_c; r_c = r_p; r_p = col(gd, j + 2);
        gw_c = gw_p; gw_p = col(gw, j + 2);
        ay_c = ay_p; ay_p = col(ay, j + 2);
        cy_m = cy_c; cy_c = col(cy, j + 1);
    }
    }
}

// Face sums -> kappa: node p takes half of each of its faces' gradients.
template <typename T>
__global__ void k_v2_kappa_faces(const T *__restrict__ F, T *__restrict__ gk, int nx, int ny,
                                 T lam, size_t n) {
    for (int j = blockIdx.y; j < ny; j += gridDim.y) {
        const int i = blockIdx.x * blockDim.x + threadIdx.x;
        if (i >= nx) continue;
        const size_t p = size_t(j) * nx + i;
        T v = T(0);
        if (i > 0) v += T(0.5) * (lam * F[p - 1]);
        if (i < nx - 1) v += T(0.5) * (lam * F[p]);
        if (j > 0) v += T(0.5) * (lam * F[n + p - nx]);
        if (j < ny - 1) v += T(0.5) * (lam * F[n + p]);
        gk[p] = v;
    }
}

// Summed coefficient gradients -> faces -> nodes.
template <typename T>
__global__ void k_v2_kappa(const T *__restrict__ G, T *__restrict__ gk, int nx, int ny, T lam,
                           size_t n) {
    // n: element stride between the six arrays of G
    for (int j = blockIdx.y; j < ny; j += gridDim.y) {
        const int i = blockIdx.x * blockDim.x + threadIdx.x;
        if (i >= nx) continue;
        const size_t p = size_t(j) * nx + i;
        // face q (between q and q+1 along x) is read by row q+1 (as a) and row q (as c)
        auto fx = [&](int ii) -> T {  // gradient of face (ii, ii+1) on line j
            const size_t q = size_t(j) * nx + ii;
            T v = T(0);
            if (ii + 1 > 0 && ii + 1 < nx - 1) v += lam * (G[n + q + 1] - G[q + 1]);
            if (ii > 0 && ii < nx - 1) v += lam * (G[n + q] - G[2 * n + q]);
            return v;
        };
        auto fy = [&](int jj) -> T {  // face (jj, jj+1) on column i
            const size_t q = size_t(jj) * nx + i;
            T v = T(0);
            if (jj + 1 > 0 && jj + 1 < ny - 1) v += lam * (G[4 * n + q + nx] - G[3 * n + q + nx]);
            if (jj > 0 && jj < ny - 1) v += lam * (G[4 * n + q] - G[5 * n + q]);
            return v;
        };
        T v = T(0);
        if (i > 0) v += T(0.5) * fx(i - 1);
        if (i < nx - 1) v += T(0.5) * fx(i);
        if (j > 0) v += T(0.5) * fy(j - 1);
        if (j < ny - 1) v += T(0.5) * fy(j);
        gk[p] = v;
    }
}

// ---------------------------------------------------------------------------
struct V2Layout {
    size_t mesh;      // bytes of one mesh array (256-aligned)
    size_t scratch;   // solve / adjoint scratch
    size_t fwd, bwd;  // workspace totals
    int nseg;
};

static size_t up256(size_t v) { return (v + 255) / 256 * 256; }

static bool v2_layout(const int64_t *dims, int nsteps, int every, trid_dtype dtype, V2Layout &l) {
    if (!dims || dims[0] < 3 || dims[1] < 3 || nsteps < 0 || every < 1) return false;
    if (dtype != TRID_F32 && dtype != TRID_F64) return false;
    if (dims[0] > (int64_t(1) << 30) || dims[1] > (int64_t(1) << 30)) return false;
    const size_t esz = dtype == TRID_F32 ? 4 : 8;
    const size_t n = size_t(dims[0]) * size_t(dims[1]);
    l.mesh = up256(n * esz);
    size_t s = 0;
    for (int ax = 0; ax < 2; ++ax) {
        const size_t a = trid_solve_workspace_bytes(dims, 2, ax, dtype);
        const size_t b = trid_adjoint_workspace_bytes(dims, 2, ax, dtype);
        s = a > s ? a : s;
        s = b > s ? b : s;
    }
    l.scratch = up256(s);
    const size_t K = size_t(every);
    l.fwd = 7 * l.mesh + l.scratch;  // 6 coefficient arrays + d/w
    // coefficients 6, transposed coefficients 4, two sets of segment u/w/delta
    // 6K, g and gn 2, g_w and g_d 2, sums 6; a scratch per stream
    l.bwd = (6 + 4 + 6 * K + 2 + 2 + 6) * l.mesh + 2 * l.scratch;
    l.nseg = nsteps == 0 ? 1 : (nsteps + every - 1) / every;
    return true;
}

// Launch with programmatic dependent launch allowed (outside stream capture).
template <typename... KArgs, typename... Args>
static bool launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, cudaStream_t st,
                       Args... args) {
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cfg.attrs = attr;
    cfg.numAttrs = pdl_launch_allowed(st) ? 1 : 0;
    const cudaError_t e = cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
    if (e != cudaSuccess) {
        note_cuda_error(e);
        cudaGetLastError();
        return false;
    }
    return true;
}

template <typename T, bool KEEP>
static bool launch_v2x(const T *up, const T *dp, T *u, const T *const co[6], T *w, int nx, int ny,
                       cudaStream_t st) {
    const int threads = (nx / V2X_M + 31) / 32 * 32;
    const int vec_u = is_aligned16(u) && (!up || is_aligned16(up)) && (!dp || is_aligned16(dp));
    const dim3 grid(unsigned(ny < 65535 ? ny : 65535));
    return launch_pdl(k_v2_rhs_x<T, KEEP>, grid, dim3(unsigned(threads)), st, up, dp, u, co[0],
                      co[1], co[2], co[3], co[5], w, nx, ny, vec_u);
}

template <typename T>
static void grid2(int nx, int ny, dim3 &g, dim3 &b) {
    b = dim3(256);
    g = dim3(unsigned((nx + 255) / 256), unsigned(ny < 65535 ? ny : 65535));
}

template <typename T>
static trid_status v2_forward_step(T *u, T *dw, const T *const co[6], const int64_t *dims,
                                   char *scr, size_t scr_bytes, trid_dtype dt, cudaStream_t st) {
    const int nx = int(dims[0]), ny = int(dims[1]);
    if (v2x_fits(nx)) {  // w = X^{-1} d, d formed on the fly
        if (!launch_v2x<T, false>(nullptr, nullptr, u, co, dw, nx, ny, st)) return TRID_ERR_CUDA;
    } else {
        dim3 g, b;
        grid2<T>(nx, ny, g, b);
        if (!launch_pdl(k_v2_rhs<T>, g, b, st, u, co[0], co[2], co[3], co[5], dw, nx, ny))
            return TRID_ERR_CUDA;
        const trid_status s = trid_solve_batch_ws(co[0], co[1], co[2], dw, nullptr, dims, 2, 0,
                                                  dt, scr, scr_bytes, st);
        if (s != TRID_OK) return s;
    }
    // u += Y^{-1} w
    return trid_solve_batch_ws(co[3], co[4], co[5], dw, u, dims, 2, 1, dt, scr, scr_bytes, st);
}

// A step recomputed by the backward, keeping u (at u; formed from the
// previous state up and increment dp unless dp is NULL), w = X^{-1} d (at w)
// and delta = Y^{-1} w (at dl).  The explicit part (which also writes u) and
// the x solve (one fused launch for lines of up to 1024 points), then the y
// solve stored into dl (w stays intact).  u + delta is formed by the next step's first kernel, with the
// same rounding as the forward's accumulating y solve.
template <typename T>
static trid_status v2_recompute_step(const T *up, const T *dp, T *u, T *w, T *dl,
                                     const T *const co[6], const int64_t *dims, char *scr,
                                     size_t scr_bytes, trid_dtype dt, cudaStream_t st) {
    const int nx = int(dims[0]), ny = int(dims[1]);
    if (v2x_fits(nx)) {  // the same fused kernel as the forward, u formed on the fly
        if (!launch_v2x<T, true>(up, dp, u, co, w, nx, ny, st)) return TRID_ERR_CUDA;
    } else {
        dim3 g, b;
        grid2<T>(nx, ny, g, b);
        if (!launch_pdl(k_v2_rhs_keep<T>, g, b, st, up, dp, u, co[0], co[2], co[3], co[5], w, nx,
                        ny))
            return TRID_ERR_CUDA;
        const trid_status s = trid_solve_batch_ws(co[0], co[1], co[2], w, nullptr, dims, 2, 0, dt,
                                                  scr, scr_bytes, st);
        if (s != TRID_OK) return s;
    }
    return solve_into_ws(co[3], co[4], co[5], w, dl, dims, 2, 1, dt, scr, scr_bytes, st);
}

template <typename T>
static trid_status v2_forward(const T *u0, T *uT, const T *kap, const int64_t *dims, T lam,
                              int nsteps, int every, T *ckpt, char *ws, const V2Layout &l,
                              trid_dtype dt, cudaStream_t st) {
    const int nx = int(dims[0]), ny = int(dims[1]);
    const size_t n = size_t(nx) * ny;
    T *co[6];
    for (int k = 0; k < 6; ++k) co[k] = reinterpret_cast<T *>(ws + k * l.mesh);
    T *dw = reinterpret_cast<T *>(ws + 6 * l.mesh);
    char *scr = ws + 7 * l.mesh;
    dim3 g, b;
    grid2<T>(nx, ny, g, b);
    k_v2_coef<T><<<g, b, 0, st>>>(kap, co[0], co[1], co[2], co[3], co[4], co[5], nx, ny, lam);
    if (!launch_ok()) return TRID_ERR_CUDA;
    if (uT != u0 && cudaMemcpyAsync(uT, u0, n * sizeof(T), cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        return launch_ok(), TRID_ERR_CUDA;
    const size_t mstride = l.mesh / sizeof(T);
    if (ckpt && cudaMemcpyAsync(ckpt, u0, n * sizeof(T), cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        return launch_ok(), TRID_ERR_CUDA;
    for (int t = 0; t < nsteps; ++t) {
        const trid_status s = v2_forward_step<T>(uT, dw, co, dims, scr, l.scratch, dt, st);
        if (s != TRID_OK) return s;
        if (ckpt && (t + 1) % every == 0 && t + 1 < nsteps) {
            T *dst = ckpt + size_t((t + 1) / every) * mstride;
            if (cudaMemcpyAsync(dst, uT, n * sizeof(T), cudaMemcpyDeviceToDevice, st) != cudaSuccess)
                return launch_ok(), TRID_ERR_CUDA;
        }
    }
    return TRID_OK;
}

template <typename T>
static trid_status v2_backward(const T *guT, T *gu0, T *gk, T *gcoef, const T *kap,
                               const int64_t *dims, T lam, int nsteps, int every, const T *ckpt,
                               char *ws, const V2Layout &l, trid_dtype dt, cudaStream_t st) {
    const int nx = int(dims[0]), ny = int(dims[1]);
    const size_t n = size_t(nx) * ny;
    const size_t ms = l.mesh / sizeof(T);  // elements between mesh arrays
    T *base = reinterpret_cast<T *>(ws);
    T *co[6];
    for (int k = 0; k < 6; ++k) co[k] = base + k * ms;
    T *tr = base + 6 * ms;           // transposed x (a, c), transposed y (a, c)
    const int K = every;
    // two sets of the segment's u, w, delta (K each): the next segment is
    // recomputed into one while the current one is run in reverse from the other
    T *Us[2], *Ws[2], *Ds[2];
    for (int b = 0; b < 2; ++b) {
        Us[b] = tr + 4 * ms + size_t(b) * 3 * K * ms;
        Ws[b] = Us[b] + size_t(K) * ms;
        Ds[b] = Ws[b] + size_t(K) * ms;
    }
    T *g = Us[0] + size_t(6) * K * ms;
    T *gn = g + ms;
    T *const gw = gn + ms;  // g_w and g_d of the current step (stored by its adjoint solves)
    T *const gd = gn + 2 * ms;
    T *G = gn + 3 * ms;     // 6 sums
    char *scr = ws + (6 + 4 + 6 * size_t(K) + 2 + 2 + 6) * l.mesh;
    char *scr2 = scr + l.scratch;
    dim3 g2, b2;
    grid2<T>(nx, ny, g2, b2);
    // the column-walking reverse kernel: V2_ROWS rows per thread
    const int64_t bands = (int64_t(ny) + V2_ROWS - 1) / V2_ROWS;
    const dim3 ga(unsigned((nx + 255) / 256), unsigned(bands < 65535 ? bands : 65535));
    k_v2_coef<T><<<g2, b2, 0, st>>>(kap, co[0], co[1], co[2], co[3], co[4], co[5], nx, ny, lam);
    k_v2_transpose<T><<<g2, b2, 0, st>>>(co[0], co[2], co[3], co[5], tr, tr + ms, tr + 2 * ms,
                                         tr + 3 * ms, nx, ny);
    if (!launch_ok()) return TRID_ERR_CUDA;
    // the six coefficient-gradient sums, or (no g_coef wanted) the two face sums
    if (cudaMemsetAsync(G, 0, (gcoef ? 6 : 2) * ms * sizeof(T), st) != cudaSuccess)
        return launch_ok(), TRID_ERR_CUDA;
    if (cudaMemcpyAsync(g, guT, n * sizeof(T), cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        return launch_ok(), TRID_ERR_CUDA;
    const int nseg = l.nseg;
    // Segments are recomputed on the library's auxiliary stream and run in
    // reverse on the caller's, ordered by events: the recomputation of segment
    // s - 1 overlaps the reverse sweep of segment s.  Event e_set: the set-up
    // above is done; e_rec[b]: set b holds a recomputed segment; e_rev[b]: the
    // reverse sweep that read set b is done (set b may be overwritten).  With
    // one segment, or without the auxiliary stream or events, everything runs
    // on the caller's stream.
    cudaStream_t sb = (nseg >= 2 && nsteps > 0) ? aux_stream() : nullptr;
    cudaEvent_t ev[5] = {};
    bool two = sb != nullptr;
    for (int k = 0; k < 5 && two; ++k)
        if (cudaEventCreateWithFlags(&ev[k], cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            two = false;
        }
    struct EventsGuard {
        cudaEvent_t *e;
        ~EventsGuard() {
            for (int k = 0; k < 5; ++k)
                if (e[k]) cudaEventDestroy(e[k]);
        }
    } guard{ev};
    cudaEvent_t e_set = ev[0], e_rec[2] = {ev[1], ev[2]}, e_rev[2] = {ev[3], ev[4]};
    if (two && (cudaEventRecord(e_set, st) != cudaSuccess ||
                cudaStreamWaitEvent(sb, e_set, 0) != cudaSuccess))
        return launch_ok(), TRID_ERR_CUDA;
    for (int idx = 0; idx < nseg && nsteps > 0; ++idx) {
        const int seg = nseg - 1 - idx;
        const int b = two ? (idx & 1) : 0;
        T *U = Us[b], *W = Ws[b], *D = Ds[b];
        const int t0 = seg * K;
        const int t1 = (t0 + K < nsteps) ? t0 + K : nsteps;
        const int L = t1 - t0;
        cudaStream_t rs = two ? sb : st;  // the recomputing stream
        char *rscr = two ? scr2 : scr;
        if (two && idx >= 2 && cudaStreamWaitEvent(sb, e_rev[b], 0) != cudaSuccess)
            return launch_ok(), TRID_ERR_CUDA;
        if (cudaMemcpyAsync(U, ckpt + size_t(seg) * ms, n * sizeof(T), cudaMemcpyDeviceToDevice,
                            rs) != cudaSuccess)
            return launch_ok(), TRID_ERR_CUDA;
        for (int q = 0; q < L; ++q) {
            const T *up = q > 0 ? U + size_t(q - 1) * ms : nullptr;
            const T *dp = q > 0 ? D + size_t(q - 1) * ms : nullptr;
            const trid_status s = v2_recompute_step<T>(up, dp, U + size_t(q) * ms,
                                                       W + size_t(q) * ms, D + size_t(q) * ms, co,
                                                       dims, rscr, l.scratch, dt, rs);
            if (s != TRID_OK) return s;
        }
        if (two && (cudaEventRecord(e_rec[b], sb) != cudaSuccess ||
                    cudaStreamWaitEvent(st, e_rec[b], 0) != cudaSuccess))
            return launch_ok(), TRID_ERR_CUDA;
        for (int q = L - 1; q >= 0; --q) {
            // g_w = Y^{-T} g, g_d = X^{-T} g_w, each stored into its own buffer
            // (g and g_w stay intact for the reverse stencil kernel)
            trid_status s = solve_into_ws(tr + 2 * ms, co[4], tr + 3 * ms, g, gw, dims, 2, 1, dt,
                                          scr, l.scratch, st);
            if (s != TRID_OK) return s;
            s = solve_into_ws(tr, co[1], tr + ms, gw, gd, dims, 2, 0, dt, scr, l.scratch, st);
            if (s != TRID_OK) return s;
            auto kern = gcoef ? k_v2_rhs_adj<T, true> : k_v2_rhs_adj<T, false>;
            if (!launch_pdl(kern, ga, b2, st, g, gd, gw, U + size_t(q) * ms, W + size_t(q) * ms,
                            D + size_t(q) * ms, co[0], co[2], co[3], co[5], G, gn, nx, ny, ms))
                return TRID_ERR_CUDA;
            T *tmp = g;
            g = gn;
            gn = tmp;
        }
        if (two && cudaEventRecord(e_rev[b], st) != cudaSuccess) return launch_ok(), TRID_ERR_CUDA;
    }
    if (cudaMemcpyAsync(gu0, g, n * sizeof(T), cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        return launch_ok(), TRID_ERR_CUDA;
    if (gcoef)
        k_v2_kappa<T><<<g2, b2, 0, st>>>(G, gk, nx, ny, lam, ms);
    else
        k_v2_kappa_faces<T><<<g2, b2, 0, st>>>(G, gk, nx, ny, lam, ms);
    if (!launch_ok()) return TRID_ERR_CUDA;
    if (gcoef) {
        for (int k = 0; k < 6; ++k)
            if (cudaMemcpyAsync(gcoef + size_t(k) * n, G + size_t(k) * ms, n * sizeof(T),
                                cudaMemcpyDeviceToDevice, st) != cudaSuccess)
                return launch_ok(), TRID_ERR_CUDA;
    }
    return TRID_OK;
}

}  // namespace trid

using namespace trid;

extern "C" size_t adi2v_workspace_bytes(const int64_t *dims, int nsteps, int every,
                                        trid_dtype dtype) {
    V2Layout l;
    if (!v2_layout(dims, nsteps, every, dtype, l)) return 0;
    return l.fwd > l.bwd ? l.fwd : l.bwd;
}

extern "C" size_t adi2v_checkpoint_bytes(const int64_t *dims, int nsteps, int every,
                                         trid_dtype dtype) {
    V2Layout l;
    if (!v2_layout(dims, nsteps, every, dtype, l)) return 0;
    return size_t(l.nseg) * l.mesh;
}

static trid_status v2_common(const int64_t *dims, int nsteps, int every, trid_dtype dtype,
                             double lambda, void *ws, size_t ws_bytes, size_t need_ws,
                             V2Layout &l) {
    if (!v2_layout(dims, nsteps, every, dtype, l)) return TRID_ERR_INVALID_ARG;
    if (!(lambda > 0.0) || lambda > 1e30) return TRID_ERR_INVALID_ARG;
    if (!ws || ws_bytes < need_ws) return TRID_ERR_ALLOC;
    if ((reinterpret_cast<uintptr_t>(ws) % 256) != 0) return TRID_ERR_MISALIGNED;
    return TRID_OK;
}

extern "C" trid_status adi2v_forward(const void *u0, void *uT, const void *kappa,
                                     const int64_t *dims, double lambda, int nsteps, int every,
                                     void *ckpt, size_t ckpt_bytes, trid_dtype dtype,
                                     void *workspace, size_t workspace_bytes,
                                     trid_stream_t stream) {
    trid::NvtxScope nvtx_scope("adi2v_forward");
    V2Layout l;
    if (!v2_layout(dims, nsteps, every, dtype, l)) return TRID_ERR_INVALID_ARG;
    trid_status s = v2_common(dims, nsteps, every, dtype, lambda, workspace, workspace_bytes,
                              l.fwd, l);
    if (s != TRID_OK) return s;
    if (!u0 || !uT || !kappa) return TRID_ERR_INVALID_ARG;
    if (ckpt && ckpt_bytes < size_t(l.nseg) * l.mesh) return TRID_ERR_ALLOC;
    if (ckpt && (reinterpret_cast<uintptr_t>(ckpt) % 256) != 0) return TRID_ERR_MISALIGNED;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    char *ws = static_cast<char *>(workspace);
    if (dtype == TRID_F32)
        return v2_forward<float>(static_cast<const float *>(u0), static_cast<float *>(uT),
                                 static_cast<const float *>(kappa), dims, float(lambda), nsteps,
                                 every, static_cast<float *>(ckpt), ws, l, dtype, st);
    return v2_forward<double>(static_cast<const double *>(u0), static_cast<double *>(uT),
                              static_cast<const double *>(kappa), dims, lambda, nsteps, every,
                              static_cast<double *>(ckpt), ws, l, dtype, st);
}

extern "C" trid_status adi2v_backward(const void *g_uT, void *g_u0, void *g_kappa, void *g_coef,
                                      const void *kappa, const int64_t *dims, double lambda,
                                      int nsteps, int every, const void *ckpt, size_t ckpt_bytes,
                                      trid_dtype dtype, void *workspace, size_t workspace_bytes,
                                      trid_stream_t stream) {
    trid::NvtxScope nvtx_scope("adi2v_backward");
    V2Layout l;
    if (!v2_layout(dims, nsteps, every, dtype, l)) return TRID_ERR_INVALID_ARG;
    trid_status s = v2_common(dims, nsteps, every, dtype, lambda, workspace, workspace_bytes,
                              l.bwd, l);
    if (s != TRID_OK) return s;
    if (!g_uT || !g_u0 || !g_kappa || !kappa || !ckpt) return TRID_ERR_INVALID_ARG;
    if (ckpt_bytes < size_t(l.nseg) * l.mesh) return TRID_ERR_ALLOC;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    char *ws = static_cast<char *>(workspace);
    if (dtype == TRID_F32)
        return v2_backward<float>(static_cast<const float *>(g_uT), static_cast<float *>(g_u0),
                                  static_cast<float *>(g_kappa), static_cast<float *>(g_coef),
                                  static_cast<const float *>(kappa), dims, float(lambda), nsteps,
                                  every, static_cast<const float *>(ckpt), ws, l, dtype, st);
    return v2_backward<double>(static_cast<const double *>(g_uT), static_cast<double *>(g_u0),
                               static_cast<double *>(g_kappa), static_cast<double *>(g_coef),
                               static_cast<const double *>(kappa), dims, lambda, nsteps, every,
                               static_cast<const double *>(ckpt), ws, l, dtype, st);
}
