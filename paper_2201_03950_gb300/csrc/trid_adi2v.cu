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
//   g_w = Y^{-T} g and g_d = X^{-T} g_w   (trid_solve_batch_adjoint, which
//        also gives the coefficient gradients -g_w delta_{p-nx}, ...),
//   g_d restricted to the interior, dL/du_t = g + (transposed stencil) g_d,
//   and the stencil adds g_d (u_p - u_{p-1}) to the gradient of a_p and
//   g_d (u_p - u_{p+1}) to that of c_p (y alike).
// The coefficient arrays do not change over the steps, so their gradients are
// summed over the steps and taken to kappa once at the end.
//
// Checkpointing: the forward keeps u every `every` steps; the backward
// recomputes each segment forward from its checkpoint (keeping u_t, w_t and
// delta_t of the segment) and then runs the segment's steps in reverse.
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/trid.h"
#include "trid_internal.h"

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

// Explicit part: d = lam (Lx + Ly) u on the interior, 0 on the boundary.
template <typename T>
__global__ void k_v2_rhs(const T *__restrict__ u, const T *__restrict__ ax,
                         const T *__restrict__ cx, const T *__restrict__ ay,
                         const T *__restrict__ cy, T *__restrict__ d, int nx, int ny) {
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

template <typename T>
__global__ void k_v2_add(const T *__restrict__ a, const T *__restrict__ b, T *__restrict__ out,
                         size_t n) {
    for (size_t p = size_t(blockIdx.x) * blockDim.x + threadIdx.x; p < n;
         p += size_t(gridDim.x) * blockDim.x)
        out[p] = a[p] + b[p];
}

// Reverse of the explicit part and of the identity path, plus the summed
// coefficient gradients:  gn = g + S^T gm  (gm = g_d on the interior),
// G_k += (step gradient k) + stencil term.  Gather form: point q collects the
// stencil rows p = q, q +- 1, q +- nx that read u_q.
template <typename T>
__global__ void k_v2_rhs_adj(const T *__restrict__ g, const T *__restrict__ gd,
                             const T *__restrict__ u, const T *__restrict__ ax,
                             const T *__restrict__ cx, const T *__restrict__ ay,
                             const T *__restrict__ cy, const T *__restrict__ sg, T *__restrict__ G,
                             T *__restrict__ gn, int nx, int ny, size_t n) {
    // n: element stride between the six arrays of sg and of G
    for (int j = blockIdx.y; j < ny; j += gridDim.y) {
        const int i = blockIdx.x * blockDim.x + threadIdx.x;
        if (i >= nx) continue;
        const size_t p = size_t(j) * nx + i;
        auto gm = [&](int ii, int jj) -> T {
            return (ii > 0 && ii < nx - 1 && jj > 0 && jj < ny - 1) ? gd[size_t(jj) * nx + ii]
                                                                     : T(0);
        };
        const T g0 = gm(i, j);
        T acc = g[p] + (ax[p] + cx[p] + ay[p] + cy[p]) * g0;
        if (i > 0) acc -= cx[p - 1] * gm(i - 1, j);
        if (i < nx - 1) acc -= ax[p + 1] * gm(i + 1, j);
        if (j > 0) acc -= cy[p - nx] * gm(i, j - 1);
        if (j < ny - 1) acc -= ay[p + nx] * gm(i, j + 1);
        gn[p] = acc;
        // summed coefficient gradients: ax, bx, cx, ay, by, cy
        const T uc = u[p];
        T sa = sg[p], sc = sg[2 * n + p], ta = sg[3 * n + p], tc = sg[5 * n + p];
        if (g0 != T(0)) {
            sa += g0 * (uc - u[p - 1]);
            sc += g0 * (uc - u[p + 1]);
            ta += g0 * (uc - u[p - nx]);
            tc += g0 * (uc - u[p + nx]);
        }
        G[p] += sa;
        G[n + p] += sg[n + p];
        G[2 * n + p] += sc;
        G[3 * n + p] += ta;
        G[4 * n + p] += sg[4 * n + p];
        G[5 * n + p] += tc;
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
    // coefficients 6, segment u/w/delta 3K, g, gn, g_w, g_d 4, step grads 6, sums 6
    l.bwd = (6 + 3 * K + 4 + 6 + 6) * l.mesh + l.scratch;
    l.nseg = nsteps == 0 ? 1 : (nsteps + every - 1) / every;
    return true;
}

template <typename T>
static void grid2(int nx, int ny, dim3 &g, dim3 &b) {
    b = dim3(256);
    g = dim3(unsigned((nx + 255) / 256), unsigned(ny < 65535 ? ny : 65535));
}

template <typename T>
static trid_status v2_forward_step(T *u, T *dw, const T *const co[6], const int64_t *dims,
                                   char *scr, size_t scr_bytes, trid_dtype dt, cudaStream_t st,
                                   T *w_keep = nullptr, T *delta_keep = nullptr,
                                   T *u_next = nullptr) {
    const int nx = int(dims[0]), ny = int(dims[1]);
    dim3 g, b;
    grid2<T>(nx, ny, g, b);
    T *w = w_keep ? w_keep : dw;
    k_v2_rhs<T><<<g, b, 0, st>>>(u, co[0], co[2], co[3], co[5], w, nx, ny);
    if (!launch_ok()) return TRID_ERR_CUDA;
    trid_status s = trid_solve_batch_ws(co[0], co[1], co[2], w, nullptr, dims, 2, 0, dt, scr,
                                        scr_bytes, st);
    if (s != TRID_OK) return s;
    if (!delta_keep) {
        // u += Y^{-1} w
        return trid_solve_batch_ws(co[3], co[4], co[5], w, u, dims, 2, 1, dt, scr, scr_bytes, st);
    }
    const size_t n = size_t(nx) * ny;
    if (cudaMemcpyAsync(delta_keep, w, n * sizeof(T), cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        return launch_ok(), TRID_ERR_CUDA;
    s = trid_solve_batch_ws(co[3], co[4], co[5], delta_keep, nullptr, dims, 2, 1, dt, scr,
                            scr_bytes, st);
    if (s != TRID_OK) return s;
    if (u_next) {
        k_v2_add<T><<<1024, 256, 0, st>>>(u, delta_keep, u_next, n);
        if (!launch_ok()) return TRID_ERR_CUDA;
    }
    return TRID_OK;
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
    const int K = every;
    T *U = base + 6 * ms;            // K states
    T *W = U + size_t(K) * ms;       // K
    T *D = W + size_t(K) * ms;       // K
    T *g = D + size_t(K) * ms;
    T *gn = g + ms, *gw = gn + ms, *gd = gw + ms;
    T *sg = gd + ms;                 // 6 step gradients (ax, bx, cx, ay, by, cy)
    T *G = sg + 6 * ms;              // 6 sums
    char *scr = ws + (6 + 3 * size_t(K) + 4 + 6 + 6) * l.mesh;
    dim3 g2, b2;
    grid2<T>(nx, ny, g2, b2);
    k_v2_coef<T><<<g2, b2, 0, st>>>(kap, co[0], co[1], co[2], co[3], co[4], co[5], nx, ny, lam);
    if (!launch_ok()) return TRID_ERR_CUDA;
    if (cudaMemsetAsync(G, 0, 6 * ms * sizeof(T), st) != cudaSuccess) return launch_ok(), TRID_ERR_CUDA;
    if (cudaMemcpyAsync(g, guT, n * sizeof(T), cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        return launch_ok(), TRID_ERR_CUDA;
    const int nseg = l.nseg;
    for (int seg = nseg - 1; seg >= 0 && nsteps > 0; --seg) {
        const int t0 = seg * K;
        const int t1 = (t0 + K < nsteps) ? t0 + K : nsteps;
        const int L = t1 - t0;
        if (cudaMemcpyAsync(U, ckpt + size_t(seg) * ms, n * sizeof(T), cudaMemcpyDeviceToDevice,
                            st) != cudaSuccess)
            return launch_ok(), TRID_ERR_CUDA;
        for (int q = 0; q < L; ++q) {
            T *un = (q + 1 < L) ? U + size_t(q + 1) * ms : nullptr;
            const trid_status s = v2_forward_step<T>(U + size_t(q) * ms, gd, co, dims, scr,
                                                     l.scratch, dt, st, W + size_t(q) * ms,
                                                     D + size_t(q) * ms, un);
            if (s != TRID_OK) return s;
        }
        for (int q = L - 1; q >= 0; --q) {
            trid_status s = trid_solve_batch_adjoint(co[3], co[4], co[5], D + size_t(q) * ms, g,
                                                     sg + 3 * ms, sg + 4 * ms, sg + 5 * ms, gw,
                                                     dims, 2, 1, dt, scr, l.scratch, st);
            if (s != TRID_OK) return s;
            s = trid_solve_batch_adjoint(co[0], co[1], co[2], W + size_t(q) * ms, gw, sg, sg + ms,
                                         sg + 2 * ms, gd, dims, 2, 0, dt, scr, l.scratch, st);
            if (s != TRID_OK) return s;
            k_v2_rhs_adj<T><<<g2, b2, 0, st>>>(g, gd, U + size_t(q) * ms, co[0], co[2], co[3],
                                                co[5], sg, G, gn, nx, ny, ms);
            if (!launch_ok()) return TRID_ERR_CUDA;
            T *tmp = g;
            g = gn;
            gn = tmp;
        }
    }
    if (cudaMemcpyAsync(gu0, g, n * sizeof(T), cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        return launch_ok(), TRID_ERR_CUDA;
    k_v2_kappa<T><<<g2, b2, 0, st>>>(G, gk, nx, ny, lam, ms);
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
