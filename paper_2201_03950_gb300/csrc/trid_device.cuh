// trid_device.cuh -- device building blocks shared by every solver kernel.
//
// The method (arXiv 2201.03950) solves many independent tridiagonal systems
//     a_i x_{i-1} + b_i x_i + c_i x_{i+1} = d_i         (Section 2)
// with the Thomas recurrence, and long systems with the tiled Thomas-PCR
// hybrid of Section 3.1.  On the GPU every system is cut into tiles of M
// consecutive rows, one tile per thread held in registers:
//
//  1. tile_reduce: the modified Thomas forward/backward pass of Section 3.1
//     over the tile writes every interior unknown as
//         x_i = dh_i - ah_i x_s - ch_i x_e          (s, e = tile ends)
//     and leaves two unit-diagonal "reduced" rows per tile:
//         S: as x_{s-1} + x_s + cs x_e     = ds
//         E: ae x_s     + x_e + ce x_{e+1} = de
//  2. group_solve: the reduced system of the tiles of one system, held by
//     G = 1..32 consecutive lanes (two rows per lane), is solved with warp
//     shuffles: one cyclic-reduction step folds S into E (one row per lane
//     over the unknowns x_e), log2(G) parallel-cyclic-reduction rounds
//     (Algorithm "pcr" of Section 2) solve for x_e, and x_s follows from S.
//  3. tile_substitute: interior unknowns from (x_s, x_e).
//
// Rows beyond a system's length are identity rows (a = c = d = 0, b = 1);
// they decouple because the last real row's c is forced to 0.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "trid_debug.cuh"

namespace trid {

// ---- reciprocal ------------------------------------------------------------
// FP32: the hardware approximate reciprocal (one MUFU op, ~1 ulp), which keeps
// the recurrence far inside the 1e-5 normwise tolerance.  FP64: IEEE division.
__device__ __forceinline__ float rcp(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ double rcp(double x) { return 1.0 / x; }

// ---- per-tile modified Thomas (Section 3.1) --------------------------------
// In: a, b, c, d rows of one tile (a of the system's first row and c of its
// last row already zeroed; padding rows are identity).  Out: a, c, d hold
// ah, ch, dh of the interior rows; S and E rows returned through refs.
template <typename T, int M>
__device__ __forceinline__ void tile_reduce(T (&a)[M], const T (&b)[M], T (&c)[M], T (&d)[M],
                                            T &as, T &cs, T &ds, T &ae, T &ce, T &de) {
    static_assert(M >= 2, "tile must hold at least two rows");
    // row 0 (tile start) and row 1, normalised by their diagonal
    const T r0 = rcp(b[0]);
    T a0 = a[0] * r0, c0 = c[0] * r0, d0 = d[0] * r0;
    const T r1 = rcp(b[1]);
    a[1] *= r1; c[1] *= r1; d[1] *= r1;
    if (M == 2) {
        as = a0; cs = c0; ds = d0;
        ae = a[1]; ce = c[1]; de = d[1];
        return;
    }
#pragma unroll
    for (int i = 2; i < M; ++i) {
        const T r = rcp(b[i] - a[i] * c[i - 1]);
        d[i] = r * (d[i] - a[i] * d[i - 1]);
        a[i] = -r * (a[i] * a[i - 1]);
        c[i] = r * c[i];
    }
#pragma unroll
    for (int i = M - 3; i >= 1; --i) {
        d[i] = d[i] - c[i] * d[i + 1];
        a[i] = a[i] - c[i] * a[i + 1];
        c[i] = -(c[i] * c[i + 1]);
    }
    // S row: substitute x_{s+1} = d1 - a1 x_s - c1 x_e into row 0, renormalise
    const T rb = rcp(T(1) - c0 * a[1]);
    as = a0 * rb;
    cs = -(c0 * c[1]) * rb;
    ds = (d0 - c0 * d[1]) * rb;
    ae = a[M - 1]; ce = c[M - 1]; de = d[M - 1];
}

template <typename T, int M>
__device__ __forceinline__ void tile_substitute(const T (&a)[M], const T (&c)[M], T (&d)[M],
                                                T xs, T xe) {
    if (M == 2) { d[0] = xs; d[1] = xe; return; }
#pragma unroll
    for (int i = 1; i < M - 1; ++i) d[i] = d[i] - a[i] * xs - c[i] * xe;
    d[0] = xs;
    d[M - 1] = xe;
}

// ---- reduced solve across G consecutive lanes -------------------------------
// Every lane of the warp must call this (full-warp shuffles).  `g` = the
// lane's index inside its group of G lanes (tile index of the system).
template <typename T, int G>
__device__ __forceinline__ void group_solve(T as, T cs, T ds, T ae, T ce, T de, int g,
                                            T &xs, T &xe) {
    constexpr unsigned FULL = 0xffffffffu;
    // fold S rows into E rows: x_s of this tile from own S row, x_s of the
    // next tile from the next lane's S row
    T nas = __shfl_down_sync(FULL, as, 1, G);
    T ncs = __shfl_down_sync(FULL, cs, 1, G);
    T nds = __shfl_down_sync(FULL, ds, 1, G);
    if (g + 1 >= G) { nas = T(0); ncs = T(0); nds = T(0); }
    // row over (x_{e,g-1}, x_{e,g}, x_{e,g+1})
    T ra = -(ae * as);
    T rdiag = T(1) - ae * cs - ce * nas;
    T rc = -(ce * ncs);
    T rd = de - ae * ds - ce * nds;
    {
        const T r = rcp(rdiag);
        ra *= r; rc *= r; rd *= r;
    }
    // parallel cyclic reduction over the G unit-diagonal rows.  Each round
    // squares the coupling of a diagonally dominant reduced system; once every
    // |ra|, |rc| of the warp is below 2^-(p+4) (p the significand bits), the
    // remaining rounds change no value by more than 1/16 ulp (normwise), and
    // the warp stops.
    constexpr float negligible = sizeof(T) == 4 ? 3.7252903e-09f : 6.9388939e-18f;
#pragma unroll
    for (int s = 1; s < G; s <<= 1) {
        if (G >= 8) {
            const float cpl = float(fmax(fabs(ra), fabs(rc)));
            const unsigned top = __reduce_max_sync(FULL, __float_as_uint(cpl));
            if (__uint_as_float(top) < negligible) break;
        }
        T am = __shfl_up_sync(FULL, ra, s, G);
        T cm = __shfl_up_sync(FULL, rc, s, G);
        T dm = __shfl_up_sync(FULL, rd, s, G);
        T ap = __shfl_down_sync(FULL, ra, s, G);
        T cp = __shfl_down_sync(FULL, rc, s, G);
        T dp = __shfl_down_sync(FULL, rd, s, G);
        if (g < s) { am = T(0); cm = T(0); dm = T(0); }
        if (g + s >= G) { ap = T(0); cp = T(0); dp = T(0); }
        const T r = rcp(T(1) - ra * cm - rc * ap);
        const T na = -r * (ra * am);
        const T nc = -r * (rc * cp);
        const T nd = r * (rd - ra * dm - rc * dp);
        ra = na; rc = nc; rd = nd;
    }
    xe = rd;
    T xprev = __shfl_up_sync(FULL, xe, 1, G);
    if (g == 0) xprev = T(0);
    xs = ds - as * xprev - cs * xe;
}

// ---- vector load/store helpers for contiguous tiles -------------------------
template <typename T> struct Vec16;
template <> struct Vec16<float> { using type = float4; static constexpr int n = 4; };
template <> struct Vec16<double> { using type = double2; static constexpr int n = 2; };

template <typename T, int M>
__device__ __forceinline__ void load_contig_vec(const T *__restrict__ p, T (&r)[M]) {
    using V = typename Vec16<T>::type;
    constexpr int W = Vec16<T>::n;
    static_assert(M % W == 0, "tile must be a whole number of 16-byte vectors");
    const V *pv = reinterpret_cast<const V *>(p);
#pragma unroll
    for (int k = 0; k < M / W; ++k) {
        V v = pv[k];
        const T *e = reinterpret_cast<const T *>(&v);
#pragma unroll
        for (int j = 0; j < W; ++j) r[k * W + j] = e[j];
    }
}

template <typename T, int M>
__device__ __forceinline__ void store_contig_vec(T *p, const T (&r)[M]) {
    using V = typename Vec16<T>::type;
    constexpr int W = Vec16<T>::n;
    V *pv = reinterpret_cast<V *>(p);
#pragma unroll
    for (int k = 0; k < M / W; ++k) {
        V v;
        T *e = reinterpret_cast<T *>(&v);
#pragma unroll
        for (int j = 0; j < W; ++j) e[j] = r[k * W + j];
        pv[k] = v;
    }
}

// Systems of a mesh axis: system s has its first element at
//   base(s) = (s % inner) + (s / inner) * inner * n
// and element i at base(s) + i * stride (stride == inner for mesh axes).
struct Lines {
    int64_t nsys;
    int64_t n;
    int64_t inner;
    int64_t stride;
    __host__ __device__ int64_t base(int64_t s) const {
        return (inner == 1) ? s * n : (s % inner) + (s / inner) * inner * n;
    }
};

}  // namespace trid
