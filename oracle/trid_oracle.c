/*
 * Reference (oracle) implementation of the batched tridiagonal solver and
 * the ADI heat-diffusion step of "High Throughput Multidimensional
 * Tridiagonal Systems Solvers on FPGAs" (arXiv 2201.03950).
 *
 * THIS IS TEST INFRASTRUCTURE.  It is plain, slow, single-threaded C in
 * IEEE binary64 (compile with -ffp-contract=off so that every product and
 * sum is rounded exactly as written).  Only the tests, the smoke check and the
 * CPU-baseline leg of the benchmark may load it.  It shares no code, header,
 * table or helper with the CUDA path, and the CUDA path never calls it.
 *
 * Problem statement (Section 2, eq. tdma-single / tdma-system):
 *     a_i x_{i-1} + b_i x_i + c_i x_{i+1} = d_i,   i = 0..N-1,
 * with a_0 = c_{N-1} = 0.  Every routine here treats a_0 and c_{N-1} as zero
 * WITHOUT reading them, so callers may leave garbage there.
 *
 * Pinning (each function is checked against something other than itself in
 * tests/test_oracle.py): dense Gaussian elimination and LAPACK on tiny systems,
 * exact rational elimination, Toeplitz eigenvector closed forms, manufactured
 * solutions, the residual invariant, the discrete heat-equation eigenmode decay
 * factor, agreement of three independent algorithms (Thomas, PCR, tiled
 * hybrid), the adjoint dot-product identity and central finite differences.
 * Parity pinned for every function: none is "parity unpinned".
 *
 * Return value of every function: 0 on success, -1 on a bad argument or a
 * failed allocation, -2 on an exact zero pivot.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Thomas algorithm -- Section 2, Algorithm "thomas".                         */
/*   forward:  d*_0 = d_0/b_0, c*_0 = c_0/b_0;                                */
/*             r = 1/(b_i - a_i c*_{i-1}); d*_i = r (d_i - a_i d*_{i-1});     */
/*             c*_i = r c_i                      for i = 1..N-1               */
/*   backward: x_{N-1} = d*_{N-1};  x_i = d*_i - c*_i x_{i+1}, i = N-2..0      */
/* Algorithm "thomas" leaves x_{N-1} = d*_{N-1} implicit (it overwrites d);   */
/* it is written out here.                                                    */
/* ------------------------------------------------------------------------ */
int orc_thomas(int64_t n, const double *a, const double *b, const double *c,
               const double *d, double *x)
{
    if (n < 1) return n == 0 ? 0 : -1;
    double *cs = (double *)malloc((size_t)n * sizeof(double));
    double *ds = (double *)malloc((size_t)n * sizeof(double));
    if (!cs || !ds) { free(cs); free(ds); return -1; }
    int rc = 0;
    if (b[0] == 0.0) { rc = -2; goto out; }
    ds[0] = d[0] / b[0];
    cs[0] = (n > 1 ? c[0] : 0.0) / b[0];
    for (int64_t i = 1; i < n; ++i) {
        double ci = (i == n - 1) ? 0.0 : c[i];
        double den = b[i] - a[i] * cs[i - 1];
        if (den == 0.0) { rc = -2; goto out; }
        double r = 1.0 / den;
        ds[i] = r * (d[i] - a[i] * ds[i - 1]);
        cs[i] = r * ci;
    }
    x[n - 1] = ds[n - 1];
    for (int64_t i = n - 2; i >= 0; --i) x[i] = ds[i] - cs[i] * x[i + 1];
out:
    free(cs); free(ds);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Parallel cyclic reduction -- Section 2, Algorithm "pcr".                   */
/* Rows are first normalised so that b_i = 1.  P is the smallest integer with */
/* 2^P >= N.  Round p (stride s = 2^{p-1}) updates every row from the values  */
/* of the previous round (Jacobi style, two buffers):                         */
/*   r  = 1 / (1 - a_i c_{i-s} - c_i a_{i+s})                                 */
/*   a' = -r a_i a_{i-s};  c' = -r c_i c_{i+s};                               */
/*   d' =  r (d_i - a_i d_{i-s} - c_i d_{i+s})                                */
/* Reading (the paper is silent): a neighbour index outside [0, N) stands for */
/* a row with a = c = d = 0, consistent with a_0 = c_{N-1} = 0.               */
/* After P rounds x_i = d_i.                                                  */
/* ------------------------------------------------------------------------ */
int orc_pcr(int64_t n, const double *a, const double *b, const double *c,
            const double *d, double *x)
{
    if (n < 1) return n == 0 ? 0 : -1;
    size_t sz = (size_t)n * sizeof(double);
    double *A0 = malloc(sz), *C0 = malloc(sz), *D0 = malloc(sz);
    double *A1 = malloc(sz), *C1 = malloc(sz), *D1 = malloc(sz);
    int rc = 0;
    if (!A0 || !C0 || !D0 || !A1 || !C1 || !D1) { rc = -1; goto out; }
    for (int64_t i = 0; i < n; ++i) {
        if (b[i] == 0.0) { rc = -2; goto out; }
        double ai = (i == 0) ? 0.0 : a[i];
        double ci = (i == n - 1) ? 0.0 : c[i];
        A0[i] = ai / b[i];
        C0[i] = ci / b[i];
        D0[i] = d[i] / b[i];
    }
    int P = 0;
    while (((int64_t)1 << P) < n) ++P;
    for (int p = 1; p <= P; ++p) {
        int64_t s = (int64_t)1 << (p - 1);
        for (int64_t i = 0; i < n; ++i) {
            double am = 0.0, cm = 0.0, dm = 0.0, ap = 0.0, cp = 0.0, dp = 0.0;
            if (i - s >= 0) { am = A0[i - s]; cm = C0[i - s]; dm = D0[i - s]; }
            if (i + s < n)  { ap = A0[i + s]; cp = C0[i + s]; dp = D0[i + s]; }
            double den = 1.0 - A0[i] * cm - C0[i] * ap;
            if (den == 0.0) { rc = -2; goto out; }
            double r = 1.0 / den;
            A1[i] = -r * (A0[i] * am);
            C1[i] = -r * (C0[i] * cp);
            D1[i] = r * (D0[i] - A0[i] * dm - C0[i] * dp);
        }
        double *t;
        t = A0; A0 = A1; A1 = t;
        t = C0; C0 = C1; C1 = t;
        t = D0; D0 = D1; D1 = t;
    }
    memcpy(x, D0, sz);
out:
    free(A0); free(C0); free(D0); free(A1); free(C1); free(D1);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Dense Gaussian elimination with partial pivoting: the textbook solution of */
/* A x = rhs for a general nonsingular n x n matrix (row-major).  Used only   */
/* as a brute-force check of the tridiagonal routines on tiny systems.        */
/* ------------------------------------------------------------------------ */
int orc_dense_solve(int64_t n, const double *A_in, const double *rhs, double *x)
{
    if (n < 1) return n == 0 ? 0 : -1;
    double *A = malloc((size_t)(n * n) * sizeof(double));
    double *y = malloc((size_t)n * sizeof(double));
    if (!A || !y) { free(A); free(y); return -1; }
    memcpy(A, A_in, (size_t)(n * n) * sizeof(double));
    memcpy(y, rhs, (size_t)n * sizeof(double));
    int rc = 0;
    for (int64_t k = 0; k < n; ++k) {
        int64_t piv = k;
        double best = A[k * n + k] < 0 ? -A[k * n + k] : A[k * n + k];
        for (int64_t r = k + 1; r < n; ++r) {
            double v = A[r * n + k] < 0 ? -A[r * n + k] : A[r * n + k];
            if (v > best) { best = v; piv = r; }
        }
        if (best == 0.0) { rc = -2; goto out; }
        if (piv != k) {
            for (int64_t j = 0; j < n; ++j) {
                double t = A[k * n + j]; A[k * n + j] = A[piv * n + j]; A[piv * n + j] = t;
            }
            double t = y[k]; y[k] = y[piv]; y[piv] = t;
        }
        for (int64_t r = k + 1; r < n; ++r) {
            double f = A[r * n + k] / A[k * n + k];
            if (f == 0.0) continue;
            for (int64_t j = k; j < n; ++j) A[r * n + j] -= f * A[k * n + j];
            y[r] -= f * y[k];
        }
    }
    for (int64_t k = n - 1; k >= 0; --k) {
        double s = y[k];
        for (int64_t j = k + 1; j < n; ++j) s -= A[k * n + j] * x[j];
        x[k] = s / A[k * n + k];
    }
out:
    free(A); free(y);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Tiled hybrid (Section 3.1, eqs. thomasthomas / thomaspcr).                 */
/* The system is cut into tiles [s, e].  A modified Thomas pass over a tile   */
/* expresses every interior unknown through the tile's own end unknowns:      */
/*     x_i = dh_i - ah_i x_s - ch_i x_e ,   s < i < e.                        */
/*   forward,  rows s and s+1 normalised by b; for i = s+2..e:                */
/*       r = 1/(b_i - a_i ch_{i-1}); ah_i = -r a_i ah_{i-1};                  */
/*       ch_i = r c_i;  dh_i = r (d_i - a_i dh_{i-1})                         */
/*   backward, for i = e-2..s+1:                                              */
/*       dh_i -= ch_i dh_{i+1}; ah_i -= ch_i ah_{i+1}; ch_i = -ch_i ch_{i+1}  */
/* Row e then reads  ah_e x_s + x_e + ch_e x_{e+1} = dh_e  and row s, after   */
/* substituting x_{s+1}, reads                                               */
/*     ah_s x_{s-1} + (1 - ch_s ah_{s+1}) x_s - ch_s ch_{s+1} x_e             */
/*         = dh_s - ch_s dh_{s+1}.                                            */
/* Over the unknowns (x_{s_0}, x_{e_0}, x_{s_1}, x_{e_1}, ...) these rows     */
/* form a tridiagonal "reduced" system of size 2t, solved here with Thomas    */
/* (use_pcr = 0, the Thomas-Thomas variant) or PCR (use_pcr = 1, the          */
/* Thomas-PCR variant).  The interior is then substituted back.               */
/* Readings (the paper is silent): tiles have length m except the last, which */
/* takes the remainder; a remainder shorter than 3 is merged into the tile    */
/* before it.  Systems with n < 3 are solved by the Thomas routine directly.  */
/* ------------------------------------------------------------------------ */
int orc_tiled(int64_t n, int64_t m, int use_pcr, const double *a,
              const double *b, const double *c, const double *d, double *x)
{
    if (n < 0 || m < 3) return -1;
    if (n < 3) return orc_thomas(n, a, b, c, d, x);
    int64_t t = n / m;
    if (t < 1) t = 1;
    int64_t rem = n - t * m;
    /* tile k covers [k*m, k*m + m - 1]; the last covers up to n-1 */
    if (rem >= 3) t += 1;
    size_t sz = (size_t)n * sizeof(double);
    size_t rz = (size_t)(2 * t) * sizeof(double);
    double *ah = malloc(sz), *ch = malloc(sz), *dh = malloc(sz);
    double *ra = malloc(rz), *rb = malloc(rz), *rc_ = malloc(rz), *rd = malloc(rz), *rx = malloc(rz);
    int rc = 0;
    if (!ah || !ch || !dh || !ra || !rb || !rc_ || !rd || !rx) { rc = -1; goto out; }
    for (int64_t k = 0; k < t; ++k) {
        int64_t s = k * m;
        int64_t e = (k == t - 1) ? n - 1 : s + m - 1;
        /* forward */
        for (int64_t i = s; i <= s + 1; ++i) {
            if (b[i] == 0.0) { rc = -2; goto out; }
            double ai = (i == 0) ? 0.0 : a[i];
            double ci = (i == n - 1) ? 0.0 : c[i];
            ah[i] = ai / b[i];
            ch[i] = ci / b[i];
            dh[i] = d[i] / b[i];
        }
        for (int64_t i = s + 2; i <= e; ++i) {
            double ci = (i == n - 1) ? 0.0 : c[i];
            double den = b[i] - a[i] * ch[i - 1];
            if (den == 0.0) { rc = -2; goto out; }
            double r = 1.0 / den;
            ah[i] = -r * (a[i] * ah[i - 1]);
            ch[i] = r * ci;
            dh[i] = r * (d[i] - a[i] * dh[i - 1]);
        }
        /* backward */
        for (int64_t i = e - 2; i >= s + 1; --i) {
            dh[i] = dh[i] - ch[i] * dh[i + 1];
            ah[i] = ah[i] - ch[i] * ah[i + 1];
            ch[i] = -(ch[i] * ch[i + 1]);
        }
        /* reduced rows 2k (tile start) and 2k+1 (tile end) */
        ra[2 * k] = ah[s];
        rb[2 * k] = 1.0 - ch[s] * ah[s + 1];
        rc_[2 * k] = -(ch[s] * ch[s + 1]);
        rd[2 * k] = dh[s] - ch[s] * dh[s + 1];
        ra[2 * k + 1] = ah[e];
        rb[2 * k + 1] = 1.0;
        rc_[2 * k + 1] = ch[e];
        rd[2 * k + 1] = dh[e];
    }
    rc = use_pcr ? orc_pcr(2 * t, ra, rb, rc_, rd, rx)
                 : orc_thomas(2 * t, ra, rb, rc_, rd, rx);
    if (rc) goto out;
    for (int64_t k = 0; k < t; ++k) {
        int64_t s = k * m;
        int64_t e = (k == t - 1) ? n - 1 : s + m - 1;
        double xs = rx[2 * k], xe = rx[2 * k + 1];
        x[s] = xs;
        x[e] = xe;
        for (int64_t i = s + 1; i <= e - 1; ++i) x[i] = dh[i] - ah[i] * xs - ch[i] * xe;
    }
out:
    free(ah); free(ch); free(dh); free(ra); free(rb); free(rc_); free(rd); free(rx);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* A batch of nsys independent contiguous systems of length n each (system k  */
/* occupies [k*n, (k+1)*n)), solved one after another with orc_thomas.        */
/* ------------------------------------------------------------------------ */
int orc_thomas_lines(int64_t nsys, int64_t n, const double *a, const double *b,
                     const double *c, const double *d, double *x)
{
    for (int64_t k = 0; k < nsys; ++k) {
        int rc = orc_thomas(n, a + k * n, b + k * n, c + k * n, d + k * n, x + k * n);
        if (rc) return rc;
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Systems laid along one axis of a 1D/2D/3D mesh (Section 2.1).  The mesh is */
/* column-major: element (i0, i1, i2) sits at i0 + n0 (i1 + n1 i2).  For      */
/* solve_dim k there are prod(dims)/n_k systems of length n_k, element i of a */
/* system sitting at base + i * stride_k.  accumulate = 0 writes x into out;  */
/* accumulate = 1 adds x into out (the "u = u + d" update of Algorithm adi).  */
/* ------------------------------------------------------------------------ */
int orc_solve_mesh(const double *a, const double *b, const double *c,
                   const double *d, double *out, const int64_t *dims, int ndim,
                   int solve_dim, int accumulate)
{
    if (ndim < 1 || ndim > 3 || solve_dim < 0 || solve_dim >= ndim) return -1;
    int64_t n3[3] = {1, 1, 1};
    for (int k = 0; k < ndim; ++k) { if (dims[k] < 0) return -1; n3[k] = dims[k]; }
    int64_t stride[3] = {1, n3[0], n3[0] * n3[1]};
    int64_t n = n3[solve_dim];
    int64_t st = stride[solve_dim];
    if (n == 0) return 0;
    /* the two axes that enumerate systems */
    int o1 = (solve_dim == 0) ? 1 : 0;
    int o2 = (solve_dim == 2) ? 1 : 2;
    size_t sz = (size_t)n * sizeof(double);
    double *la = malloc(sz), *lb = malloc(sz), *lc = malloc(sz), *ld = malloc(sz), *lx = malloc(sz);
    int rc = 0;
    if (!la || !lb || !lc || !ld || !lx) { rc = -1; goto out; }
    for (int64_t j2 = 0; j2 < n3[o2]; ++j2) {
        for (int64_t j1 = 0; j1 < n3[o1]; ++j1) {
            int64_t base = j1 * stride[o1] + j2 * stride[o2];
            for (int64_t i = 0; i < n; ++i) {
                int64_t p = base + i * st;
                la[i] = a[p]; lb[i] = b[p]; lc[i] = c[p]; ld[i] = d[p];
            }
            rc = orc_thomas(n, la, lb, lc, ld, lx);
            if (rc) goto out;
            for (int64_t i = 0; i < n; ++i) {
                int64_t p = base + i * st;
                if (accumulate) out[p] += lx[i]; else out[p] = lx[i];
            }
        }
    }
out:
    free(la); free(lb); free(lc); free(ld); free(lx);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Binary32 twin of orc_solve_mesh (Algorithm "thomas" per system, Section    */
/* 2.1 line enumeration), every operation rounded to float.  It exists only   */
/* as the like-for-like (FP32) CPU baseline of the benchmark; the FP64        */
/* routines above remain the reference the GPU path is checked against.      */
/* ------------------------------------------------------------------------ */
static int thomas_f32(int64_t n, const float *a, const float *b, const float *c,
                      const float *d, float *cp, float *dp, float *x)
{
    if (b[0] == 0.0f) return -2;
    dp[0] = d[0] / b[0];
    cp[0] = (n > 1 ? c[0] : 0.0f) / b[0];
    for (int64_t i = 1; i < n; ++i) {
        float ci = (i == n - 1) ? 0.0f : c[i];
        float den = b[i] - a[i] * cp[i - 1];
        if (den == 0.0f) return -2;
        float r = 1.0f / den;
        dp[i] = r * (d[i] - a[i] * dp[i - 1]);
        cp[i] = r * ci;
    }
    x[n - 1] = dp[n - 1];
    for (int64_t i = n - 2; i >= 0; --i) x[i] = dp[i] - cp[i] * x[i + 1];
    return 0;
}

int orc_solve_mesh_f32(const float *a, const float *b, const float *c, const float *d,
                       float *out, const int64_t *dims, int ndim, int solve_dim)
{
    if (ndim < 1 || ndim > 3 || solve_dim < 0 || solve_dim >= ndim) return -1;
    int64_t n3[3] = {1, 1, 1};
    for (int k = 0; k < ndim; ++k) { if (dims[k] < 0) return -1; n3[k] = dims[k]; }
    int64_t stride[3] = {1, n3[0], n3[0] * n3[1]};
    int64_t n = n3[solve_dim], st = stride[solve_dim];
    if (n == 0) return 0;
    int o1 = (solve_dim == 0) ? 1 : 0;
    int o2 = (solve_dim == 2) ? 1 : 2;
    size_t sz = (size_t)n * sizeof(float);
    float *la = malloc(sz), *lb = malloc(sz), *lc = malloc(sz), *ld = malloc(sz);
    float *lx = malloc(sz), *cp = malloc(sz), *dp = malloc(sz);
    int rc = 0;
    if (!la || !lb || !lc || !ld || !lx || !cp || !dp) { rc = -1; goto out; }
    for (int64_t j2 = 0; j2 < n3[o2]; ++j2) {
        for (int64_t j1 = 0; j1 < n3[o1]; ++j1) {
            int64_t base = j1 * stride[o1] + j2 * stride[o2];
            for (int64_t i = 0; i < n; ++i) {
                int64_t p = base + i * st;
                la[i] = a[p]; lb[i] = b[p]; lc[i] = c[p]; ld[i] = d[p];
            }
            rc = thomas_f32(n, la, lb, lc, ld, cp, dp, lx);
            if (rc) goto out;
            for (int64_t i = 0; i < n; ++i) out[base + i * st] = lx[i];
        }
    }
out:
    free(la); free(lb); free(lc); free(ld); free(lx); free(cp); free(dp);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* ADI heat diffusion, Section 4.1, Algorithm adi, in delta form:             */
/*   1. d = lambda * (sum of the 2*ndim axis neighbours - 2*ndim*u) at        */
/*      interior nodes, d = 0 on boundary nodes (the explicit RHS stencil,    */
/*      7-point in 3D, 5-point in 2D);                                        */
/*   2. solve along x, then y, then z, each in place on d, with the constant  */
/*      operator tridiag(-lambda, 1 + 2 lambda, -lambda) on interior rows and */
/*      identity rows (a = c = 0, b = 1) at the two Dirichlet boundary nodes; */
/*   3. u = u + d.                                                            */
/* Readings: Algorithm "adi" prints garbled coefficients (a = c = -gamma/2,  */
/* b = gamma); they are read as a = c = -lambda, b = 1 + 2 lambda.  The       */
/* boundary is Dirichlet zero (boundary nodes never change).  ndim is 2 or 3. */
/* ------------------------------------------------------------------------ */
int orc_adi(double *u, const int64_t *dims, int ndim, double lambda, int nsteps)
{
    if (ndim < 2 || ndim > 3 || nsteps < 0) return -1;
    int64_t n3[3] = {1, 1, 1};
    for (int k = 0; k < ndim; ++k) { if (dims[k] < 1) return -1; n3[k] = dims[k]; }
    int64_t total = n3[0] * n3[1] * n3[2];
    int64_t stride[3] = {1, n3[0], n3[0] * n3[1]};
    int64_t nmax = n3[0];
    if (n3[1] > nmax) nmax = n3[1];
    if (n3[2] > nmax) nmax = n3[2];
    double *dd = malloc((size_t)total * sizeof(double));
    size_t lz = (size_t)nmax * sizeof(double);
    double *la = malloc(lz), *lb = malloc(lz), *lc = malloc(lz), *ld = malloc(lz), *lx = malloc(lz);
    int rc = 0;
    if (!dd || !la || !lb || !lc || !ld || !lx) { rc = -1; goto out; }
    for (int step = 0; step < nsteps; ++step) {
        /* 1. explicit RHS */
        for (int64_t k = 0; k < n3[2]; ++k)
            for (int64_t j = 0; j < n3[1]; ++j)
                for (int64_t i = 0; i < n3[0]; ++i) {
                    int64_t p = i + stride[1] * j + stride[2] * k;
                    int interior = i > 0 && i < n3[0] - 1 && j > 0 && j < n3[1] - 1;
                    if (ndim == 3) interior = interior && k > 0 && k < n3[2] - 1;
                    if (!interior) { dd[p] = 0.0; continue; }
                    double s = u[p - 1] + u[p + 1] + u[p - stride[1]] + u[p + stride[1]];
                    if (ndim == 3) s += u[p - stride[2]] + u[p + stride[2]];
                    dd[p] = lambda * (s - 2.0 * ndim * u[p]);
                }
        /* 2. implicit solves along x, y (and z), in place on d */
        for (int ax = 0; ax < ndim; ++ax) {
            int64_t n = n3[ax], st = stride[ax];
            for (int64_t i = 0; i < n; ++i) {
                int bnd = (i == 0 || i == n - 1);
                la[i] = bnd ? 0.0 : -lambda;
                lb[i] = bnd ? 1.0 : 1.0 + 2.0 * lambda;
                lc[i] = bnd ? 0.0 : -lambda;
            }
            int o1 = (ax == 0) ? 1 : 0;
            int o2 = (ax == 2) ? 1 : 2;
            for (int64_t j2 = 0; j2 < n3[o2]; ++j2)
                for (int64_t j1 = 0; j1 < n3[o1]; ++j1) {
                    int64_t base = j1 * stride[o1] + j2 * stride[o2];
                    for (int64_t i = 0; i < n; ++i) ld[i] = dd[base + i * st];
                    rc = orc_thomas(n, la, lb, lc, ld, lx);
                    if (rc) goto out;
                    for (int64_t i = 0; i < n; ++i) dd[base + i * st] = lx[i];
                }
        }
        /* 3. accumulate */
        for (int64_t p = 0; p < total; ++p) u[p] += dd[p];
    }
out:
    free(dd); free(la); free(lb); free(lc); free(ld); free(lx);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Variable-length batch: system k occupies [offsets[k], offsets[k+1]).       */
/* ------------------------------------------------------------------------ */
int orc_solve_varlen(const double *a, const double *b, const double *c,
                     const double *d, double *x, const int64_t *offsets,
                     int64_t nsys)
{
    for (int64_t k = 0; k < nsys; ++k) {
        int64_t s = offsets[k], n = offsets[k + 1] - offsets[k];
        if (n < 0) return -1;
        int rc = orc_thomas(n, a + s, b + s, c + s, d + s, x + s);
        if (rc) return rc;
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Adjoint of one solve x = A^{-1} d.  Given g_x = dL/dx:                     */
/*   g_d = A^{-T} g_x, where A^T has sub-diagonal c_{i-1}, diagonal b_i and  */
/*   super-diagonal a_{i+1};                                                  */
/*   g_a_i = -g_d_i x_{i-1},  g_b_i = -g_d_i x_i,  g_c_i = -g_d_i x_{i+1},     */
/* with g_a_0 = g_c_{N-1} = 0 (those entries are not part of A).              */
/* ------------------------------------------------------------------------ */
int orc_adjoint(int64_t n, const double *a, const double *b, const double *c,
                const double *x, const double *gx, double *ga, double *gb,
                double *gc, double *gd)
{
    if (n < 1) return n == 0 ? 0 : -1;
    size_t sz = (size_t)n * sizeof(double);
    double *ta = malloc(sz), *tc = malloc(sz);
    if (!ta || !tc) { free(ta); free(tc); return -1; }
    for (int64_t i = 0; i < n; ++i) {
        ta[i] = (i == 0) ? 0.0 : c[i - 1];
        tc[i] = (i == n - 1) ? 0.0 : a[i + 1];
    }
    int rc = orc_thomas(n, ta, b, tc, gx, gd);
    free(ta); free(tc);
    if (rc) return rc;
    for (int64_t i = 0; i < n; ++i) {
        ga[i] = (i == 0) ? 0.0 : -gd[i] * x[i - 1];
        gb[i] = -gd[i] * x[i];
        gc[i] = (i == n - 1) ? 0.0 : -gd[i] * x[i + 1];
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Variable-diffusivity 2D ADI and its gradient.                             */
/*                                                                          */
/* The ADI step of Section 4.1 (Algorithm "adi", delta form, Dirichlet      */
/* boundary) with the constant lambda replaced by lambda * kappa at the cell */
/* faces.  The paper has no variable-coefficient form; the reading used     */
/* here: face values are arithmetic means of the two nodes,                 */
/*   kx_p = (kappa_p + kappa_{p+1}) / 2,  ky_p = (kappa_p + kappa_{p+nx})/2, */
/* and the x operator of a line has, on rows 0 < i < nx-1,                  */
/*   a_p = -lambda kx_{p-1},  c_p = -lambda kx_p,  b_p = 1 - a_p - c_p,      */
/* identity rows at i = 0 and i = nx-1 (y alike, stride nx).  A step is     */
/*   d_p = -c_p (u_{p+1} - u_p) + a_p (u_p - u_{p-1})    (x part)            */
/*         -c'_p (u_{p+nx} - u_p) + a'_p (u_p - u_{p-nx}) (y part)           */
/* at interior points (0 on the boundary), w = X^{-1} d, delta = Y^{-1} w,   */
/* u <- u + delta.  With kappa = 1 this is orc_adi in 2D.                    */
/* ------------------------------------------------------------------------ */
static void v2_coef(const double *kappa, int64_t nx, int64_t ny, double lam,
                    double *ax, double *bx, double *cx, double *ay, double *by, double *cy)
{
    for (int64_t j = 0; j < ny; ++j)
        for (int64_t i = 0; i < nx; ++i) {
            int64_t p = i + nx * j;
            if (i == 0 || i == nx - 1) { ax[p] = 0.0; bx[p] = 1.0; cx[p] = 0.0; }
            else {
                double kl = 0.5 * (kappa[p - 1] + kappa[p]);
                double kr = 0.5 * (kappa[p] + kappa[p + 1]);
                ax[p] = -lam * kl; cx[p] = -lam * kr; bx[p] = 1.0 - ax[p] - cx[p];
            }
            if (j == 0 || j == ny - 1) { ay[p] = 0.0; by[p] = 1.0; cy[p] = 0.0; }
            else {
                double kl = 0.5 * (kappa[p - nx] + kappa[p]);
                double kr = 0.5 * (kappa[p] + kappa[p + nx]);
                ay[p] = -lam * kl; cy[p] = -lam * kr; by[p] = 1.0 - ay[p] - cy[p];
            }
        }
}

static int v2_interior(int64_t i, int64_t j, int64_t nx, int64_t ny)
{
    return i > 0 && i < nx - 1 && j > 0 && j < ny - 1;
}

/* Solve along x (axis 0, stride 1) or y (axis 1, stride nx) on every line. */
static int v2_solve_lines(int axis, int64_t nx, int64_t ny, const double *a, const double *b,
                          const double *c, const double *d, double *x)
{
    int64_t n = axis == 0 ? nx : ny, nl = axis == 0 ? ny : nx;
    int64_t st = axis == 0 ? 1 : nx, ls = axis == 0 ? nx : 1;
    size_t sz = (size_t)n * sizeof(double);
    double *la = malloc(sz), *lb = malloc(sz), *lc = malloc(sz), *ld = malloc(sz), *lx = malloc(sz);
    int rc = (la && lb && lc && ld && lx) ? 0 : -1;
    for (int64_t l = 0; l < nl && rc == 0; ++l)
        for (int64_t k = 0; k < n; ++k) {
            int64_t p = l * ls + k * st;
            la[k] = a[p]; lb[k] = b[p]; lc[k] = c[p]; ld[k] = d[p];
            if (k == n - 1) {
                rc = orc_thomas(n, la, lb, lc, ld, lx);
                for (int64_t q = 0; q < n && rc == 0; ++q) x[l * ls + q * st] = lx[q];
            }
        }
    free(la); free(lb); free(lc); free(ld); free(lx);
    return rc;
}

/* One step from u: d, w = X^{-1} d, delta = Y^{-1} w (u is not modified). */
static int v2_step(const double *u, int64_t nx, int64_t ny, const double *co[6], double *d,
                   double *w, double *delta)
{
    const double *ax = co[0], *bx = co[1], *cx = co[2], *ay = co[3], *by = co[4], *cy = co[5];
    for (int64_t j = 0; j < ny; ++j)
        for (int64_t i = 0; i < nx; ++i) {
            int64_t p = i + nx * j;
            if (!v2_interior(i, j, nx, ny)) { d[p] = 0.0; continue; }
            d[p] = -cx[p] * (u[p + 1] - u[p]) + ax[p] * (u[p] - u[p - 1])
                 - cy[p] * (u[p + nx] - u[p]) + ay[p] * (u[p] - u[p - nx]);
        }
    int rc = v2_solve_lines(0, nx, ny, ax, bx, cx, d, w);
    if (rc == 0) rc = v2_solve_lines(1, nx, ny, ay, by, cy, w, delta);
    return rc;
}

int orc_adi2v(double *u, const double *kappa, const int64_t *dims, double lam, int nsteps)
{
    if (!dims || dims[0] < 1 || dims[1] < 1 || nsteps < 0) return -1;
    int64_t nx = dims[0], ny = dims[1], n = nx * ny;
    double *buf = malloc((size_t)n * 9 * sizeof(double));
    if (!buf) return -1;
    double *co[6];
    for (int k = 0; k < 6; ++k) co[k] = buf + (size_t)k * n;
    double *d = buf + 6 * n, *w = buf + 7 * n, *delta = buf + 8 * n;
    v2_coef(kappa, nx, ny, lam, co[0], co[1], co[2], co[3], co[4], co[5]);
    int rc = 0;
    for (int t = 0; t < nsteps && rc == 0; ++t) {
        rc = v2_step(u, nx, ny, (const double **)co, d, w, delta);
        for (int64_t p = 0; p < n && rc == 0; ++p) u[p] += delta[p];
    }
    free(buf);
    return rc;
}

/* Gradient of L = mean((u_T - target)^2) with respect to u_0 and kappa,    */
/* by reverse mode over stored states.  Per step, with g = dL/du_{t+1}:      */
/*   g_w = Y^{-T} g, g_d = X^{-T} g_w (orc_adjoint, which also returns the  */
/*   coefficient gradients -g_w delta_{p-nx} ... and -g_d w_{p-1} ...);      */
/*   g_d is zero off the interior (d is fixed to 0 there);                  */
/*   dL/du_t = g + (transposed stencil of d) g_d;                           */
/*   the stencil adds g_d (u_p - u_{p-1}) to the gradient of a_p and        */
/*   g_d (u_p - u_{p+1}) to that of c_p (y alike).                          */
/* The coefficient gradients summed over the steps (raw, per array, when    */
/* g_coef is not NULL: ax, bx, cx, ay, by, cy) are then taken to the faces  */
/* (a_p = -lam kx_{p-1}, c_p = -lam kx_p, b_p = 1 + lam (kx_{p-1} + kx_p))    */
/* and to the nodes (each face is the mean of its two nodes).                */
/* ------------------------------------------------------------------------ */
int orc_adi2v_grad(const double *u0, const double *kappa, const double *target,
                   const int64_t *dims, double lam, int nsteps, double *loss,
                   double *g_u0, double *g_kappa, double *g_coef)
{
    if (!dims || dims[0] < 1 || dims[1] < 1 || nsteps < 0) return -1;
    int64_t nx = dims[0], ny = dims[1], n = nx * ny;
    size_t T = (size_t)nsteps;
    double *st = malloc((size_t)n * (3 * T + 1) * sizeof(double));
    double *buf = malloc((size_t)n * 20 * sizeof(double));
    int64_t lmax = nx > ny ? nx : ny;
    double *lv = malloc((size_t)lmax * 9 * sizeof(double));
    if (!st || !buf || !lv) { free(st); free(buf); free(lv); return -1; }
    double *co[6], *G[6];
    for (int k = 0; k < 6; ++k) { co[k] = buf + (size_t)k * n; G[k] = buf + (size_t)(6 + k) * n; }
    double *d = buf + 12 * n, *g = buf + 13 * n, *gw = buf + 14 * n, *gd = buf + 15 * n;
    double *gu = buf + 16 * n, *gk = buf + 17 * n, *gkx = buf + 18 * n, *gky = buf + 19 * n;
    v2_coef(kappa, nx, ny, lam, co[0], co[1], co[2], co[3], co[4], co[5]);
    for (size_t q = 0; q < (size_t)n * 6; ++q) G[0][q] = 0.0;
    /* forward, keeping u_t, w_t, delta_t */
    double *U = st, *W = st + (size_t)n * (T + 1), *D = st + (size_t)n * (2 * T + 1);
    memcpy(U, u0, (size_t)n * sizeof(double));
    int rc = 0;
    for (size_t t = 0; t < T && rc == 0; ++t) {
        rc = v2_step(U + t * n, nx, ny, (const double **)co, d, W + t * n, D + t * n);
        for (int64_t p = 0; p < n; ++p) U[(t + 1) * n + p] = U[t * n + p] + D[t * n + p];
    }
    if (rc) goto out;
    double L = 0.0;
    for (int64_t p = 0; p < n; ++p) {
        double r = U[T * n + p] - target[p];
        L += r * r;
        g[p] = 2.0 * r / (double)n;
    }
    if (loss) *loss = L / (double)n;
    for (size_t tt = T; tt-- > 0 && rc == 0;) {
        const double *u = U + tt * n, *w = W + tt * n, *dl = D + tt * n;
        /* y lines: g_w = Y^{-T} g, coefficient gradients with x = delta */
        for (int64_t i = 0; i < nx && rc == 0; ++i) {
            double *la = lv, *lb = lv + lmax, *lc = lv + 2 * lmax, *lx = lv + 3 * lmax;
            double *lg = lv + 4 * lmax, *oa = lv + 5 * lmax, *ob = lv + 6 * lmax, *oc = lv + 7 * lmax;
            double *lgd = lv + 8 * lmax;
            for (int64_t j = 0; j < ny; ++j) {
                int64_t p = i + nx * j;
                la[j] = co[3][p]; lb[j] = co[4][p]; lc[j] = co[5][p]; lx[j] = dl[p]; lg[j] = g[p];
            }
            rc = orc_adjoint(ny, la, lb, lc, lx, lg, oa, ob, oc, lgd);
            for (int64_t j = 0; j < ny && rc == 0; ++j) {
                int64_t p = i + nx * j;
                G[3][p] += oa[j]; G[4][p] += ob[j]; G[5][p] += oc[j]; gw[p] = lgd[j];
            }
        }
        /* x lines: g_d = X^{-T} g_w, with x = w */
        for (int64_t j = 0; j < ny && rc == 0; ++j) {
            double *la = lv, *lb = lv + lmax, *lc = lv + 2 * lmax, *lx = lv + 3 * lmax;
            double *lg = lv + 4 * lmax, *oa = lv + 5 * lmax, *ob = lv + 6 * lmax, *oc = lv + 7 * lmax;
            double *lgd = lv + 8 * lmax;
            for (int64_t i = 0; i < nx; ++i) {
                int64_t p = i + nx * j;
                la[i] = co[0][p]; lb[i] = co[1][p]; lc[i] = co[2][p]; lx[i] = w[p]; lg[i] = gw[p];
            }
            rc = orc_adjoint(nx, la, lb, lc, lx, lg, oa, ob, oc, lgd);
            for (int64_t i = 0; i < nx && rc == 0; ++i) {
                int64_t p = i + nx * j;
                G[0][p] += oa[i]; G[1][p] += ob[i]; G[2][p] += oc[i]; gd[p] = lgd[i];
            }
        }
        if (rc) break;
        /* stencil of d: transposed into dL/du_t, and into the a, c gradients */
        for (int64_t p = 0; p < n; ++p) gu[p] = g[p];
        for (int64_t j = 1; j < ny - 1; ++j)
            for (int64_t i = 1; i < nx - 1; ++i) {
                int64_t p = i + nx * j;
                double gm = gd[p];
                gu[p + 1] += -co[2][p] * gm;
                gu[p - 1] += -co[0][p] * gm;
                gu[p + nx] += -co[5][p] * gm;
                gu[p - nx] += -co[3][p] * gm;
                gu[p] += (co[0][p] + co[2][p] + co[3][p] + co[5][p]) * gm;
                G[0][p] += gm * (u[p] - u[p - 1]);
                G[2][p] += gm * (u[p] - u[p + 1]);
                G[3][p] += gm * (u[p] - u[p - nx]);
                G[5][p] += gm * (u[p] - u[p + nx]);
            }
        for (int64_t p = 0; p < n; ++p) g[p] = gu[p];
    }
    if (rc) goto out;
    memcpy(g_u0, g, (size_t)n * sizeof(double));
    if (g_coef) memcpy(g_coef, G[0], (size_t)n * 6 * sizeof(double));
    /* to the faces: gkx[q] is the face between q and q+1 */
    for (int64_t p = 0; p < n; ++p) { gkx[p] = 0.0; gky[p] = 0.0; gk[p] = 0.0; }
    for (int64_t j = 0; j < ny; ++j)
        for (int64_t i = 0; i < nx; ++i) {
            int64_t p = i + nx * j;
            if (i > 0 && i < nx - 1) {
                gkx[p - 1] += lam * (G[1][p] - G[0][p]);
                gkx[p] += lam * (G[1][p] - G[2][p]);
            }
            if (j > 0 && j < ny - 1) {
                gky[p - nx] += lam * (G[4][p] - G[3][p]);
                gky[p] += lam * (G[4][p] - G[5][p]);
            }
        }
    /* to the nodes */
    for (int64_t j = 0; j < ny; ++j)
        for (int64_t i = 0; i < nx; ++i) {
            int64_t p = i + nx * j;
            if (i < nx - 1) { gk[p] += 0.5 * gkx[p]; gk[p + 1] += 0.5 * gkx[p]; }
            if (j < ny - 1) { gk[p] += 0.5 * gky[p]; gk[p + nx] += 0.5 * gky[p]; }
        }
    memcpy(g_kappa, gk, (size_t)n * sizeof(double));
out:
    free(st); free(buf); free(lv);
    return rc;
}
