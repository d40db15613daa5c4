"""Pins for the oracle: checks against facts fixed by the mathematics, not by
the oracle itself.  Each ``pin_*`` takes an oracle library handle (the real one
or a deliberately broken build, see test_oracle_mutants.py) and returns
``(ok, worst_error)``.

Sources of truth used here (none of them re-types an oracle formula):
  * LAPACK via numpy.linalg.solve on the assembled dense matrix;
  * exact rational Gaussian elimination (fractions.Fraction) on tiny systems;
  * eigenvectors of constant-coefficient (Toeplitz) tridiagonal matrices;
  * manufactured solutions d = A x* (the definition of the problem);
  * the discrete heat-equation eigenmode decay factor of the ADI step;
  * dense Kronecker-product assembly of one ADI step on a tiny mesh;
  * the transpose identity <A^{-1} d, g> = <d, A^{-T} g> and central finite
    differences for the adjoint;
  * for the diffusivity-field ADI: the constant-field case against the
    constant-coefficient step, a flux-form (D^T K D) dense assembly of the
    operators, and central finite differences of its loss.
"""
from __future__ import annotations

import math
from fractions import Fraction

import numpy as np

import oracle
from paper_2201_03950_gb300 import inputs


def dense_matrix(a, b, c):
    """Assemble the N x N matrix of eq. tdma-system (a_0, c_{N-1} dropped)."""
    n = len(b)
    A = np.zeros((n, n))
    for i in range(n):
        A[i, i] = b[i]
        if i > 0:
            A[i, i - 1] = a[i]
        if i < n - 1:
            A[i, i + 1] = c[i]
    return A


def rel(x, ref):
    x = np.asarray(x, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    if not np.all(np.isfinite(x)):
        return float("inf")  # a NaN would slip through max() comparisons
    scale = max(np.max(np.abs(ref)), 1e-300)
    return float(np.max(np.abs(x - ref)) / scale)


def _random_dominant(n, seed):
    a, b, c, d = inputs.dominant_system((n,), seed=seed, dtype=np.float64)
    return a, b, c, d


SOLVERS = {
    "thomas": lambda lib, a, b, c, d: oracle.thomas(a, b, c, d, lib=lib),
    "pcr": lambda lib, a, b, c, d: oracle.pcr(a, b, c, d, lib=lib),
    "tiled_thomas_m3": lambda lib, a, b, c, d: oracle.tiled(a, b, c, d, 3, False, lib=lib),
    "tiled_pcr_m4": lambda lib, a, b, c, d: oracle.tiled(a, b, c, d, 4, True, lib=lib),
    "tiled_thomas_m8": lambda lib, a, b, c, d: oracle.tiled(a, b, c, d, 8, False, lib=lib),
    "tiled_pcr_m16": lambda lib, a, b, c, d: oracle.tiled(a, b, c, d, 16, True, lib=lib),
}


def pin_lapack(lib, tol=1e-12):
    """P1: every solver against LAPACK on random dominant systems, N <= 70,
    with garbage in the unread a_0 / c_{N-1} slots."""
    worst = 0.0
    for n in (1, 2, 3, 4, 5, 7, 8, 9, 17, 31, 33, 50, 53, 64, 70):
        a, b, c, d = _random_dominant(n, seed=100 + n)
        ref = np.linalg.solve(dense_matrix(a, b, c), d)
        a = a.copy(); c = c.copy()
        a[0] = 123.0
        c[-1] = -77.0
        for fn in SOLVERS.values():
            worst = max(worst, rel(fn(lib, a, b, c, d), ref))
        worst = max(worst, rel(oracle.dense_solve(dense_matrix(a, b, c), d, lib=lib), ref))
    return worst <= tol, worst


def pin_dense_general(lib, tol=1e-11):
    """Dense Gaussian elimination with pivoting against LAPACK on general
    (non-tridiagonal, pivoting-requiring) matrices."""
    rng = np.random.default_rng(7)
    worst = 0.0
    for n in (1, 2, 3, 6, 11, 20):
        A = rng.standard_normal((n, n))
        A[0, 0] = 0.0  # forces a row exchange
        if n == 1:
            A[0, 0] = 0.5
        rhs = rng.standard_normal(n)
        worst = max(worst, rel(oracle.dense_solve(A, rhs, lib=lib), np.linalg.solve(A, rhs)))
    return worst <= tol, worst


def _exact_solve(a, b, c, d):
    """Gaussian elimination in exact rational arithmetic (brute force)."""
    n = len(b)
    M = [[Fraction(0)] * n for _ in range(n)]
    for i in range(n):
        M[i][i] = Fraction(b[i])
        if i > 0:
            M[i][i - 1] = Fraction(a[i])
        if i < n - 1:
            M[i][i + 1] = Fraction(c[i])
    y = [Fraction(v) for v in d]
    for k in range(n):
        p = next(r for r in range(k, n) if M[r][k] != 0)
        M[k], M[p] = M[p], M[k]
        y[k], y[p] = y[p], y[k]
        for r in range(k + 1, n):
            f = M[r][k] / M[k][k]
            for j in range(k, n):
                M[r][j] -= f * M[k][j]
            y[r] -= f * y[k]
    x = [Fraction(0)] * n
    for k in range(n - 1, -1, -1):
        s = y[k] - sum(M[k][j] * x[j] for j in range(k + 1, n))
        x[k] = s / M[k][k]
    return [float(v) for v in x]


def pin_exact_rational(lib, tol=1e-14):
    """Brute force: small-integer systems solved exactly with fractions."""
    rng = np.random.default_rng(11)
    worst = 0.0
    for n in (1, 2, 3, 4, 6, 9, 12):
        a = rng.integers(-3, 4, n).astype(np.float64)
        c = rng.integers(-3, 4, n).astype(np.float64)
        b = np.abs(a) + np.abs(c) + rng.integers(1, 4, n)
        b *= np.where(rng.random(n) < 0.5, -1.0, 1.0)  # mixed signs, still dominant
        d = rng.integers(-9, 10, n).astype(np.float64)
        ref = _exact_solve([0] + list(a[1:]), b, list(c[:-1]) + [0], d)
        for fn in SOLVERS.values():
            worst = max(worst, rel(fn(lib, a, b, c, d), ref))
    return worst <= tol, worst


def pin_toeplitz(lib, tol=1e-12):
    """P2: constant a, b, c.  v_j = rho^j sin((j+1) k pi/(n+1)), rho =
    sqrt(a/c), is an eigenvector with eigenvalue b + 2 s cos(k pi/(n+1)),
    s = sign(a) sqrt(a c); so d = v gives x = v / eigenvalue exactly."""
    worst = 0.0
    cases = [(-0.4, 2.0, -0.4), (0.3, 1.1, 0.3), (-0.2, 1.5, -0.6), (0.7, -2.5, 0.25)]
    for (av, bv, cv) in cases:
        for n in (1, 2, 5, 16, 33, 64):
            for k in sorted({1, 2, (n + 1) // 2, n}):
                if k < 1 or k > n:
                    continue
                th = k * math.pi / (n + 1)
                rho = math.sqrt(av / cv)
                s = math.copysign(math.sqrt(av * cv), av)
                j = np.arange(n)
                v = rho ** j * np.sin((j + 1) * th)
                lam = bv + 2.0 * s * math.cos(th)
                a = np.full(n, av); b = np.full(n, bv); c = np.full(n, cv)
                for fn in SOLVERS.values():
                    worst = max(worst, rel(fn(lib, a, b, c, v), v / lam))
    return worst <= tol, worst


def pin_manufactured(lib, tol=1e-12):
    """P3: draw x*, form d = A x* from the problem's definition, recover x*."""
    worst = 0.0
    rng = np.random.default_rng(5)
    for n in (3, 10, 100, 257, 1000):
        a, b, c, _ = _random_dominant(n, seed=300 + n)
        xs = rng.uniform(-1, 1, n)
        d = b * xs
        d[1:] += a[1:] * xs[:-1]
        d[:-1] += c[:-1] * xs[1:]
        for fn in SOLVERS.values():
            worst = max(worst, rel(fn(lib, a, b, c, d), xs))
    return worst <= tol, worst


def pin_mesh(lib, tol=1e-12):
    """Mesh solves: each axis against LAPACK on every line; accumulate adds;
    the unread first-a / last-c of each line may hold NaN."""
    worst = 0.0
    dims = (5, 4, 3)
    tot = 60
    a, b, c, d = inputs.dominant_system((tot,), seed=9, dtype=np.float64)
    strides = (1, 5, 20)
    for k in range(3):
        n, st = dims[k], strides[k]
        aa = a.copy(); cc = c.copy()
        x_ref = np.zeros(tot)
        others = [ax for ax in range(3) if ax != k]
        for j2 in range(dims[others[1]]):
            for j1 in range(dims[others[0]]):
                base = j1 * strides[others[0]] + j2 * strides[others[1]]
                idx = base + st * np.arange(n)
                aa[idx[0]] = np.nan
                cc[idx[-1]] = np.nan
                x_ref[idx] = np.linalg.solve(dense_matrix(a[idx], b[idx], c[idx]), d[idx])
        x = oracle.solve_mesh(aa, b, cc, d, dims, k, lib=lib)
        worst = max(worst, rel(x, x_ref))
        u0 = np.linspace(-1, 1, tot)
        u = u0.copy()
        oracle.solve_mesh(aa, b, cc, d, dims, k, out=u, lib=lib)
        worst = max(worst, rel(u - u0, x_ref))
    return worst <= tol, worst


def pin_mesh_f32(lib, tol=2e-6):
    """The binary32 mesh solve (the FP32 CPU baseline): each axis against
    LAPACK in binary64 on FP32-representable inputs, within a few FP32 ulps
    (the systems are diagonally dominant, so Thomas is stable), with NaN in
    every unread first a / last c."""
    worst = 0.0
    dims = (6, 5, 7)
    tot = 210
    a, b, c, d = (v.astype(np.float64) for v in
                  inputs.dominant_system((tot,), seed=19, dtype=np.float32))
    strides = (1, 6, 30)
    for k in range(3):
        n, st = dims[k], strides[k]
        aa = a.copy(); cc = c.copy()
        x_ref = np.zeros(tot)
        others = [ax for ax in range(3) if ax != k]
        for j2 in range(dims[others[1]]):
            for j1 in range(dims[others[0]]):
                base = j1 * strides[others[0]] + j2 * strides[others[1]]
                idx = base + st * np.arange(n)
                aa[idx[0]] = np.nan
                cc[idx[-1]] = np.nan
                x_ref[idx] = np.linalg.solve(dense_matrix(a[idx], b[idx], c[idx]), d[idx])
        x = oracle.solve_mesh_f32(aa, b, cc, d, dims, k, lib=lib)
        if x.dtype != np.float32:
            return False, float("inf")
        worst = max(worst, rel(x, x_ref))
    return worst <= tol, worst

def _mu(p, n):
    return -4.0 * math.sin(math.pi * p / (2.0 * (n - 1))) ** 2


def pin_adi_eigenmode(lib, tol=1e-11):
    """P5: u = prod sin(pi k_ax i / (n_ax - 1)) is an eigenvector of the
    stencil and of every directional operator, so one ADI step multiplies it by
    g = 1 + lam sum(mu) / prod(1 - lam mu),  mu = -4 sin^2(pi k / (2(n-1))).
    A sum of modes decays mode by mode."""
    worst = 0.0
    for dims, lam, steps in (((9, 7, 6), 0.1, 5), ((12, 10), 0.3, 7), ((17, 17, 17), 0.1, 3)):
        modes = inputs.sine_modes(dims, seed=len(dims), nmodes=3)
        u0 = inputs.sine_field(dims, modes)
        ref = np.zeros_like(u0)
        for ks, amp in modes:
            mus = [_mu(k, n) for k, n in zip(ks, dims)]
            g = 1.0 + lam * sum(mus) / np.prod([1.0 - lam * m for m in mus])
            ref += inputs.sine_field(dims, [(ks, amp * g ** steps)])
        worst = max(worst, rel(oracle.adi(u0, dims, lam, steps, lib=lib), ref))
    return worst <= tol, worst


def _axis_op(n, lam):
    T = np.eye(n)
    for i in range(1, n - 1):
        T[i, i - 1] = -lam
        T[i, i] = 1 + 2 * lam
        T[i, i + 1] = -lam
    return T


def pin_adi_dense(lib, tol=1e-12):
    """One ADI step on a tiny random mesh assembled as dense Kronecker
    products: Delta = Z^{-1} Y^{-1} X^{-1} (lam L u restricted to the interior),
    u' = u + Delta, with L the 2*ndim-neighbour Laplacian."""
    worst = 0.0
    rng = np.random.default_rng(3)
    for dims, lam in (((5, 6, 4), 0.2), ((6, 5), 0.15)):
        nd = len(dims)
        tot = int(np.prod(dims))
        u = rng.uniform(-1, 1, tot)
        grid = np.indices(tuple(reversed(dims))).reshape(nd, -1)[::-1]
        interior = np.ones(tot, dtype=bool)
        for ax in range(nd):
            interior &= (grid[ax] > 0) & (grid[ax] < dims[ax] - 1)
        u[~interior] = 0.0
        # Laplacian by explicit neighbour sums
        U = u.reshape(tuple(reversed(dims)))
        rhs = np.zeros_like(U)
        inner = tuple(slice(1, -1) for _ in range(nd))
        acc = -2.0 * nd * U[inner]
        for ax in range(nd):
            arr_ax = nd - 1 - ax
            for sh in (-1, 1):
                sl = [slice(1, -1)] * nd
                sl[arr_ax] = slice(1 + sh, U.shape[arr_ax] - 1 + sh)
                acc = acc + U[tuple(sl)]
        rhs[inner] = lam * acc
        rhs = rhs.reshape(-1)
        # x-operator acts on the contiguous index -> kron(I_z, I_y, X)
        ops = [_axis_op(n, lam) for n in dims]
        full = np.eye(1)
        mats = []
        for ax in range(nd):
            factors = [np.eye(dims[k]) if k != ax else ops[k] for k in range(nd)]
            M = np.eye(1)
            for f in reversed(factors):
                M = np.kron(M, f)
            mats.append(M)
        delta = rhs
        for M in mats:
            delta = np.linalg.solve(M, delta)
        ref = u + delta
        worst = max(worst, rel(oracle.adi(u, dims, lam, 1, lib=lib), ref))
        del full
    return worst <= tol, worst


def pin_varlen(lib, tol=1e-12):
    lengths = [1, 2, 3, 17, 5, 64]
    off = np.concatenate([[0], np.cumsum(lengths)])
    a, b, c, d = inputs.dominant_system((int(off[-1]),), seed=21, dtype=np.float64)
    x = oracle.solve_varlen(a, b, c, d, off, lib=lib)
    worst = 0.0
    for k in range(len(lengths)):
        s, e = off[k], off[k + 1]
        ref = np.linalg.solve(dense_matrix(a[s:e], b[s:e], c[s:e]), d[s:e])
        worst = max(worst, rel(x[s:e], ref))
    return worst <= tol, worst


def pin_lines(lib, tol=1e-12):
    """Batch of contiguous systems (rows of a [nsys, n] array, the checker of
    the full-size sampled GPU tests): every row against LAPACK on its own dense
    matrix, with NaN planted in each row's unread a_0 and c_{n-1}.  Shapes
    with nsys != n and several rows, so a wrong row offset or length shows."""
    worst = 0.0
    for nsys, n in ((1, 5), (3, 1), (4, 7), (7, 4), (5, 33), (9, 64)):
        a, b, c, d = inputs.dominant_system((nsys * n,), seed=300 + 7 * nsys + n,
                                            dtype=np.float64)
        a, b, c, d = (v.reshape(nsys, n).copy() for v in (a, b, c, d))
        a[:, 0] = np.nan
        c[:, -1] = np.nan
        x = oracle.thomas_lines(a, b, c, d, lib=lib)
        if x.shape != (nsys, n):
            return False, float("inf")
        for k in range(nsys):
            ref = np.linalg.solve(dense_matrix(a[k], b[k], c[k]), d[k])
            worst = max(worst, rel(x[k], ref) if np.all(np.isfinite(x[k])) else float("inf"))
    return worst <= tol, worst


def pin_adjoint(lib, tol=1e-7):
    """Adjoint: g_d against LAPACK on A^T (tight), the dot-product identity,
    and g_a, g_b, g_c, g_d against central differences of L = <g, x(a,b,c,d)>."""
    worst_tight = 0.0
    worst_fd = 0.0
    rng = np.random.default_rng(17)
    for n in (1, 2, 5, 12):
        a, b, c, d = _random_dominant(n, seed=400 + n)
        g = rng.uniform(-1, 1, n)
        A = dense_matrix(a, b, c)
        x = np.linalg.solve(A, d)
        ga, gb, gc, gd = oracle.adjoint(a, b, c, x, g, lib=lib)
        worst_tight = max(worst_tight, rel(gd, np.linalg.solve(A.T, g)))
        lhs = float(np.dot(x, g))
        rhs_ = float(np.dot(d, gd))
        worst_tight = max(worst_tight, abs(lhs - rhs_) / max(abs(lhs), 1e-30))
        h = 1e-6

        def loss(aa, bb, cc, dd):
            return float(np.dot(np.linalg.solve(dense_matrix(aa, bb, cc), dd), g))

        for arr_i, grad in ((0, ga), (1, gb), (2, gc), (3, gd)):
            fd = np.zeros(n)
            for i in range(n):
                args_p = [v.copy() for v in (a, b, c, d)]
                args_m = [v.copy() for v in (a, b, c, d)]
                args_p[arr_i][i] += h
                args_m[arr_i][i] -= h
                fd[i] = (loss(*args_p) - loss(*args_m)) / (2 * h)
            worst_fd = max(worst_fd, float(np.max(np.abs(fd - grad))))
    ok = worst_tight <= 1e-12 and worst_fd <= tol
    return ok, max(worst_tight, worst_fd)


def _flux_ops(kappa, dims, lam):
    """Dense X, Y operators and the explicit part of one step, assembled in
    flux form: L_axis = -D^T K D with D the forward difference between
    neighbouring nodes and K the face diffusivities (mean of the two nodes);
    boundary rows of X, Y become identity rows and the explicit part is
    masked to the interior."""
    nx, ny = dims
    n = nx * ny
    idx = lambda i, j: i + nx * j
    ops = []
    for axis in (0, 1):
        faces = []
        for j in range(ny):
            for i in range(nx):
                if (axis == 0 and i < nx - 1) or (axis == 1 and j < ny - 1):
                    q = idx(i + 1, j) if axis == 0 else idx(i, j + 1)
                    faces.append((idx(i, j), q))
        D = np.zeros((len(faces), n))
        K = np.zeros(len(faces))
        for f, (p0, p1) in enumerate(faces):
            D[f, p0], D[f, p1] = -1.0, 1.0
            K[f] = 0.5 * (kappa[p0] + kappa[p1])
        L = -(D.T * K) @ D
        op = np.eye(n) - lam * L
        for j in range(ny):
            for i in range(nx):
                end = (i in (0, nx - 1)) if axis == 0 else (j in (0, ny - 1))
                if end:
                    op[idx(i, j), :] = 0.0
                    op[idx(i, j), idx(i, j)] = 1.0
        ops.append((op, L))
    mask = np.zeros(n)
    for j in range(1, ny - 1):
        for i in range(1, nx - 1):
            mask[idx(i, j)] = 1.0
    E = lam * (ops[0][1] + ops[1][1]) * mask[:, None]
    return ops[0][0], ops[1][0], E


def _flux_adi(u, kappa, dims, lam, steps):
    X, Y, E = _flux_ops(kappa, dims, lam)
    for _ in range(steps):
        u = u + np.linalg.solve(Y, np.linalg.solve(X, E @ u))
    return u


def pin_adi2v(lib, tol=1e-12):
    """Diffusivity-field 2D ADI: kappa = 1 is the constant-coefficient step;
    kappa = s with lambda equals kappa = 1 with s lambda; a varying field
    matches the dense flux-form assembly (LAPACK solves)."""
    worst = 0.0
    rng = np.random.default_rng(23)
    dims = (9, 7)
    n = 63
    u0 = rng.uniform(-1, 1, n)
    ref = oracle.adi(u0, dims, 0.3, 4, lib=lib)
    worst = max(worst, rel(oracle.adi2v(u0, np.ones(n), dims, 0.3, 4, lib=lib), ref))
    worst = max(worst, rel(oracle.adi2v(u0, np.full(n, 2.5), dims, 0.12, 4, lib=lib), ref))
    for dims, steps in (((6, 5), 3), ((4, 8), 2), ((3, 3), 2)):
        n = dims[0] * dims[1]
        u0 = rng.uniform(-1, 1, n)
        kap = rng.uniform(0.3, 2.0, n)
        got = oracle.adi2v(u0, kap, dims, 0.4, steps, lib=lib)
        worst = max(worst, rel(got, _flux_adi(u0, kap, dims, 0.4, steps)))
    return worst <= tol, worst


def pin_adi2v_grad(lib, tol=1e-6):
    """Loss gradient of the diffusivity-field ADI against central finite
    differences of the dense flux-form forward: every component of g_kappa
    and g_u0 on a tiny mesh, and the raw coefficient gradients (ax .. cy)
    against differences of a forward whose six coefficient arrays are
    perturbed directly."""
    rng = np.random.default_rng(29)
    dims, steps, lam = (5, 4), 2, 0.35
    nx, ny = dims
    n = nx * ny
    u0 = rng.uniform(-1, 1, n)
    kap = rng.uniform(0.4, 1.8, n)
    tg = rng.uniform(-1, 1, n)
    loss, gu, gk, gc = oracle.adi2v_grad(u0, kap, tg, dims, lam, steps, lib=lib)

    def L_of(u, k):
        return float(np.mean((_flux_adi(u, k, dims, lam, steps) - tg) ** 2))

    h = 1e-6
    worst = abs(loss - L_of(u0, kap)) / abs(loss)
    scale = max(np.max(np.abs(gu)), np.max(np.abs(gk)))
    for p in range(n):
        e = np.zeros(n)
        e[p] = h
        fu = (L_of(u0 + e, kap) - L_of(u0 - e, kap)) / (2 * h)
        fk = (L_of(u0, kap + e) - L_of(u0, kap - e)) / (2 * h)
        worst = max(worst, abs(fu - gu[p]) / scale, abs(fk - gk[p]) / scale)

    # raw coefficient arrays as independent inputs
    X0, Y0, E0 = _flux_ops(kap, dims, lam)

    def coef_arrays(op, axis):
        a, b, c = np.zeros(n), np.zeros(n), np.zeros(n)
        st = 1 if axis == 0 else nx
        for j in range(ny):
            for i in range(nx):
                p = i + nx * j
                b[p] = op[p, p]
                end = (i in (0, nx - 1)) if axis == 0 else (j in (0, ny - 1))
                if not end:
                    a[p], c[p] = op[p, p - st], op[p, p + st]
        return a, b, c

    base = list(coef_arrays(X0, 0)) + list(coef_arrays(Y0, 1))

    def L_coef(arrs):
        ops = []
        for axis in (0, 1):
            a, b, c = arrs[3 * axis: 3 * axis + 3]
            st = 1 if axis == 0 else nx
            op = np.zeros((n, n))
            for j in range(ny):
                for i in range(nx):
                    p = i + nx * j
                    op[p, p] = b[p]
                    end = (i in (0, nx - 1)) if axis == 0 else (j in (0, ny - 1))
                    if not end:
                        op[p, p - st], op[p, p + st] = a[p], c[p]
            ops.append(op)
        # explicit part from the off-diagonal coefficients alone (the
        # diagonal b enters only the implicit operators): at interior p,
        # d_p = sum over axes of -c_p (u_{p+s} - u_p) + a_p (u_p - u_{p-s})
        E = np.zeros((n, n))
        for axis in (0, 1):
            a, _, c = arrs[3 * axis: 3 * axis + 3]
            st = 1 if axis == 0 else nx
            for j in range(1, ny - 1):
                for i in range(1, nx - 1):
                    p = i + nx * j
                    E[p, p - st] -= a[p]
                    E[p, p + st] -= c[p]
                    E[p, p] += a[p] + c[p]
        u = u0.copy()
        for _ in range(steps):
            u = u + np.linalg.solve(ops[1], np.linalg.solve(ops[0], E @ u))
        return float(np.mean((u - tg) ** 2))

    gscale = max(np.max(np.abs(gc)), 1e-30)
    for k in range(6):
        for p in rng.choice(n, 6, replace=False):
            i, j = p % nx, p // nx
            interior_row = (0 < i < nx - 1) if k < 3 else (0 < j < ny - 1)
            if k % 3 != 1 and not interior_row:
                continue  # a, c of an identity row are not part of the operator
            ap = [v.copy() for v in base]
            am = [v.copy() for v in base]
            ap[k][p] += h
            am[k][p] -= h
            fd = (L_coef(ap) - L_coef(am)) / (2 * h)
            worst = max(worst, abs(fd - gc[k][p]) / gscale)
    return worst <= tol, worst


ALL_PINS = [pin_lapack, pin_dense_general, pin_exact_rational, pin_toeplitz, pin_manufactured,
            pin_mesh, pin_mesh_f32, pin_adi_eigenmode, pin_adi_dense, pin_varlen, pin_lines, pin_adjoint, pin_adi2v,
            pin_adi2v_grad]
