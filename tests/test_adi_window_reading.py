"""The windowed y and z solves of the 3D ADI step, restated on the CPU and
checked against the oracle's step (no GPU).

The ADI operator tridiag(-lambda, 1 + 2 lambda, -lambda) (identity rows at the
two boundary nodes) is diagonally dominant with an inverse that decays
geometrically away from the diagonal, at the rate rho = |c*| of Thomas'
back-substitution factor on an infinite line.  The GPU path solves the rows of
a tile (32 y rows, or 16 z rows) by Thomas on a window of the tile plus H = 8
rows on each side, with the couplings across the window's ends dropped and the
physical boundary rows kept; x is solved exactly.  The host takes that path
only when the dropped couplings reach a tile row with a factor below 2^-28.
Here the schedule is restated in FP64 with dense solves per window, and the
step must match the oracle to within that bound, while a window one row
shorter must be visibly worse (the windows are not trivially exact).
"""
import numpy as np
import pytest

import oracle
from paper_2201_03950_gb300 import inputs

H = 8


def axis_operator(n, lam):
    A = np.eye(n)
    for i in range(1, n - 1):
        A[i, i - 1] = -lam
        A[i, i] = 1 + 2 * lam
        A[i, i + 1] = -lam
    return A


def windowed_solve(d, lam, tile, h, axis):
    """Solve along `axis` of the 3D array d tile by tile: each tile's rows
    from a dense solve of the operator restricted to [tile - h, tile + h]."""
    n = d.shape[axis]
    A = axis_operator(n, lam)
    v = np.moveaxis(d, axis, 0)
    out = np.empty_like(v)
    for t0 in range(0, n, tile):
        lo, hi = max(0, t0 - h), min(n, t0 + tile + h)
        W = A[lo:hi, lo:hi]  # couplings to rows outside the window dropped
        sol = np.linalg.solve(W, v[lo:hi].reshape(hi - lo, -1)).reshape(v[lo:hi].shape)
        out[t0:t0 + tile] = sol[t0 - lo:t0 - lo + tile]
    return np.moveaxis(out, 0, axis)


def rhs(u, lam):
    d = np.zeros_like(u)
    s = (u[2:, 1:-1, 1:-1] + u[:-2, 1:-1, 1:-1] + u[1:-1, 2:, 1:-1] + u[1:-1, :-2, 1:-1]
         + u[1:-1, 1:-1, 2:] + u[1:-1, 1:-1, :-2])
    d[1:-1, 1:-1, 1:-1] = lam * (s - 6 * u[1:-1, 1:-1, 1:-1])
    return d


def window_step(u, lam, h):
    """u <- Z^-1 (Z u + Y^-1 X^-1 d), with windowed Y (32-row tiles) and Z
    (16-row tiles) solves; u is indexed [z, y, x]."""
    nz = u.shape[0]
    d = rhs(u, lam)
    d = np.moveaxis(np.linalg.solve(axis_operator(u.shape[2], lam),
                                    np.moveaxis(d, 2, 0).reshape(u.shape[2], -1)
                                    ).reshape(np.moveaxis(d, 2, 0).shape), 0, 2)
    d = windowed_solve(d, lam, 32, h, axis=1)
    Z = axis_operator(nz, lam)
    zu = np.moveaxis(np.tensordot(Z, u, axes=(1, 0)), 0, 0)
    return windowed_solve(zu + d, lam, 16, h, axis=0)


@pytest.mark.parametrize("dims", [(24, 96, 48), (16, 64, 32), (40, 32, 80)], ids=str)
def test_windowed_step_matches_oracle(dims):
    nx, ny, nz = dims
    lam = 0.1
    rng = np.random.default_rng(nx + ny + nz)
    u0 = inputs.sine_field(dims, inputs.sine_modes(dims, seed=2))
    u0 = u0 + rng.uniform(-0.3, 0.3, u0.size)  # boundary values too: they must stay fixed
    ref = oracle.adi(u0, dims, lam, 1)
    u = u0.reshape(nz, ny, nx)
    scale = np.max(np.abs(ref))
    err = np.max(np.abs(window_step(u, lam, H).reshape(-1) - ref)) / scale
    assert err <= 2.0 ** -28
    # a window one row shorter on each side loses accuracy: the bound is tight
    err_short = np.max(np.abs(window_step(u, lam, H - 2).reshape(-1) - ref)) / scale
    assert err_short > 10 * err


def window_thomas_factors(n, lam, tile_rows, t, h):
    """Thomas factors of the window of tile t (rows t*tile_rows - h + j): forward
    f_j = F_j v_j + FA_j f_{j-1}, backward x_j = f_j - C_j x_{j+1}; rows outside
    the line are absent (all factors 0), couplings across the window ends dropped."""
    W = tile_rows + 2 * h
    A = axis_operator(n, lam)
    y0 = t * tile_rows - h
    F, FA, C = np.zeros(W), np.zeros(W), np.zeros(W)
    cprev, prev = 0.0, False
    for j in range(W):
        y = y0 + j
        if y < 0 or y >= n:
            cprev, prev = 0.0, False
            continue
        a = A[y, y - 1] if (prev and y > 0) else 0.0
        c = A[y, y + 1] if (j < W - 1 and y + 1 < n) else 0.0
        den = A[y, y] - a * cprev
        F[j], FA[j], C[j] = 1.0 / den, -a / den, c / den
        cprev, prev = C[j], True
    return F, FA, C


@pytest.mark.parametrize("tile_rows,n,t", [(32, 256, 3), (32, 256, 0), (32, 256, 7), (32, 64, 1),
                                           (16, 256, 5), (16, 32, 0)], ids=str)
def test_window_split_by_linearity(tile_rows, n, t):
    """The GPU's split of a tile's window solve: x_tile = x0 + T h + B b, with
    h = sum_k Wt_k v_k the forward value the halo above leaves at its last row
    and b the value x at the first row below the tile that the halo below alone
    produces.  Equivalently the blocks (tile rows x halo rows) of the window's
    inverse have rank one (a tridiagonal inverse is semiseparable).  Checked
    against a dense solve of the window."""
    lam, h = 0.1, H
    W = tile_rows + 2 * h
    y0 = t * tile_rows - h
    A = axis_operator(n, lam)
    rows = [y for y in range(y0, y0 + W)]
    ok = [0 <= y < n for y in rows]
    Wm = np.eye(W)  # absent rows: identity with zero right-hand side
    for i in range(W):
        for j in range(W):
            if ok[i] and ok[j] and abs(i - j) <= 1:
                Wm[i, j] = A[rows[i], rows[j]]
    rng = np.random.default_rng(t + n)
    v = np.where(ok, rng.uniform(-1, 1, W), 0.0)
    x_dense = np.linalg.solve(Wm, v)[h:h + tile_rows]
    F, FA, C = window_thomas_factors(n, lam, tile_rows, t, h)
    # the tile alone (both halos zero): forward over the tile, x after it per unit f
    f = np.zeros(W)
    for j in range(h, W):
        f[j] = F[j] * (v[j] if h <= j < h + tile_rows else 0.0) + FA[j] * f[j - 1]
    x = np.zeros(W)
    x[W - 1] = f[W - 1]
    for j in range(W - 2, h - 1, -1):
        x[j] = f[j] - C[j] * x[j + 1]
    x0 = x[h:h + tile_rows]
    # halo above: h_val from its rows; T the response to a unit forward value at row h - 1
    hval = 0.0
    for j in range(h):
        hval = F[j] * v[j] + FA[j] * hval
    f = np.zeros(W)
    f[h - 1] = 1.0
    for j in range(h, W):
        f[j] = FA[j] * f[j - 1]
    x = np.zeros(W)
    x[W - 1] = f[W - 1]
    for j in range(W - 2, h - 1, -1):
        x[j] = f[j] - C[j] * x[j + 1]
    T = x[h:h + tile_rows]
    # halo below: b = x at row h + tile_rows from its rows alone; B the response to it
    f = np.zeros(W)
    for j in range(h + tile_rows, W):
        f[j] = F[j] * v[j] + FA[j] * f[j - 1]
    xb = f[W - 1]
    for j in range(W - 2, h + tile_rows - 1, -1):
        xb = f[j] - C[j] * xb
    B = np.zeros(tile_rows)
    xv = 1.0
    for j in range(h + tile_rows - 1, h - 1, -1):
        xv = -C[j] * xv
        B[j - h] = xv
    split = x0 + T * hval + B * xb
    assert np.max(np.abs(split - x_dense)) <= 1e-14 * max(1.0, np.max(np.abs(x_dense)))
    # rank one: the tile-by-halo blocks of the window's inverse
    inv = np.linalg.inv(Wm)
    for blk in (inv[h:h + tile_rows, :h], inv[h:h + tile_rows, h + tile_rows:]):
        s = np.linalg.svd(blk, compute_uv=False)
        assert s[1:].max(initial=0.0) <= 1e-12 * max(s[0], 1e-300)
