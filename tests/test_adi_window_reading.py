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
