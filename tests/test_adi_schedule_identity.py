"""The 3D ADI step as the two-pass GPU schedule computes it, restated on the
CPU with dense per-axis operators and checked against the oracle's step.

The oracle follows Algorithm "adi": d = lambda * (sum of the 6 neighbours -
6u) on interior nodes (0 on boundary nodes), d <- X^-1 d, Y^-1 d, Z^-1 d, then
u <- u + d, with each axis operator tridiag(-lambda, 1 + 2 lambda, -lambda)
on interior rows and identity rows at the two boundary nodes.  The GPU
schedule computes the same step as u <- Z^-1 (Z u + Y^-1 X^-1 d): pass A
forms Z u from the z neighbours the stencil reads anyway and adds it to the
x- and y-solved right-hand side, pass B solves along z and writes u without
reading it.  Exact in exact arithmetic (Z^-1 Z u = u); here in FP64 to
rounding, with random boundary values that must stay fixed.
"""
import numpy as np
import pytest

import oracle
from paper_2201_03950_gb300 import inputs


def axis_operator(n, lam):
    A = np.eye(n)
    for i in range(1, n - 1):
        A[i, i - 1] = -lam
        A[i, i] = 1 + 2 * lam
        A[i, i + 1] = -lam
    return A


def apply_along(M, v, axis):
    """M @ line for every line of the 3D array v (index [z, y, x]) along axis."""
    return np.moveaxis(np.tensordot(M, np.moveaxis(v, axis, 0), axes=(1, 0)), 0, axis)


def rhs(u, lam):
    d = np.zeros_like(u)
    c = u[1:-1, 1:-1, 1:-1]
    s = (u[2:, 1:-1, 1:-1] + u[:-2, 1:-1, 1:-1] + u[1:-1, 2:, 1:-1] + u[1:-1, :-2, 1:-1]
         + u[1:-1, 1:-1, 2:] + u[1:-1, 1:-1, :-2])
    d[1:-1, 1:-1, 1:-1] = lam * (s - 6 * c)
    return d


@pytest.mark.parametrize("dims,lam", [((12, 10, 9), 0.1), ((7, 16, 11), 0.3), ((20, 5, 6), 1.0)],
                         ids=str)
def test_two_pass_schedule_equals_the_adi_step(dims, lam):
    nx, ny, nz = dims
    rng = np.random.default_rng(sum(dims))
    u0 = inputs.sine_field(dims, inputs.sine_modes(dims, seed=3))
    u0 = u0 + rng.uniform(-0.5, 0.5, nx * ny * nz)
    ref = oracle.adi(u0, dims, lam, 1)
    u = u0.reshape(nz, ny, nx)          # x contiguous: index [z, y, x]
    X, Y, Z = (axis_operator(n, lam) for n in (nx, ny, nz))
    w = rhs(u, lam)
    w = apply_along(np.linalg.inv(X), w, 2)
    w = apply_along(np.linalg.inv(Y), w, 1)
    e = apply_along(Z, u, 0) + w          # pass A's output
    unew = apply_along(np.linalg.inv(Z), e, 0)  # pass B
    got = unew.reshape(-1)
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))
    # boundary nodes keep their values
    bnd = np.ones((nz, ny, nx), dtype=bool)
    bnd[1:-1, 1:-1, 1:-1] = False
    assert np.array_equal(unew[bnd], u[bnd]) or np.max(np.abs(unew[bnd] - u[bnd])) <= 1e-13
