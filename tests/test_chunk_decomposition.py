"""The chunk decomposition behind the one-pass strided long-system kernel,
checked on the CPU against the oracle's Thomas solve.

A system cut into chunks of CH rows: by linearity, the solution restricted to
chunk k is x = p + q x_L + r x_R, where x_L and x_R are the unknowns just
outside the chunk, p solves the chunk with them zero, and q, r are its
responses to x_L = 1 and x_R = 1 (right-hand sides -a_first e_first and
-c_last e_last).  The chunks' first (F) and last (E) values obey
    F_k = P0_k + Q0_k E_{k-1} + R0_k F_{k+1}
    E_k = P1_k + Q1_k E_{k-1} + R1_k F_{k+1},
solved by 2x2 block elimination forward (E_k = al_k + be_k F_{k+1},
F_k = ga_k + dl_k F_{k+1}) and back from F_C = 0.  Here every chunk is solved
with numpy's dense solver, independently of the GPU code, and the result must
equal the oracle's Thomas to rounding (the decomposition is exact, not an
approximation) -- including weakly dominant systems where the responses carry
across many chunks.
"""
import numpy as np
import pytest

import oracle
from paper_2201_03950_gb300 import inputs


def dense(a, b, c):
    n = len(b)
    A = np.diag(b)
    A[np.arange(1, n), np.arange(n - 1)] = a[1:]
    A[np.arange(n - 1), np.arange(1, n)] = c[:-1]
    return A


def chunked_solve(a, b, c, d, ch):
    n = len(d)
    starts = list(range(0, n, ch))
    C = len(starts)
    P = np.zeros((C, 6))  # P0 P1 Q0 Q1 R0 R1
    sol = []
    for k, s in enumerate(starts):
        e = min(s + ch, n)
        A = dense(a[s:e], b[s:e], c[s:e])
        rhs = np.zeros((e - s, 3))
        rhs[:, 0] = d[s:e]
        if s > 0:
            rhs[0, 1] = -a[s]          # response to x_L = 1
        if e < n:
            rhs[-1, 2] = -c[e - 1]     # response to x_R = 1
        X = np.linalg.solve(A, rhs)
        sol.append(X)
        P[k] = [X[0, 0], X[-1, 0], X[0, 1], X[-1, 1], X[0, 2], X[-1, 2]]
    al = be = 0.0
    ga, dl, alk, bek = (np.zeros(C) for _ in range(4))
    for k in range(C):
        p0, p1, q0, q1, r0, r1 = P[k]
        inv = 1.0 / (1.0 - q0 * be)
        ga[k] = (p0 + q0 * al) * inv
        dl[k] = r0 * inv
        alk[k] = p1 + q1 * (al + be * ga[k])
        bek[k] = r1 + q1 * be * dl[k]
        al, be = alk[k], bek[k]
    F = np.zeros(C + 1)
    E = np.zeros(C)
    for k in range(C - 1, -1, -1):
        F[k] = ga[k] + dl[k] * F[k + 1]
        E[k] = alk[k] + bek[k] * F[k + 1]
    x = np.empty(n)
    for k, s in enumerate(starts):
        xl = E[k - 1] if k > 0 else 0.0
        xr = F[k + 1] if k + 1 < C else 0.0
        X = sol[k]
        x[s:s + len(X)] = X[:, 0] + X[:, 1] * xl + X[:, 2] * xr
    return x


@pytest.mark.parametrize("n,ch", [(1000, 256), (4096, 256), (257, 256), (700, 100), (512, 256),
                                  (3000, 250)], ids=str)
def test_chunked_equals_thomas(n, ch):
    a, b, c, d = (v.astype(np.float64) for v in inputs.dominant_system((n,), seed=n + ch))
    a[0] = 0.0
    c[-1] = 0.0
    ref = oracle.thomas_lines(a[None], b[None], c[None], d[None])[0]
    x = chunked_solve(a, b, c, d, ch)
    assert np.max(np.abs(x - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_weak_dominance_carries_across_chunks():
    """Dominance margin 1e-3: the responses to the outside unknowns are far
    from negligible over a 64-row chunk, so dropping them would be wrong; the
    chunk-level system reproduces Thomas."""
    n, ch = 2048, 64
    rng = np.random.default_rng(4)
    a = rng.uniform(-1, -0.1, n)
    c = rng.uniform(-1, -0.1, n)
    b = np.abs(a) + np.abs(c) + 1e-3
    d = rng.uniform(-1, 1, n)
    a[0] = 0.0
    c[-1] = 0.0
    ref = oracle.thomas_lines(a[None], b[None], c[None], d[None])[0]
    x = chunked_solve(a, b, c, d, ch)
    assert np.max(np.abs(x - ref)) <= 1e-9 * np.max(np.abs(ref))
    # the responses matter here: the chunks solved in isolation are far off
    isolated = np.concatenate([np.linalg.solve(dense(a[s:s + ch], b[s:s + ch], c[s:s + ch]),
                                               d[s:s + ch]) for s in range(0, n, ch)])
    assert np.max(np.abs(isolated - ref)) > 1e-3 * np.max(np.abs(ref))
