"""Adjoint of the batched solve (trid_solve_batch_adjoint) and the autograd
wrapper, against the FP64 oracle adjoint, the transpose identity and finite
differences."""
import numpy as np
import pytest

import oracle
from paper_2201_03950_gb300 import inputs, trid

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {np.float32: 2e-5, np.float64: 1e-11}


def normwise(x, ref):
    x = np.asarray(x, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    return float(np.max(np.abs(x - ref)) / max(np.max(np.abs(ref)), 1e-300))


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2201_03950_gb300 import build
    build.build()
    trid.load()


def line_index(dims, k):
    """(nsys, n) index array of every system's elements in the flat mesh."""
    n = dims[k]
    total = int(np.prod(dims))
    inner = int(np.prod(dims[:k])) if k else 1
    nsys = total // n
    s = np.arange(nsys)
    base = (s % inner) + (s // inner) * inner * n
    return base[:, None] + inner * np.arange(n)[None, :]


def oracle_adjoint(a, b, c, x, gx, idx):
    ga, gb, gc, gd = (np.zeros(a.size) for _ in range(4))
    for row in idx:
        r = oracle.adjoint(a[row], b[row], c[row], x[row], gx[row])
        for out, v in zip((ga, gb, gc, gd), r):
            out[row] = v
    return ga, gb, gc, gd


CASES = [((64, 64), 0), ((64, 64), 1), ((9, 7, 5), 2), ((37, 5, 3), 0), ((5, 300), 1),
         ((700, 4), 0), ((1,), 0), ((2, 3), 0), ((33, 2, 40), 1)]


@pytest.mark.parametrize("dtype", [np.float32, np.float64], ids=["f32", "f64"])
@pytest.mark.parametrize("dims,k", CASES, ids=[f"{'x'.join(map(str, d))}-dim{k}" for d, k in CASES])
def test_adjoint_matches_oracle(dims, k, dtype):
    total = int(np.prod(dims))
    a, b, c, d = inputs.dominant_system((total,), seed=total + k, dtype=dtype)
    gx = inputs.random_rhs((total,), seed=total + k + 1, dtype=dtype)
    x = oracle.solve_mesh(a, b, c, d, dims, k).astype(dtype)
    idx = line_index(dims, k)
    ref = oracle_adjoint(a, b, c, x, gx, idx)
    ta, tb, tc, tx, tgx = (torch.from_numpy(np.ascontiguousarray(v)).cuda() for v in (a, b, c, x, gx))
    got = trid.adjoint(ta, tb, tc, tx, tgx, dims, k)
    torch.cuda.synchronize()
    for name, g, r in zip(("g_a", "g_b", "g_c", "g_d"), got, ref):
        assert normwise(g.cpu().numpy(), r) <= TOL[dtype], name


def test_adjoint_transpose_identity_full_size():
    """256^3 FP32 along z: <A^{-1} d, g> = <d, A^{-T} g> with the GPU forward
    and adjoint results, and sampled lines against the oracle."""
    dims, k = (256, 256, 256), 2
    total = 256 ** 3
    a, b, c, d = inputs.dominant_system((total,), seed=1, dtype=np.float32)
    g = inputs.random_rhs((total,), seed=2, dtype=np.float32)
    ta, tb, tc, td, tg = (torch.from_numpy(v).cuda() for v in (a, b, c, d, g))
    tx = td.clone()
    trid.solve(ta, tb, tc, tx, dims, k)
    ga, gb, gc, gd = trid.adjoint(ta, tb, tc, tx, tg, dims, k)
    torch.cuda.synchronize()
    lhs = torch.dot(tx.double(), tg.double()).item()
    rhs = torch.dot(td.double(), gd.double()).item()
    assert abs(lhs - rhs) <= 1e-5 * (abs(lhs) + torch.linalg.vector_norm(tx.double()).item())
    idx = line_index(dims, k)
    rng = np.random.default_rng(0)
    pick = idx[rng.choice(idx.shape[0], 64, replace=False)]
    x = tx.cpu().numpy()
    gdn = gd.cpu().numpy()
    gan = ga.cpu().numpy()
    for row in pick:
        r = oracle.adjoint(a[row], b[row], c[row], x[row], g[row])
        assert normwise(gdn[row], r[3]) <= 2e-5
        assert normwise(gan[row], r[0]) <= 2e-5


def test_autograd_gradcheck_fp64():
    from paper_2201_03950_gb300.autograd import tridiag_solve
    for dims, k in (((6, 5), 0), ((6, 5), 1), ((4, 3, 5), 2), ((300,), 0)):
        total = int(np.prod(dims))
        a, b, c, d = inputs.dominant_system((total,), seed=7, dtype=np.float64)
        ts = [torch.from_numpy(v).cuda().requires_grad_(True) for v in (a, b, c, d)]
        assert torch.autograd.gradcheck(lambda A, B, C, D: tridiag_solve(A, B, C, D, dims, k), ts,
                                        eps=1e-6, atol=1e-7, rtol=1e-5)


def test_autograd_loss_gradient_matches_oracle():
    from paper_2201_03950_gb300.autograd import tridiag_solve
    dims, k = (32, 20), 1
    total = 640
    a, b, c, d = inputs.dominant_system((total,), seed=3, dtype=np.float32)
    target = inputs.random_rhs((total,), seed=4, dtype=np.float32)
    ts = [torch.from_numpy(v).cuda().requires_grad_(True) for v in (a, b, c, d)]
    x = tridiag_solve(*ts, dims, k)
    loss = ((x - torch.from_numpy(target).cuda()) ** 2).mean()
    loss.backward()
    xr = oracle.solve_mesh(a, b, c, d, dims, k)
    gx = 2.0 * (xr - target.astype(np.float64)) / total
    ref = oracle_adjoint(a, b, c, xr, gx, line_index(dims, k))
    for t, r in zip(ts, ref):
        assert normwise(t.grad.cpu().numpy(), r) <= 2e-5
