"""Contiguous systems of 256 < N <= 4096 rows (FP32), the bulk-copy staged
one-pass kernel: every team width (N <= 512, 1024, 2048, 4096), lengths just
above and below each width, batches that end in a partial stage, accumulate
and in-place modes, the unit-diagonal reduced systems of longer systems, and
unaligned arrays (served by the multi-pass path).  Whole meshes against the
FP64 oracle, element by element.  GPU only."""
import numpy as np
import pytest

import oracle
from paper_2201_03950_gb300 import inputs, trid

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-5


def normwise(x, ref):
    x = np.asarray(x, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    return float(np.max(np.abs(x - ref)) / max(np.max(np.abs(ref)), 1e-300))


def system(n, nsys, seed):
    a, b, c, d = inputs.dominant_system((n * nsys,), seed=seed, dtype=np.float32)
    return a, b, c, d


CASES = [(260, 1), (260, 9), (264, 300), (508, 17), (512, 64), (516, 5), (1020, 3), (1024, 33),
         (1028, 7), (2044, 2), (2048, 11), (2052, 3), (4092, 5), (4096, 1), (4096, 40)]


@pytest.mark.parametrize("n,nsys", CASES, ids=[f"n{n}-s{s}" for n, s in CASES])
def test_against_oracle(n, nsys):
    a, b, c, d = system(n, nsys, seed=n + nsys)
    dims = (n, nsys)
    ref = oracle.solve_mesh(a, b, c, d, dims, 0)
    ta, tb, tc, td = (torch.from_numpy(v).cuda() for v in (a, b, c, d))
    # the unread a of each first row and c of each last row
    ta[0::n] = float("nan")
    tc[n - 1::n] = float("nan")
    trid.solve(ta, tb, tc, td, dims, 0)
    torch.cuda.synchronize()
    assert normwise(td.cpu().numpy(), ref) <= TOL


@pytest.mark.parametrize("n,nsys", [(264, 13), (1024, 6), (4096, 3)], ids=str)
def test_accumulate(n, nsys):
    a, b, c, d = system(n, nsys, seed=3)
    dims = (n, nsys)
    ref = oracle.solve_mesh(a, b, c, d, dims, 0)
    u0 = inputs.random_rhs((n * nsys,), seed=4, dtype=np.float32)
    ta, tb, tc, td, tu = (torch.from_numpy(v).cuda() for v in (a, b, c, d, u0))
    d0 = td.clone()
    trid.solve(ta, tb, tc, td, dims, 0, u=tu)
    torch.cuda.synchronize()
    assert torch.equal(td, d0)
    got = tu.cpu().numpy().astype(np.float64) - u0.astype(np.float64)
    assert normwise(got, ref) <= TOL


@pytest.mark.parametrize("n", [8192, 16384], ids=str)
def test_longer_systems_reduce_into_it(n):
    """n = 8192 and 16384: the multi-pass path's reduced systems (2048 and
    4096 unit-diagonal rows) go through the one-pass kernel."""
    nsys = 5
    a, b, c, d = system(n, nsys, seed=n)
    dims = (n, nsys)
    ref = oracle.solve_mesh(a, b, c, d, dims, 0)
    ta, tb, tc, td = (torch.from_numpy(v).cuda() for v in (a, b, c, d))
    trid.solve(ta, tb, tc, td, dims, 0)
    torch.cuda.synchronize()
    assert normwise(td.cpu().numpy(), ref) <= TOL


def test_unaligned_arrays_take_the_multipass_path():
    """Arrays starting 4 bytes past a 16-byte boundary: same result as the
    aligned call within rounding (different tile boundaries)."""
    n, nsys = 1024, 9
    a, b, c, d = system(n, nsys, seed=11)
    dims = (n, nsys)
    ref = oracle.solve_mesh(a, b, c, d, dims, 0)
    bufs = []
    for v in (a, b, c, d):
        t = torch.empty(v.size + 1, dtype=torch.float32, device="cuda")
        t[1:] = torch.from_numpy(v).cuda()
        bufs.append(t[1:])
    trid.solve(*bufs, dims, 0)
    torch.cuda.synchronize()
    assert normwise(bufs[3].cpu().numpy(), ref) <= TOL


def test_matches_multipass_path_at_4096sq():
    """4096 x 4096 along x: the residual of every system and 200 sampled
    systems against the oracle."""
    n = nsys = 4096
    a, b, c, d = system(n, nsys, seed=21)
    rng = np.random.default_rng(2)
    idx = np.sort(rng.choice(nsys, 200, replace=False))
    ta, tb, tc, td = (torch.from_numpy(v).cuda() for v in (a, b, c, d))
    d0 = td.clone()
    trid.solve(ta, tb, tc, td, (n, nsys), 0)
    torch.cuda.synchronize()
    x = td.view(nsys, n)
    A, B, C, D = (t.view(nsys, n).double() for t in (ta, tb, tc, d0))
    X = x.double()
    r = B * X - D
    r[:, 1:] += A[:, 1:] * X[:, :-1]
    r[:, :-1] += C[:, :-1] * X[:, 1:]
    scale = (A.abs() + B.abs() + C.abs()).max() * X.abs().max() + D.abs().max()
    assert (r.abs().max() / scale).item() <= 8 * n * float(np.finfo(np.float32).eps)
    xs = x.cpu().numpy()[idx]
    rows = [slice(k * n, (k + 1) * n) for k in idx]
    ref = oracle.thomas_lines(*(np.stack([v[s] for s in rows]) for v in (a, b, c, d)))
    assert normwise(xs, ref) <= TOL


def test_many_batches_every_system_checked():
    """8192 systems of 4096 rows (two warp teams per block taking the batches
    in turn), solved three times: the residual of every system, each time.
    Guards the stage ring's invariant that a stage always serves the same
    team group (a group waiting on another group's stage could read a batch
    that is not yet there)."""
    n, nsys = 4096, 8192
    a, b, c, d = system(n, nsys, seed=77)
    ta, tb, tc, td0 = (torch.from_numpy(v).cuda() for v in (a, b, c, d))
    A, B, C, D = (t.view(nsys, n).double() for t in (ta, tb, tc, td0))
    scale = (A.abs() + B.abs() + C.abs()).max()
    for _ in range(3):
        td = td0.clone()
        trid.solve(ta, tb, tc, td, (n, nsys), 0)
        torch.cuda.synchronize()
        X = td.view(nsys, n).double()
        r = B * X - D
        r[:, 1:] += A[:, 1:] * X[:, :-1]
        r[:, :-1] += C[:, :-1] * X[:, 1:]
        per_sys = r.abs().amax(dim=1) / (scale * X.abs().amax(dim=1) + D.abs().amax(dim=1))
        assert per_sys.max().item() <= 8 * n * float(np.finfo(np.float32).eps)
