"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Tolerances: normwise max|x - x_ref| / max|x_ref| <= 1e-5 for FP32 and 1e-12 for
FP64 (inputs are diagonally dominant; the FP32 inputs are widened exactly to
FP64 for the oracle).  Small and ragged sizes are compared element by element
over the whole mesh; the full-size meshes on sampled systems the oracle
solves one by one, plus the residual |A x - d| over every system.
"""
import numpy as np
import pytest

import oracle
from paper_2201_03950_gb300 import inputs, trid

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {np.float32: 1e-5, np.float64: 1e-12}


def normwise(x, ref):
    x = np.asarray(x, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    return float(np.max(np.abs(x - ref)) / max(np.max(np.abs(ref)), 1e-300))


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2201_03950_gb300 import build
    build.build()
    assert torch.cuda.is_available()
    trid.load()


def to_dev(*arrs):
    return [torch.from_numpy(np.ascontiguousarray(v)).cuda() for v in arrs]


def run_mesh(dims, solve_dim, dtype, seed=0, accumulate=False, poison=True):
    total = int(np.prod(dims))
    a, b, c, d = inputs.dominant_system((total,), seed=seed, dtype=dtype)
    ref = oracle.solve_mesh(a, b, c, d, dims, solve_dim)
    ta, tb, tc, td = to_dev(a, b, c, d)
    if poison:
        # the unread a of each line's first row and c of its last row
        n = dims[solve_dim]
        stride = int(np.prod(dims[:solve_dim])) if solve_dim else 1
        idx = np.arange(total).reshape(tuple(reversed(dims)))
        first = np.take(idx, 0, axis=len(dims) - 1 - solve_dim).reshape(-1)
        last = np.take(idx, n - 1, axis=len(dims) - 1 - solve_dim).reshape(-1)
        assert stride >= 1
        ta[torch.from_numpy(first).cuda()] = float("nan")
        tc[torch.from_numpy(last).cuda()] = float("nan")
    if accumulate:
        u0 = inputs.random_rhs((total,), seed=seed + 1, dtype=dtype)
        tu = to_dev(u0)[0]
        d_before = td.clone()
        trid.solve(ta, tb, tc, td, dims, solve_dim, u=tu)
        torch.cuda.synchronize()
        assert torch.equal(td, d_before), "accumulate mode must leave d unmodified"
        got = tu.cpu().numpy().astype(np.float64) - u0.astype(np.float64)
        return got, ref
    trid.solve(ta, tb, tc, td, dims, solve_dim)
    torch.cuda.synchronize()
    return td.cpu().numpy(), ref


SMALL_CASES = [
    ((64, 64), 0), ((64, 64), 1),                      # 2D 64x64 (x then y)
    ((1,), 0), ((2,), 0), ((3,), 0), ((5,), 0), ((8,), 0), ((9,), 0), ((255,), 0), ((256,), 0),
    ((257,), 0), ((1000,), 0), ((3, 40), 0), ((7, 33), 1), ((31, 5, 9), 0), ((31, 5, 9), 1),
    ((31, 5, 9), 2), ((33, 17, 12), 2), ((100, 7), 0), ((100, 7), 1), ((37, 256), 1),
    ((37, 2, 256), 2), ((256, 3, 2), 0), ((13, 300), 1), ((300, 13), 0), ((9, 4, 600), 2),
    ((2050, 3), 0), ((5, 2050), 1), ((40, 9000), 1), ((9000, 3), 0),
]


@pytest.mark.parametrize("dtype", [np.float32, np.float64], ids=["f32", "f64"])
@pytest.mark.parametrize("dims,solve_dim", SMALL_CASES,
                         ids=[f"{'x'.join(map(str, d))}-dim{k}" for d, k in SMALL_CASES])
def test_mesh_elementwise(dims, solve_dim, dtype):
    got, ref = run_mesh(dims, solve_dim, dtype, seed=sum(dims) + solve_dim)
    assert np.all(np.isfinite(got))
    assert normwise(got, ref) <= TOL[dtype]


@pytest.mark.parametrize("dtype", [np.float32, np.float64], ids=["f32", "f64"])
@pytest.mark.parametrize("dims,solve_dim", [((64, 64), 0), ((31, 5, 9), 1), ((33, 17, 12), 2),
                                            ((600, 5), 0), ((6, 700), 1)])
def test_accumulate(dims, solve_dim, dtype):
    got, ref = run_mesh(dims, solve_dim, dtype, seed=3, accumulate=True)
    assert normwise(got, ref) <= 2 * TOL[dtype]


def test_config1_x_then_y():
    """2D 64x64 FP32: solve along x, then along y on the result."""
    dims = (64, 64)
    a, b, c, d = inputs.dominant_system((4096,), seed=0, dtype=np.float32)
    a2, b2, c2, _ = inputs.dominant_system((4096,), seed=1, dtype=np.float32)
    x1 = oracle.solve_mesh(a, b, c, d, dims, 0)
    x2 = oracle.solve_mesh(a2, b2, c2, x1, dims, 1)
    ta, tb, tc, td, ta2, tb2, tc2 = to_dev(a, b, c, d, a2, b2, c2)
    trid.solve(ta, tb, tc, td, dims, 0)
    trid.solve(ta2, tb2, tc2, td, dims, 1)
    assert normwise(td.cpu().numpy(), x2) <= 2e-5


def test_empty_mesh_is_noop():
    t = torch.zeros(0, device="cuda")
    trid.solve(t, t, t, t, (0, 5), 1)
    trid.solve(t, t, t, t, (7, 0, 3), 0)


def sampled_lines(dims, solve_dim, nsample, seed):
    """Indices (into the flat mesh) of `nsample` random whole systems."""
    n = dims[solve_dim]
    total = int(np.prod(dims))
    nsys = total // n
    rng = np.random.default_rng(seed)
    sys = rng.choice(nsys, size=min(nsample, nsys), replace=False)
    sys = np.unique(np.concatenate([sys, [0, nsys - 1]]))
    inner = int(np.prod(dims[:solve_dim])) if solve_dim else 1
    base = (sys % inner) + (sys // inner) * inner * n
    return base[:, None] + inner * np.arange(n)[None, :]


def residual_check(ta, tb, tc, td0, tx, dims, solve_dim, eps):
    """max_i |(A x - d)_i| / (|A|_inf |x|_inf + |d|_inf) over every system,
    evaluated with plain torch ops in FP64."""
    shp = tuple(reversed(dims))
    ax = len(dims) - 1 - solve_dim
    A, B, C, D, X = (t.double().reshape(shp) for t in (ta, tb, tc, td0, tx))
    r = B * X
    n = shp[ax]
    lo = [slice(None)] * len(shp)
    hi = [slice(None)] * len(shp)
    lo[ax] = slice(0, n - 1)
    hi[ax] = slice(1, n)
    r[tuple(hi)] += A[tuple(hi)] * X[tuple(lo)]
    r[tuple(lo)] += C[tuple(lo)] * X[tuple(hi)]
    r = r - D
    anorm = (A.abs() + B.abs() + C.abs()).max()
    val = (r.abs().max() / (anorm * X.abs().max() + D.abs().max())).item()
    assert val <= 8 * n * eps, f"residual {val:.3e}"
    return val


FULL = [((256, 256, 256), 0, np.float32), ((256, 256, 256), 1, np.float32),
        ((256, 256, 256), 2, np.float32), ((256, 256, 256), 0, np.float64),
        ((256, 256, 256), 1, np.float64), ((256, 256, 256), 2, np.float64),
        ((4096, 4096), 0, np.float32), ((4096, 4096), 1, np.float32)]


@pytest.mark.parametrize("dims,solve_dim,dtype", FULL,
                         ids=[f"{'x'.join(map(str, d))}-dim{k}-{t.__name__}" for d, k, t in FULL])
def test_full_size_sampled(dims, solve_dim, dtype):
    total = int(np.prod(dims))
    a, b, c, d = inputs.dominant_system((total,), seed=42 + solve_dim, dtype=dtype)
    idx = sampled_lines(dims, solve_dim, 300, seed=7)
    ref = oracle.thomas_lines(a[idx], b[idx], c[idx], d[idx])
    ta, tb, tc, td = to_dev(a, b, c, d)
    td0 = td.clone()
    trid.solve(ta, tb, tc, td, dims, solve_dim)
    torch.cuda.synchronize()
    x = td.cpu().numpy()
    assert np.all(np.isfinite(x))
    assert normwise(x[idx], ref) <= TOL[dtype]
    eps = float(np.finfo(dtype).eps)
    residual_check(ta, tb, tc, td0, td, dims, solve_dim, eps)


def test_long_path_workspace_entry_point():
    """trid_solve_batch_ws with caller scratch equals trid_solve_batch."""
    dims, k = (3000, 40), 0
    a, b, c, d = inputs.dominant_system((120000,), seed=5, dtype=np.float32)
    ta, tb, tc, td = to_dev(a, b, c, d)
    td2 = td.clone()
    need = trid.solve_workspace_bytes(dims, k, torch.float32)
    assert need > 0
    ws = torch.empty(need, dtype=torch.uint8, device="cuda")
    trid.solve(ta, tb, tc, td, dims, k, workspace=ws)
    trid.solve(ta, tb, tc, td2, dims, k)
    torch.cuda.synchronize()
    assert torch.equal(td, td2)
    ref = oracle.solve_mesh(a, b, c, d, dims, k)
    assert normwise(td.cpu().numpy(), ref) <= 1e-5


def test_error_codes_through_gpu_path():
    t = torch.zeros(64, device="cuda")
    with pytest.raises(trid.TridError) as e:
        trid.solve(t, t, t, t, (64,), 0, u=t)
    assert e.value.status == 1


# ---------------------------------------------------------------- ADI step
def adi_closed_form(dims, modes, lam, steps):
    import math
    out = np.zeros(int(np.prod(dims)))
    for ks, amp in modes:
        mus = [-4.0 * math.sin(math.pi * k / (2.0 * (n - 1))) ** 2 for k, n in zip(ks, dims)]
        g = 1.0 + lam * sum(mus) / np.prod([1.0 - lam * m for m in mus])
        out += inputs.sine_field(dims, [(ks, amp * g ** steps)])
    return out


def run_adi(u0, dims, lam, steps, dtype):
    tu = to_dev(u0.astype(dtype))[0]
    ws = torch.empty(trid.adi_workspace_bytes(dims, tu.dtype), dtype=torch.uint8, device="cuda")
    trid.adi_step(tu, dims, lam, steps, ws)
    torch.cuda.synchronize()
    return tu.cpu().numpy()


ADI_SMALL = [((9, 7, 6), 0.1, 3), ((40, 36, 33), 0.1, 10), ((64, 64, 64), 0.1, 5),
             ((33, 257 - 1, 17), 0.2, 2), ((12, 10), 0.3, 7), ((128, 100), 0.1, 20),
             ((3, 3, 3), 0.1, 2), ((24, 100, 7), 0.15, 3), ((16, 8, 5), 0.1, 2),
             ((256, 256, 3), 0.1, 2), ((32, 250, 9), 0.1, 2), ((8, 3, 4), 0.1, 1),
             ((200, 17, 12), 0.25, 2), ((64, 64, 160), 0.1, 2), ((32, 40, 250), 0.1, 1),
             ((256, 20, 40), 0.1, 1),
             # two-pass 3D schedule (all extents multiples of 16, nz >= 32)
             ((256, 32, 48), 0.1, 3), ((16, 16, 32), 0.3, 4), ((32, 256, 32), 0.2, 2),
             ((48, 80, 64), 0.15, 3), ((256, 256, 32), 0.1, 2), ((128, 48, 256), 0.1, 2),
             # windowed 3D schedule (FP32: nx % 8, ny % 32, nz % 16, lambda small enough):
             # three y tile kinds, lanes beyond the x line, one z tile, many z tiles
             ((256, 96, 64), 0.1, 2), ((24, 128, 16), 0.1, 3), ((200, 160, 80), 0.1, 2),
             ((8, 32, 32), 0.1, 2), ((64, 64, 256), 0.05, 2),
             # one 32-row tile per plane: several planes per CTA (16, 8, 4, 2),
             # widths that do not fill the lane groups
             ((16, 32, 48), 0.1, 2), ((24, 32, 32), 0.1, 3), ((64, 32, 16), 0.1, 2),
             ((120, 32, 32), 0.1, 2), ((40, 32, 80), 0.1, 2)]


@pytest.mark.parametrize("dtype", [np.float32, np.float64], ids=["f32", "f64"])
@pytest.mark.parametrize("dims,lam,steps", ADI_SMALL,
                         ids=[f"{'x'.join(map(str, d))}-{s}steps" for d, _, s in ADI_SMALL])
def test_adi_elementwise(dims, lam, steps, dtype):
    rng = np.random.default_rng(sum(dims))
    u0 = inputs.sine_field(dims, inputs.sine_modes(dims, seed=1)) + 0.0
    # add a random interior perturbation so that the test is not eigen-only
    pert = rng.uniform(-0.2, 0.2, u0.shape)
    grid = np.indices(tuple(reversed(dims))).reshape(len(dims), -1)[::-1]
    interior = np.ones(u0.size, dtype=bool)
    for ax, n in enumerate(dims):
        interior &= (grid[ax] > 0) & (grid[ax] < n - 1)
    u0 = (u0 + np.where(interior, pert, 0.0)).astype(dtype)
    ref = oracle.adi(u0, dims, lam, steps)
    got = run_adi(u0, dims, lam, steps, dtype)
    assert normwise(got, ref) <= TOL[dtype]


@pytest.mark.parametrize("dtype", [np.float32, np.float64], ids=["f32", "f64"])
@pytest.mark.parametrize("dims,lam", [((64, 48, 32), 0.2), ((40, 36, 33), 0.2), ((48, 32), 0.2),
                                      ((64, 64, 32), 0.1), ((256, 64, 48), 0.1)], ids=str)
def test_adi_nonzero_boundary(dims, lam, dtype):
    """Random u everywhere, boundary included: the boundary values must stay
    fixed and enter the neighbours' stencils exactly as in the oracle."""
    rng = np.random.default_rng(7)
    u0 = rng.uniform(-1.0, 1.0, int(np.prod(dims))).astype(dtype)
    ref = oracle.adi(u0, dims, lam, 3)
    got = run_adi(u0, dims, lam, 3, dtype)
    assert normwise(got, ref) <= TOL[dtype]


def test_adi_full_size_closed_form():
    """256^3 FP32, lambda = 0.1, 100 steps from 3 sine eigenmodes: the result
    must match the exact discrete decay A g^100 of each mode."""
    dims, lam, steps = (256, 256, 256), 0.1, 100
    modes = inputs.sine_modes(dims, seed=0)
    u0 = inputs.sine_field(dims, modes, dtype=np.float32)
    got = run_adi(u0, dims, lam, steps, np.float32)
    ref = adi_closed_form(dims, modes, lam, steps)
    assert normwise(got, ref) <= 1e-5
