"""Library lifecycle through the C ABI: trid_init pre-sizes the scratch pool so
that a multi-pass solve can be captured into a CUDA graph (nothing is
allocated inside the capture), and trid_finalize frees the pool and forgets
the device's cached state, after which every entry point works again."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2201_03950_gb300 import build, inputs, trid

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DIMS = (1500, 40)  # 40 FP64 systems of 1500 rows: the multi-pass path, needs scratch


@pytest.fixture(scope="module")
def lib():
    build.build()
    assert torch.cuda.is_available()
    return trid.load()


def _problem(seed):
    total = DIMS[0] * DIMS[1]
    a, b, c, d = inputs.dominant_system((total,), seed=seed, dtype=np.float64)
    ref = oracle.thomas_lines(*(v.reshape(DIMS[1], DIMS[0]) for v in (a, b, c, d))).reshape(-1)
    return [torch.from_numpy(v).cuda() for v in (a, b, c, d)], ref


def _normwise(x, ref):
    return float(np.max(np.abs(x - ref)) / np.max(np.abs(ref)))


def test_init_presizes_pool_for_graph_capture_and_finalize_resets(lib):
    need = lib.trid_solve_workspace_bytes((ctypes.c_int64 * 2)(*DIMS), 2, 0, 1)
    assert need > 0
    trid.finalize()  # no pool on this device from earlier tests
    trid.init(need)
    (ta, tb, tc, td), ref = _problem(seed=11)
    work = td.clone()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):  # would fail if the call grew the pool here
        trid.solve(ta, tb, tc, work, DIMS, 0)
    for _ in range(2):
        work.copy_(td)
        g.replay()
        torch.cuda.synchronize()
        assert _normwise(work.cpu().numpy(), ref) <= 1e-12
    del g
    torch.cuda.synchronize()

    trid.finalize()
    # after finalize: the pool is regrown on demand, the allocation-free
    # array's address and the status word are looked up again
    (ta, tb, tc, td), ref = _problem(seed=12)
    for fn in (trid.solve, trid.solve_noalloc):
        work = td.clone()
        fn(ta, tb, tc, work, DIMS, 0)
        torch.cuda.synchronize()
        assert _normwise(work.cpu().numpy(), ref) <= 1e-12
    assert trid.device_status() == 0


def test_init_is_idempotent_and_only_grows(lib):
    trid.init(0)
    trid.init(1 << 20)
    trid.init(1 << 10)  # smaller request keeps the larger pool
    (ta, tb, tc, td), ref = _problem(seed=13)
    trid.solve(ta, tb, tc, td, DIMS, 0)
    torch.cuda.synchronize()
    assert _normwise(td.cpu().numpy(), ref) <= 1e-12


def test_finalize_then_overlapped_backward(lib):
    """The differentiable ADI backward with several segments uses the
    library's auxiliary stream; after trid_finalize destroys it, the next call
    creates it again and gives the same bits as before (and as one segment,
    which runs on the caller's stream only)."""
    dims, lam, steps = (64, 48), 0.2, 9
    n = dims[0] * dims[1]
    u0 = torch.from_numpy(inputs.target_field(dims, seed=1).astype(np.float32)).cuda()
    kap = torch.from_numpy(inputs.diffusivity_field(dims, seed=2).astype(np.float32)).cuda()
    g = torch.from_numpy(inputs.random_rhs((n,), seed=3, dtype=np.float32)).cuda()

    def grads(every):
        _, ck = trid.adi2v_forward(u0, kap, dims, lam, steps, every)
        gu, gk, _ = trid.adi2v_backward(g, kap, dims, lam, steps, every, ck)
        torch.cuda.synchronize()
        return gu.cpu().numpy(), gk.cpu().numpy()

    before = grads(3)  # three segments: recomputation on the auxiliary stream
    trid.finalize()
    after = grads(3)
    single = grads(9)  # one segment
    for a, b, c in zip(before, after, single):
        assert np.array_equal(a, b)
        assert np.array_equal(a, c)
    assert trid.device_status() == 0
