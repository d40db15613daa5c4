"""The allocation-free entry point trid_solve_batch_noalloc.

It serves callers that cannot let a library call cudaMalloc (their own pool
owns the device memory, or they cannot afford the synchronisation of growing
a pool): the long-system scratch lives in one fixed device array.  Checked
here, through the C ABI, against trid_solve_batch on two calls in a row (the
second call reuses the array holding the first call's contents).  This file
is collected last so that a failure here leaves every other test already run.
"""
import ctypes

import numpy as np
import pytest

from paper_2201_03950_gb300 import build, inputs, trid

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {np.float32: 1e-5, np.float64: 1e-12}


def normwise(x, ref):
    x = np.asarray(x, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    return float(np.max(np.abs(x - ref)) / max(np.max(np.abs(ref)), 1e-300))


@pytest.fixture(scope="module")
def lib():
    build.build()
    assert torch.cuda.is_available()
    return trid.load()


def _call(lib, fn, ta, tb, tc, td, dims, k, dtype_code):
    dc = (ctypes.c_int64 * len(dims))(*dims)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return fn(ctypes.c_void_p(ta.data_ptr()), ctypes.c_void_p(tb.data_ptr()),
              ctypes.c_void_p(tc.data_ptr()), ctypes.c_void_p(td.data_ptr()), None, dc, len(dims),
              k, dtype_code, stream)


# (dims, axis, dtype, uses_scratch): the cases marked True are off the
# one-pass long-system path (FP64, longer than 4096 rows, or a contiguous
# length that is not a multiple of 4), so they run the multi-pass solve
# through the fixed array; the others are taken by the one-pass kernels.
CASES = [((3000, 40), 0, np.float32, False), ((48, 2100), 1, np.float32, False),
         ((1500, 30), 0, np.float64, True), ((200, 4, 600), 2, np.float32, False),
         ((5000, 64), 0, np.float32, True), ((64, 5000), 1, np.float32, True),
         ((1030, 50), 0, np.float32, True)]


def _off_one_pass(dims, k, dtype):
    n = dims[k]
    return dtype == np.float64 or n > 4096 or (k == 0 and n % 4 != 0)


@pytest.mark.parametrize("dims,k,dtype,uses_scratch", CASES)
def test_noalloc_matches_trid_solve_batch_twice(lib, dims, k, dtype, uses_scratch):
    total = int(np.prod(dims))
    code = 0 if dtype == np.float32 else 1
    need = lib.trid_solve_workspace_bytes((ctypes.c_int64 * len(dims))(*dims), len(dims), k, code)
    assert 0 < need <= lib_max()
    assert _off_one_pass(dims, k, dtype) == uses_scratch
    for call in range(2):  # two calls in a row share the fixed scratch array
        a, b, c, d = inputs.dominant_system((total,), seed=70 + call, dtype=dtype)
        ta, tb, tc, td = (torch.from_numpy(v).cuda() for v in (a, b, c, d))
        td_ref = td.clone()
        assert _call(lib, lib.trid_solve_batch, ta, tb, tc, td_ref, dims, k, code) == 0
        assert _call(lib, lib.trid_solve_batch_noalloc, ta, tb, tc, td, dims, k, code) == 0
        torch.cuda.synchronize()
        assert normwise(td.cpu().numpy(), td_ref.cpu().numpy()) <= TOL[dtype]


def lib_max():
    return 32 << 20


def test_noalloc_rejects_problems_beyond_its_scratch(lib):
    dims = (8192, 4096)  # needs more than the fixed 32 MiB
    need = lib.trid_solve_workspace_bytes((ctypes.c_int64 * 2)(*dims), 2, 0, 0)
    assert need > lib_max()
    # full-size arrays, so that no path the dispatch might take could reach
    # outside them; the problem is rejected on the host all the same
    ts = [torch.zeros(dims[0] * dims[1], device="cuda") for _ in range(4)]
    dc = (ctypes.c_int64 * 2)(*dims)
    p = [ctypes.c_void_p(t.data_ptr()) for t in ts]
    st = lib.trid_solve_batch_noalloc(p[0], p[1], p[2], p[3], None, dc, 2, 0, 0, None)
    torch.cuda.synchronize()
    assert st == 5  # TRID_ERR_ALLOC
    assert all(int(torch.count_nonzero(t)) == 0 for t in ts)  # nothing written
    del ts


def test_noalloc_short_systems_need_no_scratch(lib):
    dims = (256, 64)
    a, b, c, d = inputs.dominant_system((256 * 64,), seed=3, dtype=np.float32)
    ta, tb, tc, td = (torch.from_numpy(v).cuda() for v in (a, b, c, d))
    ref = td.clone()
    trid.solve(ta, tb, tc, ref, dims, 0)
    trid.solve_noalloc(ta, tb, tc, td, dims, 0)
    torch.cuda.synchronize()
    assert normwise(td.cpu().numpy(), ref.cpu().numpy()) <= 1e-5


@pytest.mark.parametrize("k", [0, 1], ids=["x", "y"])
def test_noalloc_one_pass_long_systems_need_no_scratch(lib, k):
    """4096 x 4096 FP32: the multi-pass scratch of this problem exceeds the
    fixed array, but the one-pass long-system kernels take it without
    scratch, so the allocation-free call solves it (the same kernels as
    trid_solve_batch: identical bits)."""
    dims = (4096, 4096)
    need = lib.trid_solve_workspace_bytes((ctypes.c_int64 * 2)(*dims), 2, k, 0)
    assert need > lib_max()
    a, b, c, d = inputs.dominant_system((4096 * 4096,), seed=31 + k, dtype=np.float32)
    ta, tb, tc, td = (torch.from_numpy(v).cuda() for v in (a, b, c, d))
    td_ref = td.clone()
    assert _call(lib, lib.trid_solve_batch, ta, tb, tc, td_ref, dims, k, 0) == 0
    assert _call(lib, lib.trid_solve_batch_noalloc, ta, tb, tc, td, dims, k, 0) == 0
    torch.cuda.synchronize()
    assert torch.equal(td, td_ref)
