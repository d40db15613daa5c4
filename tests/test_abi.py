"""The C-ABI library: builds, loads, exports every declared symbol, and rejects
bad arguments on the host before any launch (no GPU needed)."""
import ctypes
import os
import re

import pytest

from paper_2201_03950_gb300 import build, trid

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return trid.load()


def declared_functions():
    names = []
    for f in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not f.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", f)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^\s*[A-Za-z_][\w\s\*]*?\b(\w+)\s*\(", text, flags=re.M)
    return sorted(set(n for n in names if n not in ("defined",)))


def test_header_declares_entry_points():
    names = declared_functions()
    for required in ("trid_solve_batch", "trid_solve_batch_ws", "adi_step", "adi_workspace_bytes",
                     "trid_get_device_status", "trid_status_string"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), f"libtrid.so does not export {name}"


def test_status_strings(lib):
    for code, name in trid.STATUS.items():
        assert lib.trid_status_string(code).decode() == name
    assert b"sm_103a" in lib.trid_version()


def _dims(*v):
    return (ctypes.c_int64 * len(v))(*v)


def test_invalid_arguments_rejected_on_host(lib):
    p = ctypes.c_void_p(256)  # never dereferenced: rejected before any launch
    d3 = _dims(4, 4, 4)
    # bad ndim / solve_dim / dtype / dims
    assert lib.trid_solve_batch(p, p, p, p, None, d3, 0, 0, 0, None) == 1
    assert lib.trid_solve_batch(p, p, p, p, None, d3, 4, 0, 0, None) == 1
    assert lib.trid_solve_batch(p, p, p, p, None, d3, 3, 3, 0, None) == 1
    assert lib.trid_solve_batch(p, p, p, p, None, d3, 3, -1, 0, None) == 1
    assert lib.trid_solve_batch(p, p, p, p, None, d3, 3, 0, 7, None) == 1
    assert lib.trid_solve_batch(p, p, p, p, None, _dims(4, -1, 4), 3, 0, 0, None) == 1
    assert lib.trid_solve_batch(p, p, p, p, None, None, 3, 0, 0, None) == 1
    # NULL arrays
    assert lib.trid_solve_batch(None, p, p, p, None, d3, 3, 0, 0, None) == 1
    assert lib.trid_solve_batch(p, p, p, None, None, d3, 3, 0, 0, None) == 1
    # misaligned pointer for the element size
    q = ctypes.c_void_p(258)
    assert lib.trid_solve_batch(q, p, p, p, None, d3, 3, 0, 0, None) == 3
    assert lib.trid_solve_batch(ctypes.c_void_p(260), p, p, p, None, d3, 3, 0, 1, None) == 3
    # u aliasing a coefficient array
    assert lib.trid_solve_batch(p, p, p, p, p, d3, 3, 0, 0, None) == 1
    # empty mesh: valid, nothing to do (no launch)
    assert lib.trid_solve_batch(None, None, None, None, None, _dims(0, 4, 4), 3, 1, 0, None) == 0
    # overflow of the element count
    big = _dims(1 << 40, 1 << 30, 1)
    assert lib.trid_solve_batch(p, p, p, p, None, big, 3, 0, 0, None) == 1
    # workspace entry point: too small scratch for a long system
    long_dims = _dims(4096, 16)
    need = lib.trid_solve_workspace_bytes(long_dims, 2, 0, 0)
    assert need > 0
    assert lib.trid_solve_batch_ws(p, p, p, p, None, long_dims, 2, 0, 0, p, need - 1, None) == 5


def test_workspace_sizes(lib):
    assert lib.trid_solve_workspace_bytes(_dims(256, 256, 256), 3, 0, 0) == 0
    assert lib.trid_solve_workspace_bytes(_dims(256, 256, 256), 3, 2, 1) == 0
    assert lib.trid_solve_workspace_bytes(_dims(4096, 4096), 2, 1, 0) > 0
    assert lib.trid_solve_workspace_bytes(_dims(4, 4), 2, 2, 0) == 0  # invalid -> 0
    ws = lib.adi_workspace_bytes(_dims(256, 256, 256), 3, 0)
    assert ws >= 256 ** 3 * 4 and ws % 256 == 0
    assert lib.adi_workspace_bytes(_dims(2, 5), 2, 0) == 0


def test_adi_invalid_arguments(lib):
    p = ctypes.c_void_p(256)
    d = _dims(8, 8, 8)
    need = lib.adi_workspace_bytes(d, 3, 0)
    assert lib.adi_step(p, d, 1, 0.1, 1, 0, p, need, None) == 1          # ndim 1
    assert lib.adi_step(p, _dims(2, 8, 8), 3, 0.1, 1, 0, p, need, None) == 1
    assert lib.adi_step(p, d, 3, -0.1, 1, 0, p, need, None) == 1         # lambda <= 0
    assert lib.adi_step(p, d, 3, 0.1, -1, 0, p, need, None) == 1         # nsteps < 0
    assert lib.adi_step(None, d, 3, 0.1, 1, 0, p, need, None) == 1
    assert lib.adi_step(p, d, 3, 0.1, 1, 0, p, need - 1, None) == 5      # small workspace
    assert lib.adi_step(p, d, 3, 0.1, 1, 0, p, need, None) == 1          # u aliases workspace
    assert lib.adi_step(p, d, 3, 0.1, 1, 0, ctypes.c_void_p(1 << 20 | 8), need, None) == 3


def test_binding_refuses_missing_library(tmp_path):
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        trid.load(str(tmp_path / "missing.so"))


def test_varlen_histogram_key_buckets_and_dtype():
    """The autotuner's cache key: dtype, then systems per ceil-log2 length
    bucket (lengths 0 and 1 not counted), trailing empty buckets dropped."""
    import numpy as np
    off = np.array([0, 1, 3, 7, 8, 16, 33, 33], dtype=np.int64)  # lengths 1,2,4,1,8,17,0
    assert trid.varlen_histogram_key(off, "torch.float32") == "f32:0,1,1,1,0,1"
    assert trid.varlen_histogram_key(off, "torch.float64").startswith("f64:")
