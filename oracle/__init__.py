"""Oracle: plain FP64 CPU reference of the batched tridiagonal solve and ADI step.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import this package.  The
CUDA library never imports, links or calls it, and it imports nothing from the
CUDA path.

The arithmetic lives in ``trid_oracle.c`` (plain C, binary64, built with
``-ffp-contract=off``); this module compiles it with gcc on first use and wraps
it with ctypes over contiguous float64 numpy arrays.  Every function follows a
passage of arXiv 2201.03950 (cited in the C source):

* ``thomas``        -- Algorithm "thomas" (Section 2)
* ``pcr``           -- Algorithm "pcr" (Section 2)
* ``tiled``         -- tiled Thomas-Thomas / Thomas-PCR hybrid (Section 3.1)
* ``solve_mesh``    -- systems along one axis of a column-major mesh (Section 2.1)
* ``solve_mesh_f32`` -- the same in binary32 (the benchmark's like-for-like FP32
  CPU baseline only; never a parity reference)
* ``adi``           -- ADI heat diffusion step, Algorithm "adi" (Section 4.1)
* ``solve_varlen``  -- a batch of systems of different lengths
* ``adjoint``       -- transpose solve and coefficient gradients of one solve
* ``adi2v``         -- 2D ADI with a diffusivity field kappa (faces: node means)
* ``adi2v_grad``    -- its loss gradient w.r.t. u_0 and kappa (reverse mode)
* ``dense_solve``   -- Gaussian elimination with partial pivoting (brute force)

All parity is pinned (tests/test_oracle.py); no function is "parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "trid_oracle.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

CFLAGS = ["-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math"]


def build(force: bool = False, extra_flags: list[str] | None = None, out: str | None = None) -> str:
    """Compile ``trid_oracle.c`` into a shared library and return its path."""
    out = out or _LIB_PATH
    os.makedirs(os.path.dirname(out), exist_ok=True)
    if not force and extra_flags is None and os.path.exists(out) and \
            os.path.getmtime(out) >= os.path.getmtime(_SRC):
        return out
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", *CFLAGS, *(extra_flags or []), _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def _bind(lib):
    i64, i32, f64 = ctypes.c_int64, ctypes.c_int, ctypes.c_double
    P = ctypes.c_void_p
    sig = {
        "orc_thomas": [i64, P, P, P, P, P],
        "orc_pcr": [i64, P, P, P, P, P],
        "orc_dense_solve": [i64, P, P, P],
        "orc_tiled": [i64, i64, i32, P, P, P, P, P],
        "orc_thomas_lines": [i64, i64, P, P, P, P, P],
        "orc_solve_mesh": [P, P, P, P, P, P, i32, i32, i32],
        "orc_solve_mesh_f32": [P, P, P, P, P, P, i32, i32],
        "orc_adi": [P, P, i32, f64, i32],
        "orc_solve_varlen": [P, P, P, P, P, P, i64],
        "orc_adjoint": [i64, P, P, P, P, P, P, P, P, P],
        "orc_adi2v": [P, P, P, f64, i32],
        "orc_adi2v_grad": [P, P, P, P, f64, i32, P, P, P, P],
    }
    for name, args in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = ctypes.c_int
    return lib


def load(path: str | None = None):
    """Load (building if needed) the oracle library.  ``path`` loads a variant."""
    global _lib
    if path is not None:
        return _bind(ctypes.CDLL(path))
    with _lock:
        if _lib is None:
            _lib = _bind(ctypes.CDLL(build()))
    return _lib


def _f64(x) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(x, dtype=np.float64))


def _p(x: np.ndarray):
    return x.ctypes.data_as(ctypes.c_void_p)


def _check(rc: int, what: str):
    if rc == -2:
        raise ZeroDivisionError(f"oracle {what}: exact zero pivot")
    if rc != 0:
        raise ValueError(f"oracle {what}: bad argument (rc={rc})")


def thomas(a, b, c, d, lib=None) -> np.ndarray:
    lib = lib or load()
    a, b, c, d = map(_f64, (a, b, c, d))
    x = np.empty_like(d)
    _check(lib.orc_thomas(d.size, _p(a), _p(b), _p(c), _p(d), _p(x)), "thomas")
    return x


def pcr(a, b, c, d, lib=None) -> np.ndarray:
    lib = lib or load()
    a, b, c, d = map(_f64, (a, b, c, d))
    x = np.empty_like(d)
    _check(lib.orc_pcr(d.size, _p(a), _p(b), _p(c), _p(d), _p(x)), "pcr")
    return x


def tiled(a, b, c, d, m: int, use_pcr: bool, lib=None) -> np.ndarray:
    lib = lib or load()
    a, b, c, d = map(_f64, (a, b, c, d))
    x = np.empty_like(d)
    _check(lib.orc_tiled(d.size, m, int(use_pcr), _p(a), _p(b), _p(c), _p(d), _p(x)), "tiled")
    return x


def dense_solve(A, rhs, lib=None) -> np.ndarray:
    lib = lib or load()
    A, rhs = _f64(A), _f64(rhs)
    x = np.empty_like(rhs)
    _check(lib.orc_dense_solve(rhs.size, _p(A), _p(rhs), _p(x)), "dense_solve")
    return x


def thomas_lines(a, b, c, d, lib=None) -> np.ndarray:
    """Solve each row of 2D arrays [nsys, n] as one system."""
    lib = lib or load()
    a, b, c, d = map(_f64, (a, b, c, d))
    nsys, n = d.shape
    x = np.full_like(d, np.nan)  # a row the solver skips stays NaN
    _check(lib.orc_thomas_lines(nsys, n, _p(a), _p(b), _p(c), _p(d), _p(x)), "thomas_lines")
    return x


def _dims_c(dims):
    arr = (ctypes.c_int64 * 3)(*(list(dims) + [1] * (3 - len(dims))))
    return arr


def solve_mesh(a, b, c, d, dims, solve_dim: int, out=None, lib=None) -> np.ndarray:
    """Solve along ``solve_dim`` of a column-major mesh with shape ``dims``
    (dims[0] contiguous).  Arrays are flat (or any shape with that element
    order).  With ``out`` given, x is added into it (accumulate); otherwise a
    new array holding x is returned."""
    lib = lib or load()
    a, b, c, d = (_f64(v).reshape(-1) for v in (a, b, c, d))
    acc = out is not None
    if acc:
        if out.dtype != np.float64 or not out.flags.c_contiguous:
            raise TypeError("out must be a contiguous float64 array")
        res = out.reshape(-1)
    else:
        res = np.empty_like(d)
    _check(lib.orc_solve_mesh(_p(a), _p(b), _p(c), _p(d), _p(res), _dims_c(dims), len(dims),
                              solve_dim, int(acc)), "solve_mesh")
    return out if acc else res


def solve_mesh_f32(a, b, c, d, dims, solve_dim: int, out=None, lib=None) -> np.ndarray:
    """``solve_mesh`` in binary32 (x written to ``out`` or a new array)."""
    lib = lib or load()
    a, b, c, d = (np.ascontiguousarray(v, dtype=np.float32).reshape(-1) for v in (a, b, c, d))
    res = np.full_like(d, np.nan) if out is None else out.reshape(-1)  # unwritten stays NaN
    if res.dtype != np.float32 or not res.flags.c_contiguous:
        raise TypeError("out must be a contiguous float32 array")
    _check(lib.orc_solve_mesh_f32(_p(a), _p(b), _p(c), _p(d), _p(res), _dims_c(dims), len(dims),
                                  solve_dim), "solve_mesh_f32")
    return res


def adi(u, dims, lam: float, nsteps: int, lib=None) -> np.ndarray:
    """Return u after ``nsteps`` ADI steps (u is not modified)."""
    lib = lib or load()
    w = _f64(u).reshape(-1).copy()
    _check(lib.orc_adi(_p(w), _dims_c(dims), len(dims), float(lam), int(nsteps)), "adi")
    return w


def solve_varlen(a, b, c, d, offsets, lib=None) -> np.ndarray:
    lib = lib or load()
    a, b, c, d = map(_f64, (a, b, c, d))
    off = np.ascontiguousarray(np.asarray(offsets, dtype=np.int64))
    x = np.empty_like(d)
    _check(lib.orc_solve_varlen(_p(a), _p(b), _p(c), _p(d), _p(x), _p(off), off.size - 1),
           "solve_varlen")
    return x


def adjoint(a, b, c, x, gx, lib=None):
    """Return (g_a, g_b, g_c, g_d) for one system."""
    lib = lib or load()
    a, b, c, x, gx = map(_f64, (a, b, c, x, gx))
    ga, gb, gc, gd = (np.empty_like(x) for _ in range(4))
    _check(lib.orc_adjoint(x.size, _p(a), _p(b), _p(c), _p(x), _p(gx), _p(ga), _p(gb), _p(gc),
                           _p(gd)), "adjoint")
    return ga, gb, gc, gd


def adi2v(u, kappa, dims, lam: float, nsteps: int, lib=None) -> np.ndarray:
    """2D ADI with diffusivity field ``kappa``: u after ``nsteps`` steps."""
    lib = lib or load()
    w = _f64(u).reshape(-1).copy()
    k = _f64(kappa).reshape(-1)
    _check(lib.orc_adi2v(_p(w), _p(k), _dims_c(dims), float(lam), int(nsteps)), "adi2v")
    return w


def adi2v_grad(u0, kappa, target, dims, lam: float, nsteps: int, lib=None):
    """Return (loss, g_u0, g_kappa, g_coef) for L = mean((u_T - target)^2);
    g_coef is [6, n]: summed raw gradients of ax, bx, cx, ay, by, cy."""
    lib = lib or load()
    u0, k, tg = (_f64(v).reshape(-1) for v in (u0, kappa, target))
    gu, gk = np.empty_like(u0), np.empty_like(u0)
    gc = np.empty((6, u0.size))
    loss = ctypes.c_double(0.0)
    _check(lib.orc_adi2v_grad(_p(u0), _p(k), _p(tg), _dims_c(dims), float(lam), int(nsteps),
                              ctypes.byref(loss), _p(gu), _p(gk), _p(gc)), "adi2v_grad")
    return loss.value, gu, gk, gc
