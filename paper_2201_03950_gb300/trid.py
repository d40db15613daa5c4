"""Thin ctypes binding of the C ABI in ``include/trid.h`` (libtrid.so).

Argument marshalling only: device pointers come from torch CUDA tensors
(``tensor.data_ptr()``), the stream from ``torch.cuda.current_stream()``, and
every step of the computation runs in the library's CUDA kernels.  There is no
CPU fallback: if the library is missing or fails to load, every call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

TRID_F32, TRID_F64 = 0, 1
STATUS = {0: "TRID_OK", 1: "TRID_ERR_INVALID_ARG", 2: "TRID_ERR_UNSUPPORTED",
          3: "TRID_ERR_MISALIGNED", 4: "TRID_ERR_CUDA", 5: "TRID_ERR_ALLOC",
          6: "TRID_ERR_TIMEOUT"}

_lock = threading.Lock()
_lib = None


class TridError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        msg = f"{what}: {STATUS.get(status, status)}"
        if status == 4 and _lib is not None:
            msg += f" ({_lib.trid_last_cuda_error().decode()})"
        super().__init__(msg)


def lib_path() -> str:
    """The library ``load()`` opens: the debug build (device-side index checks,
    ``build.build(debug_bounds=True)``) when TRID_DEBUG_BOUNDS=1, else the
    release build."""
    return _build.LIB_DBG if os.environ.get("TRID_DEBUG_BOUNDS") == "1" else _build.LIB


def load(path: str | None = None):
    """Load libtrid.so (built in-tree by ``build.build()``); raise if absent."""
    global _lib
    with _lock:
        if _lib is None or path is not None:
            p = path or lib_path()
            if not os.path.exists(p):
                raise RuntimeError(f"CUDA library {p} is missing: run build() first "
                                   "(there is no CPU fallback)")
            L = ctypes.CDLL(p)
            _bind(L)
            if path is not None:
                return L
            _lib = L
    return _lib


def _bind(L):
    P, i32, i64, f64, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double, ctypes.c_size_t
    sigs = {
        "trid_solve_batch": ([P, P, P, P, P, P, i32, i32, i32, P], i32),
        "trid_solve_batch_ws": ([P, P, P, P, P, P, i32, i32, i32, P, sz, P], i32),
        "trid_solve_batch_noalloc": ([P, P, P, P, P, P, i32, i32, i32, P], i32),
        "trid_solve_workspace_bytes": ([P, i32, i32, i32], sz),
        "trid_solve_batch_varlen": ([P, P, P, P, P, P, i64, i64, i64, i32, P, sz, P], i32),
        "trid_solve_varlen_workspace_bytes": ([i64], sz),
        "trid_solve_batch_varlen_cfg": ([P, P, P, P, P, P, i64, i64, i64, i32, P, sz, P, P], i32),
        "trid_varlen_autotune_workspace_bytes": ([i64, i64, i32], sz),
        "trid_varlen_autotune": ([P, P, P, P, P, i64, i64, i64, i32, P, sz, P, P, P], i32),
        "trid_solve_batch_adjoint": ([P, P, P, P, P, P, P, P, P, P, i32, i32, i32, P, sz, P], i32),
        "trid_adjoint_workspace_bytes": ([P, i32, i32, i32], sz),
        "adi_step": ([P, P, i32, f64, i32, i32, P, sz, P], i32),
        "adi_workspace_bytes": ([P, i32, i32], sz),
        "adi_batched_workspace_bytes": ([i64, P, i32, i32], sz),
        "adi_step_batched": ([P, i64, P, i32, f64, i32, i32, P, sz, P], i32),
        "adi2v_workspace_bytes": ([P, i32, i32, i32], sz),
        "adi2v_checkpoint_bytes": ([P, i32, i32, i32], sz),
        "adi2v_forward": ([P, P, P, P, f64, i32, i32, P, sz, i32, P, sz, P], i32),
        "adi2v_backward": ([P, P, P, P, P, P, f64, i32, i32, P, sz, i32, P, sz, P], i32),
        "trid_get_device_status": ([P], i32),
        "trid_wait_flag": ([P, i32, f64, P], i32),
        "trid_status_string": ([i32], ctypes.c_char_p),
        "trid_last_cuda_error": ([], ctypes.c_char_p),
        "trid_version": ([], ctypes.c_char_p),
        "trid_init": ([sz], i32),
        "trid_fp64_rates": ([P, P, P], i32),
        "trid_finalize": ([], i32),
    }
    for name, (args, res) in sigs.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = res


def _dims(dims):
    n = len(dims)
    return (ctypes.c_int64 * max(n, 1))(*[int(v) for v in dims]), n


def _dtype(t) -> int:
    import torch
    if t.dtype == torch.float32:
        return TRID_F32
    if t.dtype == torch.float64:
        return TRID_F64
    raise TypeError(f"unsupported dtype {t.dtype}")


def _stream(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _check_tensors(ts, dtype_ref, numel):
    for t in ts:
        if t is None:
            continue
        if not t.is_cuda:
            raise ValueError("tensors must be CUDA tensors")
        if t.dtype != dtype_ref.dtype:
            raise TypeError("all arrays must share one dtype")
        if not t.is_contiguous() or t.numel() != numel:
            raise ValueError(f"arrays must be contiguous with {numel} elements")


def solve(a, b, c, d, dims, solve_dim: int, u=None, workspace=None, stream=None):
    """Batched solve along ``solve_dim`` of a column-major mesh ``dims``
    (dims[0] contiguous).  u is None: x overwrites d.  Otherwise u += x."""
    numel = 1
    for v in dims:
        numel *= int(v)
    _check_tensors((a, b, c, d, u), d, numel)
    L = load()
    dc, nd = _dims(dims)
    if workspace is None:
        st = L.trid_solve_batch(_ptr(a), _ptr(b), _ptr(c), _ptr(d), _ptr(u), dc, nd, solve_dim,
                                _dtype(d), _stream(stream))
    else:
        st = L.trid_solve_batch_ws(_ptr(a), _ptr(b), _ptr(c), _ptr(d), _ptr(u), dc, nd,
                                   solve_dim, _dtype(d), _ptr(workspace),
                                   workspace.numel() * workspace.element_size(), _stream(stream))
    if st != 0:
        raise TridError(st, "trid_solve_batch")
    return u if u is not None else d


def solve_noalloc(a, b, c, d, dims, solve_dim: int, u=None, stream=None):
    """As ``solve``, through trid_solve_batch_noalloc: for callers that must not
    let the library allocate device memory (the long-system scratch comes from
    a fixed 32 MiB device array; see include/trid.h)."""
    numel = 1
    for v in dims:
        numel *= int(v)
    _check_tensors((a, b, c, d, u), d, numel)
    L = load()
    dc, nd = _dims(dims)
    st = L.trid_solve_batch_noalloc(_ptr(a), _ptr(b), _ptr(c), _ptr(d), _ptr(u), dc, nd,
                                    solve_dim, _dtype(d), _stream(stream))
    if st != 0:
        raise TridError(st, "trid_solve_batch_noalloc")
    return u if u is not None else d


def adjoint(a, b, c, x, gx, dims, solve_dim: int, need_coef_grads: bool = True, stream=None):
    """Gradients of L through x = A^{-1} d along ``solve_dim``: returns
    (g_a, g_b, g_c, g_d) (the first three None if ``need_coef_grads`` is
    False).  All arrays are CUDA tensors with the forward call's layout."""
    import torch
    numel = 1
    for v in dims:
        numel *= int(v)
    _check_tensors((a, b, c, x, gx), x, numel)
    L = load()
    dc, nd = _dims(dims)
    gd = torch.empty_like(x)
    ga = torch.empty_like(x) if need_coef_grads else None
    gb = torch.empty_like(x) if need_coef_grads else None
    gc = torch.empty_like(x) if need_coef_grads else None
    nbytes = int(L.trid_adjoint_workspace_bytes(dc, nd, solve_dim, _dtype(x)))
    ws = torch.empty(max(nbytes, 1), dtype=torch.uint8, device=x.device) if nbytes else None
    st = L.trid_solve_batch_adjoint(_ptr(a), _ptr(b), _ptr(c), _ptr(x), _ptr(gx), _ptr(ga),
                                    _ptr(gb), _ptr(gc), _ptr(gd), dc, nd, solve_dim, _dtype(x),
                                    _ptr(ws), nbytes, _stream(stream))
    if st != 0:
        raise TridError(st, "trid_solve_batch_adjoint")
    return ga, gb, gc, gd


def varlen_workspace_bytes(nsys: int) -> int:
    return int(load().trid_solve_varlen_workspace_bytes(int(nsys)))


class VarlenConfig(ctypes.Structure):
    """Length classes, tile height and team size of the uneven-batch solver
    (trid_varlen_config; tile_rows 0 means 8, team_warps 0 means 4)."""
    _fields_ = [("team_max", ctypes.c_int32), ("block_max", ctypes.c_int32),
                ("tile_rows", ctypes.c_int32), ("team_warps", ctypes.c_int32)]

    def __repr__(self):
        return (f"VarlenConfig(team_max={self.team_max}, block_max={self.block_max}, "
                f"tile_rows={self.tile_rows or 8}, team_warps={self.team_warps or 4})")


def _check_offsets(offsets):
    import torch
    if not (offsets.is_cuda and offsets.dtype == torch.int64 and offsets.is_contiguous()):
        raise ValueError("offsets must be a contiguous int64 CUDA tensor")


def solve_varlen(a, b, c, d, offsets, max_len: int, u=None, workspace=None, stream=None,
                 config: VarlenConfig | None = None):
    """Batch of systems of different lengths: system k occupies rows
    [offsets[k], offsets[k+1]) (offsets: int64 CUDA tensor of nsys + 1).
    ``config``: length classes and tile height (e.g. from ``varlen_autotune``);
    None = defaults."""
    import torch
    total = d.numel()
    _check_tensors((a, b, c, d, u), d, total)
    _check_offsets(offsets)
    nsys = offsets.numel() - 1
    L = load()
    if workspace is None:
        workspace = torch.empty(varlen_workspace_bytes(max(nsys, 0)), dtype=torch.uint8,
                                device=d.device)
    args = (_ptr(a), _ptr(b), _ptr(c), _ptr(d), _ptr(u), _ptr(offsets), int(nsys), int(total),
            int(max_len), _dtype(d), _ptr(workspace), workspace.numel() * workspace.element_size(),
            _stream(stream))
    if config is None:
        st = L.trid_solve_batch_varlen(*args)
    else:
        st = L.trid_solve_batch_varlen_cfg(*args, ctypes.byref(config))
    if st != 0:
        raise TridError(st, "trid_solve_batch_varlen")
    return u if u is not None else d


def varlen_histogram_key(offsets, dtype) -> str:
    """Cache key of an uneven batch: the dtype and the number of systems in
    each power-of-two length bucket (the buckets the planning pass sorts by)."""
    import numpy as np
    off = offsets.detach().to("cpu").numpy() if hasattr(offsets, "detach") else np.asarray(offsets)
    lens = np.diff(off.astype(np.int64))
    buckets = np.zeros(64, dtype=np.int64)
    nz = lens[lens > 1]
    np.add.at(buckets, np.ceil(np.log2(nz)).astype(np.int64), 1)
    last = int(np.max(np.nonzero(buckets)[0])) + 1 if buckets.any() else 0
    return f"{'f32' if str(dtype).endswith('float32') else 'f64'}:" + ",".join(
        str(int(v)) for v in buckets[:last])


def _tune_cache_path():
    import os
    return os.environ.get("TRID_TUNE_CACHE") or os.path.join(
        os.path.expanduser("~"), ".cache", "gb300-trid", "varlen_tune.json")


def varlen_autotune(a, b, c, d, offsets, max_len: int, stream=None, cache: bool = True):
    """Time every admissible configuration (tile height, length classes) on this batch (d is
    not modified) and return (best VarlenConfig, its time in ms).  With
    ``cache`` the choice is kept in a JSON file (TRID_TUNE_CACHE, else
    ~/.cache/gb300-trid/varlen_tune.json) keyed by dtype and length histogram;
    a batch with a known key returns the stored choice (time -1.0) without
    timing anything."""
    import json
    import os
    import torch
    total = d.numel()
    _check_tensors((a, b, c, d), d, total)
    _check_offsets(offsets)
    nsys = offsets.numel() - 1
    key = varlen_histogram_key(offsets, d.dtype) if cache else None
    table = {}
    if cache:
        try:
            with open(_tune_cache_path()) as fh:
                table = json.load(fh)
        except (OSError, ValueError):
            table = {}
        hit = table.get(key)
        if hit is not None:
            return VarlenConfig(int(hit["team_max"]), int(hit["block_max"]),
                                int(hit.get("tile_rows", 8)), int(hit.get("team_warps", 4))), -1.0
    L = load()
    ws = torch.empty(max(int(L.trid_varlen_autotune_workspace_bytes(nsys, total, _dtype(d))), 1),
                     dtype=torch.uint8, device=d.device)
    best = VarlenConfig()
    ms = ctypes.c_float(0.0)
    st = L.trid_varlen_autotune(_ptr(a), _ptr(b), _ptr(c), _ptr(d), _ptr(offsets), int(nsys),
                                int(total), int(max_len), _dtype(d), _ptr(ws),
                                ws.numel(), _stream(stream), ctypes.byref(best),
                                ctypes.byref(ms))
    if st != 0:
        raise TridError(st, "trid_varlen_autotune")
    if cache:
        table[key] = {"team_max": int(best.team_max), "block_max": int(best.block_max),
                      "tile_rows": int(best.tile_rows or 8),
                      "team_warps": int(best.team_warps or 4), "ms": float(ms.value)}
        path = _tune_cache_path()
        try:
            os.makedirs(os.path.dirname(path), exist_ok=True)
            tmp = f"{path}.tmp{os.getpid()}"
            with open(tmp, "w") as fh:
                json.dump(table, fh, indent=1, sort_keys=True)
            os.replace(tmp, path)
        except OSError:
            pass  # an unwritable cache only costs a re-tune next time
    return best, float(ms.value)


def solve_workspace_bytes(dims, solve_dim: int, dtype) -> int:
    dc, nd = _dims(dims)
    code = TRID_F32 if str(dtype).endswith("float32") else TRID_F64
    return int(load().trid_solve_workspace_bytes(dc, nd, solve_dim, code))


def adi_workspace_bytes(dims, dtype) -> int:
    dc, nd = _dims(dims)
    code = TRID_F32 if str(dtype).endswith("float32") else TRID_F64
    return int(load().adi_workspace_bytes(dc, nd, code))


def adi_step(u, dims, lam: float, nsteps: int, workspace, stream=None):
    """Advance u in place by ``nsteps`` ADI steps (Dirichlet-zero boundary)."""
    numel = 1
    for v in dims:
        numel *= int(v)
    _check_tensors((u,), u, numel)
    L = load()
    dc, nd = _dims(dims)
    st = L.adi_step(_ptr(u), dc, nd, float(lam), int(nsteps), _dtype(u), _ptr(workspace),
                    workspace.numel() * workspace.element_size(), _stream(stream))
    if st != 0:
        raise TridError(st, "adi_step")
    return u


def adi_step_batched(u, nbatch: int, dims, lam: float, nsteps: int, workspace=None,
                     stream=None):
    """Advance each of the ``nbatch`` meshes stored back to back in ``u`` by
    ``nsteps`` ADI steps (see include/trid.h)."""
    import torch
    per = 1
    for v in dims:
        per *= int(v)
    _check_tensors((u,), u, per * int(nbatch))
    L = load()
    dc, nd = _dims(dims)
    need = int(L.adi_batched_workspace_bytes(int(nbatch), dc, nd, _dtype(u)))
    if workspace is None and need:
        workspace = torch.empty(need, dtype=torch.uint8, device=u.device)
    st = L.adi_step_batched(_ptr(u), int(nbatch), dc, nd, float(lam), int(nsteps), _dtype(u),
                            _ptr(workspace), 0 if workspace is None else _bytes(workspace),
                            _stream(stream))
    if st != 0:
        raise TridError(st, "adi_step_batched")
    return u


def _code(dtype) -> int:
    return TRID_F32 if str(dtype).endswith("float32") else TRID_F64


def adi2v_workspace_bytes(dims, nsteps: int, every: int, dtype) -> int:
    dc, _ = _dims(dims)
    return int(load().adi2v_workspace_bytes(dc, int(nsteps), int(every), _code(dtype)))


def adi2v_checkpoint_bytes(dims, nsteps: int, every: int, dtype) -> int:
    dc, _ = _dims(dims)
    return int(load().adi2v_checkpoint_bytes(dc, int(nsteps), int(every), _code(dtype)))


def _bytes(t):
    return t.numel() * t.element_size()


def adi2v_forward(u0, kappa, dims, lam: float, nsteps: int, every: int = 10, uT=None,
                  ckpt=None, workspace=None, stream=None):
    """2D ADI with diffusivity field ``kappa`` (see include/trid.h): returns
    (uT, ckpt).  ``ckpt`` (uint8 device tensor) keeps the states the backward
    call recomputes from; pass ckpt=False to skip keeping them."""
    import torch
    n = int(dims[0]) * int(dims[1])
    _check_tensors((u0, kappa, uT), u0, n)
    L = load()
    dc, _ = _dims(dims)
    code = _dtype(u0)
    if uT is None:
        uT = torch.empty_like(u0)
    if ckpt is None:
        ckpt = torch.empty(adi2v_checkpoint_bytes(dims, nsteps, every, u0.dtype),
                           dtype=torch.uint8, device=u0.device)
    if workspace is None:
        workspace = torch.empty(adi2v_workspace_bytes(dims, nsteps, every, u0.dtype),
                                dtype=torch.uint8, device=u0.device)
    ck = None if ckpt is False else ckpt
    st = L.adi2v_forward(_ptr(u0), _ptr(uT), _ptr(kappa), dc, float(lam), int(nsteps),
                         int(every), _ptr(ck), 0 if ck is None else _bytes(ck), code,
                         _ptr(workspace), _bytes(workspace), _stream(stream))
    if st != 0:
        raise TridError(st, "adi2v_forward")
    return uT, ck


def adi2v_backward(g_uT, kappa, dims, lam: float, nsteps: int, every: int, ckpt,
                   want_coef: bool = False, workspace=None, stream=None):
    """Returns (g_u0, g_kappa, g_coef) where g_coef is a [6, n] tensor of the
    summed gradients w.r.t. ax, bx, cx, ay, by, cy (None unless want_coef)."""
    import torch
    n = int(dims[0]) * int(dims[1])
    _check_tensors((g_uT, kappa), g_uT, n)
    L = load()
    dc, _ = _dims(dims)
    code = _dtype(g_uT)
    g_u0 = torch.empty_like(g_uT)
    g_k = torch.empty_like(g_uT)
    g_coef = torch.empty((6, n), dtype=g_uT.dtype, device=g_uT.device) if want_coef else None
    if workspace is None:
        workspace = torch.empty(adi2v_workspace_bytes(dims, nsteps, every, g_uT.dtype),
                                dtype=torch.uint8, device=g_uT.device)
    st = L.adi2v_backward(_ptr(g_uT), _ptr(g_u0), _ptr(g_k), _ptr(g_coef), _ptr(kappa), dc,
                          float(lam), int(nsteps), int(every), _ptr(ckpt), _bytes(ckpt), code,
                          _ptr(workspace), _bytes(workspace), _stream(stream))
    if st != 0:
        raise TridError(st, "adi2v_backward")
    return g_u0, g_k, g_coef


def wait_flag(flag, expect: int, timeout_s: float, stream=None):
    """Bounded device wait until the int32 CUDA tensor ``flag`` equals
    ``expect``; on expiry TRID_ERR_TIMEOUT is recorded in the device status
    word (read it with ``device_status``)."""
    import torch
    if not (flag.is_cuda and flag.dtype == torch.int32 and flag.numel() >= 1):
        raise ValueError("flag must be an int32 CUDA tensor")
    st = load().trid_wait_flag(_ptr(flag), int(expect), float(timeout_s), _stream(stream))
    if st != 0:
        raise TridError(st, "trid_wait_flag")


def device_status(stream=None) -> int:
    return int(load().trid_get_device_status(_stream(stream)))


def status_string(code: int) -> str:
    return load().trid_status_string(int(code)).decode()


def version() -> str:
    return load().trid_version().decode()


def init(pool_bytes: int = 0) -> None:
    """trid_init: set up the current device and make the scratch pool at least
    ``pool_bytes`` bytes, so later solves that fit it allocate nothing."""
    st = load().trid_init(int(pool_bytes))
    if st != 0:
        raise TridError(st, "trid_init")


def finalize() -> None:
    """trid_finalize: synchronise the current device, free the scratch pool
    and forget the library's cached state of that device."""
    st = load().trid_finalize()
    if st != 0:
        raise TridError(st, "trid_finalize")


def fp64_rates(stream=None):
    """trid_fp64_rates: (FMA, division) rates of the current device in 10^9/s."""
    f, d = ctypes.c_double(), ctypes.c_double()
    st = load().trid_fp64_rates(ctypes.byref(f), ctypes.byref(d), _stream(stream))
    if st != 0:
        raise TridError(st, "trid_fp64_rates")
    return f.value, d.value
