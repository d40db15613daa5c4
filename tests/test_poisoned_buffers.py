"""Outputs, workspaces and checkpoint buffers filled with NaN before a call:
every value the library reads from them must first be written by the call
itself, so the results must equal those of a call on freshly allocated
buffers.  A kernel that reads an unwritten output or scratch value, or leaves
part of an output unwritten, shows up as NaN here.  GPU only, through the
C ABI and its Python binding."""
import ctypes

import numpy as np
import pytest

from paper_2201_03950_gb300 import build, inputs, trid

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    build.build()
    assert torch.cuda.is_available()
    return trid.load()


def nan_bytes(nbytes):
    t = torch.empty(max(int(nbytes), 8) // 8 + 1, dtype=torch.float64, device="cuda")
    t.fill_(float("nan"))
    return t.view(torch.uint8)[: max(int(nbytes), 1)]


def dims_c(dims):
    return (ctypes.c_int64 * len(dims))(*dims), len(dims)


def P(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


@pytest.mark.parametrize("dims,k,dt", [((300, 7), 0, torch.float32), ((64, 32, 8), 2, torch.float32),
                                       ((40, 500), 1, torch.float64)], ids=str)
def test_adjoint_outputs_and_workspace_poisoned(lib, dims, k, dt):
    n = int(np.prod(dims))
    npdt = np.float32 if dt == torch.float32 else np.float64
    a, b, c, d = (torch.from_numpy(v).cuda() for v in inputs.dominant_system((n,), seed=3, dtype=npdt))
    x = d.clone()
    trid.solve(a, b, c, x, dims, k)
    gx = torch.from_numpy(inputs.random_rhs((n,), seed=4, dtype=npdt)).cuda()
    ref = trid.adjoint(a, b, c, x, gx, dims, k)
    outs = [torch.full_like(x, float("nan")) for _ in range(4)]
    dc, nd = dims_c(dims)
    code = 0 if dt == torch.float32 else 1
    nb = lib.trid_adjoint_workspace_bytes(dc, nd, k, code)
    ws = nan_bytes(nb) if nb else None
    st = lib.trid_solve_batch_adjoint(P(a), P(b), P(c), P(x), P(gx), *(P(o) for o in outs), dc, nd,
                                      k, code, P(ws), nb, stream())
    torch.cuda.synchronize()
    assert st == 0
    for got, want in zip(outs, ref):
        assert torch.equal(got, want)


@pytest.mark.parametrize("dims,k,dt", [((1500, 30), 0, torch.float64), ((5000, 16), 0, torch.float32),
                                       ((16, 5000), 1, torch.float32)], ids=str)
def test_solve_workspace_poisoned(lib, dims, k, dt):
    n = int(np.prod(dims))
    npdt = np.float32 if dt == torch.float32 else np.float64
    a, b, c, d = (torch.from_numpy(v).cuda() for v in inputs.dominant_system((n,), seed=5, dtype=npdt))
    ref = d.clone()
    trid.solve(a, b, c, ref, dims, k)
    got = d.clone()
    dc, nd = dims_c(dims)
    code = 0 if dt == torch.float32 else 1
    nb = lib.trid_solve_workspace_bytes(dc, nd, k, code)
    assert nb > 0
    ws = nan_bytes(nb)
    assert lib.trid_solve_batch_ws(P(a), P(b), P(c), P(got), None, dc, nd, k, code, P(ws), nb,
                                   stream()) == 0
    torch.cuda.synchronize()
    assert torch.equal(got, ref)


@pytest.mark.parametrize("dims,dt", [((256, 64, 48), torch.float32), ((64, 48, 32), torch.float64),
                                     ((40, 36, 33), torch.float32), ((96, 80), torch.float32)],
                         ids=str)
def test_adi_workspace_poisoned(lib, dims, dt):
    npdt = np.float32 if dt == torch.float32 else np.float64
    u0 = torch.from_numpy(inputs.sine_field(dims, inputs.sine_modes(dims, seed=2), dtype=npdt)).cuda()
    ref = u0.clone()
    ws = torch.zeros(trid.adi_workspace_bytes(dims, dt), dtype=torch.uint8, device="cuda")
    trid.adi_step(ref, dims, 0.1, 3, ws)
    got = u0.clone()
    trid.adi_step(got, dims, 0.1, 3, nan_bytes(ws.numel()))
    torch.cuda.synchronize()
    assert torch.equal(got, ref)


def test_varlen_workspace_poisoned(lib):
    lengths = inputs.loguniform_lengths(300, 16, 6000, seed=4)
    off = np.concatenate([[0], np.cumsum(lengths)]).astype(np.int64)
    tot = int(off[-1])
    a, b, c, d = (torch.from_numpy(v).cuda() for v in inputs.dominant_system((tot,), seed=6, dtype=np.float32))
    toff = torch.from_numpy(off).cuda()
    ref = d.clone()
    trid.solve_varlen(a, b, c, ref, toff, 6000)
    got = d.clone()
    trid.solve_varlen(a, b, c, got, toff, 6000,
                      workspace=nan_bytes(trid.varlen_workspace_bytes(len(lengths))))
    torch.cuda.synchronize()
    assert torch.equal(got, ref)


@pytest.mark.parametrize("dt", [torch.float32, torch.float64], ids=["f32", "f64"])
def test_adi2v_outputs_workspace_and_checkpoints_poisoned(lib, dt):
    dims, lam, steps, every = (48, 40), 0.2, 7, 3
    n = dims[0] * dims[1]
    npdt = np.float32 if dt == torch.float32 else np.float64
    u0 = torch.from_numpy(inputs.target_field(dims, seed=1).astype(npdt)).cuda()
    kap = torch.from_numpy(inputs.diffusivity_field(dims, seed=2).astype(npdt)).cuda()
    uT, ck = trid.adi2v_forward(u0, kap, dims, lam, steps, every)
    g = torch.from_numpy(inputs.random_rhs((n,), seed=3, dtype=npdt)).cuda()
    gu, gk, gc = trid.adi2v_backward(g, kap, dims, lam, steps, every, ck, want_coef=True)

    wsb = trid.adi2v_workspace_bytes(dims, steps, every, dt)
    ckb = trid.adi2v_checkpoint_bytes(dims, steps, every, dt)
    uT2 = torch.full_like(u0, float("nan"))
    ck2 = nan_bytes(ckb)
    trid.adi2v_forward(u0, kap, dims, lam, steps, every, uT=uT2, ckpt=ck2, workspace=nan_bytes(wsb))
    gu2, gk2, gc2 = trid.adi2v_backward(g, kap, dims, lam, steps, every, ck2, want_coef=True,
                                        workspace=nan_bytes(wsb))
    # and the form that keeps only the face sums of the coefficient gradients
    gu3, gk3, _ = trid.adi2v_backward(g, kap, dims, lam, steps, every, ck)
    gu4, gk4, _ = trid.adi2v_backward(g, kap, dims, lam, steps, every, ck2,
                                      workspace=nan_bytes(wsb))
    torch.cuda.synchronize()
    assert torch.equal(uT2, uT)
    for got, want in ((gu2, gu), (gk2, gk), (gc2, gc), (gu4, gu3), (gk4, gk3)):
        assert torch.equal(got, want)
