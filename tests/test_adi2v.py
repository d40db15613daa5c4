"""Differentiable 2D ADI with a diffusivity field (adi2v_forward / adi2v_backward
and the autograd wrapper) against the FP64 oracle, checkpoint invariance and
central finite differences.  GPU only."""
import numpy as np
import pytest

import oracle
from paper_2201_03950_gb300 import inputs, trid

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DT = {np.float32: torch.float32, np.float64: torch.float64}
# the solve tolerances hold for the forward and for both gradients (measured
# at 1024^2 FP32, 50 steps: 2e-7 forward, 3e-6 worst gradient; FP64 < 2e-15)
TOL_FWD = {np.float32: 1e-5, np.float64: 1e-12}
TOL_GRAD = {np.float32: 1e-5, np.float64: 1e-12}


def normwise(x, ref):
    x = np.asarray(x, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    return float(np.max(np.abs(x - ref)) / max(np.max(np.abs(ref)), 1e-300))


def problem(dims, seed, dtype):
    rng = np.random.default_rng(seed)
    u0 = inputs.target_field(dims, seed=seed + 3) + rng.uniform(-0.3, 0.3, dims[0] * dims[1])
    kap = inputs.diffusivity_field(dims, seed=seed)
    tg = inputs.target_field(dims, seed=seed + 5)
    return [v.astype(dtype) for v in (u0, kap, tg)]


def dev(x, dtype):
    return torch.from_numpy(np.ascontiguousarray(x.astype(dtype))).cuda()


def gpu_run(u0, kap, tg, dims, lam, steps, every, dtype, want_coef=False):
    """Forward and backward on the GPU.  Without want_coef the backward keeps
    only the face sums that the kappa gradient needs; with it, the six summed
    coefficient gradients too (returned last, else None)."""
    tu, tk, tt = (dev(v, dtype) for v in (u0, kap, tg))
    uT, ck = trid.adi2v_forward(tu, tk, dims, lam, steps, every)
    g = 2.0 * (uT - tt) / tu.numel()
    gu, gk, gc = trid.adi2v_backward(g, tk, dims, lam, steps, every, ck, want_coef=want_coef)
    torch.cuda.synchronize()
    return (uT.cpu().numpy(), gu.cpu().numpy(), gk.cpu().numpy(),
            gc.cpu().numpy() if gc is not None else None)


# Lines of nx a multiple of 8 up to 1024 take the fused explicit-part + x-solve
# kernel (64, 128, 16 and the 1024^2 case below), the others the separate
# kernels (33, 300, 17, 3 and 1032, just past the fused kernel's limit).
CASES = [((33, 20), 0.3, 5, 2), ((64, 48), 0.2, 12, 5), ((300, 40), 0.25, 4, 3),
         ((17, 260), 0.2, 3, 10), ((3, 3), 0.2, 2, 1), ((128, 128), 0.2, 50, 10),
         ((16, 24), 0.2, 6, 4), ((1032, 12), 0.2, 3, 2)]


@pytest.mark.parametrize("dtype", [np.float32, np.float64], ids=["f32", "f64"])
@pytest.mark.parametrize("dims,lam,steps,every", CASES,
                         ids=[f"{d[0]}x{d[1]}-{s}steps-every{e}" for d, _, s, e in CASES])
def test_forward_and_gradient_vs_oracle(dims, lam, steps, every, dtype):
    u0, kap, tg = problem(dims, sum(dims), dtype)
    ref_uT = oracle.adi2v(u0, kap, dims, lam, steps)
    loss, rgu, rgk, rgc = oracle.adi2v_grad(u0, kap, tg, dims, lam, steps)
    # both forms of the backward: face sums only, and all six coefficient gradients
    for want in (False, True):
        uT, gu, gk, gc = gpu_run(u0, kap, tg, dims, lam, steps, every, dtype, want_coef=want)
        assert normwise(uT, ref_uT) <= TOL_FWD[dtype]
        assert normwise(gu, rgu) <= TOL_GRAD[dtype]
        assert normwise(gk, rgk) <= TOL_GRAD[dtype]
        if want:
            assert normwise(gc, rgc) <= TOL_GRAD[dtype]


@pytest.mark.parametrize("dtype", [np.float32, np.float64], ids=["f32", "f64"])
def test_checkpoint_spacing_does_not_change_the_gradient(dtype):
    """Recomputing a segment from its checkpoint reproduces the forward
    states exactly, so every spacing gives the same bits."""
    dims, lam, steps = (96, 40), 0.2, 12
    u0, kap, tg = problem(dims, 5, dtype)
    for want in (False, True):
        ref = None
        for every in (1, 5, 12, 40):
            _, gu, gk, gc = gpu_run(u0, kap, tg, dims, lam, steps, every, dtype, want_coef=want)
            got = (gu, gk, gc) if want else (gu, gk)
            if ref is None:
                ref = got
            else:
                for a, b in zip(got, ref):
                    assert np.array_equal(a, b)


@pytest.mark.parametrize("dtype", [np.float32, np.float64], ids=["f32", "f64"])
def test_unaligned_state_gives_the_same_bits(dtype):
    """The fused line kernel reads the caller's u with scalar loads when it is
    not on a 16-byte boundary: the same arithmetic, so the same bits as an
    aligned buffer, forward and gradients."""
    dims, lam, steps, every = (64, 40), 0.2, 9, 4
    u0, kap, tg = problem(dims, 31, dtype)
    n = dims[0] * dims[1]
    tu, tk, tt = (dev(v, dtype) for v in (u0, kap, tg))
    outs = []
    for shift in (0, 1):
        big = torch.empty(n + 2, dtype=DT[dtype], device="cuda")
        uT_buf = big[shift:shift + n]
        assert (uT_buf.data_ptr() % 16 == 0) == (shift == 0)
        uT, ck = trid.adi2v_forward(tu, tk, dims, lam, steps, every, uT=uT_buf)
        g = 2.0 * (uT - tt) / n
        gu, gk, _ = trid.adi2v_backward(g, tk, dims, lam, steps, every, ck)
        torch.cuda.synchronize()
        outs.append([x.cpu().numpy() for x in (uT, gu, gk)])
    for a, b in zip(*outs):
        assert np.array_equal(a, b)


def test_autograd_matches_direct_calls():
    from paper_2201_03950_gb300.autograd import adi2d
    dims, lam, steps, every = (64, 48), 0.2, 10, 4
    u0, kap, tg = problem(dims, 9, np.float64)
    tu = dev(u0, np.float64).requires_grad_(True)
    tk = dev(kap, np.float64).requires_grad_(True)
    tt = dev(tg, np.float64)
    uT = adi2d(tu, tk, dims, lam, steps, every)
    loss = torch.mean((uT - tt) ** 2)
    loss.backward()
    _, gu, gk, _ = gpu_run(u0, kap, tg, dims, lam, steps, every, np.float64)
    assert np.array_equal(tu.grad.cpu().numpy(), gu)
    assert np.array_equal(tk.grad.cpu().numpy(), gk)
    rl, rgu, rgk, _ = oracle.adi2v_grad(u0, kap, tg, dims, lam, steps)
    assert abs(loss.item() - rl) <= 1e-12 * abs(rl)
    assert normwise(gu, rgu) <= TOL_GRAD[np.float64]


def test_finite_differences_fp64():
    """Directional derivatives of the GPU loss (FP64) by central differences."""
    dims, lam, steps, every = (80, 60), 0.25, 8, 3
    u0, kap, tg = problem(dims, 13, np.float64)
    tt = dev(tg, np.float64)

    def loss(u, k):
        uT, _ = trid.adi2v_forward(dev(u, np.float64), dev(k, np.float64), dims, lam, steps,
                                   every, ckpt=False)
        return float(torch.mean((uT - tt) ** 2).item())

    _, gu, gk, _ = gpu_run(u0, kap, tg, dims, lam, steps, every, np.float64)
    rng = np.random.default_rng(1)
    h = 1e-5
    for _ in range(3):
        vu = rng.normal(size=u0.size)
        vk = rng.normal(size=u0.size)
        fu = (loss(u0 + h * vu, kap) - loss(u0 - h * vu, kap)) / (2 * h)
        fk = (loss(u0, kap + h * vk) - loss(u0, kap - h * vk)) / (2 * h)
        assert abs(fu - gu @ vu) <= 1e-7 * max(abs(fu), 1e-12) + 1e-12
        assert abs(fk - gk @ vk) <= 1e-7 * max(abs(fk), 1e-12) + 1e-12


def test_full_size_1024_fp32():
    """1024 x 1024 FP32, 50 steps, checkpoints every 10, smoothed log-normal
    kappa: loss and both gradients against the FP64 oracle."""
    dims, lam, steps, every = (1024, 1024), 0.2, 50, 10
    u0, kap, tg = problem(dims, 0, np.float32)
    uT, gu, gk, _ = gpu_run(u0, kap, tg, dims, lam, steps, every, np.float32)
    rl, rgu, rgk, _ = oracle.adi2v_grad(u0, kap, tg, dims, lam, steps)
    assert normwise(uT, oracle.adi2v(u0, kap, dims, lam, steps)) <= TOL_FWD[np.float32]
    assert normwise(gu, rgu) <= TOL_GRAD[np.float32]
    assert normwise(gk, rgk) <= TOL_GRAD[np.float32]


def test_invalid_arguments():
    dims = (16, 16)
    t = torch.zeros(256, device="cuda")
    with pytest.raises(trid.TridError):
        trid.adi2v_forward(t, t, dims, -0.1, 3, 2)
    with pytest.raises(trid.TridError):
        trid.adi2v_forward(t, t, dims, 0.1, 3, 0)
    small = torch.empty(16, dtype=torch.uint8, device="cuda")
    with pytest.raises(trid.TridError):
        trid.adi2v_forward(t, t, dims, 0.1, 3, 2, workspace=small)
