"""Batched ADI (adi_step_batched): every mesh of a batch against the FP64
oracle's ADI step, for meshes resident in shared memory (all steps in one
kernel), 3D meshes stacked through the two-pass kernels, and meshes that go
through the single-mesh path.  GPU only."""
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


def batch(dims, nb, seed, dtype):
    """nb different meshes: sine-mode fields plus interior noise, and a
    random boundary on every other mesh (boundary values must stay fixed)."""
    rng = np.random.default_rng(seed)
    n = int(np.prod(dims))
    out = []
    for b in range(nb):
        u = inputs.sine_field(dims, inputs.sine_modes(dims, seed=seed + b)) \
            + rng.uniform(-0.2, 0.2, n)
        if b % 2:
            u = u + rng.uniform(-0.5, 0.5, n)
        out.append(u)
    return np.concatenate(out).astype(dtype)


CASES = [((32, 32), 6, 0.1, 40, np.float32), ((96, 96), 4, 0.1, 120, np.float32),
         ((128, 128), 3, 0.2, 30, np.float32), ((33, 17), 5, 0.3, 25, np.float32),
         ((200, 100), 2, 0.1, 5, np.float32), ((64, 64), 3, 0.1, 40, np.float64),
         ((32, 32, 32), 3, 0.1, 10, np.float32), ((24, 20, 16), 2, 0.15, 12, np.float32),
         ((16, 16, 16), 2, 0.1, 8, np.float64), ((5, 3, 7), 4, 0.2, 6, np.float64),
         # larger than one block's shared memory: 3D meshes stacked along z
         # through the two-pass kernels, or the single-mesh path
         ((64, 64, 64), 2, 0.1, 3, np.float32), ((48, 32, 64), 3, 0.2, 4, np.float64),
         ((40, 40, 40), 2, 0.1, 2, np.float32), ((256, 200), 2, 0.1, 4, np.float32),
         # one 32-row tile per plane, stacked: several planes per CTA across meshes
         ((32, 32, 32), 5, 0.1, 3, np.float32), ((64, 32, 48), 3, 0.1, 2, np.float32)]


@pytest.mark.parametrize("dims,nb,lam,steps,dtype", CASES,
                         ids=[f"{'x'.join(map(str, c[0]))}-b{c[1]}-{c[3]}steps-"
                              f"{'f32' if c[4] is np.float32 else 'f64'}" for c in CASES])
def test_batch_against_oracle(dims, nb, lam, steps, dtype):
    u0 = batch(dims, nb, sum(dims), dtype)
    tu = torch.from_numpy(u0.copy()).cuda()
    trid.adi_step_batched(tu, nb, dims, lam, steps)
    torch.cuda.synchronize()
    got = tu.cpu().numpy()
    n = int(np.prod(dims))
    for b in range(nb):
        ref = oracle.adi(u0[b * n:(b + 1) * n], dims, lam, steps)
        assert normwise(got[b * n:(b + 1) * n], ref) <= TOL[dtype], f"mesh {b}"


def test_matches_single_mesh_steps():
    """The resident path and adi_step agree on the same meshes."""
    dims, nb, lam, steps = (48, 40), 3, 0.1, 10
    u0 = batch(dims, nb, 3, np.float64)
    tb = torch.from_numpy(u0.copy()).cuda()
    trid.adi_step_batched(tb, nb, dims, lam, steps)
    n = int(np.prod(dims))
    ws = torch.empty(trid.adi_workspace_bytes(dims, torch.float64), dtype=torch.uint8,
                     device="cuda")
    for b in range(nb):
        ts = torch.from_numpy(u0[b * n:(b + 1) * n].copy()).cuda()
        trid.adi_step(ts, dims, lam, steps, ws)
        assert normwise(tb[b * n:(b + 1) * n].cpu().numpy(), ts.cpu().numpy()) <= 1e-13


def test_empty_and_invalid():
    t = torch.zeros(64, device="cuda")
    trid.adi_step_batched(torch.zeros(0, device="cuda"), 0, (8, 8), 0.1, 3)  # nothing to do
    trid.adi_step_batched(t, 1, (8, 8), 0.1, 0)
    with pytest.raises(trid.TridError):
        trid.adi_step_batched(t, 1, (8, 8), -0.1, 3)
    with pytest.raises(trid.TridError):
        trid.adi_step_batched(torch.zeros(16, device="cuda"), 1, (8, 2), 0.1, 3)
