"""The debug build (device-side index checks, TRID_DEBUG_BOUNDS=1): on valid
inputs of every path no check may fail, and the results must be those of the
release build.  The debug library runs in a child process (the variable is
read when the library is first loaded); the parent computes the same calls
with the release library.  GPU only."""
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_2201_03950_gb300 import build

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# the calls, run identically in both processes; `out` collects the results
CALLS = r'''
import numpy as np, torch
from paper_2201_03950_gb300 import inputs, trid
out = {}
def sys_(n, seed, dt):
    return [torch.from_numpy(v).cuda() for v in inputs.dominant_system((n,), seed=seed, dtype=dt)]
for dims, dt in (((256, 128, 64), np.float32), ((300, 37, 19), np.float32),
                 ((64, 48, 40), np.float64), ((5000, 16), np.float32), ((16, 5000), np.float32)):
    n = int(np.prod(dims))
    a, b, c, d = sys_(n, 7, dt)
    for k in range(len(dims)):
        x = d.clone()
        trid.solve(a, b, c, x, dims, k)
        out[f"solve_{dims}_{k}"] = x.cpu().numpy()
for dims, dt in (((256, 256, 256), np.float32), ((96, 80, 40), np.float32),
                 ((64, 48, 32), np.float64), ((96, 80), np.float32)):
    u = torch.from_numpy(inputs.sine_field(dims, inputs.sine_modes(dims, seed=2), dtype=dt)).cuda()
    ws = torch.empty(trid.adi_workspace_bytes(dims, u.dtype), dtype=torch.uint8, device="cuda")
    trid.adi_step(u, dims, 0.1, 2, ws)
    out[f"adi_{dims}"] = u.cpu().numpy()
dims = (64, 64, 64)
u = torch.from_numpy(np.concatenate([inputs.sine_field(dims, inputs.sine_modes(dims, seed=s))
                                     for s in range(3)]).astype(np.float32)).cuda()
trid.adi_step_batched(u, 3, dims, 0.1, 2)
out["adi_batched"] = u.cpu().numpy()
lengths = inputs.loguniform_lengths(300, 16, 6000, seed=4)
off = np.concatenate([[0], np.cumsum(lengths)]).astype(np.int64)
a, b, c, d = sys_(int(off[-1]), 6, np.float32)
trid.solve_varlen(a, b, c, d, torch.from_numpy(off).cuda(), 6000)
out["varlen"] = d.cpu().numpy()
dims = (48, 40)
u0 = torch.from_numpy(inputs.target_field(dims, seed=1).astype(np.float32)).cuda()
kap = torch.from_numpy(inputs.diffusivity_field(dims, seed=2).astype(np.float32)).cuda()
uT, ck = trid.adi2v_forward(u0, kap, dims, 0.2, 7, 3)
out["adi2v"] = uT.cpu().numpy()
torch.cuda.synchronize()
out["status"] = np.array(trid.device_status())
out["lib"] = np.array(trid.lib_path())
'''


def run_calls():
    scope = {}
    exec(CALLS, scope)
    return scope["out"]


def test_debug_build_clean_and_equal(tmp_path):
    dbg = build.build(debug_bounds=True)
    build.build()
    assert torch.cuda.is_available()
    path = tmp_path / "dbg.npz"
    script = CALLS + f"\nnp.savez({str(path)!r}, **{{k: v for k, v in out.items()}})\n"
    env = dict(os.environ, TRID_DEBUG_BOUNDS="1")
    r = subprocess.run([sys.executable, "-c", script], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    got = np.load(path)
    assert str(got["lib"]) == dbg  # the child ran the debug library
    assert int(got["status"]) == 0  # no index check failed
    want = run_calls()
    assert int(want["status"]) == 0
    for key, w in want.items():
        if key in ("status", "lib"):
            continue
        g = got[key]
        assert np.all(np.isfinite(g)), key
        tol = 1e-6 if w.dtype == np.float32 else 1e-14
        scale = max(float(np.max(np.abs(w))), 1e-30)
        assert float(np.max(np.abs(g - w))) <= tol * scale, key
