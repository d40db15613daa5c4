"""Uneven batches (trid_solve_batch_varlen) against the FP64 oracle."""
import numpy as np
import pytest

import oracle
from paper_2201_03950_gb300 import inputs, trid

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {np.float32: 1e-5, np.float64: 1e-12}


def per_system_err(x, ref, off):
    worst = 0.0
    for k in range(len(off) - 1):
        s, e = off[k], off[k + 1]
        if e <= s:
            continue
        r = np.asarray(ref[s:e], dtype=np.float64)
        g = np.asarray(x[s:e], dtype=np.float64)
        worst = max(worst, float(np.max(np.abs(g - r)) / max(np.max(np.abs(r)), 1e-300)))
    return worst


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2201_03950_gb300 import build
    build.build()
    trid.load()


def run(lengths, dtype, seed=0, accumulate=False, max_len=None):
    lengths = np.asarray(lengths, dtype=np.int64)
    off = np.concatenate([[0], np.cumsum(lengths)]).astype(np.int64)
    total = int(off[-1])
    a, b, c, d = inputs.dominant_system((max(total, 1),), seed=seed, dtype=dtype)
    a, b, c, d = a[:total], b[:total], c[:total], d[:total]
    ref = oracle.solve_varlen(a, b, c, d, off)
    ta, tb, tc, td = (torch.from_numpy(np.ascontiguousarray(v)).cuda() for v in (a, b, c, d))
    toff = torch.from_numpy(off).cuda()
    ml = int(lengths.max()) if max_len is None else max_len
    if accumulate:
        u0 = inputs.random_rhs((total,), seed=seed + 5, dtype=dtype)
        tu = torch.from_numpy(u0).cuda()
        trid.solve_varlen(ta, tb, tc, td, toff, ml, u=tu)
        torch.cuda.synchronize()
        got = tu.cpu().numpy().astype(np.float64) - u0.astype(np.float64)
    else:
        trid.solve_varlen(ta, tb, tc, td, toff, ml)
        torch.cuda.synchronize()
        got = td.cpu().numpy()
    return got, ref, off


EDGE = [1, 2, 3, 0, 5, 8, 9, 16, 31, 255, 256, 257, 300, 511, 512, 513, 1000, 2047, 2048, 2049,
        4100, 16384, 20000, 0, 7]


@pytest.mark.parametrize("dtype", [np.float32, np.float64], ids=["f32", "f64"])
def test_varlen_edge_lengths(dtype):
    got, ref, off = run(EDGE, dtype, seed=1)
    assert np.all(np.isfinite(got))
    assert per_system_err(got, ref, off) <= TOL[dtype]


@pytest.mark.parametrize("dtype", [np.float32, np.float64], ids=["f32", "f64"])
def test_varlen_loguniform(dtype):
    lengths = inputs.loguniform_lengths(300, 16, 16384, seed=4)
    got, ref, off = run(lengths, dtype, seed=2)
    assert per_system_err(got, ref, off) <= TOL[dtype]


def test_varlen_long_class_alignments_and_ragged_end():
    """FP32 systems longer than 4088 rows (the two-pass class) at every start
    alignment (1-3 rows of tile padding), the last system ending in the
    arrays' ragged last 16 bytes (total % 4 == 1), accumulate mode; against
    the oracle, and with a larger max_len (deeper shared-memory levels)."""
    lengths = [3, 17404, 4089, 5000, 1, 8191, 2, 12345, 16384, 7, 4090, 17401]
    assert sum(lengths) % 4 == 1
    got, ref, off = run(lengths, np.float32, seed=21)
    assert per_system_err(got, ref, off) <= TOL[np.float32]
    got2, _, _ = run(lengths, np.float32, seed=21, max_len=30000)
    assert per_system_err(got2, ref, off) <= TOL[np.float32]
    gacc, racc, _ = run(lengths, np.float32, seed=22, accumulate=True)
    assert per_system_err(gacc, racc, off) <= TOL[np.float32]


def test_varlen_accumulate_and_many_short():
    lengths = np.concatenate([np.full(3000, 17), [4096, 300], np.arange(1, 60)])
    got, ref, off = run(lengths, np.float32, seed=3, accumulate=True)
    assert per_system_err(got, ref, off) <= 2e-5


def test_varlen_invalid_system_is_flagged_and_skipped():
    # system 1 points past the arrays; its neighbours are still solved
    lengths = np.array([40, 50, 60], dtype=np.int64)
    off = np.array([0, 40, 1_000_000, 150], dtype=np.int64)  # offsets not monotone for system 1/2
    total = 150
    a, b, c, d = inputs.dominant_system((total,), seed=9, dtype=np.float32)
    ta, tb, tc, td = (torch.from_numpy(v).cuda() for v in (a, b, c, d))
    toff = torch.from_numpy(off).cuda()
    assert trid.device_status() == 0
    trid.solve_varlen(ta, tb, tc, td, toff, 64)
    torch.cuda.synchronize()
    assert trid.device_status() == 1  # TRID_ERR_INVALID_ARG recorded, then cleared
    x = td.cpu().numpy()
    ref0 = oracle.thomas(a[:40], b[:40], c[:40], d[:40])
    assert per_system_err(x[:40], ref0, [0, 40]) <= 1e-5
    assert trid.device_status() == 0


def test_varlen_empty_and_too_long_rejected_on_host():
    t = torch.zeros(8, device="cuda")
    off = torch.zeros(1, dtype=torch.int64, device="cuda")
    trid.solve_varlen(t, t, t, t, off, 8)  # nsys = 0: nothing to do
    with pytest.raises(trid.TridError):
        off2 = torch.tensor([0, 8], dtype=torch.int64, device="cuda")
        trid.solve_varlen(t, t, t, t, off2, 10_000_000)  # reduced systems do not fit


@pytest.mark.parametrize("dtype", [np.float32, np.float64], ids=["f32", "f64"])
def test_varlen_full_size_config_sampled(dtype):
    """8192 systems, lengths log-uniform in [16, 16384], FP32 and FP64:
    sampled systems against the oracle and the residual over every row."""
    lengths = inputs.loguniform_lengths(8192, 16, 16384, seed=0)
    off = np.concatenate([[0], np.cumsum(lengths)]).astype(np.int64)
    total = int(off[-1])
    a, b, c, d = inputs.dominant_system((total,), seed=0, dtype=dtype)
    ta, tb, tc, td = (torch.from_numpy(v).cuda() for v in (a, b, c, d))
    td0 = td.clone()
    trid.solve_varlen(ta, tb, tc, td, torch.from_numpy(off).cuda(), 16384)
    torch.cuda.synchronize()
    x = td.cpu().numpy()
    rng = np.random.default_rng(1)
    pick = np.unique(np.concatenate([rng.choice(8192, 150, replace=False),
                                     [int(np.argmax(lengths)), int(np.argmin(lengths))]]))
    worst = 0.0
    for k in pick:
        s, e = off[k], off[k + 1]
        ref = oracle.thomas(a[s:e], b[s:e], c[s:e], d[s:e])
        worst = max(worst, per_system_err(x[s:e], ref, [0, e - s]))
    assert worst <= TOL[dtype]
    # residual |A x - d| over all systems, in FP64 with plain torch ops
    A, B, C, D, X = (t.double() for t in (ta, tb, tc, td0, td))
    r = B * X
    first = torch.zeros(total, dtype=torch.bool, device="cuda")
    first[torch.from_numpy(off[:-1]).cuda()] = True
    last = torch.zeros(total, dtype=torch.bool, device="cuda")
    last[torch.from_numpy(off[1:] - 1).cuda()] = True
    r[1:] += torch.where(first[1:], 0.0, A[1:] * X[:-1])
    r[:-1] += torch.where(last[:-1], 0.0, C[:-1] * X[1:])
    res = ((r - D).abs().max() / ((A.abs() + B.abs() + C.abs()).max() * X.abs().max() + D.abs().max())).item()
    assert res <= (1e-5 if dtype == np.float32 else 1e-13)


CLASS_EDGES = [248, 249, 503, 504, 505, 1015, 1016, 1017, 2039, 2040, 2041, 4087, 4088, 4089,
               5000, 1, 2, 200]
CONFIGS = [(248, 248), (248, 1016), (248, 2040), (248, 4088), (504, 504), (504, 1016),
           (504, 2040), (504, 4088), (1016, 1016), (1016, 2040), (1016, 4088)]
# tiles of 16 rows (FP32): every limit doubles plus 8
CLASS_EDGES16 = [496, 497, 1007, 1008, 1009, 2031, 2032, 2033, 4079, 4080, 4081, 8175, 8176, 8177,
                 9000, 1, 2, 300]
CONFIGS16 = [(496, 496), (496, 2032), (496, 4080), (496, 8176), (1008, 1008), (1008, 2032),
             (1008, 4080), (1008, 8176), (2032, 2032), (2032, 4080), (2032, 8176)]


def run_cfg(lengths, dtype, cfg, seed=3, tile_rows=0):
    lengths = np.asarray(lengths, dtype=np.int64)
    off = np.concatenate([[0], np.cumsum(lengths)]).astype(np.int64)
    total = int(off[-1])
    a, b, c, d = inputs.dominant_system((total,), seed=seed, dtype=dtype)
    ref = oracle.solve_varlen(a, b, c, d, off)
    ta, tb, tc, td = (torch.from_numpy(np.ascontiguousarray(v)).cuda() for v in (a, b, c, d))
    toff = torch.from_numpy(off).cuda()
    trid.solve_varlen(ta, tb, tc, td, toff, int(lengths.max()),
                      config=trid.VarlenConfig(*cfg, tile_rows))
    torch.cuda.synchronize()
    return td.cpu().numpy(), ref, off


@pytest.mark.parametrize("cfg", CONFIGS, ids=[f"team{a}-block{b}" for a, b in CONFIGS])
def test_varlen_every_class_configuration(cfg):
    """Every admissible class split routes each length (incl. the class
    boundaries, each side) to a path that solves it exactly."""
    got, ref, off = run_cfg(CLASS_EDGES, np.float32, cfg)
    assert per_system_err(got, ref, off) <= TOL[np.float32]


@pytest.mark.parametrize("cfg", CONFIGS16, ids=[f"m16-team{a}-block{b}" for a, b in CONFIGS16])
def test_varlen_every_class_configuration_tile16(cfg):
    """The same with tiles of 16 rows per thread (FP32)."""
    got, ref, off = run_cfg(CLASS_EDGES16, np.float32, cfg, tile_rows=16)
    assert per_system_err(got, ref, off) <= TOL[np.float32]


TEAM2 = [((504, 504), 8), ((504, 4088), 8), ((1008, 8176), 16), ((1008, 1008), 16)]


@pytest.mark.parametrize("cfg,m", TEAM2, ids=[f"m{m}-team{a}-block{b}-2warps" for (a, b), m in TEAM2])
def test_varlen_two_warp_teams(cfg, m):
    """Teams of 2 warps (8 systems in flight per block) for the smaller team
    class, with either tile height."""
    lengths = (CLASS_EDGES if m == 8 else CLASS_EDGES16) + [100, 400, 503, 504, 1000]
    lengths = np.asarray(lengths, dtype=np.int64)
    off = np.concatenate([[0], np.cumsum(lengths)]).astype(np.int64)
    total = int(off[-1])
    a, b, c, d = inputs.dominant_system((total,), seed=4, dtype=np.float32)
    ref = oracle.solve_varlen(a, b, c, d, off)
    ta, tb, tc, td = (torch.from_numpy(np.ascontiguousarray(v)).cuda() for v in (a, b, c, d))
    trid.solve_varlen(ta, tb, tc, td, torch.from_numpy(off).cuda(), int(lengths.max()),
                      config=trid.VarlenConfig(*cfg, m, 2))
    torch.cuda.synchronize()
    assert per_system_err(td.cpu().numpy(), ref, off) <= TOL[np.float32]


def test_varlen_tile16_full_batch_residual():
    """Tiles of 16 rows on a log-uniform batch up to 16384 rows: oracle on
    every system."""
    lengths = inputs.loguniform_lengths(400, 16, 16384, seed=21)
    got, ref, off = run_cfg(lengths, np.float32, (1008, 8176), seed=8, tile_rows=16)
    assert per_system_err(got, ref, off) <= TOL[np.float32]


def test_varlen_autotune_picks_a_valid_config_and_keeps_d():
    lengths = inputs.loguniform_lengths(600, 16, 16384, seed=9)
    off = np.concatenate([[0], np.cumsum(lengths)]).astype(np.int64)
    total = int(off[-1])
    a, b, c, d = inputs.dominant_system((total,), seed=5, dtype=np.float32)
    ta, tb, tc, td = (torch.from_numpy(np.ascontiguousarray(v)).cuda() for v in (a, b, c, d))
    toff = torch.from_numpy(off).cuda()
    cfg, ms = trid.varlen_autotune(ta, tb, tc, td, toff, int(lengths.max()), cache=False)
    assert ((cfg.team_max, cfg.block_max) in CONFIGS and cfg.tile_rows in (0, 8)) or (
        (cfg.team_max, cfg.block_max) in CONFIGS16 and cfg.tile_rows == 16)
    assert cfg.team_warps in (0, 4) or (cfg.team_warps == 2 and cfg.team_max in (504, 1008))
    assert ms > 0.0
    assert np.array_equal(td.cpu().numpy(), d)  # the autotuner works on a copy
    trid.solve_varlen(ta, tb, tc, td, toff, int(lengths.max()), config=cfg)
    torch.cuda.synchronize()
    ref = oracle.solve_varlen(a, b, c, d, off)
    assert per_system_err(td.cpu().numpy(), ref, off) <= TOL[np.float32]


def test_varlen_autotune_cache_round_trip(tmp_path, monkeypatch):
    """The tuned choice is stored per (dtype, length histogram) and returned
    for a batch with the same histogram without timing (time -1)."""
    monkeypatch.setenv("TRID_TUNE_CACHE", str(tmp_path / "tune.json"))
    lengths = inputs.loguniform_lengths(200, 16, 9000, seed=12)
    off = np.concatenate([[0], np.cumsum(lengths)]).astype(np.int64)
    total = int(off[-1])
    a, b, c, d = inputs.dominant_system((total,), seed=2, dtype=np.float32)
    ta, tb, tc, td = (torch.from_numpy(np.ascontiguousarray(v)).cuda() for v in (a, b, c, d))
    toff = torch.from_numpy(off).cuda()
    cfg1, ms1 = trid.varlen_autotune(ta, tb, tc, td, toff, int(lengths.max()))
    assert ms1 > 0.0 and (tmp_path / "tune.json").exists()
    cfg2, ms2 = trid.varlen_autotune(ta, tb, tc, td, toff, int(lengths.max()))
    assert ms2 == -1.0 and (cfg2.team_max, cfg2.block_max, cfg2.tile_rows or 8,
                            cfg2.team_warps or 4) == (cfg1.team_max, cfg1.block_max,
                                                      cfg1.tile_rows or 8, cfg1.team_warps or 4)


def test_varlen_invalid_config_rejected():
    t = torch.zeros(8, device="cuda")
    toff = torch.tensor([0, 8], dtype=torch.int64, device="cuda")
    for bad in ((300, 4088, 8), (1016, 504, 8), (2040, 4088, 8), (504, 9000, 8), (1016, 4088, 16),
                (1008, 8176, 8), (1008, 8176, 12), (1016, 4088, 8, 2), (248, 4088, 8, 2),
                (504, 4088, 8, 3)):
        with pytest.raises(trid.TridError):
            trid.solve_varlen(t, t + 2, t, t, toff, 8, config=trid.VarlenConfig(*bad))
    # tiles of 16 rows are FP32 only
    t64 = torch.zeros(8, dtype=torch.float64, device="cuda")
    with pytest.raises(trid.TridError):
        trid.solve_varlen(t64, t64 + 2, t64, t64, toff, 8,
                          config=trid.VarlenConfig(1008, 8176, 16))
