#!/usr/bin/env python3
"""Benchmark of the hot path: batched tridiagonal solves along x, y and z of a
256^3 FP32 mesh plus one 3D ADI heat-diffusion step (lambda = 0.1).

One step = solve(x) + solve(y) + solve(z) + adi_step(1 step), each call timed
with CUDA events on the launching stream, with d restored from a pristine copy
and L2 flushed (a 256 MiB write, then a 256 MiB read, so no dirty line is left
for the timed call to write back) before every call, outside the events.

Metric: algorithmic bandwidth of the step in GB/s, counting 5 words per
unknown for a solve (a, b, c, d read; x written -- the paper's convention,
Table 1) and 4 words per mesh point for the 3D ADI step (the two-pass schedule
that runs: u read, e = Z u + Y^{-1} X^{-1} d written; e read, u = Z^{-1} e
written).  Before each timed call a GPU-side wait (torch.cuda._sleep) follows
the L2 flush, so that the host has enqueued the call before its start event
is reached: the events then time the call's kernels, not the host's launch.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the FP64 CPU oracle (the only reference this method
has) on the host cores on a bounded sample of the same workload.
Under torchrun (N > 1) every rank runs an independent replica (the solves
shard with no exchange); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

DIMS = (256, 256, 256)
LAM = 0.1
METRIC = "Batched tridiag solve GB/s (% HBM roofline), 256³ FP32 x/y/z; ADI step ms"
WORKLOAD = "256^3 FP32: batched solves along x, y, z (65536 systems of 256 each) + one 3D ADI step"
FALLBACK_HBM_GBS = 6800.0


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=100)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--e2e-steps", type=int, default=10)
    p.add_argument("--no-secondary", action="store_true",
                   help="skip the 4096^2 long-system measurement")
    p.add_argument("--dtype", choices=["f32", "f64"], default="f32",
                   help="f64 runs the same step in FP64 (reported separately; the headline is f32)")
    return p.parse_args()


def aggregate_ranks(ms_step, step_bytes, world, dist=None, device="cpu"):
    """Whole-job figure of `world` independent replicas (weak scaling): the
    slowest rank's time per step (max over ranks) and every rank's bytes.
    Returns (ms per step, GB/s)."""
    if world > 1:
        import torch
        t = torch.tensor([float(ms_step)], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_step = float(t.item())
    return ms_step, world * step_bytes / (ms_step * 1e-3) / 1e9


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# FP64 on GB300: the FP64 pipe, not HBM, bounds the solve.  Peak: the
# nominal FP64 rate of the part (1.25 TFLOP/s); algorithmic work: the Thomas
# recurrence's 9 operations per unknown (forward: a c*, b - ., 1/m, c r,
# a d*, d - ., . r; backward: d* - c* x, as a multiply and a subtract).
# Thomas (Algorithm "thomas") per unknown: one division (1 / (b - a c*)) and
# five multiply-type operations (the pivot, c*, two for d*, one in the back
# substitution).  With FP64 on GB300 far below FP32, the FP64 solves are
# bound by these operations; the peak is taken from the device's own rates,
# measured live (trid_fp64_rates): 6 / (5 / fma_rate + 1 / div_rate).
THOMAS_MUL_OPS = 5
THOMAS_DIV_OPS = 1


def roofline_obj(dtype, kernel, achieved_gbs, peak, peak_kind, traffic, nbytes, mean_ms,
                 fp64_rates=None):
    if dtype == "f64":
        unknowns = nbytes // (5 * 8)
        fma_g, div_g = fp64_rates
        ops = THOMAS_MUL_OPS + THOMAS_DIV_OPS
        peak_gops = ops / (THOMAS_MUL_OPS / fma_g + THOMAS_DIV_OPS / div_g)
        gops = ops * unknowns / (mean_ms * 1e-3) / 1e9
        return {"bound": "alu", "kernel": kernel, "achieved": round(gops, 2),
                "peak": round(peak_gops, 2),
                "peak_kind": (f"measured FP64 rates of this device (FMA {fma_g:.1f} G/s, "
                              f"IEEE division {div_g:.1f} G/s; Thomas mix of 5 FMA-type + 1 "
                              f"division per unknown)"),
                "unit": "Gop/s", "frac": round(gops / peak_gops, 4), "traffic": traffic,
                "algorithmic_ops_per_launch": ops * unknowns,
                "hbm_frac": round(achieved_gbs / peak, 4)}
    return {"bound": "hbm", "kernel": kernel, "achieved": round(achieved_gbs, 1),
            "peak": peak, "peak_kind": f"{peak_kind} (copy, burst)", "unit": "GB/s",
            "frac": round(achieved_gbs / peak, 4), "traffic": traffic,
            "algorithmic_bytes_per_launch": nbytes}


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            pk = json.load(f)
        return float(pk["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return FALLBACK_HBM_GBS, "fallback"


def profiled_traffic(kernel_key: str):
    """DRAM bytes per launch from the committed ncu summary, or None when the
    kernel sources changed since the counters were taken."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "traffic.md")
    if not os.path.exists(path):
        return None
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2201_03950_gb300", "csrc")
    for f in sorted(os.listdir(csrc)):
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(f.encode() + fh.read())
    digest = h.hexdigest()[:16]
    for line in open(path):
        m = re.match(r"\|\s*(\S+)\s*\|\s*([0-9.]+)\s*\|\s*([0-9a-f]{16})\s*\|", line)
        if m and m.group(1) == kernel_key:
            return float(m.group(2)) if m.group(3) == digest else None
    return None


class Clocks:
    """Samples nvidia-smi every 50 ms from the warm-up through the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.tmp = None

    def start(self):
        try:
            self.tmp = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=self.tmp, stderr=subprocess.DEVNULL)
        except (OSError, ValueError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.tmp.flush()
        rows = [r.split(",") for r in open(self.tmp.name).read().strip().splitlines()]
        os.unlink(self.tmp.name)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except ValueError:
                continue
            for name, v in zip(names, r[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


# ----------------------------------------------------------------- our arm
def run_ours(args):
    import torch
    from paper_2201_03950_gb300 import build, inputs, metrics, trid

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    build.build()
    trid.load()

    total = int(np.prod(DIMS))
    npdt = np.float32 if args.dtype == "f32" else np.float64
    tdt = torch.float32 if args.dtype == "f32" else torch.float64
    esz = np.dtype(npdt).itemsize
    a, b, c, d = inputs.dominant_system((total,), seed=rank, dtype=npdt)
    modes = inputs.sine_modes(DIMS, seed=rank)
    u0 = inputs.sine_field(DIMS, modes, dtype=npdt)
    ta, tb, tc, td0 = (torch.from_numpy(v).to(dev) for v in (a, b, c, d))
    td = torch.empty_like(td0)
    tu = torch.from_numpy(u0).to(dev)
    ws = torch.empty(trid.adi_workspace_bytes(DIMS, tdt), dtype=torch.uint8, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    flush_rd = torch.zeros(64 << 20, dtype=torch.float32, device=dev)

    class _Flush:
        """L2 flush between timed calls: a 256 MiB write, then a 256 MiB read,
        so that the cache holds none of the call's inputs and no dirty lines
        whose write-back the timed call would pay for."""

        def fill_(self, v):
            flush.fill_(v)
            torch.amax(flush_rd)

    flusher = _Flush()
    stream = torch.cuda.current_stream()

    names = ["solve_x", "solve_y", "solve_z", "adi_step"]
    # one kernel per solve; the FP32 step runs the windowed ADI schedule (two
    # kernels), FP64 the two-pass one (setup, RHS + x + y tile pass, y
    # substitution + z)
    launches_per_step = 3 + (2 if args.dtype == "f32" else 3)
    GAP_CYCLES = 100_000  # ~50 us of GPU-side wait while the host enqueues the call
    nbytes = {"solve_x": metrics.solve_bytes(total, esz), "solve_y": metrics.solve_bytes(total, esz),
              "solve_z": metrics.solve_bytes(total, esz),
              "adi_step": metrics.adi_step_bytes(total, esz)}

    def one_step(record):
        evs = []
        for k in range(3):
            td.copy_(td0)
            flusher.fill_(k + 1)
            torch.cuda._sleep(GAP_CYCLES)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            trid.solve(ta, tb, tc, td, DIMS, k, stream=stream)
            e1.record(stream)
            evs.append((names[k], e0, e1))
        flusher.fill_(7)
        torch.cuda._sleep(GAP_CYCLES)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        trid.adi_step(tu, DIMS, LAM, 1, ws, stream=stream)
        e1.record(stream)
        evs.append(("adi_step", e0, e1))
        if record is not None:
            record.append(evs)

    clocks = Clocks(local)
    clocks.start()
    for _ in range(args.warmup):
        one_step(None)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    recs = []
    t_wall = time.perf_counter()
    for _ in range(args.steps):
        one_step(recs)
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t_wall
    clock_info = clocks.stop()
    if world > 1:
        dist.barrier()
    per = {n: [] for n in names}
    for evs in recs:
        for n, e0, e1 in evs:
            per[n].append(e0.elapsed_time(e1))
    ms_step = sum(sum(v) for v in per.values()) / args.steps
    step_bytes = sum(nbytes.values())
    ms_step, value = aggregate_ranks(ms_step, step_bytes, world, dist if world > 1 else None, dev)

    # ---- secondary workload: 4096^2 FP32, few long systems (tiled Thomas-PCR
    #      passes), along x and y; same restore + flush protocol, mean of 5
    secondary = {}
    if args.dtype == "f32" and not args.no_secondary:
        dims2 = (4096, 4096)
        tot2 = dims2[0] * dims2[1]
        a2, b2, c2, d2 = inputs.dominant_system((tot2,), seed=11 + rank, dtype=np.float32)
        ta2, tb2, tc2, td2_0 = (torch.from_numpy(v).to(dev) for v in (a2, b2, c2, d2))
        td2 = torch.empty_like(td2_0)
        for k, name in ((0, "solve_4096sq_x"), (1, "solve_4096sq_y")):
            times = []
            for it in range(6):
                td2.copy_(td2_0)
                flusher.fill_(it + 3)
                torch.cuda._sleep(GAP_CYCLES)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                trid.solve(ta2, tb2, tc2, td2, dims2, k, stream=stream)
                e1.record(stream)
                torch.cuda.synchronize()
                if it:
                    times.append(e0.elapsed_time(e1))
            ms = statistics.mean(times)
            nb = metrics.solve_bytes(tot2, 4)
            secondary[name] = {"us": round(ms * 1e3, 2), "GBps": round(nb / (ms * 1e-3) / 1e9, 1),
                               "frac": round(nb / (ms * 1e-3) / 1e9 / peaks()[0], 4)}
        del ta2, tb2, tc2, td2_0, td2

        # adjoint of the 256^3 solves (g_d = A^-T g_x and the coefficient
        # gradients: 9 words per unknown -- a, b, c, x, g_x read; g_a, g_b,
        # g_c, g_d written), against the forward GB/s of the same axis
        tgx = torch.from_numpy(inputs.random_rhs((total,), seed=31 + rank, dtype=np.float32)).to(dev)
        tx = td0.clone()
        outs = [torch.empty_like(tx) for _ in range(4)]
        L = trid.load()
        import ctypes
        for k, name in ((0, "adjoint_x"), (2, "adjoint_z")):
            times = []
            dc = (ctypes.c_int64 * 3)(*DIMS)
            for it in range(6):
                flusher.fill_(it + 5)
                torch.cuda._sleep(GAP_CYCLES)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                st_ = L.trid_solve_batch_adjoint(*(ctypes.c_void_p(t.data_ptr()) for t in
                                                   (ta, tb, tc, tx, tgx, *outs)), dc, 3, k, 0,
                                                 None, 0, ctypes.c_void_p(stream.cuda_stream))
                e1.record(stream)
                torch.cuda.synchronize()
                assert st_ == 0
                if it:
                    times.append(e0.elapsed_time(e1))
            ms = statistics.mean(times)
            nb = 9 * total * 4
            gbs = nb / (ms * 1e-3) / 1e9
            fwd = nbytes[f"solve_{'xyz'[k]}"] / (statistics.mean(per[f"solve_{'xyz'[k]}"]) * 1e-3) / 1e9
            secondary[name] = {"us": round(ms * 1e3, 2), "GBps": round(gbs, 1),
                               "frac": round(gbs / peaks()[0], 4),
                               "ratio_to_forward_GBps": round(gbs / fwd, 3)}
        del tgx, tx, outs

        # differentiable 2D ADI with a diffusivity field: 1024^2 FP32, 50 steps,
        # checkpoints every 10; forward (17 words per point and step: stencil
        # 6, x solve 5, y solve into u 6) and backward (65 words per point and
        # step: segment recompute 21, two adjoint solves 2 x 9, stencil
        # transpose with the summed coefficient gradients 26)
        try:
            dv = (1024, 1024)
            nv = dv[0] * dv[1]
            u0v = torch.from_numpy(inputs.target_field(dv, seed=3, dtype=np.float32)).to(dev)
            kv = torch.from_numpy(inputs.diffusivity_field(dv, seed=0, dtype=np.float32)).to(dev)
            tv = torch.from_numpy(inputs.target_field(dv, seed=5, dtype=np.float32)).to(dev)
            stv, ev = 50, 10
            wsv = torch.empty(trid.adi2v_workspace_bytes(dv, stv, ev, torch.float32),
                              dtype=torch.uint8, device=dev)
            ckv = torch.empty(trid.adi2v_checkpoint_bytes(dv, stv, ev, torch.float32),
                              dtype=torch.uint8, device=dev)
            uTv = torch.empty_like(u0v)
            fwd_t, bwd_t = [], []
            for it in range(4):
                flusher.fill_(it + 9)
                torch.cuda._sleep(GAP_CYCLES)
                e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
                e0.record(stream)
                trid.adi2v_forward(u0v, kv, dv, 0.2, stv, ev, uT=uTv, ckpt=ckv, workspace=wsv,
                                   stream=stream)
                e1.record(stream)
                gv2 = 2.0 * (uTv - tv) / nv
                flusher.fill_(it + 10)
                torch.cuda._sleep(GAP_CYCLES)
                e1b = torch.cuda.Event(enable_timing=True)
                e1b.record(stream)
                trid.adi2v_backward(gv2, kv, dv, 0.2, stv, ev, ckv, workspace=wsv, stream=stream)
                e2.record(stream)
                torch.cuda.synchronize()
                if it:
                    fwd_t.append(e0.elapsed_time(e1))
                    bwd_t.append(e1b.elapsed_time(e2))
            mf, mb = statistics.mean(fwd_t), statistics.mean(bwd_t)
            bf, bb = 17 * nv * 4 * stv, 65 * nv * 4 * stv
            uni = nbytes["solve_x"] / (statistics.mean(per["solve_x"]) * 1e-3) / 1e9
            gf, gbk = bf / (mf * 1e-3) / 1e9, bb / (mb * 1e-3) / 1e9
            gtot = (bf + bb) / ((mf + mb) * 1e-3) / 1e9
            # the same forward + backward captured once in a CUDA graph and
            # replayed (about 6 launches per step and direction go to the graph)
            gv2 = 2.0 * (uTv - tv) / nv
            gvg = torch.cuda.CUDAGraph()
            with torch.cuda.graph(gvg):
                cs_ = torch.cuda.current_stream()
                trid.adi2v_forward(u0v, kv, dv, 0.2, stv, ev, uT=uTv, ckpt=ckv, workspace=wsv,
                                   stream=cs_)
                trid.adi2v_backward(gv2, kv, dv, 0.2, stv, ev, ckv, workspace=wsv, stream=cs_)
            gts = []
            for it in range(4):
                flusher.fill_(it + 11)
                torch.cuda._sleep(GAP_CYCLES)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                gvg.replay()
                e1.record(stream)
                torch.cuda.synchronize()
                if it:
                    gts.append(e0.elapsed_time(e1))
            mg = statistics.mean(gts)
            gg = (bf + bb) / (mg * 1e-3) / 1e9
            del gvg
            # through torch autograd (DiffADI2D: the library's captured
            # graphs replayed, inputs copied in and outputs copied out)
            from paper_2201_03950_gb300 import autograd as tag
            u0r = u0v.clone().requires_grad_(True)
            kr = kv.clone().requires_grad_(True)
            ats = []
            for it in range(5):
                u0r.grad = None
                kr.grad = None
                flusher.fill_(it + 12)
                torch.cuda._sleep(GAP_CYCLES)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                uTa = tag.adi2d(u0r, kr, dv, 0.2, stv, ev)
                ((uTa - tv) ** 2).mean().backward()
                e1.record(stream)
                torch.cuda.synchronize()
                if it > 1:  # the first call captures the graphs
                    ats.append(e0.elapsed_time(e1))
            ma = statistics.mean(ats)
            ga = (bf + bb) / (ma * 1e-3) / 1e9
            del u0r, kr, uTa
            secondary["adi2v_1024sq_50steps_ckpt10"] = {
                "forward_ms": round(mf, 3), "backward_ms": round(mb, 3),
                "forward_GBps": round(gf, 1), "backward_GBps": round(gbk, 1),
                "ratio_to_uniform_x_solve": round(gtot / uni, 3),
                "graph_forward_backward_ms": round(mg, 3),
                "graph_ratio_to_uniform_x_solve": round(gg / uni, 3),
                "autograd_forward_backward_ms": round(ma, 3),
                "autograd_ratio_to_uniform_x_solve": round(ga / uni, 3)}
            del u0v, kv, tv, wsv, ckv, uTv
        except Exception as exc:
            secondary["adi2v_1024sq_50steps_ckpt10"] = f"unavailable: {exc}"[:200]

        # batched small meshes with every step on chip: 3000 meshes of 96^2, 120
        # steps (2D, 5 words per point and step) and 72 meshes of 32^3, 100
        # steps (3D, 4 words), FP32 -- the batched ADI workloads of Section 4
        for key, bd, nbm, nst, words in (("adi_batched_2d_96sq_x3000_120steps", (96, 96), 3000, 120, 5),
                                         ("adi_batched_3d_32cube_x72_100steps", (32, 32, 32), 72, 100, 4)):
            try:
                per_m = int(np.prod(bd))
                ub0 = np.concatenate([inputs.sine_field(bd, inputs.sine_modes(bd, seed=m))
                                      for m in range(8)]).astype(np.float32)
                ub0 = np.tile(ub0, (nbm + 7) // 8)[: nbm * per_m]
                tub0 = torch.from_numpy(ub0).to(dev)
                tub = tub0.clone()
                ts_ = []
                for it in range(4):
                    tub.copy_(tub0)
                    flusher.fill_(it + 3)
                    torch.cuda._sleep(GAP_CYCLES)
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    trid.adi_step_batched(tub, nbm, bd, 0.1, nst, stream=stream)
                    e1.record(stream)
                    torch.cuda.synchronize()
                    if it:
                        ts_.append(e0.elapsed_time(e1))
                msb = statistics.mean(ts_)
                eff = words * 4 * per_m * nbm * nst / (msb * 1e-3) / 1e9
                secondary[key] = {"ms": round(msb, 3), "mesh_steps_per_s": round(nbm * nst / (msb * 1e-3)),
                                  "effective_GBps": round(eff, 1),
                                  "effective_frac_of_hbm": round(eff / peaks()[0], 3),
                                  "note": (f"{words} words per point and step counted; " +
                                           ("every step on chip (one kernel)" if len(bd) == 2 else
                                            "meshes stacked along z through the two-pass kernels"))}
                del tub0, tub
            except Exception as exc:
                secondary[key] = f"unavailable: {exc}"[:200]

        # uneven batch: 8192 systems, lengths log-uniform in [16, 16384], FP32
        # and FP64, planning + persistent solve captured in one CUDA graph and
        # replayed
        lengths = inputs.loguniform_lengths(8192, 16, 16384, seed=rank)
        off = np.concatenate([[0], np.cumsum(lengths)]).astype(np.int64)
        tot3 = int(off[-1])
        toff = torch.from_numpy(off).to(dev)
        wsv = torch.empty(trid.varlen_workspace_bytes(8192), dtype=torch.uint8, device=dev)
        for vdt, key in ((np.float32, "varlen_8192_loguniform_16_16384"),
                         (np.float64, "varlen_8192_loguniform_16_16384_f64")):
            esz3 = np.dtype(vdt).itemsize
            a3, b3, c3, d3 = inputs.dominant_system((tot3,), seed=21 + rank, dtype=vdt)
            ta3, tb3, tc3, td3_0 = (torch.from_numpy(v).to(dev) for v in (a3, b3, c3, d3))
            td3 = td3_0.clone()
            trid.solve_varlen(ta3, tb3, tc3, td3, toff, 16384, workspace=wsv, stream=stream)
            torch.cuda.synchronize()
            try:
                # length classes picked by the library's autotuner on this batch
                vcfg, vms = trid.varlen_autotune(ta3, tb3, tc3, td3, toff, 16384, stream=stream)
                gv = torch.cuda.CUDAGraph()
                with torch.cuda.graph(gv):
                    trid.solve_varlen(ta3, tb3, tc3, td3, toff, 16384, workspace=wsv,
                                      stream=torch.cuda.current_stream(), config=vcfg)
                times = []
                for it in range(6):
                    td3.copy_(td3_0)
                    flusher.fill_(it + 9)
                    torch.cuda._sleep(GAP_CYCLES)
                    e0, e1 = (torch.cuda.Event(enable_timing=True),
                              torch.cuda.Event(enable_timing=True))
                    e0.record(stream)
                    gv.replay()
                    e1.record(stream)
                    torch.cuda.synchronize()
                    if it:
                        times.append(e0.elapsed_time(e1))
                ms = statistics.mean(times)
                nb = metrics.solve_bytes(tot3, esz3)
                gbs = nb / (ms * 1e-3) / 1e9
                rec = {"unknowns": tot3, "us": round(ms * 1e3, 2), "GBps": round(gbs, 1),
                       "frac": round(gbs / peaks()[0], 4),
                       "autotuned": {"team_max": vcfg.team_max, "block_max": vcfg.block_max,
                                     "tile_rows": vcfg.tile_rows or 8,
                                     "team_warps": vcfg.team_warps or 4,
                                     "tuning_ms": round(vms, 4)},
                       "timing": "plan + persistent solve in one CUDA graph, L2 flushed"}
                if vdt == np.float32:
                    uni = nbytes["solve_x"] / (statistics.mean(per["solve_x"]) * 1e-3) / 1e9
                    rec["ratio_to_uniform_x_solve"] = round(gbs / uni, 3)
                else:
                    rec["note"] = "FP64: bound by FP64 arithmetic on this device, not by HBM"
                secondary[key] = rec
                del gv
            except Exception as exc:
                secondary[key] = f"unavailable: {exc}"[:200]
            del ta3, tb3, tc3, td3_0, td3

    # ---- ADI time stepping as a solver runs it: 100 steps captured in one
    #      CUDA graph and replayed (no flush between steps), per step
    adi_graph_ms = None
    try:
        nst = 100
        tu2 = tu.clone()
        trid.adi_step(tu2, DIMS, LAM, 1, ws, stream=stream)  # warm the host-side caches
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            trid.adi_step(tu2, DIMS, LAM, nst, ws, stream=torch.cuda.current_stream())
        g.replay()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        g.replay()
        e1.record()
        torch.cuda.synchronize()
        adi_graph_ms = e0.elapsed_time(e1) / nst
        del g, tu2
    except Exception as exc:  # graph capture is an extra measurement, never the headline
        adi_graph_ms = f"unavailable: {type(exc).__name__}: {exc}"[:200]

    # ---- end to end through the public API with pinned host buffers: every
    # step copies its inputs (a, b, c, d once -- the three solves share the
    # coefficients -- and the ADI field u) from the host and reads every result
    # (x of the three solves, u) back.  Steps run back to back as a pipeline
    # over two device buffer sets: copies in (one stream), solves (another)
    # and copies out (a third) are ordered by events, so step k's results
    # travel to the host while step k + 1's inputs travel to the device and
    # the solves overlap both.  Time = first copy in to last copy out, / K.
    host = {k: torch.from_numpy(v).pin_memory() for k, v in
            (("a", a), ("b", b), ("c", c), ("d", d), ("u", u0))}
    s_in, s_out = torch.cuda.Stream(device=dev), torch.cuda.Stream(device=dev)
    sets = []
    for q in range(2):
        if q == 0:
            arrs = {"a": ta, "b": tb, "c": tc, "u": tu}
            dk0 = td
        else:
            arrs = {k: torch.empty_like(td) for k in ("a", "b", "c", "u")}
            dk0 = torch.empty_like(td)
        arrs["d"] = [dk0, torch.empty_like(td), torch.empty_like(td)]
        arrs["host_x"] = [torch.empty(total, dtype=tdt).pin_memory() for _ in range(4)]
        sets.append(arrs)
    h2d = 4 * total * esz + total * esz
    d2h = 3 * total * esz + total * esz

    def e2e_run(nsteps):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        out_done = []
        e0.record(s_in)
        for k in range(nsteps):
            S = sets[k % 2]
            ev_in, ev_u = torch.cuda.Event(), torch.cuda.Event()
            done = [torch.cuda.Event() for _ in range(4)]
            if k >= 2:
                s_in.wait_event(out_done[k - 2])  # set S is free again
            with torch.cuda.stream(s_in):
                S["d"][0].copy_(host["d"], non_blocking=True)
                S["a"].copy_(host["a"], non_blocking=True)
                S["b"].copy_(host["b"], non_blocking=True)
                S["c"].copy_(host["c"], non_blocking=True)
                ev_in.record(s_in)
                S["u"].copy_(host["u"], non_blocking=True)
                ev_u.record(s_in)
            stream.wait_event(ev_in)
            with torch.cuda.stream(stream):
                S["d"][1].copy_(S["d"][0], non_blocking=True)
                S["d"][2].copy_(S["d"][0], non_blocking=True)
            for j in range(3):
                trid.solve(S["a"], S["b"], S["c"], S["d"][j], DIMS, j, stream=stream)
                done[j].record(stream)
            stream.wait_event(ev_u)
            trid.adi_step(S["u"], DIMS, LAM, 1, ws, stream=stream)
            done[3].record(stream)
            with torch.cuda.stream(s_out):
                for j, src in enumerate((S["d"][0], S["d"][1], S["d"][2], S["u"])):
                    s_out.wait_event(done[j])
                    S["host_x"][j].copy_(src, non_blocking=True)
                od = torch.cuda.Event()
                od.record(s_out)
                out_done.append(od)
        e1.record(s_out)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / nsteps

    e2e_ms = []
    if args.e2e_steps > 0:
        e2e_run(2)  # warm-up
        e2e_ms = [e2e_run(args.e2e_steps)]
    e2e_step_ms, e2e_val = None, None
    if e2e_ms:
        e2e_step_ms, e2e_val = aggregate_ranks(statistics.median(e2e_ms), step_bytes, world,
                                               dist if world > 1 else None, dev)

    peak, peak_kind = peaks()
    means = {n: statistics.mean(v) for n, v in per.items()}
    solve_frac = {n: {"us": round(means[n] * 1e3, 2),
                      "GBps": round(nbytes[n] / (means[n] * 1e-3) / 1e9, 1),
                      "frac": round(nbytes[n] / (means[n] * 1e-3) / 1e9 / peak, 4)}
                  for n in names}
    # the dominant call of the step: the one that takes the most time (FP64:
    # the slowest solve, whose Thomas operation count defines the ALU roofline)
    dom = max(names if args.dtype == "f32" else names[:3], key=lambda n: means[n])
    fp64_rates = trid.fp64_rates(stream) if args.dtype == "f64" else None
    achieved = nbytes[dom] / (means[dom] * 1e-3) / 1e9
    traffic = profiled_traffic(f"{dom}_{args.dtype}_256")
    out = {
        "metric": METRIC, "value": round(value, 2), "unit": "GB/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_step, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": args.dtype,
        "data": "synthetic (seeded diagonally dominant coefficients; ADI from 3 sine eigenmodes)",
        "config": {"workload": WORKLOAD, "dims": list(DIMS), "lambda": LAM,
                   "parallelism": f"replicas{world}" if world > 1 else "single",
                   "l2": "flushed before every timed call (256 MiB write, then a 256 MiB read: no "
                         "input resident, no dirty lines left); inputs 256 MiB per solve",
                   "timing": "CUDA events per call on the launching stream, summed per step"},
        "per_call": solve_frac,
        "secondary": secondary,
        "adi_step_ms": round(means["adi_step"], 4),
        "adi_step_ms_graph100": (round(adi_graph_ms, 4) if isinstance(adi_graph_ms, float)
                                 else adi_graph_ms),
        "roofline": roofline_obj(args.dtype, dom, achieved, peak, peak_kind, traffic,
                                 nbytes[dom], means[dom], fp64_rates),
        "e2e": None if e2e_val is None else {
            "value": round(e2e_val, 2), "unit": "GB/s", "ms_per_step": round(e2e_step_ms, 3),
            "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
            "timing": f"{args.e2e_steps} steps pipelined over two device buffer sets "
                      "(first copy in to last copy out, / steps)"},
        "gpu_launches": launches_per_step * args.steps,
        "clocks": clock_info,
        "wall_s_timed_region": round(t_wall, 3),
    }
    if args.dtype != "f32":
        out["metric"] = METRIC + " [FP64 variant of the step]"
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline_sample(target_s=10.0)
    if world > 1:
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(out), flush=True)


# ------------------------------------------------------- oracle (CPU) side
def oracle_step(arrs, dims_s, u_adi, dims_adi):
    """One step of the oracle on (possibly sub-sampled) meshes; returns
    (seconds, algorithmic bytes in the FP32 convention)."""
    import oracle
    from paper_2201_03950_gb300 import metrics
    a, b, c, d = arrs
    t0 = time.perf_counter()
    nb = 0
    for k in range(3):
        oracle.solve_mesh(a, b, c, d, dims_s[k], k)
        nb += 5 * int(np.prod(dims_s[k])) * 4
    oracle.adi(u_adi, dims_adi, LAM, 1)
    nb += metrics.adi_step_bytes(int(np.prod(dims_adi)), 4, len(dims_adi))
    return time.perf_counter() - t0, nb


def sample_meshes(frac: float):
    """Sub-meshes holding ~frac of the systems of each solve: the outermost
    axis that is not the solve axis is shortened, system lengths stay 256.
    The ADI sample keeps full x/y planes and ~frac of the z planes."""
    n = DIMS[0]
    m = max(3, int(round(n * frac)))
    dims_s = [(n, n, m), (n, n, m), (n, m, n)]
    return dims_s, (n, n, max(3, m))


def _oracle_solves_f32(arrs32, dims_s):
    """The three solves of a step through the oracle's binary32 mesh solve;
    returns (seconds, algorithmic bytes)."""
    import oracle
    a, b, c, d = arrs32
    t0 = time.perf_counter()
    nb = 0
    for k in range(3):
        oracle.solve_mesh_f32(a, b, c, d, dims_s[k], k)
        nb += 5 * int(np.prod(dims_s[k])) * 4
    return time.perf_counter() - t0, nb


def _timed_gbs(fn, threads: int, reps: int = 5):
    """Median over `reps` runs (after one warm-up) of the aggregate GB/s of
    `threads` concurrent calls of fn() -> (seconds, bytes); each call works on
    its own data, and the oracle's C calls release the GIL."""
    import concurrent.futures as cf
    vals = []
    with cf.ThreadPoolExecutor(max_workers=threads) as ex:
        for rep in range(reps + 1):
            t0 = time.perf_counter()
            res = list(ex.map(lambda f: f(), [fn] * threads))
            wall = time.perf_counter() - t0
            if rep > 0:
                vals.append(sum(nb for _, nb in res) / wall / 1e9)
    return statistics.median(vals)


def cpu_baseline_sample(target_s: float = 10.0):
    """The oracle as it stands on the host cores: FP64 (the oracle's own
    precision) one core and all cores, and a binary32 run of the three solves
    for a like-for-like dtype.  All-cores runs give every core its own
    independent sub-mesh (systems are independent, as OpenMP over systems
    would split them).  Each figure is the median of 5 after one warm-up."""
    import oracle
    from paper_2201_03950_gb300 import inputs
    oracle.load()
    ncores = os.cpu_count() or 1
    n = DIMS[0]

    def make(m, dtype):
        dims_s = [(n, n, m), (n, n, m), (n, m, n)]
        tot = n * n * m
        arrs = inputs.dominant_system((tot,), seed=0, dtype=np.float32)
        arrs = [v.astype(dtype) for v in arrs]
        dims_adi = (n, n, max(3, m))
        u = inputs.sine_field(dims_adi, inputs.sine_modes(dims_adi, seed=0), dtype=np.float32)
        return arrs, dims_s, u.astype(np.float64), dims_adi

    t_start = time.perf_counter()
    # one core: a 64-plane sample (a quarter of each 256^3 solve and ADI step)
    a64, ds64, u64, da64 = make(64, np.float64)
    one_f64 = _timed_gbs(lambda: oracle_step(a64, ds64, u64, da64), 1)
    a32, ds32, _, _ = make(64, np.float32)
    one_f32 = _timed_gbs(lambda: _oracle_solves_f32(a32, ds32), 1)
    # all cores: the full 256^3 step split into one sub-mesh per core
    m_core = max(3, n // ncores)
    per_core = [make(m_core, np.float64) for _ in range(ncores)]
    it = iter(range(10 ** 9))
    import threading
    lock = threading.Lock()

    def next_mesh():
        with lock:
            return per_core[next(it) % ncores]

    def step_f64():
        arrs, ds_, u_, da_ = next_mesh()
        return oracle_step(arrs, ds_, u_, da_)

    all_f64 = _timed_gbs(step_f64, ncores)
    per_core32 = [make(m_core, np.float32)[:2] for _ in range(ncores)]
    it32 = iter(range(10 ** 9))

    def solves_f32():
        with lock:
            arrs, ds_ = per_core32[next(it32) % ncores]
        return _oracle_solves_f32(arrs, ds_)

    all_f32 = _timed_gbs(solves_f32, ncores)
    secs = time.perf_counter() - t_start
    return {"value": round(one_f64, 3), "unit": "GB/s", "cores": 1, "kind": "oracle",
            "nproc": ncores,
            "sample": (f"FP64 oracle step (solves x, y, z + one ADI step) on a 256x256x64 sample, "
                       f"one core; median of 5 after a warm-up ({secs:.0f} s for all four runs)"),
            "all_cores": {"value": round(all_f64, 3), "unit": "GB/s", "cores": ncores,
                          "dtype": "f64",
                          "sample": f"full 256^3 step split into {ncores} independent "
                                    f"256x256x{m_core} sub-meshes, one thread per core"},
            "f32": {"one_core": round(one_f32, 3), "all_cores": round(all_f32, 3),
                    "unit": "GB/s", "cores": [1, ncores],
                    "sample": "binary32 oracle solves along x, y, z (no ADI step: the oracle's "
                              "ADI is FP64 only), same samples"}}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle
    from paper_2201_03950_gb300 import inputs
    oracle.load()
    # size each step so that the whole run stays within ~2 minutes
    full_step_s = 3.5
    frac = min(1.0, 120.0 / max(1, args.steps + args.warmup) / full_step_s)
    dims_s, dims_adi = sample_meshes(frac)
    total = int(np.prod(DIMS))
    arrs = [v.astype(np.float64) for v in inputs.dominant_system((total,), seed=0, dtype=np.float32)]
    u = inputs.sine_field(dims_adi, inputs.sine_modes(dims_adi, seed=0)).astype(np.float64)
    for _ in range(args.warmup):
        oracle_step(arrs, dims_s, u, dims_adi)
    secs, nbytes = 0.0, 0
    for _ in range(args.steps):
        s, nb = oracle_step(arrs, dims_s, u, dims_adi)
        secs += s
        nbytes += nb
    val = nbytes / secs / 1e9
    sample = (f"per step: FP64 oracle solves on sub-meshes {dims_s} (systems of 256) + one ADI "
              f"step on {dims_adi}, single-threaded C; {frac:.3f} of the 256^3 workload")
    out = {
        "impl": "reference", "metric": METRIC, "value": round(val, 3), "unit": "GB/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(secs / args.steps * 1e3, 2), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD + " (bounded CPU sample)", "dims": list(DIMS)},
        "cpu_baseline": {"value": round(val, 3), "unit": "GB/s", "cores": 1, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": round(val, 3), "unit": "GB/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
        "gpu_launches": 0,
    }
    print(json.dumps(out), flush=True)


def main():
    args = parse()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
