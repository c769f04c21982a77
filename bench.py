#!/usr/bin/env python3
"""Benchmark: zone-updates per second per RK stage of the per-block GRMHD
finite-volume update on GB300, FP64 and mixed forms, with the roofline.

Workload (default): the 3-D Fishbone-Moncrief torus around a Kerr black hole
(a = 0.9375, modified Kerr-Schild), 512 x 256 x 256 cells as 2048 blocks of
32 x 32 x 16 with 3 ghost cells, PPM + HLL, GLM cleaning, SSP-RK2, loop field at
beta = 100, seeded +-2% pressure perturbation.  One step = ghost fill, stage 1,
ghost fill, stage 2 (the CFL reduction rides in stage 2).  A zone-update is one
interior cell through one RK stage, so value = cells x 2 x steps / time.

Our arm:   python bench.py [--gpus N --steps K --warmup W]
Reference: python bench.py --impl reference ...  (the FP64 CPU oracle on the
           host cores, on a bounded sample of the workload)
Prints one JSON line (rank 0).
"""
from __future__ import annotations

import argparse
import json
import os
import platform
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import problems as pb  # noqa: E402

NVAR = 9  # primitive (and conserved) variables per cell
METRIC = "zone-updates/s per RK stage"
UNIT = "zone-updates/s"
# ALU peaks derived from the part's unit counts and clock: per SM and clock,
# 2 FP64 fused multiply-adds (4 flops) and 128 FP32 ones (256 flops); the SM
# count is read from the device and the clock is the maximum SM clock
FP64_FLOPS_PER_SM_CLK = 4
FP32_FLOPS_PER_SM_CLK = 256
SAMPLE_CELLS = (128, 64, 64)  # bounded CPU sample of the torus workload


def workload(name: str):
    if name == "torus_3d_large":
        g = pb.torus_3d_large()
        desc = "3-D FM torus, Kerr a=0.9375, MKS, 512x256x256 cells as 2048 blocks of 32x32x16 (+3 ghosts)"
    elif name == "torus_3d_mid":
        g = pb.torus_3d_large(cells=(256, 128, 128))
        desc = "3-D FM torus, Kerr a=0.9375, MKS, 256x128x128 cells as 256 blocks of 32x32x16 (+3 ghosts)"
    elif name == "torus_3d":
        g = pb.torus_3d()
        desc = "3-D FM torus, Kerr a=0.9375, MKS, 192x96x96 cells as 432 blocks of 16^3 (+3 ghosts)"
    elif name == "torus_2d":
        g = pb.torus_2d()
        desc = "2-D FM torus, Kerr a=0.9375, MKS, 256x256 cells as 256 blocks of 16^2 (+3 ghosts)"
    elif name == "amr_torus":
        g = pb.amr_torus()
        lev = np.bincount(g.blocks[:, 0])
        desc = (f"3-D FM torus, Kerr a=0.9375, MKS, 3 levels of 16^3 blocks ({g.nb} leaves: "
                f"{lev[0]}/{lev[1]}/{lev[2]} per level, finest inside r < 20 M), one launch per stage")
    elif name == "shock_tube_2d":
        g = pb.shock_tube_2d()
        desc = "2-D SRMHD shock tube, 128x128 cells as 16 blocks of 32^2 (+3 ghosts)"
    else:
        raise SystemExit(f"unknown workload {name}")
    return g, desc


def initial_prims(g):
    return pb.shock_tube_prims(g) if g.coords == "cart" else pb.fm_torus_prims(g)


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def alu_peaks(torch, pk, device=0):
    """Derived FP64 and FP32 peaks in TFLOP/s: SMs x max SM clock x flops per
    SM and clock.  SM count from the device; clock from MEASURED_PEAKS.json
    (2070 MHz, the part's maximum, if that file lacks it)."""
    sms = torch.cuda.get_device_properties(device).multi_processor_count
    mhz = float(pk.get("sm_max_mhz") or 2070.0)
    return {"sms": sms, "sm_max_mhz": mhz,
            "fp64_tflops": sms * mhz * 1e6 * FP64_FLOPS_PER_SM_CLK / 1e12,
            "fp32_tflops": sms * mhz * 1e6 * FP32_FLOPS_PER_SM_CLK / 1e12,
            "kind": f"derived: {sms} SMs x {mhz:.0f} MHz x {FP64_FLOPS_PER_SM_CLK} FP64 / "
                    f"{FP32_FLOPS_PER_SM_CLK} FP32 flops per SM and clock"}


def probe_peaks(gb, torch, stream):
    """The arithmetic units' measured throughput (bhac_measure_peaks), outside
    any timed region."""
    r = gb.bhac_measure_peaks(1 << 14, stream.cuda_stream)
    return {"fp64_tflops": r["fp64_flops"] / 1e12, "fp32_tflops": r["fp32_flops"] / 1e12,
            "fp64_div_per_s": r["fp64_div"], "fp64_sqrt_per_s": r["fp64_sqrt"],
            "fp64_rsqrt_per_s": r["fp64_rsqrt"], "sms": r["sms"]}


class Clocks:
    """Samples nvidia-smi every 200 ms during the timed region."""

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 8:
                self.rows.append(parts)

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None

        sm = [v for v in (num(r[0]) for r in self.rows) if v is not None]
        mx = [v for v in (num(r[1]) for r in self.rows) if v is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[4 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def aggregate_ms(ms: float, dist, device) -> float:
    """Slowest rank's time: every rank runs its own replica of the workload
    (the update has no exchange between GPUs), so the job takes the max."""
    if dist is None:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(cells: int, world: int, ms_per_step: float) -> float:
    """Zone-updates per second of the whole job: world replicas x cells x 2 stages."""
    return cells * 2 * world / (ms_per_step * 1e-3)


TUNE = True
Z_PARTS = 0  # z parts per work item of the 3-D stage kernel (0: the library's choice)


def time_form(gb, torch, g, P, form, steps, warmup, stream, count_flops=True, graph_repeats=3, graph_steps=1,
              faces=None):
    """Device-resident timing of `steps` steps of one form (direct launches,
    per-stage events), then the same step replayed from a CUDA graph:
    median over `graph_repeats` repeats of `graph_steps` replays.  With
    `faces` the grid runs constrained transport (its own kernels: no launch
    shape to tune)."""
    from paper_2108_12240_gb300 import autotune

    s = gb.Solver(g, form, stream=stream)
    if faces is not None:
        shape, tried = (0, 0, 0, 0, 0, 0), {}
    elif TUNE:
        shape, tried = autotune.tune(s, P)  # launch shape for this grid and form (outside the timed region)
    else:
        shape, tried = autotune.cached_or_default(s), {}
    if faces is None and g.ndim == 3:
        s.set_zsplit(Z_PARTS)
    s.set_prims(P)
    if faces is not None:
        s.set_faces(faces)
    dt = s.cfl_dt()
    for _ in range(warmup):
        s.step(0.0)  # device dt: the same path as the timed loop
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    sev = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(steps)]
    with torch.cuda.stream(stream):
        ev[0].record(stream)
        for k in range(steps):
            sev[k][0].record(stream)
            gb.bhac_stage(s.ctx, 1, 0.0)  # ghost fill + stage-1 kernel
            sev[k][1].record(stream)
            sev[k][2].record(stream)
            gb.bhac_stage(s.ctx, 2, 0.0)  # ghost fill + stage-2 kernel (+ CFL rate)
            sev[k][3].record(stream)
        ev[1].record(stream)
    torch.cuda.synchronize()
    total_ms = ev[0].elapsed_time(ev[1])
    stage_ms = ([sev[k][0].elapsed_time(sev[k][1]) for k in range(steps)] +
                [sev[k][2].elapsed_time(sev[k][3]) for k in range(steps)])
    # the ghost fill alone on the same state and stream
    fe = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    with torch.cuda.stream(stream):
        fe[0].record(stream)
        for _ in range(steps):
            gb.bhac_fill_ghosts(s.ctx)
        fe[1].record(stream)
    torch.cuda.synchronize()
    fill_ms = fe[0].elapsed_time(fe[1]) / steps
    out = {"ms_per_step": total_ms / steps, "stage_ms_mean": sum(stage_ms) / len(stage_ms) - fill_ms,
           "fill_ms": fill_ms, "launch_shape": {"tx": shape[0], "ty": shape[1], "threads": shape[2],
                                                 "persistent": shape[3], "min_ctas": shape[4],
                                                 "producer_warps": shape[5] if len(shape) > 5 else 0,
                                                 "z_parts": s.zsplit_in_force(),
                                                 "candidates_timed": len(tried)}}
    if graph_repeats > 0:
        if graph_steps <= 0:  # enough replays for about 50 ms per repeat
            graph_steps = max(1, min(2000, int(50.0 / max(total_ms / steps, 1e-3))))
        s.capture(1)
        for _ in range(2):
            s.replay()
        torch.cuda.synchronize()
        reps = []
        for _ in range(graph_repeats):
            ge = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
            with torch.cuda.stream(stream):
                ge[0].record(stream)
                for _ in range(graph_steps):
                    s.replay()
                ge[1].record(stream)
            torch.cuda.synchronize()
            reps.append(ge[0].elapsed_time(ge[1]) / graph_steps)
        out["graph"] = {"ms_per_step_median": statistics.median(reps), "repeats": graph_repeats,
                        "steps_per_repeat": graph_steps}
    out["launches_per_step"] = s.launches_per_step()
    out["c2p_counts"] = [int(x) for x in s.diagnostics()]
    if count_flops:
        out["flops"] = s.count_flops(max(dt, 1e-30), nsamples=4000, seed=7)
    s.close()
    return out


TRAFFIC_FILE = os.path.join(ROOT, "profiles", "traffic_stage_kernel_torus_3d_large.txt")


# the sources that decide the stage kernel's code, its arguments and the data
# layout and block order it reads (test utilities, the flop counter and the
# allocation-free CFL entry point are not among them)
KERNEL_SOURCES = ["amr.cu", "amr.h", "api.cu", "aux.cu", "bhac_device.cuh", "ctx.h", "launch.h",
                  "stage_fp64.cu", "stage_impl.cuh", "stage_mixed.cu"]


def _code_only(text: str) -> str:
    """C/C++ source without comments and with whitespace collapsed (the
    sources hold no string literal containing a comment marker)."""
    import re
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    return " ".join(text.split())


def kernel_fingerprint() -> str:
    """sha256 over the code (comments and layout removed) of KERNEL_SOURCES,
    in this order."""
    import hashlib
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2108_12240_gb300", "csrc")
    for f in KERNEL_SOURCES:
        with open(os.path.join(csrc, f), encoding="utf-8") as fh:
            h.update(f.encode() + b"\0" + _code_only(fh.read()).encode())
    return h.hexdigest()


def fill_roofline(g, form: str, fill_ms: float, hbm_gbs):
    """HBM roofline of one ghost fill (the paper's fill_gc_srl), a gather:
    per ghost cell the nine values read and written (FP64 in the FP64 form,
    the FP32 copy in the mixed form) plus the map's int32 source index and
    flag byte."""
    ghosts = g.nb * (int(np.prod([g.nx[d] + (2 * g.ng if d < g.ndim else 0) for d in range(3)]))
                     - int(np.prod(g.nx)))
    fill_bytes = ghosts * (NVAR * (4 if form.startswith("mixed") else 8) * 2 + 5)
    gbs = fill_bytes / (fill_ms * 1e-3) / 1e9 if fill_ms > 0 else None
    return {"bound": "hbm", "achieved": gbs, "peak": hbm_gbs, "unit": "GB/s",
            "frac": gbs / hbm_gbs if (gbs and hbm_gbs) else None,
            "bytes_per_fill": fill_bytes, "ghost_cells": ghosts, "ms": fill_ms}


def shape_key(ls) -> str:
    """Launch shape as recorded beside a traffic figure."""
    # the persistent schedule (which CTA takes which item) does not change the
    # per-launch DRAM bytes and is left out
    return (f"{ls['tx']}x{ls['ty']}/{ls['threads']}/minctas{ls['min_ctas']}/producers{ls['producer_warps']}"
            f"/zparts{ls.get('z_parts', 1)}")


def recorded_traffic(workload_name, form, tile):
    """DRAM bytes per stage-kernel launch from the committed ncu summary, when
    it was taken of these exact sources, this workload, form and tile; else None."""
    try:
        with open(TRAFFIC_FILE) as f:
            kv = dict(line.split(":", 1) for line in f.read().splitlines() if ":" in line and not line.startswith("#"))
    except OSError:
        return None
    kv = {k.strip(): v.strip() for k, v in kv.items()}
    if kv.get("sources_sha256") != kernel_fingerprint() or kv.get("workload") != workload_name:
        return None
    try:
        return float(kv[f"traffic {form} {tile}"].split()[0])
    except (KeyError, ValueError, IndexError):
        return None


def e2e_form(gb, torch, g, P, form, steps, stream):
    """Through the public API with host buffers: every step loads its
    primitives from pinned host memory (bhac_set_prims_host_async), runs the
    CFL reduction and the RK step, and reads its primitives back to pinned host
    memory (bhac_get_prims_host_async), all inside the timed region, which two
    host fences close on both sides.  The library's copy streams overlap the
    next step's load and this step's read-back with the kernels (the host link
    carries both directions at once)."""
    s = gb.Solver(g, form, stream=stream)
    from paper_2108_12240_gb300 import autotune
    autotune.cached_or_default(s)  # the shape time_form tuned for this grid and form
    host_in = torch.from_numpy(np.ascontiguousarray(P)).pin_memory()
    host_out = torch.empty(host_in.shape, dtype=torch.float64).pin_memory()
    nbytes = host_in.numel() * 8

    def run(k):
        s.host_fence()
        s.set_prims_host_async(host_in)
        for n in range(k):
            gb.bhac_cfl_dt(s.ctx, False)
            gb.bhac_step(s.ctx, 0.0)
            s.get_prims_host_async(host_out)
            if n + 1 < k:
                s.set_prims_host_async(host_in)
        s.host_fence()

    with torch.cuda.stream(stream):
        run(1)  # untimed warm-up: first use of the load and gather kernels and the pinned buffers
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    with torch.cuda.stream(stream):
        ev[0].record(stream)
        run(steps)
        ev[1].record(stream)
    torch.cuda.synchronize()
    ms = ev[0].elapsed_time(ev[1])
    launches = s.launches_per_step() + 2  # + the load (primitives, conserved state, CFL rate) and the gather
    s.close()
    return {"value": g.ncells * 2 * steps / (ms * 1e-3), "unit": UNIT, "h2d_bytes_per_step": nbytes,
            "d2h_bytes_per_step": nbytes, "ms_per_step": ms / steps, "kernels_per_step": launches}


def sample_grid(name):
    if name == "torus_3d_large":
        return pb.torus_3d_large(cells=SAMPLE_CELLS)
    if name == "amr_torus":
        return pb.amr_torus(root=(4, 2, 2), nblock=8)
    return workload(name)[0]


def cpu_baseline(name, budget_s=20.0):
    """The FP64 oracle (plain C, OpenMP over blocks) on a bounded sample of the
    workload: the same torus, physics and block shape at reduced resolution."""
    import oracle
    g = sample_grid(name)
    o = oracle.Oracle(g)
    o.set_prims(initial_prims(g))
    dt = o.cfl_dt()
    n = 0
    t0 = time.perf_counter()
    while True:
        o.step(dt)
        n += 1
        el = time.perf_counter() - t0
        if el > budget_s or n >= 50:
            break
    threads = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    nc = [g.nx[d] * g.nroot[d] for d in range(3)]
    return {"value": g.ncells * 2 * n / el, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"{n} oracle steps of the same problem at {nc[0]}x{nc[1]}x{nc[2]} cells "
                      f"({g.nb} blocks of {g.nx[0]}x{g.nx[1]}x{g.nx[2]}), {el:.1f} s",
            "single_thread": cpu_single_thread(name), "cpu_model": cpu_model()}


def cpu_model() -> str:
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    return platform.processor() or platform.machine()


_SINGLE = """
import sys, time, json
sys.path.insert(0, {root!r})
import oracle, problems as pb
g = pb.torus_3d_large(cells=(64, 32, 32)) if {name!r} == "torus_3d_large" else None
if g is None:
    print(json.dumps(None)); raise SystemExit
o = oracle.Oracle(g)
o.set_prims(pb.fm_torus_prims(g))
dt = o.cfl_dt()
n, t0 = 0, time.perf_counter()
while True:
    o.step(dt); n += 1
    el = time.perf_counter() - t0
    if el > {budget} or n >= 20:
        break
print(json.dumps({{"value": g.ncells * 2 * n / el, "steps": n, "seconds": el}}))
"""


def cpu_single_thread(name, budget_s=5.0):
    """The oracle on one host thread (OMP_NUM_THREADS=1, own process) on a
    64x32x32-cell sample of the same torus and block shape."""
    env = dict(os.environ, OMP_NUM_THREADS="1")
    code = _SINGLE.format(root=ROOT, name=name, budget=budget_s)
    try:
        r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=120)
        res = json.loads(r.stdout.strip().splitlines()[-1]) if r.returncode == 0 and r.stdout.strip() else None
    except (OSError, subprocess.SubprocessError, ValueError):
        res = None
    if not res:
        return None
    return {"value": res["value"], "unit": UNIT, "cores": 1,
            "sample": f"{res['steps']} oracle steps at 64x32x32 cells (4 blocks of 32x32x16), "
                      f"{res['seconds']:.1f} s"}


def reference_arm(args, rank):
    """The oracle on the host cores, each step a bounded sample of the workload."""
    if rank != 0:
        return
    import oracle
    _, desc = workload(args.workload)
    gs = sample_grid(args.workload)
    o = oracle.Oracle(gs)
    o.set_prims(initial_prims(gs))
    dt = o.cfl_dt()
    for _ in range(args.warmup):
        o.step(dt)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        o.step(dt)
    el = time.perf_counter() - t0
    threads = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    v = gs.ncells * 2 * args.steps / el
    nc = [gs.nx[d] * gs.nroot[d] for d in range(3)]
    sample = (f"each step: one oracle step of the same problem at {nc[0]}x{nc[1]}x{nc[2]} cells "
              f"({gs.nb} blocks of {gs.nx[0]}x{gs.nx[1]}x{gs.nx[2]})")
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded Fishbone-Moncrief torus)",
            "config": {"workload": desc, "sample": sample},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def shape_runs(args):
    """For a profiler capture: the workload in the given launch shapes, each
    set_launch (and, with a seventh value, bhac_set_split's chunk count),
    set_prims, cfl_dt and four device-dt steps (no timing, no output but one
    line per shape)."""
    import torch

    import paper_2108_12240_gb300 as gb

    torch.cuda.set_device(0)
    form, shapes = args.shape_runs[0], [tuple(int(x) for x in a.split(",")) for a in args.shape_runs[1:]]
    g, _ = workload(args.workload)
    P = initial_prims(g)
    stream = torch.cuda.Stream()
    s = gb.Solver(g, form, stream=stream)
    for sh in shapes:
        s.set_launch(*sh[:6])
        s.set_split(sh[6] if len(sh) > 6 else 0)
        s.set_prims(P)
        s.cfl_dt()
        for _ in range(4):
            s.step(0.0)
        torch.cuda.synchronize()
        print(form, sh, "done", flush=True)
    s.close()


def split_sweep(args):
    """Fused stage kernel against the split form (face kernel, then cell kernel
    on a second stream, in chunks): ms per step of the workload for each chunk
    count, persistent setting and register bound, both forms, with the clocks.
    One JSON line; not the bench contract line."""
    import torch

    import paper_2108_12240_gb300 as gb

    torch.cuda.set_device(0)
    g, desc = workload(args.workload)
    P = initial_prims(g)
    stream = torch.cuda.Stream()
    out = {"sweep": "split form", "workload": desc, "forms": {}}
    for form in ("mixed", "fp64"):
        s = gb.Solver(g, form, stream=stream)
        # the fused shapes the autotuner picks on this torus, then the split ones
        cases = [(0, 2, 2), (0, 1, 1)] if form == "mixed" else [(0, 1, 1), (0, 2, 2)]
        for chunks in ((1, 4, 8) if form == "mixed" else (1, 8)):
            for minb in ((1, 2, 3) if form == "mixed" else (1, 2)):
                for pers in (0, minb):
                    cases.append((chunks, pers, minb))
        rows = []
        with Clocks(0) as ck:
            for chunks, pers, minb in cases:
                s.set_launch(16, 16, 256, pers, minb, 0)
                s.set_split(chunks)
                s.set_prims(P)
                s.cfl_dt()
                for _ in range(args.warmup):
                    s.step(0.0)
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                for _ in range(args.steps):
                    s.step(0.0)
                e1.record(stream)
                torch.cuda.synchronize()
                ms = e0.elapsed_time(e1) / args.steps
                rows.append({"chunks": chunks, "persistent": pers, "min_ctas": minb, "ms_per_step": ms,
                             "zone_updates_per_s": job_value(g.ncells, 1, ms)})
                print(json.dumps({"form": form, **rows[-1]}), file=sys.stderr, flush=True)
        s.close()
        del s
        torch.cuda.empty_cache()
        out["forms"][form] = {"rows": rows, "clocks": ck.summary()}
    print(json.dumps(out), flush=True)


CONFIGS = ["shock_tube_2d", "torus_2d", "torus_3d", "amr_torus", "torus_3d_large"]


def all_configs(args):
    """Every workload configuration (0: 2-D shock tube ... 4: the 512x256x256
    torus), both forms: zone-updates/s with direct launches and with CUDA-graph
    replays (median of 15 repeats), FP64 flop fraction.  One JSON line per
    configuration; not the bench contract line."""
    import torch

    import paper_2108_12240_gb300 as gb

    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    alu = alu_peaks(torch, peaks()[0])
    for cfg, name in enumerate(CONFIGS):
        g, desc = workload(name)
        P = initial_prims(g)
        forms = {}
        for form in ("mixed", "fp64"):
            with Clocks(0) as ck:
                r = time_form(gb, torch, g, P, form, args.steps, args.warmup, stream, graph_repeats=15, graph_steps=0)
            stage_s = r["stage_ms_mean"] * 1e-3
            ach = r["flops"]["fp64_flops"] * g.ncells / stage_s / 1e12
            forms[form] = {"zone_updates_per_s": job_value(g.ncells, 1, r["ms_per_step"]),
                           "zone_updates_per_s_graph": job_value(g.ncells, 1, r["graph"]["ms_per_step_median"]),
                           "ms_per_step": r["ms_per_step"], "graph": r["graph"], "stage_ms": r["stage_ms_mean"],
                           "ghost_fill_ms": r["fill_ms"], "fp64_flops_per_zone_stage": r["flops"]["fp64_flops"],
                           "fp64_frac": ach / alu["fp64_tflops"], "launch_shape": r["launch_shape"],
                           "clocks": ck.summary()}
        state_mb = g.ncells * 9 * 8 * 2 / 1e6
        print(json.dumps({"config": cfg, "workload": name, "desc": desc, "cells": g.ncells, "blocks": g.nb,
                          "state_mb_fp64": state_mb, "l2_resident": state_mb < 100, "forms": forms}), flush=True)


def regrid_timing(args):
    """One regrid of the 3-level AMR torus (4220 leaves of 16^3), mixed form,
    cleaning and constrained transport: the device estimator, the host plan
    (thresholds 0.3 / 0.05, max level 2), the new context (host maps, arena,
    metric tables) and the device transfer, beside one step; one JSON line per
    form of div B control (CUDA events on the context's stream for the device
    parts, host wall time for the plan and the new context)."""
    import torch

    import paper_2108_12240_gb300 as gb
    from problems import ct as pct

    torch.cuda.set_device(0)
    g0 = pb.amr_torus()
    P = pb.fm_torus_prims(g0)
    st = torch.cuda.Stream()

    def ev():
        return torch.cuda.Event(enable_timing=True)

    for divb in ("glm", "ct"):
        g = g0.with_(divb=divb)
        s = gb.Solver(g, "mixed", stream=st)
        s.set_prims(P)
        if divb == "ct":
            s.set_faces(pct.fm_torus_faces(g, P))
        s.cfl_dt()
        s.step(0.0)
        torch.cuda.synchronize()
        a, b = ev(), ev()
        a.record(st)
        s.step(0.0)
        b.record(st)
        torch.cuda.synchronize()
        step_ms = a.elapsed_time(b)
        a, b = ev(), ev()
        a.record(st)
        err = s.estimate()
        b.record(st)
        torch.cuda.synchronize()
        est_ms = a.elapsed_time(b)
        t0 = time.perf_counter()
        new = gb.bhac_regrid_plan(gb.desc_of(g, "mixed"), gb.blocks_of(g), err, 0.3, 0.05, 2)
        plan_s = time.perf_counter() - t0
        t0 = time.perf_counter()
        fresh = gb.Solver(g.with_(blocks=new), "mixed", stream=st)
        torch.cuda.synchronize()
        init_s = time.perf_counter() - t0
        a, b = ev(), ev()
        a.record(st)
        gb.bhac_regrid_transfer(s.ctx, fresh.ctx)
        b.record(st)
        torch.cuda.synchronize()
        print(json.dumps({"divb": divb, "leaves": [g.nb, int(len(new))], "step_ms": step_ms, "estimate_ms": est_ms,
                          "plan_s": plan_s, "new_context_s": init_s, "transfer_ms": a.elapsed_time(b)}), flush=True)
        s.close()
        fresh.close()
        del s, fresh
        torch.cuda.empty_cache()


def sweep_blocks(args):
    """The 512x256x256 torus in several block shapes (8^3 to 32^3): zone-updates/s
    and FP64 roofline fraction per shape and form, one JSON line."""
    import torch

    import paper_2108_12240_gb300 as gb

    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    pk = peaks()[0]
    alu = alu_peaks(torch, pk)
    rows = []
    for nb in [(8, 8, 8), (16, 16, 16), (32, 32, 16), (32, 32, 32)]:
        g = pb.torus_3d_large(nblock=nb)
        P = initial_prims(g)
        for form in ("mixed", "fp64"):
            with Clocks(0) as ck:
                r = time_form(gb, torch, g, P, form, args.steps, args.warmup, stream)
            stage_s = r["stage_ms_mean"] * 1e-3
            ach = r["flops"]["fp64_flops"] * g.ncells / stage_s / 1e12
            rows.append({"block": "x".join(map(str, nb)), "blocks": g.nb, "form": form,
                         "zone_updates_per_s": job_value(g.ncells, 1, r["ms_per_step"]),
                         "stage_ms": r["stage_ms_mean"], "ghost_fill_ms": r["fill_ms"],
                         "fp64_flops_per_zone_stage": r["flops"]["fp64_flops"],
                         "fp64_frac": ach / alu["fp64_tflops"], "launch_shape": r["launch_shape"],
                         "ghost_fill": fill_roofline(g, form, r["fill_ms"], pk.get("hbm_gbs")),
                         "clocks": ck.summary()})
            print(json.dumps(rows[-1]), file=sys.stderr, flush=True)
        del P
    print(json.dumps({"sweep": "block shape", "workload": "512x256x256 torus", "rows": rows}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="torus_3d_large")
    ap.add_argument("--form", default="both", choices=["both", "mixed", "fp64"])
    ap.add_argument("--c2p", default="newton", choices=["newton", "nk"],
                    help="primary inversion: analytic Newton (default) or Jacobian-free Newton-Krylov")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-ct", action="store_true", help="skip the constrained-transport form")
    ap.add_argument("--sweep-blocks", action="store_true", help="block-shape roofline sweep instead of the bench line")
    ap.add_argument("--regrid-timing", action="store_true", help="one regrid of the AMR torus, timed by part")
    ap.add_argument("--all-configs", action="store_true", help="every workload configuration, one line each")
    ap.add_argument("--shape-runs", nargs="+", metavar="FORM_OR_SHAPE",
                    help="FORM tx,ty,threads,persistent,min_ctas,producers ...: four steps per shape, for ncu")
    ap.add_argument("--split-sweep", action="store_true",
                    help="fused stage kernel against the split form (face + cell kernels), one line")
    ap.add_argument("--z-parts", type=int, default=0,
                    help="z parts per work item of the 3-D stage kernel (0: the library's choice)")
    ap.add_argument("--no-tune", action="store_true", help="use the cached launch shape (or the default) without timing candidates")
    args = ap.parse_args()
    global TUNE, Z_PARTS
    TUNE = not args.no_tune
    Z_PARTS = args.z_parts
    if args.sweep_blocks:
        sweep_blocks(args)
        return
    if args.regrid_timing:
        regrid_timing(args)
        return
    if args.all_configs:
        all_configs(args)
        return
    if args.shape_runs:
        shape_runs(args)
        return
    if args.split_sweep:
        split_sweep(args)
        return

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        reference_arm(args, rank)
        return

    import torch

    import paper_2108_12240_gb300 as gb

    if args.warmup < 3:
        raise SystemExit("at least 3 warm-up steps")
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    # the CPU baseline first (rank 0 at N = 1), before any GPU work
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline(args.workload)

    g, desc = workload(args.workload)
    P = initial_prims(g)
    if args.c2p != "newton":
        g = g.with_(c2p=args.c2p)
        desc += f"; {args.c2p} inversion"
    stream = torch.cuda.Stream()
    forms = ["mixed", "fp64"] if args.form == "both" else [args.form]
    ct_faces = None
    if args.form == "both" and not args.no_ct and g.coords == "mks":
        # constrained transport beside the cleaning forms: the same torus with
        # its loop field as face fields, both forms
        from problems import ct as pct
        ct_faces = pct.fm_torus_faces(g, P)
        forms += ["mixed_ct", "fp64_ct"]
    results = {}
    for form in forms:
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        with Clocks(local) as ck:
            if form.endswith("_ct"):
                results[form] = time_form(gb, torch, g.with_(divb="ct"), P, form[:-3], args.steps, args.warmup,
                                          stream, faces=ct_faces)
            else:
                results[form] = time_form(gb, torch, g, P, form, args.steps, args.warmup, stream)
        results[form]["clocks"] = ck.summary()
        results[form]["ms_per_step"] = aggregate_ms(results[form]["ms_per_step"], dist, "cuda")
        # each rank advances its own full replica (weak scaling)
        results[form]["value"] = job_value(g.ncells, world, results[form]["ms_per_step"])
    head = forms[0]
    e2e = None
    if not args.no_e2e:
        if dist:
            dist.barrier()
        e2e = e2e_form(gb, torch, g, P, head, max(1, args.steps), stream)
        # the whole job: every replica's zone-updates over the slowest rank's time
        e2e["ms_per_step"] = aggregate_ms(e2e["ms_per_step"], dist, "cuda")
        e2e["value"] = job_value(g.ncells, world, e2e["ms_per_step"])
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return

    pk, pk_kind = peaks()
    alu = alu_peaks(torch, pk, local)
    with Clocks(local) as ck_probe:
        probe = probe_peaks(gb, torch, stream)
    probe["clocks"] = ck_probe.summary()

    def roofline(form):
        r = results[form]
        fl = r["flops"]
        stage_s = r["stage_ms_mean"] * 1e-3
        cells = g.ncells
        ach64 = fl["fp64_flops"] * cells / stage_s / 1e12
        # algorithmic bytes per zone-stage: FP64 288 (read P and U, write P and
        # U, nine FP64 values each); mixed 252 (the FP32 primitive copy read in
        # place of the FP64 one); constrained transport adds the face fields
        # read and written (3 x 8 B each way)
        bytes_alg = {"fp64": 288, "mixed": 252, "fp64_ct": 336, "mixed_ct": 300}[form] * cells
        traffic = recorded_traffic(args.workload, form, shape_key(r["launch_shape"])) if args.c2p == "newton" else None
        fill = fill_roofline(g, form, r["fill_ms"], pk.get("hbm_gbs"))
        return {"bound": "alu", "achieved": ach64, "peak": alu["fp64_tflops"], "unit": "TFLOP/s",
                "frac": ach64 / alu["fp64_tflops"], "traffic": traffic,
                "kernel": "ct_flux/ct_face/ct_cell kernels" if form.endswith("_ct") else "stage_kernel",
                "traffic_source": os.path.relpath(TRAFFIC_FILE, ROOT) if traffic else None,
                "traffic_over_algorithmic": traffic / bytes_alg if traffic else None,
                "stage_ms": r["stage_ms_mean"], "ghost_fill_ms": r["fill_ms"],
                "peak_kind": alu["kind"],
                "peak_probe": probe["fp64_tflops"], "frac_of_probe": ach64 / probe["fp64_tflops"],
                "fp64_flops_per_zone_stage": fl["fp64_flops"],
                "fp32_flops_per_zone_stage": fl["fp32_flops"],
                "fp32_frac_of_peak": fl["fp32_flops"] * cells / stage_s / 1e12 / alu["fp32_tflops"],
                "hbm_bytes_per_zone_stage": bytes_alg / cells,
                "hbm_frac_of_measured": bytes_alg / stage_s / 1e9 / pk["hbm_gbs"],
                "ghost_fill": fill}

    r = results[head]
    line = {
        "metric": METRIC, "value": r["value"], "unit": UNIT,
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": r["ms_per_step"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+f64" if head == "mixed" else "f64",
        "data": "synthetic (seeded Fishbone-Moncrief torus)",
        "config": {"workload": desc, "form": head, "replicas": world,
                   "l2": (f"inputs larger than L2 (arena {gb.bhac_query_sizes(gb.desc_of(g, head), gb.blocks_of(g)) / 1e9:.1f} GB"
                          f" against {getattr(torch.cuda.get_device_properties(local), 'L2_cache_size', 0) / 1e6:.0f} MB"
                          " of L2), no flush"),
                   "launch": "per step: ghost fill + stage kernel, twice; device dt; shape by autotuner"},
        "forms": {f: {"value": results[f]["value"], "ms_per_step": results[f]["ms_per_step"],
                      "roofline": roofline(f), "c2p_counts": results[f]["c2p_counts"],
                      "launch_shape": results[f]["launch_shape"],
                      "clocks": results[f]["clocks"]} for f in forms},
        "roofline": roofline(head),
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": results[head]["launches_per_step"] * args.steps,
        "clocks": results[head]["clocks"],
        "peaks": {"kind": pk_kind, "hbm_gbs": pk.get("hbm_gbs"), "alu": alu, "probe": probe},
    }
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
