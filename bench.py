"""Benchmark of the explicit SPFM step on GB300.

Workload (default): spherical grain of radius 150 at the centre of a 512^3
FP32 grid, lambda = 3, 27-point stencil, TI potential with u || [120]
(TI_<120>), dF = 0.02, dt = 0.05, periodic boundaries.  A "step" is one
explicit time step of the whole grid (one launch of the stencil kernel); the
FP64 interface diagnostics run every 50 steps inside the timed region.

Prints one JSON line (rank 0).  Under torchrun each rank runs its own replica
of the workload on its GPU (the path has no exchange step: replicas only) and
`value` sums the cells all ranks updated over the max-over-ranks time.

``--impl reference`` times the FP64 CPU oracle on the host cores instead (a
z-slab of the same grid per step) and prints the same line with
"impl": "reference".
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("SPFM cell-updates/s and % HBM roofline (1 GB300); batched/served vs plain at "
          "1e-4 vel err; p99")
UNIT = "cell-updates/s"
STATS_EVERY = 50
BYTES_PER_UPDATE = {"f32": 8, "f64": 16, "bf16": 4}   # one read + one write of phi per step
NOMINAL_HBM_GBS = 7900.0   # GB300 HBM3e nominal bandwidth, for context beside the measured peak


def finite_json(obj):
    """obj with every non-finite float (NaN, +-Inf) replaced by None and numpy
    scalars made plain, so that the line is strict JSON."""
    if isinstance(obj, np.generic):
        obj = obj.item()
    if isinstance(obj, float):
        return obj if math.isfinite(obj) else None
    if isinstance(obj, dict):
        return {str(k): finite_json(v) for k, v in obj.items()}
    if isinstance(obj, (list, tuple)):
        return [finite_json(v) for v in obj]
    return obj


def dumps(line) -> str:
    return json.dumps(finite_json(line), allow_nan=False)


def emit(line):
    print(dumps(line), flush=True)


# the keys of the final (headline) line; every study leg goes out before it as
# a line of its own ({"leg": name, ...}), so the headline stays short
HEADLINE_KEYS = ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                 "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config", "roofline",
                 "cpu_baseline", "e2e", "clocks", "gpu_launches", "stats_call", "legs")


def headline(line: dict) -> dict:
    return {k: line[k] for k in HEADLINE_KEYS if k in line}


def stats_cadence(steps: int) -> int:
    """Steps between two stats calls of the timed region: every STATS_EVERY
    steps, and at least once in any run."""
    return max(1, min(STATS_EVERY, steps))


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--dtype", default="f32", choices=["f32", "f64", "bf16"])
    ap.add_argument("--scheme", default="ti120", choices=["ti120", "fd", "local"])
    ap.add_argument("--rounding", default="nearest", choices=["nearest", "stochastic"],
                    help="rounding of the update of the timed grid (FP32/BF16)")
    ap.add_argument("--no-variants", action="store_true", help="skip the TI_n / CF timings")
    ap.add_argument("--no-bf16", action="store_true", help="skip the BF16-storage leg")
    ap.add_argument("--no-relax", action="store_true", help="skip the constant-volume shape relaxation")
    ap.add_argument("--no-friction", action="store_true", help="skip the 1D friction study")
    ap.add_argument("--no-force-scan", action="store_true", help="skip the force-oscillation scan")
    ap.add_argument("--no-kinetic", action="store_true", help="skip the 3D kinetic-anisotropy study")
    ap.add_argument("--no-tilted", action="store_true", help="skip the 256^3 tilted-plane FP32/FP64 leg")
    ap.add_argument("--n", type=int, default=512, help="grid edge")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched-vs-plain sweep")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving run")
    ap.add_argument("--serve-jobs", type=int, default=2000)
    ap.add_argument("--sweep-grids", type=int, default=256)
    ap.add_argument("--tilted-only", action="store_true",
                    help="only the 256^3 tilted plane with contact faces (FP32 TI_<111>): 5 + 50 steps, "
                         "its step rate (a small command to profile the contact-face path)")
    ap.add_argument("--batch-only", action="store_true",
                    help="only the batched sweep: build it, 32 + 64 steps, print its rate (a small "
                         "command to profile the batch kernel)")
    return ap.parse_args(argv)


def workload(args):
    from paper_1910_05180_gb300 import workloads as WL
    w = dict(WL.sphere_512cubed())
    if args.n != 512:
        w["nx"] = w["ny"] = w["nz"] = args.n
        w["ctr"] = ((args.n - 1) / 2.0,) * 3
        w["R"] = 150.0 * args.n / 512.0
        w["name"] = f"sphere_{args.n}cubed_R{w['R']:g}"
    return w


SCHEME_NAME = {"ti120": "TI_<120>", "fd": "CF+h3", "local": "TI_n"}


def arm_config(args, w, ws):
    """The `config` of the JSON line, the same for the GPU arm and the oracle arm."""
    cells = w["nx"] * w["ny"] * w["nz"]
    sr = "_sr" if getattr(args, "rounding", "nearest") == "stochastic" else ""
    return {"workload": w["name"] + f"_{args.scheme}_{args.dtype}{sr}_27pt",
            "grid": [w["nx"], w["ny"], w["nz"]], "stencil": 27, "scheme": SCHEME_NAME[args.scheme],
            "lambda": w["lam"], "dt": w["dt"], "dF": w["dF"], "bc": "periodic",
            "stats_every": stats_cadence(args.steps),
            "l2": "inputs larger than L2 (two %d MB fields)" % (cells * BYTES_PER_UPDATE[args.dtype] // 2 // 2**20),
            "parallelism": "replicas" if ws > 1 else "single"}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(ms: float, ws: int, device) -> float:
    """The largest of the ranks' times (all-reduce MAX over the default process
    group when ws > 1): the job's time is its slowest replica's."""
    if ws <= 1:
        return float(ms)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_value(cells: int, steps: int, ws: int, max_ms: float) -> float:
    """Whole-job cell-updates/s of ws independent replicas: every rank's cells
    and steps over the slowest rank's time."""
    return ws * cells * steps / (max_ms / 1e3)


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 100 ms.  The sampler
    starts before the warm-up; `mark(t0, t1)` gives the host wall-clock bounds
    of the timed region, and the summary keeps the samples that fall inside it
    (widened by one sampling period on each side, since a short timed region
    may see none otherwise)."""

    Q = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    PERIOD_MS = 100

    def __init__(self, gpu_index: int):
        self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.proc = None
        self.gpu = gpu_index
        self.window = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", str(self.PERIOD_MS)], stdout=self.file, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def wait_live(self, timeout_s: float = 5.0):
        """Return once the sampler has written its first sample (or after timeout_s)."""
        if self.proc is None:
            return
        t_end = time.time() + timeout_s
        while time.time() < t_end and os.path.getsize(self.file.name) == 0:
            time.sleep(0.02)

    def mark(self, t0: float, t1: float):
        self.window = (t0, t1)

    @staticmethod
    def parse_rows(lines, window=None, slack_s: float = 0.0):
        """Rows of the sampler's CSV; with a window, only those inside it."""
        import datetime
        rows = []
        for ln in lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 10:
                continue
            try:
                ts = datetime.datetime.strptime(parts[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
            except ValueError:
                ts = None
            rows.append((ts, parts[1:]))
        if window is not None:
            inside = [r for t, r in rows if t is not None and window[0] - slack_s <= t <= window[1] + slack_s]
            return inside, True
        return [r for _, r in rows], False

    @staticmethod
    def summarise(rows, in_window: bool) -> dict:
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        num = lambda s: s.replace(".", "", 1).isdigit()
        sm = [float(r[1]) for r in rows if num(r[1])]
        mx = [float(r[2]) for r in rows if num(r[2])]
        pw = [float(r[3]) for r in rows if num(r[3])]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "power_w_max": max(pw) if pw else None,
                "reasons": reasons, "samples": len(rows),
                "window": "timed region" if in_window else "warm-up and timed region"}

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        self.proc.wait()
        self.file.flush()
        with open(self.file.name) as f:
            lines = f.readlines()
        os.unlink(self.file.name)
        rows, in_window = self.parse_rows(lines, self.window, 1e-3 * self.PERIOD_MS)
        if not rows:      # a timed region shorter than the sampling period saw no sample
            rows, in_window = self.parse_rows(lines)
        return self.summarise(rows, in_window)


def issue_ceiling(dev, warp_inst_per_cell: float) -> float:
    """Cell updates/s at the full issue rate: SMs x 4 schedulers x the maximum
    SM clock (MEASURED_PEAKS.json, else 2070 MHz) warp instructions per
    second over the warp instructions one cell update takes."""
    import torch
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    mhz = 2070.0
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            mhz = float(json.load(f).get("sm_max_mhz", mhz))
    except (OSError, ValueError):
        pass
    return sms * 4 * mhz * 1e6 / warp_inst_per_cell


def measured_hbm_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


# the sources that decide the stencil kernel's code (its traffic record is
# dropped as soon as one of them changes)
STEP_SOURCES = ("spfm_internal.h", "step_kernel.cuh", "tiles.h", "step_f32.cu", "step_f64.cu", "step_bf16.cu",
                "step_f32_img.cu", "step_f64_img.cu", "step_bf16_img.cu")
TRAFFIC_PATH = os.path.join(ROOT, "profiles", "traffic.json")


def source_hash(names=STEP_SOURCES):
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1910_05180_gb300", "csrc")
    for name in sorted(names):
        with open(os.path.join(csrc, name), "rb") as f:
            h.update(name.encode())
            h.update(f.read())
    return h.hexdigest()[:16]


def profiled_record(kernel_key: str, field: str):
    """A figure of the committed ncu summaries (profiles/traffic.json), only
    while the kernel sources are unchanged since the capture."""
    try:
        with open(TRAFFIC_PATH) as f:
            d = json.load(f)
    except (OSError, ValueError):
        return None
    e = d.get(kernel_key)
    if not e or e.get("source_hash") != source_hash():
        return None
    return e.get(field)


def profiled_traffic(kernel_key: str):
    """DRAM bytes per launch from the committed ncu summary."""
    return profiled_record(kernel_key, "bytes_per_launch")


# ------------------------------------------------------------------ oracle arm


def _oracle_slab(w, nz_slab, scheme="ti120"):
    import oracle as O
    osch = {"ti120": O.TI_GLOBAL, "fd": O.CF, "local": O.TI_LOCAL}[scheme]
    p = O.Params(w["nx"], w["ny"], nz_slab, bc=(O.PERIODIC,) * 4 + (O.NOFLUX, O.NOFLUX),
                 n=w["u"], lam=w["lam"], dx=w["dx"], M=w["M"], Gamma=w["Gamma"], dt=w["dt"],
                 dF=w["dF"], stencil=w["stencil"], scheme=osch)
    # the slab is the z-range around the grain's centre plane
    phi = O.init_sphere(p, (w["ctr"][0], w["ctr"][1], (nz_slab - 1) / 2.0), w["R"])
    return p, phi


def oracle_slab_for(w, seconds_per_step: float) -> int:
    """z-thickness of the oracle slab whose one step takes about seconds_per_step."""
    import oracle as O
    p, phi = _oracle_slab(w, 2)
    O.step(p, phi, 1)                      # loads the library, starts the OpenMP pool
    t0 = time.perf_counter()
    O.step(p, phi, 1)
    rate = 2 * w["nx"] * w["ny"] / (time.perf_counter() - t0)
    return int(max(1, min(w["nz"], rate * seconds_per_step // (w["nx"] * w["ny"]))))


def oracle_sample(w, target_s: float = 12.0, steps: int = 3):
    """FP64 oracle rate (cell-updates/s) on a z-slab of the workload sized for
    about target_s seconds of host work over `steps` steps."""
    import oracle as O
    nz = oracle_slab_for(w, target_s / steps)
    p, phi = _oracle_slab(w, nz)
    t0 = time.perf_counter()
    O.step(p, phi, steps)
    dt = time.perf_counter() - t0
    cells = w["nx"] * w["ny"] * nz
    return cells * steps / dt, nz, dt


def cpu_cores():
    return int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    import oracle as O
    w = workload(args)
    # each timed step is one oracle step on a slab sized so that warm-up plus
    # timed steps take about 90 s of host time
    nz_slab = oracle_slab_for(w, 90.0 / max(1, args.steps + args.warmup))
    p, phi = _oracle_slab(w, nz_slab, args.scheme)
    for _ in range(args.warmup):
        phi = O.step(p, phi, 1)
    per_step = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        phi = O.step(p, phi, 1)
        per_step.append(time.perf_counter() - t0)
    cells = w["nx"] * w["ny"] * nz_slab
    tot = sum(per_step)
    value = cells * args.steps / tot
    sample = (f"one FP64 oracle step per timed step on a {w['nx']}x{w['ny']}x{nz_slab} z-slab "
              f"through the grain's centre")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": arm_config(args, w, ws),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cpu_cores(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    emit(line)
    return 0


# --------------------------------------------------------------------- GPU arm


def batched_vs_plain(n_grids: int, dev, rounding=None):
    """Orientation sweep: n_grids uneven grids (edges 32..96, random normals,
    lambda/dx in {2,3,4,6}), FP32 with stochastic rounding of the update,
    27-point TI with each grid's own n.  Times the batched path (one persistent
    launch per step, graph replay) against the plain path (spfm_step per grid
    per step; the same arithmetic, bit for bit) and measures each grid's
    velocity over steps 1000..2000 of the batched run against
    v_th = -M dF/Gamma."""
    import torch
    from paper_1910_05180_gb300 import spfm as S
    from paper_1910_05180_gb300 import workloads as WL
    rounding = S.SPFM_ROUND_STOCHASTIC if rounding is None else rounding
    jobs = WL.orientation_sweep(n_grids=n_grids)
    stream = torch.cuda.Stream(device=dev)
    with torch.cuda.stream(stream):
        grids = []
        for i, j in enumerate(jobs):
            g = S.Grid(j["nx"], j["ny"], j["nz"], dtype=S.SPFM_F32, bc=(S.SPFM_CONTACT,) * 6, n=j["n"],
                       stream=stream)
            g.set_rounding(rounding, seed=i)
            g.init_planar(j["c"], j["lam"])
            grids.append(g)
        args = [S.step_args(lam=j["lam"], dt=j["dt"], dF=j["dF"], stencil=26) for j in jobs]
        cells = sum(j["nx"] * j["ny"] * j["nz"] for j in jobs)
        b = S.Batch(grids, stream=stream)
        b.step(16, args)
        # tile policy and work-list depth chosen by the autotuner (its trial steps are real steps)
        depth, depth_ms = b.autotune(args, steps_per_trial=32)
        tiles = b.tiles()
        for g, a in zip(grids, args):
            g.step(2, lam=a.lam, dt=a.dt, dF=a.dF, stencil=26)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        plain_steps, batch_steps = 10, 320
        torch.cuda.synchronize(dev)
        ev[0].record(stream)
        for _ in range(plain_steps):
            for g, a in zip(grids, args):
                g.step(1, lam=a.lam, dt=a.dt, dF=a.dF, stencil=26)
        ev[1].record(stream)
        ev[2].record(stream)
        b.step(batch_steps, args)
        ev[3].record(stream)
        torch.cuda.synchronize(dev)
        plain = cells * plain_steps / (ev[0].elapsed_time(ev[1]) / 1e3)
        batched = cells * batch_steps / (ev[2].elapsed_time(ev[3]) / 1e3)
        # velocity accuracy on a fresh start: position after 1000 and 2000 steps
        for g, j in zip(grids, jobs):
            g.init_planar(j["c"], j["lam"])
        b.step(1000, args)
        s1 = b.stats()
        b.step(1000, args)
        s2 = b.stats()
        errs = []
        for j, a1, a2 in zip(jobs, s1, s2):
            v = (a2["position"] - a1["position"]) / (1000 * j["dt"])
            errs.append(abs(v / (-j["dF"]) - 1.0))
        errs = np.array(errs)
        b.close()
    return {"workload": f"orientation_sweep_{n_grids}grids_f32_27pt", "cells": int(cells),
            "rounding": "stochastic" if rounding == S.SPFM_ROUND_STOCHASTIC else "nearest",
            "plain_cell_updates_per_s": plain, "batched_cell_updates_per_s": batched,
            "speedup": batched / plain, "velocity_rel_err_median": float(np.median(errs)),
            "velocity_rel_err_p90": float(np.percentile(errs, 90)),
            "velocity_rel_err_max": float(errs.max()),
            "depth": depth, "depth_ms_per_step": {str(k): v for k, v in depth_ms.items()},
            "tile_policy": {0: "wide 64x16", 1: "square 32x32", 2: "fit per grid"}[tiles[0]],
            "note": "batched and plain give bit-identical fields (tests/test_gpu_batch.py)"}


def friction_1d(dev, steps: int = 24000, window: int = 200):
    """Sec. 3.1, Fig. 8: stationary velocity of a planar interface in 1D
    (64 x 1 x 1, no-flux in x, 27-point weights) against v_th = -M dF/Gamma,
    for CF + h3, CF + h5, CF + h_Abel and TI + h3 at lambda~ = 4, 3, 2.5 over a
    range of dF~.  All runs of one model step together as one batch; the frame
    moves back one cell whenever the favoured phase fills half the system
    (spfm_shift_x).  dt = min(0.002 / dF~, dt_max / 2) keeps the interface's
    advance per step at 0.002 cells where stability allows.  The velocity is the
    slope of the fixed-frame position over the last 60 % of the run; the
    oscillation is the spread of the window velocities.  Reduced step counts:
    the paper's runs take 2.5e8 steps at a far finer dt."""
    import torch
    from paper_1910_05180_gb300 import spfm as S
    models = (("CF+h3", S.SPFM_FD), ("CF+h5", S.SPFM_FD_H5), ("CF+h_Abel", S.SPFM_FD_HABEL),
              ("TI+h3", S.SPFM_TI_GLOBAL))
    lams = (4.0, 3.0, 2.5)
    dFs = (0.002, 0.005, 0.01, 0.02, 0.05, 0.1, 0.2, 0.5)
    nx = 64
    bc = (S.SPFM_NOFLUX, S.SPFM_NOFLUX) + (S.SPFM_PERIODIC,) * 4
    out = {}
    stream = torch.cuda.Stream(device=dev)
    with torch.cuda.stream(stream):
        for name, sch in models:
            res = {f"lam{lam:g}": {} for lam in lams}
            grids, args, runs = [], [], []
            for lam in lams:
                for dF in dFs:
                    g = S.Grid(nx, 1, 1, dtype=S.SPFM_F64, bc=bc, n=(1.0, 0.0, 0.0), stream=stream)
                    try:
                        dt = min(0.002 / dF, 0.5 * g.max_dt(lam=lam, dF=dF, stencil=26, scheme=sch))
                    except S.SpfmError as e:
                        res[f"lam{lam:g}"][f"{dF:g}"] = "phase unstable" if e.status == S.SPFM_EPHASE else str(e)
                        g.close()
                        continue
                    g.init_planar((nx - 1) / 2.0, lam)
                    grids.append(g)
                    args.append(S.step_args(lam=lam, dt=dt, dF=dF, stencil=26, scheme=sch))
                    runs.append((lam, dF, dt))
            b = S.Batch(grids, stream=stream)
            offset = np.zeros(len(grids))
            pos = [[] for _ in grids]
            nwin = steps // window
            for w in range(nwin):
                b.step(window, args)
                st = b.stats()
                for i, (g, sti) in enumerate(zip(grids, st)):
                    if w >= int(0.4 * nwin):
                        pos[i].append(((w + 1) * window * runs[i][2], sti["position"] + offset[i]))
                    if 1.0 - sti["volume"] / nx >= 0.5:   # dF > 0 favours phi = 0
                        g.shift_x(-1)
                        offset[i] -= 1
            b.close()
            for i, (lam, dF, dt) in enumerate(runs):
                t, x = np.array(pos[i]).T
                v = np.polyfit(t, x, 1)[0]
                vw = np.diff(x) / np.diff(t)
                vth = -dF
                res[f"lam{lam:g}"][f"{dF:g}"] = {
                    "err_mean": float(abs(v / vth - 1.0)),
                    "err_osc": float((vw.max() - vw.min()) / abs(vth)),
                    "cells_travelled": float(abs(x[-1] - x[0])), "dt": dt}
            for g in grids:
                g.close()
            out[name] = res
    return out


def orientation_paths(n_angles: int = 10, top: float = 81.0):
    """The two rotation paths of Figs. 3 and 10 (reading r22): the normal turns
    away from [100] about the [001] axis, n = (cos t, sin t, 0), and about the
    [011] axis, n = (cos t, sin t / sqrt 2, -sin t / sqrt 2), for t from 0 to
    `top` degrees, plus the [210] normal (26.57 degrees, a <120> member) on the
    first path and [11-1] (54.74 degrees, <111>) on the second."""
    out = []
    grid = list(np.linspace(0.0, top, n_angles))
    for deg in sorted(grid + [float(np.degrees(np.arctan(0.5)))]):
        t = np.radians(deg)
        out.append(("001", float(deg), (float(np.cos(t)), float(np.sin(t)), 0.0)))
    for deg in sorted(grid + [float(np.degrees(np.arctan(np.sqrt(2.0))))]):
        t = np.radians(deg)
        out.append(("011", float(deg), (float(np.cos(t)), float(np.sin(t) / np.sqrt(2.0)),
                                        float(-np.sin(t) / np.sqrt(2.0)))))
    return out


def kinetic_anisotropy(dev, models=None, lams=(4.0, 2.0, 1.0), travel: float = 4.0, window: int = 100):
    """Fig. 10: relative error of the stationary velocity of planar interfaces
    against their orientation on 120 x 10 x 10 (contact faces, Eq. 7), with
    dF = dF0 cos(t), dF0~ = 0.1, so that the x component of the velocity is the
    same for every orientation.  Models: CF, TI_<hkl> for u || [100], [110],
    [111], [120], and TI_n, all with h3.  lambda~ = 0.5 (in the paper's figure)
    is left out: its stable dt for TI_n is 9e-6, some 10^7 steps per run.
    dt = min(0.01, dt_max / 2); the run
    lasts until the interface has moved `travel` cells along x; the velocity is
    the slope of the position over the last 60 % of the run, the oscillation the
    spread of the window velocities."""
    import torch
    from paper_1910_05180_gb300 import spfm as S
    unit = lambda v: tuple(float(x) for x in np.array(v, float) / np.linalg.norm(v))
    if models is None:
        models = [("CF", S.SPFM_FD, (0.0, 0.0, 0.0)), ("TI_<100>", S.SPFM_TI_GLOBAL, unit([1, 0, 0])),
                  ("TI_<110>", S.SPFM_TI_GLOBAL, unit([1, 1, 0])), ("TI_<111>", S.SPFM_TI_GLOBAL, unit([1, 1, 1])),
                  ("TI_<120>", S.SPFM_TI_GLOBAL, unit([1, 2, 0])), ("TI_n", S.SPFM_TI_LOCAL, (0.0, 0.0, 0.0))]
    dF0, shape = 0.1, (120, 10, 10)
    paths = orientation_paths(8, 70.0)
    out = {}
    stream = torch.cuda.Stream(device=dev)
    with torch.cuda.stream(stream):
        for lam in lams:
            for name, sch, u in models:
                grids, args, meta = [], [], []
                for path, deg, n in paths:
                    dF = dF0 * np.cos(np.radians(deg))
                    g = S.Grid(*shape, dtype=S.SPFM_F32, bc=(S.SPFM_CONTACT,) * 6, n=n, u=u, stream=stream)
                    dt = min(0.01, 0.5 * g.max_dt(lam=lam, dF=dF, stencil=26, scheme=sch))
                    g.init_planar(float(np.dot(n, (np.array(shape) - 1) / 2.0)) + 2.5, lam)
                    grids.append(g)
                    args.append(S.step_args(lam=lam, dt=dt, dF=dF, stencil=26, scheme=sch))
                    meta.append((path, deg, dF, dt))
                dt_min = min(m[3] for m in meta)
                steps = int(np.ceil(travel / (dF0 * dt_min) / window)) * window
                pos = [[] for _ in grids]
                nwin = steps // window
                b = S.Batch(grids, stream=stream) if sch != S.SPFM_TI_LOCAL else None
                for w in range(nwin):
                    if b is not None:
                        b.step(window, args)
                        st = b.stats()
                    else:
                        st = []
                        for g, a in zip(grids, args):
                            g.step(window, lam=a.lam, dt=a.dt, dF=a.dF, stencil=26, scheme=sch)
                            st.append(g.stats())
                    if w >= int(0.4 * nwin):
                        for i, sti in enumerate(st):
                            pos[i].append(((w + 1) * window * meta[i][3], sti["position"]))
                if b is not None:
                    b.close()
                rows = []
                for i, (path, deg, dF, dt) in enumerate(meta):
                    t, x = np.array(pos[i]).T
                    v = np.polyfit(t, x, 1)[0]
                    vw = np.diff(x) / np.diff(t)
                    rows.append({"path": path, "deg": round(deg, 2), "err_mean": float(abs(v / (-dF) - 1.0)),
                                 "err_osc": float((vw.max() - vw.min()) / dF)})
                for g in grids:
                    g.close()
                out[f"{name}_lam{lam:g}"] = {"steps": steps, "rows": rows}
    return out


def force_scan_sum(S, n, lam, scheme, shift, u=(0.0, 0.0, 0.0), nx=300):
    """Sum over a 300 x 1 x 1 line of the discrete equilibrium expression E_p of
    Eq. 4 for the ideal profile (Eq. 3) with normal n through x = nx/2 + shift
    (contact faces, Eq. 7, supply the exact profile as every neighbour).  One
    FP64 step at dF = 0 gives R_p = (2M/(3 C_Gamma lambda^2)) E_p; here
    M = 1, C_Gamma = 2/3, so E_p = lambda^2 R_p.  u: the TI_<hkl> coupling
    direction (zero: n)."""
    g = S.Grid(nx, 1, 1, dtype=S.SPFM_F64, bc=(S.SPFM_CONTACT,) * 6, n=n, u=u)
    g.init_planar(n[0] * (nx / 2.0 + shift), lam)
    f0 = g.get_field(to_host=True).double().numpy()
    dt = 0.5 * g.max_dt(lam=lam, stencil=26, scheme=scheme)   # the sum does not depend on dt
    g.step(1, lam=lam, dt=dt, stencil=26, scheme=scheme)
    f1 = g.get_field(to_host=True).double().numpy()
    g.close()
    return float(((f1 - f0) / dt).sum() * lam ** 2)


def force_oscillation(shifts: int = 16):
    """Fig. 3: amplitude A (max - min over sub-grid shifts of the ideal profile)
    of the total grid friction force, the line sum of Eq. 4, against the
    interface orientation (two rotation paths, r22), for CF, TI_<120> and TI_n
    at lambda~ = 1 and 3."""
    from paper_1910_05180_gb300 import spfm as S
    out = {}
    u120 = (1.0 / np.sqrt(5.0), 2.0 / np.sqrt(5.0), 0.0)
    for lam in (1.0, 3.0):
        for name, sch, u in (("CF", S.SPFM_FD, (0.0, 0.0, 0.0)), ("TI_<120>", S.SPFM_TI_GLOBAL, u120),
                             ("TI_n", S.SPFM_TI_LOCAL, (0.0, 0.0, 0.0))):
            rows = []
            for path, deg, n in orientation_paths():
                vals = [force_scan_sum(S, n, lam, sch, m / shifts, u) for m in range(shifts)]
                rows.append({"path": path, "deg": round(deg, 3), "A": max(vals) - min(vals)})
            out[f"{name}_lam{lam:g}"] = rows
    return out


def shape_relaxation(dev):
    """Sec. 3.3: a cubic particle (half side 12) in 60^3, periodic, relaxed at
    constant volume by spfm_step_conserving for a fixed physical time (250),
    then the residual anisotropy eps_eff of its phi = 1/2 contour (Fig. 9b) per
    model and profile width lambda/dx, with the final volume-holding dF."""
    import torch
    from paper_1910_05180_gb300 import spfm as S
    N = 60
    ctr = ((N - 1) / 2.0,) * 3
    u120 = tuple(np.array([1.0, 2.0, 0.0]) / np.sqrt(5.0))
    out = {}
    stream = torch.cuda.Stream(device=dev)
    with torch.cuda.stream(stream):
        for lam, dt in ((4.0, 0.05), (2.0, 0.05), (1.3, 0.015)):
            steps = int(round(250.0 / dt))
            for name, sch in (("TI_n", S.SPFM_TI_LOCAL), ("TI_<120>", S.SPFM_TI_GLOBAL), ("CF", S.SPFM_FD)):
                g = S.Grid(N, N, N, dtype=S.SPFM_F32, bc=(S.SPFM_PERIODIC,) * 6, n=u120, center=ctr,
                           stream=stream)
                g.init_cube(ctr, 12.0, lam)
                v0 = g.stats()["volume"]
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                dF = g.step_conserving(steps, lam=lam, dt=dt, stencil=26, scheme=sch)
                e1.record(stream)
                sp = g.sphericity(0)
                out[f"{name}_lam{lam:g}"] = {
                    "eps_eff": sp["eps_eff"], "R_mean": sp["R_mean"], "dF": dF, "steps": steps, "dt": dt,
                    "volume_rel_drift": abs(g.stats()["volume"] / v0 - 1.0),
                    "ms_per_step": e0.elapsed_time(e1) / steps}
                g.close()
    return out


def bf16_variant(w, dev, steps: int = 100):
    """BF16 storage with FP32 arithmetic: the step rate of the default workload
    (4 B per update) and the acceptance check, the planar velocity error of a
    tilted 96x64x64 job against v_th = -M dF/Gamma next to the same job in FP32
    (accepted when it holds the 1e-4 bar)."""
    import torch
    from paper_1910_05180_gb300 import spfm as S
    stream = torch.cuda.Stream(device=dev)
    out = {}
    with torch.cuda.stream(stream):
        g = S.Grid(w["nx"], w["ny"], w["nz"], dtype=S.SPFM_BF16, bc=(S.SPFM_PERIODIC,) * 6, n=w["u"],
                   center=w["ctr"], stream=stream)
        g.init_sphere(w["ctr"], w["R"], w["lam"], w["dx"])
        kw = dict(lam=w["lam"], dx=w["dx"], dt=w["dt"], dF=w["dF"], stencil=26, scheme=S.SPFM_TI_GLOBAL)
        g.step(5, **kw)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(dev)
        e0.record(stream)
        g.step(steps, **kw)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1) / steps
        cells = w["nx"] * w["ny"] * w["nz"]
        peak, _ = measured_hbm_peak()
        out["cell_updates_per_s"] = cells / (ms / 1e3)
        out["ms_per_step"] = ms
        out["frac_hbm"] = cells * 4 / (ms / 1e3) / 1e9 / peak
        g.close()
        n = (1.0 / 3 ** 0.5,) * 3
        shape = (96, 64, 64)
        c = float(np.dot(n, (np.array(shape) - 1) / 2.0))
        for name, dt_, rnd in (("f32", S.SPFM_F32, S.SPFM_ROUND_NEAREST), ("bf16", S.SPFM_BF16, S.SPFM_ROUND_NEAREST),
                               ("f32_sr", S.SPFM_F32, S.SPFM_ROUND_STOCHASTIC),
                               ("bf16_sr", S.SPFM_BF16, S.SPFM_ROUND_STOCHASTIC)):
            h = S.Grid(*shape, dtype=dt_, bc=(S.SPFM_CONTACT,) * 6, n=n, stream=stream)
            h.set_rounding(rnd, seed=3)
            h.init_planar(c, 3.0)
            a = dict(lam=3.0, dt=0.05, dF=0.05, stencil=26, scheme=S.SPFM_TI_GLOBAL)
            h.step(1000, **a)
            p1 = h.stats()["position"]
            h.step(1000, **a)
            p2 = h.stats()["position"]
            v = (p2 - p1) / (1000 * 0.05)
            out[f"planar_velocity_rel_err_{name}"] = abs(v / -0.05 - 1.0)
            h.close()
    out["accepted"] = bool(out["planar_velocity_rel_err_bf16"] <= 1e-4)
    out["accepted_with_stochastic_rounding"] = bool(out["planar_velocity_rel_err_bf16_sr"] <= 1e-4)
    out["workload"] = w["name"] + "_ti120_bf16_27pt"
    return out


def tilted_256(dev, steps: int = 50, window: int = 400):
    """The 256^3 tilted-plane configuration (normal (1,1,1)/sqrt3 through the
    centre, contact faces, 27-point, lambda = 3 of its {2, 3, 4}) in FP32 and
    FP64 storage, TI_<111> and CF + h3: step rate over `steps` steps, fraction of
    the HBM roofline (8 or 16 B per update), and the velocity error against
    v_th = -M dF/Gamma between steps 200 and 200 + window (the first-order time
    discretisation error included: the GPU-vs-oracle velocity bar is a test)."""
    import torch
    from paper_1910_05180_gb300 import spfm as S
    from paper_1910_05180_gb300 import workloads as WL
    w = WL.tilted_111_256cubed()[1]
    peak, _ = measured_hbm_peak()
    cells = w["nx"] * w["ny"] * w["nz"]
    stream = torch.cuda.Stream(device=dev)
    out = {}
    with torch.cuda.stream(stream):
        for dname, dt_, bpu in (("f32", S.SPFM_F32, 8), ("f64", S.SPFM_F64, 16)):
            for sname, sch in (("TI_<111>", S.SPFM_TI_GLOBAL), ("CF+h3", S.SPFM_FD)):
                g = S.Grid(w["nx"], w["ny"], w["nz"], dtype=dt_, bc=(S.SPFM_CONTACT,) * 6, n=w["n"],
                           stream=stream)
                g.init_planar(w["c"], w["lam"], w["dx"])
                kw = dict(lam=w["lam"], dx=w["dx"], dt=w["dt"], dF=w["dF"], stencil=26, scheme=sch)
                g.step(5, **kw)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                torch.cuda.synchronize(dev)
                e0.record(stream)
                g.step(steps, **kw)
                e1.record(stream)
                torch.cuda.synchronize(dev)
                ms = e0.elapsed_time(e1) / steps
                g.step(200 - 5 - steps, **kw)
                p1 = g.stats()["position"]
                g.step(window, **kw)
                p2 = g.stats()["position"]
                v = (p2 - p1) / (window * w["dt"])
                out[f"{sname}_{dname}"] = {"cell_updates_per_s": cells / (ms / 1e3), "ms_per_step": ms,
                                           "frac_hbm": cells * bpu / (ms / 1e3) / 1e9 / peak,
                                           "zchunk": g.last_zchunk(),
                                           "velocity_rel_err_vs_v_th": abs(v / (-w["dF"]) - 1.0)}
                g.close()
    out["workload"] = w["name"] + "_contact_27pt"
    return out


def velocity_vs_oracle(dev, n_grids: int = 4, steps: int = 2000, window: int = 1000):
    """GPU against FP64-oracle velocities on the same jobs: the 32^3 grids of
    the orientation sweep with the smallest dF (the hardest case for FP32),
    batched, with round-to-nearest and with stochastic rounding of the update;
    velocity over the last `window` of `steps` steps.  Errors are relative to
    v_th = -M dF/Gamma (Sec. 2.1), next to the oracle's own error against it."""
    import torch
    import oracle as O
    from paper_1910_05180_gb300 import spfm as S
    from paper_1910_05180_gb300 import workloads as WL
    jobs = sorted([j for j in WL.orientation_sweep() if j["nx"] == 32], key=lambda j: j["dF"])[:n_grids]
    rows = []
    res = {}
    stream = torch.cuda.Stream(device=dev)
    for mode, rounding in (("nearest", S.SPFM_ROUND_NEAREST), ("stochastic", S.SPFM_ROUND_STOCHASTIC)):
        with torch.cuda.stream(stream):
            grids = []
            for i, j in enumerate(jobs):
                g = S.Grid(j["nx"], j["ny"], j["nz"], dtype=S.SPFM_F32, bc=(S.SPFM_CONTACT,) * 6, n=j["n"],
                           stream=stream)
                g.set_rounding(rounding, seed=i)
                g.init_planar(j["c"], j["lam"])
                grids.append(g)
            args = [S.step_args(lam=j["lam"], dt=j["dt"], dF=j["dF"], stencil=26) for j in jobs]
            b = S.Batch(grids, stream=stream)
            b.step(steps - window, args)
            s1 = b.stats()
            b.step(window, args)
            s2 = b.stats()
            res[mode] = [(a2["position"] - a1["position"]) / (window * j["dt"]) for j, a1, a2 in zip(jobs, s1, s2)]
            b.close()
            for g in grids:
                g.close()
    for i, j in enumerate(jobs):
        p = O.Params(j["nx"], j["ny"], j["nz"], bc=(O.CONTACT,) * 6, n=j["n"], lam=j["lam"], dt=j["dt"],
                     dF=j["dF"], stencil=26)
        phi = O.step(p, O.init_planar(p, j["c"]), steps - window)
        c1 = O.stats(p, phi)["position"]
        phi = O.step(p, phi, window)
        vo = (O.stats(p, phi)["position"] - c1) / (window * j["dt"])
        v_th = -j["dF"]
        rows.append({"grid": j["name"], "edge": j["nx"], "lam": j["lam"], "dF": j["dF"],
                     "oracle_vs_vth": abs(vo / v_th - 1.0),
                     "nearest_vs_oracle": abs(res["nearest"][i] - vo) / abs(v_th),
                     "stochastic_vs_oracle": abs(res["stochastic"][i] - vo) / abs(v_th)})
    return {"workload": f"orientation_sweep_32cubed_smallest_dF_{steps}steps_f32_27pt", "rows": rows}


def rounding_cost(w, dev, steps: int = 100):
    """Step time of the default workload with stochastic rounding of the update
    against round to nearest (the same grid and steps)."""
    import torch
    from paper_1910_05180_gb300 import spfm as S
    stream = torch.cuda.Stream(device=dev)
    out = {}
    cells = w["nx"] * w["ny"] * w["nz"]
    with torch.cuda.stream(stream):
        g = S.Grid(w["nx"], w["ny"], w["nz"], dtype=S.SPFM_F32, bc=(S.SPFM_PERIODIC,) * 6, n=w["u"],
                   center=w["ctr"], stream=stream)
        kw = dict(lam=w["lam"], dx=w["dx"], dt=w["dt"], dF=w["dF"], stencil=26, scheme=S.SPFM_TI_GLOBAL)
        for mode, rounding in (("nearest", S.SPFM_ROUND_NEAREST), ("stochastic", S.SPFM_ROUND_STOCHASTIC)):
            g.set_rounding(rounding, seed=1)
            g.init_sphere(w["ctr"], w["R"], w["lam"], w["dx"])
            g.step(5, **kw)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize(dev)
            e0.record(stream)
            g.step(steps, **kw)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            ms = e0.elapsed_time(e1) / steps
            out[mode] = {"ms_per_step": ms, "cell_updates_per_s": cells / (ms / 1e3)}
        g.close()
    out["cost"] = out["stochastic"]["ms_per_step"] / out["nearest"]["ms_per_step"] - 1.0
    out["workload"] = w["name"] + "_ti120_f32_27pt"
    return out


def serving_run(n_jobs: int, n_plain: int = 200):
    """Poisson stream (200 jobs/s) of velocity-measurement jobs, edges 32..192,
    FP32 with stochastic rounding, continuous batching under a 120 GB budget,
    retirement at |dv/v| < 1e-4.  Then the first n_plain jobs of the same
    stream twice: served, and through the one-launch-per-job path (the same
    windows and retirement, each job stepped and measured on its own); their
    rates give served / plain."""
    from paper_1910_05180_gb300 import workloads as WL
    from paper_1910_05180_gb300.serve import GpuBackend, PlainGpuBackend, Server, job_from_workload
    jobs = [job_from_workload(w) for w in WL.serving_stream(n_jobs=n_jobs)]
    srv = Server(GpuBackend(), hbm_budget=120e9, window=200, tol=1e-4, max_steps=20000)
    out = srv.run(jobs)
    out["workload"] = f"poisson200hz_{n_jobs}jobs_edge32-192_f32_sr_27pt"
    if n_plain:
        sub = jobs[:n_plain]
        a = Server(GpuBackend(), hbm_budget=120e9, window=200, tol=1e-4, max_steps=20000).run(sub)
        b_srv = Server(PlainGpuBackend(), hbm_budget=120e9, window=200, tol=1e-4, max_steps=20000)
        b = b_srv.run(sub)
        keep = ("wall_s", "cell_updates", "cell_updates_per_s", "latency_p50_s", "latency_p99_s", "converged")
        out["vs_plain"] = {"jobs": n_plain, "served": {k: a[k] for k in keep}, "plain": {k: b[k] for k in keep},
                           "speedup": a["cell_updates_per_s"] / b["cell_updates_per_s"]}
    return out



def run_gpu(args):
    import torch
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local if ws > 1 else 0)
    torch.cuda.set_device(dev)
    from paper_1910_05180_gb300 import spfm as S

    w = workload(args)
    dtype = {"f32": S.SPFM_F32, "f64": S.SPFM_F64, "bf16": S.SPFM_BF16}[args.dtype]
    scheme = {"ti120": S.SPFM_TI_GLOBAL, "fd": S.SPFM_FD, "local": S.SPFM_TI_LOCAL}[args.scheme]
    stream = torch.cuda.Stream(device=dev)
    with torch.cuda.stream(stream):
        g = S.Grid(w["nx"], w["ny"], w["nz"], dtype=dtype, bc=(S.SPFM_PERIODIC,) * 6, n=w["u"],
                   center=w["ctr"], stream=stream)
        if args.rounding == "stochastic":
            g.set_rounding(S.SPFM_ROUND_STOCHASTIC, seed=1)
        g.init_sphere(w["ctr"], w["R"], w["lam"], w["dx"])
    kw = dict(M=w["M"], Gamma=w["Gamma"], lam=w["lam"], dx=w["dx"], dt=w["dt"], dF=w["dF"],
              stencil=w["stencil"], scheme=scheme)
    cells = w["nx"] * w["ny"] * w["nz"]

    def barrier():
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize(dev)

    every = stats_cadence(args.steps)
    clocks = ClockSampler(dev.index if dev.index is not None else 0)
    clocks.start()
    for i in range(args.warmup):
        g.step(1, **kw)
        if (i + 1) % every == 0:
            g.stats()
    barrier()
    clocks.wait_live()
    # steps run in chunks of `every` (one spfm_step call each, so consecutive
    # kernels overlap under programmatic dependent launch); the FP64 stats run
    # after every full chunk, inside the timed region but outside the chunk events
    chunks = []
    left = args.steps
    while left > 0:
        chunks.append(min(every, left))
        left -= chunks[-1]
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in chunks]
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    launches = 0
    per_step = g.kernels_per_step()
    stats_seen = []
    host_t0 = time.time()
    t_start.record(stream)
    for (e0, e1), n in zip(ev, chunks):
        e0.record(stream)
        g.step(n, **kw)
        e1.record(stream)
        launches += per_step * n   # stencil kernel (+ ghost-face kernel unless it writes the images)
        if n == every:
            stats_seen.append(g.stats())
            launches += 2          # stats kernel + its final reduction
    t_end.record(stream)
    barrier()
    clocks.mark(host_t0, time.time())
    clk = clocks.stop()
    total_ms = max_over_ranks(t_start.elapsed_time(t_end), ws, dev)
    step_ms = sum(a.elapsed_time(b) for a, b in ev)
    value = replica_value(cells, args.steps, ws, total_ms)
    avg_kernel_ms = step_ms / args.steps
    bpu = BYTES_PER_UPDATE[args.dtype]
    peak, peak_kind = measured_hbm_peak()
    achieved = cells * bpu / (avg_kernel_ms / 1e3) / 1e9
    kernel_key = f"spfm_step_kernel_{args.dtype}_27pt_{args.scheme}_{w['nx']}"
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": args.dtype, "data": "synthetic",
        "config": arm_config(args, w, ws),
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "peak_kind": peak_kind,
                     "frac_of_nominal": achieved / NOMINAL_HBM_GBS,
                     "traffic": profiled_traffic(kernel_key),
                     "kernel": "spfm_step_kernel", "bytes_per_update": bpu,
                     "avg_launch_ms": avg_kernel_ms,
                     "timed": ("stencil kernel, which writes the periodic ghost images itself"
                               if per_step == 1 else "stencil kernel + ghost-face kernel")
                              + f"; events around {every}-step chunks"},
        "clocks": clk, "gpu_launches": launches,
        # no stats call ran when the timed region had no full chunk
        "stats_call": ({"ms": (total_ms - step_ms) / len(stats_seen), "calls": len(stats_seen),
                        "every": every, "note": "interface stats between step chunks, host round trip "
                                                "included"} if stats_seen else None),
        "legs": [],
    }

    def leg(name, result):
        """One study leg as a line of its own, printed as soon as it is done."""
        if result is not None and rank == 0:
            emit({"leg": name, **(result if isinstance(result, dict) else {"result": result})})
            line["legs"].append(name)

    if rank == 0:
        leg("last_stats", stats_seen[-1] if stats_seen else None)
        # grain anisotropy after the timed run (Sec. 3.3), FP64 on the device
        leg("grain_sphericity", g.sphericity(0))

    # the other schemes on the same grid and storage (short timed runs)
    if rank == 0 and not args.no_variants:
        variants = {}
        for name, sch in (("TI_n", S.SPFM_TI_LOCAL), ("CF+h3", S.SPFM_FD), ("TI_<120>", S.SPFM_TI_GLOBAL)):
            if sch == scheme:
                continue
            kw2 = dict(kw, scheme=sch)
            g.init_sphere(w["ctr"], w["R"], w["lam"], w["dx"])
            g.step(5, **kw2)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            nvar = 100
            barrier()
            e0.record(stream)
            g.step(nvar, **kw2)
            e1.record(stream)
            barrier()
            ms = e0.elapsed_time(e1) / nvar
            variants[name] = {"cell_updates_per_s": cells / (ms / 1e3), "ms_per_step": ms,
                              "frac_hbm": cells * bpu / (ms / 1e3) / 1e9 / peak}
            if sch == S.SPFM_TI_LOCAL:
                # TI_n is bound by instruction issue: its ceiling is the issue rate of
                # the GPU (SMs x 4 schedulers x the maximum SM clock, one warp
                # instruction each per cycle) over the warp instructions per cell
                # update of the committed capture
                wipc = profiled_record(f"spfm_step_kernel_{args.dtype}_27pt_local", "warp_inst_per_cell")
                ceil = issue_ceiling(dev, wipc) if wipc else None
                variants[name]["bound"] = "alu"
                variants[name]["warp_inst_per_cell"] = wipc
                variants[name]["issue_ceiling_cell_updates_per_s"] = ceil
                variants[name]["frac_alu"] = cells / (ms / 1e3) / ceil if ceil else None
        leg("variants", variants)

    if rank == 0 and not args.no_variants and args.dtype == "f32":
        leg("stochastic_rounding_cost", rounding_cost(w, dev))
    if rank == 0 and not args.no_bf16 and args.dtype != "bf16":
        leg("bf16_storage", bf16_variant(w, dev))
    if rank == 0 and not args.no_tilted:
        leg("tilted_256", tilted_256(dev))
    if rank == 0 and not args.no_relax:
        leg("shape_relaxation", shape_relaxation(dev))
    if rank == 0 and not args.no_friction:
        leg("friction_1d", friction_1d(dev))
    if rank == 0 and not args.no_force_scan:
        leg("force_oscillation", force_oscillation())
    if rank == 0 and not args.no_kinetic:
        leg("kinetic_anisotropy", kinetic_anisotropy(dev))

    # end to end through the public API from pinned host memory: upload the
    # initial field, E2E_STEPS steps, stats, read the field back
    e2e = None
    if not args.no_e2e:
        E2E_STEPS = 50
        host_in = g.get_field(to_host=True)
        host_out = torch.empty_like(host_in).pin_memory()
        iters = 5
        barrier()
        call_ms = []
        for _ in range(iters):
            t0 = torch.cuda.Event(enable_timing=True)
            t1 = torch.cuda.Event(enable_timing=True)
            t0.record(stream)
            S.spfm_set_field(g.handle, host_in.data_ptr(), 1)
            g.step(E2E_STEPS, **kw)
            g.stats()
            S.spfm_get_field(g.handle, host_out.data_ptr(), 1)
            t1.record(stream)
            t1.synchronize()
            call_ms.append(t0.elapsed_time(t1))
        barrier()
        # the median call: one disturbed call (a busy host) does not set the figure
        e_ms = max_over_ranks(float(np.median(call_ms)), ws, dev)
        fb = host_in.numel() * host_in.element_size()
        e2e = {"value": replica_value(cells, E2E_STEPS, ws, e_ms), "unit": UNIT,
               "h2d_bytes_per_step": fb / E2E_STEPS, "d2h_bytes_per_step": (fb + 96) / E2E_STEPS,
               "note": f"per call: host field in, {E2E_STEPS} steps, stats, host field out; median of {iters} calls",
               "call_ms": [round(x, 3) for x in call_ms]}
    line["e2e"] = e2e

    if rank == 0 and not args.no_batch:
        leg("batched", batched_vs_plain(args.sweep_grids, dev))
    if rank == 0 and not args.no_serve:
        leg("serving", serving_run(args.serve_jobs))
    if rank == 0 and not args.no_batch:
        leg("velocity_vs_oracle", velocity_vs_oracle(dev))

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        v, nzs, dt = oracle_sample(w)
        cpu = {"value": v, "unit": UNIT, "cores": cpu_cores(), "kind": "oracle",
               "sample": f"3 FP64 oracle steps on a {w['nx']}x{w['ny']}x{nzs} z-slab of the "
                         f"workload ({dt:.1f} s)"}
    line["cpu_baseline"] = cpu
    if rank == 0:
        emit(headline(line))
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def batch_only(n_grids: int):
    """The batched orientation sweep alone at the default work-list depth: 32
    warm-up steps, then 64 timed steps; prints one JSON line."""
    import torch
    from paper_1910_05180_gb300 import spfm as S
    from paper_1910_05180_gb300 import workloads as WL
    jobs = WL.orientation_sweep(n_grids=n_grids)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        grids = []
        for j in jobs:
            g = S.Grid(j["nx"], j["ny"], j["nz"], dtype=S.SPFM_F32, bc=(S.SPFM_CONTACT,) * 6, n=j["n"],
                       stream=stream)
            g.init_planar(j["c"], j["lam"])
            grids.append(g)
        args = [S.step_args(lam=j["lam"], dt=j["dt"], dF=j["dF"], stencil=26) for j in jobs]
        cells = sum(j["nx"] * j["ny"] * j["nz"] for j in jobs)
        b = S.Batch(grids, stream=stream)
        b.step(32, args)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        b.step(64, args)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / 64
        b.close()
    emit({"workload": f"orientation_sweep_{n_grids}grids_f32_27pt", "cells": cells,
          "ms_per_step": ms, "cell_updates_per_s": cells / (ms / 1e3)})
    return 0


def tilted_only(args):
    """The 256^3 tilted plane (n || [111], contact faces, lambda = 3) alone in
    FP32 storage with the TI_<111> step: 5 warm-up steps, then 50 timed; prints
    one JSON line."""
    import torch
    from paper_1910_05180_gb300 import spfm as S
    from paper_1910_05180_gb300 import workloads as WL
    w = WL.tilted_111_256cubed()[1]
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        g = S.Grid(w["nx"], w["ny"], w["nz"], dtype=S.SPFM_F32, bc=(S.SPFM_CONTACT,) * 6, n=w["n"], stream=stream)
        if args.rounding == "stochastic":
            g.set_rounding(S.SPFM_ROUND_STOCHASTIC, seed=1)
        g.init_planar(w["c"], w["lam"], w["dx"])
        kw = dict(lam=w["lam"], dx=w["dx"], dt=w["dt"], dF=w["dF"], stencil=26)
        g.step(5, **kw)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        g.step(50, **kw)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / 50
    cells = w["nx"] * w["ny"] * w["nz"]
    peak, _ = measured_hbm_peak()
    emit({"workload": w["name"] + "_contact_ti111_f32_27pt", "ms_per_step": ms,
          "cell_updates_per_s": cells / (ms / 1e3), "frac_hbm": cells * 8 / (ms / 1e3) / 1e9 / peak,
          "kernels_per_step": g.kernels_per_step()})
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.tilted_only:
        return tilted_only(args)
    if args.batch_only:
        return batch_only(args.sweep_grids)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
