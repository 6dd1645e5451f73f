"""Continuous-batching server for interface-velocity measurement jobs.

A job is one grid with a planar ideal profile (normal n through the box
centre, lambda, dF) whose steady interface velocity is wanted.  The server
  - admits arrived jobs in arrival order while their device memory (two field
    buffers and the scratch) fits into the HBM budget and a slot is free;
  - keeps every admitted job's field resident on the device and advances all
    of them together, window by window (one batch of `window` steps);
  - after each window measures each job's interface position (FP64 inversion
    of the ideal profile, Sec. 2.3), its velocity over the window, and retires
    the job once two consecutive window velocities agree within `tol`
    (relative), or after `max_steps` (reported as not converged);
  - re-forms the batch whenever jobs join or leave, so requests that arrive
    while others run share the device with them.
A job's arithmetic does not depend on the other jobs in the batch, so its
result is the same alone and in any mix.

The backend (`GpuBackend`, or a stand-in in tests) owns grids and batches; the
scheduling logic here is plain Python.
"""
from __future__ import annotations

import math
import time
import zlib
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Job:
    name: str
    arrival: float                 # seconds after the start of the run
    nx: int
    ny: int
    nz: int
    n: tuple
    c: float
    lam: float
    dF: float
    dx: float = 1.0
    M: float = 1.0
    Gamma: float = 1.0
    dt: float = 0.05
    stencil: int = 26


@dataclass
class Result:
    name: str
    arrival: float
    admitted: float
    finished: float
    steps: int
    velocity: float
    v_theory: float
    converged: bool
    cells: int

    @property
    def latency(self) -> float:
        return self.finished - self.arrival

    @property
    def rel_error(self) -> float:
        return abs(self.velocity / self.v_theory - 1.0) if self.v_theory else float("nan")


@dataclass
class _Active:
    job: Job
    handle: object
    admitted: float
    steps: int = 0
    c_prev: float = float("nan")
    v_prev: float = float("nan")
    v: float = float("nan")


def job_from_workload(w: dict) -> Job:
    return Job(name=w["name"], arrival=w.get("arrival", 0.0), nx=w["nx"], ny=w["ny"], nz=w["nz"],
               n=tuple(w["n"]), c=w["c"], lam=w["lam"], dF=w["dF"], dx=w.get("dx", 1.0),
               M=w.get("M", 1.0), Gamma=w.get("Gamma", 1.0), dt=w.get("dt", 0.05),
               stencil=w.get("stencil", 26))


def job_seed(job: Job) -> int:
    """Seed of a job's stochastic rounding: a hash of its name, so that its
    random bits (and its result) do not depend on the other jobs."""
    return zlib.crc32(job.name.encode())


class GpuBackend:
    """Grids and batches of the CUDA library: FP32 storage with stochastic
    rounding of the update by default (round to nearest drops the sub-ulp
    increments of slow interfaces near phi = 1 and biases their velocity)."""

    def __init__(self, dtype=None, stream=None, rounding=None):
        import torch

        from . import spfm as S
        self.S = S
        self.torch = torch
        self.dtype = S.SPFM_F32 if dtype is None else dtype
        self.rounding = S.SPFM_ROUND_STOCHASTIC if rounding is None else rounding
        if self.dtype == S.SPFM_F64:
            self.rounding = S.SPFM_ROUND_NEAREST
        self.stream = stream if stream is not None else torch.cuda.Stream()
        self._batch = None
        self._members = ()

    def bytes_for(self, job: Job) -> int:
        d = self.S.GridDesc()
        d.nx, d.ny, d.nz, d.dtype = job.nx, job.ny, job.nz, self.dtype
        _, _, fb, sb = self.S.spfm_layout(d)
        return 2 * fb + sb

    def create(self, job: Job):
        S = self.S
        with self.torch.cuda.stream(self.stream):
            g = S.Grid(job.nx, job.ny, job.nz, dtype=self.dtype, bc=(S.SPFM_CONTACT,) * 6, n=job.n,
                       stream=self.stream)
            g.set_rounding(self.rounding, job_seed(job))
            g.init_planar(job.c, job.lam, job.dx)
        return g

    def release(self, handle):
        if self._batch is not None:       # the batch refers to the grid: drop it first
            self._batch.close()
            self._batch = None
            self._members = ()
        handle.close()

    def step(self, entries, n_steps: int):
        S = self.S
        handles = tuple(a.handle for a in entries)
        if self._batch is None or handles != self._members:
            if self._batch is not None:
                self._batch.close()
            self._batch = S.Batch(list(handles), stream=self.stream)
            self._members = handles
        args = [S.step_args(M=a.job.M, Gamma=a.job.Gamma, lam=a.job.lam, dx=a.job.dx, dt=a.job.dt,
                            dF=a.job.dF, stencil=a.job.stencil) for a in entries]
        self._batch.step(n_steps, args)

    def positions(self, entries):
        return [s["position"] for s in self._batch.stats()]


class PlainGpuBackend(GpuBackend):
    """The one-launch-per-job path, for comparison: the same grids, rounding
    and windows, but each job is stepped by its own spfm_step launches and
    measured by its own stats call (no batch, no graph)."""

    def release(self, handle):
        handle.close()

    def step(self, entries, n_steps: int):
        for a in entries:
            j = a.job
            a.handle.step(n_steps, M=j.M, Gamma=j.Gamma, lam=j.lam, dx=j.dx, dt=j.dt, dF=j.dF,
                          stencil=j.stencil)

    def positions(self, entries):
        return [a.handle.stats()["position"] for a in entries]


class Server:
    def __init__(self, backend, hbm_budget: float = 120e9, window: int = 200, tol: float = 1e-4,
                 max_steps: int = 20000, max_slots: int = 1024, clock=time.perf_counter,
                 sleep=time.sleep):
        self.backend = backend
        self.budget = float(hbm_budget)
        self.window = int(window)
        self.tol = float(tol)
        self.max_steps = int(max_steps)
        self.max_slots = int(max_slots)
        self.clock = clock
        self.sleep = sleep
        self.used = 0.0
        self.peak_used = 0.0
        self.active: list[_Active] = []
        self.results: list[Result] = []
        self.cell_updates = 0
        self.windows = 0

    def _admit(self, pending: list, now: float):
        while pending and pending[0].arrival <= now and len(self.active) < self.max_slots:
            job = pending[0]
            need = self.backend.bytes_for(job)
            if need > self.budget:
                raise ValueError(f"job {job.name} needs {need} bytes, above the whole budget")
            if self.used + need > self.budget:
                break                      # wait for memory to free up (FIFO, no overtaking)
            pending.pop(0)
            handle = self.backend.create(job)
            self.used += need
            self.peak_used = max(self.peak_used, self.used)
            self.active.append(_Active(job=job, handle=handle, admitted=now))

    def _retire(self, entry: _Active, now: float, converged: bool):
        job = entry.job
        self.backend.release(entry.handle)
        self.used -= self.backend.bytes_for(job)
        self.results.append(Result(name=job.name, arrival=job.arrival, admitted=entry.admitted,
                                   finished=now, steps=entry.steps, velocity=entry.v,
                                   v_theory=-job.M * job.dF / job.Gamma, converged=converged,
                                   cells=job.nx * job.ny * job.nz))

    def run(self, jobs) -> dict:
        pending = sorted(jobs, key=lambda j: j.arrival)
        t0 = self.clock()
        while pending or self.active:
            now = self.clock() - t0
            self._admit(pending, now)
            if not self.active:
                if pending:
                    self.sleep(max(0.0, min(pending[0].arrival - now, 0.05)))
                continue
            entries = list(self.active)
            self.backend.step(entries, self.window)
            positions = self.backend.positions(entries)
            self.windows += 1
            now = self.clock() - t0
            done = []
            for a, c in zip(entries, positions):
                a.steps += self.window
                self.cell_updates += self.window * a.job.nx * a.job.ny * a.job.nz
                if not math.isnan(a.c_prev):
                    a.v_prev, a.v = a.v, (c - a.c_prev) / (self.window * a.job.dt)
                a.c_prev = c
                conv = (not math.isnan(a.v_prev) and not math.isnan(a.v) and a.v != 0.0
                        and abs(a.v - a.v_prev) <= self.tol * abs(a.v))
                if conv or a.steps >= self.max_steps:
                    done.append((a, conv))
            for a, conv in done:
                self.active.remove(a)
                self._retire(a, now, conv)
        wall = self.clock() - t0
        return self.summary(wall)

    def summary(self, wall: float) -> dict:
        lat = np.array([r.latency for r in self.results]) if self.results else np.zeros(1)
        errs = np.array([r.rel_error for r in self.results if r.converged]) if self.results else np.zeros(1)
        return {
            "jobs": len(self.results),
            "converged": int(sum(r.converged for r in self.results)),
            "wall_s": wall,
            "cell_updates": int(self.cell_updates),
            "cell_updates_per_s": self.cell_updates / wall if wall > 0 else float("nan"),
            "latency_p50_s": float(np.percentile(lat, 50)),
            "latency_p99_s": float(np.percentile(lat, 99)),
            "max_rel_velocity_error": float(errs.max()) if errs.size else float("nan"),
            "windows": self.windows,
            "peak_hbm_bytes": self.peak_used,
        }
