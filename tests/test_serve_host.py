"""Scheduling logic of the continuous-batching server, on CPU with a stand-in
backend and a simulated clock (no GPU)."""
import math

import pytest

from paper_1910_05180_gb300.serve import Job, Server


class FakeClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t

    def sleep(self, dt):
        self.t += max(dt, 1e-3)


class FakeBackend:
    """Interfaces that move at v_th after a one-window transient; stepping costs
    simulated time proportional to the cells in the batch."""

    def __init__(self, clock, cost_per_cell_step=1e-11):
        self.clock = clock
        self.cost = cost_per_cell_step
        self.live = {}
        self.batches = []

    def bytes_for(self, job):
        return job.nx * job.ny * job.nz * 8

    def create(self, job):
        h = object()
        self.live[h] = {"job": job, "c": job.c, "steps": 0}
        return h

    def release(self, h):
        del self.live[h]

    def step(self, entries, n):
        self.batches.append(len(entries))
        cells = 0
        for a in entries:
            st = self.live[a.handle]
            j = st["job"]
            v = -j.M * j.dF / j.Gamma
            if st["steps"] == 0:
                v *= 0.9           # transient in the first window
            st["c"] += v * n * j.dt
            st["steps"] += n
            cells += j.nx * j.ny * j.nz
        self.clock.t += self.cost * cells * n

    def positions(self, entries):
        return [self.live[a.handle]["c"] for a in entries]


def _jobs(k, edge=32, dt_arrival=0.001):
    return [Job(name=f"j{i}", arrival=i * dt_arrival, nx=edge, ny=edge, nz=edge, n=(1.0, 0.0, 0.0),
                c=10.0, lam=3.0, dF=0.01 * (1 + i % 5)) for i in range(k)]


def test_all_jobs_finish_converged_with_exact_velocity():
    clock = FakeClock()
    be = FakeBackend(clock)
    srv = Server(be, hbm_budget=1e9, window=200, tol=1e-4, clock=clock, sleep=clock.sleep)
    out = srv.run(_jobs(20))
    assert out["jobs"] == 20 and out["converged"] == 20
    for r in srv.results:
        assert r.steps == 600      # transient window, then two equal windows
        assert math.isclose(r.velocity, r.v_theory, rel_tol=1e-12)
        assert r.latency > 0
    assert out["latency_p99_s"] >= out["latency_p50_s"]


def test_admission_respects_the_memory_budget_and_order():
    clock = FakeClock()
    be = FakeBackend(clock)
    per_job = 32 ** 3 * 8
    srv = Server(be, hbm_budget=3.5 * per_job, window=200, clock=clock, sleep=clock.sleep)
    srv.run(_jobs(10, dt_arrival=0.0))     # all queued at once: the budget binds
    assert srv.peak_used <= 3.5 * per_job
    assert max(be.batches) == 3            # never more than three resident jobs
    admitted = [r.admitted for r in sorted(srv.results, key=lambda r: r.arrival)]
    assert admitted == sorted(admitted)    # FIFO admission
    assert srv.used == 0


def test_jobs_that_arrive_later_join_a_running_batch():
    clock = FakeClock()
    be = FakeBackend(clock, cost_per_cell_step=1e-9)
    srv = Server(be, hbm_budget=1e12, window=200, clock=clock, sleep=clock.sleep)
    jobs = _jobs(6, dt_arrival=0.002)
    srv.run(jobs)
    assert max(be.batches) > 1             # continuous batching: jobs overlap on the device


def test_job_above_the_whole_budget_is_rejected():
    clock = FakeClock()
    srv = Server(FakeBackend(clock), hbm_budget=100.0, clock=clock, sleep=clock.sleep)
    with pytest.raises(ValueError):
        srv.run(_jobs(1))


def test_unconverged_jobs_stop_at_the_step_cap():
    class Noisy(FakeBackend):
        def positions(self, entries):
            return [self.live[a.handle]["c"] + (1e-3 if self.live[a.handle]["steps"] % 400 else 0.0)
                    for a in entries]

    clock = FakeClock()
    srv = Server(Noisy(clock), hbm_budget=1e9, window=200, max_steps=2000, clock=clock, sleep=clock.sleep)
    out = srv.run(_jobs(2))
    assert out["converged"] == 0 and all(r.steps == 2000 for r in srv.results)
