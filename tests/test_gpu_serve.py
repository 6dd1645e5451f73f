"""Serving on the GPU: continuous batching of velocity-measurement jobs, and
the same result for a job alone and in a mix."""
import numpy as np
import pytest
import torch

from paper_1910_05180_gb300 import spfm as S
from paper_1910_05180_gb300 import workloads as WL
from paper_1910_05180_gb300.serve import GpuBackend, Job, Server, job_from_workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    S.load()


def _small_stream(k=8):
    jobs = []
    for w in WL.serving_stream(n_jobs=k):
        w = dict(w)
        w["nx"] = w["ny"] = w["nz"] = min(w["nx"], 64)
        w["c"] = float(np.dot(w["n"], [(w["nx"] - 1) / 2.0] * 3))
        w["arrival"] *= 0.1
        jobs.append(job_from_workload(w))
    return jobs


def test_serving_mix_matches_the_oracle_velocity():
    """Every job of a served mix converges, and its final window velocity is
    the FP64 oracle's for the same job and window within 1e-4 of v_th."""
    import oracle as O
    jobs = _small_stream(8)
    srv = Server(GpuBackend(), hbm_budget=120e9, window=200, tol=1e-4, max_steps=4000)
    out = srv.run(jobs)
    assert out["jobs"] == 8
    assert out["converged"] == 8
    for r in srv.results:
        j = next(x for x in jobs if x.name == r.name)
        p = O.Params(j.nx, j.ny, j.nz, bc=(O.CONTACT,) * 6, n=j.n, lam=j.lam, dt=j.dt, dF=j.dF, stencil=26)
        phi = O.step(p, O.init_planar(p, j.c), r.steps - 200)
        c1 = O.stats(p, phi)["position"]
        c2 = O.stats(p, O.step(p, phi, 200))["position"]
        vo = (c2 - c1) / (200 * j.dt)
        assert abs(r.velocity - vo) <= 1e-4 * abs(r.v_theory), (r.name, r.velocity, vo)
    assert out["latency_p99_s"] >= out["latency_p50_s"] > 0


def test_job_result_same_alone_and_in_a_mix():
    jobs = _small_stream(6)
    target = jobs[3]
    mix = Server(GpuBackend(), hbm_budget=120e9, window=200, max_steps=4000)
    mix.run(jobs)
    alone = Server(GpuBackend(), hbm_budget=120e9, window=200, max_steps=4000)
    alone.run([Job(**{**target.__dict__, "arrival": 0.0})])
    a = next(r for r in mix.results if r.name == target.name)
    b = alone.results[0]
    assert a.steps == b.steps
    assert a.velocity == b.velocity       # bit-identical arithmetic per job


def test_plain_path_gives_the_served_results():
    """The one-launch-per-job backend (the baseline of the serving leg) runs
    the same arithmetic: every job retires after the same steps with the same
    velocity as in the continuous batch."""
    from paper_1910_05180_gb300.serve import PlainGpuBackend
    jobs = _small_stream(5)
    served = Server(GpuBackend(), hbm_budget=120e9, window=200, max_steps=4000)
    served.run(jobs)
    plain = Server(PlainGpuBackend(), hbm_budget=120e9, window=200, max_steps=4000)
    plain.run(jobs)
    a = {r.name: r for r in served.results}
    for r in plain.results:
        assert r.steps == a[r.name].steps
        # fields are bit-identical; the positions come from the batched and the
        # single-grid stats reductions, which sum in different orders
        assert abs(r.velocity - a[r.name].velocity) <= 1e-13
