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


def test_serving_mix_converges_to_v_theory():
    jobs = _small_stream(8)
    srv = Server(GpuBackend(), hbm_budget=120e9, window=200, tol=1e-4, max_steps=4000)
    out = srv.run(jobs)
    assert out["jobs"] == 8
    assert out["converged"] == 8
    for r in srv.results:
        assert r.rel_error < 5e-4, (r.name, r.rel_error)
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
