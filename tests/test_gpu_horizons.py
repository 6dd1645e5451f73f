"""GPU against the FP64 oracle at the workloads' own step counts.

Each workload's field and interface velocity are compared after the step
count the workload states, on a replica small enough for the oracle where the
full size is out of its reach:

- tilted plane (n || [111], contact faces, 27-point, lambda in {2, 3, 4} with
  the seeded dF, dt = 0.05): the full 5000 steps on a 48^3 replica, FP64 and
  FP32 storage, TI_<111> and CF + h3;
- orientation sweep: seven of its grids (the smallest dF values and two large
  ones) over the full 2000 steps, stepped as one batch;
- serving stream: six of its jobs (edges 32 and 80, dF from 1e-4 to 2e-2),
  served together; each job's final window velocity against an oracle run of
  the same job over the same steps.

The sweep and the stream run FP32 with stochastic rounding of the update
(SPFM_ROUND_STOCHASTIC); round to nearest is recorded beside it: it drops the
sub-ulp increments of slow interfaces near phi = 1 and misses the velocity
bar below dF ~ 5e-4.

Field bars: max|phi_gpu - phi_oracle| <= 1e-12 (FP64), 2e-5 (FP32).  Velocity
bar: |v_gpu - v_oracle| <= 1e-4 |v_th| with v_th = -M dF/Gamma (Sec. 2.1); for
SPFM v_oracle equals v_th to the time-discretisation error, and for a pinned
CF interface (v_oracle ~ 0) the theoretical speed keeps the scale meaningful.
The 128^3 grain replica is in test_gpu_replica.py.

Set SPFM_RECORD=<file> to append each measured error as a JSON line.
"""
import functools
import json
import os

import numpy as np
import pytest
import torch

import oracle as O
from paper_1910_05180_gb300 import spfm as S
from paper_1910_05180_gb300 import workloads as WL
from paper_1910_05180_gb300.serve import GpuBackend, Job, Server, job_from_workload

pytestmark = pytest.mark.gpu

FIELD_TOL = {S.SPFM_F64: 1e-12, S.SPFM_F32: 2e-5}
VEL_TOL = 1e-4
DNAME = {S.SPFM_F64: "f64", S.SPFM_F32: "f32"}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    S.load()


def record(**kw):
    path = os.environ.get("SPFM_RECORD")
    if path:
        with open(path, "a") as f:
            f.write(json.dumps(kw) + "\n")


def vel_err(v, vo, v_th):
    return abs(v - vo) / abs(v_th)


# ------------------------------------------------------------ tilted plane

C2_EDGE = 48
C2_SCHEMES = {"TI": (S.SPFM_TI_GLOBAL, O.TI_GLOBAL), "CF": (S.SPFM_FD, O.CF)}


def _c2(lam):
    w = next(x for x in WL.tilted_111_256cubed() if x["lam"] == lam)
    N = C2_EDGE
    return dict(w, nx=N, ny=N, nz=N, c=float(np.dot(w["n"], [(N - 1) / 2.0] * 3)))


@functools.lru_cache(maxsize=None)
def _c2_oracle(lam, scheme):
    """Oracle run of the 48^3 replica: positions at 4000 and 5000 steps, final field."""
    w = _c2(lam)
    p = O.Params(w["nx"], w["ny"], w["nz"], bc=(O.CONTACT,) * 6, n=w["n"], lam=lam, dt=w["dt"],
                 dF=w["dF"], stencil=26, scheme=C2_SCHEMES[scheme][1])
    phi = O.step(p, O.init_planar(p, w["c"]), w["steps"] - 1000)
    c1 = O.stats(p, phi)["position"]
    phi = O.step(p, phi, 1000)
    c2 = O.stats(p, phi)["position"]
    return phi, c1, c2


@pytest.mark.parametrize("scheme", ["TI", "CF"])
@pytest.mark.parametrize("lam", [2.0, 3.0, 4.0])
@pytest.mark.parametrize("dtype", [S.SPFM_F64, S.SPFM_F32])
def test_tilted_plane_replica_5000_steps(dtype, lam, scheme):
    w = _c2(lam)
    g = S.Grid(w["nx"], w["ny"], w["nz"], dtype=dtype, bc=(S.SPFM_CONTACT,) * 6, n=w["n"])
    g.init_planar(w["c"], lam, w["dx"])
    kw = dict(lam=lam, dx=w["dx"], dt=w["dt"], dF=w["dF"], stencil=26, scheme=C2_SCHEMES[scheme][0])
    g.step(w["steps"] - 1000, **kw)
    c1 = g.stats()["position"]
    g.step(1000, **kw)
    c2 = g.stats()["position"]
    phi_o, c1o, c2o = _c2_oracle(lam, scheme)
    err = float(np.abs(g.get_field(to_host=True).double().numpy() - phi_o).max())
    T = 1000 * w["dt"]
    v, vo, v_th = (c2 - c1) / T, (c2o - c1o) / T, -w["dF"]
    ve = vel_err(v, vo, v_th)
    record(workload="tilted111", edge=C2_EDGE, lam=lam, scheme=scheme, dtype=DNAME[dtype],
           steps=w["steps"], field_err=err, vel_err_vs_oracle=ve, vel_err_vs_vth=abs(v / v_th - 1))
    g.close()
    assert err <= FIELD_TOL[dtype], err
    assert ve <= VEL_TOL, (v, vo, v_th)


# ------------------------------------------------------- orientation sweep


def _sweep_pick():
    jobs = WL.orientation_sweep()
    by_dF = sorted(range(len(jobs)), key=lambda i: jobs[i]["dF"])
    small = [i for i in by_dF if jobs[i]["nx"] <= 64][:4] + [by_dF[0]]   # by_dF[0] is a 96^3 grid
    large = [i for i in by_dF[::-1] if jobs[i]["nx"] == 32][:2]
    return [jobs[i] for i in sorted(set(small + large))]


def _sweep_batched(jobs, rounding):
    grids = []
    for i, j in enumerate(jobs):
        g = S.Grid(j["nx"], j["ny"], j["nz"], dtype=S.SPFM_F32, bc=(S.SPFM_CONTACT,) * 6, n=j["n"])
        g.set_rounding(rounding, seed=i)
        g.init_planar(j["c"], j["lam"])
        grids.append(g)
    args = [S.step_args(lam=j["lam"], dt=j["dt"], dF=j["dF"], stencil=26) for j in jobs]
    b = S.Batch(grids)
    b.step(1000, args)
    s1 = b.stats()
    b.step(1000, args)
    s2 = b.stats()
    out = [(g.get_field(to_host=True).double().numpy(), a1["position"], a2["position"])
           for g, a1, a2 in zip(grids, s1, s2)]
    b.close()
    for g in grids:
        g.close()
    return out


def test_sweep_grids_batched_2000_steps():
    """FP32 with stochastic rounding meets both bars on every picked grid;
    round to nearest is measured beside it (recorded, not asserted: it misses
    the velocity bar at dF ~ 3e-4)."""
    jobs = _sweep_pick()
    runs = {"SR": _sweep_batched(jobs, S.SPFM_ROUND_STOCHASTIC), "RN": _sweep_batched(jobs, S.SPFM_ROUND_NEAREST)}
    fails = []
    for i, j in enumerate(jobs):
        p = O.Params(j["nx"], j["ny"], j["nz"], bc=(O.CONTACT,) * 6, n=j["n"], lam=j["lam"], dt=j["dt"],
                     dF=j["dF"], stencil=26)
        phi = O.step(p, O.init_planar(p, j["c"]), 1000)
        c1o = O.stats(p, phi)["position"]
        phi = O.step(p, phi, 1000)
        c2o = O.stats(p, phi)["position"]
        T = 1000 * j["dt"]
        vo, v_th = (c2o - c1o) / T, -j["dF"]
        for mode, res in runs.items():
            field, c1, c2 = res[i]
            err = float(np.abs(field - phi).max())
            v = (c2 - c1) / T
            ve = vel_err(v, vo, v_th)
            record(workload="orientation_sweep", grid=j["name"], edge=j["nx"], lam=j["lam"], dF=j["dF"],
                   dtype="f32", rounding=mode, steps=2000, field_err=err, vel_err_vs_oracle=ve,
                   vel_err_vs_vth=abs(v / v_th - 1))
            if mode == "SR" and (err > FIELD_TOL[S.SPFM_F32] or ve > VEL_TOL):
                fails.append((j["name"], j["nx"], j["dF"], err, ve))
    assert not fails, fails


# ----------------------------------------------------------- serving stream

SERVE_PICK = ("job753", "job1235", "job314", "job261", "job369", "job136")


def test_served_jobs_match_oracle_velocity():
    """Served with stochastic rounding (the server's default), every job's
    final window velocity is the oracle's within the bar; a round-to-nearest
    server is measured beside it (recorded, not asserted)."""
    ws = {w["name"]: w for w in WL.serving_stream(n_jobs=2000)}
    jobs = [Job(**{**job_from_workload(ws[name]).__dict__, "arrival": 0.0}) for name in SERVE_PICK]
    fails = []
    oracle_cache = {}
    for mode, rounding in (("SR", S.SPFM_ROUND_STOCHASTIC), ("RN", S.SPFM_ROUND_NEAREST)):
        srv = Server(GpuBackend(rounding=rounding), hbm_budget=120e9, window=200, tol=1e-4, max_steps=20000)
        srv.run(jobs)
        for r in srv.results:
            j = next(x for x in jobs if x.name == r.name)
            key = (j.name, r.steps)
            if key not in oracle_cache:
                p = O.Params(j.nx, j.ny, j.nz, bc=(O.CONTACT,) * 6, n=j.n, lam=j.lam, dt=j.dt, dF=j.dF,
                             stencil=26)
                phi = O.step(p, O.init_planar(p, j.c), r.steps - 200)
                c1o = O.stats(p, phi)["position"]
                phi = O.step(p, phi, 200)
                c2o = O.stats(p, phi)["position"]
                oracle_cache[key] = (c2o - c1o) / (200 * j.dt)
            vo = oracle_cache[key]
            v_th = -j.M * j.dF / j.Gamma
            ve = vel_err(r.velocity, vo, v_th)
            record(workload="serving_stream", job=r.name, edge=j.nx, lam=j.lam, dF=j.dF, dtype="f32",
                   rounding=mode, steps=r.steps, converged=r.converged, vel_err_vs_oracle=ve,
                   vel_err_vs_vth=abs(r.velocity / v_th - 1), oracle_vel_err_vs_vth=abs(vo / v_th - 1))
            if mode == "SR" and (not r.converged or ve > VEL_TOL):
                fails.append((r.name, j.dF, r.steps, r.converged, ve))
    assert not fails, fails
