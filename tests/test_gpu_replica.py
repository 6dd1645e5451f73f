"""The 128^3 replica of the grain workload (Sec. 3.3 setting, downscaled):
R = 37.5, lambda = 3, dF = 0.08 (the same R/R* as R = 150 at dF = 0.02),
periodic, 27-point, dt = 0.05.  FP32 on the GPU against the FP64 oracle on the
same start: the field within 2e-5 and the radial velocity dR/dt of the radius
estimator (Sec. 2.3 inversion, radial form) within 1e-4 relative.

Horizons: the workload's full 10000 steps for both schemes (velocity over the
last 1000); the TI_n oracle runs at about a third of the TI_<120> rate, some
five minutes of host time.

Set SPFM_RECORD=<file> to append the measured errors as a JSON line.
"""
import json
import os

import numpy as np
import pytest
import torch

import oracle as O
from paper_1910_05180_gb300 import spfm as S
from paper_1910_05180_gb300 import workloads as WL

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    S.load()


@pytest.mark.parametrize("scheme,oscheme,n1,n2", [(S.SPFM_TI_GLOBAL, O.TI_GLOBAL, 9000, 1000),
                                                  (S.SPFM_TI_LOCAL, O.TI_LOCAL, 9000, 1000)])
def test_grain_replica_field_and_velocity(scheme, oscheme, n1, n2):
    w = WL.sphere_replica_128cubed()
    N, ctr, R = w["nx"], w["ctr"], w["R"]
    kw = dict(lam=w["lam"], dx=w["dx"], dt=w["dt"], dF=w["dF"], stencil=26, scheme=scheme)
    g = S.Grid(N, N, N, dtype=S.SPFM_F32, bc=(S.SPFM_PERIODIC,) * 6, n=w["u"], center=ctr)
    p = O.Params(N, N, N, bc=(O.PERIODIC,) * 6, n=tuple(w["u"]), lam=w["lam"], dx=w["dx"], dt=w["dt"],
                 dF=w["dF"], stencil=26, scheme=oscheme)
    phi0 = O.init_sphere(p, ctr, R)
    g.set_field(torch.from_numpy(phi0).float().cuda())
    start = g.get_field(to_host=True).double().numpy()   # the FP32 values the GPU starts from

    g.step(n1, **kw)
    r1 = g.stats()["radius"]
    phi = O.step(p, start, n1)
    r1o = O.stats(p, phi, ctr)["radius"]
    g.step(n2, **kw)
    r2 = g.stats()["radius"]
    phi = O.step(p, phi, n2)
    r2o = O.stats(p, phi, ctr)["radius"]

    err = float(np.abs(g.get_field(to_host=True).double().numpy() - phi).max())
    T = n2 * w["dt"]
    v, vo = (r2 - r1) / T, (r2o - r1o) / T
    path = os.environ.get("SPFM_RECORD")
    if path:
        with open(path, "a") as f:
            f.write(json.dumps({"workload": "sphere_replica_128", "scheme": "TI_n" if oscheme == O.TI_LOCAL
                                else "TI_<120>", "dtype": "f32", "steps": n1 + n2, "field_err": err,
                                "vel_err_vs_oracle": abs(v / vo - 1.0), "radius": r2}) + "\n")
    assert err <= 2e-5, err
    assert vo > 0.0                       # the grain grows: dF beats the curvature term
    assert abs(v / vo - 1.0) < 1e-4, (v, vo)
