"""Seeded synthetic workloads shaped like the paper's studies.

Only sizes, orientations and parameter draws live here (no phase-field
arithmetic): both the CUDA path and the FP64 oracle build their own initial
fields from these recipes.  Seeds: numpy.random.default_rng(seed) with the
seed equal to the workload's index (0-4).
"""
from __future__ import annotations

import numpy as np


def unit(v):
    v = np.asarray(v, dtype=np.float64)
    return v / np.linalg.norm(v)


def random_normal(rng) -> np.ndarray:
    """Uniform direction on the unit sphere (normalised Gaussian)."""
    return unit(rng.normal(size=3))


def planar_100_128x32x32():
    """Planar (1,0,0) interface at x = 40 on 128x32x32, 7-point, FP64,
    lambda = 4, M = Gamma = dx = 1, dt = 0.1, dF = 0.05, no-flux in x,
    periodic in y/z, 1000 steps."""
    return dict(name="planar100_128x32x32_fp64_7pt", nx=128, ny=32, nz=32, n=(1.0, 0.0, 0.0),
                c=40.0, lam=4.0, dx=1.0, M=1.0, Gamma=1.0, dt=0.1, dF=0.05, stencil=6,
                bc=("noflux", "noflux", "periodic", "periodic", "periodic", "periodic"), steps=1000)


def tilted_111_256cubed(seed: int = 1):
    """Tilted planar interface, normal (1,1,1)/sqrt3 through the box centre on
    256^3, 27-point, lambda in {2,3,4}, dF ~ U[0.001, 0.1] (one per lambda),
    dt = 0.05, 5000 steps, contact-angle BCs on all faces."""
    rng = np.random.default_rng(seed)
    dFs = rng.uniform(0.001, 0.1, size=3)
    n = tuple(unit([1, 1, 1]))
    N = 256
    return [dict(name=f"tilted111_256cubed_lam{lam:g}", nx=N, ny=N, nz=N, n=n,
                 c=float(np.dot(n, [(N - 1) / 2.0] * 3)), lam=float(lam), dx=1.0, M=1.0,
                 Gamma=1.0, dt=0.05, dF=float(dF), stencil=26, bc=("contact",) * 6, steps=5000)
            for lam, dF in zip((2.0, 3.0, 4.0), dFs)]


def orientation_sweep(seed: int = 2, n_grids: int = 256):
    """Batched orientation sweep: edges from {32,48,64,96}, normals uniform on
    the sphere, lambda/dx from {2,3,4,6}, dF ~ U[1e-4, 0.1], 27-point, dt = 0.05,
    contact-angle BCs, each plane through its box centre."""
    rng = np.random.default_rng(seed)
    jobs = []
    for i in range(n_grids):
        N = int(rng.choice([32, 48, 64, 96]))
        n = random_normal(rng)
        lam = float(rng.choice([2.0, 3.0, 4.0, 6.0]))
        dF = float(rng.uniform(1e-4, 0.1))
        jobs.append(dict(name=f"sweep{i}", nx=N, ny=N, nz=N, n=tuple(n),
                         c=float(np.dot(n, [(N - 1) / 2.0] * 3)), lam=lam, dx=1.0, M=1.0,
                         Gamma=1.0, dt=0.05, dF=dF, stencil=26, bc=("contact",) * 6))
    return jobs


def serving_stream(seed: int = 3, n_jobs: int = 2000, rate_hz: float = 200.0):
    """Poisson arrivals of velocity-measurement requests: edge U{32..192 step 16},
    normal on the sphere, lambda/dx U{2..6}, dF log-uniform [1e-4, 1e-1]."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate_hz, size=n_jobs))
    jobs = []
    for i in range(n_jobs):
        N = int(rng.choice(np.arange(32, 193, 16)))
        n = random_normal(rng)
        lam = float(rng.choice([2.0, 3.0, 4.0, 5.0, 6.0]))
        dF = float(np.exp(rng.uniform(np.log(1e-4), np.log(1e-1))))
        jobs.append(dict(name=f"job{i}", arrival=float(t[i]), nx=N, ny=N, nz=N, n=tuple(n),
                         c=float(np.dot(n, [(N - 1) / 2.0] * 3)), lam=lam, dx=1.0, M=1.0,
                         Gamma=1.0, dt=0.05, dF=dF, stencil=26, bc=("contact",) * 6))
    return jobs


def sphere_512cubed():
    """Spherical grain (phi = 0 inside) of radius 150 at the centre of 512^3,
    lambda = 3, 27-point, dF = 0.02, periodic, dt = 0.05, 10000 steps; the
    128^3 replica has R = 37.5 and dF = 0.08 (same R/R*)."""
    N = 512
    return dict(name="sphere_512cubed_R150", nx=N, ny=N, nz=N, ctr=((N - 1) / 2.0,) * 3, R=150.0,
                lam=3.0, dx=1.0, M=1.0, Gamma=1.0, dt=0.05, dF=0.02, stencil=26,
                bc=("periodic",) * 6, steps=10000, u=tuple(unit([1, 2, 0])))


def sphere_replica_128cubed():
    N = 128
    return dict(name="sphere_128cubed_R37.5", nx=N, ny=N, nz=N, ctr=((N - 1) / 2.0,) * 3, R=37.5,
                lam=3.0, dx=1.0, M=1.0, Gamma=1.0, dt=0.05, dF=0.08, stencil=26,
                bc=("periodic",) * 6, steps=10000, u=tuple(unit([1, 2, 0])))


BC_CODE = {"periodic": 0, "noflux": 1, "contact": 2}


def bc_codes(w):
    return tuple(BC_CODE[b] for b in w["bc"])
