"""GPU parity: the CUDA path, called through the C ABI, against the FP64 oracle.

Bars: FP64 max |phi_gpu - phi_oracle| <= 1e-12, FP32 <= 2e-5, interface velocity
within 1e-4 relative.  Sizes span several tiles with ragged tails; the
full-size cases compare sampled cells against oracle runs on their dependency
cones.
"""
import math

import numpy as np
import pytest
import torch

import oracle as O
from paper_1910_05180_gb300 import spfm as S
from paper_1910_05180_gb300 import workloads as WL

pytestmark = pytest.mark.gpu

TOL = {S.SPFM_F64: 1e-12, S.SPFM_F32: 2e-5}
SCHEME_O = {S.SPFM_TI_GLOBAL: O.TI_GLOBAL, S.SPFM_FD: O.CF, S.SPFM_TI_LOCAL: O.TI_LOCAL,
            S.SPFM_FD_H5: O.CF_H5, S.SPFM_FD_HABEL: O.CF_HABEL}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    S.load()


def make_pair(nx, ny, nz, dtype, bc, n, lam, dx=1.0, M=1.0, Gamma=1.0, dt=0.05, dF=0.0,
              stencil=26, scheme=S.SPFM_TI_GLOBAL, gamma=(0, 0, 0), C_gamma=0.0):
    g = S.Grid(nx, ny, nz, dtype=dtype, bc=bc, n=n, gamma=gamma, C_gamma=C_gamma)
    p = O.Params(nx, ny, nz, bc=bc, n=tuple(n), lam=lam, dx=dx, M=M, Gamma=Gamma, dt=dt, dF=dF,
                 stencil=stencil, scheme=SCHEME_O[scheme], gamma=gamma, C_gamma=C_gamma)
    return g, p


def upload(g, phi64, dtype):
    t = torch.from_numpy(phi64).to(S.TORCH_DTYPE[dtype])
    g.set_field(t.cuda())
    return t.double().numpy()     # the values the GPU actually starts from


def gpu_field(g):
    return g.get_field(to_host=True).double().numpy()


def rng_normal(seed):
    return WL.random_normal(np.random.default_rng(seed))


# ------------------------------------------------------------------ init


@pytest.mark.parametrize("dtype", [S.SPFM_F64, S.SPFM_F32])
def test_init_planar_and_sphere(dtype):
    n = rng_normal(1)
    g, p = make_pair(45, 23, 9, dtype, (S.SPFM_CONTACT,) * 6, n, lam=2.5, dx=0.7)
    g.init_planar(7.1, 2.5, 0.7)
    ref = O.init_planar(p, 7.1)
    tol = 2e-15 if dtype == S.SPFM_F64 else 6e-8   # CUDA and libm tanh differ by a few ulps
    assert np.abs(gpu_field(g) - ref).max() <= tol
    ctr = (14.2, 8.1, 3.3)
    g.init_sphere(ctr, 6.0, 2.5, 0.7)
    ref = O.init_sphere(p, ctr, 6.0)
    assert np.abs(gpu_field(g) - ref).max() <= tol


# ------------------------------------------------------------ step parity

CASES = [
    # (shape, bc, stencil, scheme)
    ((37, 21, 19), (S.SPFM_CONTACT,) * 6, 26, S.SPFM_TI_GLOBAL),
    ((37, 21, 19), (S.SPFM_CONTACT,) * 6, 18, S.SPFM_TI_GLOBAL),
    ((37, 21, 19), (S.SPFM_CONTACT,) * 6, 6, S.SPFM_TI_GLOBAL),
    ((70, 18, 35), (S.SPFM_PERIODIC,) * 6, 26, S.SPFM_TI_GLOBAL),
    ((67, 33, 17), (S.SPFM_NOFLUX, S.SPFM_NOFLUX, S.SPFM_PERIODIC, S.SPFM_PERIODIC,
                    S.SPFM_CONTACT, S.SPFM_CONTACT), 26, S.SPFM_FD),
    ((37, 21, 19), (S.SPFM_CONTACT,) * 6, 6, S.SPFM_FD),
    ((5, 3, 2), (S.SPFM_CONTACT,) * 6, 26, S.SPFM_TI_GLOBAL),
    ((1, 1, 40), (S.SPFM_PERIODIC,) * 4 + (S.SPFM_NOFLUX,) * 2, 26, S.SPFM_TI_GLOBAL),
    # degenerate and tile-crossing extents
    ((1, 1, 1), (S.SPFM_PERIODIC,) * 6, 26, S.SPFM_TI_GLOBAL),
    ((3, 1, 1), (S.SPFM_CONTACT,) * 6, 26, S.SPFM_FD),
    ((1, 50, 1), (S.SPFM_NOFLUX,) * 6, 18, S.SPFM_TI_GLOBAL),
    ((130, 2, 3), (S.SPFM_PERIODIC,) * 2 + (S.SPFM_CONTACT,) * 4, 26, S.SPFM_TI_LOCAL),
    ((65, 17, 33), (S.SPFM_CONTACT,) * 6, 26, S.SPFM_FD_HABEL),
    ((64, 16, 32), (S.SPFM_CONTACT,) * 6, 26, S.SPFM_FD_H5),
    # all faces periodic with rows of whole 32-byte sectors (nx a multiple of 8
    # FP32 / 4 FP64 cells): the step writes its own ghost images
    ((64, 18, 35), (S.SPFM_PERIODIC,) * 6, 26, S.SPFM_TI_GLOBAL),
    ((8, 1, 1), (S.SPFM_PERIODIC,) * 6, 26, S.SPFM_FD),
    ((136, 3, 1), (S.SPFM_PERIODIC,) * 6, 18, S.SPFM_TI_LOCAL),
    ((4, 5, 6), (S.SPFM_PERIODIC,) * 6, 26, S.SPFM_TI_GLOBAL),   # images in FP64 only
    ((16, 1, 7), (S.SPFM_PERIODIC,) * 6, 6, S.SPFM_FD_H5),
    # no periodic face: the step computes the contact and no-flux ghosts as it
    # reads them (x ghosts inside a chunk, one-row and one-plane grids, TI_n)
    ((45, 23, 21), (S.SPFM_CONTACT,) * 6, 26, S.SPFM_TI_LOCAL),
    ((6, 2, 2), (S.SPFM_NOFLUX, S.SPFM_CONTACT, S.SPFM_CONTACT, S.SPFM_NOFLUX, S.SPFM_CONTACT, S.SPFM_CONTACT),
     26, S.SPFM_TI_GLOBAL),
    ((33, 17, 1), (S.SPFM_CONTACT,) * 6, 18, S.SPFM_FD),
    ((70, 1, 3), (S.SPFM_CONTACT,) * 4 + (S.SPFM_NOFLUX,) * 2, 26, S.SPFM_TI_GLOBAL),
]


@pytest.mark.parametrize("dtype", [S.SPFM_F64, S.SPFM_F32])
@pytest.mark.parametrize("case", range(len(CASES)))
def test_step_parity_small(dtype, case):
    shape, bc, stencil, scheme = CASES[case]
    nx, ny, nz = shape
    n = rng_normal(10 + case)
    if nx == 1 and ny == 1:
        n = np.array([0.0, 0.0, 1.0])
    lam = 2.0 + 0.5 * (case % 3)
    g, p = make_pair(nx, ny, nz, dtype, bc, n, lam=lam, dt=0.05, dF=0.03, stencil=stencil,
                     scheme=scheme)
    rng = np.random.default_rng(100 + case)
    c = float(n @ (np.array(shape) - 1) / 2.0)
    phi0 = O.init_planar(p, c) + 0.01 * rng.random(p.shape)   # not an exact solution
    start = upload(g, phi0, dtype)
    steps = 40
    g.step(steps, M=1.0, Gamma=1.0, lam=lam, dx=1.0, dt=0.05, dF=0.03, stencil=stencil,
           scheme=scheme)
    ref = O.step(p, start, steps)
    err = np.abs(gpu_field(g) - ref).max()
    assert err <= TOL[dtype], err


def test_step_count_and_ping_pong_agree():
    """n single steps and one n-step call give identical fields."""
    n = rng_normal(3)
    g1, _ = make_pair(40, 20, 12, S.SPFM_F32, (S.SPFM_CONTACT,) * 6, n, lam=3.0)
    g2, _ = make_pair(40, 20, 12, S.SPFM_F32, (S.SPFM_CONTACT,) * 6, n, lam=3.0)
    for g in (g1, g2):
        g.init_planar(float(n @ [20, 10, 6]), 3.0)
    g1.step(7, lam=3.0, dt=0.05, dF=0.02)
    for _ in range(7):
        g2.step(1, lam=3.0, dt=0.05, dF=0.02)
    assert torch.equal(g1.get_field(), g2.get_field())


# ------------------------------------------------ periodic ghost images


@pytest.mark.parametrize("dtype", [S.SPFM_F64, S.SPFM_F32, S.SPFM_BF16])
@pytest.mark.parametrize("shape", [(32, 1, 1), (48, 5, 1), (144, 33, 3), (20, 3, 2)])
def test_periodic_ghost_layer_is_the_exact_wrap(dtype, shape):
    """All faces periodic: after every step the ghost layer (edges and corners
    included) holds the periodic wrap of the interior, value for value, both
    where the step kernel writes the images itself (nx a whole number of
    32-byte sectors) and where the face kernel does (nx = 20 in FP32 / BF16)."""
    nx, ny, nz = shape
    n = rng_normal(41)
    g, p = make_pair(nx, ny, nz, dtype, (S.SPFM_PERIODIC,) * 6, n, lam=2.5)
    rng = np.random.default_rng(42)
    phi0 = O.init_planar(p, float(n @ (np.array(shape) - 1) / 2.0)) + 0.01 * rng.random(p.shape)
    upload(g, phi0, dtype)
    for steps in (1, 2, 5):
        g.step(steps, lam=2.5, dt=0.05, dF=0.03, stencil=26)
        full = g.current_with_ghosts().double().cpu().numpy()
        assert np.array_equal(full, np.pad(full[1:-1, 1:-1, 1:-1], 1, mode="wrap"))


def _ghosted_reference(phi, bc, n, lam, dx, dtype):
    """The ghost layer the face rule gives, built in numpy in the storage
    precision: periodic wrap, no-flux copy of the face cell, contact shift
    (1 - a) v / (1 - a (2 v - 1)) with a = tanh(2 s dx n_axis / lambda) (s = -1
    on the low face), every operation rounded on its own, axes x, y, z in turn."""
    ft = np.float32 if dtype == S.SPFM_F32 else np.float64
    nz, ny, nx = phi.shape
    sizes = (nx, ny, nz)
    idx, hit = [], []
    for ax, N in enumerate(sizes):
        c = np.arange(-1, N + 1)
        src = np.clip(c, 0, N - 1)
        face = np.full(c.shape, -1)
        if bc[2 * ax] == S.SPFM_PERIODIC:
            src = c % N
        else:
            if bc[2 * ax] == S.SPFM_CONTACT:
                face[0] = 2 * ax
            if bc[2 * ax + 1] == S.SPFM_CONTACT:
                face[-1] = 2 * ax + 1
        idx.append(src)
        hit.append(face)
    v = phi.astype(ft)[np.ix_(idx[2], idx[1], idx[0])]
    # the host library's libm tanh, as the C library computes the couplings
    a = [ft(math.tanh(2.0 * (-1.0 if f % 2 == 0 else 1.0) * dx * float(n[f // 2]) / lam)) for f in range(6)]
    one, two = ft(1), ft(2)
    for ax in range(3):
        shape = [1, 1, 1]
        shape[2 - ax] = sizes[ax] + 2
        fh = hit[ax].reshape(shape)
        for f in (2 * ax, 2 * ax + 1):
            m = np.broadcast_to(fh == f, v.shape)
            if not m.any():
                continue
            x = v[m]
            d = one - a[f] * (two * x - one)
            v[m] = ((one - a[f]) * x) / d
    return v


@pytest.mark.parametrize("dtype", [S.SPFM_F64, S.SPFM_F32])
@pytest.mark.parametrize("shape,bc", [
    ((48, 5, 3), (S.SPFM_CONTACT,) * 6),
    ((64, 2, 1), (S.SPFM_NOFLUX, S.SPFM_CONTACT, S.SPFM_PERIODIC, S.SPFM_PERIODIC, S.SPFM_CONTACT, S.SPFM_NOFLUX)),
    ((136, 33, 4), (S.SPFM_PERIODIC, S.SPFM_PERIODIC, S.SPFM_CONTACT, S.SPFM_CONTACT, S.SPFM_NOFLUX, S.SPFM_NOFLUX)),
    ((20, 6, 5), (S.SPFM_CONTACT,) * 6),
    ((48, 7, 3), (S.SPFM_PERIODIC,) * 6),    # the step kernel's images
])
def test_ghost_layer_matches_the_face_rule_exactly(dtype, shape, bc):
    """After every step the whole ghost layer (faces, edges, corners) holds the
    face rule applied to the interior, bit for bit: periodic, no-flux and
    contact faces in every combination (the face kernel), and all-periodic
    rows of whole 32-byte sectors (the step kernel's images).  A grid with no
    periodic face keeps no ghost layer in memory between steps (the step
    computes those ghosts as it reads them); an energy stats call, which reads
    the ghosts, refreshes it first."""
    nx, ny, nz = shape
    n = rng_normal(43)
    lam = 2.5
    g, p = make_pair(nx, ny, nz, dtype, bc, n, lam=lam)
    rng = np.random.default_rng(44)
    phi0 = O.init_planar(p, float(n @ (np.array(shape) - 1) / 2.0)) + 0.01 * rng.random(p.shape)
    upload(g, phi0, dtype)
    inline = S.SPFM_PERIODIC not in bc
    if inline:
        assert g.kernels_per_step() == 1
    for steps in (1, 2, 5):
        g.step(steps, lam=lam, dt=0.05, dF=0.03, stencil=26)
        if inline:
            g.stats(S.SPFM_STATS_ENERGY)
        full = g.current_with_ghosts().double().cpu().numpy()
        want = _ghosted_reference(full[1:-1, 1:-1, 1:-1], bc, n, lam, 1.0, dtype).astype(np.float64)
        bad = np.argwhere(full != want)
        assert bad.size == 0, (len(bad), bad[:4].tolist(), np.abs(full - want).max())


def test_periodic_image_steps_around_conserving_steps():
    """Steps that write their own ghost images, then constant-volume steps
    (face kernel after the correction), then image steps again, on one
    periodic FP64 grid: the field stays on the oracle's."""
    N, lam = 32, 2.5
    u = tuple(np.array([1.0, 2.0, 0.0]) / np.sqrt(5.0))
    g, p = make_pair(N, N, N, S.SPFM_F64, (S.SPFM_PERIODIC,) * 6, u, lam=lam, dt=0.05, dF=0.04)
    p0 = O.Params(N, N, N, bc=(O.PERIODIC,) * 6, n=u, lam=lam, dt=0.05, stencil=26, scheme=O.TI_GLOBAL)
    start = upload(g, O.init_cube(p, ((N - 1) / 2.0,) * 3, 8.0), S.SPFM_F64)
    g.step(5, lam=lam, dt=0.05, dF=0.04)
    g.step_conserving(5, lam=lam, dt=0.05)
    g.step(5, lam=lam, dt=0.05, dF=0.04)
    ref = O.step(p, start, 5)
    ref, _ = O.step_conserving(p0, ref, 5)
    ref = O.step(p, ref, 5)
    assert np.abs(gpu_field(g) - ref).max() <= 1e-12


def wrapped_cone_reference(phi_start, sample, T, p_kwargs):
    """Value of one cell of an all-periodic grid after T steps, from an oracle
    run on the (2T+1)^3 box of its dependency cone, indices wrapped."""
    nz, ny, nx = phi_start.shape
    k, j, i = sample
    idx = [np.arange(c - T, c + T + 1) % n for c, n in ((k, nz), (j, ny), (i, nx))]
    sub = np.ascontiguousarray(phi_start[np.ix_(*idx)])
    w = 2 * T + 1
    p = O.Params(w, w, w, bc=(O.NOFLUX,) * 6, **p_kwargs)
    return O.step(p, sub, T)[T, T, T]


def test_grain_512cubed_sampled_cone_parity():
    """The benchmark's grain in its launch configuration: 512^3 FP32, R = 150,
    TI_<120>, 27-point, all faces periodic (the step writes its own ghost
    images), 4 steps; 72 sampled cells (corners, edges, faces, across the
    interface, random) against oracle runs on their wrapped dependency cones."""
    w = WL.sphere_512cubed()
    N, T = w["nx"], 4
    g = S.Grid(N, N, N, dtype=S.SPFM_F32, bc=(S.SPFM_PERIODIC,) * 6, n=w["u"], center=w["ctr"])
    p = O.Params(N, N, N, bc=(O.PERIODIC,) * 6, n=w["u"], lam=w["lam"])
    start = upload(g, O.init_sphere(p, w["ctr"], w["R"]), S.SPFM_F32)
    g.step(T, lam=w["lam"], dt=w["dt"], dF=w["dF"], stencil=26)
    out = g.current().double().cpu().numpy()
    rng = np.random.default_rng(7)
    pts = [(z, y, x) for z in (0, N - 1) for y in (0, N - 1) for x in (0, N - 1)]
    pts += [(0, int(a), N - 1) for a in rng.integers(0, N, 8)]                 # edges
    pts += [(int(a), int(b), 0) for a, b in rng.integers(0, N, (8, 2))]        # faces
    pts += [(N - 1, int(a), int(b)) for a, b in rng.integers(0, N, (8, 2))]
    for d in rng.normal(size=(24, 3)):                                        # the interface
        q = np.array(w["ctr"]) + (w["R"] + rng.uniform(-3, 3)) * d / np.linalg.norm(d)
        pts.append(tuple(int(round(v)) % N for v in q[::-1]))
    pts += [tuple(int(v) for v in rng.integers(0, N, 3)) for _ in range(16)]
    kw = dict(n=w["u"], lam=w["lam"], dt=w["dt"], dF=w["dF"], stencil=26, scheme=O.TI_GLOBAL)
    errs = [abs(out[s] - wrapped_cone_reference(start, s, T, kw)) for s in pts]
    assert max(errs) <= TOL[S.SPFM_F32], max(errs)
    assert sum(1e-6 < out[s] < 1 - 1e-6 for s in pts) >= 16    # the samples do cross the band


# ---------------------------------------------------------------- stats


@pytest.mark.parametrize("dtype", [S.SPFM_F64, S.SPFM_F32])
def test_stats_and_energy_match_oracle(dtype):
    n = rng_normal(7)
    g, p = make_pair(50, 40, 30, dtype, (S.SPFM_CONTACT,) * 6, n, lam=2.0, stencil=26)
    rng = np.random.default_rng(8)
    phi0 = O.init_planar(p, float(n @ [25, 20, 15])) * (1 + 0.01 * rng.random(p.shape))
    start = upload(g, phi0, dtype)
    g.step(0, lam=2.0, dt=0.05)                       # sets the stats model
    st = g.stats(S.SPFM_STATS_ENERGY)
    ref = O.stats(p, start, (0.0, 0.0, 0.0))
    for k in ("volume", "S_w", "S_c", "phi_min", "phi_max", "position"):
        assert abs(st[k] - ref[k]) <= 1e-12 * max(1.0, abs(ref[k])), (k, st[k], ref[k])
    e_ref = O.energy(p, start)
    # an FP32 grid stores its contact-angle ghost cells in FP32 (the oracle's are
    # FP64), and the forward differences of Eq. 1 read them
    e_tol = 1e-12 if dtype == S.SPFM_F64 else 1e-8
    assert abs(st["energy"] - e_ref) <= e_tol * abs(e_ref)
    # radius estimator on a sphere
    ctr = (24.5, 19.5, 14.5)
    g.init_sphere(ctr, 9.0, 2.0)
    st = g.stats()
    ref = O.stats(p, O.init_sphere(p, ctr, 9.0), ctr)
    assert abs(st["radius"] - ref["radius"]) <= (1e-12 if dtype == S.SPFM_F64 else 1e-6)


@pytest.mark.parametrize("dtype", [S.SPFM_F64, S.SPFM_F32, S.SPFM_BF16])
def test_stats_value_mix_matches_oracle(dtype):
    """Every kind of value the stats pass screens differently: exact 0 and 1,
    band values, values a few ulps either side of both band limits, tiny
    (down to subnormal) and negative values, and a few large ones (rows whose
    sum leaves the fixed-point range), on a ragged x extent, with many
    32-cell flushes of the band queue and a partial one at the end."""
    nx, ny, nz = 203, 17, 11
    n = rng_normal(11)
    ctr = (101.3, 8.2, 5.7)
    g = S.Grid(nx, ny, nz, dtype=dtype, n=n, center=ctr)
    p = O.Params(nx, ny, nz, n=tuple(n), lam=3.0)
    rng = np.random.default_rng(12)
    shape = p.shape
    kind = rng.integers(0, 9, size=shape)
    u = rng.uniform(-1.0, 1.0, size=shape)
    choices = [
        np.zeros(shape), np.ones(shape), rng.uniform(0.0, 1.0, size=shape),
        1e-6 * (1.0 + 1e-6 * u),                   # around the lower band limit
        (1.0 - 1e-6) + 3e-7 * u,                   # around the upper band limit
        10.0 ** rng.uniform(-42.0, -7.0, size=shape),
        -rng.uniform(0.0, 1e-3, size=shape),
        1.0 + rng.uniform(0.0, 1e-5, size=shape),
        rng.uniform(0.0, 1.0, size=shape),
    ]
    phi = np.choose(kind, choices)
    phi[3, 5, 7] = 300.0
    phi[9, 16, 200] = 5e3
    start = upload(g, phi, dtype)
    g.step(0, lam=3.0, dt=0.05)
    st = g.stats()
    ref = O.stats(p, start, ctr)
    assert ref["S_w"] > 0.0
    for k in ("volume", "S_w", "S_c", "S_r", "phi_min", "phi_max", "position", "radius"):
        assert abs(st[k] - ref[k]) <= 1e-12 * max(1.0, abs(ref[k])), (k, st[k], ref[k])


# --------------------------------------------------------------- config 1


@pytest.mark.parametrize("scheme", [S.SPFM_TI_GLOBAL, S.SPFM_FD])
def test_planar_100_fp64_1000_steps(scheme):
    """Planar (1,0,0) interface, 128x32x32 FP64, 7-point, 1000 steps: field
    parity <= 1e-12 and interface velocity against the oracle's (1e-4) and,
    for SPFM, against v_th = -M dF/Gamma (1e-4)."""
    w = WL.planar_100_128x32x32()
    bc = WL.bc_codes(w)
    g, p = make_pair(w["nx"], w["ny"], w["nz"], S.SPFM_F64, bc, w["n"], lam=w["lam"], dt=w["dt"],
                     dF=w["dF"], stencil=w["stencil"], scheme=scheme)
    g.init_planar(w["c"], w["lam"], w["dx"])
    phi = O.init_planar(p, w["c"])
    half = w["steps"] // 2
    args = dict(M=1.0, Gamma=1.0, lam=w["lam"], dx=1.0, dt=w["dt"], dF=w["dF"], stencil=6, scheme=scheme)
    g.step(half, **args)
    c1 = g.stats()["position"]
    phi = O.step(p, phi, half)
    c1o = O.stats(p, phi)["position"]
    g.step(w["steps"] - half, **args)
    c2 = g.stats()["position"]
    phi = O.step(p, phi, w["steps"] - half)
    c2o = O.stats(p, phi)["position"]
    assert np.abs(gpu_field(g) - phi).max() <= 1e-12
    T = (w["steps"] - half) * w["dt"]
    v, vo = (c2 - c1) / T, (c2o - c1o) / T
    assert abs(v / vo - 1) < 1e-4
    if scheme == S.SPFM_TI_GLOBAL:
        assert abs(v / (-w["dF"]) - 1) < 1e-4


# ----------------------------------------------------- full-size sampled


def cone_reference(phi_start, shape, bc, sample, T, p_kwargs):
    """Value of one cell after T steps, from an oracle run on the sub-box that
    holds its dependency cone (cut faces T cells away from the sample)."""
    nz, ny, nx = shape
    idx = []
    sub_bc = []
    for ax, (c, N) in enumerate(zip(sample[::-1], (nx, ny, nz))):
        lo, hi = max(0, c - T), min(N - 1, c + T)
        idx.append((lo, hi))
        sub_bc.append(bc[2 * ax] if lo == 0 else O.NOFLUX)
        sub_bc.append(bc[2 * ax + 1] if hi == N - 1 else O.NOFLUX)
    (x0, x1), (y0, y1), (z0, z1) = idx
    sub = np.ascontiguousarray(phi_start[z0:z1 + 1, y0:y1 + 1, x0:x1 + 1])
    p = O.Params(x1 - x0 + 1, y1 - y0 + 1, z1 - z0 + 1, bc=tuple(sub_bc), **p_kwargs)
    # the contact BC and estimator use absolute positions only through n and
    # differences, so a sub-box needs no origin shift
    out = O.step(p, sub, T)
    k, j, i = sample
    return out[k - z0, j - y0, i - x0]


@pytest.mark.parametrize("dtype", [S.SPFM_F32, S.SPFM_F64])
def test_tilted_256cubed_sampled_cone_parity(dtype):
    """256^3, normal (1,1,1)/sqrt3, 27-point SPFM, contact BCs on all faces, in
    the launch configuration of the benchmark: 4 steps, 64 sampled cells
    (corners, edges, faces, interior, interface) against dependency-cone oracle
    runs."""
    w = WL.tilted_111_256cubed()[0]
    N, T = w["nx"], 4
    bc = WL.bc_codes(w)
    g = S.Grid(N, N, N, dtype=dtype, bc=bc, n=w["n"])
    p = O.Params(N, N, N, bc=bc, n=w["n"], lam=w["lam"])
    phi0 = O.init_planar(p, w["c"])
    start = upload(g, phi0, dtype)
    g.step(T, lam=w["lam"], dt=w["dt"], dF=w["dF"], stencil=26)
    out = g.current().double().cpu().numpy()
    rng = np.random.default_rng(5)
    pts = [(z, y, x) for z in (0, N - 1) for y in (0, N - 1) for x in (0, N - 1)]
    pts += [tuple(int(v) for v in rng.integers(0, N, 3)) for _ in range(24)]
    pts += [(int(v), int(v), int(v)) for v in rng.integers(100, 156, 16)]   # across the interface
    pts += [(0, int(a), int(b)) for a, b in rng.integers(0, N, (8, 2))]
    pts += [(int(a), N - 1, int(b)) for a, b in rng.integers(0, N, (8, 2))]
    kw = dict(n=w["n"], lam=w["lam"], dt=w["dt"], dF=w["dF"], stencil=26, scheme=O.TI_GLOBAL)
    errs = [abs(out[s] - cone_reference(start, (N, N, N), bc, s, T, kw)) for s in pts]
    assert max(errs) <= TOL[dtype], max(errs)


# ------------------------------------------------------------------ TI_n


@pytest.mark.parametrize("dtype", [S.SPFM_F64, S.SPFM_F32])
@pytest.mark.parametrize("stencil", [26, 18, 6])
def test_ti_local_normal_sphere_parity(dtype, stencil):
    """TI_n on a curved interface (grain of radius 11, periodic 44x40x36) against
    the oracle's TI_n (local normal from the profile inversion)."""
    shape = (44, 40, 36)
    g, p = make_pair(*shape, dtype, (S.SPFM_PERIODIC,) * 6, (1.0, 0.0, 0.0), lam=3.0, dt=0.05,
                     dF=0.02, stencil=stencil, scheme=S.SPFM_TI_LOCAL)
    ctr = (21.3, 19.6, 17.2)
    phi0 = O.init_sphere(p, ctr, 11.0)
    start = upload(g, phi0, dtype)
    g.step(30, lam=3.0, dt=0.05, dF=0.02, stencil=stencil, scheme=S.SPFM_TI_LOCAL)
    ref = O.step(p, start, 30)
    err = np.abs(gpu_field(g) - ref).max()
    assert err <= TOL[dtype], err


@pytest.mark.parametrize("dtype", [S.SPFM_F64, S.SPFM_F32])
def test_ti_local_normal_tilted_plane_parity(dtype):
    n = rng_normal(44)
    shape = (37, 21, 19)
    g, p = make_pair(*shape, dtype, (S.SPFM_CONTACT,) * 6, n, lam=2.5, dt=0.05, dF=0.03, stencil=26,
                     scheme=S.SPFM_TI_LOCAL)
    rng = np.random.default_rng(45)
    phi0 = O.init_planar(p, float(n @ (np.array(shape) - 1) / 2.0)) + 0.005 * rng.random(p.shape)
    start = upload(g, phi0, dtype)
    g.step(25, lam=2.5, dt=0.05, dF=0.03, stencil=26, scheme=S.SPFM_TI_LOCAL)
    ref = O.step(p, start, 25)
    assert np.abs(gpu_field(g) - ref).max() <= TOL[dtype]


# ------------------------------------------------------------ sphericity


@pytest.mark.parametrize("ctr,R", [((19.4, 17.8, 15.3), 9.5), ((12.6, 21.3, 11.9), 7.5)])
@pytest.mark.parametrize("dtype", [S.SPFM_F64, S.SPFM_F32])
def test_sphericity_matches_oracle(dtype, ctr, R):
    """Sec. 3.3 eps_eff from the nonlinear contour points, after TI_n relaxation;
    the second grain sits far from the box centre, where only the particle's own
    barycentre gives the oracle's radii."""
    shape = (40, 36, 32)
    g, p = make_pair(*shape, dtype, (S.SPFM_PERIODIC,) * 6, (1.0, 0.0, 0.0), lam=3.0, dt=0.05,
                     dF=0.0, stencil=26, scheme=S.SPFM_TI_LOCAL)
    phi0 = O.init_sphere(p, ctr, R)
    start = upload(g, phi0, dtype)
    g.step(20, lam=3.0, dt=0.05, dF=0.0, stencil=26, scheme=S.SPFM_TI_LOCAL)
    field = gpu_field(g)
    got = g.sphericity(0)
    ref = O.sphericity(p, field, inside_phase=0)
    assert got["n_points"] == ref["n_points"]
    for k in ("eps_eff", "R_mean", "R_min", "R_max"):
        assert abs(got[k] - ref[k]) <= 1e-11 * max(1.0, abs(ref[k])), (k, got[k], ref[k])
    assert np.allclose(got["barycentre"], ref["barycentre"], rtol=0, atol=1e-10)
