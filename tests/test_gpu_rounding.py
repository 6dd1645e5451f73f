"""Stochastic rounding of the update (SPFM_ROUND_STOCHASTIC) on the GPU.

- Unbiasedness: on a uniform periodic field every cell has the same exact
  update phi0 + dt R (Eq. 2, R from the oracle in FP64).  Rounded to nearest,
  every cell lands on the same neighbour of that value; rounded stochastically,
  the mean over the cells is the exact update within its binomial spread.
- Parity: the FP32 field stays within 2e-5 of the FP64 oracle for every
  kernel kind (CF, TI with 1..13 coupling groups, TI_n), stencil and boundary
  mix, including the all-periodic kernels that write their own ghost images.
- Reproducibility: the same seed gives the same field bit for bit; a batch
  gives the field of the same grid stepped alone, across graph replays.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1910_05180_gb300 import spfm as S
from paper_1910_05180_gb300 import workloads as WL

pytestmark = pytest.mark.gpu

SCHEME_O = {S.SPFM_TI_GLOBAL: O.TI_GLOBAL, S.SPFM_TI_LOCAL: O.TI_LOCAL, S.SPFM_FD: O.CF}
UNIT = WL.unit


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    S.load()


def _upload(g, phi64, dtype):
    t = torch.from_numpy(phi64).to(S.TORCH_DTYPE[dtype])
    g.set_field(t.cuda())
    return t.double().numpy()


@pytest.mark.parametrize("dtype", [S.SPFM_F32, S.SPFM_BF16])
@pytest.mark.parametrize("frac", [0.05, 0.3, 0.7])
def test_stochastic_rounding_is_unbiased(dtype, frac):
    """Uniform phi0 = 0.9 on 64^3 periodic, TI with u || [120] (4 groups), one
    step with dt chosen so that the exact increment is `frac` of a unit in the
    last place of the storage type at phi0."""
    shape, lam, dF = (64, 64, 64), 3.0, 0.01
    u = tuple(UNIT([1.0, 2.0, 0.0]))
    phi0 = float(torch.tensor(0.9, dtype=S.TORCH_DTYPE[dtype]).double())
    ulp = 2.0 ** -24 if dtype == S.SPFM_F32 else 2.0 ** -8    # spacing of [0.5, 1)
    p = O.Params(*shape, n=u, lam=lam, dF=dF, stencil=26)
    R, _ = O.rhs(p, np.full(p.shape, phi0))
    R0 = float(R.flat[0])
    assert np.all(R == R0)
    dt = frac * ulp / abs(R0)
    exact = phi0 + dt * R0
    for mode in (S.SPFM_ROUND_NEAREST, S.SPFM_ROUND_STOCHASTIC):
        g = S.Grid(*shape, dtype=dtype, bc=(S.SPFM_PERIODIC,) * 6, n=u)
        g.set_rounding(mode, seed=7)
        _upload(g, np.full(p.shape, phi0), dtype)
        g.step(1, lam=lam, dt=dt, dF=dF, stencil=26)
        f = g.get_field(to_host=True).double().numpy()
        N = f.size
        vals = np.unique(f)
        if mode == S.SPFM_ROUND_NEAREST:
            assert len(vals) == 1               # every cell took the same neighbour
        else:
            # two neighbours of the exact value, in the proportion of the distances
            assert set(vals) <= {phi0, phi0 + np.sign(R0) * ulp}
            f_up = np.mean(f != phi0)
            sigma = np.sqrt(frac * (1 - frac) / N)
            assert abs(f_up - frac) < 6 * sigma, (f_up, frac, sigma)
            assert abs(f.mean() - exact) < 6 * sigma * ulp
        g.close()


CASES = [
    # (shape, bc, stencil, scheme, u)
    ((37, 21, 19), (S.SPFM_CONTACT,) * 6, 26, S.SPFM_TI_GLOBAL, None),             # 13 groups
    ((40, 24, 20), (S.SPFM_CONTACT,) * 6, 26, S.SPFM_TI_GLOBAL, (1.0, 2.0, 0.0)),  # 4 groups
    ((37, 21, 19), (S.SPFM_CONTACT,) * 6, 18, S.SPFM_TI_GLOBAL, None),
    ((37, 21, 19), (S.SPFM_CONTACT,) * 6, 6, S.SPFM_TI_GLOBAL, None),
    ((67, 33, 17), (S.SPFM_NOFLUX, S.SPFM_NOFLUX, S.SPFM_PERIODIC, S.SPFM_PERIODIC,
                    S.SPFM_CONTACT, S.SPFM_CONTACT), 26, S.SPFM_FD, None),
    ((130, 2, 3), (S.SPFM_PERIODIC,) * 2 + (S.SPFM_CONTACT,) * 4, 26, S.SPFM_TI_LOCAL, None),
    # all faces periodic, rows of whole 32-byte sectors: the image-writing kernels
    ((64, 18, 35), (S.SPFM_PERIODIC,) * 6, 26, S.SPFM_TI_GLOBAL, (1.0, 2.0, 0.0)),
    ((64, 18, 35), (S.SPFM_PERIODIC,) * 6, 26, S.SPFM_FD, None),
    ((136, 3, 4), (S.SPFM_PERIODIC,) * 6, 18, S.SPFM_TI_LOCAL, None),
    ((5, 3, 2), (S.SPFM_CONTACT,) * 6, 26, S.SPFM_TI_GLOBAL, None),
]


@pytest.mark.parametrize("case", range(len(CASES)))
def test_stochastic_rounding_parity_f32(case):
    shape, bc, stencil, scheme, u = CASES[case]
    rng = np.random.default_rng(300 + case)
    n = WL.random_normal(rng)
    uu = tuple(UNIT(u)) if u else (0.0, 0.0, 0.0)
    lam, dt, dF, steps = 2.5, 0.05, 0.03, 40
    g = S.Grid(*shape, dtype=S.SPFM_F32, bc=bc, n=tuple(n), u=uu)
    g.set_rounding(S.SPFM_ROUND_STOCHASTIC, seed=case)
    p = O.Params(*shape, bc=bc, n=tuple(n), u=uu, lam=lam, dt=dt, dF=dF, stencil=stencil,
                 scheme=SCHEME_O[scheme])
    phi0 = O.init_planar(p, float(n @ (np.array(shape) - 1) / 2.0)) + 0.01 * rng.random(p.shape)
    start = _upload(g, phi0, S.SPFM_F32)
    g.step(steps, lam=lam, dt=dt, dF=dF, stencil=stencil, scheme=scheme)
    ref = O.step(p, start, steps)
    err = np.abs(g.get_field(to_host=True).double().numpy() - ref).max()
    assert err <= 2e-5, err


def _grain(seed, mode, steps, dtype=S.SPFM_F32):
    w = WL.sphere_replica_128cubed()
    N = 64
    ctr = ((N - 1) / 2.0,) * 3
    g = S.Grid(N, N, N, dtype=dtype, bc=(S.SPFM_PERIODIC,) * 6, n=w["u"], center=ctr)
    g.set_rounding(mode, seed=seed)
    g.init_sphere(ctr, 18.0, w["lam"])
    g.step(steps, lam=w["lam"], dt=w["dt"], dF=w["dF"], stencil=26)
    return g.get_field()


def test_stochastic_rounding_is_reproducible():
    a = _grain(11, S.SPFM_ROUND_STOCHASTIC, 30)
    b = _grain(11, S.SPFM_ROUND_STOCHASTIC, 30)
    c = _grain(12, S.SPFM_ROUND_STOCHASTIC, 30)
    r = _grain(11, S.SPFM_ROUND_NEAREST, 30)
    assert torch.equal(a, b)
    assert not torch.equal(a, c) and not torch.equal(a, r)
    assert (a.double() - c.double()).abs().max().item() < 1e-6


@pytest.mark.parametrize("dtype", [S.SPFM_F32, S.SPFM_BF16])
def test_stochastic_batch_equals_single_grids_bitwise(dtype):
    """Each grid draws its bits from its own step count: batched (graph
    replays, an odd remainder, a second call) equals stepped alone, also for a
    grid that had taken steps of its own before joining the batch."""
    rng = np.random.default_rng(5)
    shapes = [(32, 32, 32), (48, 40, 36), (67, 33, 17), (20, 20, 70)]
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        sets = []
        jobs = []
        for shape in shapes:
            n = WL.random_normal(rng)
            jobs.append(dict(shape=shape, n=tuple(n), lam=float(rng.choice([2.0, 3.0, 4.0])),
                             dF=float(rng.uniform(1e-4, 0.05)), c=float(n @ (np.array(shape) - 1) / 2.0)))
        for _ in range(2):
            gs = []
            for i, j in enumerate(jobs):
                g = S.Grid(*j["shape"], dtype=dtype, bc=(S.SPFM_CONTACT,) * 6, n=j["n"], stream=stream)
                g.set_rounding(S.SPFM_ROUND_STOCHASTIC, seed=100 + i)
                g.init_planar(j["c"], j["lam"])
                gs.append(g)
            sets.append(gs)
        batched, alone = sets
        # the first grid starts with 5 steps of its own in both sets
        for gs in sets:
            gs[0].step(5, lam=jobs[0]["lam"], dt=0.05, dF=jobs[0]["dF"], stencil=26)
        args = [S.step_args(lam=j["lam"], dt=0.05, dF=j["dF"], stencil=26) for j in jobs]
        b = S.Batch(batched, stream=stream)
        b.step(37, args)
        b.step(20, args)
        for g, a in zip(alone, args):
            g.step(57, lam=a.lam, dt=a.dt, dF=a.dF, stencil=26)
        stream.synchronize()
        for gb, ga in zip(batched, alone):
            assert torch.equal(gb.get_field(), ga.get_field())
        b.close()


def test_batch_refuses_mixed_rounding():
    g1 = S.Grid(16, 16, 16, dtype=S.SPFM_F32, bc=(S.SPFM_CONTACT,) * 6)
    g2 = S.Grid(16, 16, 16, dtype=S.SPFM_F32, bc=(S.SPFM_CONTACT,) * 6)
    for g in (g1, g2):
        g.init_planar(8.0, 3.0)
    g2.set_rounding(S.SPFM_ROUND_STOCHASTIC, 1)
    b = S.Batch([g1, g2])
    with pytest.raises(S.SpfmError) as e:
        b.step(1, [S.step_args(lam=3.0, dt=0.05, stencil=26)] * 2)
    assert e.value.status == S.SPFM_EINVAL and "rounding" in str(e.value)
    b.close()


def test_conserving_steps_take_the_rounding_mode():
    """Constant-volume steps round their step as the grid's mode says: the same
    seed gives the same field, round to nearest another one."""
    N, lam = 32, 2.5
    ctr = ((N - 1) / 2.0,) * 3
    out = []
    for mode, seed in ((S.SPFM_ROUND_STOCHASTIC, 4), (S.SPFM_ROUND_STOCHASTIC, 4), (S.SPFM_ROUND_NEAREST, 4)):
        g = S.Grid(N, N, N, dtype=S.SPFM_F32, bc=(S.SPFM_PERIODIC,) * 6, n=tuple(UNIT([1.0, 2.0, 0.0])))
        g.set_rounding(mode, seed=seed)
        g.init_cube(ctr, 8.0, lam)
        g.step_conserving(20, lam=lam, dt=0.05, stencil=26)
        out.append(g.get_field())
        g.close()
    assert torch.equal(out[0], out[1])
    assert not torch.equal(out[0], out[2])
