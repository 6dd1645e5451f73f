"""The z-chunk of the step launches changes nothing in the field.

Each CTA of a step launch marches one z-chunk; a chunk reads one halo plane
on each side and, on grids with no periodic face, its producer warp rebuilds
the ghosts of the faces its planes touch (Eq. 7 at contact faces) before it
releases them.  For every kernel family (FP64, FP32 and BF16 storage; CF, TI
with 3 and 13 coupling groups, TI_n; 6/18/26 neighbours; all faces periodic
with the kernels that write their own images, no periodic face with the
ghosts built inside the kernel, a mix with the face kernel; round to nearest
and stochastic rounding) the field after a few steps is the same bit for bit
for chunks of 1, 2, 3, 4, 5 and 7 planes, the per-launch choice (0) and one
chunk over the whole grid; that field is the FP64 oracle's within the bar of
its storage type.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1910_05180_gb300 import spfm as S
from paper_1910_05180_gb300 import workloads as WL

pytestmark = pytest.mark.gpu

P, C, N = S.SPFM_PERIODIC, S.SPFM_CONTACT, S.SPFM_NOFLUX
SCHEME_O = {S.SPFM_TI_GLOBAL: O.TI_GLOBAL, S.SPFM_TI_LOCAL: O.TI_LOCAL, S.SPFM_FD: O.CF}
TOL = {S.SPFM_F64: 1e-12, S.SPFM_F32: 2e-5, S.SPFM_BF16: None}
U120 = (1.0, 2.0, 0.0)

CASES = [
    # (shape, bc, dtype, stencil, scheme, u, stochastic)
    ((64, 18, 35), (P,) * 6, S.SPFM_F32, 26, S.SPFM_TI_GLOBAL, U120, False),      # image kernel
    ((37, 21, 19), (C,) * 6, S.SPFM_F32, 26, S.SPFM_TI_GLOBAL, None, False),      # 13 groups, inline ghosts
    ((40, 24, 20), (C,) * 6, S.SPFM_F32, 26, S.SPFM_TI_GLOBAL, U120, True),
    ((37, 21, 19), (C,) * 6, S.SPFM_F32, 18, S.SPFM_TI_GLOBAL, U120, False),
    ((37, 21, 19), (N, N, C, C, N, C), S.SPFM_F32, 6, S.SPFM_FD, None, False),
    ((67, 33, 17), (N, N, P, P, C, C), S.SPFM_F32, 26, S.SPFM_FD, None, False),    # face kernel
    ((70, 20, 13), (C,) * 6, S.SPFM_F32, 26, S.SPFM_TI_LOCAL, None, False),
    ((64, 16, 22), (P,) * 6, S.SPFM_F32, 26, S.SPFM_TI_LOCAL, None, True),
    ((37, 21, 19), (C,) * 6, S.SPFM_F64, 26, S.SPFM_TI_GLOBAL, None, False),
    ((32, 18, 21), (P,) * 6, S.SPFM_F64, 26, S.SPFM_TI_GLOBAL, U120, False),
    ((40, 24, 20), (C,) * 6, S.SPFM_BF16, 26, S.SPFM_TI_GLOBAL, U120, True),
    ((64, 18, 35), (P,) * 6, S.SPFM_BF16, 26, S.SPFM_FD, None, False),
]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    S.load()


@pytest.mark.parametrize("case", range(len(CASES)))
def test_field_independent_of_zchunk(case):
    shape, bc, dtype, stencil, scheme, u, sr = CASES[case]
    rng = np.random.default_rng(900 + case)
    n = WL.random_normal(rng)
    uu = tuple(WL.unit(u)) if u else (0.0, 0.0, 0.0)
    lam, dt, dF, steps = 2.5, 0.05 if scheme != S.SPFM_TI_LOCAL else 0.02, 0.03, 6
    p = O.Params(*shape, bc=bc, n=tuple(n), u=uu, lam=lam, dt=dt, dF=dF, stencil=stencil, scheme=SCHEME_O[scheme])
    # a noisy plane kept inside (0.005, 0.999): beyond 1 - 1e-6 the profile
    # inversion of TI_n clamps phi, and FP32 and FP64 may take that branch on
    # different cells
    phi0 = 0.005 + 0.99 * O.init_planar(p, float(n @ (np.array(shape) - 1) / 2.0)) + 0.004 * rng.random(p.shape)
    host = torch.from_numpy(phi0).to(S.TORCH_DTYPE[dtype])
    fields = {}
    for zc in (shape[2], 0, 1, 2, 3, 4, 5, 7):
        g = S.Grid(*shape, dtype=dtype, bc=bc, n=tuple(n), u=uu)
        if sr:
            g.set_rounding(S.SPFM_ROUND_STOCHASTIC, seed=case)
        g.set_zchunk(zc)
        g.set_field(host.cuda())
        g.step(steps, lam=lam, dt=dt, dF=dF, stencil=stencil, scheme=scheme)
        assert g.stats()["nonfinite"] == 0.0
        fields[zc] = g.get_field(to_host=True)
        g.close()
    whole = fields[shape[2]]
    for zc, f in fields.items():
        assert torch.equal(f, whole), (zc, (f.double() - whole.double()).abs().max().item())
    if TOL[dtype] is not None:
        ref = O.step(p, host.double().numpy(), steps)
        assert np.abs(whole.double().numpy() - ref).max() <= TOL[dtype]


@pytest.mark.parametrize("policy", [S.SPFM_TILES_WIDE, S.SPFM_TILES_SQUARE])
@pytest.mark.parametrize("scheme", [S.SPFM_TI_GLOBAL, S.SPFM_FD])
@pytest.mark.parametrize("stencil", [6, 18, 26])
def test_batch_equals_single_grids_bitwise(stencil, scheme, policy):
    """The persistent batch kernel (other tile shapes, its own z-depth, a
    work-list over several grids) gives each grid the field of the single-grid
    kernel bit for bit, for every stencil and both potentials."""
    rng = np.random.default_rng(40 + stencil)
    shapes = [(37, 21, 19), (48, 40, 36), (20, 20, 70)]
    us = [U120, None, (1.0, 1.0, 1.0)]
    jobs = []
    for shape, u in zip(shapes, us):
        n = WL.random_normal(rng)
        jobs.append(dict(shape=shape, n=tuple(n), u=tuple(WL.unit(u)) if u else (0.0, 0.0, 0.0),
                         lam=float(rng.choice([2.0, 3.0, 4.0])), dF=float(rng.uniform(1e-3, 0.05)),
                         c=float(n @ (np.array(shape) - 1) / 2.0)))
    sets = []
    for _ in range(2):
        gs = []
        for j in jobs:
            g = S.Grid(*j["shape"], dtype=S.SPFM_F32, bc=(C,) * 6, n=j["n"], u=j["u"])
            g.init_planar(j["c"], j["lam"])
            gs.append(g)
        sets.append(gs)
    batched, alone = sets
    args = [S.step_args(lam=j["lam"], dt=0.05, dF=j["dF"], stencil=stencil, scheme=scheme) for j in jobs]
    b = S.Batch(batched)
    b.set_tiles(policy)
    b.step(23, args)
    torch.cuda.synchronize()
    for g, a in zip(alone, args):
        g.step(23, lam=a.lam, dt=a.dt, dF=a.dF, stencil=stencil, scheme=scheme)
    for gb, ga in zip(batched, alone):
        fb, fa = gb.get_field(), ga.get_field()
        assert torch.equal(fb, fa), (fb.double() - fa.double()).abs().max().item()
    b.close()
    for g in batched + alone:
        g.close()
