"""Batches: many uneven grids stepped by one persistent launch per step.

Each grid of a batch must end bit-identical to the same grid stepped alone
(the per-cell arithmetic is the same), across captured-graph replays and odd
remainders, and within the FP32 bar of the FP64 oracle.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1910_05180_gb300 import spfm as S
from paper_1910_05180_gb300 import workloads as WL

pytestmark = pytest.mark.gpu

SHAPES = [(32, 32, 32), (48, 40, 36), (67, 33, 17), (20, 20, 70), (96, 16, 24)]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    S.load()


def _jobs(seed, dtype=S.SPFM_F32, scheme=S.SPFM_TI_GLOBAL):
    rng = np.random.default_rng(seed)
    jobs = []
    for shape in SHAPES:
        n = WL.random_normal(rng)
        lam = float(rng.choice([2.0, 3.0, 4.0, 6.0]))
        dF = float(rng.uniform(1e-4, 0.05))
        jobs.append(dict(shape=shape, n=tuple(n), lam=lam, dF=dF,
                         c=float(n @ (np.array(shape) - 1) / 2.0)))
    return jobs


def _grids(jobs, dtype, stream):
    gs = []
    for j in jobs:
        g = S.Grid(*j["shape"], dtype=dtype, bc=(S.SPFM_CONTACT,) * 6, n=j["n"], stream=stream)
        g.init_planar(j["c"], j["lam"])
        gs.append(g)
    return gs


def _args(jobs, scheme=S.SPFM_TI_GLOBAL):
    return [S.step_args(lam=j["lam"], dt=0.05, dF=j["dF"], stencil=26, scheme=scheme) for j in jobs]


@pytest.mark.parametrize("scheme", [S.SPFM_TI_GLOBAL, S.SPFM_FD])
def test_batch_equals_single_grid_bitwise(scheme):
    jobs = _jobs(1)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        batched = _grids(jobs, S.SPFM_F32, stream)
        alone = _grids(jobs, S.SPFM_F32, stream)
        b = S.Batch(batched, stream=stream)
        args = _args(jobs, scheme)
        for n_steps in (37, 20, 1):          # graph replays + odd remainders + parity flips
            b.step(n_steps, args)
            for g, a in zip(alone, args):
                g.step(n_steps, lam=a.lam, dt=a.dt, dF=a.dF, stencil=26, scheme=scheme)
        stream.synchronize()
        for gb, ga in zip(batched, alone):
            assert torch.equal(gb.get_field(), ga.get_field())
            assert torch.equal(gb.current_with_ghosts(), ga.current_with_ghosts())


def test_batch_matches_oracle():
    jobs = _jobs(2)[:3]
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        gs = _grids(jobs, S.SPFM_F32, stream)
        starts = [g.get_field().double().numpy() for g in gs]
        b = S.Batch(gs, stream=stream)
        b.step(24, _args(jobs))
        stream.synchronize()
    for g, j, st in zip(gs, jobs, starts):
        p = O.Params(*j["shape"], bc=(O.CONTACT,) * 6, n=j["n"], lam=j["lam"], dt=0.05, dF=j["dF"], stencil=26)
        ref = O.step(p, st, 24)
        assert np.abs(g.get_field().double().numpy() - ref).max() <= 2e-5


def test_batch_stats_equal_single_stats():
    jobs = _jobs(3)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        gs = _grids(jobs, S.SPFM_F64, stream)
        b = S.Batch(gs, stream=stream)
        b.step(10, _args(jobs))
        bst = b.stats(S.SPFM_STATS_ENERGY)
        for g, s in zip(gs, bst):
            one = g.stats(S.SPFM_STATS_ENERGY)
            for k in ("volume", "S_w", "S_c", "position", "energy", "phi_min", "phi_max", "steps", "time"):
                assert abs(s[k] - one[k]) <= 1e-12 * max(1.0, abs(one[k])), (k, s[k], one[k])


def test_batch_rejects_mixed_stencils():
    jobs = _jobs(4)[:2]
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        gs = _grids(jobs, S.SPFM_F32, stream)
        b = S.Batch(gs, stream=stream)
        args = _args(jobs)
        args[1].stencil = 18
        with pytest.raises(S.SpfmError) as e:
            b.step(1, args)
        assert e.value.status == S.SPFM_EINVAL


@pytest.mark.parametrize("policy", [S.SPFM_TILES_WIDE, S.SPFM_TILES_SQUARE, S.SPFM_TILES_FIT])
def test_tile_policies_equal_single_grids_bitwise(policy):
    """The tile shape of a grid's items (64 x 16 or 32 x 32 cells, or per grid
    the one that pads its extent least, here a mix) changes only the
    work-list: after graph replays and an odd remainder the fields are
    bit-identical to the same grids stepped alone."""
    jobs = _jobs(7)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        batched = _grids(jobs, S.SPFM_F32, stream)
        alone = _grids(jobs, S.SPFM_F32, stream)
        b = S.Batch(batched, stream=stream)
        b.set_tiles(policy)
        assert b.tiles()[0] == policy
        args = _args(jobs)
        b.step(37, args)
        for g, a in zip(alone, args):
            g.step(37, lam=a.lam, dt=a.dt, dF=a.dF, stencil=26)
        stream.synchronize()
        for gb, ga in zip(batched, alone):
            assert torch.equal(gb.get_field(), ga.get_field())


def test_autotuned_batch_equals_single_grids_bitwise():
    """The autotuner's trial steps are real steps, and the tile policy and
    depth it picks change only the work-list: fields stay bit-identical to
    single grids."""
    jobs = _jobs(5)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        batched = _grids(jobs, S.SPFM_F32, stream)
        alone = _grids(jobs, S.SPFM_F32, stream)
        b = S.Batch(batched, stream=stream)
        args = _args(jobs)
        depth, ms = b.autotune(args, steps_per_trial=16)
        assert depth in S.BATCH_DEPTHS and all(v > 0.0 for v in ms.values())
        assert b.tiles() in [(p, depth) for p in (S.SPFM_TILES_WIDE, S.SPFM_TILES_SQUARE, S.SPFM_TILES_FIT)]
        tuned = (3 + len(S.BATCH_DEPTHS)) * 32
        b.step(21, args)
        for g, a in zip(alone, args):
            g.step(tuned + 21, lam=a.lam, dt=a.dt, dF=a.dF, stencil=26)
        stream.synchronize()
        for gb, ga in zip(batched, alone):
            assert gb.stats()["steps"] == ga.stats()["steps"] == tuned + 21
            assert torch.equal(gb.get_field(), ga.get_field())
