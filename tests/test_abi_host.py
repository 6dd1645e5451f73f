"""Host-side checks of the C ABI that need no GPU: the library loads, exports
every entry point declared in include/*.h, computes layouts, and rejects bad
arguments before any CUDA call (validation runs first in every entry point).
"""
import ctypes
import glob
import heapq
import math
import os
import random
import re

import numpy as np
import pytest

from paper_1910_05180_gb300 import build as B
from paper_1910_05180_gb300 import spfm as S

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return S.load()


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(spfm_[a-z0-9_]+)\s*\(",
                             text, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n
    # and the binding marshals every one of them
    bound = {s[0] for s in S.SIGNATURES}
    assert set(names) <= bound, set(names) - bound


def _desc(nx=10, ny=7, nz=5, dtype=S.SPFM_F32, bc=(S.SPFM_PERIODIC,) * 6, n=(1.0, 0.0, 0.0)):
    d = S.GridDesc()
    d.nx, d.ny, d.nz, d.dtype = nx, ny, nz, dtype
    for i in range(6):
        d.bc[i] = bc[i]
    for i in range(3):
        d.n[i] = n[i]
    return d


@pytest.mark.parametrize("dtype,per32", [(S.SPFM_F64, 4), (S.SPFM_F32, 8), (S.SPFM_BF16, 16)])
def test_layout_rows_are_whole_32_byte_sectors(lib, dtype, per32):
    for nx in (1, 3, 4, 17, 128, 130):
        px, xo, fb, sb = S.spfm_layout(_desc(nx=nx, dtype=dtype))
        assert xo == per32 and px % per32 == 0 and xo + nx + 1 <= px < xo + nx + 1 + per32
        es = {S.SPFM_F64: 8, S.SPFM_F32: 4, S.SPFM_BF16: 2}[dtype]
        assert fb == px * (7 + 2) * (5 + 2) * es
        assert sb > 0


def _fake_grid(lib, **kw):
    """A handle over fake, aligned pointers: fine for calls that fail validation."""
    d = _desc(**kw)
    _, _, _, sb = S.spfm_layout(d)
    d.field[0], d.field[1] = 0x10000, 0x20000
    d.scratch, d.scratch_bytes = 0x30000, sb
    return S.spfm_create_grid(d)


def test_kernels_per_step_follows_the_periodic_image_rule(lib):
    """One launch per step when the step writes its own periodic ghost images
    (every face periodic, nx a whole number (>= 2) of 32-byte sectors, ny >= 2)
    or when no face is periodic (the step computes the contact and no-flux
    ghosts as it reads them); otherwise the ghost-face kernel follows each
    step."""
    P, C = (S.SPFM_PERIODIC,) * 6, (S.SPFM_CONTACT,) * 6
    mixed = (S.SPFM_PERIODIC,) * 4 + (S.SPFM_NOFLUX,) * 2
    closed = (S.SPFM_NOFLUX,) * 2 + (S.SPFM_CONTACT,) * 4
    cases = [
        (dict(nx=16, ny=2, nz=1, dtype=S.SPFM_F32, bc=P), 1),
        (dict(nx=512, ny=512, nz=512, dtype=S.SPFM_F32, bc=P), 1),
        (dict(nx=8, ny=5, nz=5, dtype=S.SPFM_F32, bc=P), 2),      # one sector only
        (dict(nx=20, ny=5, nz=5, dtype=S.SPFM_F32, bc=P), 2),     # not whole sectors
        (dict(nx=16, ny=1, nz=5, dtype=S.SPFM_F32, bc=P), 2),     # ny = 1
        (dict(nx=16, ny=5, nz=5, dtype=S.SPFM_F32, bc=C), 1),
        (dict(nx=7, ny=1, nz=3, dtype=S.SPFM_F64, bc=closed), 1),
        (dict(nx=16, ny=5, nz=5, dtype=S.SPFM_F32, bc=mixed), 2),
        (dict(nx=8, ny=5, nz=5, dtype=S.SPFM_F64, bc=P), 1),
        (dict(nx=4, ny=5, nz=5, dtype=S.SPFM_F64, bc=P), 2),
        (dict(nx=32, ny=5, nz=5, dtype=S.SPFM_BF16, bc=P), 1),
        (dict(nx=16, ny=5, nz=5, dtype=S.SPFM_BF16, bc=P), 2),
    ]
    for kw, want in cases:
        h = _fake_grid(lib, **kw)
        try:
            assert S.spfm_kernels_per_step(h) == want, kw
        finally:
            S.spfm_destroy_grid(h)
    assert S.spfm_kernels_per_step(None) == -1


def test_create_grid_validation(lib):
    d = _desc(nx=0)
    with pytest.raises(S.SpfmError) as e:
        S.spfm_create_grid(d)
    assert e.value.status == S.SPFM_EINVAL
    d = _desc(n=(1.0, 1.0, 0.0))
    d.field[0], d.field[1], d.scratch, d.scratch_bytes = 0x10000, 0x20000, 0x30000, 1 << 20
    with pytest.raises(S.SpfmError) as e:
        S.spfm_create_grid(d)
    assert "|n|" in str(e.value)
    d = _desc(bc=(S.SPFM_PERIODIC, S.SPFM_NOFLUX) + (S.SPFM_PERIODIC,) * 4)
    d.field[0], d.field[1], d.scratch, d.scratch_bytes = 0x10000, 0x20000, 0x30000, 1 << 20
    with pytest.raises(S.SpfmError):
        S.spfm_create_grid(d)
    d = _desc()
    d.field[0], d.field[1], d.scratch, d.scratch_bytes = 0x10008, 0x20000, 0x30000, 1 << 20
    with pytest.raises(S.SpfmError):
        S.spfm_create_grid(d)      # unaligned field
    d = _desc()
    d.field[0], d.field[1], d.scratch, d.scratch_bytes = 0x10000, 0x20000, 0x30000, 8
    with pytest.raises(S.SpfmError) as e:
        S.spfm_create_grid(d)
    assert e.value.status == S.SPFM_ENOMEM


def test_step_validation_before_any_launch(lib):
    h = _fake_grid(lib)
    try:
        with pytest.raises(S.SpfmError) as e:
            S.spfm_step(h, 1, 1.0, 1.0, 4.0, 1.0, 0.1, 0.0, 7, S.SPFM_TI_GLOBAL)
        assert e.value.status == S.SPFM_EINVAL
        with pytest.raises(S.SpfmError) as e:
            S.spfm_step(h, 1, 1.0, 1.0, -4.0, 1.0, 0.1, 0.0, 26, S.SPFM_TI_GLOBAL)
        assert e.value.status == S.SPFM_EINVAL
        # 7-point, D = M = 1: Laplacian spectral radius 12 -> dt must stay below 1/6
        with pytest.raises(S.SpfmError) as e:
            S.spfm_step(h, 1, 1.0, 1.0, 4.0, 1.0, 0.2, 0.0, 6, S.SPFM_FD)
        assert e.value.status == S.SPFM_EUNSTABLE
    finally:
        S.spfm_destroy_grid(h)


def test_phase_stability_limit_of_cf(lib):
    """Sec. 3.1: CF + h3 needs |dF dx/Gamma| < 8/(3 C_Gamma lambda/dx)."""
    h = _fake_grid(lib)
    try:
        lam, Cg = 4.0, 2.0 / 3.0
        limit = 8.0 / (3.0 * Cg * lam)
        with pytest.raises(S.SpfmError) as e:
            S.spfm_step(h, 0, 1.0, 1.0, lam, 1.0, 0.01, 1.001 * limit, 26, S.SPFM_FD)
        assert e.value.status == S.SPFM_EPHASE
        # just below the limit passes validation (0 steps: nothing is launched)
        S.spfm_step(h, 0, 1.0, 1.0, lam, 1.0, 0.01, 0.999 * limit, 26, S.SPFM_FD)
        # TI has no such limit in this form
        S.spfm_step(h, 0, 1.0, 1.0, lam, 1.0, 0.01, 1.5 * limit, 26, S.SPFM_TI_GLOBAL)
    finally:
        S.spfm_destroy_grid(h)


def test_euler_bound_matches_spectral_radius(lib):
    """The EUNSTABLE bound uses the exact spectral radius of the Laplacian part
    (6.67 D for the default 26-neighbour weights) plus the potential curvature."""
    h = _fake_grid(lib, n=(1.0, 0.0, 0.0))
    try:
        lam = 40.0   # potential curvature small at large lambda
        # D = 1: c1 = 1/2, c2 = 1/12, c3 = 1/24; bound = 20/3 + pot
        pot = 0.0
        w = [0.5] * 3 + [1.0 / 12] * 6 + [1.0 / 24] * 4     # c_k = D w_k / |r_k|^2
        d = [(1, 0, 0), (0, 1, 0), (0, 0, 1), (1, 1, 0), (0, 1, 1), (1, 0, 1), (1, -1, 0), (0, 1, -1),
             (1, 0, -1), (1, 1, 1), (-1, 1, 1), (1, -1, 1), (1, 1, -1)]
        for k in range(13):
            a = math.tanh(2.0 * d[k][0] / lam)
            pot += 4 * w[k] * a * a / (1 - a * a)
        bound = 20.0 / 3.0 + pot
        S.spfm_step(h, 0, 1.0, 1.0, lam, 1.0, 0.999 * 2 / bound, 0.0, 26, S.SPFM_TI_GLOBAL)
        with pytest.raises(S.SpfmError) as e:
            S.spfm_step(h, 0, 1.0, 1.0, lam, 1.0, 1.001 * 2 / bound, 0.0, 26, S.SPFM_TI_GLOBAL)
        assert e.value.status == S.SPFM_EUNSTABLE
    finally:
        S.spfm_destroy_grid(h)


def test_rounding_mode_validation(lib):
    """Stochastic rounding is for FP32 and BF16 storage; unknown modes are refused."""
    for dtype in (S.SPFM_F32, S.SPFM_BF16):
        h = _fake_grid(lib, dtype=dtype)
        assert lib.spfm_set_rounding(h, S.SPFM_ROUND_STOCHASTIC, 12345) == S.SPFM_OK
        assert lib.spfm_set_rounding(h, S.SPFM_ROUND_NEAREST, 0) == S.SPFM_OK
        assert lib.spfm_set_rounding(h, 7, 0) == S.SPFM_EINVAL
        lib.spfm_destroy_grid(h)
    h = _fake_grid(lib, dtype=S.SPFM_F64)
    assert lib.spfm_set_rounding(h, S.SPFM_ROUND_STOCHASTIC, 1) == S.SPFM_EINVAL
    assert b"FP32 and BF16" in lib.spfm_last_error(h)
    assert lib.spfm_set_rounding(h, S.SPFM_ROUND_NEAREST, 1) == S.SPFM_OK
    lib.spfm_destroy_grid(h)
    assert lib.spfm_set_rounding(None, S.SPFM_ROUND_NEAREST, 0) == S.SPFM_EINVAL


def test_zchunk_validation(lib):
    """The z-chunk knob takes 0 (per launch) or any positive plane count."""
    h = _fake_grid(lib)
    assert lib.spfm_last_zchunk(h) == 0          # no step launched yet
    for zc in (0, 1, 7, 10 ** 6):
        assert lib.spfm_set_zchunk(h, zc) == S.SPFM_OK
    assert lib.spfm_set_zchunk(h, -1) == S.SPFM_EINVAL
    assert b"zchunk" in lib.spfm_last_error(h)
    lib.spfm_destroy_grid(h)
    assert lib.spfm_set_zchunk(None, 0) == S.SPFM_EINVAL
    assert lib.spfm_last_zchunk(None) == -1


def _dispatch_makespan(tiles, nz, zc, slots, h=1, w=2):
    """Greedy dispatch, CTA by CTA in launch order (z-chunks outermost), of the
    launch's CTAs to `slots` slots: a CTA takes its planes + h units, w more
    when it had to wait for a slot."""
    free = [0] * slots
    end, n = 0, 0
    for c in range(-(-nz // zc)):
        d = min(zc, nz - c * zc) + h
        for _ in range(tiles):
            t = heapq.heappop(free) + (w if n >= slots else 0)
            heapq.heappush(free, t + d)
            end, n = max(end, t + d), n + 1
    return end


def test_zchunk_model_is_the_dispatch_argmin(lib):
    """For launches of few rounds the chunk length is the one of 4..64 planes
    whose greedy dispatch ends first (ties to the longer chunk), checked against
    a CTA-by-CTA simulation; launches of many rounds, and kernels with fewer
    than three CTAs per SM, take about `target` CTAs in chunks of 16 planes or
    more."""
    rng = random.Random(3)
    for _ in range(40):
        tiles, nz = rng.randint(1, 40), rng.randint(5, 120)
        per_sm, sms = rng.choice([3, 4]), rng.choice([2, 5, 9])
        slots, target = per_sm * sms, 6 * 4 * sms
        got = lib.spfm_debug_pick_zchunk(tiles, nz, per_sm, sms, target)
        if tiles * -(-nz // 16) >= 4 * slots:
            chunks = max(1, min(-(-target // tiles), max(1, nz // 16)))
            assert got == -(-nz // chunks)
        else:
            spans = {z: _dispatch_makespan(tiles, nz, z, slots) for z in range(4, min(nz, 64) + 1)}
            best = min(spans.values())
            assert got == max(z for z, v in spans.items() if v == best), (tiles, nz, slots, got)


@pytest.mark.parametrize("tiles,nz,per_sm,want", [
    (16, 128, 4, 4),      # 128^3 FP32 (64 x 16 tiles): 32 chunks fill one round
    (30, 160, 4, 8),
    (36, 192, 4, 12),
    (56, 224, 4, 22),
    (64, 256, 4, 28),     # 256^3 tilted plane: 576 CTAs + 64 of 4 planes
    (256, 512, 4, 35),    # 512^3: many rounds, 3840 CTAs of 35 planes
    (64, 256, 2, 16),     # TI_n (two CTAs per SM): the rule of many rounds
    (64, 3, 4, 3),        # a grid of at most 4 planes is one chunk
])
def test_zchunk_model_picks_measured_lengths(lib, tiles, nz, per_sm, want):
    """The lengths the model gives the GB300 (152 SMs) launches that were swept;
    each is the measured best or within 1 % of it."""
    assert lib.spfm_debug_pick_zchunk(tiles, nz, per_sm, 152, 6 * 4 * 152) == want


def test_zchunk_model_refuses_bad_arguments(lib):
    assert lib.spfm_debug_pick_zchunk(0, 10, 4, 152, 100) == -1
    assert lib.spfm_debug_pick_zchunk(4, 10, 0, 152, 100) == -1


def test_last_error_is_thread_local_without_grid(lib):
    with pytest.raises(S.SpfmError):
        S.spfm_layout(_desc(dtype=9))
    assert "dtype" in S.spfm_last_error(None)


def test_phase_stability_of_the_other_cf_models(lib):
    """Tab. 2 CF variants: h_Abel keeps a barrier below |dF~| = 8/(C_Gamma lambda~)
    (the barrier criterion of Sec. 3.1 applied to h_Abel; reading r20), h5 at
    any dF; spfm_max_dt answers the same validation without a launch."""
    h = _fake_grid(lib)
    try:
        lam, Cg = 4.0, 2.0 / 3.0
        limit = 8.0 / (Cg * lam)
        with pytest.raises(S.SpfmError) as e:
            S.spfm_step(h, 0, 1.0, 1.0, lam, 1.0, 0.001, 1.001 * limit, 26, S.SPFM_FD_HABEL)
        assert e.value.status == S.SPFM_EPHASE
        S.spfm_step(h, 0, 1.0, 1.0, lam, 1.0, 0.001, 0.999 * limit, 26, S.SPFM_FD_HABEL)
        S.spfm_step(h, 0, 1.0, 1.0, lam, 1.0, 0.001, 50 * limit, 26, S.SPFM_FD_H5)
        with pytest.raises(S.SpfmError) as e:
            S.spfm_max_dt(h, 1.0, 1.0, lam, 1.0, 1.001 * limit, 26, S.SPFM_FD_HABEL)
        assert e.value.status == S.SPFM_EPHASE
        for scheme in (S.SPFM_FD, S.SPFM_FD_H5, S.SPFM_FD_HABEL, S.SPFM_TI_GLOBAL, S.SPFM_TI_LOCAL):
            dt = S.spfm_max_dt(h, 1.0, 1.0, lam, 1.0, 0.01, 26, scheme)
            S.spfm_step(h, 0, 1.0, 1.0, lam, 1.0, 0.999 * dt, 0.01, 26, scheme)
            with pytest.raises(S.SpfmError) as e:
                S.spfm_step(h, 0, 1.0, 1.0, lam, 1.0, 1.001 * dt, 0.01, 26, scheme)
            assert e.value.status == S.SPFM_EUNSTABLE
        with pytest.raises(S.SpfmError) as e:
            S.spfm_step_conserving(h, 0, 1.0, 1.0, lam, 1.0, 0.01, 26, S.SPFM_FD_H5)
        assert e.value.status == S.SPFM_EINVAL
    finally:
        S.spfm_destroy_grid(h)


def test_fp32_band_limits_are_the_floats_next_to_the_fp64_limits():
    """The stats kernel tests an FP32 cell against the first float above 1e-6
    and the last float below 1 - 1e-6 (hex literals in stats.cu); those are
    the floats that select exactly the cells with 1e-6 < phi < 1 - 1e-6."""
    src = open(os.path.join(ROOT, "paper_1910_05180_gb300", "csrc", "stats.cu")).read()
    m = re.search(r"return x >= (0x[0-9a-fp.+-]+)f && x <= (0x[0-9a-fp.+-]+)f;", src)
    lo, hi = float.fromhex(m.group(1)), float.fromhex(m.group(2))
    f32 = np.float32
    assert f32(lo) == lo and f32(hi) == hi
    assert lo > 1e-6 and float(np.nextafter(f32(lo), f32(0))) <= 1e-6
    assert hi < 1 - 1e-6 and float(np.nextafter(f32(hi), f32(1))) >= 1 - 1e-6
