"""The diagnostics entry point that allocates nothing.

Some callers cannot allocate device memory (their memory belongs to another
framework's pool, or they only borrow the field they measure).  For them
spfm_interface_stats_static reduces into a fixed array inside the library.
This checks it, through the C ABI, against spfm_interface_stats on the same
field, on two calls in a row (the array keeps the previous call's contents).
"""
import numpy as np
import pytest
import torch

from paper_1910_05180_gb300 import spfm as S

pytestmark = pytest.mark.gpu

KEYS = ("volume", "S_w", "S_c", "S_r", "phi_min", "phi_max", "nonfinite", "position", "radius")


@pytest.mark.parametrize("dtype", [S.SPFM_F32, S.SPFM_F64])
def test_static_stats_match_grid_stats_twice(dtype):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    S.load()
    n = np.array([1.0, 0.6, 0.3])
    n /= np.linalg.norm(n)
    g = S.Grid(70, 45, 33, dtype=dtype, bc=(S.SPFM_CONTACT,) * 6, n=tuple(n), center=(30.0, 20.0, 15.0))
    g.init_planar(float(n @ [34.5, 22, 16]), 2.5)
    g.step(30, lam=2.5, dt=0.05, dF=0.03, stencil=26)
    ref = g.stats()
    buf = g.fields[S.spfm_current(g.handle)]
    for _ in range(2):
        got = S.spfm_interface_stats_static(g.desc, buf.data_ptr(), 2.5, 1.0)
        for k in KEYS:
            assert abs(got[k] - ref[k]) <= 1e-12 * max(1.0, abs(ref[k])), (k, got[k], ref[k])
    # a second, smaller field right after: nothing of the first call leaks in
    g2 = S.Grid(20, 12, 9, dtype=dtype, bc=(S.SPFM_CONTACT,) * 6, n=tuple(n))
    g2.init_planar(float(n @ [9.5, 5.5, 4]), 2.0)
    g2.step(0, lam=2.0, dt=0.05)
    ref2 = g2.stats()
    got2 = S.spfm_interface_stats_static(g2.desc, g2.fields[0].data_ptr(), 2.0, 1.0)
    for k in KEYS:
        assert abs(got2[k] - ref2[k]) <= 1e-12 * max(1.0, abs(ref2[k])), (k, got2[k], ref2[k])


def test_static_stats_reject_too_many_planes():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    S.load()
    d = S.GridDesc()
    d.nx, d.ny, d.nz, d.dtype = 4, 4, 1025, S.SPFM_F32
    d.n[0] = 1.0
    with pytest.raises(S.SpfmError) as e:
        S.spfm_interface_stats_static(d, 256, 2.0, 1.0)
    assert e.value.status == S.SPFM_EINVAL and "1024" in str(e.value)
