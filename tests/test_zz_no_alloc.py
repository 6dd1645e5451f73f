"""The diagnostics entry point that allocates nothing.

Some callers cannot allocate device memory (their memory belongs to another
framework's pool, or they only borrow the field they measure).  For them
spfm_interface_stats_static reduces into a fixed array inside the library.
This checks it, through the C ABI, against spfm_interface_stats on the same
field, on two calls in a row (the array keeps the previous call's contents),
and against the oracle's sums of Sec. 2.3 on that field; and that it refuses
what it cannot serve.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1910_05180_gb300 import spfm as S

pytestmark = pytest.mark.gpu

KEYS = ("volume", "S_w", "S_c", "S_r", "phi_min", "phi_max", "nonfinite", "position", "radius")


def _close(got, ref, k, rel=1e-12):
    assert abs(got[k] - ref[k]) <= rel * max(1.0, abs(ref[k])), (k, got[k], ref[k])


@pytest.mark.parametrize("dtype", [S.SPFM_F32, S.SPFM_F64, S.SPFM_BF16])
def test_static_stats_match_grid_stats_and_oracle_twice(dtype):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    S.load()
    n = np.array([1.0, 0.6, 0.3])
    n /= np.linalg.norm(n)
    shape, ctr = (70, 45, 33), (30.0, 20.0, 15.0)
    g = S.Grid(*shape, dtype=dtype, bc=(S.SPFM_CONTACT,) * 6, n=tuple(n), center=ctr)
    g.init_planar(float(n @ [34.5, 22, 16]), 2.5)
    g.step(30, lam=2.5, dt=0.05, dF=0.03, stencil=26)
    ref = g.stats()
    buf = g.fields[S.spfm_current(g.handle)]
    # the oracle's sums on the same (stored) values
    p = O.Params(*shape, n=tuple(n), lam=2.5)
    ref_o = O.stats(p, g.get_field(to_host=True).double().numpy(), ctr)
    for _ in range(2):
        got = S.spfm_interface_stats_static(g.desc, buf.data_ptr(), 2.5, 1.0)
        for k in KEYS:
            _close(got, ref, k)
            _close(got, ref_o, k)
    # a second, smaller field right after: nothing of the first call leaks in
    g2 = S.Grid(20, 12, 9, dtype=dtype, bc=(S.SPFM_CONTACT,) * 6, n=tuple(n))
    g2.init_planar(float(n @ [9.5, 5.5, 4]), 2.0)
    g2.step(0, lam=2.0, dt=0.05)
    ref2 = g2.stats()
    got2 = S.spfm_interface_stats_static(g2.desc, g2.fields[0].data_ptr(), 2.0, 1.0)
    for k in KEYS:
        _close(got2, ref2, k)


def test_static_stats_reject_what_they_cannot_serve():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    S.load()
    d = S.GridDesc()
    d.nx, d.ny, d.nz, d.dtype = 4, 4, 1025, S.SPFM_F32
    d.n[0] = 1.0
    with pytest.raises(S.SpfmError) as e:
        S.spfm_interface_stats_static(d, 256, 2.0, 1.0)
    assert e.value.status == S.SPFM_EINVAL and "1024" in str(e.value)
    # a face above 2^30 cells, refused before any launch as spfm_create_grid does
    d.nx, d.ny, d.nz = 1 << 20, 1 << 10, 4
    with pytest.raises(S.SpfmError) as e:
        S.spfm_interface_stats_static(d, 256, 2.0, 1.0)
    assert e.value.status == S.SPFM_EINVAL and "2^30" in str(e.value)
    d.nx, d.ny, d.nz = 4, 4, 4
    d.n[0] = 0.5
    with pytest.raises(S.SpfmError) as e:
        S.spfm_interface_stats_static(d, 256, 2.0, 1.0)
    assert e.value.status == S.SPFM_EINVAL and "|n|" in str(e.value)
