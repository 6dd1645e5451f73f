"""Failure reporting of the step kernel's bounded waits, made to run out on the
device without a fault: spfm_debug_skip_copy makes the next step's first CTA
skip one plane's copy, so its consumers' wait for that stage gives up (after
about 2 s); the kernel still waits for every copy it did issue, returns, and
the next stats call reports SPFM_ETIMEOUT.  The context stays usable: after a
re-initialisation the same grid steps normally and matches the oracle.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1910_05180_gb300 import spfm as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    S.load()


@pytest.mark.parametrize("bc", [(S.SPFM_PERIODIC,) * 6, (S.SPFM_CONTACT,) * 6])
def test_bounded_wait_gives_up_and_reports_timeout(bc):
    n = np.array([1.0, 0.4, 0.2])
    n /= np.linalg.norm(n)
    shape = (64, 32, 40)          # periodic: the image-writing kernel; contact: face kernel after
    c = float(n @ (np.array(shape) - 1) / 2.0)
    kw = dict(lam=3.0, dt=0.05, dF=0.02, stencil=26)
    g = S.Grid(*shape, dtype=S.SPFM_F32, bc=bc, n=tuple(n))
    g.init_planar(c, 3.0)
    g.step(2, **kw)
    assert g.stats()["nonfinite"] == 0.0           # no error before the hook
    S.spfm_debug_skip_copy(g.handle)
    g.step(3, **kw)
    with pytest.raises(S.SpfmError) as e:
        g.stats()
    assert e.value.status == S.SPFM_ETIMEOUT
    torch.cuda.synchronize()                       # the context still answers
    # one-shot: after a re-initialisation the grid steps normally
    g.init_planar(c, 3.0)
    g.step(10, **kw)
    g.stats()
    p = O.Params(*shape, bc=bc, n=tuple(n), lam=3.0, dt=0.05, dF=0.02, stencil=26)
    start = O.init_planar(p, c).astype(np.float32).astype(np.float64)
    ref = O.step(p, start, 10)
    err = np.abs(g.get_field(to_host=True).double().numpy() - ref).max()
    assert err <= 2e-5, err
