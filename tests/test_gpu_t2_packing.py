"""cc_pack_t2 / cc_unpack_t2: the doubles amplitudes in their i < j, a < b
quarter (the antisymmetry of Eq. amp) and back, through the C ABI.  Packing
is a gather and unpacking a gather with sign flips, so both are checked bit for
bit: against the packed array formed on the host with the pair index, and as
a round trip that must return the antisymmetric input exactly."""
import numpy as np
import pytest
import torch

import ccinputs
from gpu_util import DEV

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cc():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2409_06759_b300 as cc
    return cc


def _pairs(n):
    return [(p, q) for p in range(n) for q in range(p + 1, n)]


@pytest.mark.parametrize("complex_", [False, True])
@pytest.mark.parametrize("o,v", [(5, 45), (2, 70), (1, 33), (12, 100), (3, 2)])
def test_pack_and_unpack_t2(cc, o, v, complex_):
    _, t2 = ccinputs.random_amplitudes(o, v, seed=o * 100 + v, scale1=0.1, scale2=0.1, complex_=complex_)
    dt = torch.complex128 if complex_ else torch.float64
    dtype = cc.CC_C128 if complex_ else cc.CC_F64
    n = cc.cc_packed_t2_elems(o, v)
    assert n == (o * (o - 1) // 2) * (v * (v - 1) // 2)
    full = torch.tensor(t2, dtype=dt, device=DEV)
    packed = torch.full((max(n, 1),), 7.0, dtype=dt, device=DEV)
    cc.cc_pack_t2(o, v, full, packed, dtype=dtype)
    back = torch.full((o, o, v, v), 3.0, dtype=dt, device=DEV)
    cc.cc_unpack_t2(o, v, packed, back, dtype=dtype)
    torch.cuda.synchronize()
    po, pv = _pairs(o), _pairs(v)
    want = np.array([t2[i, j, a, b] for (i, j) in po for (a, b) in pv]).reshape(len(po), len(pv))
    if n:
        assert np.array_equal(packed.cpu().numpy()[:n].reshape(len(po), len(pv)), want)
    assert np.array_equal(back.cpu().numpy(), t2)


def test_pack_rejects_bad_arguments(cc):
    x = torch.zeros(16, dtype=torch.float64, device=DEV)
    with pytest.raises(RuntimeError):
        cc.cc_pack_t2(0, 4, x, x)
    with pytest.raises(RuntimeError):
        cc.cc_unpack_t2(2, 2, x, x, dtype=99)
