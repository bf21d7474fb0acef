"""cc_energy_noalloc: the energy for callers that cannot allocate device memory.

Its block partial sums live in a fixed device array of the library instead of
a caller workspace.  This file sorts last so that, in a run that stops at the
first failure, every other test has already run; it passes alone in a fresh
process as well.  Checked through the C ABI against cc_energy (which takes a
workspace) on two calls in a row, within the energy tolerance of the other
GPU tests (1e-13 Eh); and the size limit is enforced before any pointer is read.
"""
import numpy as np
import pytest
import torch

import ccinputs
from gpu_util import DEV, small_case, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cc():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2409_06759_b300 as cc
    from paper_2409_06759_b300 import engine
    return cc, engine


@pytest.mark.parametrize("o,v,seed", [(5, 9, 61), (10, 40, 62)])
def test_noalloc_energy_matches_workspace_energy_twice(cc, o, v, seed):
    ccm, engine = cc
    s, B, t1, t2 = small_case(o, v, seed, L=8, scale=6.0, tscale=0.05)
    eng = engine.Engine(engine.DeviceSystem(o, v, s.eps_occ, s.eps_vir, B, device=DEV))
    T1, T2 = to_dev(t1), to_dev(t2)
    ref = torch.zeros(2, dtype=torch.float64, device=DEV)
    ccm.cc_energy(eng.plan, eng.sys.ints(), T1, T2, ref, eng.ws)
    for call in range(2):
        e = torch.full((2,), np.nan, dtype=torch.float64, device=DEV)
        ccm.cc_energy_noalloc(o, v, eng.sys.ints(), T1, T2, e)
        torch.cuda.synchronize()
        assert abs(e[0].item() - ref[0].item()) < 1e-13, call
        assert e[1].item() == 0.0


def test_noalloc_energy_without_t1(cc):
    ccm, engine = cc
    o, v = 4, 7
    s, B, t1, t2 = small_case(o, v, 63)
    eng = engine.Engine(engine.DeviceSystem(o, v, s.eps_occ, s.eps_vir, B, device=DEV))
    T2 = to_dev(t2)
    ref = torch.zeros(2, dtype=torch.float64, device=DEV)
    ccm.cc_energy(eng.plan, eng.sys.ints(), None, T2, ref, eng.ws)
    e = torch.zeros(2, dtype=torch.float64, device=DEV)
    ccm.cc_energy_noalloc(o, v, eng.sys.ints(), None, T2, e)
    torch.cuda.synchronize()
    assert abs(e[0].item() - ref[0].item()) < 1e-13


def test_noalloc_energy_rejects_oversize(cc):
    ccm, _ = cc
    o, v = 50, 200                 # o^2 v^2 = 1e8 > 67,108,864
    n = o * o * v * v
    big = torch.zeros(n, dtype=torch.float64, device=DEV)   # valid memory even if it were read
    t1 = torch.zeros(o, v, dtype=torch.float64, device=DEV)
    e = torch.zeros(2, dtype=torch.float64, device=DEV)
    f = torch.zeros(o + v, dtype=torch.float64, device=DEV)
    with pytest.raises(ccm.CCError) as ei:
        ccm.cc_energy_noalloc(o, v, dict(f_occ=f, f_vir=f, oovv=big), t1, big, e)
    assert ei.value.status == 1
    assert "no-allocation limit" in str(ei.value)
