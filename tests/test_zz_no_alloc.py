"""cc_energy_noalloc: the energy for callers that cannot allocate device memory
(code under a host application that owns the device heap, or in a region where
a cudaMalloc would be refused or would synchronise the device).

Its block partial sums live in a fixed device array of the library instead of
a caller workspace.  This file sorts last so that, in a run that stops at the
first failure, every other test has already run; it passes alone in a fresh
process as well.  Checked through the C ABI against cc_energy (which takes a
workspace) on two calls in a row, within the energy tolerance of the other
GPU tests (1e-13 relative), for FP64 and complex128, at sizes up to the
o=40 v=200 system (3907 of the 4096 partials) where it is also compared with
the oracle's energy; and the size limit is enforced before any pointer is
read.
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


def _twice_against_cc_energy(ccm, eng, o, v, T1, T2, cplx):
    ref = torch.zeros(2, dtype=torch.float64, device=DEV)
    ccm.cc_energy(eng.plan, eng.sys.ints(), T1, T2, ref, eng.ws)
    out = []
    for call in range(2):
        e = torch.full((2,), np.nan, dtype=torch.float64, device=DEV)
        ccm.cc_energy_noalloc(o, v, eng.sys.ints(), T1, T2, e)
        torch.cuda.synchronize()
        got, want = e.cpu().numpy(), ref.cpu().numpy()
        scale = max(abs(want[0]), abs(want[1]), 1e-300)
        assert abs(got[0] - want[0]) <= 1e-13 * scale, call
        if cplx:
            assert abs(got[1] - want[1]) <= 1e-13 * scale, call
        else:
            assert got[1] == 0.0
        out.append(got)
    return out


@pytest.mark.parametrize("o,v,seed", [(5, 9, 61), (10, 40, 62)])
def test_noalloc_energy_matches_workspace_energy_twice(cc, o, v, seed):
    ccm, engine = cc
    s, B, t1, t2 = small_case(o, v, seed, L=8, scale=6.0, tscale=0.05)
    eng = engine.Engine(engine.DeviceSystem(o, v, s.eps_occ, s.eps_vir, B, device=DEV))
    _twice_against_cc_energy(ccm, eng, o, v, to_dev(t1), to_dev(t2), False)


def test_noalloc_complex_energy_matches_workspace_energy_twice(cc):
    ccm, engine = cc
    o, v = 6, 23
    s = ccinputs.make_system(o, v, L=8, seed=64, complex_=True)
    t1, t2 = ccinputs.random_amplitudes(o, v, seed=64, scale1=0.05, scale2=0.05, complex_=True)
    eng = engine.Engine(engine.DeviceSystem(o, v, s.eps_occ, s.eps_vir, s.B * 6.0, device=DEV))
    z = lambda x: torch.tensor(np.ascontiguousarray(x), dtype=torch.complex128, device=DEV)
    got = _twice_against_cc_energy(ccm, eng, o, v, z(t1), z(t2), True)
    assert abs(got[0][1]) > 0.0


@pytest.mark.slow
def test_noalloc_energy_at_the_benchmark_size(cc):
    """o=40, v=200: 3907 of the 4096 partials; against cc_energy and against
    the oracle's energy of the same amplitudes (block oracle, from B)."""
    from oracle import cc_blocks
    ccm, engine = cc
    s = ccinputs.make_system(**ccinputs.CONFIG_LADDER)
    o, v = s.o, s.v
    t1, t2 = ccinputs.random_amplitudes(o, v, seed=3, scale1=0.01, scale2=0.01)
    # a one-statement plan: cc_energy takes its scratch from this plan's small workspace
    eng = engine.Engine(engine.DeviceSystem(o, v, s.eps_occ, s.eps_vir, s.B, device=DEV, blocks=("oovv",)),
                        list_text="R2[ijab] = 0.25 V[ijab]")
    got = _twice_against_cc_energy(ccm, eng, o, v, to_dev(t1), to_dev(t2), False)
    want = cc_blocks.ccsd_energy(o, v, cc_blocks.integral_blocks(o, v, s.B, names=("oovv",)), t1, t2)
    assert abs(got[1][0] - want) <= 1e-12 * abs(want)


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
    assert abs(e[0].item() - ref[0].item()) < 1e-13 * abs(ref[0].item())


def test_noalloc_energy_rejects_oversize_before_reading(cc):
    """o^2 v^2 = 1e8 > 67,108,864: rejected on the host with the limit message.
    The integral and amplitude pointers are NULL, so a size check that let the
    call through would stop at the host's pointer check (another message, this
    test fails) without launching anything."""
    ccm, _ = cc
    o, v = 50, 200
    one = torch.zeros(1, dtype=torch.float64, device=DEV)
    e = torch.zeros(2, dtype=torch.float64, device=DEV)
    for dt in (ccm.CC_F64, ccm.CC_C128):
        with pytest.raises(ccm.CCError) as ei:
            ccm.cc_energy_noalloc(o, v, dict(f_occ=one, f_vir=one), None, None, e, dtype=dt)
        assert ei.value.status == 1
        assert "no-allocation limit" in str(ei.value)


def test_noalloc_energy_rejects_an_unknown_dtype(cc):
    ccm, _ = cc
    one = torch.zeros(1, dtype=torch.float64, device=DEV)
    e = torch.zeros(2, dtype=torch.float64, device=DEV)
    with pytest.raises(ccm.CCError) as ei:
        ccm.cc_energy_noalloc(1, 1, dict(f_occ=one, f_vir=one), None, None, e, dtype=7)
    assert ei.value.status == 1
