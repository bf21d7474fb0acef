"""Failure detection without a GPU fault: the tensor-core kernels' bounded
mbarrier wait, made to run out on a barrier nothing arrives at, returns a
timeout status to the host and leaves the context usable."""
import numpy as np
import pytest
import torch

import oracle
from gpu_util import DEV, oracle_V, small_case, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cc():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2409_06759_b300 as cc
    from paper_2409_06759_b300 import engine
    return cc, engine


def test_bounded_wait_times_out_and_context_survives(cc):
    ccm, engine = cc
    assert ccm.cc_selftest_wait_timeout(2_000_000) == 8          # CC_ERR_TIMEOUT: the wait gave up
    assert "as designed" in ccm.cc_last_error()
    # the context still runs work (tensor-core route included)
    o, v = 3, 8
    s, B, t1, t2 = small_case(o, v, 3, L=6, scale=6.0, tscale=0.05)
    dsys = engine.DeviceSystem(o, v, s.eps_occ, s.eps_vir, B, device=DEV)
    eng = engine.Engine(dsys, list_name="ccsd_vvvv", precision="bf16x6", route_all=True)
    r1, r2 = eng.residual(to_dev(t1), to_dev(t2))
    torch.cuda.synchronize()
    o1, o2 = oracle.ccsd_residual(o, v, s.eps, oracle_V(o, v, B), t1, t2)
    assert np.abs(r2.cpu().numpy() - o2).max() <= 1e-5 * np.abs(o2).max()
