"""FP64 path on the GPU vs the FP64 oracle (parity), through the C ABI.

Tolerances: the residual elements within 1e-9 and the energy within 1e-10 Eh
(the stated FP64-path bar); both sides compute in FP64, so the observed gaps
are rounding-order differences of ~1e-15 relative.
"""
import numpy as np
import pytest
import torch

import ccinputs
import oracle
from gpu_util import DEV, block_slices, oracle_V, small_case, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cc():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2409_06759_b300 as cc
    from paper_2409_06759_b300 import engine
    return cc, engine


@pytest.mark.parametrize("o,v,L", [(1, 1, 3), (2, 3, 5), (4, 6, 6), (7, 19, 9), (10, 40, 120)])
def test_integral_blocks_match_oracle(cc, o, v, L):
    _, engine = cc
    s = ccinputs.make_system(o, v, L=L, seed=3)
    B = s.B * 6.0
    dsys = engine.DeviceSystem(o, v, s.eps_occ, s.eps_vir, B, device=DEV)
    ref = block_slices(oracle_V(o, v, B), o)
    for nm, blk in ref.items():
        got = dsys.block(nm).cpu().numpy()
        assert np.abs(got - blk).max() <= 1e-14 + 1e-13 * np.abs(blk).max(), nm


@pytest.mark.parametrize("list_name", ["ccsd", "ccsd_vvvv"])
@pytest.mark.parametrize("o,v,seed", [(1, 2, 1), (2, 3, 2), (3, 5, 3), (5, 7, 4), (4, 17, 5), (6, 70, 6),
                                      (10, 40, 7)])
def test_residual_matches_oracle(cc, list_name, o, v, seed):
    _, engine = cc
    s, B, t1, t2 = small_case(o, v, seed, L=8 if v < 40 else 120, scale=6.0 if v < 40 else 1.0)
    dsys = engine.DeviceSystem(o, v, s.eps_occ, s.eps_vir, B, device=DEV)
    eng = engine.Engine(dsys, list_name=list_name)
    r1, r2 = eng.residual(to_dev(t1), to_dev(t2))
    torch.cuda.synchronize()
    V = oracle_V(o, v, B)
    o1, o2 = oracle.ccsd_residual(o, v, s.eps, V, t1, t2)
    g1, g2 = r1.cpu().numpy(), r2.cpu().numpy()
    assert np.abs(g1 - o1).max() < 1e-9
    assert np.abs(g2 - o2).max() < 1e-9
    scale = max(np.abs(o1).max(), np.abs(o2).max())
    assert np.abs(g2 - o2).max() <= 1e-12 * scale
    # antisymmetry holds exactly enough
    assert np.abs(g2 + g2.transpose(1, 0, 2, 3)).max() <= 1e-13 * scale
    assert np.abs(g2 + g2.transpose(0, 1, 3, 2)).max() <= 1e-13 * scale


def test_energy_matches_oracle(cc):
    _, engine = cc
    o, v = 5, 9
    s, B, t1, t2 = small_case(o, v, 11)
    dsys = engine.DeviceSystem(o, v, s.eps_occ, s.eps_vir, B, device=DEV)
    eng = engine.Engine(dsys)
    e = eng.energy(to_dev(t1), to_dev(t2))
    ref = oracle.ccsd_energy(o, v, oracle_V(o, v, B), t1, t2)
    assert abs(e - ref) < 1e-13


def test_residual_is_repeatable_bitwise(cc):
    _, engine = cc
    o, v = 4, 11
    s, B, t1, t2 = small_case(o, v, 12)
    eng = engine.Engine(engine.DeviceSystem(o, v, s.eps_occ, s.eps_vir, B, device=DEV))
    a = [x.clone() for x in eng.residual(to_dev(t1), to_dev(t2))]
    b = eng.residual(to_dev(t1), to_dev(t2))
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])


@pytest.mark.parametrize("list_name", ["ccsd", "ccsd_vvvv"])
def test_solve_small_config_matches_oracle(cc, list_name):
    """o=10, v=40, L=120 (the small CCSD workload): same Jacobi+DIIS trajectory."""
    _, engine = cc
    s = ccinputs.make_system(**ccinputs.CONFIG_SMALL)
    o, v = s.o, s.v
    dsys = engine.DeviceSystem.from_system(s, device=DEV)
    sol = engine.Solver(engine.Engine(dsys, list_name=list_name))
    z1 = torch.zeros(o, v, dtype=torch.float64, device=DEV)
    z2 = torch.zeros(o, o, v, v, dtype=torch.float64, device=DEV)
    res = sol.solve(z1, z2, max_iter=60, tol=1e-8)
    ref = oracle.ccsd_solve(o, v, s.eps, oracle_V(o, v, s.B), tol=1e-8, maxiter=60)
    assert res.converged and ref["status"] == 0
    assert res.iterations == ref["iters"]
    assert np.abs(np.array(res.energies) - ref["energies"]).max() < 1e-12
    assert abs(res.energy - ref["energy"]) < 1e-10
    assert np.abs(z2.cpu().numpy() - ref["t2"]).max() < 1e-10


def test_solve_two_electrons_equals_fci(cc):
    import detspace
    _, engine = cc
    o, v = 2, 6
    s = ccinputs.make_system(o, v, L=6, seed=12)
    B = s.B * 6.0
    dsys = engine.DeviceSystem(o, v, s.eps_occ, s.eps_vir, B, device=DEV)
    sol = engine.Solver(engine.Engine(dsys))
    z1 = torch.zeros(o, v, dtype=torch.float64, device=DEV)
    z2 = torch.zeros(o, o, v, v, dtype=torch.float64, device=DEV)
    res = sol.solve(z1, z2, max_iter=100, tol=1e-12)
    assert res.converged
    assert abs(res.energy - detspace.fci_correlation(o, v, s.eps, oracle_V(o, v, B))) < 1e-12


def test_solve_resume_continues_the_same_trajectory(cc):
    _, engine = cc
    o, v = 4, 12
    s, B, _, _ = small_case(o, v, 13)
    dsys = engine.DeviceSystem(o, v, s.eps_occ, s.eps_vir, B, device=DEV)
    eng = engine.Engine(dsys)
    z = lambda: (torch.zeros(o, v, dtype=torch.float64, device=DEV),
                 torch.zeros(o, o, v, v, dtype=torch.float64, device=DEV))
    a1, a2 = z()
    straight = engine.Solver(eng).solve(a1, a2, max_iter=7, tol=0.0)
    b1, b2 = z()
    sol = engine.Solver(eng)
    p1 = sol.solve(b1, b2, max_iter=3, tol=0.0)
    p2 = sol.solve(b1, b2, max_iter=4, tol=0.0, resume=True)
    assert np.allclose(p1.energies + p2.energies, straight.energies, rtol=0, atol=1e-14)
    assert torch.allclose(a2, b2, rtol=0, atol=1e-15)


def test_bad_arguments_return_status(cc):
    ccm, engine = cc
    o, v = 3, 4
    s, B, t1, t2 = small_case(o, v, 14)
    eng = engine.Engine(engine.DeviceSystem(o, v, s.eps_occ, s.eps_vir, B, device=DEV))
    r1 = torch.empty(o, v, dtype=torch.float64, device=DEV)
    r2 = torch.empty(o, o, v, v, dtype=torch.float64, device=DEV)
    small_ws = torch.empty(4, dtype=torch.float64, device=DEV)
    with pytest.raises(ccm.CCError) as ei:
        ccm.cc_residual(eng.plan, eng.sys.ints(), to_dev(t1), to_dev(t2), r1, r2, small_ws)
    assert ei.value.status == 9
    with pytest.raises(ccm.CCError) as ei:
        ccm.cc_residual(eng.plan, eng.sys.ints(), None, to_dev(t2), r1, r2, eng.ws)
    assert ei.value.status == 1
