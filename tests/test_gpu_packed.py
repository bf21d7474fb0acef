"""Packed index pairs (lists/ccsd_packed.txt): the particle ladder and the
tau<mn||ef> part of W_mnij over e < f, producing only i < j, a < b, against
the oracle (small sizes, every element), the unpacked plan (full size) and the
oracle's solve."""
import numpy as np
import pytest
import torch

import ccinputs
import oracle
from gpu_util import DEV, assert_elementwise, list_bounds, oracle_V, small_case, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cc():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2409_06759_b300 as cc
    from paper_2409_06759_b300 import engine
    return cc, engine


@pytest.mark.parametrize("o,v,seed", [(2, 3, 1), (3, 5, 2), (4, 9, 3), (7, 33, 4), (10, 40, 5)])
def test_packed_fp64_residual_matches_oracle(cc, o, v, seed):
    _, engine = cc
    s, B, t1, t2 = small_case(o, v, seed, L=8, scale=6.0, tscale=0.05)
    dsys = engine.DeviceSystem(o, v, s.eps_occ, s.eps_vir, B, device=DEV)
    eng = engine.Engine(dsys, list_name="ccsd_packed")
    r1, r2 = eng.residual(to_dev(t1), to_dev(t2))
    torch.cuda.synchronize()
    o1, o2 = oracle.ccsd_residual(o, v, s.eps, oracle_V(o, v, B), t1, t2)
    scale = max(np.abs(o1).max(), np.abs(o2).max())
    assert np.abs(r1.cpu().numpy() - o1).max() <= 1e-12 * scale
    assert np.abs(r2.cpu().numpy() - o2).max() <= 1e-12 * scale


@pytest.mark.parametrize("prec,rel", [("bf16x3", 2e-4), ("bf16x6", 2e-6)])
@pytest.mark.parametrize("o,v", [(3, 8), (6, 30)])
def test_packed_mixed_residual_matches_oracle(cc, prec, rel, o, v):
    """Every element within the element-wise bound of the packed plan's routes
    (a packed contraction sums half the pairs twice: the same bound with the
    packed K); the error norm as an extra check."""
    ccm, engine = cc
    s, B, t1, t2 = small_case(o, v, 7, L=8, scale=6.0, tscale=0.05)
    dsys = engine.DeviceSystem(o, v, s.eps_occ, s.eps_vir, B, device=DEV)
    eng = engine.Engine(dsys, list_name="ccsd_packed", precision=prec, route_all=True)
    r1, r2 = eng.residual(to_dev(t1), to_dev(t2))
    torch.cuda.synchronize()
    V = oracle_V(o, v, B)
    o1, o2 = oracle.ccsd_residual(o, v, s.eps, V, t1, t2)
    _, [(e1, e2)] = list_bounds(ccm.load_list("ccsd_packed"), o, v, s.eps, V, t1, t2, [eng.plan])
    assert_elementwise([r1, r2], [o1, o2], [e1, e2], what=f"packed {prec}")
    d = np.sqrt(np.sum((r1.cpu().numpy() - o1) ** 2) + np.sum((r2.cpu().numpy() - o2) ** 2))
    assert d <= rel * np.sqrt(np.sum(o1 ** 2) + np.sum(o2 ** 2))


def test_packed_solves_small_config(cc):
    """o=10, v=40: the packed FP64 plan reaches the oracle energy (1e-10 Eh);
    the packed bf16x6 plan refined by the packed FP64 plan too."""
    _, engine = cc
    s = ccinputs.make_system(**ccinputs.CONFIG_SMALL)
    o, v = s.o, s.v
    ref = oracle.ccsd_solve(o, v, s.eps, oracle_V(o, v, s.B), tol=1e-9, maxiter=60)
    dsys = engine.DeviceSystem.from_system(s, device=DEV)
    fp64 = engine.Engine(dsys, list_name="ccsd_packed")
    z = lambda: (torch.zeros(o, v, dtype=torch.float64, device=DEV),
                 torch.zeros(o, o, v, v, dtype=torch.float64, device=DEV))
    a1, a2 = z()
    r = engine.Solver(fp64).solve(a1, a2, max_iter=60, tol=1e-9)
    assert r.converged and abs(r.energy - ref["energy"]) < 1e-10
    mixed = engine.Engine(dsys, list_name="ccsd_packed", precision="bf16x6")
    b1, b2 = z()
    r2 = engine.Solver(mixed, refine=fp64).solve(b1, b2, max_iter=60, tol=1e-9, switch_tol=1e-7)
    assert r2.converged and abs(r2.energy - ref["energy"]) < 1e-10


@pytest.mark.slow
def test_packed_full_size_matches_unpacked(cc):
    """o=40, v=200: the packed FP64 residual against the unpacked one over the
    whole array and against sampled oracle elements."""
    _, engine = cc
    s = ccinputs.make_system(**ccinputs.CONFIG_LADDER)
    o, v = s.o, s.v
    t1, t2 = ccinputs.random_amplitudes(o, v, seed=0, scale1=0.01, scale2=0.01)
    dsys = engine.DeviceSystem.from_system(s, device=DEV)
    T1, T2 = to_dev(t1), to_dev(t2)
    p = engine.Engine(dsys, list_name="ccsd_packed")
    p1, p2 = p.residual(T1, T2)
    torch.cuda.synchronize()
    p1, p2 = p1.cpu(), p2.cpu()
    del p
    u = engine.Engine(dsys, list_name="ccsd_vvvv")
    u1, u2 = u.residual(T1, T2)
    torch.cuda.synchronize()
    u1, u2 = u1.cpu(), u2.cpu()
    n = max(u1.abs().max().item(), u2.abs().max().item())
    assert (p1 - u1).abs().max().item() <= 1e-12 * n and (p2 - u2).abs().max().item() <= 1e-12 * n
    idx = np.array([[0, 1, 0, 1], [o - 1, o - 2, v - 1, v - 2], [3, 17, 150, 42]])
    want = oracle.ccsd_r2_sample(o, v, s.B, s.eps, t1, t2, idx)
    assert np.abs(p2.numpy()[tuple(idx.T)] - want).max() < 1e-9


def _pair(p, q, n):
    return p * (2 * n - p - 1) // 2 + (q - p - 1)


@pytest.mark.parametrize("o,v", [(3, 7), (4, 25)])
def test_packed_vvvv_block_matches_oracle(cc, o, v):
    _, engine = cc
    s, B, _, _ = small_case(o, v, 41, L=8)
    dsys = engine.DeviceSystem(o, v, s.eps_occ, s.eps_vir, B, device=DEV, packed_vvvv=True)
    assert "vvvv" not in dsys.blocks
    V = oracle_V(o, v, B)[o:, o:, o:, o:]
    P = v * (v - 1) // 2
    iu = [(a, b) for a in range(v) for b in range(a + 1, v)]
    assert [_pair(a, b, v) for a, b in iu] == list(range(P))
    want = np.array([[V[a, b, e, f] for e, f in iu] for a, b in iu])
    got = dsys.blocks["vvvv_packed"].view(P, P).cpu().numpy()
    assert np.abs(got - want).max() <= 1e-14 * np.abs(want).max()


@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
def test_packed_vvvv_residual_matches_oracle(cc, prec):
    """A system holding <ab||ef> only packed: the packed list reads it in place."""
    ccm, engine = cc
    o, v = 6, 30
    s, B, t1, t2 = small_case(o, v, 42, L=8, scale=6.0, tscale=0.05)
    dsys = engine.DeviceSystem(o, v, s.eps_occ, s.eps_vir, B, device=DEV, packed_vvvv=True)
    eng = engine.Engine(dsys, list_name="ccsd_packed", precision=prec, route_all=prec != "fp64")
    used = eng.plan.describe()["integrals_used"]
    assert "vvvv_packed" in used and "vvvv" not in used
    r1, r2 = eng.residual(to_dev(t1), to_dev(t2))
    torch.cuda.synchronize()
    V = oracle_V(o, v, B)
    o1, o2 = oracle.ccsd_residual(o, v, s.eps, V, t1, t2)
    if prec == "fp64":
        assert_elementwise([r1, r2], [o1, o2], [np.full(o1.shape, 1e-12), np.full(o2.shape, 1e-12)])
    else:
        _, [(e1, e2)] = list_bounds(ccm.load_list("ccsd_packed"), o, v, s.eps, V, t1, t2, [eng.plan])
        assert_elementwise([r1, r2], [o1, o2], [e1, e2], what="packed-input bf16x3")
    d = np.sqrt(np.sum((r1.cpu().numpy() - o1) ** 2) + np.sum((r2.cpu().numpy() - o2) ** 2))
    assert d <= (1e-13 if prec == "fp64" else 2e-4) * np.sqrt(np.sum(o1 ** 2) + np.sum(o2 ** 2))


@pytest.mark.slow
def test_packed_vvvv_full_size(cc):
    """o=40, v=200: the chunked packed builder against the full block, and the
    packed-input residual against the unpacked plan."""
    _, engine = cc
    s = ccinputs.make_system(**ccinputs.CONFIG_LADDER)
    o, v = s.o, s.v
    full = engine.DeviceSystem.from_system(s, device=DEV)
    pk = engine.DeviceSystem.from_system(s, device=DEV, packed_vvvv=True)
    P = v * (v - 1) // 2
    rng = np.random.default_rng(3)
    ab = rng.integers(0, v, (64, 4))
    ab = ab[(ab[:, 0] < ab[:, 1]) & (ab[:, 2] < ab[:, 3])]
    Vf = full.block("vvvv")
    Vp = pk.blocks["vvvv_packed"].view(P, P)
    for a, b, e, f in ab:
        assert abs(Vp[_pair(a, b, v), _pair(e, f, v)].item() - Vf[a, b, e, f].item()) < 1e-15
    t1, t2 = ccinputs.random_amplitudes(o, v, seed=0, scale1=0.01, scale2=0.01)
    T1, T2 = to_dev(t1), to_dev(t2)
    r = [x.cpu() for x in engine.Engine(pk, list_name="ccsd_packed").residual(T1, T2)]
    del pk
    u = [x.cpu() for x in engine.Engine(full, list_name="ccsd_vvvv").residual(T1, T2)]
    n = max(b.abs().max().item() for b in u)
    assert max((a - b).abs().max().item() for a, b in zip(r, u)) <= 1e-12 * n
