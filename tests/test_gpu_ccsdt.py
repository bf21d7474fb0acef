"""CCSDT (the generated list, lists/ccsdt.txt) on the GPU against the
definition oracle (oracle/cc_definition.c: <Phi_l| exp(-T) H_N exp(T) |Phi_0>
from CI coefficients, independent of the list and its derivation), the
determinant-space FCI (three electrons: CCSDT is exact), and the split-bf16
route against the FP64 route."""
import itertools

import numpy as np
import pytest
import torch

import ccinputs
import detspace
import list_exec
import oracle
from gpu_util import DEV, assert_elementwise, list_bounds

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cc():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2409_06759_b300 as cc
    from paper_2409_06759_b300 import engine
    return cc, engine


def dev(x, cplx=False):
    return torch.tensor(np.ascontiguousarray(x), dtype=torch.complex128 if cplx else torch.float64, device=DEV)


def case(o, v, seed, L=6, scale=6.0, tscale=0.1, cplx=False):
    s = ccinputs.make_system(o, v, L=L, seed=seed, complex_=cplx)
    B = s.B * scale
    t1, t2, t3 = ccinputs.random_amplitudes(o, v, seed=seed, scale1=tscale, scale2=tscale, triples=True,
                                            complex_=cplx)
    return s, B, t1, t2, t3


def all_idx(o, v, rank):
    return np.array([list(i) + list(a) for i in itertools.product(range(o), repeat=rank)
                     for a in itertools.product(range(v), repeat=rank)])


@pytest.mark.parametrize("cplx", [False, True])
@pytest.mark.parametrize("o,v,seed", [(3, 4, 1), (3, 6, 2)])
def test_ccsdt_residual_matches_definition_oracle(cc, cplx, o, v, seed):
    """Every element of R1, R2, R3."""
    _, engine = cc
    s, B, t1, t2, t3 = case(o, v, seed, cplx=cplx)
    dsys = engine.DeviceSystem(o, v, s.eps_occ, s.eps_vir, B, device=DEV)
    eng = engine.Engine(dsys, list_name="ccsdt")
    r = eng.residual(dev(t1, cplx), dev(t2, cplx), t3=dev(t3, cplx))
    torch.cuda.synchronize()
    for rank in (1, 2, 3):
        idx = all_idx(o, v, rank)
        want = oracle.cc_definition_elements(o, v, B, s.eps, t1, t2, t3, rank=rank, idx=idx)
        got = r[rank - 1].cpu().numpy()[tuple(idx.T)]
        assert np.abs(got - want).max() < 1e-12 * max(1.0, np.abs(want).max()), rank


def test_ccsdt_residual_ragged_multi_tile(cc):
    """o=5, v=17 (several GEMM tiles, ragged tails): the whole arrays against
    the einsum reading of the list, sampled elements against the definition oracle."""
    _, engine = cc
    o, v = 5, 17
    s, B, t1, t2, t3 = case(o, v, 3, L=8, tscale=0.05)
    dsys = engine.DeviceSystem(o, v, s.eps_occ, s.eps_vir, B, device=DEV)
    eng = engine.Engine(dsys, list_name="ccsdt")
    r1, r2, r3 = eng.residual(dev(t1), dev(t2), t3=dev(t3))
    torch.cuda.synchronize()
    g3 = r3.cpu().numpy()
    V = oracle.antisym_integrals(o, v, B)
    e1, e2, e3 = list_exec.run_list(eng.plan.text, o, v, s.eps, V, t1, t2, t3)
    scale = np.abs(e3).max()
    assert np.abs(g3 - e3).max() < 1e-12 * scale
    assert np.abs(r2.cpu().numpy() - e2).max() < 1e-12 * np.abs(e2).max()
    rng = np.random.default_rng(0)
    idx = np.concatenate([rng.integers(0, o, (5, 3)), rng.integers(0, v, (5, 3))], 1)
    idx[0] = (0, 1, 2, 0, 1, 2)
    idx[1] = (o - 1, o - 2, o - 3, v - 1, v - 2, v - 3)
    want = oracle.cc_definition_elements(o, v, B, s.eps, t1, t2, t3, rank=3, idx=idx)
    assert np.abs(g3[tuple(idx.T)] - want).max() < 1e-12 * scale


def test_ccsdt_three_electrons_equals_fci(cc):
    """CCSDT is exact for three electrons: the converged GPU energy is the FCI
    correlation energy of the determinant-space Hamiltonian."""
    _, engine = cc
    o, v = 3, 6
    s = ccinputs.make_system(o, v, L=6, seed=7)
    B = s.B * 6.0
    e_fci = detspace.fci_correlation(o, v, s.eps, oracle.antisym_integrals(o, v, B))
    dsys = engine.DeviceSystem(o, v, s.eps_occ, s.eps_vir, B, device=DEV)
    eng = engine.Engine(dsys, list_name="ccsdt")
    z = [torch.zeros(*sh, dtype=torch.float64, device=DEV) for sh in ((o, v), (o, o, v, v), (o, o, o, v, v, v))]
    res = engine.Solver(eng).solve(z[0], z[1], t3=z[2], max_iter=100, tol=1e-10)
    assert res.converged
    assert abs(res.energy - e_fci) < 1e-10
    # the converged amplitudes make every residual element vanish (definition oracle)
    t1, t2, t3 = (x.cpu().numpy() for x in z)
    idx = all_idx(o, v, 3)[::7]
    r3 = oracle.cc_definition_elements(o, v, B, s.eps, t1, t2, t3, rank=3, idx=idx)
    assert np.abs(r3).max() < 1e-8


def _reference_with_bounds(ccm, o, v, s, B, t1, t2, t3, plans, n_def=40, seed=0):
    """The einsum reading of the CCSDT list (values and the element-wise bound of
    each plan's routes), itself checked on sampled elements against the
    definition oracle, which shares nothing with the list."""
    V = oracle.antisym_integrals(o, v, B)
    vals, bounds = list_bounds(ccm.load_list("ccsdt"), o, v, s.eps, V, t1, t2, plans, t3=t3)
    rng = np.random.default_rng(seed)
    idx3 = np.concatenate([rng.integers(0, o, (n_def, 3)), rng.integers(0, v, (n_def, 3))], 1)
    want = oracle.cc_definition_elements(o, v, B, s.eps, t1, t2, t3, rank=3, idx=idx3)
    assert np.abs(vals[2][tuple(idx3.T)] - want).max() < 1e-12 * max(1.0, np.abs(want).max())
    return vals, bounds


@pytest.mark.parametrize("kconcat", [True, False])
@pytest.mark.parametrize("prec,rel", [("bf16x3", 1e-4), ("bf16x6", 1e-6)])
def test_ccsdt_split_route_matches_reference(cc, prec, rel, kconcat):
    """Every R1, R2, R3 element of the all-tensor-core route within the
    element-wise bound of its routes (accumulating statements merged into one
    GEMM each, or one GEMM per statement); the FP64 route within 1e-9; the
    error norm against the FP64 route as an extra check."""
    ccm, engine = cc
    o, v = 4, 20
    s, B, t1, t2, t3 = case(o, v, 4, L=8, tscale=0.05)
    dsys = engine.DeviceSystem(o, v, s.eps_occ, s.eps_vir, B, device=DEV)
    T = (dev(t1), dev(t2), dev(t3))
    fe = engine.Engine(dsys, list_name="ccsdt")
    me = engine.Engine(dsys, list_name="ccsdt", precision=prec, route_all=True, kconcat=kconcat)
    assert any("stmts" in st for st in me.plan.describe()["steps"]) == kconcat
    f = fe.residual(T[0], T[1], t3=T[2])
    m = me.residual(T[0], T[1], t3=T[2])
    torch.cuda.synchronize()
    vals, [bound] = _reference_with_bounds(ccm, o, v, s, B, t1, t2, t3, [me.plan])
    assert_elementwise(m, vals, bound, what=f"ccsdt {prec}")
    assert_elementwise(f, vals, [np.full(x.shape, 1e-9) for x in vals], slack=1e-12, what="ccsdt fp64")
    d = np.sqrt(sum(((a - b).cpu().numpy() ** 2).sum() for a, b in zip(f, m)))
    n = np.sqrt(sum((a.cpu().numpy() ** 2).sum() for a in f))
    assert d <= rel * n, (d, n)


@pytest.mark.slow
def test_ccsdt_full_size_sampled_elements(cc):
    """o=8, v=64, L=96 (the CCSDT workload): sampled R1, R2, R3 elements
    against the definition oracle, R3 antisymmetry."""
    _, engine = cc
    s = ccinputs.make_system(**ccinputs.CONFIG_CCSDT)
    o, v = s.o, s.v
    t1, t2, t3 = ccinputs.random_amplitudes(o, v, seed=0, scale1=0.01, scale2=0.01, triples=True)
    dsys = engine.DeviceSystem.from_system(s, device=DEV)
    eng = engine.Engine(dsys, list_name="ccsdt")
    r1, r2, r3 = eng.residual(dev(t1), dev(t2), t3=dev(t3))
    torch.cuda.synchronize()
    rng = np.random.default_rng(1)
    idx3 = np.concatenate([rng.integers(0, o, (3, 3)), rng.integers(0, v, (3, 3))], 1)
    idx3[0] = (0, 1, 2, 0, 1, 2)
    idx3[1] = (o - 1, o - 2, o - 3, v - 1, v - 2, v - 3)
    want = oracle.cc_definition_elements(o, v, s.B, s.eps, t1, t2, t3, rank=3, idx=idx3)
    got = r3[tuple(torch.as_tensor(idx3.T))].cpu().numpy()
    assert np.abs(got - want).max() < 1e-9
    idx2 = np.array([[0, 1, 0, 1], [o - 1, 2, v - 1, 5]])
    want2 = oracle.cc_definition_elements(o, v, s.B, s.eps, t1, t2, t3, rank=2, idx=idx2)
    assert np.abs(r2[tuple(torch.as_tensor(idx2.T))].cpu().numpy() - want2).max() < 1e-9
    g = r3[:4, :4, :4, :16, :16, :16].cpu().numpy()
    scale = np.abs(g).max()
    assert np.abs(g + g.transpose(1, 0, 2, 3, 4, 5)).max() <= 1e-13 * scale
    assert np.abs(g - g.transpose(1, 2, 0, 3, 4, 5)).max() <= 1e-13 * scale
    assert np.abs(g + g.transpose(0, 1, 2, 4, 3, 5)).max() <= 1e-13 * scale


@pytest.mark.parametrize("kconcat", [True, False])
def test_ccsdt_default_mixed_plan_matches_reference(cc, kconcat):
    """The bench's mixed plan (tensor-core route for the contractions that fill
    128 x bn x 64 tiles, FP32 arithmetic for the skinny rank-o updates of T3,
    accumulating statements K-concatenated into one GEMM where that saves
    output passes), o=6 v=36: every element within the element-wise bound of
    its routes, and the error norm against the FP64 plan as an extra check."""
    ccm, engine = cc
    o, v = 6, 36
    s, B, t1, t2, t3 = case(o, v, 5, L=16, scale=1.0, tscale=0.01)
    dsys = engine.DeviceSystem(o, v, s.eps_occ, s.eps_vir, B, device=DEV)
    T = (dev(t1), dev(t2), dev(t3))
    f = engine.Engine(dsys, list_name="ccsdt").residual(T[0], T[1], t3=T[2])
    f = [x.cpu() for x in f]
    mixed = engine.Engine(dsys, list_name="ccsdt", precision="bf16x3", kconcat=kconcat)
    assert sum("stmts" in st for st in mixed.plan.describe()["steps"]) >= (8 if kconcat else 0)
    kinds = {st["kind"] for st in mixed.plan.describe()["steps"]}
    assert "gemm_bf16split" in kinds and kinds & {"gemm_f32", "gemm_rows_f32"}
    m = [x.cpu() for x in mixed.residual(T[0], T[1], t3=T[2])]
    vals, [bound] = _reference_with_bounds(ccm, o, v, s, B, t1, t2, t3, [mixed.plan], n_def=12)
    assert_elementwise(m, vals, bound, what="ccsdt default mixed plan")
    d = np.sqrt(sum(((a - b).numpy() ** 2).sum() for a, b in zip(f, m)))
    n = np.sqrt(sum((a.numpy() ** 2).sum() for a in f))
    assert d <= 1e-4 * n, (d, n)
