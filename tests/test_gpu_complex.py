"""Complex128 path (complex spin orbitals, Hermitian integrals) vs the complex
oracle build and the complex determinant-space pins behind it.

FP64 route: complex GEMMs and accumulates in double2 arithmetic, compared to
the oracle at 1e-11 relative.  Split route: one real GEMM of doubled K per
complex contraction (the smaller operand embedded as [[Re, -Im], [Im, Re]],
the other stacked as [Re; Im]).  Its element bound is the real one (see
test_gpu_mixed.py) with two changes: each real or imaginary output part sums
two real products per complex one, so the bound on sum_k |a_ik||b_kj|
(moduli) is doubled, and the FP32 accumulation runs over 2K terms.
"""
import numpy as np
import pytest
import torch

import ccinputs
import list_exec
import oracle
from gpu_util import DEV, assert_elementwise, block_slices, list_bounds

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cc():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2409_06759_b300 as cc
    from paper_2409_06759_b300 import engine
    return cc, engine


def complex_case(o, v, seed, L=6, scale=6.0, tscale=0.05):
    s = ccinputs.make_system(o, v, L=L, seed=seed, complex_=True)
    B = s.B * scale
    t1, t2 = ccinputs.random_amplitudes(o, v, seed=seed, scale1=tscale, scale2=tscale, complex_=True)
    return s, B, t1, t2


def zdev(x):
    return torch.tensor(np.ascontiguousarray(x), dtype=torch.complex128, device=DEV)


@pytest.mark.parametrize("o,v,L", [(2, 5, 3), (5, 19, 11), (8, 33, 20)])
def test_complex_integral_blocks_match_oracle(cc, o, v, L):
    _, engine = cc
    s, B, _, _ = complex_case(o, v, 31, L=L)
    dsys = engine.DeviceSystem(o, v, s.eps_occ, s.eps_vir, B, device=DEV)
    ref = block_slices(oracle.antisym_integrals(o, v, B), o)
    for name, want in ref.items():
        got = dsys.block(name).cpu().numpy()
        assert np.abs(got - want).max() <= 1e-14 * max(1.0, np.abs(want).max()), name


@pytest.mark.parametrize("list_name", ["ccsd", "ccsd_vvvv"])
@pytest.mark.parametrize("o,v,seed", [(2, 3, 1), (3, 8, 2), (5, 19, 3), (8, 33, 4)])
def test_complex_fp64_residual_matches_oracle(cc, list_name, o, v, seed):
    _, engine = cc
    s, B, t1, t2 = complex_case(o, v, seed)
    dsys = engine.DeviceSystem(o, v, s.eps_occ, s.eps_vir, B, device=DEV)
    eng = engine.Engine(dsys, list_name=list_name, precision="fp64")
    r1, r2 = eng.residual(zdev(t1), zdev(t2))
    torch.cuda.synchronize()
    o1, o2 = oracle.ccsd_residual(o, v, s.eps, oracle.antisym_integrals(o, v, B), t1, t2)
    scale = max(np.abs(o1).max(), np.abs(o2).max())
    assert np.abs(o2.imag).max() > 1e-3 * scale        # a genuinely complex case
    assert np.abs(r1.cpu().numpy() - o1).max() <= 1e-11 * scale
    assert np.abs(r2.cpu().numpy() - o2).max() <= 1e-11 * scale


# statements whose integral references resolve with a conjugation (bra and
# ket swapped against the stored block) and ones that do not, over the
# copy, outer-product, GEMV and GEMM shapes
STATEMENTS = [
    ("R2[ijab] = V[abij]", 1),
    ("R2[ijab] = P(ab) T1[ia] * T1[jb]", 2),
    ("R2[ijab] = P(ij) T1[ie] * V[abej]", 2),
    ("R2[ijab] = -1 P(ab) T1[ma] * V[mbij]", 2),
    ("R1[ia] = -1 T1[nf] * V[naif]", 1),
    ("R1[ia] = -0.5 T2[mnae] * V[nmei]", 1),
    ("R2[ijab] = 0.5 T2[ijef] * V[abef]", 1),
    ("R2[ijab] = P(ij) P(ab) T2[imae] * V[mbej]", 4),
]


@pytest.mark.parametrize("k", range(len(STATEMENTS)))
def test_complex_fp64_statements(cc, k):
    ccm, engine = cc
    text, _ = STATEMENTS[k]
    o, v = 5, 21
    s, B, t1, t2 = complex_case(o, v, 40 + k)
    dsys = engine.DeviceSystem(o, v, s.eps_occ, s.eps_vir, B, device=DEV)
    eng = engine.Engine(dsys, list_text=text, precision="fp64")
    r1 = torch.zeros(o, v, dtype=torch.complex128, device=DEV)
    r2 = torch.zeros(o, o, v, v, dtype=torch.complex128, device=DEV)
    ccm.cc_residual(eng.plan, dsys.ints(), zdev(t1), zdev(t2), r1, r2, eng.ws)
    torch.cuda.synchronize()
    e1, e2 = list_exec.run_list(text, o, v, s.eps, oracle.antisym_integrals(o, v, B), t1, t2)
    scale = max(np.abs(e1).max(), np.abs(e2).max())
    assert np.abs(r1.cpu().numpy() - e1).max() <= 1e-12 * scale
    assert np.abs(r2.cpu().numpy() - e2).max() <= 1e-12 * scale


def _abs_bound(text, o, v, eps, V, t1, t2):
    """max_ij sum_k |a_ik||b_kj| (moduli) of the statement's plain contraction."""
    rhs = text.split("=", 1)[1].split()
    plain = text.split("=", 1)[0] + "= " + " ".join(
        w for w in rhs if not w.startswith("P(") and not w.lstrip("-").replace(".", "").isdigit())
    z = np.zeros_like(eps)
    a1, a2 = list_exec.run_list(plain, o, v, z, np.abs(V), np.abs(t1), np.abs(t2))
    return max(np.abs(a1).max(), np.abs(a2).max())


SPLIT = [
    ("R2[ijab] = 0.5 T2[ijef] * V[abef]", lambda o, v: v * v, 1),
    ("R2[ijab] = P(ij) P(ab) T2[imae] * V[mbej]", lambda o, v: o * v, 4),
    ("R1[ia] = -0.5 T2[imef] * V[maef]", lambda o, v: o * v * v, 1),
    ("R2[ijab] = P(ij) T1[ie] * V[abej]", lambda o, v: v, 2),
    ("R2[ijab] = 0.5 T2[mnab] * V[mnij]", lambda o, v: o * o, 1),
]


@pytest.mark.parametrize("prec,first", [("bf16x3", 3 * 2.0 ** -16), ("bf16x6", 3 * 2.0 ** -24)])
@pytest.mark.parametrize("o,v", [(3, 20), (5, 70), (2, 9)])
@pytest.mark.parametrize("k", range(len(SPLIT)))
def test_complex_split_statement(cc, prec, first, o, v, k):
    ccm, engine = cc
    text, kfun, nterms = SPLIT[k]
    s, B, t1, t2 = complex_case(o, v, 60 + k, L=8, tscale=0.1)
    dsys = engine.DeviceSystem(o, v, s.eps_occ, s.eps_vir, B, device=DEV)
    eng = engine.Engine(dsys, list_text=text, precision=prec, route_all=True)
    assert any(st["kind"] == "gemm_bf16split" for st in eng.plan.describe()["steps"])
    r1 = torch.zeros(o, v, dtype=torch.complex128, device=DEV)
    r2 = torch.zeros(o, o, v, v, dtype=torch.complex128, device=DEV)
    ccm.cc_residual(eng.plan, dsys.ints(), zdev(t1), zdev(t2), r1, r2, eng.ws)
    torch.cuda.synchronize()
    V = oracle.antisym_integrals(o, v, B)
    e1, e2 = list_exec.run_list(text, o, v, s.eps, V, t1, t2)
    first_tok = text.split("=", 1)[1].split()[0]
    fac = abs(float(first_tok)) if first_tok[0] in "-0123456789" else 1.0
    kacc = 2 * kfun(o, v) if prec == "bf16x3" else min(2 * kfun(o, v), 128)
    tol = 2 * nterms * fac * (first + kacc * 2.0 ** -24) * _abs_bound(text, o, v, s.eps, V, t1, t2) + 1e-15
    err = max(np.abs(r1.cpu().numpy() - e1).max(), np.abs(r2.cpu().numpy() - e2).max())
    assert err <= tol, (err, tol)
    mag = max(np.abs(e1).max(), np.abs(e2).max())
    assert err <= 1e-3 * mag


@pytest.mark.parametrize("prec,rel", [("bf16x3", 4e-4), ("bf16x6", 2e-6)])
@pytest.mark.parametrize("o,v,route_all", [(3, 8, True), (6, 30, True), (9, 37, False)])
def test_complex_mixed_full_residual_vs_oracle(cc, prec, rel, o, v, route_all):
    """Every complex R1, R2 element of the split route against the complex
    oracle within the element-wise bound of the plan's routes (moduli, twice
    the real rule), and the error norm as an extra check."""
    ccm, engine = cc
    s, B, t1, t2 = complex_case(o, v, 9, L=8)
    dsys = engine.DeviceSystem(o, v, s.eps_occ, s.eps_vir, B, device=DEV)
    eng = engine.Engine(dsys, list_name="ccsd_vvvv", precision=prec, route_all=route_all)
    r1, r2 = eng.residual(zdev(t1), zdev(t2))
    torch.cuda.synchronize()
    V = oracle.antisym_integrals(o, v, B)
    o1, o2 = oracle.ccsd_residual(o, v, s.eps, V, t1, t2)
    _, [(e1, e2)] = list_bounds(ccm.load_list("ccsd_vvvv"), o, v, s.eps, V, t1, t2, [eng.plan])
    assert_elementwise([r1, r2], [o1, o2], [e1, e2], what=f"complex {prec} o={o} v={v}")
    d = np.sqrt(np.sum(np.abs(r1.cpu().numpy() - o1) ** 2) + np.sum(np.abs(r2.cpu().numpy() - o2) ** 2))
    ref = np.sqrt(np.sum(np.abs(o1) ** 2) + np.sum(np.abs(o2) ** 2))
    assert d <= rel * ref


def test_complex_energy_matches_oracle(cc):
    _, engine = cc
    o, v = 6, 23
    s, B, t1, t2 = complex_case(o, v, 12)
    dsys = engine.DeviceSystem(o, v, s.eps_occ, s.eps_vir, B, device=DEV)
    eng = engine.Engine(dsys, list_name="ccsd")
    e = eng.energy(zdev(t1), zdev(t2))
    want = oracle.ccsd_energy(o, v, oracle.antisym_integrals(o, v, B), t1, t2)
    assert isinstance(e, complex) and abs(want.imag) > 1e-6
    assert abs(e - want) <= 1e-13 * max(1.0, abs(want))


def test_complex_solve_matches_oracle(cc):
    """FP64 Jacobi + DIIS on a complex system: the converged complex energy
    equals the oracle's; the split route with FP64 defect correction reaches
    the same energy."""
    _, engine = cc
    o, v = 6, 24
    s = ccinputs.make_system(o, v, L=16, seed=5, complex_=True)
    ref = oracle.ccsd_solve(o, v, s.eps, oracle.antisym_integrals(o, v, s.B), tol=1e-9, maxiter=80)
    assert ref["status"] == 0
    dsys = engine.DeviceSystem.from_system(s, device=DEV)
    z = lambda: (torch.zeros(o, v, dtype=torch.complex128, device=DEV),
                 torch.zeros(o, o, v, v, dtype=torch.complex128, device=DEV))
    fp64 = engine.Engine(dsys, list_name="ccsd")
    a1, a2 = z()
    res = engine.Solver(fp64).solve(a1, a2, max_iter=80, tol=1e-9)
    assert res.converged and isinstance(res.energy, complex)
    assert abs(res.energy - ref["energy"]) < 1e-10
    mixed = engine.Engine(dsys, list_name="ccsd_vvvv", precision="bf16x6", route_all=True)
    b1, b2 = z()
    res2 = engine.Solver(mixed, refine=fp64).solve(b1, b2, max_iter=80, tol=1e-9, switch_tol=1e-7)
    assert res2.converged and abs(res2.energy - ref["energy"]) < 1e-10


def test_complex_two_electrons_equals_fci(cc):
    """Two electrons: CCSD is exact, so the converged complex-orbital energy is
    the (real) FCI correlation energy of the determinant-space Hamiltonian."""
    import detspace
    _, engine = cc
    o, v = 2, 7
    s, B, _, _ = complex_case(o, v, 13, L=5)
    V = oracle.antisym_integrals(o, v, B)
    e_fci = detspace.fci_correlation(o, v, s.eps, V)
    dsys = engine.DeviceSystem(o, v, s.eps_occ, s.eps_vir, B, device=DEV)
    eng = engine.Engine(dsys, list_name="ccsd")
    t1 = torch.zeros(o, v, dtype=torch.complex128, device=DEV)
    t2 = torch.zeros(o, o, v, v, dtype=torch.complex128, device=DEV)
    res = engine.Solver(eng).solve(t1, t2, max_iter=100, tol=1e-11)
    assert res.converged
    assert abs(res.energy - e_fci) < 1e-11
