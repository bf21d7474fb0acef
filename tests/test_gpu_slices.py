"""The exact-slice route (CC_PREC_SLICES): an FP64-grade contraction on the
tensor cores.  Every operand row is scaled by a power of two and cut into six
exact 7-bit bf16 slices; the 21 slice products of weight <= 5 are summed
exactly in FP32 over 128-long K chunks and drained into float-float registers.

Its error per element is below
    K (2 * 2^-41 + 7 * 2^-40) max_k|A(m,k)| max_k|B(k,n)|      (slicing, dropped weights)
  + 6 ceil(K/128) 2^-48 sum_k |A(m,k)| |B(k,n)|                 (float-float drains)
(first order; times the number of permutation terms), so it is held to the
FP64 parity bar of the other routes: every residual element within 1e-9 of
the oracle, and single contractions within the bound above.
"""
import numpy as np
import pytest
import torch

import ccinputs
import list_exec
import oracle
from gpu_util import DEV, assert_elementwise, oracle_V, small_case, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cc():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2409_06759_b300 as cc
    from paper_2409_06759_b300 import engine
    return cc, engine


def _slice_bound(text, o, v, eps, V, t1, t2, nterms, fac):
    """The bound of the module docstring for a one-statement list: the plain
    contraction of |A| |B|, and of the row maxima of A and column maxima of B."""
    rhs = text.split("=", 1)[1]
    plain = text.split("=", 1)[0] + "= " + " ".join(w for w in rhs.split()
                                                    if not w.startswith("P(") and not w.lstrip("-").replace(".", "").isdigit())
    z = np.zeros_like(eps)
    s1, s2 = list_exec.run_list(plain, o, v, z, np.abs(V), np.abs(t1), np.abs(t2))
    # K max|A row| max|B column| <= (max over the statement's operands) K |A|max |B|max, taken
    # per output element through the same contraction of the operands' maxima (an upper bound)
    ma, mb = np.abs(t2).max(), np.abs(V).max()
    mt1 = np.abs(t1).max()
    ones = lambda x, m: np.full_like(x, m)
    m1, m2 = list_exec.run_list(plain, o, v, z, ones(V, mb), ones(t1, mt1), ones(t2, ma))
    c1 = 2 * 2.0 ** -41 + 7 * 2.0 ** -40
    kmax = max(v * v, o * v * v, o * o, o * v)          # the longest contraction of STATEMENTS
    c2 = 6 * -(-kmax // 128) * 2.0 ** -48               # one float-float add per weight per chunk
    return [nterms * fac * (c1 * np.abs(m) + c2 * s) + 1e-300 for m, s in ((m1, s1), (m2, s2))]


STATEMENTS = [
    ("R2[ijab] = 0.5 T2[ijef] * V[abef]", 1),
    ("R2[ijab] = P(ij) P(ab) T2[imae] * V[mbej]", 4),
    ("R1[ia] = -0.5 T2[imef] * V[maef]", 1),
    ("R2[ijab] = 0.5 T2[mnab] * V[mnij]", 1),
]


@pytest.mark.parametrize("o,v", [(3, 20), (5, 70), (2, 9), (7, 33)])
@pytest.mark.parametrize("k", range(len(STATEMENTS)))
def test_slice_statement_within_its_bound(cc, o, v, k):
    ccm, engine = cc
    text, nterms = STATEMENTS[k]
    s, B, t1, t2 = small_case(o, v, 400 + k, L=8, scale=6.0, tscale=0.1)
    dsys = engine.DeviceSystem(o, v, s.eps_occ, s.eps_vir, B, device=DEV)
    eng = engine.Engine(dsys, list_text=text, precision="slices", route_all=True)
    kinds = [st["kind"] for st in eng.plan.describe()["steps"]]
    assert "gemm_bf16split" in kinds
    r1 = torch.zeros(o, v, dtype=torch.float64, device=DEV)
    r2 = torch.zeros(o, o, v, v, dtype=torch.float64, device=DEV)
    ccm.cc_residual(eng.plan, dsys.ints(), to_dev(t1), to_dev(t2), r1, r2, eng.ws)
    torch.cuda.synchronize()
    V = oracle_V(o, v, B)
    e1, e2 = list_exec.run_list(text, o, v, s.eps, V, t1, t2)
    first = text.split("=", 1)[1].split()[0]
    fac = abs(float(first)) if first[0] in "-0123456789" else 1.0
    b1, b2 = _slice_bound(text, o, v, s.eps, V, t1, t2, nterms, fac)
    # the -D*t part of run_list is exact FP64 on both sides
    assert_elementwise([r1, r2], [e1, e2], [b1, b2], slack=1e-15, what=text)


@pytest.mark.parametrize("list_name", ["ccsd_vvvv", "ccsd"])
@pytest.mark.parametrize("o,v,route_all", [(3, 8, True), (6, 30, True), (10, 40, False), (13, 57, False)])
def test_slice_residual_meets_the_fp64_bar(cc, list_name, o, v, route_all):
    """Every R1 and R2 element within 1e-9 of the oracle (the FP64 bar), and
    within 1e-10 of the largest element."""
    _, engine = cc
    s, B, t1, t2 = small_case(o, v, 17, L=8, scale=6.0, tscale=0.05)
    dsys = engine.DeviceSystem(o, v, s.eps_occ, s.eps_vir, B, device=DEV)
    eng = engine.Engine(dsys, list_name=list_name, precision="slices", route_all=route_all)
    kinds = {st["kind"] for st in eng.plan.describe()["steps"]}
    assert "gemm_bf16split" in kinds and not any(k.endswith("f32") for k in kinds)
    r1, r2 = eng.residual(to_dev(t1), to_dev(t2))
    torch.cuda.synchronize()
    o1, o2 = oracle.ccsd_residual(o, v, s.eps, oracle_V(o, v, B), t1, t2)
    scale = max(np.abs(o1).max(), np.abs(o2).max())
    tol = min(1e-9, 1e-10 * scale)
    assert_elementwise([r1, r2], [o1, o2], [np.full(o1.shape, tol), np.full(o2.shape, tol)], slack=0.0,
                       what=f"slices {list_name} o={o} v={v}")


def test_slice_residual_complex(cc):
    """complex128 (the 4M embedding: the embedded operand's re/im rows are
    sliced like any other rows): every element within 1e-9 of the complex oracle."""
    _, engine = cc
    o, v = 6, 23
    s = ccinputs.make_system(o, v, L=8, seed=18, complex_=True)
    B = s.B * 6.0
    t1, t2 = ccinputs.random_amplitudes(o, v, seed=18, scale1=0.05, scale2=0.05, complex_=True)
    dsys = engine.DeviceSystem(o, v, s.eps_occ, s.eps_vir, B, device=DEV)
    eng = engine.Engine(dsys, list_name="ccsd_vvvv", precision="slices", route_all=True)
    z = lambda x: torch.tensor(np.ascontiguousarray(x), dtype=torch.complex128, device=DEV)
    r1, r2 = eng.residual(z(t1), z(t2))
    torch.cuda.synchronize()
    o1, o2 = oracle.ccsd_residual(o, v, s.eps, oracle.antisym_integrals(o, v, B), t1, t2)
    scale = max(np.abs(o1).max(), np.abs(o2).max())
    tol = min(1e-9, 1e-10 * scale)
    assert_elementwise([r1, r2], [o1, o2], [np.full(o1.shape, tol), np.full(o2.shape, tol)], slack=0.0,
                       what="complex slices")


def test_every_slice_configuration_gives_the_same_residual(cc):
    """Split-K factors and the reduction epilogue of the exact-slice GEMMs
    change only the FP64 order of the chunk sums: within 1e-12 of each other."""
    ccm, engine = cc
    o, v = 9, 36
    s, B, t1, t2 = small_case(o, v, 19, L=16, scale=6.0, tscale=0.05)
    dsys = engine.DeviceSystem(o, v, s.eps_occ, s.eps_vir, B, device=DEV)
    eng = engine.Engine(dsys, list_name="ccsd_vvvv", precision="slices")
    T1, T2 = to_dev(t1), to_dev(t2)
    b1, b2 = eng.residual(T1, T2)
    torch.cuda.synchronize()
    base = torch.cat([b1.flatten(), b2.flatten()]).cpu().numpy()
    tol = np.full(base.shape, 1e-12 * np.abs(base).max())
    n = 0
    for k, st in enumerate(eng.plan.describe()["steps"]):
        if not st.get("configs") or st["kind"] != "gemm_bf16split":
            continue
        planned = (st.get("bn", 0), st["splitk"], st.get("red", 0))
        for bn, sk, red in st["configs"]:
            ccm.cc_plan_set_gemm_config(eng.plan, k, bn, sk, red)
            r1, r2 = eng.residual(T1, T2)
            torch.cuda.synchronize()
            assert_elementwise([torch.cat([r1.flatten(), r2.flatten()])], [base], [tol],
                               what=f"step {k} bn={bn} splitk={sk} red={red}")
            n += 1
        ccm.cc_plan_set_gemm_config(eng.plan, k, *planned)
    assert n > 0


def test_nan_in_the_amplitudes_reaches_the_residual(cc):
    """A non-finite amplitude is carried by the top slice, so the residual shows
    it (cc_solve's divergence check depends on that)."""
    _, engine = cc
    o, v = 5, 24
    s, B, t1, t2 = small_case(o, v, 20, L=8, scale=6.0, tscale=0.05)
    t2 = t2.copy()
    t2[0, 1, 2, 3] = np.nan
    dsys = engine.DeviceSystem(o, v, s.eps_occ, s.eps_vir, B, device=DEV)
    eng = engine.Engine(dsys, list_name="ccsd_vvvv", precision="slices", route_all=True)
    r1, r2 = eng.residual(to_dev(t1), to_dev(t2))
    torch.cuda.synchronize()
    assert not torch.isfinite(r2).all()


def test_slice_refinement_reaches_the_oracle_energy(cc):
    """o=10, v=40: the split route (bf16x3 and bf16x6) refined by the exact-slice
    plan converges on the slice residual to the oracle's energy (1e-10 Eh);
    the exact-slice plan alone from T = 0 follows the oracle's trajectory."""
    _, engine = cc
    s = ccinputs.make_system(**ccinputs.CONFIG_SMALL)
    o, v = s.o, s.v
    ref = oracle.ccsd_solve(o, v, s.eps, oracle_V(o, v, s.B), tol=1e-10, maxiter=60)
    dsys = engine.DeviceSystem.from_system(s, device=DEV)
    sl = engine.Engine(dsys, list_name="ccsd_vvvv", precision="slices", route_all=True)
    z = lambda: (torch.zeros(o, v, dtype=torch.float64, device=DEV),
                 torch.zeros(o, o, v, v, dtype=torch.float64, device=DEV))
    a1, a2 = z()
    alone = engine.Solver(sl).solve(a1, a2, max_iter=60, tol=1e-10)
    assert alone.converged and abs(alone.iterations - ref["iters"]) <= 1
    k = min(alone.iterations, ref["iters"])
    assert np.abs(np.asarray(alone.energies[:k]) - ref["energies"][:k]).max() < 1e-11
    assert abs(alone.energy - ref["energy"]) < 1e-10
    for inner in ("bf16x3", "bf16x6"):
        mixed = engine.Engine(dsys, list_name="ccsd_vvvv", precision=inner, route_all=True)
        b1, b2 = z()
        res = engine.Solver(mixed, refine=sl).solve(b1, b2, max_iter=60, tol=1e-10, switch_tol=1e-6)
        assert res.converged and res.switched_at >= 0, inner
        assert abs(res.energy - ref["energy"]) < 1e-10, (inner, res.energy - ref["energy"])
