"""Split-bf16 tensor-core route (tcgen05) vs FP64 references.

Tolerance derived from the arithmetic: with two bf16 planes per operand the
dropped lo*lo product and the plane rounding leave at most ~3*2^-16 |a||b|
per product, and FP32 accumulation over K adds at most K*2^-24 sum|a||b|
(first-order worst case).  So every element must satisfy
    |err| <= nterms * |factor| * (3*2^-16 + K*2^-24) * max sum_k |a_ik||b_kj|.
With three planes (six products) the first term drops to ~3*2^-24 and the
accumulator is drained every 128 K elements into float-float registers, so
the second term becomes min(K, 128)*2^-24.
"""
import numpy as np
import pytest
import torch

import ccinputs
import list_exec
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


STATEMENTS = [
    # (text, K as a function of (o, v), number of permutation terms)
    ("R2[ijab] = 0.5 T2[ijef] * V[abef]", lambda o, v: v * v, 1),
    ("R2[ijab] = P(ij) P(ab) T2[imae] * V[mbej]", lambda o, v: o * v, 4),
    ("R1[ia] = -0.5 T2[imef] * V[maef]", lambda o, v: o * v * v, 1),
    ("R2[ijab] = 0.5 T2[mnab] * V[mnij]", lambda o, v: o * o, 1),
]


def _abs_bound(text, o, v, eps, V, t1, t2):
    """max_ij sum_k |a_ik||b_kj| of the statement's plain contraction."""
    plain = text.split("=", 1)[0] + "= " + " ".join(w for w in text.split("=", 1)[1].split()
                                                      if not w.startswith("P(") and not w.lstrip("-").replace(".", "").isdigit())
    z = np.zeros_like(eps)
    a1, a2 = list_exec.run_list(plain, o, v, z, np.abs(V), np.abs(t1), np.abs(t2))
    return max(np.abs(a1).max(), np.abs(a2).max())


@pytest.mark.parametrize("prec,first", [("bf16x3", 3 * 2.0 ** -16), ("bf16x6", 3 * 2.0 ** -24)])
@pytest.mark.parametrize("o,v", [(3, 20), (5, 70), (2, 9), (7, 33)])
@pytest.mark.parametrize("k", range(len(STATEMENTS)))
def test_split_gemm_statement(cc, prec, first, o, v, k):
    ccm, engine = cc
    text, kfun, nterms = STATEMENTS[k]
    s, B, t1, t2 = small_case(o, v, 100 + k, L=8, scale=6.0, tscale=0.1)
    dsys = engine.DeviceSystem(o, v, s.eps_occ, s.eps_vir, B, device=DEV)
    eng = engine.Engine(dsys, list_text=text, precision=prec, route_all=True)
    assert any(st["kind"] == "gemm_bf16split" for st in eng.plan.describe()["steps"])
    r1 = torch.zeros(o, v, dtype=torch.float64, device=DEV)
    r2 = torch.zeros(o, o, v, v, dtype=torch.float64, device=DEV)
    ccm.cc_residual(eng.plan, dsys.ints(), to_dev(t1), to_dev(t2), r1, r2, eng.ws)
    torch.cuda.synchronize()
    V = oracle_V(o, v, B)
    e1, e2 = list_exec.run_list(text, o, v, s.eps, V, t1, t2)
    fac = abs(float(text.split("=", 1)[1].split()[0])) if text.split("=", 1)[1].split()[0][0] in "-0123456789" else 1.0
    kacc = kfun(o, v) if prec == "bf16x3" else min(kfun(o, v), 128)
    tol = nterms * fac * (first + kacc * 2.0 ** -24) * _abs_bound(text, o, v, s.eps, V, t1, t2) + 1e-15
    err = max(np.abs(r1.cpu().numpy() - e1).max(), np.abs(r2.cpu().numpy() - e2).max())
    assert err <= tol, (err, tol)
    mag = max(np.abs(e1).max(), np.abs(e2).max())
    assert err <= 1e-3 * mag


@pytest.mark.parametrize("prec,first", [("bf16x3", 3 * 2.0 ** -16), ("bf16x6", 3 * 2.0 ** -24)])
@pytest.mark.parametrize("o", [23, 31, 16, 25])
def test_ragged_column_tiles(cc, prec, first, o):
    """The ladder statement with N = o^2 columns at every tile width the step
    offers.  The ceil(N / BN) column tiles share N's 16-column units evenly, so
    tiles of two widths meet inside the output and the last one may pass N by
    up to 15 columns: N = 529 runs 192+176+176 at width 256, 3x112+2x96 at 128,
    6x64+3x48 at 64; N = 961 runs 256+3x240, 5x128+3x112, 13x64+3x48; N = 256
    runs full tiles; N = 625 runs 224+2x208, and 5x128 / 10x64 ending 15
    columns past N.  M = v^2 = 144 leaves a 16-row last row tile and K = 144 a
    ragged K block.  R2 starts as NaN, so a column no tile stores shows up."""
    ccm, engine = cc
    v = 12
    text, kfun, nterms = STATEMENTS[0]
    s, B, t1, t2 = small_case(o, v, 300 + o, L=8, scale=6.0, tscale=0.1)
    dsys = engine.DeviceSystem(o, v, s.eps_occ, s.eps_vir, B, device=DEV)
    eng = engine.Engine(dsys, list_text=text, precision=prec, route_all=True)
    steps = eng.plan.describe()["steps"]
    k = next(i for i, st in enumerate(steps) if st["kind"] == "gemm_bf16split")
    assert steps[k]["N"] == o * o and steps[k]["M"] == v * v
    V = oracle_V(o, v, B)
    e1, e2 = list_exec.run_list(text, o, v, s.eps, V, t1, t2)
    kacc = kfun(o, v) if prec == "bf16x3" else min(kfun(o, v), 128)
    tol = nterms * 0.5 * (first + kacc * 2.0 ** -24) * _abs_bound(text, o, v, s.eps, V, t1, t2) + 1e-15
    widths = set()
    for bn, sk, red in steps[k]["configs"]:
        ccm.cc_plan_set_gemm_config(eng.plan, k, bn, sk, red)
        r2 = torch.full((o, o, v, v), float("nan"), dtype=torch.float64, device=DEV)
        r1 = torch.zeros(o, v, dtype=torch.float64, device=DEV)
        ccm.cc_residual(eng.plan, dsys.ints(), to_dev(t1), to_dev(t2), r1, r2, eng.ws)
        torch.cuda.synchronize()
        err = np.abs(r2.cpu().numpy() - e2).max()      # a column the kernel skipped stays NaN
        assert err <= tol, (bn, err, tol)
        widths.add(bn)
    assert {64, 128} <= widths


@pytest.mark.parametrize("prec,rel", [("bf16x3", 2e-4), ("bf16x6", 1e-6)])
@pytest.mark.parametrize("o,v,route_all", [(3, 8, True), (6, 30, True), (10, 40, False), (13, 57, False)])
def test_mixed_full_residual_vs_oracle(cc, prec, rel, o, v, route_all):
    """Every R1 and R2 element of the split route against the oracle, within the
    element-wise bound of the plan's routes propagated through the list
    (list_exec.run_list_bounds); the Frobenius norm of the error as an extra
    check.  route_all sends every contraction to the tensor cores; otherwise
    the plan's own route choice (tensor cores, FP32 narrow and tiled, FP64)."""
    ccm, engine = cc
    s, B, t1, t2 = small_case(o, v, 7, L=8, scale=6.0, tscale=0.05)
    dsys = engine.DeviceSystem(o, v, s.eps_occ, s.eps_vir, B, device=DEV)
    eng = engine.Engine(dsys, list_name="ccsd_vvvv", precision=prec, route_all=route_all)
    r1, r2 = eng.residual(to_dev(t1), to_dev(t2))
    torch.cuda.synchronize()
    V = oracle_V(o, v, B)
    o1, o2 = oracle.ccsd_residual(o, v, s.eps, V, t1, t2)
    (x1, x2), [(e1, e2)] = list_bounds(ccm.load_list("ccsd_vvvv"), o, v, s.eps, V, t1, t2, [eng.plan])
    assert np.abs(x2 - o2).max() < 1e-13 and np.abs(x1 - o1).max() < 1e-13   # the einsum reading is the oracle's
    assert_elementwise([r1, r2], [o1, o2], [e1, e2], what=f"{prec} o={o} v={v}")
    d = np.sqrt(np.sum((r1.cpu().numpy() - o1) ** 2) + np.sum((r2.cpu().numpy() - o2) ** 2))
    ref = np.sqrt(np.sum(o1 ** 2) + np.sum(o2 ** 2))
    assert d <= rel * ref


def test_mixed_solve_small_config(cc):
    """o=10, v=40: split-bf16 iterations alone reach |dE| < 1e-6 Eh; with the FP64
    refine plan the converged energy matches the oracle to 1e-10 Eh."""
    _, engine = cc
    s = ccinputs.make_system(**ccinputs.CONFIG_SMALL)
    o, v = s.o, s.v
    ref = oracle.ccsd_solve(o, v, s.eps, oracle_V(o, v, s.B), tol=1e-8, maxiter=60)
    dsys = engine.DeviceSystem.from_system(s, device=DEV)
    mixed = engine.Engine(dsys, list_name="ccsd_vvvv", precision="bf16x3", route_all=True)
    fp64 = engine.Engine(dsys, list_name="ccsd")
    z = lambda: (torch.zeros(o, v, dtype=torch.float64, device=DEV),
                 torch.zeros(o, o, v, v, dtype=torch.float64, device=DEV))
    a1, a2 = z()
    alone = engine.Solver(mixed).solve(a1, a2, max_iter=40, tol=1e-8)
    assert abs(alone.energy - ref["energy"]) < 1e-6
    b1, b2 = z()
    res = engine.Solver(mixed, refine=fp64).solve(b1, b2, max_iter=60, tol=1e-8, switch_tol=1e-6)
    assert res.converged and res.switched_at >= 0
    assert abs(res.energy - ref["energy"]) < 1e-10


def test_accurate_mixed_solve_small_config(cc):
    """Three planes with chunked accumulation: the split route alone reaches the
    oracle energy within 1e-8 Eh; refined, within 1e-10 Eh."""
    _, engine = cc
    s = ccinputs.make_system(**ccinputs.CONFIG_SMALL)
    o, v = s.o, s.v
    ref = oracle.ccsd_solve(o, v, s.eps, oracle_V(o, v, s.B), tol=1e-8, maxiter=60)
    dsys = engine.DeviceSystem.from_system(s, device=DEV)
    mixed = engine.Engine(dsys, list_name="ccsd_vvvv", precision="bf16x6", route_all=True)
    z = lambda: (torch.zeros(o, v, dtype=torch.float64, device=DEV),
                 torch.zeros(o, o, v, v, dtype=torch.float64, device=DEV))
    a1, a2 = z()
    alone = engine.Solver(mixed).solve(a1, a2, max_iter=40, tol=1e-8)
    assert alone.converged and abs(alone.energy - ref["energy"]) < 1e-8
    b1, b2 = z()
    res = engine.Solver(mixed, refine=engine.Engine(dsys, list_name="ccsd")).solve(b1, b2, max_iter=60, tol=1e-8,
                                                                                  switch_tol=1e-7)
    assert res.converged and abs(res.energy - ref["energy"]) < 1e-10


@pytest.mark.parametrize("prec,kind,rel", [("fp64", "gemm_rows", 1e-13), ("bf16x3", "gemm_rows_f32", 2e-6)])
def test_narrow_gemm_route(cc, prec, kind, rel):
    """Rank-o updates (short K and one short free side) run on the narrow
    kernel, reading T2 in place: FP64 arithmetic on the FP64 plan, FP32 on the
    mixed plan (error bound K * 2^-24 relative to sum |a||b|)."""
    ccm, engine = cc
    o, v = 24, 100
    text = "X[mj] = V[mnje] * T1[ne]\nR2[ijab] = -1 P(ij) T2[imab] * X[mj]"
    s, B, t1, t2 = small_case(o, v, 21, L=8, scale=6.0, tscale=0.05)
    dsys = engine.DeviceSystem(o, v, s.eps_occ, s.eps_vir, B, device=DEV, blocks=("ooov",))
    eng = engine.Engine(dsys, list_text=text, precision=prec)
    assert kind in [st["kind"] for st in eng.plan.describe()["steps"]]
    r1 = torch.zeros(o, v, dtype=torch.float64, device=DEV)
    r2 = torch.zeros(o, o, v, v, dtype=torch.float64, device=DEV)
    ccm.cc_residual(eng.plan, dsys.ints(), to_dev(t1), to_dev(t2), r1, r2, eng.ws)
    torch.cuda.synchronize()
    (e1, e2), [(b1, b2)] = list_bounds(text, o, v, s.eps, oracle_V(o, v, B), t1, t2, [eng.plan])
    assert_elementwise([r2], [e2], [b2], slack=1e-14, what=f"narrow route {prec}")
    err = np.abs(r2.cpu().numpy() - e2).max()
    assert err <= rel * np.abs(e2).max(), err


@pytest.mark.parametrize("prec,rel", [("fp64", 1e-12), ("bf16x3", 2e-4)])
def test_autotuned_plan_keeps_the_residual(cc, prec, rel):
    """cc_plan_autotune changes only tile widths and split-K factors: every
    element of the tuned plan's residual matches the oracle within the bound
    of its (tuned) routes, 1e-9 for FP64."""
    ccm, engine = cc
    o, v = 10, 40
    s, B, t1, t2 = small_case(o, v, 31, L=16, scale=6.0, tscale=0.05)
    dsys = engine.DeviceSystem(o, v, s.eps_occ, s.eps_vir, B, device=DEV)
    name = "ccsd" if prec == "fp64" else "ccsd_vvvv"
    eng = engine.Engine(dsys, list_name=name, precision=prec)
    T1, T2 = to_dev(t1), to_dev(t2)
    eng.autotune(T1, T2, reps=2)
    d = eng.plan.describe()
    assert d["tuned"] == 1 and any(st.get("candidates", 0) > 1 for st in d["steps"])
    r1, r2 = eng.residual(T1, T2)
    torch.cuda.synchronize()
    V = oracle_V(o, v, B)
    o1, o2 = oracle.ccsd_residual(o, v, s.eps, V, t1, t2)
    if prec == "fp64":
        assert_elementwise([r1, r2], [o1, o2], [np.full(o1.shape, 1e-9), np.full(o2.shape, 1e-9)], slack=1e-12)
    else:
        _, [(e1, e2)] = list_bounds(ccm.load_list(name), o, v, s.eps, V, t1, t2, [eng.plan])
        assert_elementwise([r1, r2], [o1, o2], [e1, e2], what="tuned bf16x3")
    dd = np.sqrt(np.sum((r1.cpu().numpy() - o1) ** 2) + np.sum((r2.cpu().numpy() - o2) ** 2))
    assert dd <= rel * np.sqrt(np.sum(o1 ** 2) + np.sum(o2 ** 2))


@pytest.mark.parametrize("list_name,prec,o,v,cplx", [("ccsd_vvvv", "bf16x3", 10, 40, False),
                                                      ("ccsd_vvvv", "bf16x3", 7, 45, False),
                                                      ("ccsd", "fp64", 9, 30, False),
                                                      ("ccsd_vvvv", "bf16x3", 9, 36, True)])
def test_every_gemm_configuration_gives_the_same_residual(cc, list_name, prec, o, v, cplx):
    """Each contraction step set, one at a time, to every autotuning candidate
    (tile widths, split-K factors, and the reduction epilogue of accumulating
    contractions) reproduces the planned configuration's residual: the
    configurations differ only in the FP32 summation order inside a tile
    column (split K) or the order in which L2 adds a tile (reductions), so the
    difference stays at the split route's rounding level."""
    ccm, engine = cc
    if cplx:
        s = ccinputs.make_system(o, v, L=16, seed=33, complex_=True)
        B = s.B * 6.0
        t1, t2 = ccinputs.random_amplitudes(o, v, seed=33, scale1=0.05, scale2=0.05, complex_=True)
        T1 = torch.tensor(t1, dtype=torch.complex128, device=DEV)
        T2 = torch.tensor(t2, dtype=torch.complex128, device=DEV)
    else:
        s, B, t1, t2 = small_case(o, v, 33, L=16, scale=6.0, tscale=0.05)
        T1, T2 = to_dev(t1), to_dev(t2)
    dsys = engine.DeviceSystem(o, v, s.eps_occ, s.eps_vir, B, device=DEV)
    eng = engine.Engine(dsys, list_name=list_name, precision=prec)
    b1, b2 = eng.residual(T1, T2)
    torch.cuda.synchronize()
    base = torch.cat([b1.flatten(), b2.flatten()]).cpu().numpy()  # complex or real
    scale = np.linalg.norm(base)
    # every configuration and the planned one lie within the bound of the
    # loosest candidate (no split K) of the truth, so within twice it of each other
    _, [(e1, e2)] = list_bounds(ccm.load_list(list_name), o, v, s.eps, oracle.antisym_integrals(o, v, B), t1, t2,
                                [eng.plan], use_splitk=False)
    if prec == "fp64":
        e1, e2 = np.full(e1.shape, 1e-12), np.full(e2.shape, 1e-12)
    ebound = 2.0 * np.concatenate([e1.ravel(), e2.ravel()])
    steps = eng.plan.describe()["steps"]
    reds = 0
    for k, st in enumerate(steps):
        if not st.get("configs"):
            continue
        planned = (st.get("bn", 0), st["splitk"], st.get("red", 0))
        for bn, sk, red in st["configs"]:
            ccm.cc_plan_set_gemm_config(eng.plan, k, bn, sk, red)
            r1, r2 = eng.residual(T1, T2)
            torch.cuda.synchronize()
            got = torch.cat([r1.flatten(), r2.flatten()]).cpu().numpy()
            assert_elementwise([got], [base], [ebound], what=f"step {k} bn={bn} splitk={sk} red={red}")
            tol = 1e-5 if prec != "fp64" else 1e-13
            assert np.linalg.norm(got - base) <= tol * scale, (k, bn, sk, red)
            reds += red
        ccm.cc_plan_set_gemm_config(eng.plan, k, *planned)
    assert reds > 0
    with pytest.raises(RuntimeError):
        ccm.cc_plan_set_gemm_config(eng.plan, 0, 999, 1, 0)
