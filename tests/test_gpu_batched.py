"""Batched Jacobi + DIIS (cc_solve_batched): many independent systems of
uneven size in one call (a CUDA graph of every system's residual, then
batched update kernels), against the oracle's solve of each system and the
single-system cc_solve."""
import numpy as np
import pytest
import torch

import ccinputs
import oracle
from gpu_util import DEV

pytestmark = pytest.mark.gpu

SIZES = [(4, 20, 11), (5, 24, 12), (6, 30, 13), (4, 28, 14), (7, 22, 15), (3, 18, 16)]


@pytest.fixture(scope="module")
def cc():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2409_06759_b300 as cc
    from paper_2409_06759_b300 import engine
    return cc, engine


def zeros(o, v, cplx=False):
    dt = torch.complex128 if cplx else torch.float64
    return (torch.zeros(o, v, dtype=dt, device=DEV), torch.zeros(o, o, v, v, dtype=dt, device=DEV))


def systems(sizes, cplx=False):
    return [ccinputs.make_system(o, v, L=16, seed=sd, complex_=cplx) for o, v, sd in sizes]


def test_batched_fp64_matches_oracle_and_single_solves(cc):
    _, engine = cc
    sy = systems(SIZES)
    dsys = [engine.DeviceSystem.from_system(s, device=DEV) for s in sy]
    engs = [engine.Engine(d, list_name="ccsd") for d in dsys]
    amps = [zeros(s.o, s.v) for s in sy]
    st, res = engine.BatchSolver(engs).solve(amps, max_iter=60, tol=1e-9)
    assert st == 0
    for s, d, r, a in zip(sy, dsys, res, amps):
        ref = oracle.ccsd_solve(s.o, s.v, s.eps, oracle.antisym_integrals(s.o, s.v, s.B), tol=1e-9, maxiter=60)
        assert r.converged and abs(r.energy - ref["energy"]) < 1e-10
        single = engine.Engine(d, list_name="ccsd")
        b1, b2 = zeros(s.o, s.v)
        one = engine.Solver(single).solve(b1, b2, max_iter=60, tol=1e-9)
        assert one.iterations == r.iterations
        assert np.allclose(one.energies, r.energies, rtol=0, atol=1e-12)
        assert torch.abs(b2 - a[1]).max().item() < 1e-11


def test_batched_mixed_and_uneven_convergence(cc):
    """Split-bf16 (bf16x6) plans: every system reaches the oracle energy within
    1e-7 Eh; systems stop at their own iteration counts."""
    _, engine = cc
    sy = systems(SIZES[:4])
    engs = [engine.Engine(engine.DeviceSystem.from_system(s, device=DEV), list_name="ccsd_vvvv",
                          precision="bf16x6", route_all=True) for s in sy]
    amps = [zeros(s.o, s.v) for s in sy]
    st, res = engine.BatchSolver(engs).solve(amps, max_iter=60, tol=1e-8)
    assert st == 0
    for s, r in zip(sy, res):
        ref = oracle.ccsd_solve(s.o, s.v, s.eps, oracle.antisym_integrals(s.o, s.v, s.B), tol=1e-9, maxiter=60)
        assert r.converged and abs(r.energy - ref["energy"]) < 1e-7
    assert len({r.iterations for r in res}) >= 1


def test_batched_complex_systems(cc):
    _, engine = cc
    sy = systems(SIZES[:3], cplx=True)
    dsys = [engine.DeviceSystem.from_system(s, device=DEV) for s in sy]
    engs = [engine.Engine(d, list_name="ccsd") for d in dsys]
    amps = [zeros(s.o, s.v, True) for s in sy]
    st, res = engine.BatchSolver(engs).solve(amps, max_iter=60, tol=1e-9)
    assert st == 0
    for s, r in zip(sy, res):
        ref = oracle.ccsd_solve(s.o, s.v, s.eps, oracle.antisym_integrals(s.o, s.v, s.B), tol=1e-9, maxiter=80)
        assert isinstance(r.energy, complex) and abs(r.energy - ref["energy"]) < 1e-10


def test_batched_max_iter_reports_not_converged(cc):
    ccm, engine = cc
    sy = systems(SIZES[:2])
    engs = [engine.Engine(engine.DeviceSystem.from_system(s, device=DEV), list_name="ccsd") for s in sy]
    amps = [zeros(s.o, s.v) for s in sy]
    st, res = engine.BatchSolver(engs).solve(amps, max_iter=3, tol=1e-12)
    assert st == 7 and all(r.iterations == 3 and not r.converged for r in res)


GROUPED_SIZES = [(4, 20, 21), (6, 30, 22), (8, 36, 23), (5, 44, 24), (10, 40, 25), (3, 18, 26), (7, 52, 27)]


def test_grouped_batch_matches_oracle_and_single_solves(cc):
    """Plans with uniform steps (every contraction on the tensor cores, none
    merged) run the batch as grouped launches (one per step for all systems).
    Every system converges to the oracle energy within 1e-6 Eh (the metric's
    tolerance for the split route), and its trajectory follows the same plan
    solved on its own (cc_solve, one launch per step) to 1e-9 Eh per
    iteration."""
    ccm, engine = cc
    sy = systems(GROUPED_SIZES)
    dsys = [engine.DeviceSystem.from_system(s, device=DEV) for s in sy]
    engs = [engine.Engine(d, list_name="ccsd_vvvv", precision="bf16x3", uniform_steps=True) for d in dsys]
    sig = {tuple(st["kind"] + st["note"] for st in e.plan.describe()["steps"]) for e in engs}
    assert len(sig) == 1                      # the same steps at every size
    amps = [zeros(s.o, s.v) for s in sy]
    n0 = sum(ccm.cc_plan_launch_count(e.plan) for e in engs)
    st, res = engine.BatchSolver(engs).solve(amps, max_iter=60, tol=1e-8)
    assert st == 0
    launches = sum(ccm.cc_plan_launch_count(e.plan) for e in engs) - n0
    nsteps = len(engs[0].plan.describe()["steps"])
    iters = max(r.iterations for r in res)
    # grouped: about two launches per step and iteration for the whole batch, not per system
    assert launches < 3 * nsteps * iters + 8 * iters, (launches, nsteps, iters)
    for s, d, r in zip(sy, dsys, res):
        ref = oracle.ccsd_solve(s.o, s.v, s.eps, oracle.antisym_integrals(s.o, s.v, s.B), tol=1e-9, maxiter=60)
        assert r.converged and abs(r.energy - ref["energy"]) < 1e-6, (s.o, s.v, r.energy - ref["energy"])
        single = engine.Engine(d, list_name="ccsd_vvvv", precision="bf16x3", uniform_steps=True)
        b1, b2 = zeros(s.o, s.v)
        one = engine.Solver(single).solve(b1, b2, max_iter=60, tol=1e-8)
        assert abs(one.iterations - r.iterations) <= 1
        k = min(one.iterations, r.iterations)
        assert np.abs(np.asarray(one.energies[:k]) - np.asarray(r.energies[:k])).max() < 1e-9


def test_grouped_batch_skips_converged_systems(cc):
    """Systems that converge early stop: a system's amplitudes at its own stop
    are the same (bit for bit) whether the call ends there or runs on for the
    others, and each report's iteration count is its own."""
    _, engine = cc
    sy = systems(GROUPED_SIZES[:5])
    engs = [engine.Engine(engine.DeviceSystem.from_system(s, device=DEV), list_name="ccsd_vvvv",
                          precision="bf16x3", uniform_steps=True) for s in sy]
    solver = engine.BatchSolver(engs)
    amps = [zeros(s.o, s.v) for s in sy]
    st, res = solver.solve(amps, max_iter=60, tol=1e-7)
    assert st == 0
    its = [r.iterations for r in res]
    first = int(np.argmin(its))
    assert min(its) < max(its), its
    amps2 = [zeros(s.o, s.v) for s in sy]
    solver.solve(amps2, max_iter=its[first], tol=1e-7)
    assert torch.equal(amps[first][1], amps2[first][1]) and torch.equal(amps[first][0], amps2[first][0])


def test_autotune_cache_serves_same_shaped_contractions(cc):
    """cc_plan_autotune keeps each pick in a process-wide cache keyed by the
    contraction's route and shape: a second plan of the same system size takes
    every pick from it (no timing) and ends with the same configurations."""
    ccm, engine = cc
    s = systems([(6, 30, 31)])[0]
    d = engine.DeviceSystem.from_system(s, device=DEV)
    ccm.cc_autotune_cache(clear=True)
    a = engine.Engine(d, list_name="ccsd_vvvv", precision="bf16x3")
    a.autotune(*zeros(s.o, s.v), reps=1)
    n1, h1 = ccm.cc_autotune_cache()
    tunable = sum(1 for st in a.plan.describe()["steps"] if len(st.get("configs", [])) >= 2)
    assert n1 >= 1 and h1 <= tunable
    b = engine.Engine(d, list_name="ccsd_vvvv", precision="bf16x3")
    b.autotune(*zeros(s.o, s.v), reps=1)
    n2, h2 = ccm.cc_autotune_cache()
    assert n2 == n1 and h2 - h1 == tunable
    pick = lambda e: [(st.get("bn"), st["splitk"], st.get("red")) for st in e.plan.describe()["steps"]
                      if len(st.get("configs", [])) >= 2]
    assert pick(a) == pick(b)
