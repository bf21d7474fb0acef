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


def test_split_rounding_matches_the_library_conversion(cc):
    """The split kernels round double -> float on the integer pipe; the result is
    bit-identical to the library conversion over normal, tie, carry, tiny,
    huge, signed-zero and special values."""
    ccm, _ = cc
    rng = np.random.default_rng(0)
    vals = np.concatenate([
        rng.standard_normal(200000) * 10.0 ** rng.integers(-30, 30, 200000),
        np.array([0.0, -0.0, 1.0, -1.0, 3.0e38, -3.4028234663852886e38, 3.4028235677973366e38, 1e-38, 1e-40, 1e-46,
                  5e-324, float("inf"), -float("inf"), float("nan")]),
        # exact ties between two floats, and values just off them
        ((2.0 ** 23 + rng.integers(0, 2 ** 23, 4096)) + 0.5) * 2.0 ** rng.integers(-60, 60, 4096).astype(float),
        1.0 + np.arange(0, 2000) * 2.0 ** -52,
    ])
    x = torch.tensor(vals, dtype=torch.float64, device=DEV)
    mine = torch.empty(x.numel(), dtype=torch.float32, device=DEV)
    ref = torch.empty_like(mine)
    ccm.cc_selftest_convert(x, mine, ref)
    a = mine.cpu().numpy().view(np.uint32)
    b = ref.cpu().numpy().view(np.uint32)
    nan = np.isnan(ref.cpu().numpy())
    assert np.array_equal(a[~nan], b[~nan])
    assert np.isnan(mine.cpu().numpy()[nan]).all()


def _solver_case(engine, o=3, v=8):
    s, B, t1, t2 = small_case(o, v, 5, L=6, scale=6.0, tscale=0.05)
    dsys = engine.DeviceSystem(o, v, s.eps_occ, s.eps_vir, B, device=DEV)
    return engine.Engine(dsys, list_name="ccsd"), o, v


def test_solve_reports_max_iterations_without_converging(cc):
    """max_iter reached: CC_ERR_NOT_CONVERGED (7) with every iteration's finite
    energy and |R| reported, and the amplitudes left at the last iterate."""
    ccm, engine = cc
    eng, o, v = _solver_case(engine)
    t1 = torch.zeros(o, v, dtype=torch.float64, device=DEV)
    t2 = torch.zeros(o, o, v, v, dtype=torch.float64, device=DEV)
    res = engine.Solver(eng).solve(t1, t2, max_iter=3, tol=1e-300)
    assert res.status == 7 and not res.converged and res.iterations == 3
    assert "maximum iterations" in ccm.cc_last_error()
    assert all(np.isfinite(res.rnorms)) and all(np.isfinite(res.energies))
    assert res.rnorms[-1] < res.rnorms[0]
    assert torch.isfinite(t2).all() and t2.abs().max().item() > 0


def test_solve_stops_on_a_non_finite_residual(cc):
    """A NaN placed in the starting amplitudes on the host (the injected fault)
    makes |R| non-finite in the first iteration: cc_solve stops there with
    CC_ERR_NOT_CONVERGED and says why, and the next solve on clean inputs in
    the same context converges."""
    ccm, engine = cc
    eng, o, v = _solver_case(engine)
    t1 = torch.zeros(o, v, dtype=torch.float64, device=DEV)
    h2 = torch.zeros(o, o, v, v, dtype=torch.float64)
    h2[0, 1, 2, 3] = float("nan")
    t2 = h2.to(DEV)
    res = engine.Solver(eng).solve(t1, t2, max_iter=20, tol=1e-8)
    assert res.status == 7 and not res.converged and res.iterations == 1
    assert "divergence" in ccm.cc_last_error()
    assert not np.isfinite(res.rnorms[0])
    t1.zero_()
    t2.zero_()
    ok = engine.Solver(eng).solve(t1, t2, max_iter=60, tol=1e-8)
    assert ok.status == 0 and ok.converged
