"""Parity at the benchmark's full size (o=40, v=200, L=120), in the launch
configuration bench.py times.  The oracle cannot hold the n^4 integrals here,
so it computes sampled R2 elements one by one from B (oracle.ccsd_r2_sample,
itself pinned against the determinant brute force at small sizes); the
split-bf16 route is compared with the FP64 route over the whole array, and the
antisymmetry of R2 holds at any size.
"""
import numpy as np
import pytest
import torch

import ccinputs
import oracle
from gpu_util import DEV, to_dev

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def full():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2409_06759_b300 import engine
    s = ccinputs.make_system(**ccinputs.CONFIG_LADDER)
    t1, t2 = ccinputs.random_amplitudes(s.o, s.v, seed=0, scale1=0.01, scale2=0.01)
    dsys = engine.DeviceSystem.from_system(s, device=DEV)
    return s, t1, t2, dsys, engine


def test_fp64_residual_sampled_elements_match_oracle(full):
    s, t1, t2, dsys, engine = full
    o, v = s.o, s.v
    eng = engine.Engine(dsys, list_name="ccsd")
    r1, r2 = eng.residual(to_dev(t1), to_dev(t2))
    torch.cuda.synchronize()
    rng = np.random.default_rng(5)
    idx = np.stack([rng.integers(0, o, 6), rng.integers(0, o, 6), rng.integers(0, v, 6), rng.integers(0, v, 6)], 1)
    idx[0] = (0, 1, 0, 1)
    idx[1] = (o - 1, o - 2, v - 1, v - 2)          # ragged-tail corner
    want = oracle.ccsd_r2_sample(o, v, s.B, s.eps, t1, t2, idx)
    got = r2[idx[:, 0], idx[:, 1], idx[:, 2], idx[:, 3]].cpu().numpy()
    assert np.abs(got - want).max() < 1e-9
    g = r2.cpu().numpy()
    scale = np.abs(g).max()
    assert np.abs(g + g.transpose(1, 0, 2, 3)).max() <= 1e-13 * scale
    assert np.abs(g + g.transpose(0, 1, 3, 2)).max() <= 1e-13 * scale
    del eng


@pytest.mark.parametrize("prec,rel", [("bf16x3", 1e-5), ("bf16x6", 2e-7)])
def test_mixed_residual_matches_fp64_route(full, prec, rel):
    s, t1, t2, dsys, engine = full
    T1, T2 = to_dev(t1), to_dev(t2)
    ref = engine.Engine(dsys, list_name="ccsd")
    f1, f2 = ref.residual(T1, T2)
    torch.cuda.synchronize()
    f1, f2 = f1.cpu(), f2.cpu()
    del ref
    mix = engine.Engine(dsys, list_name="ccsd_vvvv", precision=prec)
    m1, m2 = mix.residual(T1, T2)
    torch.cuda.synchronize()
    d = torch.sqrt(((m1.cpu() - f1) ** 2).sum() + ((m2.cpu() - f2) ** 2).sum()).item()
    n = torch.sqrt((f1 ** 2).sum() + (f2 ** 2).sum()).item()
    assert d <= rel * n, (d, n)


@pytest.fixture(scope="module")
def full_c():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2409_06759_b300 import engine
    s = ccinputs.make_system(**ccinputs.CONFIG_LADDER, complex_=True)
    t1, t2 = ccinputs.random_amplitudes(s.o, s.v, seed=0, scale1=0.01, scale2=0.01, complex_=True)
    dsys = engine.DeviceSystem.from_system(s, device=DEV)
    return s, t1, t2, dsys, engine


def zdev(x):
    return torch.tensor(np.ascontiguousarray(x), dtype=torch.complex128, device=DEV)


def test_complex_residuals_at_full_size(full_c):
    """complex128 at o=40 v=200: FP64 route against sampled oracle elements
    (complex build), antisymmetry, and the bf16x3 split route (the bench's
    configuration) against the FP64 route over the whole array."""
    s, t1, t2, dsys, engine = full_c
    o, v = s.o, s.v
    T1, T2 = zdev(t1), zdev(t2)
    eng = engine.Engine(dsys, list_name="ccsd")
    r1, r2 = eng.residual(T1, T2)
    torch.cuda.synchronize()
    rng = np.random.default_rng(6)
    idx = np.stack([rng.integers(0, o, 4), rng.integers(0, o, 4), rng.integers(0, v, 4), rng.integers(0, v, 4)], 1)
    idx[0] = (0, 1, 0, 1)
    idx[1] = (o - 1, o - 2, v - 1, v - 2)
    want = oracle.ccsd_r2_sample(o, v, s.B, s.eps, t1, t2, idx)
    got = r2[idx[:, 0], idx[:, 1], idx[:, 2], idx[:, 3]].cpu().numpy()
    assert np.abs(got - want).max() < 1e-9
    f1, f2 = r1.cpu(), r2.cpu()
    g = f2.numpy()
    scale = np.abs(g).max()
    assert np.abs(g + g.transpose(1, 0, 2, 3)).max() <= 1e-13 * scale
    del eng, r1, r2
    mix = engine.Engine(dsys, list_name="ccsd_vvvv", precision="bf16x3")
    m1, m2 = mix.residual(T1, T2)
    torch.cuda.synchronize()
    d = torch.sqrt((m1.cpu() - f1).abs().pow(2).sum() + (m2.cpu() - f2).abs().pow(2).sum()).item()
    n = torch.sqrt(f1.abs().pow(2).sum() + f2.abs().pow(2).sum()).item()
    assert d <= 2e-5 * n, (d, n)
