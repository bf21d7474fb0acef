"""Parity at the benchmark's full size (o=40, v=200, L=120), in the launch
configuration bench.py times (the split-bf16 plan autotuned first).

The oracle cannot hold the n^4 integrals here, so it evaluates sampled R2
elements one by one from B (oracle.R2Sampler, the explicit-loop oracle's
sampled-element routine, pinned against the determinant brute force at small
sizes).  The samples sit on the tile edges of the dominant contraction (the
particle ladder, GEMM M = (ab) = v^2 rows in 128-row tiles, N = (ij) = o^2
columns in seven column tiles of 240/240/224/.../224), on the first and last
occupied and virtual indices, and on the exact zeros i = j and a = b.

Every sample of every route is compared with the oracle element by element:
FP64 within 1e-9 (the stated FP64 bar); the split routes within the
element-wise bound of their own routes propagated through the list
(list_exec.run_list_bounds, in its moduli form so that no n^4 tensor is
formed).  Antisymmetry of R2 holds at any size and is checked over the whole
array.
"""
import numpy as np
import pytest
import torch

import ccinputs
import list_exec
import oracle
from gpu_util import DEV, to_dev

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


def tile_edge_samples(o, v, seed):
    """(i, j, a, b) rows: 14 column-tile edges of (ij) x 19 row-tile edges of
    (ab), plus the i = j / a = b zeros and the corners."""
    n = o * o
    ntile = -(-n // 256)
    units = n // 16
    widths = [16 * (units // ntile + (1 if t < units % ntile else 0)) for t in range(ntile)]
    edges = np.cumsum([0] + widths)
    ij = sorted({int(x) for e in edges for x in (e - 1, e) if 0 <= x < n})
    m = v * v
    rb = [0, 1, 2, 40, 80, m // 128 // 2, m // 128 - 1, m // 128]
    ab = sorted({int(x) for r in rb for x in (128 * r - 1, 128 * r) if 0 <= x < m} | {m - 2, m - 1})
    rng = np.random.default_rng(seed)
    ab += [int(x) for x in rng.integers(0, m, max(0, 19 - len(ab)))]
    rows = [(p // o, p % o, q // v, q % v) for p in ij for q in ab[:19]]
    rows += [(0, 0, 3, 7), (5, 9, 11, 11), (0, 1, 0, 1), (o - 1, o - 2, v - 1, v - 2), (o - 1, o - 1, v - 1, v - 1)]
    return np.array(rows, dtype=np.int32)


def _plan(engine, dsys, name, prec, T1, T2, tune):
    eng = engine.Engine(dsys, list_name=name, precision=prec)
    if tune:
        eng.autotune(T1, T2, reps=2)
        eng.release()
    return eng


@pytest.fixture(scope="module")
def full():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2409_06759_b300 import engine
    s = ccinputs.make_system(**ccinputs.CONFIG_LADDER)
    t1, t2 = ccinputs.random_amplitudes(s.o, s.v, seed=0, scale1=0.01, scale2=0.01)
    dsys = engine.DeviceSystem.from_system(s, device=DEV)
    idx = tile_edge_samples(s.o, s.v, 5)
    with oracle.R2Sampler(s.o, s.v, s.B, s.eps, t1, t2) as smp:
        want = smp.eval(idx)
    return s, t1, t2, dsys, engine, idx, want


def test_sample_set_covers_the_tile_edges(full):
    """(the oracle's sampled routine adds and subtracts the P(ij)P(ab) partners
    one by one, so its i = j or a = b elements are zero to rounding only)"""
    s, t1, t2, dsys, engine, idx, want = full
    assert len(idx) >= 256
    z = (idx[:, 0] == idx[:, 1]) | (idx[:, 2] == idx[:, 3])
    assert z.sum() >= 4 and np.abs(want[z]).max() <= 1e-15 * np.abs(want).max()


def test_fp64_residual_sampled_elements_match_oracle(full):
    s, t1, t2, dsys, engine, idx, want = full
    eng = engine.Engine(dsys, list_name="ccsd")
    r1, r2 = eng.residual(to_dev(t1), to_dev(t2))
    torch.cuda.synchronize()
    got = r2[tuple(torch.as_tensor(idx.T.astype(np.int64)))].cpu().numpy()
    err = np.abs(got - want)
    assert err.max() < 1e-9, (err.max(), idx[np.argmax(err)])
    g = r2.cpu().numpy()
    scale = np.abs(g).max()
    assert np.abs(g + g.transpose(1, 0, 2, 3)).max() <= 1e-13 * scale
    assert np.abs(g + g.transpose(0, 1, 3, 2)).max() <= 1e-13 * scale
    del eng


@pytest.fixture(scope="module")
def split_runs(full):
    """The bf16x3 plan (autotuned, as bench.py times it) and the bf16x6 plan:
    their sampled R2 elements and the element-wise bounds of their routes."""
    s, t1, t2, dsys, engine, idx, want = full
    import paper_2409_06759_b300 as ccm
    T1, T2 = to_dev(t1), to_dev(t2)
    got, desc = {}, {}
    for prec in ("bf16x3", "bf16x6"):
        eng = _plan(engine, dsys, "ccsd_vvvv", prec, T1, T2, tune=(prec == "bf16x3"))
        r1, r2 = eng.residual(T1, T2)
        torch.cuda.synchronize()
        got[prec] = r2[tuple(torch.as_tensor(idx.T.astype(np.int64)))].cpu().numpy()
        g = r2.cpu().numpy()
        scale = np.abs(g).max()
        assert np.abs(g + g.transpose(1, 0, 2, 3)).max() <= 1e-13 * scale
        desc[prec] = eng.plan.describe()
        del eng, r1, r2, g
        torch.cuda.empty_cache()
    consts = [list_exec.route_constants(desc[p]) for p in ("bf16x3", "bf16x6")]
    _, bounds = list_exec.run_list_bounds(ccm.load_list("ccsd_vvvv"), s.o, s.v, s.eps,
                                          list_exec.BlockV(s.o, s.v, s.B), t1, t2, consts, magnitudes=True)
    bnd = {p: b[1][tuple(idx.T)] for p, b in zip(("bf16x3", "bf16x6"), bounds)}
    return got, bnd


@pytest.mark.parametrize("prec", ["bf16x3", "bf16x6"])
def test_split_residual_sampled_elements_match_oracle(full, split_runs, prec):
    s, t1, t2, dsys, engine, idx, want = full
    got, bnd = split_runs
    err = np.abs(got[prec] - want)
    lim = bnd[prec] + 1e-13 * np.abs(want).max()
    bad = err > lim
    assert not bad.any(), (prec, int(bad.sum()), idx[np.argmax(err - lim)], err.max())
    # the exact zeros stay exact on the split route too (antisymmetric by construction)
    z = (idx[:, 0] == idx[:, 1]) | (idx[:, 2] == idx[:, 3])
    assert np.all(got[prec][z] == 0.0)


def test_bf16x6_is_closer_to_the_oracle_than_bf16x3(full, split_runs):
    """The three-plane route's error is below the two-plane route's on the
    samples as a whole (an extra check on the precision ordering)."""
    s, t1, t2, dsys, engine, idx, want = full
    got, _ = split_runs
    e3 = np.linalg.norm(got["bf16x3"] - want)
    e6 = np.linalg.norm(got["bf16x6"] - want)
    assert e6 < 0.1 * e3, (e3, e6)


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
    """complex128 at o=40 v=200: the FP64 route and the bf16x3 split route (the
    bench's configuration) against sampled oracle elements (complex build),
    FP64 within 1e-9, the split route within its element-wise bound (moduli
    form, twice the real rule per complex element); antisymmetry."""
    import paper_2409_06759_b300 as ccm
    s, t1, t2, dsys, engine = full_c
    o, v = s.o, s.v
    T1, T2 = zdev(t1), zdev(t2)
    idx = tile_edge_samples(o, v, 6)[::3]
    with oracle.R2Sampler(o, v, s.B, s.eps, t1, t2) as smp:
        want = smp.eval(idx)
    sel = tuple(torch.as_tensor(idx.T.astype(np.int64)))
    eng = engine.Engine(dsys, list_name="ccsd")
    r1, r2 = eng.residual(T1, T2)
    torch.cuda.synchronize()
    got = r2[sel].cpu().numpy()
    assert np.abs(got - want).max() < 1e-9
    g = r2.cpu().numpy()
    scale = np.abs(g).max()
    assert np.abs(g + g.transpose(1, 0, 2, 3)).max() <= 1e-13 * scale
    del eng, r1, r2, g
    torch.cuda.empty_cache()
    mix = engine.Engine(dsys, list_name="ccsd_vvvv", precision="bf16x3")
    m1, m2 = mix.residual(T1, T2)
    torch.cuda.synchronize()
    gm = m2[sel].cpu().numpy()
    c = {k: 2.0 * x for k, x in list_exec.route_constants(mix.plan.describe()).items()}
    del mix, m1, m2
    torch.cuda.empty_cache()
    _, [(_, e2)] = list_exec.run_list_bounds(ccm.load_list("ccsd_vvvv"), o, v, s.eps, list_exec.BlockV(o, v, s.B),
                                             t1, t2, [c], magnitudes=True)
    lim = e2[tuple(idx.T)] + 1e-13 * np.abs(want).max()
    err = np.abs(gm - want)
    assert (err <= lim).all(), (int((err > lim).sum()), err.max())
