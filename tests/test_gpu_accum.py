"""Elementwise steps (permuted copies, outer products with permutation
operators, antisymmetrising epilogues) against the numpy executor of the
list grammar, through the C ABI.

Each statement below is chosen to land on one of the accumulate kernels
(pair antisymmetriser, row kernel with one or two sources, tiled transpose
kernel, flat copy) with alpha = 1, +-2^k or a general value and beta = 0 or 1,
at sizes whose 32-wide tiles are ragged and at o = 1, where P(ij) has only
i = j orbits (exact zeros).  The amplitudes are plain random arrays (not
antisymmetric), so every one of the four orbit members enters the sums with
its own value.  The kernels add at most nterms values per element, so the
tolerance is a few ulps of the largest term.
"""
import numpy as np
import pytest
import torch

import ccinputs
import list_exec
import oracle
from gpu_util import DEV

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cc():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2409_06759_b300 as cc
    from paper_2409_06759_b300 import engine
    return cc, engine


LISTS = [
    # pair antisymmetriser: beta 0, alpha 1 / -0.5 with beta 1 / general alpha, swapped base term
    "R2[ijab] = P(ij) P(ab) T2[ijab]",
    "R2[ijab] = T2[ijab]\nR2[ijab] += -0.5 P(ij) P(ab) T2[ijab]",
    "R2[ijab] = 0.3 P(ij) P(ab) T2[jiab]",
    # row kernel: copy (collapses to one dim), two-source outer products
    "R2[ijab] = T2[ijab]\nR2[ijab] += 0.5 P(ab) T1[ia] * T1[jb]",
    "R2[ijab] = P(ij) P(ab) T1[ia] * T1[jb]",
    "R2[ijab] = -3 P(ij) T2[ijab]",
    # a permuted copy fused with the outer product that follows it
    "R2[ijab] = T2[jiba]\nR2[ijab] += -0.25 P(ij) T1[ia] * T1[jb]",
    # tiled kernel: transposed sources, mixed direct / transposed terms
    "R2[ijab] = T2[jiba]",
    "R2[ijab] = 0.25 V[abij]",
    "R2[ijab] = T2[ijab]\nR2[ijab] += P(ab) T2[ijab]",
    "R1[ia] = 3 T1[ia]\nR2[ijab] = -1 T2[ijba]",
]

SIZES = [(3, 20), (5, 45), (2, 70), (1, 33)]


def _inputs(o, v, seed, complex_):
    s = ccinputs.make_system(o, v, L=6, seed=seed, complex_=complex_)
    rng = np.random.default_rng(seed + 1000)
    t1 = rng.standard_normal((o, v))
    t2 = rng.standard_normal((o, o, v, v))
    if complex_:
        t1 = t1 + 1j * rng.standard_normal((o, v))
        t2 = t2 + 1j * rng.standard_normal((o, o, v, v))
    return s, t1, t2


def _run(cc, text, o, v, seed, complex_):
    ccm, engine = cc
    s, t1, t2 = _inputs(o, v, seed, complex_)
    B = s.B * 6.0
    dsys = engine.DeviceSystem(o, v, s.eps_occ, s.eps_vir, B, device=DEV)
    eng = engine.Engine(dsys, list_text=text, precision="fp64")
    dt = torch.complex128 if complex_ else torch.float64
    T1 = torch.tensor(t1, dtype=dt, device=DEV)
    T2 = torch.tensor(t2, dtype=dt, device=DEV)
    r1 = torch.zeros(o, v, dtype=dt, device=DEV)
    r2 = torch.zeros(o, o, v, v, dtype=dt, device=DEV)
    ccm.cc_residual(eng.plan, dsys.ints(), T1, T2, r1, r2, eng.ws)
    torch.cuda.synchronize()
    e1, e2 = list_exec.run_list(text, o, v, s.eps, oracle.antisym_integrals(o, v, B), t1, t2)
    return r1.cpu().numpy(), r2.cpu().numpy(), e1, e2


@pytest.mark.parametrize("o,v", SIZES)
@pytest.mark.parametrize("k", range(len(LISTS)))
def test_accumulate_statement_real(cc, k, o, v):
    g1, g2, e1, e2 = _run(cc, LISTS[k], o, v, 70 + k, False)
    scale = max(1.0, np.abs(e1).max(), np.abs(e2).max())
    assert np.abs(g1 - e1).max() <= 4e-15 * scale * 4
    assert np.abs(g2 - e2).max() <= 4e-15 * scale * 4


@pytest.mark.parametrize("o,v", [(3, 20), (5, 45)])
@pytest.mark.parametrize("k", [0, 1, 3, 6, 7, 8])
def test_accumulate_statement_complex(cc, k, o, v):
    g1, g2, e1, e2 = _run(cc, LISTS[k], o, v, 90 + k, True)
    scale = max(1.0, np.abs(e1).max(), np.abs(e2).max())
    assert np.abs(g1 - e1).max() <= 4e-15 * scale * 8
    assert np.abs(g2 - e2).max() <= 4e-15 * scale * 8


@pytest.mark.parametrize("list_name,prec", [("ccsd", "fp64"), ("ccsd_vvvv", "bf16x3")])
def test_residual_is_exactly_antisymmetric(cc, list_name, prec):
    """The CCSD lists end in R2 = P(ij) P(ab) Z2; the orbit kernel writes +-X
    to all four orbit members, and the denominator update preserves the
    antisymmetry of T2, so the residual is antisymmetric bit for bit and its
    i = j and a = b planes are zero."""
    ccm, engine = cc
    o, v = 5, 45
    s = ccinputs.make_system(o, v, L=6, seed=8)
    t1, t2 = ccinputs.random_amplitudes(o, v, seed=8, scale1=0.05, scale2=0.05)
    dsys = engine.DeviceSystem(o, v, s.eps_occ, s.eps_vir, s.B * 6.0, device=DEV)
    eng = engine.Engine(dsys, list_name=list_name, precision=prec)
    r1, r2 = eng.residual(torch.tensor(t1, device=DEV), torch.tensor(t2, device=DEV))
    g2 = r2.cpu().numpy()
    assert np.abs(g2).max() > 0
    assert np.array_equal(g2, -g2.transpose(1, 0, 2, 3))
    assert np.array_equal(g2, -g2.transpose(0, 1, 3, 2))
    assert not np.any(g2[np.arange(o), np.arange(o)])
    assert not np.any(g2[:, :, np.arange(v), np.arange(v)])


TRIPLE_LISTS = [
    # the triple antisymmetriser over the occupied dims (orbit kernel): =, += with alpha, and a
    # permuted base term; over the virtual dims (transposing tiles)
    "R3[ijkabc] = P(i/jk) P(jk) T3[ijkabc]",
    "R3[ijkabc] = T3[ijkabc]\nR3[ijkabc] += -0.5 P(i/jk) P(jk) T3[ijkabc]",
    "R3[ijkabc] = 0.25 P(i/jk) P(jk) T3[jikabc]",
    "R3[ijkabc] = P(a/bc) P(bc) T3[ijkabc]",
    "R3[ijkabc] = T3[ijkabc]\nR3[ijkabc] += 0.5 P(a/bc) P(bc) T3[ijkabc]",
    "R3[ijkabc] = -2 P(a/bc) P(bc) T3[ijkacb]",
]


@pytest.mark.parametrize("o,v", [(4, 6), (5, 5), (3, 9), (3, 37)])
@pytest.mark.parametrize("k", range(len(TRIPLE_LISTS)))
def test_triple_antisymmetrisers(cc, k, o, v):
    """Six-term antisymmetrisers of a rank-3 array (plain random, so every
    orbit member enters with its own value); rows with a repeated occupied
    index come out as exact zeros."""
    ccm, engine = cc
    text = TRIPLE_LISTS[k]
    s = ccinputs.make_system(o, v, L=6, seed=k)
    rng = np.random.default_rng(200 + k)
    t1 = rng.standard_normal((o, v))
    t2 = rng.standard_normal((o, o, v, v))
    t3 = rng.standard_normal((o, o, o, v, v, v))
    dsys = engine.DeviceSystem(o, v, s.eps_occ, s.eps_vir, s.B, device=DEV)
    eng = engine.Engine(dsys, list_text=text, precision="fp64")
    T = [torch.tensor(x, device=DEV) for x in (t1, t2, t3)]
    r1, r2, r3 = eng.residual(T[0], T[1], t3=T[2])
    torch.cuda.synchronize()
    e1, e2, e3 = list_exec.run_list(text, o, v, s.eps, oracle.antisym_integrals(o, v, s.B), t1, t2, t3)
    g3 = r3.cpu().numpy()
    scale = max(1.0, np.abs(e3).max())
    assert np.abs(g3 - e3).max() <= 8 * 4e-15 * scale


@pytest.mark.parametrize("complex_", [False, True])
@pytest.mark.parametrize("o,v", [(3, 7), (5, 37)])
def test_every_integral_orientation_copies_exactly(cc, o, v, complex_):
    """R2[ijab] = V[p q r s] for all 24 orders of the letters i, j, a, b: each
    resolves onto a stored block through <pq||rs> = -<qp||rs> = -<pq||sr> =
    <rs||pq>* (a sign and, for complex orbitals, a conjugation), then a
    permuted copy.  The device blocks are loaded with the oracle's own
    integrals and T = 0, so the result must equal the einsum reading bit for
    bit (signs, conjugations and copies are exact)."""
    import itertools
    ccm, engine = cc
    s = ccinputs.make_system(o, v, L=6, seed=11, complex_=complex_)
    dsys = engine.DeviceSystem(o, v, s.eps_occ, s.eps_vir, s.B, device=DEV)
    V = oracle.antisym_integrals(o, v, s.B)
    sl = {"o": slice(0, o), "v": slice(o, o + v)}
    for name, blk in dsys.blocks.items():
        sub = V[sl[name[0]], sl[name[1]], sl[name[2]], sl[name[3]]]
        blk.copy_(torch.from_numpy(np.ascontiguousarray(sub).reshape(-1)).to(blk.dtype))
    dt = torch.complex128 if complex_ else torch.float64
    npdt = np.complex128 if complex_ else np.float64
    T1 = torch.zeros(o, v, dtype=dt, device=DEV)
    T2 = torch.zeros(o, o, v, v, dtype=dt, device=DEV)
    z1, z2 = np.zeros((o, v), dtype=npdt), np.zeros((o, o, v, v), dtype=npdt)
    for perm in itertools.permutations("ijab"):
        text = "R2[ijab] = V[" + "".join(perm) + "]"
        eng = engine.Engine(dsys, list_text=text, precision="fp64")
        r1, r2 = eng.residual(T1, T2)
        torch.cuda.synchronize()
        _, e2 = list_exec.run_list(text, o, v, s.eps, V, z1, z2)
        assert np.array_equal(r2.cpu().numpy(), e2), text
