"""The derivation of contraction lists (paper_2409_06759_b300/gen.py) against
what fixes it independently: the paper's diagram counts (Tab. gener: CCD
11, CCSD 48, CCSDT 102), the FP64 oracle (CCSD) and the determinant-space
brute force (CCSDT, with T3), for real and complex orbitals."""
import os

import numpy as np
import pytest

import ccinputs
import detspace
import list_exec
import oracle
from paper_2409_06759_b300 import gen

LISTS = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2409_06759_b300", "lists")


@pytest.mark.parametrize("method,count", [("ccd", 11), ("ccsd", 48), ("ccsdt", 102)])
def test_diagram_counts_match_the_paper(method, count):
    assert gen.count_diagrams(method) == count


def test_fast_canonical_form_agrees_with_the_full_group_search():
    """Both canonical forms induce the same partition of the raw terms into
    equal terms with the same relative signs."""
    for k, ranks in ((2, (1, 2)), (3, (1, 2, 3))):
        seen_fast, seen_brute = {}, {}
        for levels in ([2], [1, 2], [3], [1, 3], [2, 2], [1, 1, 2]):
            if any(n not in ranks for n in levels):
                continue
            for sign, hl, tls in gen.contractions(k, "V", list(levels)):
                kf, sf = gen.canonical("V", hl, tls)
                kb, sb = gen.canonical_brute("V", hl, tls)
                if kf in seen_fast:
                    kb0, rel = seen_fast[kf]
                    assert kb0 == kb and rel == sf * sb
                else:
                    seen_fast[kf] = (kb, sf * sb)
                    assert kb not in seen_brute
                    seen_brute[kb] = kf


@pytest.mark.parametrize("cplx", [False, True])
@pytest.mark.parametrize("o,v,seed", [(2, 3, 1), (3, 4, 2), (4, 5, 3)])
def test_generated_ccsd_list_matches_oracle(cplx, o, v, seed):
    text = gen.generate("ccsd", 8, 64)
    s = ccinputs.make_system(o, v, L=6, seed=seed, complex_=cplx)
    V = oracle.antisym_integrals(o, v, s.B * 6.0)
    t1, t2 = ccinputs.random_amplitudes(o, v, seed=seed, scale1=0.1, scale2=0.1, complex_=cplx)
    r1, r2 = oracle.ccsd_residual(o, v, s.eps, V, t1, t2)
    l1, l2 = list_exec.run_list(text, o, v, s.eps, V, t1, t2)
    assert np.abs(r1 - l1).max() < 1e-13 and np.abs(r2 - l2).max() < 1e-13


@pytest.mark.parametrize("cplx", [False, True])
@pytest.mark.parametrize("o,v,seed", [(3, 4, 1), (3, 5, 2)])
def test_shipped_ccsdt_list_matches_brute_force(cplx, o, v, seed):
    text = open(os.path.join(LISTS, "ccsdt.txt")).read()
    s = ccinputs.make_system(o, v, L=6, seed=seed, complex_=cplx)
    V = oracle.antisym_integrals(o, v, s.B * 6.0)
    t1, t2, t3 = ccinputs.random_amplitudes(o, v, seed=seed, scale1=0.1, scale2=0.1, triples=True, complex_=cplx)
    _, b1, b2, b3 = detspace.brute_residual(o, v, s.eps, V, t1, t2, t3)
    l1, l2, l3 = list_exec.run_list(text, o, v, s.eps, V, t1, t2, t3)
    scale = max(np.abs(b3).max(), np.abs(b2).max())
    assert np.abs(b3).max() > 1e-2                    # the triples residual is exercised
    for got, want in ((l1, b1), (l2, b2), (l3, b3)):
        assert np.abs(got - want).max() < 1e-13 * max(1.0, scale)


def test_shipped_ccsdt_list_is_the_generator_output():
    text = open(os.path.join(LISTS, "ccsdt.txt")).read()
    body = [l for l in text.splitlines() if l and not l.startswith("#")]
    fresh = [l for l in gen.generate("ccsdt", 8, 64).splitlines() if l and not l.startswith("#")]
    assert body == fresh


def test_ccsdt_list_factorisation_keeps_the_triples_ladder_as_one_gemm():
    """The o^3 v^5 particle ladder 1/2 <ab||ef> t_ijk^efc is one contraction
    of T3 with the vvvv block (trailing virtual pair contracted, no T3 copy)."""
    text = open(os.path.join(LISTS, "ccsdt.txt")).read()
    lad = [l for l in text.splitlines() if l.startswith("Z3") and "V[" in l and "T3[" in l
           and all(c in "abcdefg" for c in l.split("V[")[1][:4])]
    assert len(lad) == 1


def test_deferred_antisymmetrisation_matches_per_diagram_operators():
    """One full antisymmetriser over the weighted sum of unsymmetrised terms
    equals the per-diagram P(..) operators (both against the brute force's
    reference values through the einsum reading)."""
    o, v = 3, 5
    s = ccinputs.make_system(o, v, L=6, seed=9)
    V = oracle.antisym_integrals(o, v, s.B * 6.0)
    t1, t2, t3 = ccinputs.random_amplitudes(o, v, seed=9, scale1=0.1, scale2=0.1, triples=True)
    a = list_exec.run_list(gen.generate("ccsdt", 8, 64, defer=False), o, v, s.eps, V, t1, t2, t3)
    b = list_exec.run_list(gen.generate("ccsdt", 8, 64, defer=True), o, v, s.eps, V, t1, t2, t3)
    for x, y in zip(a, b):
        assert np.abs(x - y).max() < 1e-14
