"""The shipped contraction lists, evaluated by an independent numpy.einsum
reading of the grammar, reproduce the oracle residual (CPU)."""
import os

import numpy as np
import pytest

import ccinputs
import list_exec
import oracle

LISTS = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2409_06759_b300", "lists")


@pytest.mark.parametrize("name", ["ccsd", "ccsd_vvvv", "ccsd_packed"])
@pytest.mark.parametrize("o,v,seed", [(2, 3, 1), (3, 4, 2), (4, 5, 3)])
def test_list_matches_oracle(name, o, v, seed):
    text = open(os.path.join(LISTS, name + ".txt")).read()
    s = ccinputs.make_system(o, v, L=6, seed=seed)
    V = oracle.antisym_integrals(o, v, s.B * 6.0)
    t1, t2 = ccinputs.random_amplitudes(o, v, seed=seed, scale1=0.1, scale2=0.1)
    r1, r2 = oracle.ccsd_residual(o, v, s.eps, V, t1, t2)
    l1, l2 = list_exec.run_list(text, o, v, s.eps, V, t1, t2)
    assert np.abs(r1 - l1).max() < 1e-13
    assert np.abs(r2 - l2).max() < 1e-13


@pytest.mark.parametrize("name", ["ccsd", "ccsd_vvvv", "ccsd_packed"])
@pytest.mark.parametrize("o,v,seed", [(2, 3, 11), (3, 5, 12)])
def test_list_matches_complex_oracle(name, o, v, seed):
    """Complex orbitals: the lists name each integral in the orientation the
    projection fixes (e.g. <ab||ij> for the doubles driver), so they hold as
    written for complex Hermitian integrals."""
    text = open(os.path.join(LISTS, name + ".txt")).read()
    s = ccinputs.make_system(o, v, L=6, seed=seed, complex_=True)
    V = oracle.antisym_integrals(o, v, s.B * 6.0)
    t1, t2 = ccinputs.random_amplitudes(o, v, seed=seed, scale1=0.1, scale2=0.1, complex_=True)
    r1, r2 = oracle.ccsd_residual(o, v, s.eps, V, t1, t2)
    l1, l2 = list_exec.run_list(text, o, v, s.eps, V, t1, t2)
    assert np.abs(r2.imag).max() > 1e-3
    assert np.abs(r1 - l1).max() < 1e-13
    assert np.abs(r2 - l2).max() < 1e-13
