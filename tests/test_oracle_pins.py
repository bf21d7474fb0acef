"""Pins of the FP64 oracle against things other than itself.

* determinant-space brute force of <Phi_l| exp(-T) H_N exp(T) |Phi_0> (Eq. amp)
  for random, non-converged T at tiny o/v: every residual element and the energy;
* the converged CCSD energy equals FCI for two electrons (CCSD is exact there);
* the first Jacobi step from T = 0 gives the MP2 energy, computed here by
  second-order Moller-Plesset perturbation theory on determinant-space H elements;
* antisymmetry of R2 in (ij) and (ab); integral symmetries;
* DIIS coefficients vs the closed form c = B^-1 1 / (1^T B^-1 1);
* lambda scaling: E(lambda V) = lambda^2 E2 + lambda^3 E3 + O(lambda^4), E2 the MP2
  energy and E3 the spin-orbital MP3 closed form (itself checked against
  third-order perturbation theory in determinant space).
"""
import numpy as np
import pytest

import ccinputs
import detspace
import oracle


def _system(o, v, seed, scale=6.0):
    s = ccinputs.make_system(o, v, L=6, seed=seed)
    return s, s.B * scale


@pytest.mark.parametrize("o,v,seed", [(2, 3, 1), (3, 4, 2), (3, 5, 3), (4, 4, 4), (2, 6, 5)])
def test_residual_matches_determinant_brute_force(o, v, seed):
    s, B = _system(o, v, seed)
    V = oracle.antisym_integrals(o, v, B)
    t1, t2 = ccinputs.random_amplitudes(o, v, seed=seed, scale1=0.1, scale2=0.1)
    e_b, r1_b, r2_b = detspace.brute_residual(o, v, s.eps, detspace.antisym_from_B(B), t1, t2)
    r1, r2 = oracle.ccsd_residual(o, v, s.eps, V, t1, t2)
    e = oracle.ccsd_energy(o, v, V, t1, t2)
    scale = max(np.abs(r2_b).max(), np.abs(r1_b).max())
    assert np.abs(r1 - r1_b).max() < 1e-12 * scale
    assert np.abs(r2 - r2_b).max() < 1e-12 * scale
    assert abs(e - e_b) < 1e-13


def test_single_t1t1_sign_rule():
    """One T1*T1 product into R2: the sign of R_ij^ab fixed by 'the line from i ends in a'."""
    o, v = 2, 2
    s, B = _system(o, v, 9)
    V = oracle.antisym_integrals(o, v, B)
    t1 = np.zeros((o, v)); t1[0, 0] = 0.3; t1[1, 1] = 0.2
    t2 = np.zeros((o, o, v, v))
    _, _, r2_b = detspace.brute_residual(o, v, s.eps, V, t1, t2)
    _, r2 = oracle.ccsd_residual(o, v, s.eps, V, t1, t2)
    assert np.abs(r2 - r2_b).max() < 1e-14
    assert np.sign(r2[0, 1, 0, 1]) == np.sign(r2_b[0, 1, 0, 1])


@pytest.mark.parametrize("o,v,seed", [(2, 4, 11), (2, 6, 12)])
def test_ccsd_equals_fci_for_two_electrons(o, v, seed):
    s, B = _system(o, v, seed)
    V = oracle.antisym_integrals(o, v, B)
    res = oracle.ccsd_solve(o, v, s.eps, V, tol=1e-12, maxiter=200)
    assert res["status"] == 0
    assert abs(res["energy"] - detspace.fci_correlation(o, v, s.eps, V)) < 1e-12


@pytest.mark.parametrize("o,v,seed", [(2, 4, 21), (3, 4, 22), (3, 5, 23)])
def test_first_iteration_is_mp2(o, v, seed):
    s, B = _system(o, v, seed)
    V = oracle.antisym_integrals(o, v, B)
    res = oracle.ccsd_solve(o, v, s.eps, V, tol=0.0, maxiter=2)
    assert res["energies"][0] == 0.0
    assert abs(res["energies"][1] - detspace.mp2_det_space(o, v, s.eps, V)) < 1e-14


def test_residual_antisymmetry_and_integral_symmetry():
    o, v = 4, 6
    s, B = _system(o, v, 31)
    V = oracle.antisym_integrals(o, v, B)
    assert np.abs(V + V.transpose(1, 0, 2, 3)).max() < 1e-15
    assert np.abs(V + V.transpose(0, 1, 3, 2)).max() < 1e-15
    assert np.abs(V - V.transpose(2, 3, 0, 1)).max() < 1e-15
    assert np.abs(V - detspace.antisym_from_B(B)).max() < 1e-14
    t1, t2 = ccinputs.random_amplitudes(o, v, seed=31, scale1=0.1, scale2=0.1)
    _, r2 = oracle.ccsd_residual(o, v, s.eps, V, t1, t2)
    assert np.abs(r2 + r2.transpose(1, 0, 2, 3)).max() < 1e-14
    assert np.abs(r2 + r2.transpose(0, 1, 3, 2)).max() < 1e-14


@pytest.mark.parametrize("m", [2, 3, 5, 8])
def test_diis_coefficients_closed_form(m):
    rng = np.random.default_rng(m)
    E = rng.standard_normal((m, 50))
    Bm = E @ E.T
    c = oracle.diis_coeffs(Bm)
    w = np.linalg.solve(Bm, np.ones(m))
    ref = w / w.sum()
    assert np.abs(c - ref).max() < 1e-10
    assert abs(c.sum() - 1.0) < 1e-13


@pytest.mark.parametrize("cplx", [False, True])
@pytest.mark.parametrize("o,v,seed", [(2, 3, 61), (2, 4, 62), (3, 5, 63)])
def test_mp3_closed_form_equals_third_order_perturbation_theory(cplx, o, v, seed):
    """The MP3 closed form used by the lambda pin, against Rayleigh-Schroedinger
    third order on the determinant-space Hamiltonian (no closed form involved)."""
    s = ccinputs.make_system(o, v, L=6, seed=seed, complex_=cplx)
    V = oracle.antisym_integrals(o, v, s.B * 6.0)
    e3 = detspace.mp3_closed_form(o, v, s.eps, V)
    assert abs(e3 - detspace.mp3_det_space(o, v, s.eps, V)) < 1e-13 * max(1.0, abs(e3))


def lambda_coefficients(solve, lam):
    """Coefficients of E(l) = sum_k l^k E_k, k = 2 .. 1 + len(lam), fitted exactly
    through the converged energies at the given scales of the integrals."""
    lam = np.asarray(lam, dtype=float)
    A = np.stack([lam ** k for k in range(2, 2 + lam.size)], 1)
    return np.linalg.solve(A, np.array([solve(x) for x in lam]))


LAMBDAS = [0.01, 0.02, 0.03, 0.04, 0.05]


@pytest.mark.parametrize("o,v,seed,L", [(2, 4, 41, 6), (3, 8, 42, 6), (5, 16, 43, 12)])
def test_energy_lambda_expansion_is_mp2_then_mp3(o, v, seed, L):
    """E_CCSD(lambda V) = lambda^2 E_MP2 + lambda^3 E_MP3 + O(lambda^4): CCSD is
    exact through third order, so the lambda^3 coefficient pins the first-order
    T2 response of the particle ladder, the hole ladder and the ring terms."""
    s = ccinputs.make_system(o, v, L=L, seed=seed)
    V = oracle.antisym_integrals(o, v, s.B * 6.0)
    c = lambda_coefficients(lambda x: oracle.ccsd_solve(o, v, s.eps, V * x, tol=1e-15, maxiter=200)["energy"],
                            LAMBDAS)
    e2 = detspace.mp2_det_space(o, v, s.eps, V) if o + v <= 8 else None
    e3 = detspace.mp3_closed_form(o, v, s.eps, V)
    if e2 is not None:
        assert abs(c[0] - e2) < 1e-10 * abs(e2)
    assert abs(c[1] - e3) < 1e-7 * abs(e3)


@pytest.mark.parametrize("o,v,seed", [(2, 3, 51), (3, 5, 52), (4, 4, 53)])
def test_sampled_elements_match_brute_force_and_full_residual(o, v, seed):
    s, B = _system(o, v, seed)
    t1, t2 = ccinputs.random_amplitudes(o, v, seed=seed, scale1=0.1, scale2=0.1)
    rng = np.random.default_rng(seed)
    idx = np.stack([rng.integers(0, o, 12), rng.integers(0, o, 12), rng.integers(0, v, 12),
                    rng.integers(0, v, 12)], 1)
    got = oracle.ccsd_r2_sample(o, v, B, s.eps, t1, t2, idx)
    _, _, r2_b = detspace.brute_residual(o, v, s.eps, detspace.antisym_from_B(B), t1, t2)
    _, r2 = oracle.ccsd_residual(o, v, s.eps, oracle.antisym_integrals(o, v, B), t1, t2)
    want = r2_b[idx[:, 0], idx[:, 1], idx[:, 2], idx[:, 3]]
    assert np.abs(got - want).max() < 1e-12 * max(1.0, np.abs(r2_b).max())
    assert np.abs(got - r2[idx[:, 0], idx[:, 1], idx[:, 2], idx[:, 3]]).max() < 1e-13


# ----------------------------------------------------------------- complex128
def _csystem(o, v, seed, scale=6.0):
    s = ccinputs.make_system(o, v, L=6, seed=seed, complex_=True)
    return s, s.B * scale


@pytest.mark.parametrize("o,v,seed", [(2, 3, 71), (3, 4, 72), (3, 5, 73)])
def test_complex_residual_matches_determinant_brute_force(o, v, seed):
    s, B = _csystem(o, v, seed)
    V = oracle.antisym_integrals(o, v, B)
    assert np.abs(V - detspace.antisym_from_B(B)).max() < 1e-14
    # Hermitian antisymmetrised integrals
    assert np.abs(V - V.transpose(2, 3, 0, 1).conj()).max() < 1e-14
    t1, t2 = ccinputs.random_amplitudes(o, v, seed=seed, scale1=0.1, scale2=0.1, complex_=True)
    e_b, r1_b, r2_b = detspace.brute_residual(o, v, s.eps, V, t1, t2)
    r1, r2 = oracle.ccsd_residual(o, v, s.eps, V, t1, t2)
    e = oracle.ccsd_energy(o, v, V, t1, t2)
    scale = max(np.abs(r2_b).max(), np.abs(r1_b).max())
    assert np.abs(r1 - r1_b).max() < 1e-12 * scale
    assert np.abs(r2 - r2_b).max() < 1e-12 * scale
    assert abs(e - e_b) < 1e-13


def test_complex_ccsd_equals_fci_for_two_electrons():
    o, v = 2, 5
    s, B = _csystem(o, v, 74)
    V = oracle.antisym_integrals(o, v, B)
    res = oracle.ccsd_solve(o, v, s.eps, V, tol=1e-12, maxiter=200)
    assert res["status"] == 0
    assert abs(res["energy"] - detspace.fci_correlation(o, v, s.eps, V)) < 1e-12


def test_complex_path_with_real_B_equals_real_path():
    o, v = 3, 4
    s, B = _system(o, v, 75)
    t1, t2 = ccinputs.random_amplitudes(o, v, seed=75, scale1=0.1, scale2=0.1)
    Vr = oracle.antisym_integrals(o, v, B)
    Vc = oracle.antisym_integrals(o, v, B.astype(np.complex128))
    r1, r2 = oracle.ccsd_residual(o, v, s.eps, Vr, t1, t2)
    z1, z2 = oracle.ccsd_residual(o, v, s.eps, Vc, t1.astype(complex), t2.astype(complex))
    assert np.abs(z2.imag).max() == 0.0 and np.abs(z2.real - r2).max() < 1e-15
    assert np.abs(z1.real - r1).max() < 1e-15


def test_complex_sampled_elements_match_full_residual():
    o, v = 3, 5
    s, B = _csystem(o, v, 76)
    t1, t2 = ccinputs.random_amplitudes(o, v, seed=76, scale1=0.1, scale2=0.1, complex_=True)
    idx = np.array([[0, 1, 0, 1], [2, 0, 4, 3], [1, 2, 3, 0]])
    got = oracle.ccsd_r2_sample(o, v, B, s.eps, t1, t2, idx)
    _, r2 = oracle.ccsd_residual(o, v, s.eps, oracle.antisym_integrals(o, v, B), t1, t2)
    assert np.abs(got - r2[idx[:, 0], idx[:, 1], idx[:, 2], idx[:, 3]]).max() < 1e-13


# ------------------------------------------- definition oracle (any rank <= 3)
def _all_idx(o, v, rank):
    import itertools
    return np.array([list(i) + list(a) for i in itertools.product(range(o), repeat=rank)
                     for a in itertools.product(range(v), repeat=rank)])


@pytest.mark.parametrize("cplx", [False, True])
@pytest.mark.parametrize("o,v,seed,triples", [(2, 3, 81, False), (3, 4, 82, False), (3, 4, 83, True),
                                              (3, 5, 84, True)])
def test_definition_oracle_matches_brute_force(cplx, o, v, seed, triples):
    """cc_definition.c (CI coefficients of exp(T) Phi_0, Slater-Condon, the
    exp(-T) row) against the full-matrix determinant brute force: every
    element of R1, R2 (and R3) and the energy, CCSD and CCSDT."""
    s = ccinputs.make_system(o, v, L=5, seed=seed, complex_=cplx)
    B = s.B * 6.0
    V = oracle.antisym_integrals(o, v, B)
    amps = ccinputs.random_amplitudes(o, v, seed=seed, scale1=0.1, scale2=0.1, triples=triples, complex_=cplx)
    t1, t2, t3 = amps[0], amps[1], (amps[2] if triples else None)
    ref = detspace.brute_residual(o, v, s.eps, V, t1, t2, t3)
    e = oracle.cc_definition_elements(o, v, B, s.eps, t1, t2, t3, rank=0)
    assert abs(e - ref[0]) < 1e-13
    for rank in ((1, 2, 3) if triples else (1, 2)):
        idx = _all_idx(o, v, rank)
        got = oracle.cc_definition_elements(o, v, B, s.eps, t1, t2, t3, rank=rank, idx=idx)
        want = np.array([ref[rank][tuple(r)] for r in idx])
        assert np.abs(got - want).max() < 1e-13


@pytest.mark.parametrize("cplx", [False, True])
def test_definition_oracle_agrees_with_the_ccsd_equations(cplx):
    """Two independent oracles, one from the CCSD equations and one from the
    definition, on sampled elements of a system too large for the brute force."""
    o, v = 5, 12
    s = ccinputs.make_system(o, v, L=8, seed=85, complex_=cplx)
    B = s.B * 6.0
    t1, t2 = ccinputs.random_amplitudes(o, v, seed=85, scale1=0.1, scale2=0.1, complex_=cplx)
    r1, r2 = oracle.ccsd_residual(o, v, s.eps, oracle.antisym_integrals(o, v, B), t1, t2)
    rng = np.random.default_rng(3)
    idx2 = np.stack([rng.integers(0, o, 6), rng.integers(0, o, 6), rng.integers(0, v, 6), rng.integers(0, v, 6)], 1)
    got2 = oracle.cc_definition_elements(o, v, B, s.eps, t1, t2, None, rank=2, idx=idx2)
    assert np.abs(got2 - r2[tuple(idx2.T)]).max() < 1e-12
    idx1 = np.stack([rng.integers(0, o, 4), rng.integers(0, v, 4)], 1)
    got1 = oracle.cc_definition_elements(o, v, B, s.eps, t1, t2, None, rank=1, idx=idx1)
    assert np.abs(got1 - r1[tuple(idx1.T)]).max() < 1e-12


@pytest.mark.parametrize("cplx", [False, True])
def test_prepared_sampler_equals_one_shot_sampling(cplx):
    """The prepared sampled-element oracle (shared part built once) returns what
    the one-shot routine returns, bit for bit, over several evaluations."""
    o, v = 3, 5
    s = ccinputs.make_system(o, v, L=6, seed=57, complex_=cplx)
    t1, t2 = ccinputs.random_amplitudes(o, v, seed=57, scale1=0.1, scale2=0.1, complex_=cplx)
    idx = np.array([[0, 1, 0, 1], [2, 0, 4, 3], [1, 2, 3, 0], [1, 1, 2, 3]])
    want = oracle.ccsd_r2_sample(o, v, s.B, s.eps, t1, t2, idx)
    with oracle.R2Sampler(o, v, s.B, s.eps, t1, t2) as smp:
        for _ in range(2):
            got = smp.eval(idx)
            assert np.array_equal(got, want)
        assert np.array_equal(smp.eval(idx[1:3]), want[1:3])
