"""Pins of the block-form CCSD oracle (oracle/cc_blocks.py), none of them the
oracle itself:

* every residual element and the energy against the determinant-space brute
  force of <Phi_l| exp(-T) H_N exp(T) |Phi_0> (Eq. amp), real and complex;
* the converged energy equals FCI for two electrons;
* the first Jacobi step gives MP2 (determinant-space second order);
* the lambda^3 coefficient of E(lambda V) is the MP3 closed form;
* the integral blocks against the numpy einsum reading of Eq. ham2q;
* agreement with the explicit-loop oracle (residual, solve trajectory) on a
  system with several hundred elements per block;
* the cached converged energies (baseline/oracle_cache.json) belong to the
  current input generator, and the small entry is what the oracle computes.
"""
import json
import os

import numpy as np
import pytest

import ccinputs
import detspace
import oracle
from oracle import cc_blocks

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.parametrize("cplx", [False, True])
@pytest.mark.parametrize("o,v,seed", [(2, 3, 101), (3, 4, 102), (3, 5, 103), (4, 4, 104), (2, 6, 105)])
def test_block_residual_matches_brute_force(cplx, o, v, seed):
    s = ccinputs.make_system(o, v, L=6, seed=seed, complex_=cplx)
    B = s.B * 6.0
    t1, t2 = ccinputs.random_amplitudes(o, v, seed=seed, scale1=0.1, scale2=0.1, complex_=cplx)
    blk = cc_blocks.integral_blocks(o, v, B)
    r1, r2 = cc_blocks.ccsd_residual(o, v, s.eps, blk, t1, t2)
    e = cc_blocks.ccsd_energy(o, v, blk, t1, t2)
    e_b, r1_b, r2_b = detspace.brute_residual(o, v, s.eps, detspace.antisym_from_B(B), t1, t2)
    scale = max(np.abs(r2_b).max(), np.abs(r1_b).max())
    assert np.abs(r1 - r1_b).max() < 1e-12 * scale
    assert np.abs(r2 - r2_b).max() < 1e-12 * scale
    assert abs(e - e_b) < 1e-13


@pytest.mark.parametrize("cplx", [False, True])
def test_integral_blocks_match_einsum_reading(cplx):
    o, v = 3, 7
    s = ccinputs.make_system(o, v, L=5, seed=106, complex_=cplx)
    V = detspace.antisym_from_B(s.B)
    blk = cc_blocks.integral_blocks(o, v, s.B)
    sl = {"o": slice(0, o), "v": slice(o, o + v)}
    for nm, x in blk.items():
        ref = V[sl[nm[0]], sl[nm[1]], sl[nm[2]], sl[nm[3]]]
        assert x.shape == ref.shape and np.abs(x - ref).max() < 1e-16


@pytest.mark.parametrize("cplx", [False, True])
def test_block_ccsd_equals_fci_for_two_electrons(cplx):
    o, v = 2, 6
    s = ccinputs.make_system(o, v, L=6, seed=107, complex_=cplx)
    B = s.B * 6.0
    res = cc_blocks.ccsd_solve(o, v, s.eps, cc_blocks.integral_blocks(o, v, B), tol=1e-12, maxiter=200)
    assert res["status"] == 0
    assert abs(res["energy"] - detspace.fci_correlation(o, v, s.eps, detspace.antisym_from_B(B))) < 1e-12


def test_block_first_iteration_is_mp2():
    o, v = 3, 5
    s = ccinputs.make_system(o, v, L=6, seed=108)
    B = s.B * 6.0
    res = cc_blocks.ccsd_solve(o, v, s.eps, cc_blocks.integral_blocks(o, v, B), tol=0.0, maxiter=2)
    assert res["energies"][0] == 0.0
    assert abs(res["energies"][1] - detspace.mp2_det_space(o, v, s.eps, detspace.antisym_from_B(B))) < 1e-14


def test_block_energy_lambda_expansion_is_mp3():
    o, v = 5, 16
    s = ccinputs.make_system(o, v, L=12, seed=109)
    B = s.B * 6.0
    blk = cc_blocks.integral_blocks(o, v, B)
    lam = np.array([0.01, 0.02, 0.03, 0.04, 0.05])
    es = []
    for x in lam:
        scaled = {k: b * x for k, b in blk.items()}
        es.append(cc_blocks.ccsd_solve(o, v, s.eps, scaled, tol=1e-15, maxiter=200)["energy"])
    A = np.stack([lam ** k for k in range(2, 7)], 1)
    c = np.linalg.solve(A, np.array(es))
    e3 = detspace.mp3_closed_form(o, v, s.eps, oracle.antisym_integrals(o, v, B))
    assert abs(c[1] - e3) < 1e-7 * abs(e3)


@pytest.mark.parametrize("cplx", [False, True])
def test_block_oracle_agrees_with_explicit_loop_oracle(cplx):
    o, v = 6, 20
    s = ccinputs.make_system(o, v, L=24, seed=110, complex_=cplx)
    t1, t2 = ccinputs.random_amplitudes(o, v, seed=110, scale1=0.05, scale2=0.05, complex_=cplx)
    V = oracle.antisym_integrals(o, v, s.B)
    blk = cc_blocks.integral_blocks(o, v, s.B)
    r1, r2 = cc_blocks.ccsd_residual(o, v, s.eps, blk, t1, t2)
    q1, q2 = oracle.ccsd_residual(o, v, s.eps, V, t1, t2)
    assert np.abs(r1 - q1).max() < 1e-14 and np.abs(r2 - q2).max() < 1e-14
    a = cc_blocks.ccsd_solve(o, v, s.eps, blk, tol=1e-10, maxiter=50)
    b = oracle.ccsd_solve(o, v, s.eps, V, tol=1e-10, maxiter=50)
    assert a["iters"] == b["iters"] and a["status"] == b["status"] == 0
    assert np.abs(np.asarray(a["energies"]) - np.asarray(b["energies"])).max() < 1e-14


def _cache():
    p = os.path.join(ROOT, "baseline", "oracle_cache.json")
    if not os.path.exists(p):
        pytest.skip("no oracle cache")
    with open(p) as f:
        return json.load(f)


def test_cached_energies_belong_to_the_current_inputs():
    """Every cached entry's input fingerprint matches what the generator draws
    today, and each solve converged below the stored tolerance."""
    from oracle.cache_energies import fingerprint

    cache = _cache()
    for key, e in cache.items():
        entries = e["systems"] if "systems" in e else [e]
        for x in entries[:4]:
            s = ccinputs.make_system(x["o"], x["v"], L=x["L"], seed=x["seed"], complex_=x["dtype"] == "c128")
            assert fingerprint(s) == x["inputs_sha256_16"], key
            assert x["status"] == 0 and x["rnorms"][-1] < 1e-10, key


def test_cached_small_energy_is_the_oracles():
    cache = _cache()
    e = cache["ccsd_o10_v40_L120_seed0_f64"]
    s = ccinputs.make_system(10, 40, L=120, seed=0)
    res = oracle.ccsd_solve(10, 40, s.eps, oracle.antisym_integrals(10, 40, s.B), tol=e["tol"], maxiter=100)
    assert res["iters"] == e["iterations"]
    assert np.abs(np.asarray(res["energies"]) - np.asarray(e["energies"])).max() == 0.0
