"""Block-form FP64 oracle for spin-orbital CCSD (test infrastructure).

TEST INFRASTRUCTURE ONLY: only ``tests/``, ``__graft_entry__.smoke()``,
``bench.py``'s CPU legs and the cache writer beside this file may import it.
It shares no code with the CUDA path.

Why a second CCSD oracle: the explicit-loop oracle (``cc_oracle.c``) holds the
full n^4 integral tensor and walks it with cache-hostile strides, which is
right for small systems but would take days at o=40, v=200.  This module
computes the same quantities with the same equations, each term one library
contraction (``numpy.einsum`` / matrix product), on the integral blocks a
term reads, so a converged energy at o=40, v=200 (o^2 v^4 = 2.6e12
multiply-adds per iteration) takes minutes on a multi-core host.

What it computes (arxiv 2409.06759, Sec. II A, Eq. amp; Hamiltonian Eq. ham2q):
* integral blocks <pq||rs> = (pr|qs) - (ps|qr) with (pq|rs) = sum_L B_pq B_rs
  (no conjugation; complex Hermitian B gives Hermitian integrals), each block
  formed from B by that definition, one first index at a time;
* the CCSD residual R = RHS - D*t in the Stanton-Gauss intermediate form of
  the spin-orbital CCSD equations, term by term in the order printed below;
  the diagonal Fock matrix makes f_me = 0 and f_ae, f_mi off-diagonal = 0, so
  those terms of F_ae, F_mi, F_me vanish and are not written;
* the energy E - E_ref = 1/4 sum <ij||ab> t_ij^ab + 1/2 sum <ij||ab> t_i^a t_j^b;
* Jacobi + DIIS with the reading used throughout: error e_k = R_k/D, at most
  diis_max stored pairs, extrapolation from two on, coefficients from
  ``oracle.diis_coeffs`` (the explicit-loop oracle's own Gaussian
  elimination), the oldest pair dropped while the solve is singular, stop when
  the Frobenius norm of (R1, R2) is below tol.

Integral identities used (exact for the definition above, bit for bit, since
each (pq|rs) is the same sum of the same products):
<qp||rs> = -<pq||rs>, <pq||sr> = -<pq||rs>.

Pins (tests/test_oracle_blocks.py): every residual element and the energy
against the determinant-space brute force (real and complex), CCSD = FCI for
two electrons, MP2 and MP3 from the lambda expansion of the energy, and
agreement with the explicit-loop oracle on systems of several hundred
elements per block.
"""
from __future__ import annotations

import numpy as np

__all__ = ["integral_blocks", "ccsd_residual", "ccsd_energy", "ccsd_solve", "BLOCKS"]

# The blocks the CCSD equations below read, named by their index spaces.
BLOCKS = ("oooo", "ooov", "oovv", "ovov", "ovvv", "vvvv", "vvoo", "vvvo", "ovoo")


def _antisym_block(B: np.ndarray, o: int, spaces: str) -> np.ndarray:
    """<pq||rs> for p, q, r, s in the spaces named by ``spaces`` (e.g. 'ovvv'),
    dense [p][q][r][s]: sum_L B_pr B_qs - B_ps B_qr, one p at a time."""
    n = B.shape[1]
    sl = {"o": slice(0, o), "v": slice(o, n)}
    sp, sq, sr, ss = (sl[c] for c in spaces)
    Bpr, Bqs = B[:, sp, sr], B[:, sq, ss]
    Bps, Bqr = B[:, sp, ss], B[:, sq, sr]
    P, Q, R, S = Bpr.shape[1], Bqs.shape[1], Bpr.shape[2], Bqs.shape[2]
    out = np.empty((P, Q, R, S), dtype=B.dtype)
    for p in range(P):
        prqs = np.tensordot(Bpr[:, p, :], Bqs, axes=(0, 0))        # [r][q][s] = (pr|qs)
        psqr = np.tensordot(Bps[:, p, :], Bqr, axes=(0, 0))        # [s][q][r] = (ps|qr)
        out[p] = prqs.transpose(1, 0, 2) - psqr.transpose(1, 2, 0)
    return out


def integral_blocks(o: int, v: int, B: np.ndarray, names=BLOCKS) -> dict:
    """The integral blocks the CCSD equations read, built from B[L][n][n]."""
    B = np.ascontiguousarray(B)
    return {nm: _antisym_block(B, o, nm) for nm in names}


def _P(x: np.ndarray, a0: int, a1: int) -> np.ndarray:
    """Permutation operator P(pq) = 1 - (p<->q) on axes a0, a1."""
    return x - np.swapaxes(x, a0, a1)


def _ein(spec, *ops):
    return np.einsum(spec, *ops, optimize=True)


def ccsd_residual(o: int, v: int, eps: np.ndarray, blk: dict, t1: np.ndarray, t2: np.ndarray):
    """(R1, R2) of spin-orbital CCSD, R = RHS - D*t (Stanton-Gauss form)."""
    eo, ev = eps[:o], eps[o:]
    oooo, ooov, oovv = blk["oooo"], blk["ooov"], blk["oovv"]
    ovov, ovvv, vvvv = blk["ovov"], blk["ovvv"], blk["vvvv"]
    vvoo, vvvo, ovoo = blk["vvoo"], blk["vvvo"], blk["ovoo"]

    # tau = t2 + t_i^a t_j^b - t_i^b t_j^a ; tau~ = t2 + 1/2 (t_i^a t_j^b - t_i^b t_j^a)
    tt = _ein("ia,jb->ijab", t1, t1)
    tt = tt - tt.transpose(0, 1, 3, 2)
    tau = t2 + tt
    taut = t2 + 0.5 * tt
    del tt

    # F_ae = sum_mf t_m^f <ma||fe> - 1/2 sum_mnf tau~_mn^af <mn||ef>
    Fae = _ein("mf,mafe->ae", t1, ovvv) - 0.5 * _ein("mnaf,mnef->ae", taut, oovv)
    # F_mi = sum_en t_n^e <mn||ie> + 1/2 sum_nef tau~_in^ef <mn||ef>
    Fmi = _ein("ne,mnie->mi", t1, ooov) + 0.5 * _ein("inef,mnef->mi", taut, oovv)
    # F_me = sum_nf t_n^f <mn||ef>
    Fme = _ein("nf,mnef->me", t1, oovv)

    # W_mnij = <mn||ij> + P(ij) sum_e t_j^e <mn||ie> + 1/4 sum_ef tau_ij^ef <mn||ef>
    x = _ein("je,mnie->mnij", t1, ooov)
    Wmnij = oooo + _P(x, 2, 3) + 0.25 * _ein("ijef,mnef->mnij", tau, oovv)

    # W_abef = <ab||ef> - P(ab) sum_m t_m^b <am||ef> + 1/4 sum_mn tau_mn^ab <mn||ef>
    #   stored [ab][ef]; <am||ef> = -<ma||ef>, so the P(ab) term adds
    #   Z_b[a] - Z_a[b] with Z_c[a][e][f] = sum_m t_m^c <ma||ef>.
    Wabef = (0.25 * tau.reshape(o * o, v * v)).T @ oovv.reshape(o * o, v * v)
    Wabef += vvvv.reshape(v * v, v * v)
    Wabef = Wabef.reshape(v, v, v, v)
    for c in range(v):
        Z = np.tensordot(t1[:, c], ovvv, axes=(0, 0))
        Wabef[:, c] += Z
        Wabef[c, :] -= Z
    del Z

    # W_mbej = <mb||ej> + sum_f t_j^f <mb||ef> - sum_n t_n^b <mn||ej>
    #          - sum_nf (1/2 t_jn^fb + t_j^f t_n^b) <mn||ef>
    #   <mb||ej> = -<mb||je>,  <mn||ej> = -<mn||je>
    mbej = -ovov.transpose(0, 1, 3, 2)
    Y = 0.5 * t2 + _ein("jf,nb->jnfb", t1, t1)
    Wmbej = (mbej + _ein("jf,mbef->mbej", t1, ovvv) + _ein("nb,mnje->mbej", t1, ooov)
             - _ein("jnfb,mnef->mbej", Y, oovv))
    del Y

    # ---- T1 equation
    #   sum_e t_i^e F_ae - sum_m t_m^a F_mi + sum_me t_im^ae F_me - sum_nf t_n^f <na||if>
    #   - 1/2 sum_mef t_im^ef <ma||ef> - 1/2 sum_men t_mn^ae <nm||ei>,  <nm||ei> = -<nm||ie>
    r1 = (_ein("ie,ae->ia", t1, Fae) - _ein("ma,mi->ia", t1, Fmi) + _ein("imae,me->ia", t2, Fme)
          - _ein("nf,naif->ia", t1, ovov) - 0.5 * _ein("imef,maef->ia", t2, ovvv)
          + 0.5 * _ein("mnae,nmie->ia", t2, ooov))
    r1 -= (eo[:, None] - ev[None, :]) * t1

    # ---- T2 equation; the doubles projection of H|Phi_0> is <ab||ij>
    D2 = eo[:, None, None, None] + eo[None, :, None, None] - ev[None, None, :, None] - ev[None, None, None, :]
    r2 = vvoo.transpose(2, 3, 0, 1) - D2 * t2
    # + P(ab) sum_e t_ij^ae (F_be - 1/2 sum_m t_m^b F_me)
    Fbe2 = Fae - 0.5 * _ein("mb,me->be", t1, Fme)
    r2 += _P(_ein("ijae,be->ijab", t2, Fbe2), 2, 3)
    # - P(ij) sum_m t_im^ab (F_mj + 1/2 sum_e t_j^e F_me)
    Fmj2 = Fmi + 0.5 * _ein("je,me->mj", t1, Fme)
    r2 -= _P(_ein("imab,mj->ijab", t2, Fmj2), 0, 1)
    # + 1/2 sum_mn tau_mn^ab W_mnij
    r2 += 0.5 * _ein("mnab,mnij->ijab", tau, Wmnij)
    # + 1/2 sum_ef tau_ij^ef W_abef
    r2 += 0.5 * (tau.reshape(o * o, v * v) @ Wabef.reshape(v * v, v * v).T).reshape(o, o, v, v)
    del Wabef
    # + P(ij) P(ab) sum_me (t_im^ae W_mbej - t_i^e t_m^a <mb||ej>)
    X = _ein("imae,mbej->ijab", t2, Wmbej) - _ein("ie,ma,mbej->ijab", t1, t1, mbej)
    r2 += _P(_P(X, 0, 1), 2, 3)
    del X
    # + P(ij) sum_e t_i^e <ab||ej>
    r2 += _P(_ein("ie,abej->ijab", t1, vvvo), 0, 1)
    # - P(ab) sum_m t_m^a <mb||ij>
    r2 -= _P(_ein("ma,mbij->ijab", t1, ovoo), 2, 3)
    return r1, r2


def ccsd_energy(o: int, v: int, blk: dict, t1: np.ndarray, t2: np.ndarray):
    """E_CC - E_ref = 1/4 sum <ij||ab> t_ij^ab + 1/2 sum <ij||ab> t_i^a t_j^b (f_ia = 0)."""
    oovv = blk["oovv"]
    return 0.25 * _ein("ijab,ijab->", oovv, t2) + 0.5 * _ein("ijab,ia,jb->", oovv, t1, t1)


def ccsd_solve(o, v, eps, blk, t1=None, t2=None, tol=1e-8, maxiter=100, diis_max=8, log=None):
    """Jacobi + DIIS from (t1, t2) (zeros by default); the reading of
    ``cc_oracle.c``'s solve, with the block residual.  Returns a dict with
    status (0 converged, 2 maxiter, 3 non-finite or exploding norm), iters,
    energies, rnorms, t1, t2, energy."""
    from . import diis_coeffs

    cplx = any(np.iscomplexobj(b) for b in blk.values())
    dt = np.complex128 if cplx else np.float64
    eps = np.asarray(eps, dtype=np.float64)
    eo, ev = eps[:o], eps[o:]
    t1 = np.zeros((o, v), dt) if t1 is None else np.array(t1, dtype=dt)
    t2 = np.zeros((o, o, v, v), dt) if t2 is None else np.array(t2, dtype=dt)
    n1 = o * v
    D1 = eo[:, None] - ev[None, :]
    D2 = eo[:, None, None, None] + eo[None, :, None, None] - ev[None, None, :, None] - ev[None, None, None, :]
    D = np.concatenate([D1.ravel(), D2.ravel()])
    hx, he = [], []
    energies, rnorms = [], []
    best = np.inf
    status = 2
    for k in range(maxiter):
        r1, r2 = ccsd_residual(o, v, eps, blk, t1, t2)
        e = ccsd_energy(o, v, blk, t1, t2)
        rn = float(np.sqrt(np.sum(np.abs(r1) ** 2) + np.sum(np.abs(r2) ** 2)))
        energies.append(e)
        rnorms.append(rn)
        if log is not None:
            log(k, e, rn)
        if not np.isfinite(rn) or rn > 1e3 * best:
            status = 3
            break
        best = min(best, rn)
        if rn < tol:
            status = 0
            break
        if diis_max > 0 and len(hx) == diis_max:
            hx.pop(0)
            he.pop(0)
        ek = np.concatenate([r1.ravel(), r2.ravel()]) / D
        del r1, r2
        xk = np.concatenate([t1.ravel(), t2.ravel()]) + ek
        if diis_max > 0:
            hx.append(xk)
            he.append(ek)
        if len(hx) >= 2:
            while True:
                m = len(he)
                Bm = np.empty((m, m))
                for a in range(m):
                    for b in range(m):
                        Bm[a, b] = np.vdot(he[a], he[b]).real
                c = diis_coeffs(Bm)
                if c is not None or m <= 2:
                    break
                hx.pop(0)
                he.pop(0)
            if c is not None:
                x = np.zeros_like(hx[0])
                for a in range(len(hx)):
                    x += c[a] * hx[a]
            else:
                x = hx[-1].copy()
        else:
            x = xk
        t1 = x[:n1].reshape(o, v).copy()
        t2 = x[n1:].reshape(o, o, v, v).copy()
        del x
    return dict(status=status, iters=len(energies), energies=np.array(energies), rnorms=np.array(rnorms),
                t1=t1, t2=t2, energy=energies[-1] if energies else float("nan"))
