"""Determinant-space brute force for coupled cluster (pins the oracle).

An independent route to the quantities of Sec. II A (Eq. amp): second
quantisation on explicit Slater determinants (bit strings), with no CC
equations at all.

* ``H = sum_pq h_pq a+_p a_q + 1/4 sum_pqrs <pq||rs> a+_p a+_q a_s a_r``
  (Eq. ham2q) is built as a matrix in the N-electron determinant space, with
  ``h_pq = f_pq - sum_i <pi||qi>`` so that its Fock operator is exactly the
  diagonal ``f = diag(eps)`` used by the CC code, and ``H_N = H - E_ref``.
* ``T = T1 + T2 (+ T3)`` with the 1, 1/4, 1/36 prefactors of the cluster
  operators is built as a matrix in the same space; ``exp(+-T)`` is a
  terminating Taylor series (T only excites).
* residual elements are ``<Phi_l| exp(-T) H_N exp(T) |Phi_0>`` with
  ``Phi_ij^ab = a+_a a+_b a_j a_i Phi_0`` (the sign rule "the line from i ends
  in a", Sec. II C);  the energy is the ``Phi_0`` projection.
* FCI: the eigenvector of H with the largest weight on ``Phi_0``.
* MP2: Rayleigh-Schroedinger second order with the Moller-Plesset partition,
  ``sum_D |<D|H|Phi_0>|^2 / (E0_0 - E0_D)`` over all determinants D.
"""
from __future__ import annotations

from itertools import combinations

import numpy as np


def _popc(x: int) -> int:
    return bin(x).count("1")


def _ann(det: int, p: int):
    if not (det >> p) & 1:
        return None, 0
    return det & ~(1 << p), (-1 if _popc(det & ((1 << p) - 1)) & 1 else 1)


def _cre(det: int, p: int):
    if (det >> p) & 1:
        return None, 0
    return det | (1 << p), (-1 if _popc(det & ((1 << p) - 1)) & 1 else 1)


def apply_ops(det: int, ops):
    """Apply an operator string; ``ops`` is written left to right as in the
    formula (('c', p) = creator, ('a', p) = annihilator); the rightmost acts first."""
    sign = 1
    for kind, p in reversed(ops):
        det, s = (_cre if kind == "c" else _ann)(det, p)
        if det is None:
            return None, 0
        sign *= s
    return det, sign


class DetSpace:
    def __init__(self, o: int, v: int):
        self.o, self.v, self.n = o, v, o + v
        self.dets = [sum(1 << p for p in c) for c in combinations(range(self.n), o)]
        self.index = {d: k for k, d in enumerate(self.dets)}
        self.dim = len(self.dets)
        self.ref = (1 << o) - 1

    # ---------------------------------------------------------------- builders
    def hamiltonian(self, h: np.ndarray, V: np.ndarray) -> np.ndarray:
        n, dim = self.n, self.dim
        H = np.zeros((dim, dim), dtype=np.result_type(h, V))
        for col, d in enumerate(self.dets):
            occ = [p for p in range(n) if (d >> p) & 1]
            for q in occ:
                for p in range(n):
                    d2, s = apply_ops(d, [("c", p), ("a", q)])
                    if d2 is not None:
                        H[self.index[d2], col] += s * h[p, q]
            for r in occ:
                for s_ in occ:
                    if r == s_:
                        continue
                    for p in range(n):
                        for q in range(n):
                            if p == q:
                                continue
                            d2, sg = apply_ops(d, [("c", p), ("c", q), ("a", s_), ("a", r)])
                            if d2 is not None:
                                H[self.index[d2], col] += 0.25 * sg * V[p, q, r, s_]
        return H

    def cluster(self, t1=None, t2=None, t3=None) -> np.ndarray:
        o, v, dim = self.o, self.v, self.dim
        dt = np.result_type(*(x for x in (t1, t2, t3) if x is not None))
        T = np.zeros((dim, dim), dtype=dt)
        for col, d in enumerate(self.dets):
            occ = [i for i in range(o) if (d >> i) & 1]
            vir = [a for a in range(v) if not (d >> (o + a)) & 1]
            if t1 is not None:
                for i in occ:
                    for a in vir:
                        d2, s = apply_ops(d, [("c", o + a), ("a", i)])
                        T[self.index[d2], col] += s * t1[i, a]
            if t2 is not None:
                for i in occ:
                    for j in occ:
                        if i == j:
                            continue
                        for a in vir:
                            for b in vir:
                                if a == b:
                                    continue
                                d2, s = apply_ops(d, [("c", o + a), ("c", o + b), ("a", j), ("a", i)])
                                T[self.index[d2], col] += 0.25 * s * t2[i, j, a, b]
            if t3 is not None:
                for i, j, k in ((i, j, k) for i in occ for j in occ for k in occ if len({i, j, k}) == 3):
                    for a, b, c in ((a, b, c) for a in vir for b in vir for c in vir if len({a, b, c}) == 3):
                        d2, s = apply_ops(d, [("c", o + a), ("c", o + b), ("c", o + c),
                                              ("a", k), ("a", j), ("a", i)])
                        T[self.index[d2], col] += s * t3[i, j, k, a, b, c] / 36.0
        return T

    # ------------------------------------------------------------- projections
    def _vec_ref(self, dtype=float) -> np.ndarray:
        x = np.zeros(self.dim, dtype=dtype)
        x[self.index[self.ref]] = 1.0
        return x

    @staticmethod
    def _expm_apply(T: np.ndarray, x: np.ndarray, sign: float = 1.0) -> np.ndarray:
        acc = x.copy()
        term = x.copy()
        for k in range(1, 64):
            term = sign * (T @ term) / k
            if not np.any(term):
                break
            acc = acc + term
        return acc

    def similarity_ref(self, HN: np.ndarray, T: np.ndarray) -> np.ndarray:
        """exp(-T) H_N exp(T) |Phi_0> as a vector."""
        x = self._vec_ref(np.result_type(HN, T))
        return self._expm_apply(T, HN @ self._expm_apply(T, x, +1.0), -1.0)

    def project(self, y: np.ndarray, creators, annihilators):
        """<Phi| y>, Phi = a+_{c1} a+_{c2} .. a_{an} .. a_{a1} Phi_0 with the
        creators listed left to right and the annihilators in the order
        (i, j, k) meaning a_k a_j a_i."""
        ops = [("c", p) for p in creators] + [("a", p) for p in reversed(annihilators)]
        d, s = apply_ops(self.ref, ops)
        if d is None:
            return 0.0
        return s * y[self.index[d]]


def one_body_from_fock(eps: np.ndarray, V: np.ndarray, o: int):
    """h_pq = f_pq - sum_i <pi||qi> and E_ref = sum_i f_ii - 1/2 sum_ij <ij||ij>."""
    n = eps.size
    h = np.diag(eps).astype(V.dtype) - np.einsum("piqi->pq", V[:, :o, :, :o])
    e_ref = eps[:o].sum() - 0.5 * np.einsum("ijij->", V[:o, :o, :o, :o])
    return h, e_ref


def antisym_from_B(B: np.ndarray) -> np.ndarray:
    """<pq||rs> = (pr|qs) - (ps|qr), (pq|rs) = sum_L B_pq B_rs (numpy route)."""
    chem = np.einsum("lpq,lrs->pqrs", B, B)
    return np.einsum("prqs->pqrs", chem) - np.einsum("psqr->pqrs", chem)


def brute_residual(o, v, eps, V, t1, t2, t3=None):
    """(E_CC - E_ref, R1, R2[, R3]) by explicit second quantisation."""
    ds = DetSpace(o, v)
    h, e_ref = one_body_from_fock(eps, V, o)
    H = ds.hamiltonian(h, V)
    HN = H - e_ref * np.eye(ds.dim)
    T = ds.cluster(t1, t2, t3)
    y = ds.similarity_ref(HN, T)
    e = ds.project(y, [], [])
    r1 = np.zeros((o, v), dtype=y.dtype)
    for i in range(o):
        for a in range(v):
            r1[i, a] = ds.project(y, [o + a], [i])
    r2 = np.zeros((o, o, v, v), dtype=y.dtype)
    for i in range(o):
        for j in range(o):
            for a in range(v):
                for b in range(v):
                    if i != j and a != b:
                        r2[i, j, a, b] = ds.project(y, [o + a, o + b], [i, j])
    if t3 is None:
        return e, r1, r2
    r3 = np.zeros((o, o, o, v, v, v), dtype=y.dtype)
    for i, j, k in ((i, j, k) for i in range(o) for j in range(o) for k in range(o) if len({i, j, k}) == 3):
        for a, b, c in ((a, b, c) for a in range(v) for b in range(v) for c in range(v) if len({a, b, c}) == 3):
            r3[i, j, k, a, b, c] = ds.project(y, [o + a, o + b, o + c], [i, j, k])
    return e, r1, r2, r3


def fci_correlation(o, v, eps, V):
    """E_FCI - E_ref for the root with the largest |c_0|."""
    ds = DetSpace(o, v)
    h, e_ref = one_body_from_fock(eps, V, o)
    H = ds.hamiltonian(h, V)
    w, U = np.linalg.eigh(H)
    k = int(np.argmax(np.abs(U[ds.index[ds.ref], :])))
    return w[k] - e_ref


def mp2_det_space(o, v, eps, V):
    """Second-order Moller-Plesset energy from determinant-space H elements."""
    ds = DetSpace(o, v)
    h, e_ref = one_body_from_fock(eps, V, o)
    H = ds.hamiltonian(h, V)
    c0 = ds.index[ds.ref]
    e0 = eps[:o].sum()
    tot = 0.0
    for k, d in enumerate(ds.dets):
        if k == c0:
            continue
        ed = sum(eps[p] for p in range(ds.n) if (d >> p) & 1)
        tot += abs(H[k, c0]) ** 2 / (e0 - ed)
    return tot


def mp3_det_space(o, v, eps, V):
    """Third-order Moller-Plesset energy from determinant-space H elements:
    Rayleigh-Schroedinger E3 = <Psi1| (W - E1) |Psi1> with H0 = sum_p eps_p a+_p a_p,
    W = H - H0, E1 = <Phi_0|W|Phi_0> and Psi1 = sum_K |K> <K|W|Phi_0> / (E0_0 - E0_K)."""
    ds = DetSpace(o, v)
    h, _ = one_body_from_fock(eps, V, o)
    H = ds.hamiltonian(h, V)
    e0 = np.array([sum(eps[p] for p in range(ds.n) if (d >> p) & 1) for d in ds.dets])
    W = H - np.diag(e0)
    c0 = ds.index[ds.ref]
    denom = e0[c0] - e0
    denom[c0] = 1.0
    psi1 = W[:, c0] / denom
    psi1[c0] = 0.0
    e1 = W[c0, c0]
    return np.vdot(psi1, (W - e1 * np.eye(ds.dim)) @ psi1)


def mp3_closed_form(o, v, eps, V):
    """Spin-orbital MP3 energy with unrestricted sums and D_ij^ab = e_i + e_j - e_a - e_b:
    1/8 sum <ij||ab><ab||cd><cd||ij>/(D_ij^ab D_ij^cd)   (particle ladder)
    + 1/8 sum <ij||ab><kl||ij><ab||kl>/(D_ij^ab D_kl^ab) (hole ladder)
    + sum <ij||ab><kb||cj><ac||ik>/(D_ij^ab D_ik^ac)     (ring)."""
    eo, ev = eps[:o], eps[o:]
    D = eo[:, None, None, None] + eo[None, :, None, None] - ev[None, None, :, None] - ev[None, None, None, :]
    oovv, vvvv, oooo = V[:o, :o, o:, o:], V[o:, o:, o:, o:], V[:o, :o, :o, :o]
    ovvo, vvoo = V[:o, o:, o:, :o], V[o:, o:, :o, :o]
    w = oovv / D
    t = vvoo.transpose(2, 3, 0, 1) / D
    return (0.125 * np.einsum("ijab,abcd,ijcd->", w, vvvv, t) + 0.125 * np.einsum("ijab,klij,klab->", w, oooo, t)
            + np.einsum("ijab,kbcj,ikac->", w, ovvo, t))
