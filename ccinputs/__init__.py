"""Seeded synthetic inputs for the coupled-cluster residual.

This module only draws random numbers and lays them out; it holds none of the
method's arithmetic (no integral contraction, no antisymmetrised Hamiltonian,
no CC terms).  Both the FP64 oracle and the GPU path take their inputs from
here, and each side then builds what it needs from them on its own.

Recipe (the paper's molecular inputs are replaced by seeded synthetic data of
the same structure; the active-space sizes track the paper's H2O/LiH/CO/UF6
runs, Sec. "Geometry, basis, etc." and Tables h2o/lih):

* ``rng = numpy.random.default_rng(seed)``; draw order is fixed:
  1. occupied orbital energies ``eps_occ ~ U[-2, -0.5]`` (o values), sorted;
  2. virtual orbital energies ``eps_vir ~ U[0.5, 3]`` (v values), sorted;
  3. the factor tensor ``B[L][p][q]`` (n = o + v spin orbitals): for each L the
     upper triangle p <= q in row-major order is drawn, then mirrored.
     Real: entries N(0,1) * 0.05 / sqrt(L).
     Complex (mimics relativistic spinors): B[q][p] = conj(B[p][q]); each
     off-diagonal entry draws (re, im) as N(0,1) * 0.05 / sqrt(2L) each; the
     diagonal draws (re, im) and keeps re * 0.05 / sqrt(L).
  The chemist integrals are then (pq|rs) = sum_L B[L][p][q] B[L][r][s]; the
  consumer forms them itself.
* Batched systems use sub-seed ``seed * 1000 + s``.
* Random amplitudes for residual tests (not converged, all terms active) are
  drawn from their own generator ``default_rng(seed + 7919)`` and made
  antisymmetric in the occupied and in the virtual indices, the storage
  convention of the cluster operators (Sec. II A, Eq. for T1..T4: full,
  unrestricted sums).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

__all__ = ["CCSystem", "make_system", "random_amplitudes", "batched_sizes",
           "CONFIG_SMALL", "CONFIG_LADDER", "CONFIG_CCSDT"]

# Named workloads (spin-orbital CCSD unless stated).
CONFIG_SMALL = dict(o=10, v=40, L=120, seed=0)      # small CCSD, oracle-size
CONFIG_LADDER = dict(o=40, v=200, L=120, seed=0)    # o=40, v=200 CCSD ladder workload
CONFIG_CCSDT = dict(o=8, v=64, L=96, seed=0)        # CCSDT workload


@dataclass
class CCSystem:
    o: int
    v: int
    L: int
    seed: int
    eps_occ: np.ndarray   # [o] float64
    eps_vir: np.ndarray   # [v] float64
    B: np.ndarray         # [L][n][n] float64 or complex128

    @property
    def n(self) -> int:
        return self.o + self.v

    @property
    def eps(self) -> np.ndarray:
        return np.concatenate([self.eps_occ, self.eps_vir])


def make_system(o: int, v: int, L: int = 120, seed: int = 0, complex_: bool = False) -> CCSystem:
    rng = np.random.default_rng(seed)
    eps_occ = np.sort(rng.uniform(-2.0, -0.5, o))
    eps_vir = np.sort(rng.uniform(0.5, 3.0, v))
    n = o + v
    iu, ju = np.triu_indices(n)          # row-major order of the upper triangle
    ntri = iu.size
    if not complex_:
        z = rng.standard_normal((L, ntri)) * (0.05 / math.sqrt(L))
        B = np.zeros((L, n, n))
        B[:, iu, ju] = z
        B[:, ju, iu] = z
    else:
        z = rng.standard_normal((L, ntri, 2))
        off = (z[..., 0] + 1j * z[..., 1]) * (0.05 / math.sqrt(2 * L))
        diag = z[..., 0] * (0.05 / math.sqrt(L))
        val = np.where(iu == ju, diag, off)
        B = np.zeros((L, n, n), dtype=np.complex128)
        B[:, iu, ju] = val
        B[:, ju, iu] = np.conj(val)
        B[:, np.arange(n), np.arange(n)] = diag[:, iu == ju]
    return CCSystem(o, v, L, seed, eps_occ, eps_vir, np.ascontiguousarray(B))


def _antisym_pair(x: np.ndarray, ax0: int, ax1: int) -> np.ndarray:
    return x - np.swapaxes(x, ax0, ax1)


def random_amplitudes(o: int, v: int, seed: int = 0, scale1: float = 0.02, scale2: float = 0.02,
                      triples: bool = False, complex_: bool = False):
    """Random antisymmetric amplitudes t1[i][a], t2[i][j][a][b] (and t3[i][j][k][a][b][c])."""
    rng = np.random.default_rng(seed + 7919)

    def draw(shape, s):
        if complex_:
            return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) * (s / math.sqrt(2))
        return rng.standard_normal(shape) * s

    t1 = draw((o, v), scale1)
    x = draw((o, o, v, v), scale2)
    t2 = _antisym_pair(_antisym_pair(x, 0, 1), 2, 3) * 0.25
    out = [np.ascontiguousarray(t1), np.ascontiguousarray(t2)]
    if triples:
        x = draw((o, o, o, v, v, v), scale2)
        acc = np.zeros_like(x)
        import itertools
        for po in itertools.permutations(range(3)):
            so = _perm_sign(po)
            for pv in itertools.permutations(range(3)):
                sv = _perm_sign(pv)
                acc += so * sv * np.transpose(x, list(po) + [3 + p for p in pv])
        out.append(np.ascontiguousarray(acc / 36.0))
    return tuple(out)


def _perm_sign(p) -> int:
    s, p = 1, list(p)
    for i in range(len(p)):
        while p[i] != i:
            j = p[i]
            p[i], p[j] = p[j], p[i]
            s = -s
    return s


def batched_sizes(count: int = 64, seed: int = 0):
    """(o, v, sub_seed) for the batched workload: o ~ U[4,16], v ~ U[20,80]."""
    rng = np.random.default_rng(seed)
    o = rng.integers(4, 17, count)
    v = rng.integers(20, 81, count)
    return [(int(a), int(b), seed * 1000 + s) for s, (a, b) in enumerate(zip(o, v))]
