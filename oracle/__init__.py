"""FP64 CPU oracle for the spin-orbital CC residual (test infrastructure).

Only ``tests/``, ``__graft_entry__.smoke()``, ``bench.py``'s CPU legs and the
cache writer ``oracle/cache_energies.py`` may import this package.  It wraps ``cc_oracle.c`` (the CCSD equations, plain
C, explicit loops, OpenMP over outer loops) and ``cc_definition.c`` (residual
elements of any rank up to triples straight from <Phi_l| exp(-T) H_N exp(T)
|Phi_0>, no CC equations) through ctypes, both compiled for double and complex
double, and shares no code with the CUDA path or the list derivation.

Parity pins (all in ``tests/test_oracle_pins.py``):
* residual elements vs a determinant-space brute force of
  <Phi_l| exp(-T) H_N exp(T) |Phi_0> (Eq. amp), random T, tiny o/v;
* converged CCSD energy vs FCI for two electrons;
* first-iteration energy vs the MP2 closed form computed in determinant space;
* antisymmetry of the residual; lambda-scaling of the energy: the lambda^2
  coefficient is MP2 and the lambda^3 coefficient the MP3 closed form (itself
  checked against determinant-space third-order perturbation theory).

``ccsd_r2_sample`` (and ``R2Sampler``, which builds the shared part once)
evaluates selected residual elements of large systems from B directly (same
equations); it is pinned against the brute force and the full residual at
small sizes.

``cc_blocks`` is the same CCSD in block form (numpy, one library contraction
per term of the equations) for sizes the explicit loops cannot reach; its
pins are in ``tests/test_oracle_blocks.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cc_oracle.c")
_SRCS = [_SRC, os.path.join(_HERE, "cc_definition.c")]
_LIB = os.path.join(_HERE, "libccoracle.so")
_lib = None


class _Complex(ctypes.Structure):
    """C99 double complex returned by value (two doubles)."""
    _fields_ = [("re", ctypes.c_double), ("im", ctypes.c_double)]


def build(force: bool = False) -> str:
    """Compile cc_oracle.c twice (real orc_*, complex orz_*) into libccoracle.so."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(os.path.getmtime(x) for x in _SRCS):
        import tempfile
        with tempfile.TemporaryDirectory() as td:
            objs = []
            for src in _SRCS:
                for tag, flags in (("real", []), ("cplx", ["-DCC_COMPLEX"])):
                    obj = os.path.join(td, os.path.basename(src) + "." + tag + ".o")
                    subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", *flags, "-c", src, "-o", obj])
                    objs.append(obj)
            subprocess.check_call(["gcc", "-shared", "-fopenmp", "-o", _LIB, *objs, "-lm"])
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        dp = ctypes.POINTER(ctypes.c_double)
        L.orc_antisym_integrals.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, dp]
        L.orc_ccsd_residual.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp, dp, dp, dp, dp]
        L.orc_ccsd_energy.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp, dp]
        L.orc_ccsd_energy.restype = ctypes.c_double
        L.orc_diis_coeffs.argtypes = [ctypes.c_int, dp, dp]
        L.orc_ccsd_solve.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp, dp, dp, ctypes.c_double,
                                     ctypes.c_int, ctypes.c_int, dp, dp, ctypes.POINTER(ctypes.c_int)]
        L.orc_num_threads.restype = ctypes.c_int
        L.orc_ccsd_r2_sample.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, dp, dp, dp, ctypes.c_int,
                                         ctypes.POINTER(ctypes.c_int), dp]
        vp = ctypes.c_void_p
        L.orz_antisym_integrals.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, vp, vp]
        L.orz_ccsd_residual.argtypes = [ctypes.c_int, ctypes.c_int, dp, vp, vp, vp, vp, vp]
        L.orz_ccsd_energy.argtypes = [ctypes.c_int, ctypes.c_int, vp, vp, vp]
        L.orz_ccsd_energy.restype = _Complex
        L.orz_ccsd_solve.argtypes = [ctypes.c_int, ctypes.c_int, dp, vp, vp, vp, ctypes.c_double,
                                     ctypes.c_int, ctypes.c_int, vp, dp, ctypes.POINTER(ctypes.c_int)]
        for nm in ("orc_cc_definition_elements", "orz_cc_definition_elements"):
            getattr(L, nm).argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, vp, dp, vp, vp, vp, ctypes.c_int,
                                       ctypes.c_int, ctypes.POINTER(ctypes.c_int), vp]
        L.orz_ccsd_r2_sample.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, vp, dp, vp, vp, ctypes.c_int,
                                         ctypes.POINTER(ctypes.c_int), vp]
        for pre in ("orc", "orz"):
            f = getattr(L, pre + "_ccsd_r2_sample_prepare")
            f.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, vp, dp, vp, vp]
            f.restype = vp
            getattr(L, pre + "_ccsd_r2_sample_eval").argtypes = [vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int), vp]
            getattr(L, pre + "_ccsd_r2_sample_free").argtypes = [vp]
        _lib = L
    return _lib


def _p(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _z(a: np.ndarray):
    assert a.dtype == np.complex128 and a.flags["C_CONTIGUOUS"]
    return ctypes.c_void_p(a.ctypes.data)


def _cplx(*arrays) -> bool:
    return any(np.iscomplexobj(a) for a in arrays if a is not None)


def num_threads() -> int:
    return lib().orc_num_threads()


def antisym_integrals(o: int, v: int, B: np.ndarray) -> np.ndarray:
    """Full <pq||rs> tensor [n][n][n][n] from B[L][n][n] (Eq. ham2q); complex B gives complex V."""
    n = o + v
    if np.iscomplexobj(B):
        B = np.ascontiguousarray(B, dtype=np.complex128)
        V = np.empty((n, n, n, n), dtype=np.complex128)
        if lib().orz_antisym_integrals(o, v, B.shape[0], _z(B), _z(V)) != 0:
            raise MemoryError("oracle integral build failed")
        return V
    B = np.ascontiguousarray(B, dtype=np.float64)
    V = np.empty((n, n, n, n))
    if lib().orc_antisym_integrals(o, v, B.shape[0], _p(B), _p(V)) != 0:
        raise MemoryError("oracle integral build failed")
    return V


def ccsd_residual(o, v, eps, V, t1, t2):
    if _cplx(V, t1, t2):
        eps = np.ascontiguousarray(eps, dtype=np.float64)
        V = np.ascontiguousarray(V, dtype=np.complex128)
        t1 = np.ascontiguousarray(t1, dtype=np.complex128)
        t2 = np.ascontiguousarray(t2, dtype=np.complex128)
        r1 = np.empty((o, v), dtype=np.complex128); r2 = np.empty((o, o, v, v), dtype=np.complex128)
        if lib().orz_ccsd_residual(o, v, _p(eps), _z(V), _z(t1), _z(t2), _z(r1), _z(r2)) != 0:
            raise MemoryError("oracle residual failed")
        return r1, r2
    eps = np.ascontiguousarray(eps, dtype=np.float64)
    t1 = np.ascontiguousarray(t1, dtype=np.float64)
    t2 = np.ascontiguousarray(t2, dtype=np.float64)
    r1 = np.empty((o, v)); r2 = np.empty((o, o, v, v))
    if lib().orc_ccsd_residual(o, v, _p(eps), _p(V), _p(t1), _p(t2), _p(r1), _p(r2)) != 0:
        raise MemoryError("oracle residual failed")
    return r1, r2


def ccsd_r2_sample(o, v, B, eps, t1, t2, idx):
    """R2[i,j,a,b] for each row (i, j, a, b) of idx, integrals formed from B on
    demand (large systems)."""
    if _cplx(B, t1, t2):
        B = np.ascontiguousarray(B, dtype=np.complex128)
        eps = np.ascontiguousarray(eps, dtype=np.float64)
        t1 = np.ascontiguousarray(t1, dtype=np.complex128)
        t2 = np.ascontiguousarray(t2, dtype=np.complex128)
        idx = np.ascontiguousarray(idx, dtype=np.int32).reshape(-1, 4)
        out = np.empty(idx.shape[0], dtype=np.complex128)
        rc = lib().orz_ccsd_r2_sample(o, v, B.shape[0], _z(B), _p(eps), _z(t1), _z(t2), idx.shape[0],
                                      idx.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _z(out))
        if rc != 0:
            raise MemoryError("oracle sampled residual failed")
        return out
    B = np.ascontiguousarray(B, dtype=np.float64)
    eps = np.ascontiguousarray(eps, dtype=np.float64)
    t1 = np.ascontiguousarray(t1, dtype=np.float64)
    t2 = np.ascontiguousarray(t2, dtype=np.float64)
    idx = np.ascontiguousarray(idx, dtype=np.int32).reshape(-1, 4)
    out = np.empty(idx.shape[0])
    rc = lib().orc_ccsd_r2_sample(o, v, B.shape[0], _p(B), _p(eps), _p(t1), _p(t2), idx.shape[0],
                                  idx.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _p(out))
    if rc != 0:
        raise MemoryError("oracle sampled residual failed")
    return out


class R2Sampler:
    """Selected R2 elements of one (B, t1, t2), the shared part (integral
    blocks oovv/ooov/ovvv, tau, tau~, one-particle intermediates) built once at
    construction; ``eval(idx)`` evaluates the rows (i, j, a, b) of idx.  The
    same arithmetic as ``ccsd_r2_sample``; use as a context manager."""

    def __init__(self, o, v, B, eps, t1, t2):
        self.cplx = _cplx(B, t1, t2)
        dt = np.complex128 if self.cplx else np.float64
        self._keep = [np.ascontiguousarray(B, dtype=dt), np.ascontiguousarray(eps, dtype=np.float64),
                      np.ascontiguousarray(t1, dtype=dt), np.ascontiguousarray(t2, dtype=dt)]
        B_, eps_, t1_, t2_ = self._keep
        pre = "orz" if self.cplx else "orc"
        vp = lambda a: ctypes.c_void_p(a.ctypes.data)
        self._eval = getattr(lib(), pre + "_ccsd_r2_sample_eval")
        self._free = getattr(lib(), pre + "_ccsd_r2_sample_free")
        self.h = getattr(lib(), pre + "_ccsd_r2_sample_prepare")(o, v, B_.shape[0], vp(B_), _p(eps_), vp(t1_),
                                                                   vp(t2_))
        if not self.h:
            raise MemoryError("oracle sampled residual: prepare failed")

    def eval(self, idx):
        idx = np.ascontiguousarray(idx, dtype=np.int32).reshape(-1, 4)
        out = np.empty(idx.shape[0], dtype=np.complex128 if self.cplx else np.float64)
        if self._eval(self.h, idx.shape[0], idx.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                      ctypes.c_void_p(out.ctypes.data)) != 0:
            raise RuntimeError("oracle sampled residual failed")
        return out

    def close(self):
        if self.h:
            self._free(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        self.close()


def ccsd_energy(o, v, V, t1, t2):
    if _cplx(V, t1, t2):
        V = np.ascontiguousarray(V, dtype=np.complex128)
        t1 = np.ascontiguousarray(t1, dtype=np.complex128)
        t2 = np.ascontiguousarray(t2, dtype=np.complex128)
        e = lib().orz_ccsd_energy(o, v, _z(V), _z(t1), _z(t2))
        return complex(e.re, e.im)
    t1 = np.ascontiguousarray(t1, dtype=np.float64)
    t2 = np.ascontiguousarray(t2, dtype=np.float64)
    return lib().orc_ccsd_energy(o, v, _p(V), _p(t1), _p(t2))


def diis_coeffs(Bmat: np.ndarray):
    Bmat = np.ascontiguousarray(Bmat, dtype=np.float64)
    m = Bmat.shape[0]
    c = np.empty(m)
    rc = lib().orc_diis_coeffs(m, _p(Bmat), _p(c))
    return (c if rc == 0 else None)


def ccsd_solve(o, v, eps, V, t1=None, t2=None, tol=1e-8, maxiter=100, diis_max=8):
    """Jacobi + DIIS from (t1, t2) (zeros by default).  Returns a dict."""
    eps = np.ascontiguousarray(eps, dtype=np.float64)
    if _cplx(V, t1, t2):
        V = np.ascontiguousarray(V, dtype=np.complex128)
        t1 = np.zeros((o, v), complex) if t1 is None else np.array(t1, dtype=np.complex128, order="C")
        t2 = np.zeros((o, o, v, v), complex) if t2 is None else np.array(t2, dtype=np.complex128, order="C")
        en = np.zeros(maxiter, dtype=np.complex128); rn = np.zeros(maxiter); it = ctypes.c_int(0)
        st = lib().orz_ccsd_solve(o, v, _p(eps), _z(V), _z(t1), _z(t2), tol, maxiter, diis_max, _z(en), _p(rn),
                                  ctypes.byref(it))
        k = it.value
        return dict(status=st, iters=k, energies=en[:k], rnorms=rn[:k], t1=t1, t2=t2,
                    energy=en[k - 1] if k else complex("nan"))
    t1 = np.zeros((o, v)) if t1 is None else np.array(t1, dtype=np.float64, order="C")
    t2 = np.zeros((o, o, v, v)) if t2 is None else np.array(t2, dtype=np.float64, order="C")
    en = np.zeros(maxiter); rn = np.zeros(maxiter); it = ctypes.c_int(0)
    st = lib().orc_ccsd_solve(o, v, _p(eps), _p(V), _p(t1), _p(t2), tol, maxiter, diis_max,
                              _p(en), _p(rn), ctypes.byref(it))
    k = it.value
    return dict(status=st, iters=k, energies=en[:k], rnorms=rn[:k], t1=t1, t2=t2,
                energy=en[k - 1] if k else float("nan"))


def cc_definition_elements(o, v, B, eps, t1, t2=None, t3=None, rank=2, idx=None):
    """Residual elements of the given rank (1..3) at the index tuples idx
    [ns][2*rank] = (i.., a..), or the energy E - E_ref (rank 0), from
    <Phi_l| exp(-T) H_N exp(T) |Phi_0> directly (cc_definition.c).  T holds the
    ranks whose amplitudes are given (t2 / t3 None: absent)."""
    cplx = _cplx(B, t1, t2, t3)
    dt = np.complex128 if cplx else np.float64
    B = np.ascontiguousarray(B, dtype=dt)
    eps = np.ascontiguousarray(eps, dtype=np.float64)
    ts = [None if t is None else np.ascontiguousarray(t, dtype=dt) for t in (t1, t2, t3)]
    if rank == 0:
        idx = np.zeros((1, 0), dtype=np.int32)
    idx = np.ascontiguousarray(idx, dtype=np.int32).reshape(-1, 2 * rank) if rank else idx
    ns = idx.shape[0]
    out = np.zeros(max(ns, 1), dtype=dt)
    vp = lambda a: None if a is None else ctypes.c_void_p(a.ctypes.data)
    fn = lib().orz_cc_definition_elements if cplx else lib().orc_cc_definition_elements
    rc = fn(o, v, B.shape[0], vp(B), _p(eps), vp(ts[0]), vp(ts[1]), vp(ts[2]), rank, ns,
            idx.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), vp(out))
    if rc != 0:
        raise MemoryError("definition oracle failed (%d)" % rc)
    return out[0] if rank == 0 else out
