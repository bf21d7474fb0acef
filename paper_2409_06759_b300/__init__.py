"""ccb300 -- the coupled-cluster amplitude residual on one NVIDIA B300 (sm_103a).

Thin ctypes binding of the C ABI in ``include/cc.h`` (same function names;
argument marshalling only -- every step of the residual, energy and
Jacobi+DIIS iteration runs in the library's CUDA kernels).  Device buffers are
passed as torch tensors (or raw integer addresses); torch is used only for
device memory and streams.

The library is built in-tree (``paper_2409_06759_b300/libccb300.so``, see
``build.py``).  Importing this package without it raises ImportError: there is
no CPU fallback.
"""
from __future__ import annotations

import ctypes
import json
import os
from dataclasses import dataclass

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libccb300.so")
LISTS = os.path.join(_HERE, "lists")

CC_F64, CC_C128 = 0, 1
CC_PREC_FP64, CC_PREC_BF16X3, CC_PREC_BF16X6, CC_PREC_SLICES = 0, 2, 3, 4
PRECISIONS = {"fp64": CC_PREC_FP64, "bf16x3": CC_PREC_BF16X3, "bf16x6": CC_PREC_BF16X6, "slices": CC_PREC_SLICES}
STATUS = ["CC_OK", "CC_ERR_INVALID_ARG", "CC_ERR_PARSE", "CC_ERR_SHAPE", "CC_ERR_UNSUPPORTED", "CC_ERR_OOM",
          "CC_ERR_CUDA", "CC_ERR_NOT_CONVERGED", "CC_ERR_TIMEOUT", "CC_ERR_WORKSPACE"]

# every function include/cc.h declares
EXPORTS = ["cc_plan_create", "cc_plan_workspace_bytes", "cc_plan_describe", "cc_plan_flops", "cc_plan_destroy",
           "cc_plan_profile_enable", "cc_plan_profile_read", "cc_plan_launch_count",
           "cc_residual", "cc_energy", "cc_solve_workspace_bytes", "cc_solve", "cc_integral_block_elems",
           "cc_build_integrals_workspace_bytes", "cc_build_integrals", "cc_energy_noalloc", "cc_packed_t2_elems",
           "cc_pack_t2", "cc_unpack_t2", "cc_status_string",
           "cc_last_error", "cc_version", "cc_solve_batched_workspace_bytes", "cc_solve_batched",
           "cc_plan_autotune", "cc_autotune_cache", "cc_plan_set_gemm_config", "cc_build_vvvv_packed_workspace_bytes",
           "cc_build_vvvv_packed",
           "cc_selftest_wait_timeout", "cc_selftest_convert"]

if not os.path.exists(LIB_PATH):
    raise ImportError(f"libccb300.so is not built ({LIB_PATH}); run paper_2409_06759_b300/build.py "
                      "or __graft_entry__.build() -- there is no CPU fallback")

_lib = ctypes.CDLL(LIB_PATH)

c_void_p, c_int, c_size_t, c_double = ctypes.c_void_p, ctypes.c_int, ctypes.c_size_t, ctypes.c_double


class cc_integrals(ctypes.Structure):
    _fields_ = [("f_occ", c_void_p), ("f_vir", c_void_p), ("oooo", c_void_p), ("ooov", c_void_p),
                ("oovv", c_void_p), ("ovov", c_void_p), ("ovvv", c_void_p), ("vvvv", c_void_p),
                ("vvvv_packed", c_void_p)]


class cc_amps(ctypes.Structure):
    _fields_ = [("t1", c_void_p), ("t2", c_void_p), ("t3", c_void_p)]


class cc_resid(ctypes.Structure):
    _fields_ = [("r1", c_void_p), ("r2", c_void_p), ("r3", c_void_p)]


class cc_plan_opts(ctypes.Structure):
    _fields_ = [("struct_size", c_int), ("verbose", c_int), ("fuse_permutes", c_int), ("packed_vvvv", c_int),
                ("no_kconcat", c_int), ("uniform_steps", c_int)]


class cc_solve_opts(ctypes.Structure):
    _fields_ = [("struct_size", c_int), ("max_iter", c_int), ("tol", c_double), ("diis_max", c_int),
                ("resume", c_int), ("refine_plan", c_void_p), ("switch_tol", c_double), ("verbose", c_int)]


class cc_solve_report(ctypes.Structure):
    _fields_ = [("iterations", c_int), ("converged", c_int), ("switched_at", c_int), ("energy", c_double),
                ("rnorm", c_double), ("energies", ctypes.POINTER(c_double)), ("rnorms", ctypes.POINTER(c_double)),
                ("energy_im", c_double), ("energies_im", ctypes.POINTER(c_double))]


_P = ctypes.POINTER
_sig = {
    "cc_plan_create": (c_int, [ctypes.c_char_p, c_int, c_int, c_int, c_int, _P(cc_plan_opts), _P(c_void_p)]),
    "cc_plan_workspace_bytes": (c_int, [c_void_p, _P(c_size_t)]),
    "cc_plan_describe": (c_int, [c_void_p, ctypes.c_char_p, c_size_t, _P(c_size_t)]),
    "cc_plan_flops": (c_int, [c_void_p, _P(c_double)]),
    "cc_plan_destroy": (c_int, [c_void_p]),
    "cc_plan_profile_enable": (c_int, [c_void_p, c_int]),
    "cc_plan_profile_read": (c_int, [c_void_p, _P(c_double), _P(c_double), c_int, _P(c_int), _P(c_int)]),
    "cc_plan_launch_count": (c_int, [c_void_p, _P(ctypes.c_longlong)]),
    "cc_residual": (c_int, [c_void_p, _P(cc_integrals), _P(cc_amps), _P(cc_resid), c_void_p, c_size_t, c_void_p]),
    "cc_energy": (c_int, [c_void_p, _P(cc_integrals), _P(cc_amps), c_void_p, c_void_p, c_size_t, c_void_p]),
    "cc_solve_workspace_bytes": (c_int, [c_void_p, _P(cc_solve_opts), _P(c_size_t)]),
    "cc_solve": (c_int, [c_void_p, _P(cc_integrals), _P(cc_amps), _P(cc_solve_opts), _P(cc_solve_report),
                         c_void_p, c_size_t, c_void_p]),
    "cc_integral_block_elems": (c_int, [c_int, c_int, _P(c_size_t)]),
    "cc_build_integrals_workspace_bytes": (c_int, [c_int, c_int, c_int, c_int, _P(c_size_t)]),
    "cc_build_integrals": (c_int, [c_int, c_int, c_int, c_int, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                   c_void_p, c_void_p, c_void_p, c_size_t, c_void_p]),
    "cc_energy_noalloc": (c_int, [c_int, c_int, c_int, _P(cc_integrals), _P(cc_amps), c_void_p, c_void_p]),
    "cc_solve_batched_workspace_bytes": (c_int, [c_int, _P(c_void_p), _P(cc_solve_opts), _P(c_size_t)]),
    "cc_solve_batched": (c_int, [c_int, _P(c_void_p), _P(cc_integrals), _P(cc_amps), _P(cc_solve_opts),
                                 _P(cc_solve_report), c_void_p, c_size_t, c_void_p]),
    "cc_plan_set_gemm_config": (c_int, [c_void_p, c_int, c_int, c_int, c_int]),
    "cc_plan_autotune": (c_int, [c_void_p, _P(cc_integrals), _P(cc_amps), _P(cc_resid), c_void_p, c_size_t, c_void_p,
                                 c_int]),
    "cc_build_vvvv_packed_workspace_bytes": (c_int, [c_int, c_int, c_int, c_int, _P(c_size_t)]),
    "cc_packed_t2_elems": (ctypes.c_int64, [c_int, c_int]),
    "cc_pack_t2": (c_int, [c_int, c_int, c_int, c_void_p, c_void_p, c_void_p]),
    "cc_unpack_t2": (c_int, [c_int, c_int, c_int, c_void_p, c_void_p, c_void_p]),
    "cc_build_vvvv_packed": (c_int, [c_int, c_int, c_int, c_int, c_void_p, c_void_p, c_void_p, c_size_t, c_void_p]),
    "cc_selftest_wait_timeout": (c_int, [ctypes.c_longlong]),
    "cc_selftest_convert": (c_int, [c_void_p, ctypes.c_longlong, c_void_p, c_void_p]),
    "cc_status_string": (ctypes.c_char_p, [c_int]),
    "cc_last_error": (ctypes.c_char_p, []),
    "cc_version": (ctypes.c_char_p, []),
}
for _name, (_res, _args) in _sig.items():
    _f = getattr(_lib, _name)
    _f.restype = _res
    _f.argtypes = _args


class CCError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        msg = _lib.cc_last_error().decode(errors="replace")
        name = STATUS[status] if 0 <= status < len(STATUS) else str(status)
        super().__init__(f"{where}: {name}: {msg}")


def _check(st: int, where: str, ok=(0,)):
    if st not in ok:
        raise CCError(st, where)
    return st


def _ptr(x):
    if x is None or isinstance(x, int):
        return x
    return x.data_ptr()


def _nbytes(x) -> int:
    if x is None or isinstance(x, int):
        return 0
    return x.numel() * x.element_size()


def _stream(s):
    if s is None or isinstance(s, int):
        return s
    return s.cuda_stream


def cc_version() -> str:
    return _lib.cc_version().decode()


def cc_status_string(s: int) -> str:
    return _lib.cc_status_string(s).decode()


def cc_last_error() -> str:
    return _lib.cc_last_error().decode()


class Plan:
    """Owns a cc_plan handle (a host object)."""

    def __init__(self, handle: int, o: int, v: int, precision: int, text: str, dtype: int = 0):
        self.handle, self.o, self.v, self.precision, self.text = handle, o, v, precision, text
        self.dtype = dtype

    def __del__(self):
        h = getattr(self, "handle", None)
        if h:
            _lib.cc_plan_destroy(h)
            self.handle = None

    @property
    def workspace_bytes(self) -> int:
        return cc_plan_workspace_bytes(self)

    @property
    def flops(self) -> float:
        return cc_plan_flops(self)

    def describe(self) -> dict:
        return cc_plan_describe(self)


def load_list(name: str) -> str:
    """Contraction lists shipped with the package (``lists/<name>.txt``)."""
    with open(os.path.join(LISTS, name + ".txt")) as f:
        return f.read()


def cc_plan_create(text: str, o: int, v: int, dtype: int = CC_F64, precision=CC_PREC_FP64, verbose: int = 0,
                   _route_all: bool = False, packed_vvvv: bool = False, kconcat: bool = True,
                   uniform_steps: bool = False) -> Plan:
    if isinstance(precision, str):
        precision = PRECISIONS[precision]
    prec = precision + (100 if _route_all else 0)   # test hook: every GEMM on the split route
    h = c_void_p()
    opts = cc_plan_opts(ctypes.sizeof(cc_plan_opts), verbose, 0, int(packed_vvvv), int(not kconcat),
                        int(uniform_steps))
    _check(_lib.cc_plan_create(text.encode(), o, v, dtype, prec, ctypes.byref(opts), ctypes.byref(h)),
           "cc_plan_create")
    return Plan(h.value, o, v, precision, text, dtype)


def cc_plan_workspace_bytes(plan: Plan) -> int:
    n = c_size_t()
    _check(_lib.cc_plan_workspace_bytes(plan.handle, ctypes.byref(n)), "cc_plan_workspace_bytes")
    return n.value


def cc_plan_flops(plan: Plan) -> float:
    f = c_double()
    _check(_lib.cc_plan_flops(plan.handle, ctypes.byref(f)), "cc_plan_flops")
    return f.value


def cc_plan_describe(plan: Plan) -> dict:
    need = c_size_t()
    _check(_lib.cc_plan_describe(plan.handle, None, 0, ctypes.byref(need)), "cc_plan_describe")
    buf = ctypes.create_string_buffer(need.value)
    _check(_lib.cc_plan_describe(plan.handle, buf, need.value, ctypes.byref(need)), "cc_plan_describe")
    return json.loads(buf.value.decode())


def cc_plan_profile_enable(plan: Plan, enable: bool = True):
    _check(_lib.cc_plan_profile_enable(plan.handle, int(enable)), "cc_plan_profile_enable")


def cc_plan_profile_read(plan: Plan):
    """(ms_step[], ms_kernel[], calls) accumulated since enabling."""
    n, calls = c_int(), c_int()
    _check(_lib.cc_plan_profile_read(plan.handle, None, None, 0, ctypes.byref(n), ctypes.byref(calls)),
           "cc_plan_profile_read")
    a, b = (c_double * max(n.value, 1))(), (c_double * max(n.value, 1))()
    _check(_lib.cc_plan_profile_read(plan.handle, a, b, n.value, ctypes.byref(n), ctypes.byref(calls)),
           "cc_plan_profile_read")
    return list(a[:n.value]), list(b[:n.value]), calls.value


def cc_plan_launch_count(plan: Plan) -> int:
    c = ctypes.c_longlong()
    _check(_lib.cc_plan_launch_count(plan.handle, ctypes.byref(c)), "cc_plan_launch_count")
    return c.value


def integrals_struct(ints: dict) -> cc_integrals:
    return cc_integrals(*(_ptr(ints.get(k)) for k in ("f_occ", "f_vir", "oooo", "ooov", "oovv", "ovov", "ovvv",
                                                       "vvvv", "vvvv_packed")))


def cc_residual(plan: Plan, ints: dict, t1, t2, r1, r2, ws, stream=None, t3=None, r3=None):
    I = integrals_struct(ints)
    A = cc_amps(_ptr(t1), _ptr(t2), _ptr(t3))
    R = cc_resid(_ptr(r1), _ptr(r2), _ptr(r3))
    _check(_lib.cc_residual(plan.handle, ctypes.byref(I), ctypes.byref(A), ctypes.byref(R), _ptr(ws), _nbytes(ws),
                            _stream(stream)), "cc_residual")


def cc_plan_set_gemm_config(plan: Plan, step: int, bn: int, splitk: int, red: int = 0):
    """Sets one contraction step to one of its autotuning candidates."""
    _check(_lib.cc_plan_set_gemm_config(plan.handle, step, bn, splitk, red), "cc_plan_set_gemm_config")


def cc_plan_autotune(plan: Plan, ints: dict, t1, t2, r1, r2, ws, reps: int = 3, stream=None, t3=None, r3=None):
    """Times the GEMM candidates of every contraction and keeps the fastest
    (the residual buffers receive unspecified values)."""
    I = integrals_struct(ints)
    A = cc_amps(_ptr(t1), _ptr(t2), _ptr(t3))
    R = cc_resid(_ptr(r1), _ptr(r2), _ptr(r3))
    _check(_lib.cc_plan_autotune(plan.handle, ctypes.byref(I), ctypes.byref(A), ctypes.byref(R), _ptr(ws),
                                 _nbytes(ws), _stream(stream), reps), "cc_plan_autotune")


def cc_energy(plan: Plan, ints: dict, t1, t2, e_dev, ws, stream=None):
    I = integrals_struct(ints)
    A = cc_amps(_ptr(t1), _ptr(t2), None)
    _check(_lib.cc_energy(plan.handle, ctypes.byref(I), ctypes.byref(A), _ptr(e_dev), _ptr(ws), _nbytes(ws),
                          _stream(stream)), "cc_energy")


def cc_energy_noalloc(o: int, v: int, ints: dict, t1, t2, e_dev, stream=None, dtype=None):
    """cc_energy without a workspace, for callers that cannot allocate (see
    include/cc.h).  dtype: CC_F64 / CC_C128; by default that of t2."""
    if dtype is None:
        dtype = CC_C128 if getattr(t2, "is_complex", lambda: False)() else CC_F64
    I = integrals_struct(ints)
    A = cc_amps(_ptr(t1), _ptr(t2), None)
    _check(_lib.cc_energy_noalloc(o, v, dtype, ctypes.byref(I), ctypes.byref(A), _ptr(e_dev), _stream(stream)),
           "cc_energy_noalloc")


@dataclass
class SolveResult:
    status: int
    iterations: int
    converged: bool
    switched_at: int
    energy: float             # complex for CC_C128 plans
    rnorm: float
    energies: list
    rnorms: list


def _solve_opts(max_iter, tol, diis_max, resume, refine_plan, switch_tol, verbose):
    return cc_solve_opts(ctypes.sizeof(cc_solve_opts), max_iter, tol, diis_max, resume,
                         refine_plan.handle if refine_plan is not None else None, switch_tol, verbose)


def cc_solve_workspace_bytes(plan: Plan, diis_max: int = 8, refine_plan: Plan | None = None) -> int:
    o = _solve_opts(100, 1e-8, diis_max, 0, refine_plan, 0.0, 0)
    n = c_size_t()
    _check(_lib.cc_solve_workspace_bytes(plan.handle, ctypes.byref(o), ctypes.byref(n)), "cc_solve_workspace_bytes")
    return n.value


def cc_solve(plan: Plan, ints: dict, t1, t2, ws, max_iter: int = 100, tol: float = 1e-8, diis_max: int = 8,
             resume: bool = False, refine_plan: Plan | None = None, switch_tol: float = 0.0, verbose: int = 0,
             stream=None, t3=None) -> SolveResult:
    I = integrals_struct(ints)
    A = cc_amps(_ptr(t1), _ptr(t2), _ptr(t3))
    o = _solve_opts(max_iter, tol, diis_max, int(resume), refine_plan, switch_tol, verbose)
    en = (c_double * max(max_iter, 1))()
    ei = (c_double * max(max_iter, 1))()
    rn = (c_double * max(max_iter, 1))()
    rep = cc_solve_report(0, 0, -1, 0.0, 0.0, ctypes.cast(en, _P(c_double)), ctypes.cast(rn, _P(c_double)), 0.0,
                          ctypes.cast(ei, _P(c_double)))
    st = _lib.cc_solve(plan.handle, ctypes.byref(I), ctypes.byref(A), ctypes.byref(o), ctypes.byref(rep), _ptr(ws),
                       _nbytes(ws), _stream(stream))
    _check(st, "cc_solve", ok=(0, 7))
    k = rep.iterations
    if plan.dtype == CC_C128:
        return SolveResult(st, k, bool(rep.converged), rep.switched_at, complex(rep.energy, rep.energy_im), rep.rnorm,
                           [complex(a, b) for a, b in zip(en[:k], ei[:k])], list(rn[:k]))
    return SolveResult(st, k, bool(rep.converged), rep.switched_at, rep.energy, rep.rnorm, list(en[:k]),
                       list(rn[:k]))


def cc_autotune_cache(clear: bool = False):
    """(entries, hits) of the process-wide shape-keyed tuning cache; clear empties it."""
    e, h = ctypes.c_longlong(), ctypes.c_longlong()
    _check(_lib.cc_autotune_cache(int(clear), ctypes.byref(e), ctypes.byref(h)), "cc_autotune_cache")
    return e.value, h.value


def cc_solve_batched_workspace_bytes(plans, diis_max: int = 8) -> int:
    arr = (c_void_p * len(plans))(*[p.handle for p in plans])
    o = _solve_opts(100, 1e-8, diis_max, 0, None, 0.0, 0)
    n = c_size_t()
    _check(_lib.cc_solve_batched_workspace_bytes(len(plans), arr, ctypes.byref(o), ctypes.byref(n)),
           "cc_solve_batched_workspace_bytes")
    return n.value


def cc_solve_batched(plans, ints, amps, ws, max_iter: int = 100, tol: float = 1e-8, diis_max: int = 8,
                     stream=None):
    """Jacobi + DIIS on len(plans) independent systems.  ints: list of integral
    dicts; amps: list of (t1, t2[, t3]) device tensors (updated in place).
    Returns (status, [SolveResult per system])."""
    n = len(plans)
    parr = (c_void_p * n)(*[p.handle for p in plans])
    I = (cc_integrals * n)(*[integrals_struct(x) for x in ints])
    A = (cc_amps * n)(*[cc_amps(_ptr(a[0]), _ptr(a[1]), _ptr(a[2]) if len(a) > 2 else None) for a in amps])
    o = _solve_opts(max_iter, tol, diis_max, 0, None, 0.0, 0)
    bufs = [((c_double * max(max_iter, 1))(), (c_double * max(max_iter, 1))(), (c_double * max(max_iter, 1))())
            for _ in range(n)]
    reps = (cc_solve_report * n)(*[cc_solve_report(0, 0, -1, 0.0, 0.0, ctypes.cast(b[0], _P(c_double)),
                                                   ctypes.cast(b[1], _P(c_double)), 0.0,
                                                   ctypes.cast(b[2], _P(c_double))) for b in bufs])
    st = _lib.cc_solve_batched(n, parr, I, A, ctypes.byref(o), reps, _ptr(ws), _nbytes(ws), _stream(stream))
    _check(st, "cc_solve_batched", ok=(0, 7))
    out = []
    for p, r, b in zip(plans, reps, bufs):
        k = r.iterations
        if p.dtype == CC_C128:
            out.append(SolveResult(st, k, bool(r.converged), -1, complex(r.energy, r.energy_im), r.rnorm,
                                   [complex(x, y) for x, y in zip(b[0][:k], b[2][:k])], list(b[1][:k])))
        else:
            out.append(SolveResult(st, k, bool(r.converged), -1, r.energy, r.rnorm, list(b[0][:k]), list(b[1][:k])))
    return st, out


BLOCKS = ("oooo", "ooov", "oovv", "ovov", "ovvv", "vvvv")


def cc_integral_block_elems(o: int, v: int) -> dict:
    arr = (c_size_t * 6)()
    _check(_lib.cc_integral_block_elems(o, v, arr), "cc_integral_block_elems")
    return dict(zip(BLOCKS, arr))


def cc_build_integrals_workspace_bytes(o: int, v: int, L: int, dtype: int = CC_F64) -> int:
    n = c_size_t()
    _check(_lib.cc_build_integrals_workspace_bytes(o, v, L, dtype, ctypes.byref(n)),
           "cc_build_integrals_workspace_bytes")
    return n.value


def cc_build_integrals(o: int, v: int, L: int, B, blocks: dict, ws, dtype: int = CC_F64, stream=None):
    _check(_lib.cc_build_integrals(o, v, L, dtype, _ptr(B), *(_ptr(blocks.get(k)) for k in BLOCKS), _ptr(ws),
                                   _nbytes(ws), _stream(stream)), "cc_build_integrals")


def cc_build_vvvv_packed_workspace_bytes(o: int, v: int, L: int, dtype: int = CC_F64) -> int:
    n = c_size_t()
    _check(_lib.cc_build_vvvv_packed_workspace_bytes(o, v, L, dtype, ctypes.byref(n)),
           "cc_build_vvvv_packed_workspace_bytes")
    return n.value


def cc_build_vvvv_packed(o: int, v: int, L: int, B, out, ws, dtype: int = CC_F64, stream=None):
    _check(_lib.cc_build_vvvv_packed(o, v, L, dtype, _ptr(B), _ptr(out), _ptr(ws), _nbytes(ws), _stream(stream)),
           "cc_build_vvvv_packed")


def cc_packed_t2_elems(o: int, v: int) -> int:
    """Elements of the packed (i < j, a < b) doubles amplitudes."""
    return int(_lib.cc_packed_t2_elems(o, v))


def cc_pack_t2(o: int, v: int, t_full, t_packed, dtype: int = CC_F64, stream=None):
    """t_packed[P(i,j)][P(a,b)] = t_full[i][j][a][b] over i < j, a < b (device arrays)."""
    _check(_lib.cc_pack_t2(o, v, dtype, _ptr(t_full), _ptr(t_packed), _stream(stream)), "cc_pack_t2")


def cc_unpack_t2(o: int, v: int, t_packed, t_full, dtype: int = CC_F64, stream=None):
    """The full antisymmetric [o][o][v][v] array from its packed quarter (device arrays)."""
    _check(_lib.cc_unpack_t2(o, v, dtype, _ptr(t_packed), _ptr(t_full), _stream(stream)), "cc_unpack_t2")


def cc_selftest_wait_timeout(budget_cycles: int = 2_000_000) -> int:
    """Runs the bounded-wait self-test; returns the status (CC_ERR_TIMEOUT = 8 expected)."""
    return _lib.cc_selftest_wait_timeout(budget_cycles)


def cc_selftest_convert(x, mine, ref):
    """The split kernels' double -> float rounding and the library's, into mine / ref."""
    _check(_lib.cc_selftest_convert(_ptr(x), x.numel(), _ptr(mine), _ptr(ref)), "cc_selftest_convert")
