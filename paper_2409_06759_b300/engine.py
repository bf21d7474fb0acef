"""Device-side convenience layer over the C ABI (argument marshalling only).

Allocates device buffers with torch, builds the integral blocks with the
library's own kernels (cc_build_integrals), and wraps plans, workspaces and the
solver.  Every arithmetic step runs in libccb300.so.
"""
from __future__ import annotations

import torch

from . import (BLOCKS, CC_C128, CC_F64, cc_build_vvvv_packed, cc_build_vvvv_packed_workspace_bytes,
               cc_plan_autotune, cc_build_integrals, cc_build_integrals_workspace_bytes, cc_energy,
               cc_integral_block_elems, cc_plan_create, cc_residual, cc_solve, cc_solve_batched,
               cc_solve_batched_workspace_bytes, cc_solve_workspace_bytes, load_list)


def alloc_ws(nbytes: int, device) -> torch.Tensor:
    """Workspace buffer (torch's caching allocator returns 512-byte aligned blocks)."""
    t = torch.empty(max(1, (nbytes + 7) // 8), dtype=torch.float64, device=device)
    assert t.data_ptr() % 256 == 0
    return t


class DeviceSystem:
    """Orbital energies and the six integral blocks of one system, on the device.
    A complex factor B (complex spin orbitals) gives complex128 blocks."""

    def __init__(self, o: int, v: int, eps_occ, eps_vir, B, device="cuda:0", blocks=BLOCKS, stream=None,
                 packed_vvvv: bool = False):
        """packed_vvvv: build <ab||ef> only packed (a < b, e < f; a quarter of the
        block, never holding the full one) and leave vvvv out."""
        self.o, self.v, self.device = o, v, torch.device(device)
        self.f_occ = torch.as_tensor(eps_occ, dtype=torch.float64).to(self.device)
        self.f_vir = torch.as_tensor(eps_vir, dtype=torch.float64).to(self.device)
        Bt = torch.as_tensor(B)
        self.dtype = CC_C128 if Bt.is_complex() else CC_F64
        self.tdtype = torch.complex128 if self.dtype == CC_C128 else torch.float64
        Bd = Bt.to(self.tdtype).to(self.device).contiguous()
        L = Bd.shape[0]
        elems = cc_integral_block_elems(o, v)
        if packed_vvvv:
            blocks = tuple(k for k in blocks if k != "vvvv")
        self.packed_vvvv = packed_vvvv
        self.blocks = {k: torch.empty(elems[k], dtype=self.tdtype, device=self.device) for k in blocks}
        ws = alloc_ws(cc_build_integrals_workspace_bytes(o, v, L, self.dtype), self.device)
        cc_build_integrals(o, v, L, Bd, self.blocks, ws, dtype=self.dtype, stream=stream)
        if packed_vvvv:
            P = v * (v - 1) // 2
            self.blocks["vvvv_packed"] = torch.empty(P * P, dtype=torch.float64, device=self.device)
            del ws
            ws = alloc_ws(cc_build_vvvv_packed_workspace_bytes(o, v, L, self.dtype), self.device)
            cc_build_vvvv_packed(o, v, L, Bd, self.blocks["vvvv_packed"], ws, dtype=self.dtype, stream=stream)
        torch.cuda.synchronize(self.device)
        del ws, Bd

    @classmethod
    def from_system(cls, sysm, device="cuda:0", scale: float = 1.0, **kw):
        return cls(sysm.o, sysm.v, sysm.eps_occ, sysm.eps_vir, sysm.B * scale, device=device, **kw)

    def ints(self) -> dict:
        d = dict(f_occ=self.f_occ, f_vir=self.f_vir)
        d.update(self.blocks)
        return d

    def block(self, name: str) -> torch.Tensor:
        shape = [self.o if c == "o" else self.v for c in name]
        return self.blocks[name].view(*shape)


class Engine:
    """A plan plus its workspace for one system."""

    def __init__(self, system: DeviceSystem, list_text: str | None = None, precision="fp64",
                 route_all: bool = False, list_name: str | None = None, kconcat: bool = True,
                 uniform_steps: bool = False):
        """uniform_steps: every contraction on the tensor-core split route, none
        merged (plans of one list then have the same steps at any size, which
        lets a BatchSolver run its systems in grouped launches)."""
        if list_text is None:
            list_text = load_list(list_name or ("ccsd" if precision == "fp64" else "ccsd_vvvv"))
        self.triples = "T3[" in list_text
        self.sys = system
        self.plan = cc_plan_create(list_text, system.o, system.v, system.dtype, precision, _route_all=route_all,
                                   kconcat=kconcat, uniform_steps=uniform_steps,
                                   packed_vvvv=getattr(system, "packed_vvvv", False))
        self._ws = None

    @property
    def ws(self):
        """The plan's workspace, allocated on first use (a Solver brings its own,
        so an engine used only through a Solver never holds a second copy).  At
        least 16 KiB: cc_energy takes its scratch from the same buffer."""
        if self._ws is None:
            self._ws = alloc_ws(max(self.plan.workspace_bytes, 16384), self.sys.device)
        return self._ws

    def autotune(self, t1, t2, reps: int = 3, t3=None, stream=None):
        """cc_plan_autotune on these amplitudes (scratch residual buffers)."""
        o, v, dev, dt = self.sys.o, self.sys.v, self.sys.device, self.sys.tdtype
        r1 = torch.empty(o, v, dtype=dt, device=dev)
        r2 = torch.empty(o, o, v, v, dtype=dt, device=dev)
        r3 = torch.empty(o, o, o, v, v, v, dtype=dt, device=dev) if t3 is not None else None
        cc_plan_autotune(self.plan, self.sys.ints(), t1, t2, r1, r2, self.ws, reps=reps, stream=stream, t3=t3, r3=r3)

    def release(self):
        """Drops the workspace (allocated again on the next residual or energy)."""
        self._ws = None

    def residual(self, t1, t2, r1=None, r2=None, stream=None, t3=None, r3=None):
        """(R1, R2), or (R1, R2, R3) when t3 is given (a list with triples)."""
        o, v, dev = self.sys.o, self.sys.v, self.sys.device
        dt = self.sys.tdtype
        r1 = torch.empty(o, v, dtype=dt, device=dev) if r1 is None else r1
        r2 = torch.empty(o, o, v, v, dtype=dt, device=dev) if r2 is None else r2
        if t3 is not None and r3 is None:
            r3 = torch.empty(o, o, o, v, v, v, dtype=dt, device=dev)
        cc_residual(self.plan, self.sys.ints(), t1, t2, r1, r2, self.ws, stream=stream, t3=t3, r3=r3)
        return (r1, r2) if t3 is None else (r1, r2, r3)

    def energy(self, t1, t2, stream=None):
        """float, or complex for a complex system."""
        e = torch.zeros(2, dtype=torch.float64, device=self.sys.device)
        cc_energy(self.plan, self.sys.ints(), t1, t2, e, self.ws, stream=stream)
        if self.sys.dtype == CC_C128:
            return complex(e[0].item(), e[1].item())
        return float(e[0].item())


class Solver:
    """cc_solve with its own workspace (the DIIS history lives there)."""

    def __init__(self, engine: Engine, diis_max: int = 8, refine: Engine | None = None):
        self.eng, self.refine, self.diis_max = engine, refine, diis_max
        nb = cc_solve_workspace_bytes(engine.plan, diis_max, refine.plan if refine else None)
        self.ws = alloc_ws(nb, engine.sys.device)

    def solve(self, t1, t2, max_iter=100, tol=1e-8, resume=False, switch_tol=0.0, verbose=0, stream=None, t3=None):
        return cc_solve(self.eng.plan, self.eng.sys.ints(), t1, t2, self.ws, max_iter=max_iter, tol=tol,
                        diis_max=self.diis_max, resume=resume,
                        refine_plan=self.refine.plan if self.refine else None, switch_tol=switch_tol,
                        verbose=verbose, stream=stream, t3=t3)


class BatchSolver:
    """cc_solve_batched over several engines (one system each), one workspace."""

    def __init__(self, engines, diis_max: int = 8):
        self.engines, self.diis_max = list(engines), diis_max
        nb = cc_solve_batched_workspace_bytes([e.plan for e in self.engines], diis_max)
        self.ws = alloc_ws(nb, self.engines[0].sys.device)

    def solve(self, amps, max_iter=100, tol=1e-8, stream=None):
        """amps: list of (t1, t2[, t3]) per engine, updated in place.
        Returns (status, [SolveResult])."""
        return cc_solve_batched([e.plan for e in self.engines], [e.sys.ints() for e in self.engines], amps,
                                self.ws, max_iter=max_iter, tol=tol, diis_max=self.diis_max, stream=stream)
