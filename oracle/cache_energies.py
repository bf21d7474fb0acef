"""Writes the oracle's converged CCSD energies to baseline/oracle_cache.json.

Test infrastructure: this script calls only ``oracle/`` (and the seeded input
generator ``ccinputs``), never the CUDA path, so every stored value is the
oracle's.  The benchmark and the tests read the file to report and check the
GPU path's energy error against the oracle at sizes where an oracle solve
takes minutes to hours.

Entries are keyed by workload name and carry the workload (o, v, L, seed,
dtype), a fingerprint of the generated inputs (so a changed generator is
detected), the oracle routine, the per-iteration energies and residual norms
of the Jacobi+DIIS solve from T = 0 (the reading every solver here follows),
the energy of the first iterate with |R| < 1e-8 and the final energy.

    python -m oracle.cache_energies small      # o=10 v=40 (explicit-loop and block oracles)
    python -m oracle.cache_energies ladder     # o=40 v=200 FP64 (block oracle, ~45 GB host RAM)
    python -m oracle.cache_energies batched    # the 64 uneven batched systems
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import platform
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

CACHE = os.path.join(ROOT, "baseline", "oracle_cache.json")
TOL = 1e-11          # the stored trajectory runs past the 1e-8 stopping rule of the benchmark


def fingerprint(s) -> str:
    h = hashlib.sha256()
    h.update(np.ascontiguousarray(s.eps).tobytes())
    h.update(np.ascontiguousarray(s.B).tobytes())
    return h.hexdigest()[:16]


def load() -> dict:
    if os.path.exists(CACHE):
        with open(CACHE) as f:
            return json.load(f)
    return {}


def save(cache: dict) -> None:
    os.makedirs(os.path.dirname(CACHE), exist_ok=True)
    tmp = CACHE + ".tmp"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
        f.write("\n")
    os.replace(tmp, CACHE)


def _re(x):
    return [float(np.real(e)) for e in x]


def entry(s, res, routine, wall, dtype="f64") -> dict:
    rn = [float(r) for r in res["rnorms"]]
    en = _re(res["energies"])
    k8 = next((k for k, r in enumerate(rn) if r < 1e-8), None)
    e = {"o": s.o, "v": s.v, "L": s.L, "seed": s.seed, "dtype": dtype, "inputs_sha256_16": fingerprint(s),
         "oracle": routine, "tol": TOL, "status": int(res["status"]), "iterations": int(res["iters"]),
         "energies": en, "rnorms": rn, "energy": en[-1],
         "energy_at_tol_1e-8": en[k8] if k8 is not None else None,
         "iterations_to_tol_1e-8": (k8 + 1) if k8 is not None else None,
         "wall_s": wall, "host": platform.node(), "threads": os.cpu_count()}
    if dtype == "c128":
        e["energy_im"] = float(np.imag(res["energies"][-1]))
    return e


def run_small(cache):
    import ccinputs
    import oracle
    from oracle import cc_blocks

    s = ccinputs.make_system(10, 40, L=120, seed=0)
    t = time.time()
    V = oracle.antisym_integrals(s.o, s.v, s.B)
    res = oracle.ccsd_solve(s.o, s.v, s.eps, V, tol=TOL, maxiter=100)
    cache["ccsd_o10_v40_L120_seed0_f64"] = entry(s, res, "orc_ccsd_solve (cc_oracle.c)", time.time() - t)
    t = time.time()
    blk = cc_blocks.integral_blocks(s.o, s.v, s.B)
    res_b = cc_blocks.ccsd_solve(s.o, s.v, s.eps, blk, tol=TOL, maxiter=100)
    cache["ccsd_o10_v40_L120_seed0_f64_blocks"] = entry(s, res_b, "cc_blocks.ccsd_solve", time.time() - t)


def run_ladder(cache, complex_=False):
    import ccinputs
    from oracle import cc_blocks

    s = ccinputs.make_system(40, 200, L=120, seed=0, complex_=complex_)
    t = time.time()
    blk = cc_blocks.integral_blocks(s.o, s.v, s.B)
    t_blk = time.time() - t

    def log(k, e, rn):
        print(f"  iter {k:2d}  E = {np.real(e):.15f}  |R| = {rn:.3e}  ({time.time() - t:.0f} s)", flush=True)

    res = cc_blocks.ccsd_solve(s.o, s.v, s.eps, blk, tol=TOL, maxiter=60, log=log)
    key = "ccsd_o40_v200_L120_seed0_" + ("c128" if complex_ else "f64")
    cache[key] = entry(s, res, "cc_blocks.ccsd_solve", time.time() - t, dtype="c128" if complex_ else "f64")
    cache[key]["integral_blocks_s"] = t_blk


def run_batched(cache):
    import ccinputs
    from oracle import cc_blocks

    sizes = ccinputs.batched_sizes(64, seed=0)
    out = []
    t0 = time.time()
    for o, v, sd in sizes:
        s = ccinputs.make_system(o, v, L=120, seed=sd)
        t = time.time()
        blk = cc_blocks.integral_blocks(o, v, s.B)
        res = cc_blocks.ccsd_solve(o, v, s.eps, blk, tol=TOL, maxiter=100)
        e = entry(s, res, "cc_blocks.ccsd_solve", time.time() - t)
        for k in ("host", "threads", "tol", "oracle"):
            e.pop(k)
        out.append(e)
        print(f"  o={o:2d} v={v:2d} seed={sd:2d}  E = {e['energy']:.15f}  iters {e['iterations']}", flush=True)
    cache["ccsd_batched64_L120_seed0_f64"] = {"oracle": "cc_blocks.ccsd_solve", "tol": TOL,
                                              "systems": out, "wall_s": time.time() - t0,
                                              "host": platform.node(), "threads": os.cpu_count()}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("which", nargs="+", choices=["small", "ladder", "ladder_c128", "batched"])
    args = ap.parse_args()
    for w in args.which:
        cache = load()
        print(f"[oracle cache] {w}", flush=True)
        {"small": run_small, "ladder": run_ladder, "batched": run_batched,
         "ladder_c128": lambda c: run_ladder(c, complex_=True)}[w](cache)
        save(cache)
    print(f"[oracle cache] written {CACHE}")


if __name__ == "__main__":
    main()
