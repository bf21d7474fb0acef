"""Benchmark: CC residual TFLOP/s and s/iter on one B300, split-bf16 vs FP64.

Workload: spin-orbital CCSD, o=40 occupied, v=200 virtual, L=120, seed 0,
FP64 real, synthetic integrals (ccinputs).  One step = one iteration of
cc_solve: the full residual (every statement of the contraction list), the
energy, |R|, the Jacobi update and the DIIS extrapolation.

  python bench.py [--steps K] [--warmup W] [--gpus N] [--impl ours|reference]
                  [--dtype f64|c128] [--workload ccsd|ccsdt|batched|ladder]

The default run (N = 1) also carries:
  * time to solution (|R| < 1e-8) of every precision, each energy compared
    with the oracle's converged energy (baseline/oracle_cache.json, written by
    oracle/cache_energies.py, which calls only the oracle);
  * the oracle timed on the host cores (cpu_baseline);
  * compact results of the complex128, CCSDT and batched workloads ("c128",
    "ccsdt", "batched"; --no-suite skips them).

--dtype c128 runs the main workload with complex spin orbitals (complex
Hermitian integrals, complex amplitudes; every complex product is four real
ones, counted as such in the flops).

Under torchrun (N > 1) every rank runs an independent replica (the residual of
one system does not shard without an exchange; no collective is used on the
data path); value = all ranks' flops / the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "CC residual TFLOP/s and s/iter on 1 B300, mixed vs FP64 at |ΔE|<1e-6 Eh"
WORKLOAD = "spin-orbital CCSD o=40 v=200 L=120 seed=0, FP64 real, synthetic integrals"
SMALL = "spin-orbital CCSD o=10 v=40 L=120 seed=0, FP64 real, synthetic integrals"
WORKLOAD_C = "spin-orbital CCSD o=40 v=200 L=120 seed=0, complex128 (complex spin orbitals), synthetic integrals"
SMALL_C = "spin-orbital CCSD o=10 v=40 L=120 seed=0, complex128 (complex spin orbitals), synthetic integrals"
WORKLOAD_T = "spin-orbital CCSDT o=8 v=64 L=96 seed=0, FP64 real, synthetic integrals, generated list"
WORKLOAD_B = "batched CCSD: 64 systems, o ~ U[4,16], v ~ U[20,80], L=120, sub-seeds 0..63, FP64 real, synthetic"

# Flops of one residual evaluation of the timed split-bf16 plan (lists/ccsd_vvvv.txt) as the library
# counts them (dense 2MNK over the executed GEMMs; complex: four real products each).  Recorded here
# so that the reference arm never loads the library; tests/test_abi_cpu.py checks them against
# cc_plan_flops.
PLAN_FLOPS = {("ccsd_vvvv", 40, 200, "f64"): 8777761280000.0, ("ccsd_vvvv", 10, 40, "f64"): 1056000000.0,
              ("ccsd_vvvv", 40, 200, "c128"): 35111045120000.0, ("ccsd_vvvv", 10, 40, "c128"): 4224000000.0}

ORACLE_CACHE = os.path.join(ROOT, "baseline", "oracle_cache.json")

# DRAM bytes (read + write) of one launch of the o=40 v=200 ladder step in this benchmark's own
# iteration, from a one-pass ncu capture of the current kernel version (set to None when the kernel
# changes, until it is captured again): 11.06 GB read, mostly the <ab||ef> planes once and the tau
# planes once per wave of 148 tiles, plus 0.49 GB written
LADDER_TRAFFIC = 11.55e9


def jsonable(e):
    """A (possibly complex) energy as JSON: a number, or [re, im]."""
    return [e.real, e.imag] if isinstance(e, complex) else e


def workload_name(args, dtype=None):
    if args.size:
        return (f"spin-orbital CCSD o={args.size.split(',')[0]} v={args.size.split(',')[1]} L=120 seed=0, "
                f"{'complex128' if (dtype or args.dtype) == 'c128' else 'FP64 real'}, synthetic integrals")
    if (dtype or args.dtype) == "c128":
        return SMALL_C if args.small else WORKLOAD_C
    return SMALL if args.small else WORKLOAD


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "bf16_tflops_sustained": 1400.0}, "fallback"


def oracle_reference(o, v, dtype="f64", seed=0, L=120):
    """The oracle's cached solve of this workload, or None."""
    if not os.path.exists(ORACLE_CACHE):
        return None
    with open(ORACLE_CACHE) as f:
        cache = json.load(f)
    return cache.get(f"ccsd_o{o}_v{v}_L{L}_seed{seed}_{dtype}")


def delta_e(e, ref):
    return None if ref is None or e is None else abs(e - ref)


class Clocks:
    """nvidia-smi sampling during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                      stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.p is not None:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.p.kill()

    def summary(self):
        self.f.flush()
        self.f.seek(0)
        rows = [r.split(",") for r in self.f.read().strip().splitlines() if r.strip()]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].strip().replace(".", "").isdigit()]
        pw = [float(r[3]) for r in rows if r[3].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in rows:
            for nm, val in zip(names, r[5:9]):
                if val.strip().lower() == "active":
                    reasons.add(nm)
        load = [x for x, p in zip(sm, pw) if p > 300] or sm
        return {"sm_mhz": statistics.median(load) if load else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(rows)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if __import__("torch").cuda.is_available() else "gloo")
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x: float, world: int) -> float:
    """The slowest rank's time (replicas: every rank times its own copy of the step)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def fp64_peak_live(torch):
    """cuBLAS DGEMM 4096^3, best of 3 (the FP64 roofline denominator)."""
    n = 4096
    a = torch.randn(n, n, dtype=torch.float64, device="cuda")
    b = torch.randn(n, n, dtype=torch.float64, device="cuda")
    for _ in range(2):
        a @ b
    torch.cuda.synchronize()
    best = 1e9
    for _ in range(3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        a @ b
        e1.record()
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1) / 1e3)
    del a, b
    return 2 * n ** 3 / best / 1e12


# ---------------------------------------------------------------- the oracle on the host cores
def cpu_leg_small():
    """(run in a child process, so its thread count can be fixed) the explicit-loop oracle
    (cc_oracle.c) on the o=10 v=40 system: one residual of random amplitudes and the
    Jacobi+DIIS solve from T = 0 to |R| < 1e-8.  Prints one JSON line."""
    import ccinputs
    import oracle
    s = ccinputs.make_system(**ccinputs.CONFIG_SMALL)
    o, v = s.o, s.v
    t0 = time.perf_counter()
    V = oracle.antisym_integrals(o, v, s.B)
    t_int = time.perf_counter() - t0
    t1, t2 = ccinputs.random_amplitudes(o, v, seed=0, scale1=0.01, scale2=0.01)
    t0 = time.perf_counter()
    oracle.ccsd_residual(o, v, s.eps, V, t1, t2)
    t_res = time.perf_counter() - t0
    t0 = time.perf_counter()
    res = oracle.ccsd_solve(o, v, s.eps, V, tol=1e-8, maxiter=100)
    t_sol = time.perf_counter() - t0
    print(json.dumps({"threads": oracle.num_threads(), "integrals_s": t_int, "residual_s": t_res,
                      "solve_s": t_sol, "iterations": int(res["iters"]), "energy": float(res["energy"])}))


def cpu_small_both():
    """The o=10 v=40 oracle leg with one thread and with every host core."""
    out = {}
    for name, nthr in (("one_thread", "1"), ("all_threads", None)):
        env = dict(os.environ)
        if nthr:
            env.update(OMP_NUM_THREADS=nthr, OPENBLAS_NUM_THREADS=nthr)
        r = subprocess.run([sys.executable, os.path.abspath(__file__), "--cpu-leg", "small"], env=env,
                           capture_output=True, text=True, timeout=1200)
        out[name] = json.loads(r.stdout.strip().splitlines()[-1]) if r.returncode == 0 else {"error": r.stderr[-300:]}
    return out


def cpu_baseline(o, v, flops, complex_=False, small=None):
    """The FP64 oracle on the host cores, before any GPU work.
    value: one full residual of this workload by the block oracle (oracle/cc_blocks.py, the
    CCSD equations with one library contraction per term), integral blocks built first and
    timed apart; flops counted as the timed plan counts them, so the value's ratio to the GPU
    figure is the ratio of seconds per residual.
    Beside it: the explicit-loop oracle's per-element cost on this workload (sampled R2
    elements, shared part built first and timed apart) and its o=10 v=40 residual and solve
    with one thread and with all threads."""
    import gc

    import numpy as np

    import ccinputs
    import oracle
    from oracle import cc_blocks

    s = ccinputs.make_system(o, v, L=120, seed=0, complex_=complex_)
    t1, t2 = ccinputs.random_amplitudes(o, v, seed=0, scale1=0.01, scale2=0.01, complex_=complex_)
    out = {"unit": "TFLOP/s", "cores": os.cpu_count(), "kind": "oracle"}
    if not complex_:
        t0 = time.perf_counter()
        blk = cc_blocks.integral_blocks(o, v, s.B)
        t_setup = time.perf_counter() - t0
        t0 = time.perf_counter()
        cc_blocks.ccsd_residual(o, v, s.eps, blk, t1, t2)
        t_res = time.perf_counter() - t0
        del blk
        gc.collect()
        out.update(value=flops / t_res / 1e12, seconds_per_residual=t_res, setup_s=t_setup,
                   sample=f"one full CCSD residual at o={o} v={v} (random amplitudes) by the block-form FP64 "
                          f"oracle (numpy, OpenBLAS on the host cores); integral blocks from B built first, "
                          f"setup_s apart; value = {flops:.4g} flop (the timed plan's count) / seconds_per_residual")
    # the explicit-loop oracle's sampled elements, shared part built once
    ns = max(4, os.cpu_count() or 4)
    rng = np.random.default_rng(1)
    idx = np.stack([rng.integers(0, o, ns), rng.integers(0, o, ns), rng.integers(0, v, ns),
                    rng.integers(0, v, ns)], 1)
    t0 = time.perf_counter()
    with oracle.R2Sampler(o, v, s.B, s.eps, t1, t2) as smp:
        t_prep = time.perf_counter() - t0
        t0 = time.perf_counter()
        smp.eval(idx)
        t_el = time.perf_counter() - t0
    per_el = t_el / ns
    out["sampled_elements"] = {"elements": ns, "setup_s": t_prep, "per_element_s": per_el,
                               "threads": oracle.num_threads(),
                               "tflops": flops / (per_el * o * o * v * v) / 1e12,
                               "note": "explicit-loop oracle (cc_oracle.c), R2 elements one by one; tflops = "
                                       "flops / (per_element_s x o^2 v^2)"}
    if complex_:
        out.update(value=out["sampled_elements"]["tflops"], setup_s=t_prep,
                   sample=f"{ns} R2 elements of the o={o} v={v} complex residual by the explicit-loop oracle, "
                          f"shared part built first (setup_s apart); value = flops / (per-element s x o^2 v^2)")
    if small is not None:
        out["small_o10_v40"] = small
    return out


def run_reference(args, world, rank):
    """The reference arm: the explicit-loop FP64 oracle (cc_oracle.c) on this workload, as it
    stands, on the host cores.  Its shared part (integral blocks oovv/ooov/ovvv, tau, the
    one-particle intermediates) is built once before the warm-up; each step evaluates one R2
    element per host thread.  Only the oracle is loaded (no product library)."""
    if rank != 0:
        return
    import numpy as np

    import ccinputs
    import oracle
    cplx = args.dtype == "c128"
    o, v = (10, 40) if args.small else (40, 200)
    flops = PLAN_FLOPS[("ccsd_vvvv", o, v, "c128" if cplx else "f64")]
    s = ccinputs.make_system(o, v, L=120, seed=0, complex_=cplx)
    t1, t2 = ccinputs.random_amplitudes(o, v, seed=0, scale1=0.01, scale2=0.01, complex_=cplx)
    ns = oracle.num_threads()
    rng = np.random.default_rng(2)
    t0 = time.perf_counter()
    smp = oracle.R2Sampler(o, v, s.B, s.eps, t1, t2)
    t_setup = time.perf_counter() - t0
    times = []
    for k in range(args.warmup + args.steps):
        idx = np.stack([rng.integers(0, o, ns), rng.integers(0, o, ns), rng.integers(0, v, ns),
                        rng.integers(0, v, ns)], 1)
        t0 = time.perf_counter()
        smp.eval(idx)
        if k >= args.warmup:
            times.append(time.perf_counter() - t0)
    smp.close()
    step = sum(times) / len(times)
    value = flops * ns / float(o * o * v * v) / step / 1e12
    sample = (f"{ns} R2 elements per step (one per host thread) of the o={o} v={v} "
              f"{'complex ' if cplx else ''}residual by the explicit-loop FP64 oracle; its shared part "
              f"(integral blocks, tau, one-particle intermediates) built once before the warm-up in "
              f"{t_setup:.1f} s; value = {flops:.4g} flop x {ns}/(o^2 v^2) / step time")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": step * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128" if cplx else "f64",
            "data": "synthetic", "config": {"workload": workload_name(args)},
            "cpu_baseline": {"value": value, "unit": "TFLOP/s", "cores": ns, "kind": "oracle", "sample": sample,
                             "setup_s": t_setup},
            "e2e": {"value": value, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- the main CCSD workload
def run_ccsd(args, world, rank, local, dtype="f64", suite=False, cpu=None):
    """The CCSD iteration at o=40 v=200 (or o=10 v=40 with --small).  suite: the compact form
    run beside the main workload (no packed leg, no FP64-alone solve)."""
    import torch

    import ccinputs
    import paper_2409_06759_b300 as cc
    from paper_2409_06759_b300.engine import DeviceSystem, Engine, Solver

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    cfg = dict(ccinputs.CONFIG_SMALL if args.small else ccinputs.CONFIG_LADDER)
    if args.size:
        cfg["o"], cfg["v"] = (int(x) for x in args.size.split(","))
    o, v = cfg["o"], cfg["v"]
    cplx = dtype == "c128"
    cdt = cc.CC_C128 if cplx else cc.CC_F64
    tdt = torch.complex128 if cplx else torch.float64
    esz = 16 if cplx else 8
    pk, pk_kind = peaks()
    packed = args.packed and not suite and not cplx
    oref = oracle_reference(o, v, dtype)
    e_or = oref["energy"] if oref else None

    sysm = ccinputs.make_system(**cfg, complex_=cplx)
    t0 = time.perf_counter()
    # --packed: <ab||ef> held only packed (a < b, e < f), the full block never built
    dsys = DeviceSystem.from_system(sysm, device=dev, packed_vvvv=packed)
    t_int = time.perf_counter() - t0
    int_bytes = sum(b.numel() * b.element_size() for b in dsys.blocks.values())
    mixed_list = "ccsd_packed" if packed else "ccsd_vvvv"
    fp64_list = "ccsd_packed" if packed else "ccsd"
    mixed = Engine(dsys, list_name=mixed_list, precision=args.precision)
    fp64 = Engine(dsys, list_name=fp64_list)
    stream = torch.cuda.current_stream(dev)
    z = lambda: (torch.zeros(o, v, dtype=tdt, device=dev),
                 torch.zeros(o, o, v, v, dtype=tdt, device=dev))

    # tile widths and split-K factors of the mixed plan picked by timing (cc_plan_autotune)
    t_tune = None
    if args.load_tune and not suite:
        # replay a configuration saved by an earlier run (e.g. for a profiler run,
        # where timings taken under the profiler would mislead the autotuner)
        for k, bn, sk, red in json.load(open(args.load_tune)):
            cc.cc_plan_set_gemm_config(mixed.plan, k, bn, sk, red)
    elif not args.no_tune:
        tt = time.perf_counter()
        mixed.autotune(*z(), reps=3, stream=stream)
        mixed.release()
        torch.cuda.synchronize()
        t_tune = time.perf_counter() - tt
    if args.save_tune and rank == 0 and not suite:
        cfgs = [[k, st.get("bn", 0), st["splitk"], st.get("red", 0)] for k, st in
                enumerate(mixed.plan.describe()["steps"]) if st.get("configs")]
        json.dump(cfgs, open(args.save_tune, "w"))

    # ---- device-timed steps on the split-bf16 plan
    t1, t2 = z()
    sol = Solver(mixed)
    sol.solve(t1, t2, max_iter=args.warmup, tol=0.0, stream=stream)
    cc.cc_plan_profile_enable(mixed.plan, True)
    n0 = cc.cc_plan_launch_count(mixed.plan)
    torch.cuda.synchronize()
    barrier(world)
    torch.cuda.synchronize()
    with Clocks(local) as clk:
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sol.solve(t1, t2, max_iter=args.steps, tol=0.0, resume=True, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
    barrier(world)
    launches = cc.cc_plan_launch_count(mixed.plan) - n0
    dt = max_over_ranks(e0.elapsed_time(e1) / 1e3, world)
    ms_step, ms_kernel, calls = cc.cc_plan_profile_read(mixed.plan)
    cc.cc_plan_profile_enable(mixed.plan, False)
    desc = mixed.plan.describe()
    flops = mixed.plan.flops
    s_iter = dt / args.steps
    value = world * flops * args.steps / dt / 1e12

    # roofline of the dominant kernel (largest accumulated kernel time)
    k_dom = max(range(len(ms_kernel)), key=lambda k: ms_kernel[k])
    st = desc["steps"][k_dom]
    t_kernel = ms_kernel[k_dom] / calls / 1e3
    if st["kind"] == "gemm_bf16split":
        # tensor-pipe flops: products x 2 M N K of the real GEMM the kernel runs (for a
        # complex contraction that GEMM carries the four real products of each complex one)
        tflop = st["products"] * 2.0 * st["M"] * st["N"] * st["K"]
        achieved = tflop / t_kernel / 1e12
        # the kernel runs ~10 ms inside a ~30 ms step: the burst figure is the denominator
        peak = pk["bf16_tflops"]
        # DRAM bytes of one launch, measured by ncu on this workload (None until captured)
        traffic = None
        if (not cplx and not args.small and not packed and args.precision == "bf16x3" and (o, v) == (40, 200)
                and st["M"] == v * v and st["N"] == o * o):
            traffic = LADDER_TRAFFIC
        roof = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": traffic, "traffic_unit": "bytes per launch",
                "kernel": "tc_gemm_persistent_kernel (" + st["note"] + ")",
                "fp64_equiv_tflops": st["flops"] / t_kernel / 1e12, "ms_per_launch": t_kernel * 1e3,
                "gemm_shape": [st["M"], st["N"], st["K"]],
                "frac_of_sustained": achieved / pk["bf16_tflops_sustained"],
                "peak_kind": f"{pk_kind} bf16 burst (tensor-pipe flops = {st['products']} products x 2MNK)"}
    else:
        roof = {"bound": "fp64", "achieved": st.get("flops", 0) / t_kernel / 1e12, "peak": None, "unit": "TFLOP/s",
                "frac": None, "traffic": None, "kernel": st["note"]}

    # ---- end to end through the C ABI with host buffers: the amplitudes live on
    # the host (T2 in its packed i<j, a<b quarter, cc_pack_t2's layout); every
    # step copies them in, unpacks, iterates once, packs and copies them out
    npk = cc.cc_packed_t2_elems(o, v)
    h1 = torch.empty(o, v, dtype=tdt).pin_memory()
    h2 = torch.empty(npk, dtype=tdt).pin_memory()
    d2 = torch.empty(npk, dtype=tdt, device=dev)
    cc.cc_pack_t2(o, v, t2, d2, dtype=cdt, stream=stream)
    torch.cuda.synchronize()
    h1.copy_(t1.cpu())
    h2.copy_(d2.cpu())
    e2e_steps = max(2, min(args.steps, 4))
    torch.cuda.synchronize()
    barrier(world)
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    with torch.cuda.stream(stream):
        for _ in range(e2e_steps):
            t1.copy_(h1, non_blocking=True)
            d2.copy_(h2, non_blocking=True)
            cc.cc_unpack_t2(o, v, d2, t2, dtype=cdt, stream=stream)
            sol.solve(t1, t2, max_iter=1, tol=0.0, resume=True, stream=stream)
            cc.cc_pack_t2(o, v, t2, d2, dtype=cdt, stream=stream)
            h1.copy_(t1, non_blocking=True)
            h2.copy_(d2, non_blocking=True)
    f1.record(stream)
    torch.cuda.synchronize()
    dt_e2e = max_over_ranks(f0.elapsed_time(f1) / 1e3, world)
    nbytes = (h1.numel() + h2.numel()) * esz
    e2e = {"value": world * flops * e2e_steps / dt_e2e / 1e12, "unit": "TFLOP/s", "h2d_bytes_per_step": nbytes,
           "d2h_bytes_per_step": nbytes, "s_per_iter": dt_e2e / e2e_steps}

    line = {"metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": s_iter * 1e3, "s_per_iter": s_iter, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": f"{args.precision}: bf16 tensor-core products, fp32 "
            "accumulation, fp64 outputs/energy/DIIS" + (" (complex128 tensors)" if cplx else ""), "data": "synthetic",
            "config": {"workload": workload_name(args, dtype), "precision": args.precision,
                       "list": mixed_list, "fp64_list": fp64_list, "flops_per_iter": flops, "replicas": world,
                       "flops_counted": "packed (pair-count) flops" if packed else "unpacked flops",
                       "l2": "inputs larger than L2 (<ab||ef> split planes %.2f GB, T2 %d MB)"
                             % (2 * 2 * v ** 4 * (2 if cplx else 1) / 1e9, esz * o * o * v * v // 10 ** 6),
                       "integral_build_s": t_int, "integral_bytes": int_bytes, "autotune_s": t_tune,
                       "gemm_configs": {st["note"]: [st.get("bn", 0), st["splitk"], st.get("red", 0)]
                                        for st in desc["steps"] if st.get("configs")}},
            "roofline": roof, "e2e": e2e, "gpu_launches": launches, "clocks": clk.summary()}
    if cpu is not None:
        line["cpu_baseline"] = cpu

    # ---- time to solution (|R| < 1e-8) of every precision, each energy against the
    #      oracle's converged energy of this workload (and against the FP64 GPU leg)
    if args.no_tts:
        return line
    del sol, t1, t2
    torch.cuda.empty_cache()
    acc = Engine(dsys, list_name=mixed_list, precision="bf16x6") if args.precision != "bf16x6" else mixed

    def timed_solve(eng, refine=None, max_iter=60, **kw):
        a1, a2 = z()
        g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        sol_ = Solver(eng, refine=refine)
        torch.cuda.synchronize()
        g0.record(stream)
        r = sol_.solve(a1, a2, max_iter=max_iter, tol=1e-8, stream=stream, **kw)
        g1.record(stream)
        torch.cuda.synchronize()
        del sol_, a1, a2
        torch.cuda.empty_cache()
        return r, g0.elapsed_time(g1) / 1e3

    legs = {}
    rf = None
    if not suite:
        fpk = fp64_peak_live(torch)
        cc.cc_plan_profile_enable(fp64.plan, True)
        rf, t_f = timed_solve(fp64)
        fms, fker, fcalls = cc.cc_plan_profile_read(fp64.plan)
        cc.cc_plan_profile_enable(fp64.plan, False)
        legs["fp64"] = (rf, t_f)
        fdesc = fp64.plan.describe()
        kf = max(range(len(fker)), key=lambda k: fker[k])
        fst = fdesc["steps"][kf]
        tk = fker[kf] / fcalls / 1e3
        line["fp64"] = {"value": fp64.plan.flops * rf.iterations / t_f / 1e12, "unit": "TFLOP/s",
                        "s_per_iter": t_f / rf.iterations, "iterations": rf.iterations,
                        "time_to_solution_s": t_f, "energy": jsonable(rf.energy), "converged": rf.converged,
                        "delta_E_vs_oracle": delta_e(rf.energy, e_or),
                        "delta_E_vs_oracle_same_stop": delta_e(rf.energy, oref["energy_at_tol_1e-8"] if oref
                                                               else None),
                        "roofline": {"bound": "fp64", "kernel": "gemm_f64_kernel (" + fst["note"] + ")",
                                     "achieved": fst["flops"] / tk / 1e12, "peak": fpk, "unit": "TFLOP/s",
                                     "frac": fst["flops"] / tk / 1e12 / fpk,
                                     "peak_kind": "measured live: cuBLAS DGEMM 4096^3 best of 3"}}
    # a split route alone stalls at its rounding floor when that lies above the tolerance
    legs[args.precision + "_alone"] = timed_solve(mixed, max_iter=30)
    if acc is not mixed:
        legs["bf16x6_alone"] = timed_solve(acc, max_iter=30)
    legs["bf16x6_refined"] = timed_solve(acc, refine=fp64, switch_tol=1e-7)
    # the FP64-grade exact-slice route: alone, and as the refine plan of the split routes
    slices = Engine(dsys, list_name=mixed_list, precision="slices")
    legs["slices_alone"] = timed_solve(slices)
    legs[args.precision + "_refined_slices"] = timed_solve(mixed, refine=slices, switch_tol=1e-7)
    if acc is not mixed:
        legs["bf16x6_refined_slices"] = timed_solve(acc, refine=slices, switch_tol=1e-7)
    del slices
    torch.cuda.empty_cache()
    e_ref = e_or if e_or is not None else legs["bf16x6_refined"][0].energy
    tts = {"oracle_energy": e_or, "oracle": ("baseline/oracle_cache.json: " + oref["oracle"] + f", |R| < "
                                             f"{oref['tol']:g}") if oref else None}
    for name, (r, t) in legs.items():
        tts[name] = {"s": t, "iterations": r.iterations, "converged": r.converged, "energy": jsonable(r.energy),
                     "delta_E_vs_oracle": delta_e(r.energy, e_or),
                     "delta_E_vs_fp64": delta_e(r.energy, rf.energy) if rf is not None else None}
        if "refined" in name:
            tts[name]["switched_at"] = r.switched_at
            tts[name]["rnorms"] = [float(f"{x:.3e}") for x in r.rnorms]
        if rf is not None and name != "fp64":
            tts[name]["speedup_vs_fp64"] = legs["fp64"][1] / t
    if e_or is None:
        tts["note"] = "no cached oracle energy for this workload: delta_E_vs_refined below is against the " \
                      "bf16x6 + FP64-refined solve (converged on the FP64 residual)"
        for name, (r, t) in legs.items():
            tts[name]["delta_E_vs_refined"] = delta_e(r.energy, e_ref)
    line["tts"] = tts
    head = legs[args.precision + "_alone"][0]
    line["accuracy"] = {"headline_precision": args.precision,
                        "delta_E_vs_oracle": delta_e(head.energy, e_or),
                        "delta_E_vs_refined": delta_e(head.energy, legs["bf16x6_refined"][0].energy),
                        "time_to_solution_s": legs[args.precision + "_alone"][1],
                        "meets_1e-6": (delta_e(head.energy, e_or) < 1e-6) if e_or is not None else None}

    # ---- packed index pairs (lists/ccsd_packed.txt, <ab||ef> held only packed):
    #      s/iter of both plans and time to solution; flops counted packed
    if not suite and not packed and not cplx:
        del mixed, fp64, acc, dsys
        torch.cuda.empty_cache()
        pkd = DeviceSystem.from_system(sysm, device=dev, packed_vvvv=True)
        pm = Engine(pkd, list_name="ccsd_packed", precision=args.precision)
        pf = Engine(pkd, list_name="ccsd_packed")
        pa = Engine(pkd, list_name="ccsd_packed", precision="bf16x6")
        a1, a2 = z()
        psol = Solver(pm)
        psol.solve(a1, a2, max_iter=args.warmup, tol=0.0, stream=stream)
        torch.cuda.synchronize()
        h0, h1_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        h0.record(stream)
        psol.solve(a1, a2, max_iter=args.steps, tol=0.0, resume=True, stream=stream)
        h1_.record(stream)
        torch.cuda.synchronize()
        p_iter = h0.elapsed_time(h1_) / 1e3 / args.steps
        del psol, a1, a2
        torch.cuda.empty_cache()
        rpf, tts_pf = timed_solve(pf)
        rpm, tts_pm = timed_solve(pa, refine=pf, switch_tol=1e-7)
        line["packed"] = {"list": "ccsd_packed", "integral_bytes": sum(b.numel() * b.element_size()
                                                                       for b in pkd.blocks.values()),
                          "flops_per_iter": pm.plan.flops, "mixed_s_per_iter": p_iter,
                          "mixed_tflops_packed_flops": pm.plan.flops / p_iter / 1e12,
                          "fp64_time_to_solution_s": tts_pf, "fp64_iterations": rpf.iterations,
                          "fp64_s_per_iter": tts_pf / max(rpf.iterations, 1),
                          "mixed_refined_s": tts_pm, "mixed_refined_iterations": rpm.iterations,
                          "speedup": tts_pf / tts_pm, "delta_E": abs(rpm.energy - rpf.energy),
                          "fp64_delta_E_vs_oracle": delta_e(rpf.energy, e_or),
                          "mixed_refined_delta_E_vs_oracle": delta_e(rpm.energy, e_or),
                          "converged": rpf.converged and rpm.converged}
    return line


# ---------------------------------------------------------------- CCSDT
def run_ccsdt(args, world, rank, local, suite=False):
    """CCSDT workload: s/iter of the FP64 and split-bf16 plans of the generated
    list, the o^3 v^5 terms timed separately, time to |R| < 1e-7."""
    import numpy as np
    import torch

    import ccinputs
    import paper_2409_06759_b300 as cc
    from paper_2409_06759_b300.engine import DeviceSystem, Engine, Solver

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    cfg = dict(ccinputs.CONFIG_CCSDT)
    o, v = cfg["o"], cfg["v"]
    pk, pk_kind = peaks()
    text = cc.load_list("ccsdt")
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu and not suite:
        import oracle
        sm = ccinputs.make_system(**cfg)
        a1, a2, a3 = ccinputs.random_amplitudes(o, v, seed=0, scale1=0.01, scale2=0.01, triples=True)
        idx = np.array([[0, 1, 2, 0, 1, 2], [1, 3, 5, 2, 7, 9], [o - 1, o - 2, o - 3, v - 1, v - 2, v - 3]])
        flops = cc.cc_plan_create(text, o, v).flops
        t0 = time.perf_counter()
        oracle.cc_definition_elements(o, v, sm.B, sm.eps, a1, a2, a3, rank=3, idx=idx)
        dt = time.perf_counter() - t0
        share = len(idx) / float(o ** 3 * v ** 3)
        cpu = {"value": flops * share / dt / 1e12, "unit": "TFLOP/s", "cores": oracle.num_threads(), "kind": "oracle",
               "sample": f"{len(idx)} R3 elements of the o={o} v={v} CCSDT residual by the definition oracle "
                         "(CI coefficients of exp(T) Phi_0, Slater-Condon); value = residual flops x "
                         f"{len(idx)}/(o^3 v^3) / time"}
    sysm = ccinputs.make_system(**cfg)
    dsys = DeviceSystem.from_system(sysm, device=dev)
    stream = torch.cuda.current_stream(dev)
    z = lambda: [torch.zeros(*sh, dtype=torch.float64, device=dev) for sh in
                 ((o, v), (o, o, v, v), (o, o, o, v, v, v))]
    # the split plan as timed (accumulating statements K-concatenated), and the same
    # plan with one GEMM per statement for comparison
    unmerged = args.precision + "_one_gemm_per_statement"
    plans = {"fp64": Engine(dsys, list_text=text),
             args.precision: Engine(dsys, list_text=text, precision=args.precision)}
    if args.precision != "fp64" and not suite:
        plans[unmerged] = Engine(dsys, list_text=text, precision=args.precision, kconcat=False)
    out = {}
    t_tune = None
    mp = plans[args.precision]
    if args.load_tune and not suite:
        for k, bn, sk, red in json.load(open(args.load_tune)):
            cc.cc_plan_set_gemm_config(mp.plan, k, bn, sk, red)
    elif not args.no_tune:
        # GEMM configurations of the mixed plans picked by timing (cc_plan_autotune)
        tt = time.perf_counter()
        for nm in (args.precision, unmerged):
            if nm in plans and nm != "fp64":
                plans[nm].autotune(*z()[:2], reps=2, stream=stream, t3=z()[2])
                plans[nm].release()
            if nm == args.precision:
                torch.cuda.synchronize()
                t_tune = time.perf_counter() - tt
        torch.cuda.synchronize()
    if args.save_tune and rank == 0 and not suite:
        json.dump([[k, st.get("bn", 0), st["splitk"], st.get("red", 0)] for k, st in
                   enumerate(mp.plan.describe()["steps"]) if st.get("configs")], open(args.save_tune, "w"))
    for name, eng in plans.items():
        t1, t2, t3 = z()
        sol = Solver(eng)
        nsteps = args.steps if name != "fp64" or not suite else 1
        sol.solve(t1, t2, t3=t3, max_iter=args.warmup if name != "fp64" or not suite else 1, tol=0.0,
                  stream=stream)
        cc.cc_plan_profile_enable(eng.plan, True)
        n0 = cc.cc_plan_launch_count(eng.plan)
        torch.cuda.synchronize()
        barrier(world)
        with Clocks(local) as clk:
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            sol.solve(t1, t2, t3=t3, max_iter=nsteps, tol=0.0, resume=True, stream=stream)
            e1.record(stream)
            torch.cuda.synchronize()
        dt = max_over_ranks(e0.elapsed_time(e1) / 1e3, world)
        ms_step, ms_kernel, calls = cc.cc_plan_profile_read(eng.plan)
        cc.cc_plan_profile_enable(eng.plan, False)
        desc = eng.plan.describe()
        steps = desc["steps"]
        # the o^3 v^5 terms: the GEMM steps of that size and their statements' epilogues
        big = {s_["stmt"] for s_ in steps if s_["kind"].startswith("gemm") and s_.get("flops", 0) >= o ** 3 * v ** 5}
        t_big = sum(ms_step[k] for k, s_ in enumerate(steps) if s_["stmt"] in big) / calls / 1e3
        k_dom = max(range(len(ms_kernel)), key=lambda k: ms_kernel[k])
        st = steps[k_dom]
        t_k = ms_kernel[k_dom] / calls / 1e3
        # share of the iteration's kernel time on the tensor cores
        t_all = sum(ms_kernel) / calls / 1e3
        t_tc = sum(ms_kernel[k] for k, s_ in enumerate(steps) if s_["kind"] == "gemm_bf16split") / calls / 1e3
        out[name] = {"s_per_iter": dt / nsteps, "tflops": world * eng.plan.flops * nsteps / dt / 1e12,
                     "steps": len(steps), "merged_steps": sum(1 for s_ in steps if "stmts" in s_),
                     "o3v5_s_per_iter": t_big, "o3v5_statements": len(big),
                     "launches": cc.cc_plan_launch_count(eng.plan) - n0,
                     "tensor_core_share_of_step_time": t_tc / t_all if t_all > 0 else None,
                     "dominant": {"kernel": st["note"], "kind": st["kind"], "ms_per_launch": t_k * 1e3,
                                  "fp64_equiv_tflops": st.get("flops", 0) / t_k / 1e12,
                                  "shape": [st.get("M"), st.get("N"), st.get("K")]},
                     "clocks": clk.summary()}
        if st["kind"] == "gemm_bf16split":
            ach = st["products"] * 2.0 * st["M"] * st["N"] * st["K"] / t_k / 1e12
            out[name]["roofline"] = {"bound": "tensor", "achieved": ach, "peak": pk["bf16_tflops"],
                                     "unit": "TFLOP/s", "frac": ach / pk["bf16_tflops"], "traffic": None,
                                     "kernel": "tc_gemm (" + st["note"] + ")",
                                     "peak_kind": f"{pk_kind} bf16 burst"}
        del sol, t1, t2, t3
        torch.cuda.empty_cache()
    # time to |R| < 1e-7: FP64 alone, the split route alone, and the accurate split route with
    # FP64 defect correction
    tts = {}
    if not args.no_tts:
        acc = Engine(dsys, list_text=text, precision="bf16x6")
        legs = [(args.precision + "_alone", plans[args.precision], None), ("bf16x6_refined", acc, plans["fp64"])]
        if not suite:
            legs.insert(0, ("fp64", plans["fp64"], None))
        for name, eng, ref in legs:
            t1, t2, t3 = z()
            sol = Solver(eng, refine=ref)
            torch.cuda.synchronize()
            g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            g0.record(stream)
            r = sol.solve(t1, t2, t3=t3, max_iter=80, tol=1e-7, stream=stream,
                          switch_tol=1e-6 if ref is not None else 0.0)
            g1.record(stream)
            torch.cuda.synchronize()
            tts[name] = {"s": g0.elapsed_time(g1) / 1e3, "iterations": r.iterations, "energy": r.energy,
                         "converged": r.converged}
            del sol, t1, t2, t3
            torch.cuda.empty_cache()
        ref_name = "fp64" if "fp64" in tts else "bf16x6_refined"
        for name in tts:
            if name != ref_name:
                tts[name]["delta_E_vs_" + ref_name] = abs(tts[name]["energy"] - tts[ref_name]["energy"])
        if "fp64" in tts:
            tts["speedup"] = tts["fp64"]["s"] / tts["bf16x6_refined"]["s"]
        tts["note"] = ("no oracle energy: a converged CCSDT oracle solve at o=8 v=64 is out of the "
                       "definition oracle's reach; the residual is pinned element by element instead")
    m = out[args.precision]
    line = {"metric": METRIC, "value": m["tflops"], "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": m["s_per_iter"] * 1e3, "s_per_iter": m["s_per_iter"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": f"{args.precision}: bf16 tensor-core products, fp32 accumulation, fp64 outputs/energy/DIIS",
            "data": "synthetic",
            "config": {"workload": WORKLOAD_T, "precision": args.precision, "list": "ccsdt (generated)",
                       "flops_per_iter": plans["fp64"].plan.flops, "replicas": world,
                       "l2": "inputs larger than L2 (T3 1.07 GB)", "autotune_s": t_tune},
            "roofline": m.get("roofline"), "gpu_launches": m["launches"], "clocks": m["clocks"],
            "plans": out, "tts": tts}
    if cpu is not None:
        line["cpu_baseline"] = cpu
    return line


LADDER_TEXT = "R2[ijab] = 0.5 T2[ijef] * V[abef]"


def run_ladder(args, world, rank, local):
    """The particle ladder R2 = 1/2 sum_ef t_ij^ef <ab||ef> alone (Eq. 2's
    o^2 v^4 term, one split-route GEMM step): the dominant kernel of the CCSD
    iteration in isolation, at a size (--ladder-size o,v) where a profiler
    capture of every metric ends quickly."""
    import torch

    import ccinputs
    import paper_2409_06759_b300 as cc
    from paper_2409_06759_b300.engine import DeviceSystem, Engine

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    o, v = (int(x) for x in args.ladder_size.split(","))
    pk, pk_kind = peaks()
    dsys = DeviceSystem.from_system(ccinputs.make_system(o=o, v=v, L=120, seed=0), device=dev)
    eng = Engine(dsys, list_text=LADDER_TEXT, precision=args.precision)
    a1, a2 = ccinputs.random_amplitudes(o, v, seed=0)
    t1 = torch.tensor(a1, device=dev)
    t2 = torch.tensor(a2, device=dev)
    r1, r2 = torch.empty_like(t1), torch.empty_like(t2)
    stream = torch.cuda.current_stream(dev)
    for _ in range(args.warmup):
        eng.residual(t1, t2, r1, r2, stream=stream)
    cc.cc_plan_profile_enable(eng.plan, True)
    n0 = cc.cc_plan_launch_count(eng.plan)
    torch.cuda.synchronize()
    barrier(world)
    with Clocks(local) as clk:
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            eng.residual(t1, t2, r1, r2, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
    dt = max_over_ranks(e0.elapsed_time(e1) / 1e3, world)
    ms_step, ms_kernel, calls = cc.cc_plan_profile_read(eng.plan)
    steps = eng.plan.describe()["steps"]
    k = next(i for i, st in enumerate(steps) if st["kind"].startswith("gemm"))
    st = steps[k]
    t_k = ms_kernel[k] / calls / 1e3
    split = st["kind"] == "gemm_bf16split"
    tflop = (st["products"] if split else 1) * 2.0 * st["M"] * st["N"] * st["K"]
    ach = tflop / t_k / 1e12
    value = world * eng.plan.flops * args.steps / dt / 1e12
    if not split:
        fpk = fp64_peak_live(torch)
    return {"metric": "particle-ladder contraction TFLOP/s on 1 B300", "value": value, "unit": "TFLOP/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": (f"{args.precision}: bf16 tensor-core products, fp32 accumulation, fp64 output" if split
                      else "fp64"),
            "data": "synthetic",
            "config": {"workload": f"particle ladder {LADDER_TEXT} o={o} v={v} L=120 seed=0",
                       "gemm_shape": [st["M"], st["N"], st["K"]], "tile_width": st.get("bn"),
                       "l2": "operands larger than L2 at o>=20 v>=100 (<ab||ef> planes >= 400 MB)"},
            "roofline": {"bound": "tensor", "achieved": ach, "peak": pk["bf16_tflops"], "unit": "TFLOP/s",
                         "frac": ach / pk["bf16_tflops"], "traffic": None,
                         "kernel": "tc_gemm_persistent_kernel (" + st["note"] + ")", "ms_per_launch": t_k * 1e3,
                         "peak_kind": f"{pk_kind} bf16 burst (tensor-pipe flops = {st['products']} products x 2MNK)"}
            if split else
            {"bound": "fp64", "achieved": ach, "peak": fpk, "unit": "TFLOP/s", "frac": ach / fpk, "traffic": None,
             "kernel": "gemm_f64_kernel (" + st["note"] + ")", "ms_per_launch": t_k * 1e3,
             "peak_kind": "measured live: cuBLAS DGEMM 4096^3 best of 3"},
            "gpu_launches": cc.cc_plan_launch_count(eng.plan) - n0, "clocks": clk.summary()}


# ---------------------------------------------------------------- batched
def run_batched(args, world, rank, local, suite=False):
    """64 independent CCSD systems of uneven size solved together
    (cc_solve_batched) to |R| < 1e-8: aggregate TFLOP/s of the FP64 and the
    split-bf16 plans, per-system |dE| against the oracle's solves, and the same
    systems solved one after another for comparison."""
    import torch

    import ccinputs
    import paper_2409_06759_b300 as cc
    from paper_2409_06759_b300.engine import BatchSolver, DeviceSystem, Engine, Solver

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    sizes = ccinputs.batched_sizes(64, seed=0)
    if args.batched_quick and args.batched_count:
        sizes = sizes[:args.batched_count]          # profiler captures on a smaller device footprint
    sysl = [ccinputs.make_system(o, v, L=120, seed=sd) for o, v, sd in sizes]
    dsys = [DeviceSystem.from_system(s, device=dev) for s in sysl]
    stream = torch.cuda.current_stream(dev)
    zeros = lambda s: (torch.zeros(s.o, s.v, dtype=torch.float64, device=dev),
                       torch.zeros(s.o, s.o, s.v, s.v, dtype=torch.float64, device=dev))
    oracle_e = None
    if os.path.exists(ORACLE_CACHE):
        with open(ORACLE_CACHE) as f:
            ent = json.load(f).get("ccsd_batched64_L120_seed0_f64")
        if ent:
            oracle_e = [x["energy"] for x in ent["systems"]]
    out = {}
    K = max(args.steps, 2) * 2

    def timed(solver, iters, tol):
        amps = [zeros(s) for s in sysl]
        torch.cuda.synchronize()
        barrier(world)
        g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        g0.record(stream)
        st, res = solver.solve(amps, max_iter=iters, tol=tol, stream=stream)
        g1.record(stream)
        torch.cuda.synchronize()
        return max_over_ranks(g0.elapsed_time(g1) / 1e3, world), res

    # bf16x3_grouped: plans with uniform steps, so cc_solve_batched runs the batch as
    # one grouped launch per step (the other variants: one graph branch per system)
    variants = (("fp64", "ccsd", "fp64"), ("bf16x3", "ccsd_vvvv", "bf16x3"), ("bf16x3_grouped", "ccsd_vvvv", "bf16x3"),
                ("bf16x6", "ccsd_vvvv", "bf16x6"))
    if args.batched_quick:
        # profiler captures: the headline (grouped, uniform-step bf16x3) plans, three
        # iterations of cc_solve_batched
        engs = [Engine(d, list_name="ccsd_vvvv", precision="bf16x3", uniform_steps=True) for d in dsys]
        t2, res = timed(BatchSolver(engs), 3, 0.0)
        return {"metric": "batched quick run (profiler capture)", "value": None, "unit": "s",
                "ms_3_iterations": t2 * 1e3, "launches": sum(cc.cc_plan_launch_count(e.plan) for e in engs)}
    with Clocks(local) as clk:
        for name, lst, prec in variants:
            grouped = name.endswith("_grouped")
            engs = [Engine(d, list_name=lst, precision=prec, uniform_steps=grouped) for d in dsys]
            flops = [e.plan.flops for e in engs]
            t_tune = time.perf_counter()
            if not grouped:                                # (grouped launches pick their own tiles)
                for e_, s_ in zip(engs, sysl):             # tile widths and split-K picked by timing
                    e_.autotune(*zeros(s_), reps=2, stream=stream)
                    e_.release()
            t_tune = time.perf_counter() - t_tune
            solver = BatchSolver(engs)
            timed(solver, 2, 0.0)                          # warm-up
            # steady state: (2 + K) minus 2 iterations, each system's own iteration counts
            n0 = sum(cc.cc_plan_launch_count(e.plan) for e in engs)
            ta, ra = timed(solver, 2, 0.0)
            n1 = sum(cc.cc_plan_launch_count(e.plan) for e in engs)
            tb, rb = timed(solver, 2 + K, 0.0)
            n2 = sum(cc.cc_plan_launch_count(e.plan) for e in engs)
            work = sum(f * (b.iterations - a.iterations) for f, a, b in zip(flops, ra, rb))
            steady = (tb - ta)
            # the whole solve to |R| < 1e-8 (setup included: static caches, graph capture)
            tts, res = timed(solver, 60, 1e-8)
            out[name] = {"steady_s_per_iter": steady / K, "steady_tflops": world * work / steady / 1e12,
                         "steady_launches_per_iter": ((n2 - n1) - (n1 - n0)) / K,
                         "solve_s": tts, "solve_tflops": world * sum(f * r.iterations for f, r in zip(flops, res))
                         / tts / 1e12, "converged": sum(r.converged for r in res),
                         "iterations": [r.iterations for r in res], "energies": [r.energy for r in res],
                         "autotune_s": t_tune}
            del solver, engs
            torch.cuda.empty_cache()
        # the FP64 systems one after another (single-system cc_solve), for comparison
        t_seq = 0.0
        if not suite:
            for d, s in zip(dsys, sysl):
                e = Engine(d, list_name="ccsd")
                a1, a2 = zeros(s)
                g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                g0.record(stream)
                Solver(e).solve(a1, a2, max_iter=60, tol=1e-8, stream=stream)
                g1.record(stream)
                torch.cuda.synchronize()
                t_seq += g0.elapsed_time(g1) / 1e3
    ef = out["fp64"]["energies"]
    for name, _, _ in variants:
        if name != "fp64":
            out[name]["max_abs_dE_vs_fp64"] = max(abs(a - b) for a, b in zip(out[name]["energies"], ef))
        if oracle_e is not None:
            out[name]["max_abs_dE_vs_oracle"] = max(abs(a - b) for a, b in zip(out[name]["energies"], oracle_e))
    for v_ in out.values():
        del v_["energies"]
    head = "bf16x3_grouped"
    m = out[head]
    line = {"metric": METRIC, "value": m["steady_tflops"], "unit": "TFLOP/s", "n_gpus": world, "steps": K,
            "warmup": 2, "ms_per_step": m["steady_s_per_iter"] * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None,
            "dtype": "bf16x3: bf16 tensor-core products, fp32 accumulation, fp64 outputs/energy/DIIS",
            "data": "synthetic",
            "config": {"workload": WORKLOAD_B, "step": "one batched iteration of all 64 systems (grouped launches, "
                       "one per plan step for the whole batch, captured as one graph + batched updates); steady "
                       "state = (2+K)-iteration call minus 2-iteration call", "headline_variant": head,
                       "systems": len(sizes), "sizes": [[o, v] for o, v, _ in sizes]},
            "roofline": None, "gpu_launches": int(m["steady_launches_per_iter"] * K), "clocks": clk.summary(),
            "variants": out, "oracle": "baseline/oracle_cache.json (cc_blocks.ccsd_solve per system)"
            if oracle_e is not None else None}
    if not suite:
        line["fp64_sequential_solve_s"] = t_seq
        line["batching_speedup_fp64_solve"] = t_seq / out["fp64"]["solve_s"]
    return line


def compact(line, keys):
    return {k: line[k] for k in keys if k in line}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="bf16x3", choices=["bf16x3", "bf16x6", "fp64"],
                    help="precision of the timed plan (fp64: the FP64 route, e.g. for profiler captures)")
    ap.add_argument("--size", default=None, help="o,v of the CCSD workload instead of o=40 v=200 (profiler "
                    "captures of the iteration's kernels on a smaller case)")
    ap.add_argument("--small", action="store_true", help="o=10 v=40 instead of o=40 v=200")
    ap.add_argument("--no-tts", action="store_true", help="skip the time-to-solution legs")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-baseline leg")
    ap.add_argument("--no-suite", action="store_true", help="skip the complex128, CCSDT and batched results")
    ap.add_argument("--dtype", default="f64", choices=["f64", "c128"])
    ap.add_argument("--no-tune", action="store_true", help="skip cc_plan_autotune on the timed plan")
    ap.add_argument("--save-tune", default=None, help="write the timed plan's GEMM configurations (JSON)")
    ap.add_argument("--load-tune", default=None, help="set the timed plan's GEMM configurations from a file "
                    "written by --save-tune instead of autotuning")
    ap.add_argument("--packed", action="store_true",
                    help="lists with packed index pairs (ladder over e<f; flops counted packed)")
    ap.add_argument("--workload", default="ccsd", choices=["ccsd", "ccsdt", "batched", "ladder"],
                    help="ccsdt: the o=8 v=64 CCSDT workload (generated list); batched: 64 uneven CCSD systems; "
                         "ladder: the particle-ladder contraction alone (profiler captures)")
    ap.add_argument("--ladder-size", default="20,100", help="o,v of --workload ladder")
    ap.add_argument("--batched-count", type=int, default=0,
                    help="--batched-quick: the first N of the 64 systems (profiler captures)")
    ap.add_argument("--batched-quick", action="store_true",
                    help="--workload batched: bf16x3 only, untuned, one two-iteration solve (profiler captures)")
    ap.add_argument("--cpu-leg", default=None, choices=["small"], help=argparse.SUPPRESS)
    args = ap.parse_args()
    if args.cpu_leg == "small":
        cpu_leg_small()
        return
    world, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, world, rank)
        return
    if args.workload != "ccsd":
        line = {"ccsdt": run_ccsdt, "batched": run_batched, "ladder": run_ladder}[args.workload](args, world, rank,
                                                                                              local)
    else:
        # the oracle's host legs run before any GPU work (rank 0, N = 1 only)
        cpu = None
        if rank == 0 and world == 1 and not args.no_cpu:
            o, v = (10, 40) if args.small else (40, 200)
            small = cpu_small_both()
            cpu = cpu_baseline(o, v, PLAN_FLOPS[("ccsd_vvvv", o, v, args.dtype)], complex_=args.dtype == "c128",
                               small=small)
        line = run_ccsd(args, world, rank, local, dtype=args.dtype, cpu=cpu)
        if world == 1 and not args.no_suite and args.dtype == "f64" and not args.small and not args.packed \
                and not args.size:
            import torch
            torch.cuda.empty_cache()
            c = run_ccsd(args, world, rank, local, dtype="c128", suite=True)
            line["c128"] = compact(c, ("value", "s_per_iter", "roofline", "e2e", "tts", "accuracy", "gpu_launches"))
            line["c128"]["workload"] = c["config"]["workload"]
            del c
            torch.cuda.empty_cache()
            t = run_ccsdt(args, world, rank, local, suite=True)
            line["ccsdt"] = compact(t, ("value", "s_per_iter", "roofline", "plans", "tts", "gpu_launches"))
            line["ccsdt"]["workload"] = WORKLOAD_T
            torch.cuda.empty_cache()
            b = run_batched(args, world, rank, local, suite=True)
            line["batched"] = compact(b, ("value", "ms_per_step", "variants", "oracle", "gpu_launches"))
            line["batched"]["workload"] = WORKLOAD_B
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
