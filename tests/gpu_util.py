"""Shared helpers of the GPU tests (inputs from ccinputs, expected values from oracle/)."""
import numpy as np
import torch

import ccinputs
import oracle

DEV = torch.device("cuda:0")


def small_case(o, v, seed, L=6, scale=6.0, tscale=0.05):
    s = ccinputs.make_system(o, v, L=L, seed=seed)
    B = s.B * scale
    t1, t2 = ccinputs.random_amplitudes(o, v, seed=seed, scale1=tscale, scale2=tscale)
    return s, B, t1, t2


def to_dev(x):
    return torch.tensor(np.ascontiguousarray(x), dtype=torch.float64, device=DEV)


def oracle_V(o, v, B):
    return oracle.antisym_integrals(o, v, np.ascontiguousarray(B))


def block_slices(V, o):
    n = V.shape[0]
    sl = {"o": slice(0, o), "v": slice(o, n)}
    return {nm: V[sl[nm[0]], sl[nm[1]], sl[nm[2]], sl[nm[3]]] for nm in
            ("oooo", "ooov", "oovv", "ovov", "ovvv", "vvvv")}


def assert_elementwise(got, want, bound, slack=1e-13, what=""):
    """|got - want| <= bound + slack * max|want| for every element of every
    (got, want, bound) triple; the message names the worst element."""
    for k, (g, w, b) in enumerate(zip(got, want, bound)):
        g = g.cpu().numpy() if hasattr(g, "cpu") else np.asarray(g)
        w, b = np.asarray(w), np.asarray(b)
        assert g.shape == w.shape == b.shape, (what, k, g.shape, w.shape, b.shape)
        err = np.abs(g - w)
        lim = b + slack * max(np.abs(w).max(), 1e-300)
        bad = err > lim
        if bad.any():
            q = np.unravel_index(np.argmax(err - lim), err.shape)
            raise AssertionError(f"{what} output {k}: {int(bad.sum())} of {err.size} elements outside the bound; "
                                 f"worst at {q}: |err| {err[q]:.3e} > {lim[q]:.3e} (value {w[q]:.3e})")


def list_bounds(text, o, v, eps, V, t1, t2, plans, t3=None, use_splitk=True):
    """Values of the list's einsum reading and, for each plan, the element-wise
    error bound of its routes (list_exec.route_constants); complex moduli
    double the bound (each real component is bounded by the real rule)."""
    import list_exec
    cplx = np.iscomplexobj(t2)
    consts = []
    for p in plans:
        c = list_exec.route_constants(p.describe(), use_splitk=use_splitk)
        consts.append({k: (2.0 * x if cplx else x) for k, x in c.items()})
    vals, bounds = list_exec.run_list_bounds(text, o, v, eps, V, t1, t2, consts, t3=t3)
    return vals, bounds
