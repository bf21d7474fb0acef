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
