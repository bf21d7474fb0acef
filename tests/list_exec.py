"""numpy.einsum executor of a contraction list (test helper).

An independent reading of the list grammar (one binary Contraction per line,
Sec. II C) used to pin the shipped CCSD lists against the oracle on the CPU:
every statement is evaluated with ``numpy.einsum`` on the full antisymmetrised
integral tensor, so a wrong factor, sign, index or permutation operator in a
list shows up as a residual mismatch.
"""
from __future__ import annotations

import re

import numpy as np

_REF = re.compile(r"([A-Za-z_][A-Za-z0-9_]*)((?:\[[^\]]*\])+)")
_TOK = re.compile(r"[a-z][0-9]*")


def _space(tok: str) -> str:
    if len(tok) == 1:
        if "a" <= tok <= "h":
            return "v"
        if "i" <= tok <= "n":
            return "o"
    elif tok[0] == "p":
        return "v"
    elif tok[0] == "h":
        return "o"
    raise ValueError(f"bad index {tok}")


def _letters(brackets: str):
    return _TOK.findall(brackets.replace("[", " ").replace("]", " "))


def _expand_perm(ps):
    terms = [(1.0, {})]
    for letters, slash in ps:
        ops = [(1.0, {})]
        if not slash:
            p, q = letters
            ops.append((-1.0, {p: q, q: p}))
        else:
            for q in letters[1:]:
                ops.append((-1.0, {letters[0]: q, q: letters[0]}))
        new = []
        for s1, m1 in terms:
            for s2, m2 in ops:
                comb = {}
                for l in set(m1) | set(m2):
                    x = m1.get(m2.get(l, l), m2.get(l, l))
                    if x != l:
                        comb[l] = x
                new.append((s1 * s2, comb))
        terms = new
    return terms


def _relabel(x, labels, mp):
    """(sigma x)[idx] = x[sigma idx], (sigma idx)(l) = idx(mp(l)): x's axis for
    letter l takes the output axis of letter mp(l)."""
    a = [labels.index(mp.get(l, l)) for l in labels]
    return np.transpose(x, np.argsort(a))


def run_list(text: str, o: int, v: int, eps, V, t1, t2, t3=None):
    """Returns (R1, R2) -- or (R1, R2, R3) when t3 is given -- including the
    -D*t terms, like the engine."""
    n = o + v
    sl = {"o": slice(0, o), "v": slice(o, n)}
    env, out = {}, {}

    def amp_order(letters):
        return [l for l in letters if _space(l) == "o"] + [l for l in letters if _space(l) == "v"]

    def get(name, letters):
        if name in ("T1", "T2", "T3", "t", "T"):
            return {2: t1, 4: t2, 6: t3}[len(letters)], amp_order(letters)
        if name == "V":
            sp = [_space(l) for l in letters]
            return V[sl[sp[0]], sl[sp[1]], sl[sp[2]], sl[sp[3]]], list(letters)
        return env[name], list(letters)

    for raw in text.splitlines():
        line = raw.split("#")[0].strip()
        if not line:
            continue
        m = re.match(r"\s*([A-Za-z_][A-Za-z0-9_]*)((?:\[[^\]]*\])+)\s*(\+=|-=|=)\s*(.*)$", line)
        oname, obr, op, rest = m.groups()
        olet = _letters(obr)
        fac = 1.0
        mf = re.match(r"\s*([+-]?\s*(?:\d+\.?\d*|\.\d+)(?:[eE][+-]?\d+)?)(?:\s*/\s*(\d+))?\s*(.*)$", rest)
        if mf:
            fac = float(mf.group(1).replace(" ", ""))
            if mf.group(2):
                fac /= float(mf.group(2))
            rest = mf.group(3)
        elif rest.strip().startswith("-"):
            fac = -1.0
            rest = rest.strip()[1:]
        perms = []
        for pm in re.finditer(r"P\(([^)]*)\)", rest):
            body = pm.group(1)
            if "/" in body:
                a, b = body.split("/")
                perms.append((_TOK.findall(a) + _TOK.findall(b), True))
            else:
                perms.append((_TOK.findall(body), False))
        rest = re.sub(r"P\([^)]*\)", " ", rest)
        ops = [get(nm, _letters(br)) for nm, br in _REF.findall(rest)]
        olet_store = amp_order(olet) if oname.startswith("R") else olet
        letters = sorted(set(sum((l for _, l in ops), [])) | set(olet_store))
        sym = {l: chr(ord("A") + k) for k, l in enumerate(letters)}
        spec = ",".join("".join(sym[l] for l in lab) for _, lab in ops) + "->" + "".join(sym[l] for l in olet_store)
        x = np.einsum(spec, *[a for a, _ in ops])
        val = np.zeros_like(x)
        for s, mp in _expand_perm(perms):
            val = val + s * _relabel(x, olet_store, mp)
        val = fac * val
        tgt = out if oname.startswith("R") else env
        if op == "=":
            tgt[oname] = val.copy()
        elif op == "+=":
            tgt[oname] = tgt.get(oname, np.zeros_like(val)) + val
        else:
            tgt[oname] = tgt.get(oname, np.zeros_like(val)) - val
    # the engine adds -D*t to the residuals the list writes (and only to those)
    eo, ev = eps[:o], eps[o:]
    d1 = eo[:, None] - ev[None, :]
    d2 = eo[:, None, None, None] + eo[None, :, None, None] - ev[None, None, :, None] - ev[None, None, None, :]
    r1 = out["R1"] - d1 * t1 if "R1" in out else np.zeros((o, v))
    r2 = out["R2"] - d2 * t2 if "R2" in out else np.zeros((o, o, v, v))
    if t3 is None:
        return r1, r2
    d3 = (eo[:, None, None, None, None, None] + eo[None, :, None, None, None, None]
          + eo[None, None, :, None, None, None] - ev[None, None, None, :, None, None]
          - ev[None, None, None, None, :, None] - ev[None, None, None, None, None, :])
    r3 = out["R3"] - d3 * t3 if "R3" in out else np.zeros((o, o, o, v, v, v))
    return r1, r2, r3
