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


# ------------------------------------------------------------------ error bounds
U32 = 2.0 ** -24
U64 = 2.0 ** -53


def route_constants(describe: dict, use_splitk: bool = True) -> dict:
    """Relative rounding constant c of each statement (ordinal in the list text)
    from a plan description: a statement whose contraction runs on a route with
    constant c has |err| <= c * |factor| * sum_k |a_ik||b_kj| per output element
    of its plain contraction (before its permutation operators).

    * split bf16 on tensor cores, FP32 accumulation of K' = K / splitk terms:
      two planes (3 products): 3*2^-16 + K'*2^-24 (dropped lo*lo product and
      plane rounding, then the first-order worst case of FP32 accumulation);
      three planes (6 products, accumulators drained into float-float every
      128 terms): 3*2^-24 + min(K', 128)*2^-24;
    * FP32 arithmetic on FP64 data: (3 + K)*2^-24 (operand and product
      rounding, accumulation);
    * FP64 routes: (2 + K)*2^-53; copies, permutes and antisymmetrisers: 2^-52.
    Complex statements run as real GEMMs of doubled K (4M embedding), so K
    doubles.  A statement with several steps takes the largest constant.
    use_splitk=False takes K' = K (the bound of every split-K candidate).
    A K-concatenated step (several accumulating statements summed in one GEMM,
    its "stmts") gives each member the constant of the whole K: the GEMM's
    accumulation error is bounded by that constant times the sum over all
    members of |factor| sum_k |a||b|, which is the sum of the members' bounds."""
    cplx = describe.get("dtype") == 1
    out = {}
    for st in describe["steps"]:
        k = st.get("K", 1) * (2 if cplx else 1)
        kp = max(1, -(-k // max(1, st.get("splitk", 1)))) if use_splitk else k
        kind = st["kind"]
        if kind == "gemm_bf16split":
            if st.get("products", 3) >= 6:
                c = 3 * U32 + min(kp, 128) * U32
            else:
                c = 3 * 2.0 ** -16 + kp * U32
        elif kind.endswith("f32"):
            c = (3 + k) * U32
        elif kind.startswith("gemm") or kind.startswith("gemv"):
            c = (2 + k) * U64
        else:
            c = 2 * U64
        for si in st.get("stmts", [st["stmt"]]):
            out[si] = max(out.get(si, 0.0), c)
    return out


class BlockV:
    """<pq||rs> by space pattern, each block built once from B by the oracle's
    block routine: stands in for the full n^4 tensor in run_list_bounds at
    sizes where that tensor does not fit."""

    def __init__(self, o, v, B):
        from oracle import cc_blocks
        self.o, self.v, self.B, self._mk, self._c = o, v, np.ascontiguousarray(B), cc_blocks._antisym_block, {}

    def __getitem__(self, key):
        sp = "".join("o" if s.start == 0 else "v" for s in key)
        if sp not in self._c:
            self._c[sp] = self._mk(self.B, self.o, sp)
        return self._c[sp]


def run_list_bounds(text: str, o: int, v: int, eps, V, t1, t2, consts, t3=None, magnitudes=False):
    """The list's values (as run_list) and first-order element-wise bounds on
    the error of an execution whose statements round with the relative
    constants ``consts`` (one dict per bound, statement ordinal -> c; see
    route_constants).  Returns (values, bounds): values = (R1, R2[, R3]),
    bounds = [(E1, E2[, E3]) per constant dict].  Inputs (T, V) are exact; an
    intermediate carries its bound into every later statement that reads it:
        E(out) += |factor| * sum_P [ c * (|A| |B|) + E_A |B| + |A| E_B ].
    magnitudes=True never forms the signed values: every tensor is replaced by a
    bound on its moduli (inputs by their moduli, an intermediate by
    |factor| sum_P |A| |B| of its statements), which keeps the bounds rigorous
    (looser where the intermediates cancel) at the cost of one real
    contraction per statement; the returned values are then those moduli
    bounds."""
    n = o + v
    sl = {"o": slice(0, o), "v": slice(o, n)}
    nb = len(consts)
    env, out, err = {}, {}, {}
    ein = lambda spec, *x: np.einsum(spec, *x, optimize=True)

    def amp_order(letters):
        return [l for l in letters if _space(l) == "o"] + [l for l in letters if _space(l) == "v"]

    if magnitudes:
        t1, t2 = np.abs(t1), np.abs(t2)
        t3 = None if t3 is None else np.abs(t3)

    def get(name, letters):
        if name in ("T1", "T2", "T3", "t", "T"):
            return {2: t1, 4: t2, 6: t3}[len(letters)], amp_order(letters), None
        if name == "V":
            sp = [_space(l) for l in letters]
            blk = V[sl[sp[0]], sl[sp[1]], sl[sp[2]], sl[sp[3]]]
            return (np.abs(blk) if magnitudes else blk), list(letters), None
        return env[name], list(letters), err[name]

    stmt = -1
    for raw in text.splitlines():
        line = raw.split("#")[0].strip()
        if not line:
            continue
        stmt += 1
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
        letters = sorted(set(sum((l for _, l, _ in ops), [])) | set(olet_store))
        sym = {l: chr(ord("A") + k) for k, l in enumerate(letters)}
        spec = ",".join("".join(sym[l] for l in lab) for _, lab, _ in ops) + "->" + "".join(sym[l] for l in olet_store)
        arrs = [a for a, _, _ in ops]
        if magnitudes:
            fac = abs(fac)
            absx = ein(spec, *arrs)
            x = absx
        else:
            x = ein(spec, *arrs)
            absx = ein(spec, *[np.abs(a) for a in arrs])
        ex = []
        for q in range(nb):
            e = consts[q].get(stmt, 0.0) * absx
            for k, (a, _, ea) in enumerate(ops):
                if ea is not None:
                    e = e + ein(spec, *[ea[q] if kk == k else np.abs(b) for kk, (b, _, _) in enumerate(ops)])
            ex.append(e)
        val = np.zeros_like(x)
        ev = [np.zeros(x.shape) for _ in range(nb)]
        for s, mp in _expand_perm(perms):
            val = val + (1.0 if magnitudes else s) * _relabel(x, olet_store, mp)
            for q in range(nb):
                ev[q] = ev[q] + _relabel(ex[q], olet_store, mp)
        val = fac * val
        ev = [abs(fac) * e for e in ev]
        tgt = out if oname.startswith("R") else env
        if op == "=":
            tgt[oname] = val.copy()
            err[oname] = ev
        else:
            tgt[oname] = tgt.get(oname, np.zeros_like(val)) + (val if op == "+=" or magnitudes else -val)
            old = err.get(oname, [0.0] * nb)
            err[oname] = [a + b for a, b in zip(old, ev)]
        del x, absx, ex
    eo, ev_ = eps[:o], eps[o:]
    d1 = eo[:, None] - ev_[None, :]
    d2 = eo[:, None, None, None] + eo[None, :, None, None] - ev_[None, None, :, None] - ev_[None, None, None, :]
    if magnitudes:
        d1, d2 = -np.abs(d1), -np.abs(d2)
    r1 = out["R1"] - d1 * t1 if "R1" in out else np.zeros((o, v))
    r2 = out["R2"] - d2 * t2 if "R2" in out else np.zeros((o, o, v, v))
    e1 = [err["R1"][q] if "R1" in err else np.zeros((o, v)) for q in range(nb)]
    e2 = [err["R2"][q] if "R2" in err else np.zeros((o, o, v, v)) for q in range(nb)]
    if t3 is None:
        return (r1, r2), [(e1[q], e2[q]) for q in range(nb)]
    d3 = (eo[:, None, None, None, None, None] + eo[None, :, None, None, None, None]
          + eo[None, None, :, None, None, None] - ev_[None, None, None, :, None, None]
          - ev_[None, None, None, None, :, None] - ev_[None, None, None, None, None, :])
    r3 = out["R3"] - d3 * t3 if "R3" in out else np.zeros((o, o, o, v, v, v))
    e3 = [err["R3"][q] if "R3" in err else np.zeros((o, o, o, v, v, v)) for q in range(nb)]
    return (r1, r2, r3), [(e1[q], e2[q], e3[q]) for q in range(nb)]
