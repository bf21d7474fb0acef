"""Derivation of coupled-cluster residual equations as contraction lists.

This is the derivation step of arxiv 2409.06759 (Sec. II A-C): from the CC
equations <Phi_l| exp(-T) H_N exp(T) |Phi_0> = 0 (Eq. amp) to an ordered list
of binary contractions (the "Contraction" objects of Sec. II C) that the
planner executes.  The paper enumerates diagrams with the integer-string
scheme of Kallay and Surjan (Fig. algo:gen) and applies interpretation rules to
line graphs; this module reaches the same algebraic terms by enumerating Wick
contractions directly:

  * R_l = <Phi_l| (H_N exp(T))_C |Phi_0>: the bra string of level k,
    <Phi_0| i+ j+ .. b a, one Hamiltonian vertex (V = 1/4 <pq||rs> p+ q+ s r,
    or F = f_pq p+ q), and up to four cluster operators
    T_n = (1/n!)^2 t_{i..}^{a..} a+ .. i, each connected to the vertex;
  * every complete contraction (hole lines: creator left of annihilator,
    occupied; particle lines: annihilator left of creator, virtual) gives one
    signed product; the sign is (-1)^(crossings) of the pairing;
  * products are brought to a canonical form (antisymmetry of <pq||rs> within
    its bra and ket pairs and of t within its occupied and virtual sets,
    reordering of equal-rank amplitudes, dummy renaming) and summed exactly
    (fractions);
  * terms related by permutations of external indices are grouped into one
    term with permutation operators P(pq) / P(p/qr) (one "diagram");
  * each diagram is factorised into binary contractions (the constraint of
    Fig. algo:remove) in the order of least flops whose intermediates stay
    below a size cap.

The integrals keep the orientation the derivation gives them (no bra-ket
swap is used), so the lists hold for complex Hermitian integrals as written.

Usage:  python -m paper_2409_06759_b300.gen ccsdt > lists/ccsdt.txt
"""
from __future__ import annotations

import functools
import itertools
import sys
from fractions import Fraction
from math import factorial

OCC_EXT = "ijklmn"[:3]
VIR_EXT = "abc"


# ----------------------------------------------------------------- operators
class Op:
    """One creation/annihilation operator of the contraction string.
    space: 'o', 'v' or None (Hamiltonian indices: fixed by the contraction)."""
    __slots__ = ("grp", "slot", "cre", "space", "ext")

    def __init__(self, grp, slot, cre, space, ext=None):
        self.grp, self.slot, self.cre, self.space, self.ext = grp, slot, cre, space, ext


def bra_ops(k):
    """<Phi_0| i1+ .. ik+ ak .. a1 (the adjoint of a1+ .. ak+ ik .. i1 |Phi_0>)."""
    ops = [Op("bra", q, True, "o", OCC_EXT[q]) for q in range(k)]
    ops += [Op("bra", k + q, False, "v", VIR_EXT[q]) for q in reversed(range(k))]
    return ops


def ham_ops(kind):
    if kind == "V":   # 1/4 <pq||rs> p+ q+ s r: slots (p, q, r, s) = (0, 1, 2, 3)
        return [Op("H", 0, True, None), Op("H", 1, True, None), Op("H", 3, False, None), Op("H", 2, False, None)]
    return [Op("H", 0, True, None), Op("H", 1, False, None)]   # f_pq p+ q


def t_ops(g, n):
    """T_n = (1/n!)^2 t[i1..in][a1..an] a1+ .. an+ in .. i1: slots 0..n-1 occupied, n..2n-1 virtual."""
    ops = [Op(g, n + q, True, "v") for q in range(n)]
    ops += [Op(g, q, False, "o") for q in reversed(range(n))]
    return ops


def crossings(pairs):
    c = 0
    for a in range(len(pairs)):
        x1, y1 = pairs[a]
        for b in range(len(pairs)):
            x2, y2 = pairs[b]
            if x1 < x2 < y1 < y2:
                c += 1
    return c


def contractions(k, hkind, levels):
    """All complete contractions of <bra_k| H T_levels[0] T_levels[1] ..|0> in
    which every T is connected to H.  Yields (sign, H labels, [T labels])."""
    string = bra_ops(k) + ham_ops(hkind)
    for g, n in enumerate(levels):
        string += t_ops(g, n)
    pos = {id(op): p for p, op in enumerate(string)}
    hops = [op for op in string if op.grp == "H"]
    others = [op for op in string if op.grp != "H"]

    def partners(h):
        """(partner, space, is_bra) for a Hamiltonian operator."""
        out = []
        for x in others:
            if x.grp == "bra":
                # bra op is left of H: needs (bra ann vir, H cre) or (bra cre occ, H ann)
                if (h.cre and not x.cre and x.space == "v") or (not h.cre and x.cre and x.space == "o"):
                    out.append((x, x.space))
            else:
                # T op is right of H: (H cre occ, T ann occ) or (H ann vir, T cre vir)
                if (h.cre and not x.cre and x.space == "o") or (not h.cre and x.cre and x.space == "v"):
                    out.append((x, x.space))
        return out

    plist = [partners(h) for h in hops]
    nlev = len(levels)
    for choice in itertools.product(*plist):
        used = [x for x, _ in choice]
        if len({id(x) for x in used}) != len(used):
            continue
        connected = {x.grp for x in used if x.grp != "bra"}
        if len(connected) != nlev:
            continue
        uid = {id(x) for x in used}
        rb_o = [x for x in others if x.grp == "bra" and x.space == "o" and id(x) not in uid]
        rb_v = [x for x in others if x.grp == "bra" and x.space == "v" and id(x) not in uid]
        rt_o = [x for x in others if x.grp != "bra" and x.space == "o" and id(x) not in uid]
        rt_v = [x for x in others if x.grp != "bra" and x.space == "v" and id(x) not in uid]
        if len(rb_o) != len(rt_o) or len(rb_v) != len(rt_v):
            continue
        for po in itertools.permutations(rt_o):
            for pv in itertools.permutations(rt_v):
                pairs = []
                hl = [None] * len(hops)
                tl = [[None] * (2 * n) for n in levels]
                dummy = 0
                for h, (x, sp) in zip(hops, choice):
                    a, b = sorted((pos[id(h)], pos[id(x)]))
                    pairs.append((a, b))
                    if x.grp == "bra":
                        hl[h.slot] = x.ext
                    else:
                        lab = f"#{dummy}{sp}"
                        dummy += 1
                        hl[h.slot] = lab
                        tl[x.grp][x.slot] = lab
                for bx, tx in list(zip(rb_o, po)) + list(zip(rb_v, pv)):
                    pairs.append((pos[id(bx)], pos[id(tx)]))
                    tl[tx.grp][tx.slot] = bx.ext
                yield (-1) ** crossings(pairs), tuple(hl), [tuple(x) for x in tl]


# ------------------------------------------------------------ canonical form
def perm_sign(p):
    s, seen = 1, [False] * len(p)
    for i in range(len(p)):
        if not seen[i]:
            j, c = i, 0
            while not seen[j]:
                seen[j] = True
                j = p[j]
                c += 1
            if c % 2 == 0:
                s = -s
    return s


_PERMS = {n: [(p, perm_sign(p)) for p in itertools.permutations(range(n))] for n in range(5)}


def canonical(hkind, hl, tls):
    """(key, sign): a canonical relabelled form of the term and the sign that
    takes the term to it.

    For a fixed order of the amplitudes, every antisymmetric index group (the
    bra and ket pairs of <pq||rs>, the occupied and virtual sets of each t) is
    sorted: external letters first, by name; then dummies by the group at their
    other end.  Two dummies that tie connect the same two groups; their order
    in the amplitude's group is made to follow their order in the vertex's
    group.  Dummies are then renamed by first appearance.  The key is the
    smallest over the orders of equal-rank amplitudes.
    """
    levels = [len(t) // 2 for t in tls]
    nt = len(tls)
    hgroups = [(0, 1), (2, 3)] if hkind == "V" else [(0,), (1,)]
    # each dummy's endpoints: (vertex group, amplitude index, amplitude group)
    hpos = {}
    for gi, g in enumerate(hgroups):
        for slot in g:
            lab = hl[slot]
            if lab[0] == "#":
                hpos[lab] = gi
    tpos = {}
    for ti, t in enumerate(tls):
        n = len(t) // 2
        for q, lab in enumerate(t):
            if lab[0] == "#":
                tpos[lab] = (ti, 0 if q < n else 1)
    order = sorted(range(nt), key=lambda g: levels[g])
    groups = [list(g) for _, g in itertools.groupby(order, key=lambda g: levels[g])]
    best = None
    for orders in itertools.product(*[list(itertools.permutations(g)) for g in groups]):
        seq = [g for grp in orders for g in grp]
        rank = {ti: r for r, ti in enumerate(seq)}
        sign = 1
        hout = list(hl)
        for gi, g in enumerate(hgroups):
            labs = [hl[s_] for s_ in g]
            keyed = sorted(range(len(labs)), key=lambda q: (0, labs[q]) if labs[q][0] != "#"
                           else (1, rank[tpos[labs[q]][0]], labs[q][-1]))
            sign *= perm_sign(keyed)
            for q, s_ in enumerate(g):
                hout[s_] = labs[keyed[q]]
        # position of each dummy inside its vertex group after sorting (tie breaker)
        hrank = {}
        for gi, g in enumerate(hgroups):
            for q, s_ in enumerate(g):
                if hout[s_][0] == "#":
                    hrank[hout[s_]] = (gi, q)
        touts = []
        for ti in seq:
            t = tls[ti]
            n = len(t) // 2
            newt = []
            for part in (t[:n], t[n:]):
                keyed = sorted(range(len(part)), key=lambda q: (0, part[q]) if part[q][0] != "#"
                               else (1,) + hrank[part[q]])
                sign *= perm_sign(keyed)
                newt.extend(part[q] for q in keyed)
            touts.append(newt)
        ren = {}
        out = []
        for lab in hout + [x for t in touts for x in t]:
            if lab[0] == "#":
                if lab not in ren:
                    ren[lab] = f"#{len(ren):02d}{lab[-1]}"
                out.append(ren[lab])
            else:
                out.append(lab)
        key = (hkind, tuple(levels[g] for g in seq), tuple(out))
        if best is None or key < best[0]:
            best = (key, sign)
    return best


def canonical_brute(hkind, hl, tls):
    """Reference canonical form: the smallest key over the whole symmetry group
    (slow; used to check `canonical`)."""
    levels = [len(t) // 2 for t in tls]
    hvars = [((hl[0], hl[1], hl[2], hl[3]), 1), ((hl[1], hl[0], hl[2], hl[3]), -1),
             ((hl[0], hl[1], hl[3], hl[2]), -1), ((hl[1], hl[0], hl[3], hl[2]), 1)] if hkind == "V" else [(hl, 1)]
    tvars = []
    for t in tls:
        n = len(t) // 2
        vs = []
        for po, so in _PERMS[n]:
            for pv, sv in _PERMS[n]:
                vs.append((tuple(t[q] for q in po) + tuple(t[n + q] for q in pv), so * sv))
        tvars.append(vs)
    best = None
    # equal-rank amplitudes may be reordered: canonical order by rank, all orders within a rank
    order = sorted(range(len(tls)), key=lambda g: levels[g])
    groups = [list(g) for _, g in itertools.groupby(order, key=lambda g: levels[g])]
    for orders in itertools.product(*[list(itertools.permutations(g)) for g in groups]):
        seq = [g for grp in orders for g in grp]
        for hv, hs in hvars:
            for tv in itertools.product(*[tvars[g] for g in seq]):
                ren, nd = {}, 0
                labels = list(hv) + [lab for t, _ in tv for lab in t]
                out = []
                for lab in labels:
                    if lab.startswith("#"):
                        if lab not in ren:
                            ren[lab] = f"#{nd:02d}{lab[-1]}"
                            nd += 1
                        out.append(ren[lab])
                    else:
                        out.append(lab)
                key = (hkind, tuple(levels[g] for g in seq), tuple(out))
                if best is None or key < best[0]:
                    s = hs
                    for _, ts in tv:
                        s *= ts
                    best = (key, s)
    return best


def derive(k, ranks, hkinds=("V",)):
    """Canonical terms of R_k (k = 0: the energy) with cluster operators of the
    given ranks: {key: Fraction coefficient}, zero sums dropped."""
    terms = {}
    for hkind in hkinds:
        maxc = 4 if hkind == "V" else 2        # a vertex connects to at most this many operators
        for l in range(0, maxc + 1):
            for levels in itertools.combinations_with_replacement(sorted(ranks), l):
                # excitation balance: the vertex changes the level by -2..+2 (V), -1..+1 (F)
                exc = sum(levels)
                if abs(exc - k) > (2 if hkind == "V" else 1):
                    continue
                mult = Fraction(1)
                for n in set(levels):
                    mult /= factorial(levels.count(n))
                for n in levels:
                    mult /= factorial(n) ** 2
                hfac = Fraction(1, 4) if hkind == "V" else Fraction(1)
                for sign, hl, tls in contractions(k, hkind, list(levels)):
                    key, s = canonical(hkind, hl, tls)
                    terms[key] = terms.get(key, Fraction(0)) + hfac * mult * sign * s
    return {k_: c for k_, c in terms.items() if c != 0}


# ---------------------------------------------------- diagrams (P operators)
def relabel_key(key, mp):
    hkind, levels, labs = key
    return hkind, levels, tuple(mp.get(x, x) for x in labs)


def key_to_term(key):
    """Split a canonical key back into (hkind, H labels, [T labels])."""
    hkind, levels, labs = key
    nh = 4 if hkind == "V" else 2
    hl = labs[:nh]
    tls, p = [], nh
    for n in levels:
        tls.append(tuple(labs[p:p + 2 * n]))
        p += 2 * n
    return hkind, hl, tls


def _op_expansions(letters):
    """Permutation-operator choices over one set of external letters, with their
    expansion as signed relabellings (text, [(map, sign)])."""
    n = len(letters)
    out = [("", [({}, 1)])]
    if n >= 2:
        for p, q in itertools.combinations(letters, 2):
            out.append((f"P({p}{q})", [({}, 1), ({p: q, q: p}, -1)]))
    if n == 3:
        for d in letters:
            rest = [x for x in letters if x != d]
            exp = [({}, 1)] + [({d: r, r: d}, -1) for r in rest]
            out.append((f"P({d}/{''.join(rest)})", exp))
        # full antisymmetriser: P(i/jk) P(jk)
        d, r1, r2 = letters
        exp = []
        for mp1, s1 in [({}, 1), ({d: r1, r1: d}, -1), ({d: r2, r2: d}, -1)]:
            for mp2, s2 in [({}, 1), ({r1: r2, r2: r1}, -1)]:
                # composition: apply mp2 first, then mp1
                comp = {x: mp1.get(mp2.get(x, x), mp2.get(x, x)) for x in letters}
                exp.append(({x: y for x, y in comp.items() if x != y}, s1 * s2))
        out.append((f"P({d}/{r1}{r2}) P({r1}{r2})", exp))
    return out


def diagrams(k, terms):
    """Groups the terms of R_k into diagrams: [(coef, text_of_P_ops, key,
    nterms)], each standing for the sum over its P expansion (nterms signed
    relabellings) of sign * coef * term."""
    left = dict(terms)
    out = []
    occ_ops = _op_expansions(list(OCC_EXT[:k]))
    vir_ops = _op_expansions(list(VIR_EXT[:k]))
    catalogue = []
    for (to, eo), (tv, ev) in itertools.product(occ_ops, vir_ops):
        exp = [({**mo, **mv}, so * sv) for mo, so in eo for mv, sv in ev]
        catalogue.append(((to + " " + tv).strip(), exp))
    catalogue.sort(key=lambda c: -len(c[1]))
    while left:
        rep = min(left)
        c = left[rep]
        hk, hl, tls = key_to_term(rep)
        done = False
        for text, exp in catalogue:
            contrib = {}
            for mp, s in exp:
                hk2, l2, labs = relabel_key(rep, mp)
                kk, s2 = canonical(*key_to_term((hk2, l2, labs)))
                contrib[kk] = contrib.get(kk, Fraction(0)) + c * s * s2
            contrib = {x: y for x, y in contrib.items() if y != 0}
            if contrib and all(left.get(x) == y for x, y in contrib.items()):
                for x in contrib:
                    del left[x]
                out.append((c, text, rep, len(exp)))
                done = True
                break
        if not done:
            raise RuntimeError(f"no permutation operator covers the orbit of {rep}")
    return out


# ------------------------------------------------------------ factorisation
def tensor_text(name, labs):
    return name + "[" + "".join(labs) + "]"


def letter_space(lab):
    """Index space of a list letter: i..n and h<k> occupied, a..h and p<k> virtual."""
    if lab.startswith("#"):
        return lab[-1]
    if lab[0] in "ijklmn" or (lab[0] == "h" and len(lab) > 1):
        return "o"
    return "v"


def _trees(items):
    """Every sequence of pairwise contractions of the items (bushy trees included)."""
    if len(items) == 1:
        yield []
        return
    for x, y in itertools.combinations(range(len(items)), 2):
        node = ("@", items[x], items[y])
        rest = [items[q] for q in range(len(items)) if q not in (x, y)] + [node]
        for tail in _trees(rest):
            yield [(items[x], items[y], node)] + tail


class Factoriser:
    """Turns diagrams into binary contraction statements (least flops, with
    every intermediate at most `cap` elements)."""

    def __init__(self, o, v, cap):
        self.o, self.v, self.cap = o, v, cap
        self.lines = []
        self.nint = 0
        self.defs = {}      # signature -> intermediate name

    def size(self, labs):
        s = 1
        for x in labs:
            s *= self.o if letter_space(x) == "o" else self.v
        return s

    @staticmethod
    def num(f):
        return f"{f.numerator}" if f.denominator == 1 else f"{f.numerator}/{f.denominator}"

    def emit(self, k, coef, ptext, key, target=None, first=False):
        """Statements of one diagram.  target: write the unsymmetrised term into
        this accumulator instead of R_k (no P operators; '=' when first)."""
        hk, hl, tls = key_to_term(key)
        occ, vir = OCC_EXT[:k], VIR_EXT[:k]
        free_o = [c for c in "ijklmn" if c not in occ] + [f"h{q}" for q in range(1, 10)]
        free_v = [c for c in "abcdefg" if c not in vir] + [f"p{q}" for q in range(1, 10)]
        mp = {}
        for lab in list(hl) + [x for t in tls for x in t]:
            if lab.startswith("#") and lab not in mp:
                mp[lab] = free_o.pop(0) if lab[-1] == "o" else free_v.pop(0)
        tens = [("V" if hk == "V" else "F", tuple(mp.get(x, x) for x in hl))]
        tens += [("T%d" % (len(t) // 2), tuple(mp.get(x, x) for x in t)) for t in tls]
        out = tuple(occ) + tuple(vir)
        best = None
        for seq in _trees([("t", q) for q in range(len(tens))]):
            r = self._cost(tens, seq, out)
            if r is not None and (best is None or r[0] < best[0]):
                best = r
        if best is None:
            raise RuntimeError("no factorisation within the intermediate cap for " + str(key))
        _, labels, seq = best
        names = {}

        def ref(node):
            if node[0] == "t":
                return tens[node[1]]
            return names[id(node)], labels[id(node)]

        res = "R%d" % k
        head = f"{res}[{''.join(out)}] += {self.num(coef)}{(' ' + ptext) if ptext else ''} "
        if target is not None:
            head = f"{target}[{''.join(out)}] {'=' if first else '+='} {self.num(coef)} "
        if not seq:
            self.lines.append(head + tensor_text(*ref(("t", 0))))
            return
        for q, (x, y, node) in enumerate(seq):
            a, b = ref(x), ref(y)
            if q == len(seq) - 1:
                self.lines.append(head + tensor_text(*a) + " * " + tensor_text(*b))
                continue
            # an intermediate already defined with the same operands and index
            # pattern is reused under this statement's letters (no recomputation)
            sig = min(self._signature(a, b, labels[id(node)]), self._signature(b, a, labels[id(node)]))
            if sig in self.defs:
                names[id(node)] = self.defs[sig]
                continue
            self.nint += 1
            names[id(node)] = self.defs[sig] = f"X{self.nint}"
            self.lines.append(f"{tensor_text(*ref(node))} = {tensor_text(*a)} * {tensor_text(*b)}")

    @staticmethod
    def _signature(a, b, out):
        ren = {}
        for lab in list(a[1]) + list(b[1]) + list(out):
            if lab not in ren:
                ren[lab] = letter_space(lab) + str(len(ren))
        return (a[0], tuple(ren[x] for x in a[1]), b[0], tuple(ren[x] for x in b[1]), tuple(ren[x] for x in out))

    def _cost(self, tens, seq, out):
        """(flops, labels by node, seq) of one contraction sequence, None when an
        intermediate exceeds the cap."""
        need = {}
        for _, labs in tens:
            for x in labs:
                need[x] = need.get(x, 0) + 1
        for x in out:
            need[x] = need.get(x, 0) + 1
        labels = {}

        def labs_of(node):
            return tens[node[1]][1] if node[0] == "t" else labels[id(node)]

        flops = 0
        for q, (x, y, node) in enumerate(seq):
            la, lb = labs_of(x), labs_of(y)
            union = list(dict.fromkeys(la + lb))
            flops += 2 * self.size(union)
            for lab in la + lb:
                need[lab] -= 1
            keep = [lab for lab in union if need[lab] > 0]
            if q < len(seq) - 1 and self.size(keep) > self.cap:
                return None
            keep = tuple([l for l in keep if letter_space(l) == "o"] + [l for l in keep if letter_space(l) == "v"])
            for lab in keep:
                need[lab] += 1
            labels[id(node)] = keep
        return flops, labels, seq


METHODS = {"ccd": (2,), "ccsd": (1, 2), "ccsdt": (1, 2, 3)}


FULL_P = {2: "P(ij) P(ab)", 3: "P(i/jk) P(jk) P(a/bc) P(bc)"}


def generate(method, o, v, cap=None, header="", defer=True):
    """Contraction list text of a method (METHODS) for extents (o, v), which
    only steer the factorisation order and the intermediate cap.

    defer: the unsymmetrised term X of every diagram of R_k (k >= 2) is
    accumulated into one buffer Z_k with weight nterms / (k!)^2, and R_k gets
    the full antisymmetriser A of Z_k once.  X is antisymmetric under the
    stabiliser H of its orbit (|H| = (k!)^2 / nterms), so the diagram's
    P-operator sum equals A(X) / |H|: one antisymmetrising pass per residual
    instead of one per diagram.  This holds for antisymmetric amplitudes, the
    convention of every tensor the lists read."""
    ranks = METHODS[method]
    cap = cap if cap is not None else (o ** 3) * (v ** 3)
    fz = Factoriser(o, v, cap)
    lines = [header] if header else []
    for k in ranks:
        terms = derive(k, ranks)
        dg = diagrams(k, terms)
        fz.lines.append(f"# R{k}: {len(dg)} diagrams")
        use_z = defer and k >= 2
        for q, (coef, ptext, key, nterms) in enumerate(dg):
            if use_z:
                w = coef * Fraction(nterms, factorial(k) ** 2)
                fz.emit(k, w, "", key, target=f"Z{k}", first=q == 0)
            else:
                fz.emit(k, coef, ptext, key)
        if use_z:
            idx = OCC_EXT[:k] + VIR_EXT[:k]
            if k == 3:
                # A = A_occ A_vir: two passes of six terms instead of one of 36
                fz.lines.append(f"W3[{idx}] = P(a/bc) P(bc) Z3[{idx}]")
                fz.lines.append(f"R3[{idx}] += P(i/jk) P(jk) W3[{idx}]")
            else:
                fz.lines.append(f"R{k}[{idx}] += {FULL_P[k]} Z{k}[{idx}]")
    return "\n".join(lines + fz.lines) + "\n"


def count_diagrams(method):
    """Number of distinct diagrams (energy and every residual, with a general,
    non-diagonal Fock operator): the count the paper tabulates per method."""
    ranks = METHODS[method]
    total = 0
    for k in (0,) + tuple(ranks):
        terms = derive(k, ranks, hkinds=("F", "V"))
        total += len(diagrams(k, terms)) if k > 0 else len(terms)
    return total


HEADER = """# Spin-orbital {name} residual as an ordered list of binary contractions,
# derived by paper_2409_06759_b300/gen.py (Wick contractions of
# <Phi_l| (H_N exp(T))_C |Phi_0>, Eq. amp; {ndiag} diagrams with a general Fock
# operator, as in Tab. gener) and factorised for o={o}, v={v}
# (least flops, intermediates <= o^3 v^3 elements).  Diagonal Fock terms are
# not listed: the engine adds -D*t.  Regenerate with
#   python -m paper_2409_06759_b300.gen {method} {o} {v}
"""


def main(argv):
    method = argv[1] if len(argv) > 1 else "ccsd"
    o = int(argv[2]) if len(argv) > 2 else 8
    v = int(argv[3]) if len(argv) > 3 else 64
    head = HEADER.format(name=method.upper(), ndiag=count_diagrams(method), o=o, v=v, method=method)
    sys.stdout.write(generate(method, o, v, header=head.rstrip("\n")))


if __name__ == "__main__":
    main(sys.argv)
