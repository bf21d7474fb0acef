"""C-ABI library checks that need no GPU: the .so loads, exports every symbol
include/cc.h declares, and the parser/planner (host only) behaves."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def cc():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2409_06759_b300 as cc
    return cc


def header_functions():
    txt = open(os.path.join(ROOT, "include", "cc.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(cc_[a-z0-9_]+)\s*\(", txt)))


def test_exports_every_declared_symbol(cc):
    lib = ctypes.CDLL(cc.LIB_PATH)
    names = header_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(cc.EXPORTS) == names


def test_version_and_status(cc):
    assert "sm_103a" in cc.cc_version()
    assert cc.cc_status_string(0) == "ok"
    assert cc.cc_status_string(2) == "parse error"


@pytest.mark.parametrize("name", ["ccsd", "ccsd_vvvv"])
def test_plan_ccsd_structure(cc, name):
    o, v = 40, 200
    p = cc.cc_plan_create(cc.load_list(name), o, v, precision="fp64")
    d = p.describe()
    gemms = [s for s in d["steps"] if s["kind"].startswith("gemm")]
    assert sum(s["flops"] for s in gemms) == pytest.approx(p.flops)
    ladder = [s for s in gemms if s["M"] * s["N"] * s["K"] == (v * v) * (o * o) * (v * v)]
    assert len(ladder) == 1, "one o^2 v^4 ladder GEMM"
    # the ladder runs as a plain GEMM: no permute or epilogue in its statement
    st = ladder[0]["stmt"]
    assert not [s for s in d["steps"] if s["stmt"] == st and s["kind"] == "accum"]
    assert p.flops < 1.3 * (2 * o**2 * v**4 + 6 * o**3 * v**3 + 10 * o**4 * v**2)


def test_plan_mixed_routes_big_gemms(cc):
    o, v = 40, 200
    p = cc.cc_plan_create(cc.load_list("ccsd_vvvv"), o, v, precision="bf16x3")
    d = p.describe()
    mixed = [s for s in d["steps"] if s["kind"] == "gemm_bf16split"]
    assert mixed and max(s["flops"] for s in mixed) == 2.0 * o**2 * v**4
    lad = [s for s in mixed if s["flops"] == 2.0 * o**2 * v**4][0]
    assert lad["products"] == 3
    assert lad["a_static"] or lad["b_static"], "the <ab||ef> planes are cached"


@pytest.mark.parametrize("text,frag", [
    ("R2[ijab] = V[ijab] * T2[ijab] * T1[ia]", "binary"),
    ("R2[ijab] = X[ijab]", "before a defining"),
    ("R2[ijqb] = V[ijqb]", "neither occupied"),
    ("R2[ijab] = V[ijab", "bracket"),
    ("X[ijab] += T2[ijab]", "before a defining"),
    ("R2[ijab] = T2[ijae] * V[ebcd]", "output indices"),
    ("R2[ijab] = 0.5 P(ia) T2[ijab]", "mixes occupied"),
    ("T2[ijab] = V[ijab]", "inputs"),
])
def test_parse_errors(cc, text, frag):
    with pytest.raises(cc.CCError) as ei:
        cc.cc_plan_create(text, 3, 4)
    assert frag in str(ei.value)
    assert "line 1" in str(ei.value)


def test_paper_bracket_form_is_accepted(cc):
    """t[ef][ij] (upper/lower, as printed in the paper) names the same tensor as T2[ijef]."""
    a = cc.cc_plan_create("R2[ijab] = 0.5 t[ef][ij] * V[ab][ef]", 3, 5).describe()
    b = cc.cc_plan_create("R2[ijab] = 0.5 T2[ijef] * V[abef]", 3, 5).describe()
    ga = [s for s in a["steps"] if s["kind"] == "gemm_f64"][0]
    gb = [s for s in b["steps"] if s["kind"] == "gemm_f64"][0]
    for k in ("M", "N", "K", "sAm", "sAk", "sBk", "sBn", "alpha"):
        assert ga[k] == gb[k]


def test_integral_block_resolution_signs(cc):
    """<mb||ej> comes from the ovov block with a minus sign (ket swap)."""
    d = cc.cc_plan_create("X[mbej] = V[mbej]", 3, 5).describe()
    acc = [s for s in d["steps"] if s["kind"] == "accum"][0]
    assert acc["alpha"] == -1.0
    assert {t["name"] for t in d["tensors"]} >= {"V_ovov"}


def test_integral_block_elems(cc):
    e = cc.cc_integral_block_elems(3, 5)
    assert e == dict(oooo=81, ooov=135, oovv=225, ovov=225, ovvv=375, vvvv=625)


def test_workspace_grows_with_size(cc):
    small = cc.cc_plan_create(cc.load_list("ccsd"), 4, 8).workspace_bytes
    big = cc.cc_plan_create(cc.load_list("ccsd"), 8, 16).workspace_bytes
    assert 0 < small < big


def test_complex_plan_structure(cc):
    """Complex plans: the same steps as the real plan with four times the real
    flops; integral references whose bra and ket are swapped against the
    stored block are read conjugated."""
    o, v = 6, 20
    for name in ("ccsd", "ccsd_vvvv"):
        r = cc.cc_plan_create(cc.load_list(name), o, v, dtype=cc.CC_F64)
        z = cc.cc_plan_create(cc.load_list(name), o, v, dtype=cc.CC_C128)
        assert z.describe()["dtype"] == 1
        assert z.flops == pytest.approx(4 * r.flops)
        assert z.workspace_bytes > 1.8 * r.workspace_bytes
    drv = cc.cc_plan_create("R2[ijab] = V[abij]", 3, 5, dtype=cc.CC_C128).describe()
    assert [s["conj_a"] for s in drv["steps"] if s["kind"] == "accum"] == [1]
    drv = cc.cc_plan_create("R2[ijab] = V[ijab]", 3, 5, dtype=cc.CC_C128).describe()
    assert [s["conj_a"] for s in drv["steps"] if s["kind"] == "accum"] == [0]
    # real lists never conjugate
    drv = cc.cc_plan_create("R2[ijab] = V[abij]", 3, 5).describe()
    assert [s["conj_a"] for s in drv["steps"] if s["kind"] == "accum"] == [0]


def test_complex_split_route_doubles_k(cc):
    """On the split route a complex contraction is one real GEMM of doubled K,
    with the smaller operand embedded (its rows doubled) and the larger stacked."""
    o, v = 8, 40
    p = cc.cc_plan_create("R2[ijab] = 0.5 T2[ijef] * V[abef]", o, v, dtype=cc.CC_C128, precision="bf16x3")
    g = [s for s in p.describe()["steps"] if s["kind"] == "gemm_bf16split"][0]
    assert g["K"] == 2 * v * v
    assert {g["M"], g["N"]} == {v * v, 2 * o * o}
    assert g["flops"] == 8.0 * o * o * v ** 4
    small = "a" if g["M"] == 2 * o * o else "b"
    assert g["cplx_" + small] == 2 and g["cplx_" + ("b" if small == "a" else "a")] == 1


def test_batched_argument_checks(cc):
    """cc_solve_batched validates before any device work: one plan per system."""
    p = cc.cc_plan_create(cc.load_list("ccsd"), 3, 5)
    q = cc.cc_plan_create(cc.load_list("ccsd"), 4, 6)
    n1 = cc.cc_solve_batched_workspace_bytes([p])
    n2 = cc.cc_solve_batched_workspace_bytes([p, q])
    assert 0 < n1 < n2
    with pytest.raises(cc.CCError) as ei:
        cc.cc_solve_batched([p, p], [{}, {}], [(None, None), (None, None)], None)
    assert "plan of its own" in str(ei.value)


def test_packed_pairs_plan(cc):
    """Declared pairs: the ladder runs as pack + one GEMM over pairs + unpack,
    with the pair-count flops; the integral operand is packed once (static)."""
    o, v = 8, 30
    p = cc.cc_plan_create(cc.load_list("ccsd_packed"), o, v)
    q = cc.cc_plan_create(cc.load_list("ccsd_vvvv"), o, v)
    d = p.describe()
    kinds = [s["kind"] for s in d["steps"]]
    assert kinds.count("pack") == 4 and kinds.count("unpack") == 2
    P, Q = o * (o - 1) // 2, v * (v - 1) // 2
    lad = [s for s in d["steps"] if s["kind"].startswith("gemm") and s["K"] == Q and Q in (s["M"], s["N"])]
    assert lad and lad[0]["flops"] == 2.0 * P * Q * Q
    assert p.flops < q.flops - 2.0 * o * o * v ** 4 * 0.8


@pytest.mark.parametrize("text,frag", [
    ("R2[ijab] = 0.5 T2[(ij)(ef)] * V[(ab)(fe)] * T1[ia]", "binary"),
    ("R2[ijab] = T2[(ij)(ef)] * V[(ae)(bf)]", "declared pair"),
    ("R2[ijab] = T2[(i)(jab)]", "exactly two"),
    ("R2[ijab] = T2[(ij(ab))]", "nested"),
])
def test_packed_pair_errors(cc, text, frag):
    with pytest.raises(cc.CCError) as ei:
        cc.cc_plan_create(text, 3, 5)
    assert frag in str(ei.value)


def test_packed_pairs_reject_complex(cc):
    with pytest.raises(cc.CCError) as ei:
        cc.cc_plan_create(cc.load_list("ccsd_packed"), 3, 5, dtype=cc.CC_C128)
    assert "real" in str(ei.value)


def test_wait_selftest_budget_checked_before_device_work(cc):
    assert cc.cc_selftest_wait_timeout(10) == 1          # CC_ERR_INVALID_ARG


def test_autotune_candidates_and_config_replay(cc):
    """Host-side candidate lists of the o=40 v=200 split-bf16 plan: every
    tunable step offers its planned configuration; on the tensor route the
    tile widths are 64/128/256; accumulating steps without split K also offer
    the reduction epilogue; cc_plan_set_gemm_config takes exactly the listed
    configurations and the description reports the one set."""
    o, v = 40, 200
    p = cc.cc_plan_create(cc.load_list("ccsd_vvvv"), o, v, precision="bf16x3")
    steps = p.describe()["steps"]
    tunable = [(k, s) for k, s in enumerate(steps) if s.get("configs")]
    assert len(tunable) >= 10
    reds = 0
    for k, s in tunable:
        cfgs = [tuple(c) for c in s["configs"]]
        planned = (s.get("bn", 0), s["splitk"], s.get("red", 0))
        assert planned in cfgs, (k, planned, cfgs)
        assert len(set(cfgs)) == len(cfgs)
        if s["kind"] == "gemm_bf16split":
            assert {c[0] for c in cfgs} <= {64, 128, 256}
        for bn, sk, red in cfgs:
            if red:
                assert sk == 1 and s["beta"] == 1, (k, s["note"])
                reds += 1
    assert reds > 0
    k, s = next((k, s) for k, s in tunable if any(c[2] for c in s["configs"]))
    bn, sk, red = next(c for c in s["configs"] if c[2])
    cc.cc_plan_set_gemm_config(p, k, bn, sk, red)
    got = p.describe()["steps"][k]
    assert (got.get("bn", 0), got["splitk"], got.get("red", 0)) == (bn, sk, red)
    with pytest.raises(RuntimeError):
        cc.cc_plan_set_gemm_config(p, k, 96, 1, 0)
    with pytest.raises(RuntimeError):
        cc.cc_plan_set_gemm_config(p, len(steps), bn, sk, red)


@pytest.mark.parametrize("name", ["ccsd", "ccsd_vvvv", "ccsd_packed", "ccsdt"])
def test_parser_round_trips_its_statements(cc, name):
    """The planner's normalised rendering of each statement (factor, P(..)
    operators, operands, packed-pair declarations) parses back to the same
    plan: identical statements, steps and flop count."""
    o, v = (4, 9) if name != "ccsdt" else (3, 5)
    p = cc.cc_plan_create(cc.load_list(name), o, v, precision="fp64")
    d = p.describe()
    q = cc.cc_plan_create("\n".join(d["statements"]), o, v, precision="fp64")
    e = q.describe()
    assert e["statements"] == d["statements"]
    assert e["steps"] == d["steps"]
    assert q.flops == p.flops


def test_bench_flop_constants_match_the_plans(cc):
    """bench.py records the timed plan's flops so that its reference arm never
    loads this library; they must equal cc_plan_flops."""
    import bench
    for (name, o, v, dt), flops in bench.PLAN_FLOPS.items():
        p = cc.cc_plan_create(cc.load_list(name), o, v, dtype=cc.CC_C128 if dt == "c128" else cc.CC_F64,
                              precision=cc.CC_PREC_BF16X3)
        assert p.flops == flops, (name, o, v, dt)


def test_slices_plan_routes(cc):
    """The exact-slice precision: every bulk GEMM on the tensor cores with six
    planes (21 products, 64-wide tiles), every other route FP64 (no FP32)."""
    p = cc.cc_plan_create(cc.load_list("ccsd_vvvv"), 40, 200, precision="slices")
    d = p.describe()
    kinds = {st["kind"] for st in d["steps"]}
    assert "gemm_bf16split" in kinds and not any(k.endswith("f32") for k in kinds)
    for st in d["steps"]:
        if st["kind"] == "gemm_bf16split":
            assert st["products"] == 21 and st["bn"] == 64
            assert all(c[0] == 64 for c in st.get("configs", []))
    lad = next(st for st in d["steps"] if st["note"] == "V_vvvv*tau -> Z2")
    # six bf16 planes and one int32 exponent per row of the 40000 x 40000 block
    assert d["cache_bytes"] >= 6 * 40000 * 40000 * 2 + 40000 * 4
    assert lad["flops"] == 2.0 * 40000 * 1600 * 40000


def test_k_concatenated_steps(cc):
    """Split-route plans merge accumulating statements into one pass over their
    output when the output's letters fall on the same operand positions (K
    concatenation, on the split route or the narrow kernel): every member
    accumulates into the step's output, each statement is planned once, the
    merged K is at most the members' total, the FLOP count is unchanged;
    FP64, exact-slice and complex plans, and kconcat=False, merge nothing;
    the cached ladder block is never re-split into a merged step."""
    text = cc.load_list("ccsdt")
    stmts = [l.split("#")[0].strip() for l in text.splitlines() if l.split("#")[0].strip()]
    for prec in ("bf16x3", "bf16x6"):
        d = cc.cc_plan_create(text, 8, 64, precision=prec).describe()
        ref = cc.cc_plan_create(text, 8, 64, precision=prec, kconcat=False).describe()
        assert not any("stmts" in st for st in ref["steps"])
        assert d["flops"] == pytest.approx(ref["flops"], rel=1e-12)
        merged = [st for st in d["steps"] if "stmts" in st]
        # the sums of operands that several members share run as copies before their step
        sums = [st for st in d["steps"] if st["note"].startswith("operand sum")]
        assert all(st["kind"] == "accum" for st in sums) and len(sums) >= 10
        assert len(merged) >= 8 and len(d["steps"]) - len(sums) < len(ref["steps"]) - 40
        seen = {}
        for st in d["steps"]:
            if st in sums:
                continue
            for si in st.get("stmts", [st["stmt"]]):
                seen.setdefault(si, set()).add(id(st))
        assert sorted(seen) == list(range(len(stmts)))
        kref = {}
        for st in ref["steps"]:
            if st["kind"].startswith("gemm"):
                kref[st["stmt"]] = st["K"]
        for st in merged:
            out = st["note"].rsplit("-> ", 1)[1]
            assert len(st["stmts"]) >= 2 and st["stmts"] == sorted(st["stmts"])
            for si in st["stmts"]:
                lhs, rhs = stmts[si].split("=", 1)
                assert lhs.rstrip("+-").strip().startswith(out + "[") and lhs.rstrip()[-1] in "+-", stmts[si]
                assert "P(" not in rhs
                assert seen[si] == {id(st)}          # a member runs in its merged step only
            # statements that share an operand contract it once with the sum of their
            # other operands: K is at most the members' total
            assert 0 < st["K"] <= sum(kref[si] for si in st["stmts"])
            if st["kind"] == "gemm_bf16split":
                assert st["Kp"] % 64 == 0 and st["Kp"] >= st["K"]
    for prec, dt in (("fp64", cc.CC_F64), ("slices", cc.CC_F64), ("bf16x3", cc.CC_C128)):
        d = cc.cc_plan_create(text, 6, 30, dtype=dt, precision=prec).describe()
        assert not any("stmts" in st for st in d["steps"]), (prec, dt)
    lad = cc.cc_plan_create(cc.load_list("ccsd_vvvv"), 40, 200, precision="bf16x3").describe()
    step = next(st for st in lad["steps"] if "V_vvvv*tau" in st["note"])
    assert "stmts" not in step and step["note"] == "V_vvvv*tau -> Z2"


def test_uniform_steps_plans_are_alike_at_every_size(cc):
    """uniform_steps: every contraction on the split route, none merged, so the
    step list is the same at any o, v (what grouped batch execution needs);
    the batched workspace then holds the grouped tables too."""
    text = cc.load_list("ccsd_vvvv")
    sigs = set()
    plans = []
    for o, v in ((4, 20), (16, 80), (7, 33), (12, 25)):
        p = cc.cc_plan_create(text, o, v, precision="bf16x3", uniform_steps=True)
        d = p.describe()
        # contractions with a two-index operand (T1, F) on the narrow kernel, the rest on the tensor cores
        assert all(st["kind"] in ("accum", "gemm_bf16split", "gemm_rows_f32") for st in d["steps"])
        stmts = d["statements"]
        for st in d["steps"]:
            if st["kind"].startswith("gemm"):
                ops = stmts[st["stmt"]].split("=", 1)[1]
                two = any(len(x.split("]")[0]) == 2 for x in ops.split("[")[1:])
                assert (st["kind"] == "gemm_rows_f32") == two, stmts[st["stmt"]]
        assert not any("stmts" in st for st in d["steps"])
        sigs.add(tuple((st["kind"], st["note"]) for st in d["steps"]))
        plans.append(p)
    assert len(sigs) == 1
    with pytest.raises(cc.CCError):
        cc.cc_plan_create(text, 4, 20, precision="fp64", uniform_steps=True)
    with pytest.raises(cc.CCError):
        cc.cc_plan_create(text, 4, 20, dtype=cc.CC_C128, precision="bf16x3", uniform_steps=True)
    grouped = cc.cc_solve_batched_workspace_bytes(plans, 8)
    plain = cc.cc_solve_batched_workspace_bytes(
        [cc.cc_plan_create(text, o, v, precision="bf16x3") for o, v in ((4, 20), (16, 80), (7, 33), (12, 25))], 8)
    assert grouped > 0 and plain > 0
