"""CPU tests of the C-ABI library: it loads, exports every symbol that
include/sel.h declares, fails loudly without a GPU, and its predicate
compiler (host logic) produces programs whose meaning equals the oracle's."""
import ctypes as C
import os
import re

import numpy as np
import pytest
import torch

import datagen as dg
import oracle
import paper_1806_08384_b300 as sel
from tests import program_emulator as emu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(sel_[a-z0-9_]+)\s*\(", src))
    return sorted(names)


def test_library_exports_every_declared_symbol():
    names = declared_functions()
    assert "sel_count" in names and "sel_pushdown" in names and "sel_count_batch" in names
    lib = C.CDLL(sel.LIB_PATH)
    missing = [n for n in names if not hasattr(lib, n)]
    assert missing == []


@pytest.mark.skipif(torch.cuda.is_available(), reason="checks the no-GPU behaviour")
def test_context_fails_loudly_without_gpu():
    h = C.c_void_p()
    st = sel.lib.sel_ctx_create(None, C.byref(h))
    assert st == sel.SEL_ERR_CUDA
    assert sel.lib.sel_last_error().decode() != ""


def _compile(table, tree):
    return sel.Predicate(sel.Table(table.columns), tree)


def test_not_is_pushed_to_the_leaves():
    t = dg.tiny_table(8)
    p = _compile(t, dg.p_not(dg.p_and(dg.p_cmp(0, "<", 2), dg.p_or(dg.p_cmp(0, "=", 3), dg.p_not(dg.p_cmp(3, ">", dg.DATE_BASE))))))
    txt = p.describe()
    assert "NOT" not in txt
    # NOT(a AND (b OR NOT c)) = NOT a OR (NOT b AND c)
    assert txt.count("OR") == 1 and txt.count("AND") == 1


@pytest.mark.parametrize("tree,expect", [
    (dg.p_cmp(0, "<", -(1 << 40)), "CONST neg=1"),
    (dg.p_cmp(0, "<", 1 << 40), "CONST neg=0"),
    (dg.p_cmp(0, ">=", -(2 ** 31)), "CONST neg=0"),
    (dg.p_cmp(0, "<>", 1 << 35), "CONST neg=0"),
    (dg.p_in(0, []), "CONST neg=1"),
    (dg.p_in(0, [3, 1, 2, 2]), "RANGE32 slot=0 neg=0 lo=1 span=2"),
    (dg.p_in(0, [1, 5, 9]), "MASK32 slot=0 neg=0 lo=1 word=0x111"),
    (dg.p_in(0, [1, 5000]), "IN32"),
    (dg.p_in(0, [1, 100, 5000]), "HASH32"),
    (dg.p_in(0, list(range(0, 40, 3))), "HASH32"),
    (dg.p_in(0, list(range(0, 3000, 3))), "BITMAP"),
    (dg.p_in(1, [1, 5, 9]), "HASH64"),
    (dg.p_in(1, [-(2 ** 62), 5]), "IN64"),
    (dg.p_between(0, 5, 4), "CONST neg=1"),
    (dg.p_between(2, 3.0, 1.0), "CONST neg=1"),
    (dg.p_cmp(2, "<", float("-inf")), "CONST neg=1"),
    (dg.p_cmp(2, ">", float("inf")), "CONST neg=1"),
    (dg.p_cmp(1, "<", -(2 ** 63)), "CONST neg=1"),
    (dg.p_cmp(1, "<=", 2 ** 63 - 1), "CONST neg=0"),
    (dg.p_like(4, ""), "RANGE32 slot=0 neg=0 lo=0 span=4"),
    (dg.p_and(dg.P_TRUE, dg.p_cmp(0, "=", 1)), "RANGE32 slot=0 neg=0 lo=1 span=0"),
    (dg.p_or(dg.P_TRUE, dg.p_cmp(0, "=", 1)), "CONST neg=0"),
])
def test_leaf_lowering(tree, expect):
    t = dg.tiny_table(8)
    assert expect in _compile(t, tree).describe()


def test_leaf_before_and_or_combines_into_top():
    """A leaf (or LOAD) directly followed by AND/OR folds into the top of the
    mask stack: the operator's instruction disappears, the program's meaning
    does not (the emulator models the folded form)."""
    t = dg.tiny_table(64, seed=9)
    chain = dg.p_and(dg.p_cmp(0, ">", 1), dg.p_cmp(3, ">", dg.DATE_BASE), dg.p_cmp(1, "<", 5))
    txt = _compile(t, chain).describe()
    body = txt.strip().splitlines()[3:]
    assert len(body) == 3 and body[0].split()[0] != "AND"
    assert [ln.split()[-1] for ln in body[1:]] == ["+AND", "+AND"]
    dnf = dg.p_or(dg.p_and(dg.p_cmp(0, ">", 1), dg.p_cmp(1, "<", 5)), dg.p_cmp(2, "<", 0.5))
    txt = _compile(t, dnf).describe()
    assert "+AND" in txt and "+OR" in txt and not any(ln.strip() == "AND" for ln in txt.splitlines())
    ot = oracle.OTable.from_table(t)
    arrays = [c.data.numpy() for c in t.columns]
    for tree in (chain, dnf):
        got = emu.evaluate(_compile(t, tree).describe(), arrays, t.n_rows)
        assert int(got.sum()) == oracle.count(ot, tree)


def test_unsorted_dictionary_prefix_is_a_bitmap():
    d = [b"ab", b"c", b"ax", b"d", b"aa"]
    col = dg.Column(dg.ColumnSpec("s", "dict", "zipf", n_values=5), torch.zeros(4, dtype=torch.int32), d)
    p = sel.Predicate(sel.Table([col]), dg.p_like(0, "a"))
    assert "BITMAP slot=0 neg=0 lo=0 nbits=5 words=0x15" in p.describe()


@pytest.mark.parametrize("tree,status", [
    (dg.p_like(0, "a"), sel.SEL_ERR_TYPE),
    (dg.p_like(2, "a"), sel.SEL_ERR_TYPE),
    (dg.p_cmp(9, "<", 1), sel.SEL_ERR_INVALID_ARG),
    (dg.p_in(0, list(range(5000))), sel.SEL_ERR_UNSUPPORTED),
    (dg.p_and(*[dg.p_cmp(0, "=", i) for i in range(65)]), sel.SEL_ERR_UNSUPPORTED),
])
def test_compile_errors(tree, status):
    t = dg.tiny_table(8)
    with pytest.raises(sel.SelError) as e:
        _compile(t, tree)
    assert e.value.status == status


def test_malformed_postfix_is_rejected():
    t = sel.Table(dg.tiny_table(4).columns)
    arr = (sel.sel_node * 2)()
    arr[0].kind, arr[0].col = sel.N_CMP, 0
    arr[1].kind, arr[1].n_children = sel.N_AND, 2        # AND of 2 with one operand on the stack
    h = C.c_void_p()
    assert sel.lib.sel_compile_predicate(t.ref(), arr, 2, C.byref(h)) == sel.SEL_ERR_INVALID_ARG
    arr2 = (sel.sel_node * 2)()
    arr2[0].kind = arr2[1].kind = sel.N_TRUE                # two trees left on the stack
    assert sel.lib.sel_compile_predicate(t.ref(), arr2, 2, C.byref(h)) == sel.SEL_ERR_INVALID_ARG


def test_stack_depth_is_bounded_by_operand_ordering():
    t = dg.tiny_table(4)

    def balanced(lo, hi):
        if hi - lo == 1:
            return dg.p_cmp(0, "=", lo % 4)
        mid = (lo + hi) // 2
        k = "and" if (hi - lo) % 4 else "or"
        return (k, [balanced(lo, mid), balanced(mid, hi)])
    txt = _compile(t, balanced(0, 64)).describe()
    assert emu.need(txt) <= 7
    # a right-deep chain needs no more than 2 entries once reordered
    chain = dg.p_cmp(0, "=", 0)
    for i in range(30):
        chain = ("or", [dg.p_cmp(0, "=", i % 4), ("and", [dg.p_cmp(3, ">", dg.DATE_BASE), chain])])
    assert emu.need(_compile(t, chain).describe()) <= 3


@pytest.mark.parametrize("n", [0, 1, 33, 257])
def test_compiled_programs_match_oracle(n):
    """Compiler + device-program semantics vs the oracle on random trees."""
    t = dg.tiny_table(n, seed=n + 100)
    ot = oracle.OTable.from_table(t)
    arrays = [c.data.numpy() for c in t.columns]
    rng = np.random.default_rng(n)
    for _ in range(150):
        tree = dg.random_tree(t, rng, depth=4)
        got = emu.evaluate(_compile(t, tree).describe(), arrays, n)
        ids = oracle.select(ot, tree)
        want = np.zeros(n, bool)
        want[ids] = True
        assert np.array_equal(got, want), tree


def test_every_single_clause_matches_oracle():
    n = 97
    t = dg.tiny_table(n, seed=5)
    ot = oracle.OTable.from_table(t)
    arrays = [c.data.numpy() for c in t.columns]
    for col in range(len(t.columns)):
        consts = dg.tiny_constants(t, col)
        trees = [dg.p_cmp(col, op, c) for op in ("=", "<>", "<", "<=", ">", ">=") for c in consts]
        trees += [dg.p_between(col, a, b) for a in consts for b in consts]
        trees += [dg.p_in(col, consts[:k]) for k in range(len(consts) + 1)]
        if t.columns[col].type == "dict":
            trees += [dg.p_like(col, w[:k].decode()) for w in t.columns[col].dictionary for k in range(len(w) + 1)]
        for tree in trees:
            for tr in (tree, dg.p_not(tree)):
                got = emu.evaluate(_compile(t, tr).describe(), arrays, n)
                assert int(got.sum()) == oracle.count(ot, tr), tr


def test_repeated_leaves_are_evaluated_once():
    """A leaf that occurs in several AND groups is saved once and reloaded."""
    t = dg.gen_table("cfg2", dg.config2_specs(), 3000, "cpu")
    ot = oracle.OTable.from_table(t)
    arrays = [c.data.numpy() for c in t.columns]
    saw_load = False
    for s in dg.CONFIG2_TARGETS:
        for seed in range(4):
            tree = dg.config2_predicate(s, seed=seed)
            txt = _compile(t, tree).describe()
            saw_load |= "LOAD m=" in txt
            got = emu.evaluate(txt, arrays, t.n_rows)
            assert int(got.sum()) == oracle.count(ot, tree), tree
    assert saw_load
    a = dg.p_in(2, [1, 5, 9])
    txt = _compile(t, dg.p_or(dg.p_and(a, dg.p_cmp(0, "<", 9)), dg.p_and(a, dg.p_cmp(1, ">", 9)),
                              dg.p_and(dg.p_not(a), dg.p_cmp(5, "=", 9)))).describe()
    assert txt.count("HASH64") == 2 and txt.count("LOAD") == 1   # NOT a is a different leaf


@pytest.mark.parametrize("n_vals", [3, 5, 8, 17, 64, 256])
def test_hashed_in_lists_match_oracle(n_vals):
    """IN lists lowered to perfect multiply-shift hash tables (int32 and int64
    columns, values far apart, negated too): the emulated tables give the
    oracle's counts, and members outside the table's rows still miss."""
    t = dg.gen_table("cfg2", dg.config2_specs(), 4000, "cpu")
    ot = oracle.OTable.from_table(t)
    arrays = [c.data.numpy() for c in t.columns]
    rng = np.random.default_rng(n_vals)
    for col in (0, 2, 7):
        data = arrays[col]
        present = [int(x) for x in rng.choice(data, size=min(n_vals, 2 * n_vals // 3 + 1), replace=False)]
        absent = [int(x) for x in rng.integers(-(2 ** 31), 2 ** 31, size=n_vals - len(present))]
        vals = present + absent
        for tr in (dg.p_in(col, vals), dg.p_not(dg.p_in(col, vals))):
            txt = _compile(t, tr).describe()
            if n_vals <= 64:   # a single multiply-shift table holds up to about 64 values within 8 KB
                assert ("HASH64" if col == 2 else "HASH32") in txt, txt[:200]
            got = emu.evaluate(txt, arrays, t.n_rows)
            assert int(got.sum()) == oracle.count(ot, tr)
