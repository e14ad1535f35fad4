"""Pins for the CPU oracle: facts fixed by the paper and by mathematics, not by
the oracle itself.

Each ``pin_*`` function takes a loaded oracle library (the real one, or a
deliberately mutated copy) and returns a list of failure strings.  The pins:

* closed forms on constructed columns (a seeded permutation of the row index,
  i mod m, exact small floats, a hand-made sorted dictionary);
* order-statistic and histogram counts computed by different methods
  (``np.searchsorted`` on the sorted column, ``np.bincount`` of codes with
  ``bytes.startswith`` over the dictionary);
* the four rows the paper prints in §1.2 (table "Column vs. row stores"),
  with counts worked by hand (tests/golden/col_vs_row_table.json);
* boolean identities of two-valued logic on random trees: the partition
  count(A) = count(A and B) + count(A and not B), inclusion-exclusion for OR,
  De Morgan, complement, TRUE -> n, FALSE -> 0, BETWEEN widening monotone.
"""
from __future__ import annotations

import json
import os

import numpy as np
import torch

import datagen as dg
import oracle
from datagen import p_and, p_between, p_cmp, p_in, p_like, p_not, p_or

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _table(arrays, types, dicts=None):
    dicts = dicts or [None] * len(arrays)
    return oracle.OTable(arrays, types, dicts)


def pin_permutation_closed_forms(lib):
    """c = seeded bijection of 0..n-1: every range has a known size."""
    fails = []
    n = 5000
    perm = np.random.default_rng(7).permutation(n).astype(np.int32)
    t = _table([perm], ["i32"])
    for a, b in [(0, 0), (0, n - 1), (17, 4000), (4999, 4999), (10, 9), (-5, 3), (4990, 6000)]:
        want = max(0, min(b, n - 1) - max(a, 0) + 1)
        got = oracle.count(t, p_between(0, a, b), lib=lib)
        if got != want:
            fails.append(f"between {a},{b}: {got} != {want}")
    for x in [-1, 0, 1, 2500, n - 1, n]:
        lt, le = min(max(x, 0), n), min(max(x + 1, 0), n)
        want = {"<": lt, "<=": le, ">": n - le, ">=": n - lt,
                "=": 1 if 0 <= x < n else 0, "<>": n - (1 if 0 <= x < n else 0)}
        for op, w in want.items():
            got = oracle.count(t, p_cmp(0, op, x), lib=lib)
            if got != w:
                fails.append(f"perm {op} {x}: {got} != {w}")
    # the selected row ids are the inverse permutation of [a, b], ascending
    inv = np.argsort(perm)
    ids = oracle.select(t, p_between(0, 100, 1999), lib=lib)
    if not np.array_equal(ids, np.sort(inv[100:2000])):
        fails.append("select between: row ids differ from the inverse permutation")
    ids = oracle.select(t, p_not(p_between(0, 100, 1999)), lib=lib)
    if not np.array_equal(ids, np.sort(np.concatenate([inv[:100], inv[2000:]]))):
        fails.append("select not-between: row ids differ")
    return fails


def pin_modulo_closed_forms(lib):
    """c = i mod m: count(c < t) = floor(n/m) * t + min(t, n mod m)."""
    fails = []
    for n, m in [(1000, 7), (4097, 32), (33, 40)]:
        col = (np.arange(n) % m).astype(np.int32)
        t_ = _table([col], ["i32"])
        for t in [0, 1, m // 2, m - 1, m]:
            want = (n // m) * t + min(t, n % m)
            got = oracle.count(t_, p_cmp(0, "<", t), lib=lib)
            if got != want:
                fails.append(f"mod n={n} m={m} < {t}: {got} != {want}")
        vals = [0, m - 1, m // 3, 0, m + 5]           # duplicates and a value outside the domain
        distinct = sorted({v for v in vals if 0 <= v < m})
        want = sum((n // m) + (1 if v < n % m else 0) for v in distinct)
        got = oracle.count(t_, p_in(0, vals), lib=lib)
        if got != want:
            fails.append(f"mod IN: {got} != {want}")
        if oracle.count(t_, p_in(0, []), lib=lib) != 0:
            fails.append("empty IN is not FALSE")
    return fails


def pin_float_closed_forms(lib):
    """Exact small floats: c = float(i) for i < 2^24, plus signed zeros."""
    fails = []
    n = 3000
    col = np.arange(n, dtype=np.float32)
    t = _table([col], ["f32"])
    cases = [(p_cmp(0, "<", 10.5), 11), (p_cmp(0, "<", 10.0), 10), (p_cmp(0, "<=", 10.0), 11),
             (p_cmp(0, ">", 2998.5), 1), (p_cmp(0, ">=", 0.0), n), (p_cmp(0, "=", 7.0), 1),
             (p_cmp(0, "<>", 7.0), n - 1), (p_between(0, 5.0, 9.0), 5), (p_between(0, 9.0, 5.0), 0),
             (p_between(0, -0.0, 0.0), 1), (p_cmp(0, "<", -0.0), 0), (p_cmp(0, "<=", -0.0), 1),
             (p_in(0, [1.0, 2.0, 2.0, 0.5]), 2), (p_cmp(0, "<", float("inf")), n),
             (p_cmp(0, ">", float("-inf")), n), (p_cmp(0, "<", float("-inf")), 0)]
    for tree, want in cases:
        got = oracle.count(t, tree, lib=lib)
        if got != want:
            fails.append(f"float {tree}: {got} != {want}")
    z = np.array([-0.0, 0.0, -0.0, 1.0], dtype=np.float32)
    tz = _table([z], ["f32"])
    for tree, want in [(p_cmp(0, "=", 0.0), 3), (p_cmp(0, "=", -0.0), 3), (p_cmp(0, "<", 0.0), 0),
                       (p_cmp(0, ">=", 0.0), 4), (p_between(0, 0.0, 0.0), 3)]:
        got = oracle.count(tz, tree, lib=lib)
        if got != want:
            fails.append(f"signed zero {tree}: {got} != {want}")
    return fails


def pin_int64_and_widening(lib):
    """int64 values beyond 32 bits, and int32 columns vs constants outside int32."""
    fails = []
    n = 1000
    c64 = (np.arange(n, dtype=np.int64) - 500) * (1 << 33)
    c32 = (np.arange(n, dtype=np.int64) - 500).astype(np.int32)
    t = _table([c64, c32], ["i64", "i32"])
    cases = [(p_cmp(0, "<", 0), 500), (p_cmp(0, "<", 1), 501), (p_cmp(0, "<=", -(1 << 33)), 500),
             (p_between(0, -(3 << 33), 3 << 33), 7), (p_cmp(0, "=", 1 << 33), 1),
             (p_cmp(1, "<", 1 << 40), n), (p_cmp(1, ">", -(1 << 40)), n), (p_cmp(1, "=", (1 << 32) + 5), 0),
             (p_between(1, -(1 << 35), 0), 501), (p_cmp(1, ">=", 2 ** 31), 0)]
    for tree, want in cases:
        got = oracle.count(t, tree, lib=lib)
        if got != want:
            fails.append(f"int64 {tree}: {got} != {want}")
    return fails


def pin_like_closed_forms(lib):
    """Hand-made sorted dictionary; codes i mod 6 plus out-of-range codes."""
    fails = []
    d = [b"a", b"ab", b"abc", b"b", b"ba", b"c"]
    n = 600
    codes = (np.arange(n) % 6).astype(np.int32)
    codes[::50] = -1
    codes[1::50] = 6
    t = _table([codes], ["dict"], [d])
    valid = codes[(codes >= 0) & (codes < 6)]
    per = np.bincount(valid, minlength=6)
    for prefix in ["", "a", "ab", "abc", "abcd", "b", "c", "z", "B"]:
        want = int(sum(per[i] for i, w in enumerate(d) if w.startswith(prefix.encode())))
        got = oracle.count(t, p_like(0, prefix), lib=lib)
        if got != want:
            fails.append(f"like {prefix!r}: {got} != {want}")
    return fails


def pin_order_statistics(lib):
    """Random columns: range counts from the sorted column (searchsorted) and
    equality/IN/LIKE counts from histograms (bincount)."""
    fails = []
    tab = dg.gen_table("pins", dg.config2_specs(), 20_000, "cpu")
    ot = oracle.OTable.from_table(tab)
    rng = np.random.default_rng(3)
    for ci in range(len(tab.columns)):
        a = ot.arrays[ci]
        if ot.types[ci] == "dict":
            d = ot.dicts[ci]
            hist = np.bincount(a, minlength=len(d))
            for pre in ["a", "k", "zz", ""]:
                want = int(sum(hist[k] for k, w in enumerate(d) if w.startswith(pre.encode())))
                got = oracle.count(ot, p_like(ci, pre), lib=lib)
                if got != want:
                    fails.append(f"hist like col {ci} {pre!r}: {got} != {want}")
            continue
        s = np.sort(a)
        for _ in range(4):
            x, y = (a[int(i)] for i in rng.integers(0, len(a), 2))
            lo, hi = (x, y) if x <= y else (y, x)
            lo, hi = (float(lo), float(hi)) if ot.types[ci] == "f32" else (int(lo), int(hi))
            want = int(np.searchsorted(s, hi, "right") - np.searchsorted(s, lo, "left"))
            got = oracle.count(ot, p_between(ci, lo, hi), lib=lib)
            if got != want:
                fails.append(f"sorted between col {ci}: {got} != {want}")
            want = int(np.searchsorted(s, lo, "left"))
            got = oracle.count(ot, p_cmp(ci, "<", lo), lib=lib)
            if got != want:
                fails.append(f"sorted < col {ci}: {got} != {want}")
            uniq, cnt = np.unique(a, return_counts=True)
            vals = [a[int(i)] for i in rng.integers(0, len(a), 3)]
            vals = [float(v) if ot.types[ci] == "f32" else int(v) for v in vals]
            want = int(sum(cnt[np.searchsorted(uniq, v)] for v in set(vals)))
            got = oracle.count(ot, p_in(ci, vals), lib=lib)
            if got != want:
                fails.append(f"unique-count IN col {ci}: {got} != {want}")
    return fails


def _golden_tree(q, names):
    k = q[0]
    if k in ("and", "or"):
        return (k, [_golden_tree(c, names) for c in q[1]])
    if k == "not":
        return ("not", _golden_tree(q[1], names))
    return (k, names[q[1]]) + tuple(q[2:])


def load_golden_paper_table():
    with open(os.path.join(GOLDEN, "col_vs_row_table.json")) as f:
        g = json.load(f)
    names = {n: i for i, n in enumerate(g["columns"])}
    arrays, types, dicts = [], [], []
    for n, c in g["columns"].items():
        types.append(c["type"])
        arrays.append(np.array(c["values"], dtype=np.int32))
        dicts.append([w.encode() for w in c["dictionary"]] if "dictionary" in c else None)
    queries = [(_golden_tree(q["where"], names), q["count"], q["rows"]) for q in g["queries"]]
    return arrays, types, dicts, queries


def pin_paper_table(lib):
    fails = []
    arrays, types, dicts, queries = load_golden_paper_table()
    t = _table(arrays, types, dicts)
    for tree, want, rows in queries:
        got = oracle.count(t, tree, lib=lib)
        ids = oracle.select(t, tree, lib=lib)
        if got != want or list(ids) != rows:
            fails.append(f"paper table {tree}: {got} {list(ids)} != {want} {rows}")
    return fails


def pin_boolean_identities(lib, n_trees=60):
    fails = []
    rng = np.random.default_rng(11)
    for n in (0, 1, 3, 33, 257):
        tab = dg.tiny_table(n, seed=n)
        ot = oracle.OTable.from_table(tab)
        cnt = lambda tr: oracle.count(ot, tr, lib=lib)
        if cnt(dg.P_TRUE) != n or cnt(dg.P_FALSE) != 0:
            fails.append(f"n={n}: TRUE/FALSE")
        for _ in range(n_trees // 5):
            A = dg.random_tree(tab, rng)
            B = dg.random_tree(tab, rng)
            cA, cB = cnt(A), cnt(B)
            cAB, cAnB = cnt(p_and(A, B)), cnt(p_and(A, p_not(B)))
            if cA != cAB + cAnB:
                fails.append(f"partition n={n}")
            if cnt(p_or(A, B)) != cA + cB - cAB:
                fails.append(f"inclusion-exclusion n={n}")
            if cnt(p_not(p_and(A, B))) != cnt(p_or(p_not(A), p_not(B))):
                fails.append(f"De Morgan n={n}")
            if cnt(p_not(A)) != n - cA:
                fails.append(f"complement n={n}")
            if cnt(p_and(A)) != cA or cnt(p_or(A)) != cA or cnt(("and", [])) != n or cnt(("or", [])) != 0:
                fails.append(f"unary/empty AND-OR n={n}")
        for _ in range(4):
            c = int(rng.integers(0, 4))
            lo, hi = sorted(int(x) for x in rng.integers(-1, 5, 2))
            if cnt(p_between(0, lo, hi)) > cnt(p_between(0, lo - 1, hi + 1)):
                fails.append("BETWEEN widening not monotone")
    return fails


ALL_PINS = [pin_permutation_closed_forms, pin_modulo_closed_forms, pin_float_closed_forms,
            pin_int64_and_widening, pin_like_closed_forms, pin_order_statistics, pin_paper_table,
            pin_boolean_identities]


def run_all(lib):
    out = []
    for p in ALL_PINS:
        try:
            out += [f"{p.__name__}: {f}" for f in p(lib)]
        except Exception as e:            # a mutant may also break the oracle's own consistency checks
            out.append(f"{p.__name__}: raised {type(e).__name__}: {e}")
    return out
