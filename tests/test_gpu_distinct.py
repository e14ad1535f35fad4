"""V(sigma_P(R), A) on the GPU (sel_count_distinct) against the oracle
(oracle/join.py): the same distinct count and row count, for every column type,
with and without a pushed-down selection, including the all-ones int64 value
(the hash set's empty marker) and -0.0 / +0.0; and the join-size estimate."""
import numpy as np
import pytest
import torch

import datagen as dg
import oracle
import paper_1806_08384_b300 as sel
from oracle import join

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n", [0, 1, 2, 255, 4097, 100_003])
def test_tiny_tables_every_column(ctx, dev, n):
    t = dg.tiny_table(n, seed=n + 5)
    ot = oracle.OTable.from_table(t)
    T = sel.Table(t.to(dev).columns)
    rng = np.random.default_rng(n)
    for col in range(len(t.columns)):
        assert ctx.count_distinct(T, col) == join.count_distinct(ot, col), col
        for _ in range(4):
            tree = dg.random_tree(t, rng, depth=3)
            assert ctx.count_distinct(T, col, sel.Predicate(T, tree)) == join.count_distinct(ot, col, tree), (col, tree)


def test_marker_value_and_signed_zero(ctx, dev):
    n = 50_000
    rng = np.random.default_rng(3)
    i64 = rng.integers(-3, 3, n).astype(np.int64)          # includes -1: all ones as 64 bits
    f32 = rng.choice(np.array([0.0, -0.0, 2.5, -7.0], np.float32), n)
    i32 = rng.integers(-2, 2, n).astype(np.int32)          # -1 sign-extends to all ones too
    specs = [dg.ColumnSpec("a", "i64", "uniform", -3, 3), dg.ColumnSpec("b", "f32", "uniform", 0.0, 1.0),
             dg.ColumnSpec("c", "i32", "uniform", -2, 2)]
    cols = [dg.Column(s, torch.from_numpy(a).to(dev)) for s, a in zip(specs, (i64, f32, i32))]
    T = sel.Table(cols)
    ot = oracle.OTable([i64, f32, i32], ["i64", "f32", "i32"], [None] * 3)
    for col in range(3):
        assert ctx.count_distinct(T, col) == join.count_distinct(ot, col), col
        tree = dg.p_cmp(2, ">=", 0)
        assert ctx.count_distinct(T, col, sel.Predicate(T, tree)) == join.count_distinct(ot, col, tree), col


def test_config2_medium_and_join_estimate(ctx, dev):
    t = dg.gen_table("cfg2", dg.config2_specs(), 2_000_003, dev)
    ot = oracle.OTable.from_table(t)
    T = sel.Table(t.columns)
    for s in (1e-3, 0.1):
        tree = dg.config2_predicate(s, seed=4)
        p = sel.Predicate(T, tree)
        for col in range(8):
            assert ctx.count_distinct(T, col, p) == join.count_distinct(ot, col, tree, threads=8), (s, col)
    vr, rr = ctx.count_distinct(T, 2, sel.Predicate(T, dg.config2_predicate(0.01, seed=4)))
    vs, rs = ctx.count_distinct(T, 2)
    assert sel.join_size_estimate(rr, rs, vr, vs) == join.join_size_estimate(rr, rs, vr, vs)


@pytest.mark.slow
def test_full_size_key_columns(ctx, dev):
    """300M rows: V of the int64 Zipf key over all rows and under a selection."""
    t = dg.config2_table(device=dev)
    T = sel.Table(t.columns)
    k2 = t.columns[2].data
    assert ctx.count_distinct(T, 2) == (int(torch.unique(k2).numel()), t.n_rows)
    tree = dg.config2_predicate(0.01)
    d, r = ctx.count_distinct(T, 2, sel.Predicate(T, tree))
    st, cnt, cols, ids = ctx.pushdown(sel.Predicate(T, tree), T, [2], r)
    assert cnt == r and d == int(torch.unique(cols[0]).numel())
