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


@pytest.mark.parametrize("seed", range(3))
def test_join_count_tiny(ctx, dev, seed):
    rng = np.random.default_rng(seed)
    tr = dg.tiny_table(int(rng.integers(0, 30_000)), seed=seed)
    ts = dg.tiny_table(int(rng.integers(0, 3_000)), seed=seed + 100)
    otr, ots = oracle.OTable.from_table(tr), oracle.OTable.from_table(ts)
    Tr, Ts = sel.Table(tr.to(dev).columns), sel.Table(ts.to(dev).columns)
    for col in range(5):   # same-type key columns: i32, i64, f32, date, dict
        for _ in range(3):
            pr = dg.random_tree(tr, rng, depth=3) if rng.random() < 0.8 else None
            ps = dg.random_tree(ts, rng, depth=3) if rng.random() < 0.8 else None
            got = ctx.join_count(Tr, col, sel.Predicate(Tr, pr) if pr else None, Ts, col,
                                 sel.Predicate(Ts, ps) if ps else None)
            assert got == join.join_count(otr, col, pr, ots, col, ps), (col, pr, ps)


def test_join_count_star_dimension(ctx, dev):
    """Fact a0 (uniform over 2^31) would rarely meet a dimension key: join the fact's
    Zipf column a1 (1000 values) with each dimension's key under their predicates."""
    tabs = dg.config3_tables(fact_rows=2_000_000, device=dev)
    ot = [oracle.OTable.from_table(t) for t in tabs]
    T = [sel.Table(t.columns) for t in tabs]
    probes = dg.config3_predicates()
    fact_tree = next(tr for ti, tr in probes if ti == 0)
    for k in range(1, len(tabs)):
        dim_tree = next(tr for ti, tr in probes if ti == k)
        got = ctx.join_count(T[0], 1, sel.Predicate(T[0], fact_tree), T[k], 0, sel.Predicate(T[k], dim_tree))
        assert got == join.join_count(ot[0], 1, fact_tree, ot[k], 0, dim_tree, threads=8), k


def test_join_count_type_rules(ctx, dev):
    t = dg.tiny_table(100, seed=1)
    T = sel.Table(t.to(dev).columns)
    with pytest.raises(sel.SelError) as e:
        ctx.join_count(T, 0, None, T, 2, None)       # int32 with float32
    assert e.value.status == sel.SEL_ERR_TYPE
    with pytest.raises(sel.SelError) as e:
        ctx.join_count(T, 0, None, T, 1, None)       # int32 with int64
    assert e.value.status == sel.SEL_ERR_UNSUPPORTED
