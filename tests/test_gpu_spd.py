"""Algorithm 1 EvaluateAndPushDown in the library (sel_evaluate_and_push_down)
against its oracle (oracle/spd.py): the same decision for every relation, the
same exact counts and maxSize, and for pushed relations the same projected
rows in the same order."""
import numpy as np
import pytest

import datagen as dg
import oracle
import paper_1806_08384_b300 as sel
from oracle import spd

pytestmark = pytest.mark.gpu


def check(ctx, tables, trees, projs, min_size, ratio, max_rows=0):
    T = [sel.Table(t.columns) for t in tables]
    preds = [sel.Predicate(Ti, tr) if tr is not None else None for Ti, tr in zip(T, trees)]
    got = sel.evaluate_and_push_down(ctx, list(zip(T, preds, projs)), min_table_size=min_size,
                                     max_selectivity=ratio, max_rows=max_rows)
    want = spd.evaluate_and_push_down([(oracle.OTable.from_table(t), tr, p) for t, tr, p in zip(tables, trees, projs)],
                                      min_size, ratio, max_rows, threads=8)
    for i, (g, w) in enumerate(zip(got, want)):
        assert (g["decision"], g["count"], g["max_size"]) == (w["decision"], w["count"], w["max_size"]), i
        if w["decision"] == "pushed":
            assert np.array_equal(g["rowids"].cpu().numpy(), w["rowids"]), i
            for a, b in zip(g["columns"], w["columns"]):
                assert np.array_equal(a.cpu().numpy(), b), i
    return [g["decision"] for g in got]


@pytest.mark.parametrize("seed", range(4))
def test_random_relation_sets(ctx, dev, seed):
    rng = np.random.default_rng(seed)
    sizes = [int(x) for x in rng.choice([100, 5_000, 40_000, 70_001, 150_000], size=6)]
    tables = [dg.tiny_table(n, seed=seed * 10 + i, device=dev) for i, n in enumerate(sizes)]
    trees = [None if rng.random() < 0.15 else dg.random_tree(t, rng, depth=3) for t in tables]
    projs = [[0, 1, 2, 3, 4][: int(rng.integers(1, 6))] for _ in tables]
    seen = check(ctx, tables, trees, projs, min_size=1_000, ratio=float(rng.choice([0.05, 0.3, 0.7])))
    assert "probe" in seen


def test_star_schema_decisions(ctx, dev):
    """Config-3-shaped star with the fact table cut to 3M rows: the largest
    relation (here the 16M-row dimension) is probed, the 2k-row dimension is
    skipped, each other relation is pushed down or reverted by its count."""
    tabs = dg.config3_tables(fact_rows=3_000_000, device=dev)
    probes = dg.config3_predicates()
    trees = [next(tr for ti, tr in probes if ti == k) for k in range(len(tabs))]
    projs = [[0, 1]] * len(tabs)
    largest = int(np.argmax([t.n_rows for t in tabs]))
    for kw in ({"ratio": 0.05}, {"ratio": 0.0, "max_rows": 50_000}):
        seen = check(ctx, tabs, trees, projs, min_size=10_000, **kw)
        assert seen[largest] == "probe" and seen[1] == "too_small"
        assert all(d in ("pushed", "reverted") for i, d in enumerate(seen) if i not in (largest, 1))
