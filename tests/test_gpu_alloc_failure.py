"""Failure detection without a GPU fault: an allocation made to fail on the
host (sel_debug_fail_allocation) is reported as SEL_ERR_OOM by every entry
point that allocates -- context creation, a predicate's first upload, batch
plan creation, the push-down's scratch, distinct counts, join counts and the
learned estimator -- and the context keeps working afterwards (the same call
then succeeds and is exact against the oracle)."""
import numpy as np
import pytest
import torch

import datagen as dg
import oracle
import paper_1806_08384_b300 as sel

pytestmark = pytest.mark.gpu


@pytest.fixture()
def small(dev):
    t = dg.gen_table("cfg2", dg.config2_specs(), 100_003, dev)
    yield t, oracle.OTable.from_table(t), sel.Table(t.columns)
    sel.debug_fail_allocation(0)


def _oom(fn):
    with pytest.raises(sel.SelError) as e:
        fn()
    assert e.value.status == sel.SEL_ERR_OOM, e.value


@pytest.mark.parametrize("nth", [1, 2, 3])
def test_context_creation(small, nth):
    sel.debug_fail_allocation(nth)
    _oom(lambda: sel.Context())
    sel.debug_fail_allocation(0)
    ctx = sel.Context()
    t, ot, T = small
    tree = dg.config2_predicate(1e-2)
    assert ctx.count(sel.Predicate(T, tree), T) == oracle.count(ot, tree)


def test_count_pushdown_and_plans(small):
    t, ot, T = small
    trees = [dg.config2_predicate(s) for s in dg.CONFIG2_TARGETS]
    want = [oracle.count(ot, tr) for tr in trees]
    ctx = sel.Context()
    p = sel.Predicate(T, trees[0])
    sel.debug_fail_allocation(1)                    # the count buffer of a fresh context
    _oom(lambda: ctx.count(p, T))
    assert ctx.count(p, T) == want[0]
    q = sel.Predicate(T, trees[1])                  # first use of this predicate: its upload
    sel.debug_fail_allocation(1)
    _oom(lambda: ctx.count(q, T))
    assert ctx.count(q, T) == want[1]
    proj = [t.index(c) for c in dg.CONFIG2_PROJECTION]
    fresh = sel.Context()
    fresh.count(p, T)
    sel.debug_fail_allocation(1)                    # the push-down's scratch (row masks and counts)
    _oom(lambda: fresh.pushdown(p, T, proj, want[0]))
    st, n, cols, ids = fresh.pushdown(p, T, proj, want[0])
    assert st == sel.SEL_OK and n == want[0]
    assert np.array_equal(ids.cpu().numpy(), oracle.select(ot, trees[0]))
    preds = [sel.Predicate(T, tr) for tr in trees]
    for nth in (1, 2, 3):                           # program blob, counts, bucket blob
        sel.debug_fail_allocation(nth)
        _oom(lambda: sel.BatchPlan(ctx, preds, [T] * len(preds), autotune=False))
    sel.debug_fail_allocation(0)
    assert sel.BatchPlan(ctx, preds, [T] * len(preds), autotune=False).run() == want


def test_distinct_join_and_estimator(small):
    t, ot, T = small
    k = t.index("k2")
    pred = sel.Predicate(T, dg.config2_predicate(1e-1))
    ctx = sel.Context()
    ctx.count(pred, T)
    sel.debug_fail_allocation(1)
    _oom(lambda: ctx.count_distinct(T, k, pred))
    d, r = ctx.count_distinct(T, k, pred)
    assert d == len(np.unique(t.columns[k].data.cpu().numpy()[oracle.select(ot, dg.config2_predicate(1e-1))]))
    ctx2 = sel.Context()
    ctx2.count(pred, T)
    sel.debug_fail_allocation(1)
    _oom(lambda: ctx2.join_count(T, 0, pred, T, 0, None))
    c, _, _ = ctx2.join_count(T, 0, pred, T, 0, None)
    assert c >= r
    sel.debug_fail_allocation(1)
    _oom(lambda: sel.Estimator(ctx, T, sample_rows=1024, seed=1))
    est = sel.Estimator(ctx, T, sample_rows=1024, seed=1)
    two = sel.Predicate(T, dg.p_and(dg.p_cmp(0, "<", 1 << 30), dg.p_cmp(3, "<", dg.f32(100.0))))
    feat, ok = est.featurize([two])     # an AND of 2 leaves has a feature form
    assert bool(ok[0])


def test_bad_arming_is_rejected():
    with pytest.raises(sel.SelError) as e:
        sel.debug_fail_allocation(-1)
    assert e.value.status == sel.SEL_ERR_INVALID_ARG
