"""Batched probes on the GPU: one persistent launch (replayed from a CUDA
graph, shape from the autotuner) gives the same exact counts as separate
sel_count calls and as the oracle."""
import os

import numpy as np
import pytest
import torch

import datagen as dg
import oracle
import paper_1806_08384_b300 as sel

pytestmark = pytest.mark.gpu
THREADS = max(1, min(32, os.cpu_count() or 1))


def test_batch_mixed_tables(ctx, dev):
    tabs = [dg.tiny_table(n, seed=n) for n in (0, 1, 257, 5000, 70_001)]
    ots = [oracle.OTable.from_table(t) for t in tabs]
    Ts = [sel.Table(t.to(dev).columns) for t in tabs]
    rng = np.random.default_rng(5)
    preds, tables, want = [], [], []
    for i in range(60):
        k = int(rng.integers(0, len(tabs)))
        tree = dg.random_tree(tabs[k], rng, depth=3)
        preds.append(sel.Predicate(Ts[k], tree))
        tables.append(Ts[k])
        want.append(oracle.count(ots[k], tree))
    got = ctx.count_batch(preds, tables)
    assert got == want
    assert got == [ctx.count(p, T) for p, T in zip(preds, tables)]


def test_star_schema_batch(ctx, dev):
    """The 64-probe star of config 3 with the fact table cut to 3M rows."""
    tabs = dg.config3_tables(fact_rows=3_000_000, device=dev)
    ots = [oracle.OTable.from_table(t) for t in tabs]
    Ts = [sel.Table(t.columns) for t in tabs]
    probes = dg.config3_predicates()
    preds = [sel.Predicate(Ts[k], tree) for k, tree in probes]
    tables = [Ts[k] for k, _ in probes]
    want = [oracle.count(ots[k], tree, threads=THREADS) for k, tree in probes]
    plan = sel.BatchPlan(ctx, preds, tables, autotune=True)
    info = plan.info()
    assert info["tile_rows"] % 256 == 0 and info["stages"] >= 2 and info["ms"] > 0
    assert plan.run() == want
    assert plan.run() == want                       # graph replay
    out = torch.zeros(len(preds), dtype=torch.int64, device="cuda")
    plan.run(device_out=out)
    torch.cuda.synchronize()
    assert out.cpu().tolist() == want


def test_more_tables_than_one_launch_holds(ctx, dev):
    tabs = [dg.tiny_table(1000 + 37 * i, seed=i) for i in range(11)]
    ots = [oracle.OTable.from_table(t) for t in tabs]
    Ts = [sel.Table(t.to(dev).columns) for t in tabs]
    rng = np.random.default_rng(9)
    preds, tables, want = [], [], []
    for i, t in enumerate(tabs):
        for _ in range(3):
            tree = dg.random_tree(t, rng, depth=3)
            preds.append(sel.Predicate(Ts[i], tree))
            tables.append(Ts[i])
            want.append(oracle.count(ots[i], tree))
    assert sel.BatchPlan(ctx, preds, tables, autotune=False).run() == want


def test_256_probes_one_table(ctx, dev):
    """Config 5's probe set (selectivities 1e-6 .. 0.9) on a 4M-row prefix."""
    t = dg.config5_table(n=4_000_000, device=dev)
    ot = oracle.OTable.from_table(t)
    T = sel.Table(t.columns)
    trees = dg.config5_predicates()
    preds = [sel.Predicate(T, tr) for tr in trees]
    got = sel.BatchPlan(ctx, preds, [T] * len(preds), autotune=True).run()
    want = [oracle.count(ot, tr, threads=THREADS) for tr in trees]
    assert got == want


@pytest.mark.parametrize("autotune", [False, True])
def test_plans_above_256_probes_a_table_run_as_parts(ctx, dev, autotune):
    """600 probes on one table and 40 on another: the plan runs as three
    parts of at most 256 probes a table (the second table's probes all in the
    first part), every part adding into the same counts; interleaved order,
    host and device outputs, graph replay."""
    t1 = dg.gen_table("cfg2", dg.config2_specs(), 200_003, dev)
    t2 = dg.tiny_table(50_001, seed=5, device=dev)
    o1, o2 = oracle.OTable.from_table(t1), oracle.OTable.from_table(t2)
    T1, T2 = sel.Table(t1.columns), sel.Table(t2.columns)
    rng = np.random.default_rng(31)
    trees1 = [dg.random_dnf_predicate(dg.config2_specs(), rng) for _ in range(600)]
    trees2 = [dg.random_tree(t2, rng, depth=3) for _ in range(40)]
    preds, tables, want = [], [], []
    it2 = iter(trees2)
    for k, tr in enumerate(trees1):
        preds.append(sel.Predicate(T1, tr))
        tables.append(T1)
        want.append(oracle.count(o1, tr, threads=THREADS))
        if k % 15 == 0:
            tr2 = next(it2, None)
            if tr2 is not None:
                preds.append(sel.Predicate(T2, tr2))
                tables.append(T2)
                want.append(oracle.count(o2, tr2))
    plan = sel.BatchPlan(ctx, preds, tables, autotune=autotune)
    assert plan.run() == want
    assert plan.run() == want                                   # graph replay
    out = torch.full((len(preds),), -1, dtype=torch.int64, device=dev)
    plan.run(device_out=out)
    torch.cuda.synchronize()
    assert out.cpu().tolist() == want
    assert ctx.count_batch(preds, tables) == want              # the cached-plan entry point
