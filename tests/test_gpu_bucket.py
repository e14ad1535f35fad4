"""The column-bucket batch kernel on the GPU against the oracle: exact counts.

Plans are forced onto the bucket kernel (sel_ctx_set_batch_kernel mode 2) and
run over tiny tables of every ragged size, the edge-value table (float32 +-0,
infinities, NaN, denormals, the ends of int32 and int64), config 2's probes
on a 300,001-row table in several launch shapes (tile rows, stages, 8, 11,
15 or 16 consumer warps), several blocks of probes on one table: 2 blocks
(block form: shared bucket search, per-warp bucket buffers, remapped gm
tables) and 3 to 5 blocks (quad form: per-row bucket records, a quarter-warp
per row, quads of 3 blocks and of 1 block), a 10-column table that keeps the
block form, and the five tables of config 3's star in one launch."""
import os

import numpy as np
import pytest
import torch

import datagen as dg
import oracle
import paper_1806_08384_b300 as sel
from tests.test_bucket_host import _edge_table, _edge_trees, _fits

pytestmark = pytest.mark.gpu
THREADS = max(1, min(32, os.cpu_count() or 1))


def _bucket_ctx():
    c = sel.Context()
    c.set_batch_kernel(2)
    return c


def _run(ctx, preds, tables, autotune=False):
    plan = sel.BatchPlan(ctx, preds, tables, autotune=autotune)
    assert plan.info()["kernel"] == "bucket"
    return plan.run()


@pytest.mark.parametrize("n", [0, 1, 2, 31, 32, 33, 255, 256, 257, 4097, 70_001])
def test_random_trees_tiny(dev, n):
    t = dg.tiny_table(n, seed=n)
    ot = oracle.OTable.from_table(t)
    T = sel.Table(t.to(dev).columns)
    rng = np.random.default_rng(500 + n)
    fit = _fits(sel.Table(t.columns), [dg.random_tree(t, rng, depth=3) for _ in range(150)])
    preds = [sel.Predicate(T, tr) for tr in fit]
    want = [oracle.count(ot, tr) for tr in fit]
    for variant in ((16, 1), (8, 2)):
        ctx = _bucket_ctx()
        ctx.set_scan_variant(*variant)
        assert _run(ctx, preds, [T] * len(preds)) == want
        assert _run(ctx, preds[:40], [T] * 40) == want[:40]    # one block (no bucket buffer)


def test_edge_values(dev):
    t = _edge_table()
    ot = oracle.OTable.from_table(t)
    T = sel.Table(t.to(dev).columns)
    trees = _edge_trees()
    preds = [sel.Predicate(T, tr) for tr in trees]
    assert _run(_bucket_ctx(), preds, [T] * len(preds)) == [oracle.count(ot, tr) for tr in trees]


@pytest.fixture(scope="module")
def medium():
    t = dg.gen_table("cfg2", dg.config2_specs(), 300_001, "cuda")
    return t, oracle.OTable.from_table(t), sel.Table(t.columns)


@pytest.mark.parametrize("shape", [(256, 2, 8, 1), (768, 3, 8, 2), (2048, 4, 16, 1), (0, 0, 0, 0), (0, 2, 16, 2),
                                   (16384, 3, 8, 1), (1280, 3, 16, 2), (256, 3, 8, 2), (0, 3, 15, 1), (2816, 3, 11, 2),
                                   (0, 4, 15, 2), (768, 2, 11, 1)])
def test_config2_shapes(medium, shape):
    """Ragged last tile (n = 300,001), tiles with fewer chunks than warps, every
    ring depth, one or two chunks per pass (an odd chunk count leaves the last
    group with one chunk)."""
    t, ot, T = medium
    ctx = _bucket_ctx()
    tile, stages, warps, group = shape
    ctx.set_scan_shape(tile, stages, 0)
    if warps:
        ctx.set_scan_variant(warps, group)
    trees = [dg.config2_predicate(s, seed=k) for s in dg.CONFIG2_TARGETS for k in range(3)]
    preds = [sel.Predicate(T, tr) for tr in trees]
    assert _run(ctx, preds, [T] * len(preds)) == [oracle.count(ot, tr, threads=THREADS) for tr in trees]


@pytest.mark.parametrize("variant", [(8, 1), (16, 1), (8, 2), (16, 2), (15, 1), (11, 2), (11, 1)])
def test_several_blocks_on_one_table(dev, variant):
    """256 probes (4 blocks of 64: one quad), 129 (a quad of 3 blocks, the
    last with 1 probe), 128 (2 blocks: the block form) and 300 random
    estimator-workload probes (5 blocks: 2 quads, the second of 1 block)."""
    t = dg.config5_table(n=1_000_003, device=dev)
    ot = oracle.OTable.from_table(t)
    T = sel.Table(t.columns)
    ctx = _bucket_ctx()
    ctx.set_scan_variant(*variant)
    trees = dg.config5_predicates(256, seed=4)
    preds = [sel.Predicate(T, tr) for tr in trees]
    want = [oracle.count(ot, tr, threads=THREADS) for tr in trees]
    assert _run(ctx, preds, [T] * len(preds)) == want
    assert _run(ctx, preds[:129], [T] * 129) == want[:129]
    assert _run(ctx, preds[:128], [T] * 128) == want[:128]
    t2 = dg.gen_table("cfg2", dg.config2_specs(), 200_000, dev)
    ot2, T2 = oracle.OTable.from_table(t2), sel.Table(t2.columns)
    rng = np.random.default_rng(11)
    trees = [dg.random_dnf_predicate(dg.config2_specs(), rng) for _ in range(300)]
    preds = [sel.Predicate(T2, tr) for tr in trees]
    assert _run(ctx, preds, [T2] * len(preds)) == [oracle.count(ot2, tr, threads=THREADS) for tr in trees]


def test_ten_columns_keep_the_block_form(dev):
    specs = [dg.ColumnSpec(f"c{i}", "i32", "uniform", 0, 50) for i in range(10)]
    t = dg.gen_table("wide10", specs, 200_003, dev)
    ot, T = oracle.OTable.from_table(t), sel.Table(t.columns)
    rng = np.random.default_rng(12)
    trees = [dg.random_dnf_predicate(specs, rng) for _ in range(256)]
    preds = [sel.Predicate(T, tr) for tr in trees]
    assert _run(_bucket_ctx(), preds, [T] * len(preds)) == [oracle.count(ot, tr, threads=THREADS) for tr in trees]


def test_star_schema_one_launch(dev):
    tabs = dg.config3_tables(fact_rows=2_000_000, device=dev)
    ots = [oracle.OTable.from_table(t) for t in tabs]
    Ts = [sel.Table(t.columns) for t in tabs]
    probes = dg.config3_predicates()
    preds = [sel.Predicate(Ts[k], tree) for k, tree in probes]
    tables = [Ts[k] for k, _ in probes]
    want = [oracle.count(ots[k], tree, threads=THREADS) for k, tree in probes]
    plan = sel.BatchPlan(_bucket_ctx(), preds, tables, autotune=True)
    assert plan.info()["kernel"] == "bucket"
    assert plan.run() == want
    assert plan.run() == want                       # graph replay
    out = torch.zeros(len(preds), dtype=torch.int64, device="cuda")
    plan.run(device_out=out)
    torch.cuda.synchronize()
    assert out.cpu().tolist() == want


def test_kernel_modes(medium):
    t, ot, T = medium
    trees = [dg.config2_predicate(s, seed=2) for s in dg.CONFIG2_TARGETS]
    preds = [sel.Predicate(T, tr) for tr in trees]
    want = [oracle.count(ot, tr, threads=THREADS) for tr in trees]
    ctx = sel.Context()
    plan = sel.BatchPlan(ctx, preds, [T] * len(preds), autotune=False)
    assert plan.info()["kernel"] == "bucket"          # the default whenever the probes fit
    assert plan.run() == want
    ctx.set_batch_kernel(1)
    plan = sel.BatchPlan(ctx, preds, [T] * len(preds), autotune=False)
    assert plan.info()["kernel"] == "interpreter"
    assert plan.run() == want
    ctx.set_batch_kernel(2)
    wide = dg.p_or(*[dg.p_cmp(0, "=", k) for k in range(5)])
    wide = dg.p_and(wide, dg.p_or(dg.p_cmp(1, "<", 5), dg.p_cmp(3, ">", dg.f32(10.0))))
    with pytest.raises(sel.SelError) as e:
        sel.BatchPlan(ctx, [sel.Predicate(T, wide)], [T], autotune=False)
    assert e.value.status == sel.SEL_ERR_UNSUPPORTED
    ctx.set_batch_kernel(0)                            # a batch that does not fit runs on the interpreter
    plan = sel.BatchPlan(ctx, preds + [sel.Predicate(T, wide)], [T] * (len(preds) + 1), autotune=False)
    assert plan.info()["kernel"] == "interpreter"
    assert plan.run() == want + [oracle.count(ot, wide, threads=THREADS)]
