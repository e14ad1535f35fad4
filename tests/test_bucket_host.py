"""The column-bucket form of a batch of probes, evaluated on the CPU from the
same tables the GPU kernel reads (sel_debug_bucket_count_host), against the
oracle: exact counts, CPU only.

This checks everything of the form except the device code: the DNF
conversion of compiled programs, every leaf kind's change points in the raw
bit order of its column (including float32 +-0, infinities, NaN, denormals
and the ends of the int32 and int64 ranges), the bucket search, the blocks of
64 probes, the remap of global to local buckets and the per-field counting."""
import math

import numpy as np
import pytest
import torch

import datagen as dg
import oracle
import paper_1806_08384_b300 as sel
from datagen import p_and, p_between, p_cmp, p_in, p_not, p_or


def _host_counts(preds, T):
    return sel.debug_bucket_count_host(preds, T)


def _quads(preds, T):
    return sel.debug_bucket_count_host(preds, T, with_quads=True)[2]


def _fits(T, trees):
    """The trees whose programs fit the form (each checked alone), in order."""
    out = []
    for tr in trees:
        try:
            _host_counts([sel.Predicate(T, tr)], T)
            out.append(tr)
        except sel.SelError as e:
            assert e.status == sel.SEL_ERR_UNSUPPORTED
    return out


@pytest.mark.parametrize("n", [0, 1, 31, 257, 4097])
def test_random_trees_tiny(n):
    t = dg.tiny_table(n, seed=n)
    ot = oracle.OTable.from_table(t)
    T = sel.Table(t.columns)
    rng = np.random.default_rng(77 + n)
    trees = [dg.random_tree(t, rng, depth=3) for _ in range(300)]
    fit = _fits(T, trees)
    assert len(fit) >= 200            # most depth-3 trees have at most 4 AND-groups
    preds = [sel.Predicate(T, tr) for tr in fit]
    got, blocks = _host_counts(preds, T)
    assert blocks == (len(fit) + 63) // 64
    want = [oracle.count(ot, tr) for tr in fit]
    assert got == want
    # 3 or more blocks take the quad form (here 4 blocks, one quad); 2 blocks
    # the block form with remapped tables
    assert _quads(preds, T) == (blocks + 3) // 4 and blocks >= 3
    got2, blocks2 = _host_counts(preds[:128], T)
    assert blocks2 == 2 and _quads(preds[:128], T) == 0 and got2 == want[:128]
    got3 = _host_counts(preds[:129], T)[0]      # a quad of 3 blocks, the last of 1 probe
    assert _quads(preds[:129], T) == 1 and got3 == want[:129]


def _edge_table():
    """Columns whose values sit on every edge the bit-order buckets have."""
    f = np.array([0.0, -0.0, np.inf, -np.inf, np.nan, -np.nan, 1e-45, -1e-45, 1.0, -1.0, 2.0, -2.0,
                  np.float32(1.0) + np.float32(2 ** -23), np.float32(3.4028235e38), -np.float32(3.4028235e38),
                  0.5, -0.5, 1.5], np.float32)
    i = np.array([-2 ** 31, 2 ** 31 - 1, -1, 0, 1, 2, 5, -5, 7, 8, 100, -100, 2 ** 30, -2 ** 30,
                  3, 4, 6, 9], np.int32)
    l = np.array([-2 ** 63, 2 ** 63 - 1, -1, 0, 1, 2 ** 32, -2 ** 32, 2 ** 32 + 1, 5, -5, 7, 1 << 40,
                  -(1 << 40), 3, 4, 6, 8, 9], np.int64)
    reps = 40
    rng = np.random.default_rng(5)
    cols = []
    for arr in (f, i, l):
        cols.append(np.concatenate([np.tile(arr, reps), rng.permutation(np.tile(arr, 3))]))
    specs = [dg.ColumnSpec("f", "f32", "uniform", 0.0, 1.0), dg.ColumnSpec("i", "i32", "uniform", 0, 4),
             dg.ColumnSpec("l", "i64", "uniform", 0, 4)]
    return dg.Table("edges", [dg.Column(s, torch.from_numpy(np.ascontiguousarray(a)), None)
                              for s, a in zip(specs, cols)])


def _edge_trees():
    fc = [0.0, -0.0, math.inf, -math.inf, dg.f32(1e-45), dg.f32(-1e-45), 1.0, -1.0, 2.0, 0.5, dg.f32(3.4028235e38)]
    ic = [-2 ** 31, 2 ** 31 - 1, -1, 0, 1, 5, 7, 8, -5, 2 ** 30]
    lc = [-2 ** 63, 2 ** 63 - 1, -1, 0, 1, 2 ** 32, -2 ** 32, 5, 1 << 40]
    trees = []
    for col, cs in ((0, fc), (1, ic), (2, lc)):
        for c in cs:
            for op in ("=", "<>", "<", "<=", ">", ">="):
                trees.append(p_cmp(col, op, c))
        for a in cs:
            for b in cs:
                trees.append(p_between(col, a, b))
        trees.append(p_in(col, cs[:4]))
        trees.append(p_in(col, cs[3:]))
        trees.append(p_not(p_in(col, cs[1:6])))
        trees.append(p_in(col, cs + cs[:2]))      # duplicates
    trees.append(p_in(1, list(range(0, 40, 3))))   # a sparse set: hash table
    trees.append(p_in(1, list(range(-3, 29))))     # consecutive: one range
    trees.append(p_in(1, [0, 2, 5, 9, 30]))        # within 32 values: one word
    trees.append(p_in(1, list(range(0, 600, 7)) + [2 ** 30]))   # large sparse set
    trees.append(p_in(2, list(range(-40, 40, 9))))  # int64 hash table
    trees.append(p_in(0, [0.0, 1.0, -2.0, math.inf]))
    trees.append(p_or(p_and(p_cmp(0, ">=", -1.0), p_cmp(0, "<", 2.0)), p_not(p_cmp(1, "=", 5))))
    trees.append(p_and(p_cmp(0, ">", -math.inf), p_cmp(0, "<", math.inf)))   # every number, no NaN
    trees.append(p_not(p_and(p_cmp(0, ">", -math.inf), p_cmp(0, "<", math.inf))))
    trees.append(dg.P_TRUE)
    trees.append(dg.P_FALSE)
    trees.append(p_not(dg.P_TRUE))
    return trees


def test_edge_values_of_every_leaf_kind():
    t = _edge_table()
    ot = oracle.OTable.from_table(t)
    T = sel.Table(t.columns)
    trees = _edge_trees()
    preds = [sel.Predicate(T, tr) for tr in trees]
    got, blocks = _host_counts(preds, T)
    assert blocks > 1
    want = [oracle.count(ot, tr) for tr in trees]
    bad = [(tr, g, w) for tr, g, w in zip(trees, got, want) if g != w]
    assert bad == []


def test_one_probe_at_a_time_equals_the_batch():
    """Each probe alone (one block, identity remap) equals its count inside a
    batch of several blocks (shared bucket search, remapped gm tables)."""
    t = _edge_table()
    T = sel.Table(t.columns)
    trees = _edge_trees()[::7]
    preds = [sel.Predicate(T, tr) for tr in trees]
    batch, blocks = _host_counts(preds * 3, T)
    assert blocks >= 2
    alone = [_host_counts([p], T)[0][0] for p in preds]
    assert batch == alone * 3


def test_config_shaped_batches():
    """Config 2's OR of 3 ANDs and config 5's 256 probes (4 blocks) on prefixes."""
    t2 = dg.gen_table("cfg2", dg.config2_specs(), 30_011, "cpu")
    ot2, T2 = oracle.OTable.from_table(t2), sel.Table(t2.columns)
    trees = [dg.config2_predicate(s, seed=k) for s in dg.CONFIG2_TARGETS for k in range(4)]
    got, _ = _host_counts([sel.Predicate(T2, tr) for tr in trees], T2)
    assert got == [oracle.count(ot2, tr) for tr in trees]
    t5 = dg.gen_table("cfg5", dg.config5_specs(), 20_003, "cpu")
    ot5, T5 = oracle.OTable.from_table(t5), sel.Table(t5.columns)
    trees = dg.config5_predicates(256, seed=3)
    got, blocks = _host_counts([sel.Predicate(T5, tr) for tr in trees], T5)
    assert blocks == 4
    assert got == [oracle.count(ot5, tr) for tr in trees]
    assert _quads([sel.Predicate(T5, tr) for tr in trees], T5) == 1
    rng = np.random.default_rng(9)
    trees = [dg.random_dnf_predicate(dg.config2_specs(), rng) for _ in range(300)]
    got, blocks = _host_counts([sel.Predicate(T2, tr) for tr in trees], T2)
    assert blocks == 5
    assert _quads([sel.Predicate(T2, tr) for tr in trees], T2) == 2     # the second quad holds 1 block
    assert got == [oracle.count(ot2, tr) for tr in trees]


def test_quad_form_needs_at_most_eight_columns():
    """A table of 10 columns keeps the block form at 4 blocks; 8 columns take
    quads (rows of a column no probe of a quad reads are all ones)."""
    specs = [dg.ColumnSpec(f"c{i}", "i32", "uniform", 0, 50) for i in range(10)]
    t = dg.gen_table("wide10", specs, 5_003, "cpu")
    ot, T = oracle.OTable.from_table(t), sel.Table(t.columns)
    rng = np.random.default_rng(12)
    trees = [dg.random_dnf_predicate(specs, rng) for _ in range(256)]
    preds = [sel.Predicate(T, tr) for tr in trees]
    got, blocks = _host_counts(preds, T)
    assert blocks == 4 and _quads(preds, T) == 0
    assert got == [oracle.count(ot, tr) for tr in trees]
    t8 = dg.gen_table("wide8", specs[:8], 5_003, "cpu")
    ot8, T8 = oracle.OTable.from_table(t8), sel.Table(t8.columns)
    trees = [dg.random_dnf_predicate(specs[:8], rng) for _ in range(200)]
    trees += [dg.p_between(0, 3, 9)] * 64      # a fourth block that reads one column only
    preds = [sel.Predicate(T8, tr) for tr in trees]
    got, blocks = _host_counts(preds, T8)
    assert blocks == 5 and _quads(preds, T8) == 2
    assert got == [oracle.count(ot8, tr) for tr in trees]


def test_programs_beyond_four_groups_are_refused():
    t = dg.tiny_table(100)
    T = sel.Table(t.columns)
    wide = p_or(*[p_cmp(0, "=", k) for k in range(3)], p_cmp(1, "<", 0), p_cmp(2, ">", 1.0))
    with pytest.raises(sel.SelError) as e:
        _host_counts([sel.Predicate(T, wide)], T)
    assert e.value.status == sel.SEL_ERR_UNSUPPORTED
    assert "groups" in str(e.value)


def test_spread_boundaries_and_extreme_values():
    """Many ranges spread over the whole int32 and float32 domains (the cell
    search: a cell table over the boundaries' span, at most 3 boundaries per
    cell) with data at and around every boundary and at the type's ends."""
    rng = np.random.default_rng(21)
    lo = rng.integers(-2 ** 31, 2 ** 31 - 2 ** 24, 60)
    hi = lo + rng.integers(0, 2 ** 24, 60)
    flo = np.sort(rng.normal(0, 3, (60, 2)).astype(np.float32), axis=1)
    edge_i = np.concatenate([lo, hi, lo - 1, hi + 1, [-2 ** 31, -1, 0, 1, 2 ** 31 - 1]]).clip(-2 ** 31, 2 ** 31 - 1)
    ivals = np.concatenate([edge_i, rng.integers(-2 ** 31, 2 ** 31, 4000)]).astype(np.int32)
    edge_f = np.concatenate([flo.ravel(), np.nextafter(flo.ravel(), np.float32(np.inf)),
                             np.nextafter(flo.ravel(), np.float32(-np.inf)),
                             np.array([0.0, -0.0, np.inf, -np.inf, np.nan], np.float32)])
    fvals = np.concatenate([edge_f, rng.normal(0, 3, ivals.shape[0] - edge_f.shape[0])]).astype(np.float32)
    specs = [dg.ColumnSpec("i", "i32", "uniform", 0, 4), dg.ColumnSpec("f", "f32", "uniform", 0.0, 1.0)]
    t = dg.Table("spread", [dg.Column(specs[0], torch.from_numpy(ivals), None),
                            dg.Column(specs[1], torch.from_numpy(fvals), None)])
    ot, T = oracle.OTable.from_table(t), sel.Table(t.columns)
    trees = [p_between(0, int(a), int(b)) for a, b in zip(lo, hi)]
    trees += [p_between(1, float(a), float(b)) for a, b in flo]
    trees += [p_or(p_between(0, int(lo[k]), int(hi[k])), p_not(p_between(1, float(flo[k][0]), float(flo[k][1]))))
              for k in range(10)]
    got, _ = _host_counts([sel.Predicate(T, tr) for tr in trees], T)
    assert got == [oracle.count(ot, tr) for tr in trees]
