"""Selection push-down on the GPU (§3.3, Algorithm 1 Execute) against the
oracle: identical projected rows, in ascending row order, identical row ids,
and the maxSize contract (count > max_rows -> SEL_ERR_TOO_LARGE, exact count)."""
import os

import numpy as np
import pytest
import torch

import datagen as dg
import oracle
import paper_1806_08384_b300 as sel

pytestmark = pytest.mark.gpu
THREADS = max(1, min(32, os.cpu_count() or 1))


def check_pushdown(ctx, T, ot, tree, proj, max_rows=None, rowids=True):
    p = sel.Predicate(T, tree)
    want_ids = oracle.select(ot, tree, threads=THREADS)
    max_rows = len(want_ids) if max_rows is None else max_rows
    st, n, cols, ids = ctx.pushdown(p, T, proj, max_rows, rowids=rowids)
    assert n == len(want_ids), tree
    if n > max_rows:
        assert st == sel.SEL_ERR_TOO_LARGE and cols is None
        return n
    assert st == sel.SEL_OK
    if rowids:
        assert np.array_equal(ids.cpu().numpy(), want_ids)
    for c, out in zip(proj, cols):
        assert np.array_equal(out.cpu().numpy(), ot.arrays[c][want_ids]), (tree, c)
    return n


@pytest.fixture(params=[sel.SEL_PD_TWO_PASS, sel.SEL_PD_ONE_PASS], ids=["two_pass", "one_pass"])
def method(request, ctx):
    """Runs the test with each push-down method (the context is the test's own)."""
    ctx.set_pushdown_method(request.param)
    return request.param


@pytest.fixture()
def one_pass(ctx):
    ctx.set_pushdown_method(sel.SEL_PD_ONE_PASS)


@pytest.mark.parametrize("n", [0, 1, 3, 33, 255, 256, 257, 1023, 1025, 4097, 20_000, 32768, 32769, 70_001])
def test_random_trees_tiny(ctx, dev, method, n):
    t = dg.tiny_table(n, seed=n + 7)
    ot = oracle.OTable.from_table(t)
    T = sel.Table(t.to(dev).columns)
    rng = np.random.default_rng(77 + n)
    proj = [0, 1, 2, 3, 4]
    for _ in range(25):
        tree = dg.random_tree(t, rng, depth=4)
        check_pushdown(ctx, T, ot, tree, proj)


@pytest.fixture(scope="module")
def medium():
    t = dg.gen_table("cfg2", dg.config2_specs(), 1_000_003, "cuda")
    return t, oracle.OTable.from_table(t), sel.Table(t.columns)


def proj_cfg2(t):
    return [t.index(c) for c in dg.CONFIG2_PROJECTION]


# The persistent kernel takes 3-chunk groups by default (768 rows: 1536 and
# the default tile), 2-chunk groups for requested tiles that are multiples of
# 512 rows only (1024, 2048, 2560, 3584, 4096, 8192); 256 and 1280 are neither
# and run on the one-CTA-per-tile kernel.
@pytest.mark.parametrize("tile_rows", [0, 256, 768, 1024, 1280, 1536, 2048, 2304, 2560, 3584, 4096, 8192])
def test_config2_selectivities(ctx, medium, method, tile_rows):
    t, ot, T = medium
    ctx.set_scan_shape(tile_rows, 0, 0)
    for s in dg.CONFIG2_TARGETS:
        check_pushdown(ctx, T, ot, dg.config2_predicate(s, seed=11), proj_cfg2(t))


@pytest.mark.parametrize("variant", [(12, 3), (12, 2), (12, 1), (16, 2), (16, 1), (8, 2), (8, 1)])
def test_persistent_variants(ctx, dev, medium, one_pass, variant):
    """Every persistent push-down variant (consumer warps x chunks per warp), on
    the 1,000,003-row table (ragged last super-tile and sub-tile) and on sizes at
    super-tile boundaries."""
    t, ot, T = medium
    ctx.set_scan_variant(*variant)
    for s in (1e-3, 0.1):
        check_pushdown(ctx, T, ot, dg.config2_predicate(s, seed=21), proj_cfg2(t))
    if variant[1] in (1, 3):   # 3-chunk sub-tiles: 42 of them make a 32256-row super-tile
        ctx.set_scan_shape(768, 0, 0)
        check_pushdown(ctx, T, ot, dg.config2_predicate(0.1, seed=22), proj_cfg2(t))
        ctx.set_scan_shape(0, 0, 0)
    for n in (32768, 65537):
        tt = dg.tiny_table(n, seed=n)
        ott = oracle.OTable.from_table(tt)
        TT = sel.Table(tt.to(dev).columns)
        rng = np.random.default_rng(n)
        for _ in range(6):
            check_pushdown(ctx, TT, ott, dg.random_tree(tt, rng, depth=4), [0, 1, 2, 3, 4])


@pytest.mark.parametrize("super_rows", [65536, 131072, 99_840, 256])
def test_super_tile_sizes(ctx, dev, medium, one_pass, super_rows):
    """Super-tiles above the default 32768 rows (the masks and chunk prefixes
    of up to 512 chunks per buffer), one that is no multiple of the sub-tile
    and one smaller than the sub-tile (one sub-tile per super-tile), on the
    1,000,003-row table and on a table of 3 super-tiles and a ragged part."""
    t, ot, T = medium
    ctx.set_pushdown_super_rows(super_rows)
    try:
        for s in (1e-3, 0.1, 0.5):
            check_pushdown(ctx, T, ot, dg.config2_predicate(s, seed=23), proj_cfg2(t))
        tt = dg.tiny_table(3 * 131072 + 777, seed=9)
        ott = oracle.OTable.from_table(tt)
        TT = sel.Table(tt.to(dev).columns)
        rng = np.random.default_rng(super_rows)
        for _ in range(4):
            check_pushdown(ctx, TT, ott, dg.random_tree(tt, rng, depth=4), [0, 1, 2, 3, 4])
    finally:
        ctx.set_pushdown_super_rows(0)


@pytest.mark.parametrize("super_rows", [0, 65536])
def test_four_byte_projections(ctx, dev, medium, method, super_rows):
    """Projections of 4-byte columns only: 6 such columns (two rounds of 4
    loads a write batch), 1 column, and no column with row ids only, at
    selectivities from 1e-4 to 0.5."""
    t, ot, T = medium
    narrow = [t.index(c) for c in ("k0", "k1", "f0", "f1", "d", "s0")]
    ctx.set_pushdown_super_rows(super_rows)
    try:
        for s in (1e-4, 1e-2, 0.1, 0.5):
            tree = dg.config2_predicate(s, seed=31)
            check_pushdown(ctx, T, ot, tree, narrow)
            check_pushdown(ctx, T, ot, tree, [t.index("f1")], rowids=False)
        check_pushdown(ctx, T, ot, dg.config2_predicate(0.1, seed=32), [], rowids=True)
        # a limit inside a write group: the first max_rows rows are written,
        # nothing after them
        tree = dg.config2_predicate(1e-2, seed=33)
        want = oracle.select(ot, tree, threads=THREADS)
        m = len(want) - 77
        outs = [torch.full((m + 64,), 7, dtype=t.columns[j].data.dtype, device="cuda") for j in narrow]
        ids = torch.full((m + 64,), -5, dtype=torch.int64, device="cuda")
        st, cnt, _, _ = ctx.pushdown(sel.Predicate(T, tree), T, narrow, m, out_cols=outs, out_rowids=ids)
        assert st == sel.SEL_ERR_TOO_LARGE and cnt == len(want)
        assert np.array_equal(ids[:m].cpu().numpy(), want[:m]) and bool((ids[m:] == -5).all())
        for j, o in zip(narrow, outs):
            assert np.array_equal(o[:m].cpu().numpy(), ot.arrays[j][want[:m]]) and bool((o[m:] == 7).all())
    finally:
        ctx.set_pushdown_super_rows(0)


def test_bad_super_rows_are_rejected(ctx):
    for r in (-256, 100, 131072 + 256, 1 << 20):
        with pytest.raises(sel.SelError):
            ctx.set_pushdown_super_rows(r)


def test_projection_of_non_predicate_columns_and_no_rowids(ctx, medium, method):
    t, ot, T = medium
    tree = dg.p_between(t.index("f0"), 100.0, 2000.0)
    check_pushdown(ctx, T, ot, tree, [t.index("k2"), t.index("s1"), t.index("f0")], rowids=False)
    check_pushdown(ctx, T, ot, tree, [], rowids=True)


def test_max_rows_contract(ctx, medium, method):
    t, ot, T = medium
    tree = dg.config2_predicate(1e-2, seed=12)
    n = oracle.count(ot, tree, threads=THREADS)
    assert n > 10
    p = sel.Predicate(T, tree)
    proj = proj_cfg2(t)
    # exactly at the limit: materialised (Algorithm 1 throws only when count > maxSize)
    check_pushdown(ctx, T, ot, tree, proj, max_rows=n)
    # one below: rejected, exact count reported, nothing written past max_rows
    m = n - 1
    guard = 64
    outs = [torch.full((m + guard,), 7, dtype=c.data.dtype, device="cuda") for c in (t.columns[j] for j in proj)]
    ids = torch.full((m + guard,), -5, dtype=torch.int64, device="cuda")
    st, cnt, _, _ = ctx.pushdown(p, T, proj, m, out_cols=outs, out_rowids=ids)
    assert st == sel.SEL_ERR_TOO_LARGE and cnt == n
    for o in outs:
        assert bool((o[m:] == 7).all())
    assert bool((ids[m:] == -5).all())
    # ratio 0 (the overhead runs of Ch5): only an empty selection is pushed down
    st, cnt, _, _ = ctx.pushdown(p, T, proj, 0)
    assert st == sel.SEL_ERR_TOO_LARGE and cnt == n
    st, cnt, cols, _ = ctx.pushdown(sel.Predicate(T, dg.P_FALSE), T, proj, 0)
    assert st == sel.SEL_OK and cnt == 0
    # the written prefix of a rejected push-down is still the start of the true result
    want = oracle.select(ot, tree, threads=THREADS)
    assert np.array_equal(ids[:m].cpu().numpy(), want[:m])
    # a limit that cuts the result inside a super-tile: the first max_rows rows
    # in row order are written, nothing after them
    m = n // 3
    ids.fill_(-5)
    for o in outs:
        o.fill_(7)
    st, cnt, _, _ = ctx.pushdown(p, T, proj, m, out_cols=outs, out_rowids=ids)
    assert st == sel.SEL_ERR_TOO_LARGE and cnt == n
    assert np.array_equal(ids[:m].cpu().numpy(), want[:m])
    assert bool((ids[m:] == -5).all())
    for c, o in zip(proj, outs):
        assert np.array_equal(o[:m].cpu().numpy(), ot.arrays[c][want[:m]])
        assert bool((o[m:] == 7).all())


def test_unaligned_columns(ctx, medium, method):
    t, ot, _ = medium
    cols = [dg.Column(c.spec, c.data[3:], c.dictionary) for c in t.columns]
    T = sel.Table(cols)
    sub = oracle.OTable([a[3:] for a in ot.arrays], ot.types, ot.dicts)
    for s in (1e-3, 0.5):
        check_pushdown(ctx, T, sub, dg.config2_predicate(s, seed=13), proj_cfg2(t))


@pytest.mark.parametrize("tile_rows", [1024, 2048, 3584, 4096, 1280, -65536])
def test_lookback_wait_times_out_and_context_recovers(ctx, dev, one_pass, tile_rows):
    """A tile that never publishes makes its successors' bounded waits run out:
    the call returns SEL_ERR_TIMEOUT, and the context works afterwards (the
    persistent kernel, whose look-back unit is a super-tile of up to 32768
    rows -- 32256 for 3584-row sub-tiles --, and the one-CTA-per-tile kernel
    for 1280-row tiles)."""
    t = dg.tiny_table(4 * 32768 + 1000, seed=3)
    ot = oracle.OTable.from_table(t)
    T = sel.Table(t.to(dev).columns)
    tree = dg.p_cmp(0, "<", 2)
    p = sel.Predicate(T, tree)
    if tile_rows < 0:                                # 65536-row super-tiles of the default sub-tile
        ctx.set_pushdown_super_rows(-tile_rows)
    else:
        ctx.set_scan_shape(tile_rows, 0, 0)
    ctx.debug_pushdown_fault(1 if tile_rows < 0 else 2, 50_000_000)   # never publishes; waits give up after 50 ms
    with pytest.raises(sel.SelError) as e:
        ctx.pushdown(p, T, [0], T.n_rows)
    assert e.value.status == sel.SEL_ERR_TIMEOUT
    ctx.debug_pushdown_fault(-1, 0)
    check_pushdown(ctx, T, ot, tree, [0, 1, 2])
    assert ctx.count(p, T) == oracle.count(ot, tree)
    ctx.set_pushdown_super_rows(0)


def test_bad_method_is_rejected(ctx):
    for m in (-1, 3, 100):
        with pytest.raises(sel.SelError):
            ctx.set_pushdown_method(m)


@pytest.mark.parametrize("variant", [(16, 2), (16, 1), (8, 2), (8, 1), (8, 4), (15, 2), (15, 3)])
def test_two_pass_count_variants(ctx, dev, medium, variant):
    """The two-pass method's first pass is the count scan: every variant of it
    leaves the same masks and counts."""
    t, ot, T = medium
    ctx.set_pushdown_method(sel.SEL_PD_TWO_PASS)
    ctx.set_scan_variant(*variant)
    for s in (1e-3, 0.1):
        check_pushdown(ctx, T, ot, dg.config2_predicate(s, seed=24), proj_cfg2(t))
    ctx.set_scan_shape(1792, 0, 0)   # 7 chunks a tile: chunk groups that straddle a segment
    check_pushdown(ctx, T, ot, dg.config2_predicate(0.5, seed=25), proj_cfg2(t))


# Sizes at the two-pass method's boundaries: 16384-row segments (one scatter
# warp each) and groups of 64 segments (1,048,576 rows, one offset each).
@pytest.mark.parametrize("n", [16383, 16384, 16385, 16384 * 64, 16384 * 64 + 1, 2 * 16384 * 64 + 16384 * 3 + 99])
def test_two_pass_segment_boundaries(ctx, dev, n):
    t = dg.tiny_table(n, seed=n % 1000 + 3)
    ot = oracle.OTable.from_table(t)
    T = sel.Table(t.to(dev).columns)
    ctx.set_pushdown_method(sel.SEL_PD_TWO_PASS)
    rng = np.random.default_rng(n)
    for _ in range(6):
        check_pushdown(ctx, T, ot, dg.random_tree(t, rng, depth=4), [0, 1, 2, 3, 4])
    # every row, and every row but the limit
    check_pushdown(ctx, T, ot, dg.P_TRUE, [0, 1, 2, 3, 4])
    st, cnt, _, ids = ctx.pushdown(sel.Predicate(T, dg.P_TRUE), T, [0], n - 5)
    assert st == sel.SEL_ERR_TOO_LARGE and cnt == n


@pytest.mark.slow
def test_config2_full_size(ctx, dev):
    t = dg.config2_table(device=dev)
    T = sel.Table(t.columns)
    ot = oracle.OTable.from_table(t)
    for s in (1e-4, 1e-2, 0.5):
        check_pushdown(ctx, T, ot, dg.config2_predicate(s), proj_cfg2(t))


def test_context_sets_the_l2_fetch_granularity_hint(ctx):
    """sel_ctx_create leaves the process's L2 fetch granularity hint at 32
    bytes (the push-down's gathers read single values)."""
    import ctypes
    rt = ctypes.CDLL("libcudart.so.13")   # the runtime the library loaded
    v = ctypes.c_size_t(0)
    assert rt.cudaDeviceGetLimit(ctypes.byref(v), 5) == 0   # cudaLimitMaxL2FetchGranularity
    assert v.value == 32


def test_split_event_marks_the_end_of_the_count_pass(ctx, medium):
    """sel_ctx_set_pushdown_split_event: the event is recorded between a
    two-pass push-down's count pass and its scatter, so start <= split <= end;
    the one-pass method does not record it; NULL turns the hook off."""
    t, ot, T = medium
    tree = dg.config2_predicate(0.1, seed=41)
    p = sel.Predicate(T, tree)
    proj = proj_cfg2(t)
    n = oracle.count(ot, tree, threads=THREADS)
    outs = [torch.empty(n, dtype=t.columns[j].data.dtype, device="cuda") for j in proj]
    ids = torch.empty(n, dtype=torch.int64, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    a, m, b = (torch.cuda.Event(enable_timing=True) for _ in range(3))
    ctx.set_pushdown_method(sel.SEL_PD_TWO_PASS)
    m.record()
    torch.cuda.synchronize()
    a.record()
    ctx.set_pushdown_split_event(m)
    ctx.pushdown_async(p, T, proj, n, outs, ids, cnt)
    ctx.set_pushdown_split_event(None)
    b.record()
    torch.cuda.synchronize()
    assert int(cnt.item()) == n
    assert 0.0 < a.elapsed_time(m) <= a.elapsed_time(b)
    assert np.array_equal(ids.cpu().numpy(), oracle.select(ot, tree, threads=THREADS))
    # the one-pass method leaves the event where it was
    m2 = torch.cuda.Event(enable_timing=True)
    m2.record()
    torch.cuda.synchronize()
    a.record()
    ctx.set_pushdown_method(sel.SEL_PD_ONE_PASS)
    ctx.set_pushdown_split_event(m2)
    ctx.pushdown_async(p, T, proj, n, outs, ids, cnt)
    ctx.set_pushdown_split_event(None)
    torch.cuda.synchronize()
    assert a.elapsed_time(m2) < 0.0
