"""Exact COUNT on the GPU (§3.1) against the oracle: bit-exact u64 counts."""
import numpy as np
import pytest
import torch

import datagen as dg
import oracle
import paper_1806_08384_b300 as sel

pytestmark = pytest.mark.gpu

TINY_SIZES = [0, 1, 2, 3, 31, 32, 33, 127, 128, 129, 255, 256, 257, 4097, 10_000]


@pytest.mark.parametrize("n", TINY_SIZES)
def test_random_trees_tiny(ctx, dev, n):
    t = dg.tiny_table(n, seed=n)
    ot = oracle.OTable.from_table(t)
    T = sel.Table(t.to(dev).columns)
    rng = np.random.default_rng(1000 + n)
    for _ in range(40):
        tree = dg.random_tree(t, rng, depth=4)
        p = sel.Predicate(T, tree)
        assert ctx.count(p, T) == oracle.count(ot, tree), tree


def _medium(n=300_001):
    return dg.gen_table("cfg2", dg.config2_specs(), n, "cuda")


@pytest.fixture(scope="module")
def medium():
    t = _medium()
    return t, oracle.OTable.from_table(t), sel.Table(t.columns)


@pytest.mark.parametrize("shape", [(256, 2, 1), (512, 3, 2), (2048, 4, 1), (8192, 2, 1), (1024, 6, 3), (0, 0, 0)])
def test_scan_shapes_config2(ctx, medium, shape):
    """Several tiles, every pipeline depth, a ragged last tile (n = 300,001)."""
    t, ot, T = medium
    ctx.set_scan_shape(*shape)
    for s in dg.CONFIG2_TARGETS:
        tree = dg.config2_predicate(s, seed=1)
        p = sel.Predicate(T, tree)
        assert ctx.count(p, T) == oracle.count(ot, tree, threads=8)


VARIANTS = [(8, 1), (8, 2), (16, 1), (16, 2), (8, 4), (15, 2), (15, 3)]


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("shape", [(256, 3, 1), (768, 4, 1), (4096, 3, 1), (1024, 4, 2), (16384, 3, 1),
                                   (512, 2, 1), (1024, 2, 1)])
def test_scan_variants_config2(ctx, medium, variant, shape):
    """Every kernel variant (consumer warps x chunks per pass) on tiles with an
    odd number of chunks (a half-empty last group) and a ragged last tile, and
    on tiles with far fewer chunk groups than warps over a 2-stage ring (most
    warps skip most tiles and come back to a stage one ring later)."""
    t, ot, T = medium
    ctx.set_scan_variant(*variant)
    ctx.set_scan_shape(*shape)
    try:
        for s in (1e-3, 0.1):
            tree = dg.config2_predicate(s, seed=3)
            assert ctx.count(sel.Predicate(T, tree), T) == oracle.count(ot, tree, threads=8)
    finally:
        ctx.set_scan_variant(0, 0)
        ctx.set_scan_shape(0, 0, 0)


@pytest.mark.parametrize("variant", VARIANTS)
def test_narrow_rows_in_large_tiles(ctx, medium, variant):
    """One 4- or 8-byte column per row: tiles of up to 16384 rows (64-128 KB stages)."""
    t, ot, T = medium
    ctx.set_scan_variant(*variant)
    for shape in ((16384, 3, 1), (12288, 2, 1), (0, 0, 0)):
        ctx.set_scan_shape(*shape)
        for tree in (dg.p_between(0, 1 << 28, 1 << 30), dg.p_cmp(2, "<", 1000), dg.p_cmp(3, ">=", dg.f32(5e4)),
                     dg.p_not(dg.p_in(7, [3, 99, 1234, 777, 5]))):
            assert ctx.count(sel.Predicate(T, tree), T) == oracle.count(ot, tree, threads=8), (shape, tree)


@pytest.mark.parametrize("variant", VARIANTS)
def test_variants_tiny(ctx, dev, variant):
    ctx.set_scan_variant(*variant)
    try:
        for n in (1, 255, 257, 513, 4097):
            t = dg.tiny_table(n, seed=77 + n)
            ot = oracle.OTable.from_table(t)
            T = sel.Table(t.to(dev).columns)
            rng = np.random.default_rng(77 + n)
            for _ in range(20):
                tree = dg.random_tree(t, rng, depth=4)
                assert ctx.count(sel.Predicate(T, tree), T) == oracle.count(ot, tree), tree
    finally:
        ctx.set_scan_variant(0, 0)


def test_bad_variant_is_rejected(ctx):
    for w, g in [(4, 1), (8, 3), (0, 1), (32, 2), (16, 4), (15, 4), (11, 3), (12, 4), (13, 1)]:
        with pytest.raises(sel.SelError):
            ctx.set_scan_variant(w, g)


def test_bucket_only_variant_keeps_the_count_default(ctx, medium):
    """11 and 15 consumer warps exist for the batch plans' bucket kernel only,
    12 for the push-down only: the other kernels keep their own defaults."""
    t, ot, T = medium
    tree = dg.config2_predicate(1e-2, seed=5)
    want = oracle.count(ot, tree)
    try:
        for w, g in [(15, 1), (11, 2), (12, 2), (12, 3)]:
            ctx.set_scan_variant(w, g)
            P = sel.Predicate(T, tree)
            assert ctx.count(P, T) == want
            status, n, _, _ = ctx.pushdown(P, T, [0], max_rows=T.n_rows)
            assert status == sel.SEL_OK and n == want
    finally:
        ctx.set_scan_variant(0, 0)


def test_unaligned_columns_take_the_plain_path(ctx, medium):
    t, ot, _ = medium
    cols = [dg.Column(c.spec, c.data[1:], c.dictionary) for c in t.columns]   # base + 4/8 bytes
    T = sel.Table(cols)
    sub = oracle.OTable([a[1:] for a in ot.arrays], ot.types, ot.dicts)
    for s in (1e-3, 0.5):
        tree = dg.config2_predicate(s, seed=2)
        assert ctx.count(sel.Predicate(T, tree), T) == oracle.count(sub, tree, threads=8)


def test_config1_full(ctx, dev):
    t = dg.config1_table(device=dev)
    ot = oracle.OTable.from_table(t)
    T = sel.Table(t.columns)
    for seed in range(5):
        tree = dg.config1_predicate(seed)
        got = ctx.count(sel.Predicate(T, tree), T)
        assert got == oracle.count(ot, tree)
        assert got > 0


def test_constants_and_async(ctx, medium):
    t, ot, T = medium
    n = T.n_rows
    assert ctx.count(sel.Predicate(T, dg.P_TRUE), T) == n
    assert ctx.count(sel.Predicate(T, dg.P_FALSE), T) == 0
    assert ctx.count(sel.Predicate(T, dg.p_or(dg.p_cmp(0, ">=", 0), dg.p_cmp(0, "<", 0))), T) == n
    out = torch.full((1,), -1, dtype=torch.int64, device="cuda")
    tree = dg.config2_predicate(0.1, seed=3)
    ctx.count_async(sel.Predicate(T, tree), T, out)
    torch.cuda.synchronize()
    assert int(out.item()) == oracle.count(ot, tree, threads=8)


@pytest.mark.parametrize("variant", [(16, 1), (8, 2)])
@pytest.mark.parametrize("n_vals", [2, 3, 5, 17, 64, 100, 300])
def test_set_lowerings(ctx, medium, variant, n_vals):
    """IN lists in every lowering (MASK32 word, value compares, perfect hash
    tables, bitmaps, long lists) on int32, int64, float and dictionary
    columns, plain and negated, about two thirds of the values present."""
    t, ot, T = medium
    ctx.set_scan_variant(*variant)
    rng = np.random.default_rng(500 + n_vals)
    for col in range(8):
        data = t.columns[col].data[:50_000].cpu().numpy()
        k = min(n_vals, len(np.unique(data)))
        present = rng.choice(np.unique(data), size=max(1, 2 * k // 3), replace=False).tolist()
        if t.columns[col].type == "f32":
            absent = [dg.f32(float(x)) for x in rng.random(n_vals - len(present)) * 7]
        elif t.columns[col].type == "dict":
            absent = [int(x) for x in rng.integers(0, len(t.columns[col].dictionary), n_vals - len(present))]
        else:
            absent = [int(x) for x in rng.integers(-(2 ** 31), 2 ** 31, n_vals - len(present))]
        vals = present + absent
        for tr in (dg.p_in(col, vals), dg.p_not(dg.p_in(col, vals)),
                   dg.p_and(dg.p_in(col, vals), dg.p_cmp(5, ">", dg.DATE_BASE + 100))):
            assert ctx.count(sel.Predicate(T, tr), T) == oracle.count(ot, tr, threads=8), (col, n_vals)


def test_large_sets_and_prefixes(ctx, medium):
    t, ot, T = medium
    s1 = t.index("s1")
    k2 = t.index("k2")
    d = t.columns[s1].dictionary
    trees = [dg.p_like(s1, d[i][:1].decode()) for i in (0, 3000, 9999)]
    trees += [dg.p_in(s1, list(range(0, 3000, 7))), dg.p_in(s1, list(range(0, 600, 2)) + [9999])]
    vals = [int(v) for v in dg.zipf_rank_values(t.columns[k2].spec)[:50]]
    trees += [dg.p_in(k2, vals), dg.p_not(dg.p_in(k2, vals[:3]))]
    trees += [dg.p_cmp(t.index("f1"), "<", 1.0), dg.p_in(t.index("f0"), [float(x) for x in ot.arrays[3][:20]])]
    for tree in trees:
        assert ctx.count(sel.Predicate(T, tree), T) == oracle.count(ot, tree, threads=8), tree


def test_boolean_identities_on_gpu(ctx, medium):
    """Identities that hold at any size: partition, inclusion-exclusion, complement."""
    t, ot, T = medium
    n = T.n_rows
    A = dg.config2_predicate(0.1, seed=5)
    B = dg.config2_predicate(0.5, seed=6)
    c = lambda tr: ctx.count(sel.Predicate(T, tr), T)
    cA, cB, cAB = c(A), c(B), c(dg.p_and(A, B))
    assert cA == cAB + c(dg.p_and(A, dg.p_not(B)))
    assert c(dg.p_or(A, B)) == cA + cB - cAB
    assert c(dg.p_not(A)) == n - cA
    assert c(dg.p_not(dg.p_and(A, B))) == c(dg.p_or(dg.p_not(A), dg.p_not(B)))


def test_type_mismatch_is_rejected(ctx, medium):
    t, ot, T = medium
    p = sel.Predicate(T, dg.p_cmp(0, "<", 5))
    cols = list(t.columns)
    cols[0] = dg.Column(dg.ColumnSpec("x", "f32", "normal"), cols[3].data, None)
    with pytest.raises(sel.SelError) as e:
        ctx.count(p, sel.Table(cols))
    assert e.value.status == sel.SEL_ERR_TYPE


@pytest.mark.slow
def test_config2_full_size(ctx, dev):
    """300M rows, the five target selectivities, exact vs the (threaded) oracle."""
    t = dg.config2_table(device=dev)
    T = sel.Table(t.columns)
    ot = oracle.OTable.from_table(t)
    for s in dg.CONFIG2_TARGETS:
        tree = dg.config2_predicate(s)
        assert ctx.count(sel.Predicate(T, tree), T) == oracle.count(ot, tree, threads=32)
