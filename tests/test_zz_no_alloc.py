"""sel_pushdown_noalloc: the push-down for callers that cannot allocate device
memory (for example code running inside its own device memory manager, where
a nested cudaMalloc would re-enter it).  The entry point keeps its scratch in
a fixed array inside the library and writes only to caller-owned outputs.

Checked against the regular entry point (sel_pushdown) on two calls in a row,
so that the shared array's leftovers from the first call cannot leak into the
second.  Integer results: the comparison is exact.  This file is collected
last; it passes alone in a fresh process and after the other tests."""
import numpy as np
import pytest
import torch

import datagen as dg
import paper_1806_08384_b300 as sel

pytestmark = pytest.mark.gpu


def _expected(ctx, pred, T, proj):
    st, n, cols, ids = ctx.pushdown(pred, T, proj, T.n_rows)
    assert st == sel.SEL_OK
    return n, [c.clone() for c in cols], ids.clone()


def test_noalloc_matches_regular_pushdown_on_two_calls(dev):
    t = dg.gen_table("cfg2", dg.config2_specs(), 1_000_003, dev)
    T = sel.Table(t.columns)
    proj = [t.index(c) for c in dg.CONFIG2_PROJECTION]
    trees = [dg.config2_predicate(0.1, seed=21), dg.config2_predicate(1e-3, seed=22)]
    preds = [sel.Predicate(T, tr) for tr in trees]
    ctx = sel.Context()
    want = [_expected(ctx, p, T, proj) for p in preds]
    cap = T.n_rows
    for p, (n, cols, ids) in zip(preds, want):          # two calls in a row, one shared array
        outs = [torch.full((cap,), -1, dtype=t.columns[c].data.dtype, device=dev) for c in proj]
        rid = torch.full((cap,), -1, dtype=torch.int64, device=dev)
        cnt = torch.full((1,), -1, dtype=torch.int64, device=dev)
        err = torch.full((1,), 7, dtype=torch.int32, device=dev)
        sel.pushdown_noalloc(p, T, proj, cap, outs, rid, cnt, err)
        torch.cuda.synchronize()
        assert int(err.item()) == 0
        assert int(cnt.item()) == n
        assert torch.equal(rid[:n], ids)
        for o, c in zip(outs, cols):
            assert torch.equal(o[:n], c)
        assert bool((rid[n:] == -1).all())


def test_noalloc_rejects_tables_beyond_its_fixed_scratch(dev):
    col = torch.zeros(1024, dtype=torch.int32, device=dev)
    c = dg.Column(dg.ColumnSpec("x", "i32", "uniform", 0, 4), col, None)
    big = sel.Table([c], n_rows=600_000_000)           # descriptor only: rejected before any launch
    p = sel.Predicate(big, dg.p_cmp(0, "<", 2))
    cnt = torch.zeros(1, dtype=torch.int64, device=dev)
    with pytest.raises(sel.SelError) as e:
        sel.pushdown_noalloc(p, big, [0], 10, [col], None, cnt)
    assert e.value.status == sel.SEL_ERR_UNSUPPORTED
    assert "tiles" in str(e.value)
