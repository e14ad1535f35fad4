"""sel_pushdown_noalloc: the push-down for callers that cannot allocate device
memory (for example code running inside its own device memory manager, where
a nested cudaMalloc would re-enter it).  The entry point keeps its scratch in
a fixed array inside the library and writes only to caller-owned outputs.

Checked on two calls in a row, so that the shared array's leftovers from the
first call cannot leak into the second: against the CPU oracle (row ids and
every projected value, bit for bit) and against the regular entry point
(sel_pushdown).  Integer and byte results: the comparison is exact.  This file
is collected last; it passes alone in a fresh process and after the other
tests."""
import numpy as np
import pytest
import torch

import datagen as dg
import oracle
import paper_1806_08384_b300 as sel

pytestmark = pytest.mark.gpu


def _regular(ctx, pred, T, proj):
    st, n, cols, ids = ctx.pushdown(pred, T, proj, T.n_rows)
    assert st == sel.SEL_OK
    return n, [c.clone() for c in cols], ids.clone()


def test_noalloc_matches_oracle_and_regular_pushdown_on_two_calls(dev):
    t = dg.gen_table("cfg2", dg.config2_specs(), 1_000_003, dev)
    ot = oracle.OTable.from_table(t)
    T = sel.Table(t.columns)
    proj = [t.index(c) for c in dg.CONFIG2_PROJECTION]
    trees = [dg.config2_predicate(0.1, seed=21), dg.config2_predicate(1e-3, seed=22)]
    preds = [sel.Predicate(T, tr) for tr in trees]
    ctx = sel.Context()
    regular = [_regular(ctx, p, T, proj) for p in preds]
    cap = T.n_rows
    for tr, p, (n_reg, cols_reg, ids_reg) in zip(trees, preds, regular):   # two calls, one shared array
        want_ids = oracle.select(ot, tr)
        outs = [torch.full((cap,), -1, dtype=t.columns[c].data.dtype, device=dev) for c in proj]
        rid = torch.full((cap,), -1, dtype=torch.int64, device=dev)
        cnt = torch.full((1,), -1, dtype=torch.int64, device=dev)
        err = torch.full((1,), 7, dtype=torch.int32, device=dev)
        sel.pushdown_noalloc(p, T, proj, cap, outs, rid, cnt, err)
        torch.cuda.synchronize()
        n = int(cnt.item())
        assert int(err.item()) == 0
        assert n == len(want_ids) == n_reg
        got_ids = rid[:n].cpu().numpy()
        assert np.array_equal(got_ids, want_ids)
        assert torch.equal(rid[:n], ids_reg)
        for o, c, r in zip(outs, proj, cols_reg):
            got = o[:n].cpu().numpy()
            want = ot.arrays[c][want_ids]
            assert got.dtype == want.dtype and got.tobytes() == want.tobytes()
            assert torch.equal(o[:n], r)
        assert bool((rid[n:] == -1).all())


def test_noalloc_requires_the_error_output(dev):
    t = dg.gen_table("cfg1", dg.config1_specs(), 4096, dev)
    T = sel.Table(t.columns)
    p = sel.Predicate(T, dg.p_cmp(0, "<", 500_000))
    out = torch.zeros(4096, dtype=torch.int32, device=dev)
    cnt = torch.zeros(1, dtype=torch.int64, device=dev)
    with pytest.raises(sel.SelError) as e:
        sel.pushdown_noalloc(p, T, [0], 4096, [out], None, cnt, None)
    assert e.value.status == sel.SEL_ERR_INVALID_ARG


def test_noalloc_rejects_tables_beyond_its_fixed_scratch(dev):
    col = torch.zeros(1024, dtype=torch.int32, device=dev)
    c = dg.Column(dg.ColumnSpec("x", "i32", "uniform", 0, 4), col, None)
    big = sel.Table([c], n_rows=600_000_000)           # descriptor only: rejected before any launch
    p = sel.Predicate(big, dg.p_cmp(0, "<", 2))
    cnt = torch.zeros(1, dtype=torch.int64, device=dev)
    err = torch.zeros(1, dtype=torch.int32, device=dev)
    with pytest.raises(sel.SelError) as e:
        sel.pushdown_noalloc(p, big, [0], 10, [col], None, cnt, err)
    assert e.value.status == sel.SEL_ERR_UNSUPPORTED
    assert "tiles" in str(e.value)
