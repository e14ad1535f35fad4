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


def test_noalloc_call_captured_in_a_graph_replays_its_own_program(dev):
    """The call can be captured in a CUDA graph once the first call on the
    device is done: the program reaches the scratch array as kernel
    parameters, so the graph holds it.  Between the capture and the replay
    another call with another program rewrites the shared array; the replay
    must still give the captured predicate's rows (against the oracle)."""
    t = dg.gen_table("cfg2", dg.config2_specs(), 300_001, dev)
    ot = oracle.OTable.from_table(t)
    T = sel.Table(t.columns)
    proj = [t.index(c) for c in ("k0", "f0")]
    tree_a, tree_b = dg.config2_predicate(1e-2, seed=41), dg.config2_predicate(0.1, seed=42)
    pa, pb = sel.Predicate(T, tree_a), sel.Predicate(T, tree_b)
    cap = T.n_rows

    def bufs():
        return ([torch.full((cap,), -1, dtype=t.columns[c].data.dtype, device=dev) for c in proj],
                torch.full((cap,), -1, dtype=torch.int64, device=dev),
                torch.zeros(1, dtype=torch.int64, device=dev), torch.zeros(1, dtype=torch.int32, device=dev))

    outs_a, rid_a, cnt_a, err_a = bufs()
    outs_b, rid_b, cnt_b, err_b = bufs()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):          # the first call on the device, outside the capture
        sel.pushdown_noalloc(pa, T, proj, cap, outs_a, rid_a, cnt_a, err_a, stream=s)
    s.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        sel.pushdown_noalloc(pa, T, proj, cap, outs_a, rid_a, cnt_a, err_a, stream=s)
    for o in outs_a:
        o.fill_(-1)
    rid_a.fill_(-1)
    cnt_a.zero_()
    sel.pushdown_noalloc(pb, T, proj, cap, outs_b, rid_b, cnt_b, err_b)   # rewrites the shared array
    torch.cuda.synchronize()
    g.replay()
    torch.cuda.synchronize()
    want = oracle.select(ot, tree_a, threads=8)
    n = int(cnt_a.item())
    assert int(err_a.item()) == 0 and n == len(want)
    assert np.array_equal(rid_a[:n].cpu().numpy(), want) and bool((rid_a[n:] == -1).all())
    for o, c in zip(outs_a, proj):
        assert o[:n].cpu().numpy().tobytes() == ot.arrays[c][want].tobytes()
    want_b = oracle.select(ot, tree_b, threads=8)
    assert int(err_b.item()) == 0 and int(cnt_b.item()) == len(want_b)
    assert np.array_equal(rid_b[:len(want_b)].cpu().numpy(), want_b)
