"""The learned estimator on the GPU against its CPU oracle (oracle/mlp.py).

Features are compared bit for bit (after the oracle's values are rounded to
BF16 like the GPU's); the forward pass, the gradients of the Gaussian NLL and
the Adam step within the tolerance the arithmetic allows: FP32 accumulation
in a different order plus BF16 rounding points that may flip by one BF16 ulp,
so |gpu - oracle| <= 2e-2 * (1 + |oracle|) element-wise for outputs and
<= 2e-2 * max|oracle| per tensor for gradients.  The gate is compared with the
oracle's gate, its exact fallbacks with oracle.count."""
import math

import numpy as np
import pytest
import torch

import datagen as dg
import oracle
from oracle import mlp as om
import paper_1806_08384_b300 as sel
from paper_1806_08384_b300 import baselines

pytestmark = pytest.mark.gpu
M = 4096
SEED = 20180612


@pytest.fixture(scope="module")
def setup():
    t = dg.gen_table("cfg2", dg.config2_specs(), 400_000, "cuda")
    T = sel.Table(t.columns)
    ctx = sel.Context()
    est = sel.Estimator(ctx, T, sample_rows=M, seed=SEED)
    cdfs = [om.CDF(c.data.cpu().numpy(), SEED, i, M) for i, c in enumerate(t.columns)]
    dicts = [c.dictionary for c in t.columns]
    rng = np.random.default_rng(7)
    trees = [dg.random_dnf_predicate(dg.config2_specs(), rng) for _ in range(600)]
    trees += [dg.config2_predicate(s, seed=k) for s in dg.CONFIG2_TARGETS for k in range(3)]
    trees += [dg.p_and(dg.p_or(dg.p_cmp(0, "<", 5), dg.p_cmp(1, ">", 7)), dg.p_cmp(3, "<", 1.0)),   # not DNF
              dg.p_or(*[dg.p_cmp(i % 8, ">=", 0) for i in range(4)])]                              # 4 groups
    return t, T, ctx, est, cdfs, dicts, trees


def test_features_bit_exact(setup):
    t, T, ctx, est, cdfs, dicts, trees = setup
    preds = [sel.Predicate(T, tr) for tr in trees]
    feat, ok = est.featurize(preds)
    got = feat.float().cpu().numpy()
    okh = ok.cpu().numpy().astype(bool)
    for i, tr in enumerate(trees):
        f, fok = om.featurize(tr, cdfs, dicts)
        assert okh[i] == fok, tr
        want = om.bf16_round(f)
        other = np.ones(144, bool)
        other[23::24] = False
        assert np.array_equal(got[i][other], want[other]), (tr, np.nonzero(got[i] != want))
        # the log-selectivity term: both sides round a float64 log; allow one BF16 ulp
        ls_g, ls_w = got[i][23::24], want[23::24]
        assert np.all(np.abs(ls_g - ls_w) <= np.abs(ls_w) * 2 ** -7 + 1e-12), (tr, ls_g, ls_w)
    assert okh[:600].all()                   # every random OR-of-ANDs has a feature form
    assert not okh[-1] and not okh[-2]       # nested shapes and 4 groups have none


def _features(setup, n):
    t, T, ctx, est, cdfs, dicts, trees = setup
    preds = [sel.Predicate(T, tr) for tr in trees[:n]]
    feat, ok = est.featurize(preds)
    return feat, feat.float().cpu().numpy()


def test_forward_matches_oracle(setup):
    est = setup[3]
    P = om.init_params(5)
    rng = np.random.default_rng(1)
    for k in ("b1", "b2", "b3", "b4"):
        P[k] = (rng.standard_normal(P[k].shape) * 0.05).astype(np.float32)
    est.set_params(sel.flatten(P))
    feat, X = _features(setup, 600)
    out = est.forward(feat).cpu().numpy()
    ref = om.forward(P, X)["out"]
    assert np.all(np.abs(out - ref) <= 2e-2 * (1 + np.abs(ref))), float(np.abs(out - ref).max())


def test_fused_forward_equals_layer_by_layer(setup):
    """The one-kernel inference pass and the layer-by-layer pass of training
    (three GEMM launches, activations through global memory, the head kernel)
    round and sum alike: the same bits, on a ragged batch of several
    128-row tiles and on a batch of one row; both within the oracle's
    tolerance."""
    est = setup[3]
    P = om.init_params(9)
    rng = np.random.default_rng(3)
    for k in ("b1", "b2", "b3", "b4"):
        P[k] = (rng.standard_normal(P[k].shape) * 0.05).astype(np.float32)
    est.set_params(sel.flatten(P))
    feat, X = _features(setup, 611)
    try:
        for rows in (611, 1):
            f = feat[:rows].contiguous()
            est.set_fused(True)
            fused = est.forward(f)
            est.set_fused(False)
            layered = est.forward(f)
            torch.cuda.synchronize()
            assert torch.equal(fused, layered), float((fused - layered).abs().max())
            ref = om.forward(P, X[:rows])["out"]
            out = fused.cpu().numpy()
            assert np.all(np.abs(out - ref) <= 2e-2 * (1 + np.abs(ref))), float(np.abs(out - ref).max())
    finally:
        est.set_fused(True)


def test_gradients_and_adam_match_oracle(setup):
    est = setup[3]
    P = om.init_params(11)
    est.set_params(sel.flatten(P))
    feat, X = _features(setup, 512)
    y = np.log1p(np.random.default_rng(2).integers(0, 10 ** 6, 512)).astype(np.float32)
    yd = torch.from_numpy(y).cuda()
    loss = est.train_step(feat, yd, sel.train_cfg(apply_update=0))
    ref_loss, G = om.loss_and_grads(P, X, y)
    assert abs(loss - ref_loss) <= 2e-2 * (1 + abs(ref_loss))
    g = sel.unflatten(est.get_grads())
    for k in G:
        scale = max(float(np.abs(G[k]).max()), 1e-12)
        assert float(np.abs(g[k] - G[k]).max()) <= 2e-2 * scale, k
    # Adam on the GPU's own gradients (a fresh gradient of the same batch)
    est.set_params(sel.flatten(P))
    est.train_step(feat, yd, sel.train_cfg(apply_update=0))
    g_gpu = sel.unflatten(est.get_grads())
    est.set_params(sel.flatten(P))
    est.train_step(feat, yd, sel.train_cfg(lr=1e-3, apply_update=1))
    after = sel.unflatten(est.get_params())
    Pm = {k: v.copy() for k, v in P.items()}
    Mo = {k: np.zeros(v.shape) for k, v in P.items()}
    Vo = {k: np.zeros(v.shape) for k, v in P.items()}
    om.adam_step(Pm, g_gpu, Mo, Vo, t=1, lr=1e-3)
    for k in P:
        diff = np.abs(after[k] - Pm[k])
        # the sign of a tiny gradient may differ between two runs (atomic sums): allow <= 0.5 % of entries
        assert np.mean(diff > 1e-6) <= 5e-3, k


def test_training_versus_the_independence_estimate(setup):
    t, T, ctx, est, cdfs, dicts, _ = setup
    rng = np.random.default_rng(3)
    trees = [dg.random_dnf_predicate(dg.config2_specs(), rng) for _ in range(24_000)]
    preds = [sel.Predicate(T, tr) for tr in trees]
    counts = np.array(sel.count_many(ctx, preds, T), dtype=np.uint64)
    n_train = 20_000
    model = sel.Estimator(ctx, T, sample_rows=M, seed=SEED)
    loss = model.train(preds[:n_train], counts[:n_train], sel.train_cfg(epochs=40, batch=256, lr=1e-3, seed=1))
    assert math.isfinite(loss)
    test_p, test_c = preds[n_train:], counts[n_train:]
    feat, ok = model.featurize(test_p)
    out = model.forward(feat).cpu().numpy()
    okm = ok.cpu().numpy().astype(bool)
    q_mlp = om.q_error(np.expm1(out[:, 0]), test_c)[okm]
    ind = baselines.independence_selectivity(feat.float().cpu().numpy()) * T.n_rows
    q_ind = om.q_error(ind, test_c)[okm]
    sig = np.exp(0.5 * np.clip(out[:, 1], -8, 8))[okm]
    acc = sig <= np.median(sig)
    print(f"q-error p50/p95: mlp {np.median(q_mlp):.3f}/{np.percentile(q_mlp, 95):.3f}  "
          f"gated(50%) {np.median(q_mlp[acc]):.3f}/{np.percentile(q_mlp[acc], 95):.3f}  "
          f"independence {np.median(q_ind):.3f}/{np.percentile(q_ind, 95):.3f}  final loss {loss:.4f}")
    # The network's tail beats the independence assumption on correlated clauses (same-column
    # ranges, §1.1's "B < y1 AND B > y2"); its confident half is accurate enough to skip the scan.
    assert np.percentile(q_mlp, 95) < np.percentile(q_ind, 95)
    assert np.median(q_mlp) <= 1.6
    assert np.percentile(q_mlp[acc], 95) <= 3.0


def _distinct_gap_tau(sig):
    """A threshold halfway between two neighbouring distinct sigmas near the
    median, with a gap far above float32 rounding, so that no sigma sits on it."""
    s = np.unique(sig[np.isfinite(sig)])
    mid = len(s) // 2
    for k in list(range(mid, len(s) - 1)) + list(range(mid - 1, -1, -1)):
        if s[k + 1] - s[k] > 1e-4 * s[k + 1]:
            return float(0.5 * (s[k] + s[k + 1]))
    raise AssertionError("no gap between sigmas")


def test_gate_against_the_oracle_gate(setup, tmp_path):
    """sel_mlp_estimate against oracle.mlp.gate with exact counts from oracle.count:
    (1) fed the network outputs the GPU computed on the same features, every
    decision, sigma and estimate agrees (fallbacks bit-exact, accepted
    estimates the same expm1 of the same float32 mu); (2) fed the oracle's own
    features and forward pass with the model's parameters, sigmas and
    estimates agree within the forward tolerance and every decision agrees
    outside the band that tolerance allows around tau."""
    t, T, ctx, est, cdfs, dicts, trees = setup
    P = om.init_params(13)
    rng = np.random.default_rng(13)
    for k in ("b1", "b2", "b3", "b4"):
        P[k] = (rng.standard_normal(P[k].shape) * 0.05).astype(np.float32)
    est.set_params(sel.flatten(P))
    sub = trees[:200] + [trees[-1]]                     # the last one has no feature form
    preds = [sel.Predicate(T, tr) for tr in sub]
    ot = oracle.OTable.from_table(t)
    exact = np.array([oracle.count(ot, tr, threads=8) for tr in sub], dtype=np.uint64)
    feat, ok = est.featurize(preds)
    okh = ok.cpu().numpy().astype(bool)
    assert okh[:-1].all() and not okh[-1]
    out = est.forward(feat).cpu().numpy().astype(np.float64)

    # (1) the gate's rule on the GPU network's outputs
    _, sig_all, _ = om.gate(out[:, 0], out[:, 1], okh, math.inf, exact)
    taus = [0.0, math.inf, _distinct_gap_tau(sig_all)]
    for tau in taus:
        we, ws, wu = om.gate(out[:, 0], out[:, 1], okh, tau, exact)
        e, s, u = est.estimate(preds, T, tau=tau)
        assert np.array_equal(u.astype(bool), wu), tau
        assert np.array_equal(e, we), tau
        fin = np.isfinite(ws)
        assert np.array_equal(np.isfinite(s), fin)
        assert np.all(np.abs(s[fin] - ws[fin]) <= 1e-6 * ws[fin]), tau
    assert 0 < int(np.sum(~om.gate(out[:, 0], out[:, 1], okh, taus[2], exact)[2])) < len(sub) - 1

    # (2) the same against the oracle's features and forward pass
    X = np.stack([om.featurize(tr, cdfs, dicts)[0] for tr in sub])
    ref = om.forward(sel.unflatten(est.get_params()), X)
    tol_lv = 2e-2 * (1 + np.abs(ref["lv"]))
    tol_mu = 2e-2 * (1 + np.abs(ref["mu"]))
    tau = taus[2]
    we, ws, wu = om.gate(ref["mu"], ref["lv"], okh, tau, exact)
    e, s, u = est.estimate(preds, T, tau=tau)
    u = u.astype(bool)
    fin = np.isfinite(ws)
    assert np.all(np.abs(np.log(s[fin]) - np.log(ws[fin])) <= 0.5 * tol_lv[fin] + 1e-6)
    clear = ~fin | (np.abs(np.log(ws) - math.log(tau)) > 0.5 * tol_lv + 1e-6)
    assert clear.sum() >= len(sub) // 2
    assert np.array_equal(u[clear], wu[clear])
    both_exact = u & wu
    assert np.array_equal(e[both_exact], we[both_exact])
    both_est = ~u & ~wu
    assert np.all(np.abs(np.log1p(e[both_est]) - np.log1p(we[both_est])) <= tol_mu[both_est])

    path = str(tmp_path / "m.bin")
    est.save(path)
    again = sel.Estimator.load(ctx, path)
    assert torch.equal(est.forward(feat), again.forward(feat))


def test_repeated_featurize_reuses_the_staged_records(setup):
    """The same predicate list featurized again (the staged clause records are
    reused), interleaved with other lists, gives identical features and flags."""
    t, T, ctx, est, cdfs, dicts, trees = setup
    a = sel.PredicateList([sel.Predicate(T, tr) for tr in trees[:300]])
    b = [sel.Predicate(T, tr) for tr in trees[300:450]]
    fa, oa = est.featurize(a)
    fa2, oa2 = est.featurize(a)
    fb, ob = est.featurize(b)
    fa3, oa3 = est.featurize(a)
    fb2, ob2 = est.featurize(b[:149] + [b[149]])   # equal predicates, new list object
    for f, o in ((fa2, oa2), (fa3, oa3)):
        assert torch.equal(f, fa) and torch.equal(o, oa)
    assert torch.equal(fb2, fb) and torch.equal(ob2, ob)
    fresh, _ = est.featurize([sel.Predicate(T, tr) for tr in trees[:300]])   # recompiled: new ids
    assert torch.equal(fresh, fa)


def test_launch_count_includes_the_estimator(setup):
    """sel_ctx_launch_count counts every kernel the context launches, the
    estimator's included: featurize is one kernel, the forward pass one fused
    kernel (three GEMMs and the head layer by layer), and a training step a
    whole number of launches that is the same every time; a training run made
    of steps counts each step once."""
    t, T, ctx, est, cdfs, dicts, trees = setup
    preds = [sel.Predicate(T, tr) for tr in trees[:64]]
    l0 = ctx.launches
    feat, _ = est.featurize(preds)
    assert ctx.launches - l0 == 1
    l1 = ctx.launches
    est.forward(feat)
    assert ctx.launches - l1 == 1
    est.set_fused(False)
    try:
        l1 = ctx.launches
        est.forward(feat)
        assert ctx.launches - l1 == 4
    finally:
        est.set_fused(True)
    y = torch.zeros(64, dtype=torch.float32, device=feat.device)
    cfg = sel.train_cfg(batch=64, lr=0.0, apply_update=0)
    l2 = ctx.launches
    est.train_step(feat, y, cfg)
    per_step = ctx.launches - l2
    assert per_step >= 8
    l3 = ctx.launches
    est.train_step(feat, y, cfg)
    assert ctx.launches - l3 == per_step
