"""Pins for the estimator oracle (oracle/mlp.py), CPU only.

* BF16 rounding equals torch's own float32 -> bfloat16 conversion (a library
  routine written independently), including ties;
* SplitMix64 reproduces the published test vectors of its reference code;
* the analytic gradients equal central finite differences of the loss (in
  float64 with rounding off);
* the Gaussian NLL and its gradient at closed-form points;
* Adam's first step moves each parameter by lr * g / (|g| + eps);
* CDF features partition the sample: < a, BETWEEN a..b and > b cover it once;
* the hand-worked features, gate, tau rule and network of tests/mlp_pins.py,
  and a planted mistake in each part of a copy of the oracle (a dropped
  complement, a shifted one-hot, a wrong log base, a strict gate, ...) fails
  at least one of those pins.
"""
import math
import os
import types

import numpy as np
import pytest
import torch

import datagen as dg
from oracle import mlp
from tests import mlp_pins


def test_bf16_rounding_matches_torch():
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.standard_normal(10000).astype(np.float32) * 10 ** rng.uniform(-5, 5, 10000),
                        np.array([1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, -(1.0 + 2 ** -8), 65504.5, 0.0, -0.0],
                                 np.float32)]).astype(np.float32)
    # exact ties: low 16 bits 0x8000 with even and odd bit 16
    ties = np.array([0x3F808000, 0x3F818000, 0xBF808000, 0x40008000], np.uint32).view(np.float32)
    x = np.concatenate([x, ties])
    want = torch.from_numpy(x).to(torch.bfloat16).to(torch.float32).numpy()
    assert np.array_equal(mlp.bf16_round(x).view(np.uint32), want.view(np.uint32))


def test_splitmix64_published_vectors():
    g = 0x9E3779B97F4A7C15
    z = np.array([1234567, 1234567 + g, 1234567 + 2 * g], dtype=object)
    z = np.array([int(v) % (1 << 64) for v in z], dtype=np.uint64)
    assert [int(v) for v in mlp.splitmix64(z)] == [6457827717110365317, 3203168211198807973,
                                                    9817491932198370423]


def test_gradients_match_finite_differences():
    rng = np.random.default_rng(1)
    P = mlp.init_params(3)
    for k in P:
        if k.startswith("b"):
            P[k] = (rng.standard_normal(P[k].shape) * 0.1).astype(np.float32)
    P = {k: v.astype(np.float64) for k, v in P.items()}
    X = rng.random((6, mlp.N_FEAT))
    y = rng.random(6) * 5
    loss, G = mlp.loss_and_grads(P, X, y, exact=True)
    h = 1e-6
    for k in ("W1", "b1", "W2", "b3", "W3", "W4", "b4"):
        for _ in range(6):
            idx = tuple(int(rng.integers(0, s)) for s in P[k].shape)
            Pp = {q: v.copy() for q, v in P.items()}
            Pm = {q: v.copy() for q, v in P.items()}
            Pp[k][idx] += h
            Pm[k][idx] -= h
            cp = mlp.forward(Pp, X, exact=True)
            cm = mlp.forward(Pm, X, exact=True)
            fd = (mlp.nll(cp["mu"], cp["lv"], y) - mlp.nll(cm["mu"], cm["lv"], y)) / (2 * h)
            assert abs(fd - G[k][idx]) <= 1e-5 * max(1.0, abs(fd)), (k, idx, fd, G[k][idx])


def test_nll_closed_forms():
    y = np.array([1.0, 2.0])
    assert math.isclose(mlp.nll(y, np.array([0.3, -0.7]), y), 0.5 * (0.3 - 0.7) / 2)
    # lv = 0, residual r: loss = 0.5 * mean(r^2)
    assert math.isclose(mlp.nll(np.zeros(2), np.zeros(2), y), 0.5 * (1 + 4) / 2)


def test_adam_first_step_is_lr_sign():
    P = {"w": np.array([1.0, -2.0, 0.5], np.float32)}
    G = {"w": np.array([0.3, -1e-3, 5.0])}
    M = {"w": np.zeros(3)}
    V = {"w": np.zeros(3)}
    mlp.adam_step(P, G, M, V, t=1, lr=0.01, eps=1e-8)
    want = np.array([1.0, -2.0, 0.5]) - 0.01 * G["w"] / (np.abs(G["w"]) + 1e-8)
    assert np.allclose(P["w"], want, rtol=0, atol=1e-6)


def test_cdf_features_partition_the_sample():
    t = dg.gen_table("cfg2", dg.config2_specs(), 50_000, "cpu")
    for ci in (0, 3, 4, 5):
        a = t.columns[ci].data.numpy()
        cdf = mlp.CDF(a, seed=7, col=ci, m=4096)
        lo, hi = (a[17], a[4242]) if a[17] <= a[4242] else (a[4242], a[17])
        lo, hi = (float(lo), float(hi)) if a.dtype == np.float32 else (int(lo), int(hi))
        below = mlp.leaf_bounds(("cmp", ci, "<", lo), cdf)
        mid = mlp.leaf_bounds(("between", ci, lo, hi), cdf)
        above = mlp.leaf_bounds(("cmp", ci, ">", hi), cdf)
        mass = (below[1] - below[0]) + (mid[1] - mid[0]) + (above[1] - above[0])
        assert abs(mass - 1.0) < 1e-6
        assert below[1] == mid[0] and mid[1] == above[0]
    s1 = t.index("s1")
    cdf = mlp.CDF(t.columns[s1].data.numpy(), seed=7, col=s1, m=4096)
    assert mlp.leaf_bounds(("like", s1, ""), cdf, t.columns[s1].dictionary) == (0.0, 1.0)
    vals = sorted(set(int(v) for v in cdf.s))
    assert mlp.leaf_bounds(("in", s1, vals), cdf) == (0.0, 1.0)


def test_dnf_shapes():
    a, b, c = dg.p_cmp(0, "<", 1), dg.p_cmp(1, ">", 2), dg.p_cmp(2, "=", 3)
    g = mlp.dnf_groups(dg.p_not(dg.p_or(a, b)))           # NOT(a OR b) = NOT a AND NOT b
    assert g == [[(a, True), (b, True)]]
    g = mlp.dnf_groups(dg.p_or(dg.p_and(a, b), c))
    assert g == [[(a, False), (b, False)], [(c, False)]]
    assert mlp.dnf_groups(dg.p_and(a, dg.p_or(b, c))) is None
    f, ok = mlp.featurize(dg.p_or(*[dg.p_and(a, b)] * 4), [None] * 8, [None] * 8)
    assert not ok


# ----------------------------------------------------------------------------
# hand-worked pins (tests/mlp_pins.py) and planted mistakes in copies of the oracle
# ----------------------------------------------------------------------------



@pytest.mark.parametrize("pin", mlp_pins.ALL_PINS, ids=lambda p: p.__name__)
def test_estimator_pin(pin):
    assert pin(mlp) == []


MLP_MUTANTS = {
    "ne_complement_dropped": ("    if ne:\n        p = 1.0 - p\n", ""),
    "not_complement_dropped": ("    if neg:\n        p = 1.0 - p\n", ""),
    "log_base_m": ("/ math.log(2.0 * m)", "/ math.log(1.0 * m)"),
    "log_floor_1_over_m": ("max(p, 0.5 / m)", "max(p, 1.0 / m)"),
    "column_onehot_shifted": ("f[o + col] = 1.0", "f[o + col + 1] = 1.0"),
    "operator_onehot_offset": ("f[o + 8 + op_index(leaf)] = 1.0", "f[o + 9 + op_index(leaf)] = 1.0"),
    "not_flag_slot": ("f[o + 17] = 1.0", "f[o + 16] = 1.0"),
    "group_onehot_offset": ("f[o + 20 + gi] = 1.0", "f[o + 21 + gi] = 1.0"),
    "op_index_in_like_swapped": ('{"between": 6, "in": 7, "like": 8}', '{"between": 6, "in": 8, "like": 7}'),
    "lt_counts_equal_rows": ('        if op == "<":\n            return 0.0, cdf.frac(cdf.below(v))',
                             '        if op == "<":\n            return 0.0, cdf.frac(cdf.upto(v))'),
    "between_hi_exclusive": ("cdf.frac(max(lo, cdf.upto(leaf[3])))", "cdf.frac(max(lo, cdf.below(leaf[3])))"),
    "in_duplicates_counted": ("vals = sorted(set(leaf[2]))", "vals = sorted(leaf[2])"),
    "like_prefix_ignored": ("if w.startswith(pre)]", "if w[:1] == pre[:1]]"),
    "sample_column_offset": ("((col + 1) << 40)", "(col << 40)"),
    "relu_dropped": ("a = r(np.maximum(z, 0.0).astype(", "a = r(np.asarray(z).astype("),
    "heads_swapped": ('c["mu"] = out[:, 0]\n    c["lv"] = np.clip(out[:, 1], LV_MIN, LV_MAX)',
                      'c["mu"] = out[:, 1]\n    c["lv"] = np.clip(out[:, 0], LV_MIN, LV_MAX)'),
    "bias_dropped": ('z = a @ r(P[f"W{l}"]).T + P[f"b{l}"].astype(np.float64)', 'z = a @ r(P[f"W{l}"]).T'),
    "gate_sigma_without_half": ("math.exp(0.5 * lv[i])", "math.exp(lv[i])"),
    "gate_strict_accept": ("not (sigma[i] <= tau)", "not (sigma[i] < tau)"),
    "gate_exp_not_expm1": ("max(0.0, math.expm1(mu[i]))", "max(0.0, math.exp(mu[i]))"),
    "gate_no_floor": ("max(0.0, math.expm1(mu[i]))", "math.expm1(mu[i])"),
    "gate_ignores_feature_form": ("used[i] = (not ok[i]) or not (sigma[i] <= tau)", "used[i] = not (sigma[i] <= tau)"),
    "gate_no_clamp": ("lv = np.clip(np.asarray(lv, np.float64), LV_MIN, LV_MAX)", "lv = np.asarray(lv, np.float64)"),
    "tau_median": ("percentile(acc, q) <= max_q", "percentile(acc, 50.0) <= max_q"),
    "tau_smallest": ("            best = t\n", "            best = t if best == 0.0 else best\n"),
    "percentile_nearest_lower": ("return s[lo] + (h - lo) * (s[lo + 1] - s[lo])", "return s[lo]"),
    "q_error_unclamped": ("e = np.maximum(np.asarray(est, np.float64), 1.0)", "e = np.asarray(est, np.float64)"),
}


@pytest.mark.parametrize("name", sorted(MLP_MUTANTS))
def test_estimator_pins_catch_planted_mistake(name):
    src = open(os.path.join(os.path.dirname(mlp.__file__), "mlp.py")).read()
    old, new = MLP_MUTANTS[name]
    assert src.count(old) == 1, f"mutation anchor for {name} not unique"
    mod = types.ModuleType(f"mlp_mutant_{name}")
    mod.__file__ = mlp.__file__
    with np.errstate(all="ignore"):
        exec(compile(src.replace(old, new), f"<mutant {name}>", "exec"), mod.__dict__)
        fails = mlp_pins.run_all(mod)
    assert fails, f"no pin catches mutant {name}"
