"""Pins for the estimator oracle (oracle/mlp.py): facts fixed by hand-worked
cases, closed forms and identities, not by the oracle itself.

Each ``pin_*`` takes the oracle module (the real one, or a copy with a planted
mistake) and returns a list of failure strings.

The constructed samples have m = 16 rows, so every sample fraction is a
multiple of 1/16 and the log-selectivity term ln(max(p, 1/(2m))) / ln(2m)
has the closed form -k/5 whenever p = 2^-k (ln 32 = 5 ln 2); p = 0 takes the
floor 1/32 and gives -1.  Column 0 holds 0 once, 1 once, 2 twice, 3 four times
and 4 eight times (masses 1/16, 1/16, 1/8, 1/4, 1/2); column 1 is a
dictionary column over ["ab", "ac", "b", "ba", "c"] holding codes 0 and 1
twice each and codes 2, 3, 4 four times each.
"""
from __future__ import annotations

import math

import numpy as np

from datagen import p_and, p_between, p_cmp, p_in, p_like, p_not, p_or

C0 = [0, 1, 2, 2, 3, 3, 3, 3, 4, 4, 4, 4, 4, 4, 4, 4]
C1 = [0, 0, 1, 1, 2, 2, 2, 2, 3, 3, 3, 3, 4, 4, 4, 4]
DICT1 = [b"ab", b"ac", b"b", b"ba", b"c"]
SLOT_OP = {"=": 0, "<>": 1, "<": 2, "<=": 3, ">": 4, ">=": 5, "between": 6, "in": 7, "like": 8}


def _cdfs(m):
    return [m.CDF.from_sample(np.array(C0, np.int32)), m.CDF.from_sample(np.array(C1, np.int32))]


def _check(fails, what, got, want, tol=0.0):
    if isinstance(want, tuple):
        ok = len(got) == len(want) and all(abs(float(g) - float(w)) <= tol for g, w in zip(got, want))
    else:
        ok = abs(float(got) - float(want)) <= tol
    if not ok:
        fails.append(f"{what}: {got!r} != {want!r}")


def pin_sample_index_formula(m):
    """idx_i = splitmix64(seed + (col + 1) 2^40 + i) mod n: with seed + 2^40 =
    1234567 (col 0, i 0), the state is the one of SplitMix64's published
    first output, 6457827717110365317."""
    fails = []
    seed = (1234567 - (1 << 40)) % (1 << 64)
    n = 1_000_003
    want = 6457827717110365317 % n
    # consecutive i advance the state by 1, not by the golden gamma: only i = 0 is a published vector
    got = m.sample_indices(seed, 0, 3, n)
    if int(got[0]) != want:
        fails.append(f"sample index 0: {int(got[0])} != {want}")
    got = m.sample_indices((1234567 - (2 << 40)) % (1 << 64), 1, 1, n)   # col 1 adds 2 * 2^40
    if int(got[0]) != want:
        fails.append(f"column offset: {int(got[0])} != {want}")
    return fails


def pin_leaf_bounds_hand_worked(m):
    """[F_lo, F_hi] of every leaf kind on the constructed samples, by hand."""
    fails = []
    c0, c1 = _cdfs(m)
    cases = [
        (p_cmp(0, "<", 3), (0.0, 4 / 16)),
        (p_cmp(0, "<=", 3), (0.0, 8 / 16)),
        (p_cmp(0, ">", 3), (8 / 16, 1.0)),
        (p_cmp(0, ">=", 3), (4 / 16, 1.0)),
        (p_cmp(0, "=", 2), (2 / 16, 4 / 16)),
        (p_cmp(0, "<>", 2), (2 / 16, 4 / 16)),
        (p_cmp(0, "=", 7), (1.0, 1.0)),
        (p_between(0, 1, 3), (1 / 16, 8 / 16)),
        (p_between(0, 3, 1), (4 / 16, 4 / 16)),          # lo > hi: empty
        (p_in(0, [0, 1, 2, 2, 9]), (0.0, 4 / 16)),       # duplicates once, 9 absent
        (p_in(0, [4]), (0.0, 8 / 16)),
        (p_in(0, []), (0.0, 0.0)),
    ]
    for leaf, want in cases:
        _check(fails, f"bounds {leaf}", m.leaf_bounds(leaf, c0), want)
    like = [("a", (0.0, 4 / 16)), ("b", (0.0, 8 / 16)), ("ba", (0.0, 4 / 16)), ("", (0.0, 1.0)),
            ("c", (0.0, 4 / 16)), ("e", (0.0, 0.0)), ("abc", (0.0, 0.0))]
    for pre, want in like:
        _check(fails, f"like {pre!r}", m.leaf_bounds(p_like(1, pre), c1, DICT1), want)
    return fails


def pin_log_selectivity_closed_forms(m):
    """p = 2^-k gives -k/5; p = 0 takes the floor 1/32 and gives -1; p = 1 gives 0."""
    fails = []
    c0, c1 = _cdfs(m)
    cases = [(p_cmp(0, "=", 4), -1 / 5), (p_cmp(0, "=", 3), -2 / 5), (p_cmp(0, "=", 2), -3 / 5),
             (p_cmp(0, "=", 1), -4 / 5), (p_cmp(0, "=", 7), -1.0), (p_cmp(0, ">=", 0), 0.0),
             (p_in(0, [0, 1, 2, 3]), -1 / 5), (p_like(1, "b"), -1 / 5), (p_like(1, "ab"), -3 / 5)]
    for leaf, want in cases:
        f, ok = m.featurize(leaf, [c0, c1], [None, DICT1])
        if not ok:
            fails.append(f"{leaf}: no feature form")
            continue
        _check(fails, f"log-selectivity {leaf}", f[23], np.float32(want))
    return fails


def pin_complement_identities(m):
    """A leaf whose value set is a complement has the log-selectivity of a
    plain leaf with the same value set: c <> 3 as c IN {0,1,2,4};
    NOT(c < 3) as c >= 3; NOT(c1 LIKE 'a') as c1 IN {2,3,4};
    NOT(c <> 2) as c = 2 (two complements)."""
    fails = []
    cdfs = _cdfs(m)
    dicts = [None, DICT1]
    pairs = [(p_cmp(0, "<>", 3), p_in(0, [0, 1, 2, 4])),
             (p_not(p_cmp(0, "<", 3)), p_cmp(0, ">=", 3)),
             (p_not(p_like(1, "a")), p_in(1, [2, 3, 4])),
             (p_not(p_cmp(0, "<>", 2)), p_cmp(0, "=", 2)),
             (p_not(p_in(0, [4])), p_cmp(0, "<", 4))]
    for a, b in pairs:
        fa, oka = m.featurize(a, cdfs, dicts)
        fb, okb = m.featurize(b, cdfs, dicts)
        if not (oka and okb):
            fails.append(f"{a} / {b}: no feature form")
            continue
        if fa[23] != fb[23]:
            fails.append(f"log-selectivity of {a} = {fa[23]} but of {b} = {fb[23]}")
    return fails


def pin_feature_vector_hand_worked(m):
    """The whole 144-float vector of (c0 < 3 AND NOT c1 LIKE 'a') OR c0 IN {0,1,2,2,9},
    written out slot by slot from the layout: column one-hot at 0..7, operator
    one-hot at 8..16 (= <> < <= > >= BETWEEN IN LIKE), NOT flag at 17, F_lo at
    18, F_hi at 19, OR-group one-hot at 20..22, log-selectivity at 23."""
    fails = []
    cdfs = _cdfs(m)
    tree = p_or(p_and(p_cmp(0, "<", 3), p_not(p_like(1, "a"))), p_in(0, [0, 1, 2, 2, 9]))
    f, ok = m.featurize(tree, cdfs, [None, DICT1])
    want = np.zeros(144, np.float32)
    # slot 0: c0 < 3 (group 0), p = 1/4
    want[0] = 1; want[8 + 2] = 1; want[18] = 0; want[19] = 0.25; want[20] = 1; want[23] = np.float32(-0.4)
    # slot 1: NOT c1 LIKE 'a' (group 0), bounds of the un-negated set [0, 1/4]
    o = 24
    want[o + 1] = 1; want[o + 8 + 8] = 1; want[o + 17] = 1; want[o + 18] = 0; want[o + 19] = 0.25; want[o + 20] = 1
    # its log-selectivity (p = 3/4) is pinned by the identity with c1 IN {2,3,4}
    fi, _ = m.featurize(p_in(1, [2, 3, 4]), cdfs, [None, DICT1])
    want[o + 23] = fi[23]
    # slot 2: c0 IN {0,1,2,2,9} (group 1), p = 1/4
    o = 48
    want[o + 0] = 1; want[o + 8 + 7] = 1; want[o + 18] = 0; want[o + 19] = 0.25; want[o + 21] = 1
    want[o + 23] = np.float32(-0.4)
    if not ok:
        fails.append("hand-worked predicate has no feature form")
    elif not np.array_equal(f, want):
        fails.append(f"feature vector differs at {np.nonzero(f != want)[0].tolist()}")
    return fails


def pin_operator_slots(m):
    """Every operator sets exactly its one-hot position 8 + k of the layout."""
    fails = []
    cdfs = _cdfs(m)
    leaves = [p_cmp(0, op, 2) for op in ("=", "<>", "<", "<=", ">", ">=")] + \
        [p_between(0, 1, 2), p_in(0, [1]), p_like(1, "b")]
    names = ["=", "<>", "<", "<=", ">", ">=", "between", "in", "like"]
    for leaf, name in zip(leaves, names):
        f, ok = m.featurize(leaf, cdfs, [None, DICT1])
        hot = np.nonzero(f[8:18])[0].tolist()
        if not ok or hot != [SLOT_OP[name]]:
            fails.append(f"operator {name}: one-hot at {hot}")
        col = np.nonzero(f[0:8])[0].tolist()
        if col != [leaf[1]]:
            fails.append(f"operator {name}: column one-hot at {col}")
    # three groups: the group one-hot follows the OR's order
    tree = p_or(p_cmp(0, "=", 1), p_cmp(0, "=", 2), p_cmp(1, "=", 3))
    f, ok = m.featurize(tree, cdfs, [None, DICT1])
    for s in range(3):
        g = np.nonzero(f[s * 24 + 20:s * 24 + 23])[0].tolist()
        if g != [s]:
            fails.append(f"group one-hot of slot {s}: {g}")
    return fails


def pin_network_hand_wired(m):
    """A hand-wired network with one live unit per layer and biases on every
    layer; every value is exact in BF16:
    row e0: a1 = (2, 1), a2 = 3*2 + 1 - 0.5 = 6.5, a3 = 0.5*6.5 + 0.25 = 3.5,
            mu = 3.5 + 0.25 = 3.75, lv = -3.5 + 0.5 = -3;
    row -e0: a1 = (0, 1) (ReLU), a2 = 0.5, a3 = 0.5, mu = 0.75, lv = 0."""
    fails = []
    P = {k: np.zeros(s, np.float32) for k, s in m.PARAM_SHAPES}
    P["W1"][0, 0] = 2.0
    P["b1"][1] = 1.0
    P["W2"][0, 0] = 3.0
    P["W2"][0, 1] = 1.0
    P["b2"][0] = -0.5
    P["W3"][0, 0] = 0.5
    P["b3"][0] = 0.25
    P["W4"][0, 0] = 1.0
    P["W4"][1, 0] = -1.0
    P["b4"][:] = [0.25, 0.5]
    X = np.zeros((2, m.N_FEAT), np.float32)
    X[0, 0] = 1.0
    X[1, 0] = -1.0
    c = m.forward(P, X)
    _check(fails, "mu", tuple(c["mu"]), (3.75, 0.75))
    _check(fails, "lv", tuple(c["lv"]), (-3.0, 0.0))
    P["b4"][1] = 20.0                                  # the log-variance clamp at 8
    _check(fails, "lv clamp", tuple(m.forward(P, X)["lv"]), (8.0, 8.0))
    return fails


def pin_gate_hand_worked(m):
    """The gate's rule on hand-worked points: mu = ln 100 -> 99; mu = 0 -> 0;
    mu < 0 -> 0 (clamped); lv = 2 ln 0.5 -> sigma 0.5, accepted at tau = 0.5
    (sigma <= tau) and answered exactly at tau = 0.49; lv = 100 -> clamp 8 ->
    sigma = e^4; no feature form -> exact with sigma = inf even at tau = inf."""
    fails = []
    mu = [math.log(100.0), 0.0, -3.0, 1.0, 1.0, 2.0]
    lv = [2 * math.log(0.5), 2 * math.log(0.5), 2 * math.log(0.5), 100.0, -100.0, 0.0]
    ok = [True, True, True, True, True, False]
    exact = [7, 8, 9, 10, 11, 12]
    est, sig, used = m.gate(mu, lv, ok, 0.5, exact)
    _check(fails, "sigma", tuple(sig[:5]), (0.5, 0.5, 0.5, math.exp(4.0), math.exp(-4.0)), 1e-12)
    if not math.isinf(sig[5]):
        fails.append(f"sigma without a feature form: {sig[5]}")
    if list(used) != [False, False, False, True, False, True]:
        fails.append(f"decisions at tau 0.5: {list(used)}")
    _check(fails, "estimates at tau 0.5", tuple(est), (99.0, 0.0, 0.0, 10.0, math.e - 1.0, 12.0), 1e-9)
    est, sig, used = m.gate(mu, lv, ok, 0.49, exact)
    if list(used) != [True, True, True, True, False, True]:
        fails.append(f"decisions at tau 0.49: {list(used)}")
    est, sig, used = m.gate(mu, lv, ok, math.inf, exact)
    if list(used) != [False] * 5 + [True]:
        fails.append(f"decisions at tau inf: {list(used)}")
    return fails


def pin_choose_tau_hand_worked(m):
    """sigma = (0.1, 0.2, 0.3, 0.4, inf) with q-errors (1, 1.5, 3, 1.2, -):
    95th percentiles of the accepted sets are 1, 1.475, 2.85, 2.775, so
    max_q = 2 picks 0.2 and max_q = 3 picks 0.4; max_q = 0.5 picks nothing (0)."""
    fails = []
    sig = [0.1, 0.2, 0.3, 0.4, math.inf]
    est = [10.0, 15.0, 30.0, 12.0, 0.0]
    exact = [10, 10, 10, 10, 5]
    _check(fails, "tau(max_q=2)", m.choose_tau(sig, est, exact, 2.0), 0.2)
    _check(fails, "tau(max_q=3)", m.choose_tau(sig, est, exact, 3.0), 0.4)
    _check(fails, "tau(max_q=0.5)", m.choose_tau(sig, est, exact, 0.5), 0.0)
    _check(fails, "p95 of 1..101", m.percentile(list(range(1, 102)), 95.0), 96.0, 1e-12)
    _check(fails, "p95 of (1, 1.5, 3)", m.percentile([3.0, 1.0, 1.5], 95.0), 2.85, 1e-12)
    return fails


def pin_q_error_definition(m):
    """q = max(e, t) / min(e, t) with both clamped to >= 1."""
    fails = []
    _check(fails, "q-errors", tuple(m.q_error([10, 5, 0, 0.5, 3], [5, 10, 0, 7, 3])), (2.0, 2.0, 1.0, 7.0, 1.0))
    return fails


ALL_PINS = [pin_sample_index_formula, pin_leaf_bounds_hand_worked, pin_log_selectivity_closed_forms,
            pin_complement_identities, pin_feature_vector_hand_worked, pin_operator_slots,
            pin_network_hand_wired, pin_gate_hand_worked, pin_choose_tau_hand_worked, pin_q_error_definition]


def run_all(m):
    fails = []
    for p in ALL_PINS:
        try:
            fails += [f"{p.__name__}: {x}" for x in p(m)]
        except Exception as e:          # a mutant may raise instead of returning a wrong value
            fails.append(f"{p.__name__}: raised {type(e).__name__}: {e}")
    return fails
