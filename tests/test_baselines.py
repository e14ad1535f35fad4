"""The traditional (independence) estimator used as the learned estimator's
baseline, pinned by the numbers the paper prints (§1.1, Ch2)."""
import numpy as np

from paper_1806_08384_b300 import baselines as b


def test_worked_and_estimate():
    # §1.1: 0.2 x 0.167 x 0.167 x 0.27 ~= 0.0015 for the four ANDed predicates
    assert round(b.combine_and([0.2, 0.167, 0.167, 0.27]), 4) == 0.0015


def test_or_is_sum_minus_joint():
    # Ch2: (C = z1 OR C = z2) -> 1/V + 1/V - (1/V)^2
    v = 1 / 7
    assert abs(b.combine_or([v, v]) - (v + v - v * v)) < 1e-15


def test_from_features():
    f = np.zeros((1, 144), np.float32)
    # group 0: two leaves with masses 0.5 and 0.2; group 1: one negated leaf of mass 0.9
    for s, (lo, hi, g, neg) in enumerate([(0.25, 0.75, 0, 0), (0.0, 0.2, 0, 0), (0.0, 0.9, 1, 1)]):
        o = s * 24
        f[0, o + s] = 1                      # column one-hot
        f[0, o + 18], f[0, o + 19] = lo, hi
        f[0, o + 20 + g] = 1
        f[0, o + 17] = neg
    want = 1 - (1 - 0.5 * 0.2) * (1 - 0.1)
    assert abs(b.independence_selectivity(f)[0] - want) < 1e-6
