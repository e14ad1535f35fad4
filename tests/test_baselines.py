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


def test_paper_cardinality_of_the_worked_selection():
    # §1.1: |R| = 600 million rows, combined factor about 0.0015 -> sigma(R) about 0.9 million rows
    assert round(600e6 * b.combine_and([0.2, 0.167, 0.167, 0.27]) / 1e6, 1) == 0.9


def test_textbook_heuristics_on_the_ch2_formula():
    # |R| * 1/V(R,A) * 1/3 * 1/3 * (1/V(R,C) + 1/V(R,C) - (1/V(R,C))^2) for
    # R.A = x AND R.B < y1 AND R.B > y2 AND (R.C = z1 OR R.C = z2)
    va, vc = 5.0, 4.0
    tree = ("and", [("cmp", 0, "=", 1), ("cmp", 1, "<", 9), ("cmp", 1, ">", 2),
                    ("or", [("cmp", 2, "=", 7), ("cmp", 2, "=", 8)])])
    want = (1 / va) * (1 / 3) * (1 / 3) * (1 / vc + 1 / vc - (1 / vc) ** 2)
    assert abs(b.textbook_selectivity(tree, [va, 10, vc]) - want) < 1e-15
    # IN of two values is the same OR of equalities; BETWEEN is the two inequalities
    tin = ("and", [("cmp", 0, "=", 1), ("between", 1, 2, 9), ("in", 2, [7, 8])])
    assert abs(b.textbook_selectivity(tin, [va, 10, vc]) - want) < 1e-15
    assert abs(b.textbook_selectivity(("not", ("cmp", 0, "=", 1)), [va]) - (1 - 1 / va)) < 1e-15


def test_equi_depth_histogram_worked_example():
    # Ch2: an equality on a value spread over three buckets of depth 30 with 2, 1 and 7
    # distinct values: 30/2 + 30/1 + 30/7 = 49.3
    h = b.EquiDepthHistogram(lo=[10, 16, 16, 30], hi=[16, 16, 25, 40], distinct=[2, 1, 7, 5], depth=30)
    assert round(h.eq_rows(16), 1) == 49.3
    assert round(h.eq_rows(35), 6) == 6.0      # one bucket: 30 / 5


def test_equi_depth_histogram_ranges():
    rng = np.random.default_rng(0)
    x = rng.integers(0, 1000, 200_000)
    h = b.EquiDepthHistogram.build(x, n_rows=len(x), buckets=50)
    for c in (10, 250, 500, 999):
        est = h.below_rows(c, inclusive=False)
        assert abs(est - np.sum(x < c)) <= 0.03 * len(x)
    sel_ = b.histogram_selectivity(("between", 0, 100, 299), [h])
    assert abs(sel_ - np.mean((x >= 100) & (x <= 299))) < 0.03


def test_sampling_scale_factor():
    # |sigma(R')| * |R| / |R'|
    assert b.sampling_estimate(12, 4096, 300_000_000) == 12 * 300_000_000 / 4096
