"""Pins for the join-size oracle (oracle/join.py), CPU only: the plan sizes
the paper works out in §1.1 for its three-relation query, and distinct counts
checked against constructions whose answer is known."""
import numpy as np

import datagen as dg
import oracle
from oracle import join


def test_paper_plan_sizes():
    # |R| = 600M, |S| = 5M, |T| = 1M; S.A and T.B are distinct keys.
    # Estimated sigma(R): 0.9M rows -> (sigma(R) join S) = 0.9M;  (T join S) = 5M;
    # with the actual selectivity 0.167, sigma(R) has 100.2M rows -> (sigma(R) join S) = 100.2M
    assert join.join_size_estimate(900_000, 5_000_000, 900_000, 5_000_000) == 900_000
    assert join.join_size_estimate(5_000_000, 1_000_000, 1_000_000, 1_000_000) == 5_000_000
    assert round(join.join_size_estimate(int(600e6 * 0.167), 5_000_000, 5_000_000, 5_000_000) / 1e6, 1) == 100.2
    assert join.join_size_estimate(0, 10, 0, 0) == 0.0


def test_distinct_counts_by_construction():
    n = 10_000
    perm = np.random.default_rng(1).permutation(n).astype(np.int32)
    mod = (np.arange(n) % 37).astype(np.int64) - 18
    f = np.array([0.0, -0.0, 1.5, -1.5, 1.5] * (n // 5), np.float32)
    t = oracle.OTable([perm, mod, f], ["i32", "i64", "f32"], [None, None, None])
    assert join.count_distinct(t, 0) == (n, n)                    # a permutation: n distinct values
    assert join.count_distinct(t, 1) == (37, n)                   # i mod 37
    assert join.count_distinct(t, 2) == (3, n)                    # -0.0 and +0.0 are one value
    # under a selection: perm < 100 selects 100 rows with 100 distinct values
    assert join.count_distinct(t, 0, dg.p_cmp(0, "<", 100)) == (100, 100)
    d, r = join.count_distinct(t, 1, dg.p_cmp(0, "<", 100))
    assert r == 100 and d == len(set(mod[perm < 100].tolist()))
    assert join.count_distinct(t, 1, dg.P_FALSE) == (0, 0)


def test_join_count_brute_force_and_key_join():
    rng = np.random.default_rng(5)
    a = rng.integers(0, 6, 300).astype(np.int32)
    b = rng.integers(2, 9, 200).astype(np.int32)
    r = oracle.OTable([a], ["i32"], [None])
    s = oracle.OTable([b], ["i32"], [None])
    brute = sum(1 for x in a for y in b if x == y)
    assert join.join_count(r, 0, None, s, 0, None) == (brute, 300, 200)
    sel_r = dg.p_cmp(0, ">=", 3)
    brute = sum(1 for x in a if x >= 3 for y in b if x == y)
    assert join.join_count(r, 0, sel_r, s, 0, None)[0] == brute
    # a join on S's distinct key (§1.1: primary keys are distinct): every selected R row matches once,
    # so the join has exactly |sigma(R)| rows, as the plan sizes of §1.1 assume
    keys = np.arange(1000, dtype=np.int64)
    fk = rng.integers(0, 1000, 5000).astype(np.int64)
    rr = oracle.OTable([fk], ["i64"], [None])
    ss = oracle.OTable([keys], ["i64"], [None])
    c, nr, ns = join.join_count(rr, 0, dg.p_cmp(0, "<", 100), ss, 0, None)
    assert c == nr == int(np.sum(fk < 100)) and ns == 1000
