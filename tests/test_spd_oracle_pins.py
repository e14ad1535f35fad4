"""Pins for the Algorithm 1 oracle (oracle/spd.py), CPU only.

Each case is built so that the answer follows from the algorithm's text
(Ch4 §4.2) by hand: a relation enters the queue only when its size is
strictly greater than PUSH_DOWN_MIN_TABLE_SIZE, the largest one is popped and
never pushed down, maxSize = R.size * PUSH_DOWN_MAX_SELECTIVITY and the
push-down is reverted exactly when count > maxSize.  Column 0 of every table
is the row index, so the count of `c0 < k` is min(k, n)."""
import numpy as np

import datagen as dg
import oracle
from oracle import spd


def rel(n, k=None, proj=(0,)):
    """A relation of n rows (c0 = row index, c1 = 7 * row index) whose pushed-down
    selection `c0 < k` selects min(k, n) rows; k None: no selection."""
    t = oracle.OTable([np.arange(n, dtype=np.int32), (7 * np.arange(n)).astype(np.int64)], ["i32", "i64"],
                      [None, None])
    return t, (None if k is None else dg.p_cmp(0, "<", k)), list(proj)


def decisions(res):
    return [r["decision"] for r in res]


def test_queue_order_min_size_and_probe():
    # sizes 10, 50, 30, 50, 5 with PUSH_DOWN_MIN_TABLE_SIZE 10: sizes 10 and 5 stay out (not > 10);
    # the first 50 (input order breaks the tie) is the probed relation
    rels = [rel(10, 1), rel(50, 1), rel(30, 1), rel(50, 1), rel(5, 1)]
    res = spd.evaluate_and_push_down(rels, min_table_size=10, max_selectivity=0.5)
    assert decisions(res) == ["too_small", "probe", "pushed", "pushed", "too_small"]
    assert [r["count"] for r in res] == [0, 0, 1, 1, 0]


def test_max_size_is_floored_and_the_test_is_strict():
    # size 10, ratio 0.25: maxSize = floor(2.5) = 2; count 2 is pushed down, count 3 reverted
    big = rel(100)
    res = spd.evaluate_and_push_down([big, rel(10, 2), rel(10, 3)], min_table_size=0, max_selectivity=0.25)
    assert decisions(res) == ["probe", "pushed", "reverted"]
    assert [r["max_size"] for r in res] == [0, 2, 2]
    assert [r["count"] for r in res] == [0, 2, 3]
    assert list(res[1]["rowids"]) == [0, 1]


def test_ratio_zero_still_pushes_an_empty_selection():
    # maxSize = 0: count 0 is not > 0, so the (empty) selection is pushed down
    res = spd.evaluate_and_push_down([rel(100), rel(20, 0), rel(20, 1)], min_table_size=0, max_selectivity=0.0)
    assert decisions(res) == ["probe", "pushed", "reverted"]
    assert res[1]["count"] == 0 and len(res[1]["rowids"]) == 0


def test_absolute_max_size_replaces_the_ratio():
    res = spd.evaluate_and_push_down([rel(1000), rel(500, 40), rel(500, 41)], min_table_size=0,
                                     max_selectivity=0.9, max_rows=40)
    assert decisions(res) == ["probe", "pushed", "reverted"]
    assert [r["max_size"] for r in res] == [0, 40, 40]


def test_no_selection_and_single_relation():
    assert decisions(spd.evaluate_and_push_down([rel(10, 3)], 0, 1.0)) == ["probe"]
    res = spd.evaluate_and_push_down([rel(30), rel(20)], 0, 1.0)
    assert decisions(res) == ["probe", "no_predicate"]
    assert decisions(spd.evaluate_and_push_down([], 0, 1.0)) == []


def test_projected_columns_follow_the_selected_rows():
    res = spd.evaluate_and_push_down([rel(64), rel(40, 5, proj=(1, 0))], 0, 0.5)
    assert res[1]["decision"] == "pushed"
    c1, c0 = res[1]["columns"]
    assert list(c0) == [0, 1, 2, 3, 4] and list(c1) == [0, 7, 14, 21, 28]
