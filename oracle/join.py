"""CPU oracle of the join-size estimate's inputs (§1.1, §3.2).  TEST
INFRASTRUCTURE ONLY (imported by tests; never by the library).

* V(sigma_P(R), A): the number of distinct values of column A over the rows
  that satisfy P (all rows without P).  The rows come from the row-by-row
  evaluator (``oracle.select``), the distinct values from a Python set of the
  selected values; float32 -0.0 and +0.0 are one value (they compare equal).
* |R join S| = |R||S| / max(V(R,A), V(S,A)).
* The exact COUNT(*) of sigma_P(R) join sigma_Q(S) on R.a = S.b: for every
  selected row of R, the number of selected rows of S with an equal key
  (a Counter of S's selected keys).
"""
from __future__ import annotations

from collections import Counter
from typing import Optional, Tuple

import numpy as np

from . import OTable, select


def count_distinct(t: OTable, col: int, tree: Optional[tuple] = None, threads: int = 1) -> Tuple[int, int]:
    a = t.arrays[col]
    rows = np.arange(t.n_rows) if tree is None else select(t, tree, threads=threads)
    vals = a[rows]
    if vals.dtype == np.float32:
        vals = np.where(vals == 0, np.float32(0.0), vals)   # -0.0 == +0.0
    return len(set(vals.tolist())), int(len(rows))


def join_size_estimate(rows_r: int, rows_s: int, distinct_r: int, distinct_s: int) -> float:
    v = max(distinct_r, distinct_s)
    return 0.0 if v == 0 else rows_r * rows_s / v


def _keys(t: OTable, col: int, tree: Optional[tuple], threads: int):
    a = t.arrays[col]
    rows = np.arange(t.n_rows) if tree is None else select(t, tree, threads=threads)
    vals = a[rows]
    if vals.dtype == np.float32:
        vals = np.where(vals == 0, np.float32(0.0), vals)
    return vals.tolist()


def join_count(r: OTable, col_r: int, tree_r: Optional[tuple], s: OTable, col_s: int, tree_s: Optional[tuple],
               threads: int = 1) -> Tuple[int, int, int]:
    kr = _keys(r, col_r, tree_r, threads)
    ks = Counter(_keys(s, col_s, tree_s, threads))
    return sum(ks.get(k, 0) for k in kr), len(kr), sum(ks.values())
