"""CPU oracle of Algorithm 1, EvaluateAndPushDown (Ch4 §4.2).  TEST
INFRASTRUCTURE ONLY (imported by tests; never by the library).

The steps, in the algorithm's order:
  1. the queue listRA holds every scanned relation R with
     R.size > PUSH_DOWN_MIN_TABLE_SIZE, ordered by size, largest first (the
     paper does not order equal sizes; here they keep their input order);
  2. listRA.pop() removes the largest relation, the one to be probed;
  3. for each remaining R, in queue order, whose selection was pushed down:
     maxSize = R.size * PUSH_DOWN_MAX_SELECTIVITY (floored; or a given
     absolute maxSize), then Execute(compound, isSPD = true, maxSize): the
     COUNT first, an exception (the push-down is reverted) when
     count > maxSize, otherwise the selected rows of the projected columns,
     in row order.
Relations outside the queue, and relations without a pushed-down selection,
are left alone.  Counts and rows come from the row-by-row evaluator in
``oracle.c`` (``oracle.pushdown``).
"""
from __future__ import annotations

from typing import List, Optional, Sequence, Tuple

from . import OTable, max_rows_for_ratio, pushdown


def evaluate_and_push_down(relations: Sequence[Tuple[OTable, Optional[tuple], Sequence[int]]],
                           min_table_size: int, max_selectivity: float = 0.0, max_rows: int = 0,
                           threads: int = 1) -> List[dict]:
    """relations: (table, predicate tree or None, projected columns) per scan.
    Returns per relation: decision (probe / too_small / no_predicate / pushed /
    reverted), count, max_size, and for pushed ones the columns and row ids."""
    out = [{"decision": "too_small", "count": 0, "max_size": 0} for _ in relations]
    queue = [i for i, (t, _, _) in enumerate(relations) if t.n_rows > min_table_size]
    queue.sort(key=lambda i: -relations[i][0].n_rows)   # stable: equal sizes keep input order
    if not queue:
        return out
    out[queue[0]]["decision"] = "probe"
    for i in queue[1:]:
        t, tree, proj = relations[i]
        if tree is None:
            out[i]["decision"] = "no_predicate"
            continue
        ms = max_rows if max_rows else max_rows_for_ratio(t.n_rows, max_selectivity)
        st, n, cols, ids = pushdown(t, tree, proj, ms, threads=threads)
        out[i].update(count=n, max_size=ms)
        if st == "TOO_LARGE":
            out[i]["decision"] = "reverted"
        else:
            out[i].update(decision="pushed", columns=cols, rowids=ids)
    return out
