"""The traditional estimator the paper argues against (Ch2), as the baseline
the learned estimator's q-error is compared with.

Each leaf gets the single-column selectivity its statistics give (here the
sample-CDF mass F_hi - F_lo carried in the feature vector, or its complement
for <> and for a negated leaf); an AND multiplies the factors (independence,
the product of §1.1's worked estimate 0.2 x 0.167 x 0.167 x 0.27 = 0.0015)
and an OR adds them minus the joint probability (Ch2), i.e. 1 - prod(1 - p)
over the OR's operands.
"""
from __future__ import annotations

import numpy as np

SLOT, N_SLOTS = 24, 6


def combine_and(ps) -> float:
    out = 1.0
    for p in ps:
        out *= p
    return out


def combine_or(ps) -> float:
    out = 1.0
    for p in ps:
        out *= 1.0 - p
    return 1.0 - out


def independence_selectivity(features: np.ndarray) -> np.ndarray:
    """Selectivity per predicate from its 144 features (rows of a float array)."""
    f = np.asarray(features, np.float64).reshape(-1, N_SLOTS, SLOT)
    out = np.zeros(f.shape[0])
    for i in range(f.shape[0]):
        groups = {}
        for s in range(N_SLOTS):
            slot = f[i, s]
            if slot[:8].max() < 0.5:     # unused slot (no column)
                continue
            p = max(0.0, slot[19] - slot[18])
            if slot[8 + 1] > 0.5:        # <>: complement of the equality mass
                p = 1.0 - p
            if slot[17] > 0.5:           # NOT
                p = 1.0 - p
            g = int(np.argmax(slot[20:23]))
            groups.setdefault(g, []).append(p)
        out[i] = combine_or([combine_and(ps) for ps in groups.values()]) if groups else 0.0
    return out


# ----------------------------------------------------------------------------
# Ch2's other traditional estimators, on predicate trees (the same tuples the
# library compiles: ("cmp", col, op, v), ("between", col, lo, hi), ("in", col,
# values), ("like", col, prefix), ("and"/"or", [...]), ("not", x), ("true",),
# ("false",)).  They are baselines for the exact count and the learned
# estimator; none of them is on the library's path.
# ----------------------------------------------------------------------------

class EquiDepthHistogram:
    """Equi-depth histogram of one column (Ch2): B buckets holding the same
    number of values D = T(R) / B, each with its value range [lo, hi] and its
    number of distinct values V(b).  Built from a sample of the column, the
    depth scaled to the table's row count."""

    def __init__(self, lo: np.ndarray, hi: np.ndarray, distinct: np.ndarray, depth: float):
        self.lo = np.asarray(lo, np.float64)
        self.hi = np.asarray(hi, np.float64)
        self.distinct = np.maximum(np.asarray(distinct, np.float64), 1.0)
        self.depth = float(depth)

    @classmethod
    def build(cls, sample: np.ndarray, n_rows: int, buckets: int = 64) -> "EquiDepthHistogram":
        s = np.sort(np.asarray(sample, np.float64))
        edges = np.linspace(0, len(s), buckets + 1).astype(np.int64)
        lo, hi, dv = [], [], []
        for a, b in zip(edges[:-1], edges[1:]):
            if b <= a:
                continue
            part = s[a:b]
            lo.append(part[0])
            hi.append(part[-1])
            dv.append(len(np.unique(part)))
        return cls(lo, hi, dv, float(n_rows) / max(1, len(lo)))

    @property
    def n_rows(self) -> float:
        return self.depth * len(self.lo)

    def eq_rows(self, x: float) -> float:
        """|sigma_{A=x}(R)| = sum over the buckets that contain x of D / V(b)."""
        inside = (self.lo <= x) & (x <= self.hi)
        return float(np.sum(self.depth / self.distinct[inside]))

    def below_rows(self, x: float, inclusive: bool) -> float:
        """Rows with A < x (A <= x): whole buckets below x, plus the share of a
        bucket x falls in, values spread uniformly over its range."""
        total = 0.0
        for lo, hi, dv in zip(self.lo, self.hi, self.distinct):
            if hi < x or (inclusive and hi <= x):
                total += self.depth
            elif lo < x or (inclusive and lo <= x):
                if hi > lo:
                    total += self.depth * (x - lo) / (hi - lo)
                if inclusive:
                    total += self.depth / dv   # the value x itself
        return min(total, self.n_rows)


def _leaf_values(node, dicts):
    """The set of equality values a set-like leaf stands for (IN list, LIKE codes)."""
    if node[0] == "in":
        return list(node[2])
    d = dicts[node[1]]
    p = node[2].encode() if isinstance(node[2], str) else node[2]
    return [code for code, s in enumerate(d) if s.startswith(p)]


def textbook_selectivity(tree, distinct, dicts=None) -> float:
    """Ch2's heuristics: A = x -> 1/V(R,A); an inequality -> 1/3 (BETWEEN, the
    paper's `B < y1 AND B > y2`, -> 1/3 * 1/3); IN and LIKE -> an OR of
    equalities; AND multiplies, OR adds minus the joint probability, NOT
    complements."""
    k = tree[0]
    if k == "true":
        return 1.0
    if k == "false":
        return 0.0
    if k == "not":
        return 1.0 - textbook_selectivity(tree[1], distinct, dicts)
    if k == "and":
        return combine_and([textbook_selectivity(c, distinct, dicts) for c in tree[1]])
    if k == "or":
        return combine_or([textbook_selectivity(c, distinct, dicts) for c in tree[1]])
    v = max(1.0, float(distinct[tree[1]]))
    if k == "cmp":
        op = tree[2]
        if op == "=":
            return 1.0 / v
        if op == "<>":
            return 1.0 - 1.0 / v
        return 1.0 / 3.0
    if k == "between":
        return 1.0 / 9.0
    if k in ("in", "like"):
        return combine_or([1.0 / v] * len(set(_leaf_values(tree, dicts))))
    raise ValueError(k)


def histogram_selectivity(tree, hists: list, dicts=None) -> float:
    """One equi-depth histogram per column (Ch2) for every leaf, the leaves
    combined as independent (AND: product; OR: sum minus joint probability)."""
    k = tree[0]
    if k == "true":
        return 1.0
    if k == "false":
        return 0.0
    if k == "not":
        return 1.0 - histogram_selectivity(tree[1], hists, dicts)
    if k == "and":
        return combine_and([histogram_selectivity(c, hists, dicts) for c in tree[1]])
    if k == "or":
        return combine_or([histogram_selectivity(c, hists, dicts) for c in tree[1]])
    h = hists[tree[1]]
    n = h.n_rows
    if k == "cmp":
        op, x = tree[2], float(tree[3])
        if op == "=":
            r = h.eq_rows(x)
        elif op == "<>":
            r = n - h.eq_rows(x)
        elif op in ("<", "<="):
            r = h.below_rows(x, op == "<=")
        else:
            r = n - h.below_rows(x, op == ">")
        return min(max(r / n, 0.0), 1.0)
    if k == "between":
        lo, hi = float(tree[2]), float(tree[3])
        if lo > hi:
            return 0.0
        return min(max((h.below_rows(hi, True) - h.below_rows(lo, False)) / n, 0.0), 1.0)
    if k in ("in", "like"):
        return min(sum(h.eq_rows(float(x)) for x in set(_leaf_values(tree, dicts))) / n, 1.0)
    raise ValueError(k)


def row_sample(columns, sample_rows: int, seed: int):
    """R': sample_rows rows of the table drawn uniformly with replacement
    (a seeded torch generator on the columns' device); returns columns
    (``.type``, ``.data``, ``.dictionary``) holding the sampled rows, whose
    selection the library's count kernel then counts."""
    import torch
    dev = columns[0].data.device
    n = int(columns[0].data.numel())
    g = torch.Generator(device=dev)
    g.manual_seed(seed)
    rows = torch.randint(0, n, (sample_rows,), generator=g, device=dev)
    return [SampledColumn(c.type, c.data[rows].contiguous(), c.dictionary) for c in columns]


class SampledColumn:
    """A sampled column: type name, data tensor and dictionary (or None)."""

    def __init__(self, type_name: str, data, dictionary):
        self.type, self.data, self.dictionary = type_name, data, dictionary


def sampling_estimate(sample_count: int, sample_rows: int, n_rows: int) -> float:
    """|sigma(R)| = |sigma(R')| * |R| / |R'| (Ch2), R' a random row sample."""
    return float(sample_count) * float(n_rows) / float(max(1, sample_rows))
