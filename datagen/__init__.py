"""Seeded synthetic inputs: columnar tables and predicate trees.

This module is shared by the CUDA path's tests/bench and by the CPU oracle.
It holds no arithmetic of the method itself (no predicate evaluation, no
counting, no compaction): it only draws table columns from stated
distributions and builds predicate trees with seeded constants.

Workload shapes stand in for the TPC-H / SSB data the paper measured on
(Ch5 "Evaluation", §5.1 Setup): one very large fact table, smaller dimension
tables, skewed (Zipf) keys, dictionary-encoded strings and dates spread over
about seven years.  Nothing from any benchmark suite is reproduced.

Predicate trees use a neutral nested-tuple form:

    ("and", [child, ...])          n-ary conjunction (n >= 1)
    ("or",  [child, ...])          n-ary disjunction (n >= 1)
    ("not", child)
    ("cmp", col, op, value)        op in "=", "<>", "<", "<=", ">", ">="
    ("between", col, lo, hi)       inclusive on both ends
    ("in", col, [v, ...])          set membership, duplicates allowed
    ("like", col, "prefix")        LIKE 'prefix%' on a dictionary column
    ("true",) / ("false",)

``col`` is a column index into the table.  Constants for float32 columns are
Python floats that are exactly representable in binary32; constants for the
integer-like columns are Python ints.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Callable, List, Optional, Sequence

import numpy as np
import torch

MASTER_SEED = 20180612
CHUNK_ROWS = 1 << 24          # rows drawn per generator stream (fixed => prefixes are stable)
DATE_BASE = 8035              # 1992-01-01 as days since 1970-01-01
DATE_SPAN = 2555              # about seven years of days

TYPES = ("i32", "i64", "f32", "date", "dict")
TYPE_WIDTH = {"i32": 4, "i64": 8, "f32": 4, "date": 4, "dict": 4}
TORCH_DTYPE = {"i32": torch.int32, "i64": torch.int64, "f32": torch.float32,
               "date": torch.int32, "dict": torch.int32}

_M64 = (1 << 64) - 1


def splitmix64(x: int) -> int:
    """SplitMix64 finaliser (Steele, Lea, Flood 2014) on a Python int."""
    x = (x + 0x9E3779B97F4A7C15) & _M64
    z = x
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
    return z ^ (z >> 31)


def mix_seed(*parts) -> int:
    """Derive a 63-bit stream seed from the master seed and any labels."""
    h = MASTER_SEED
    for p in parts:
        if isinstance(p, str):
            for ch in p.encode():
                h = splitmix64(h ^ ch)
        else:
            h = splitmix64(h ^ (int(p) & _M64))
    return h & ((1 << 63) - 1)


# ----------------------------------------------------------------------------
# column specifications
# ----------------------------------------------------------------------------

@dataclasses.dataclass
class ColumnSpec:
    name: str
    type: str                 # one of TYPES
    dist: str                 # uniform | zipf | normal | lognormal | date | index
    lo: float = 0.0           # uniform lower bound (inclusive)
    hi: float = 0.0           # uniform upper bound (exclusive)
    n_values: int = 0         # zipf / dict domain size
    s: float = 1.0            # zipf exponent
    dict_seed: int = 0        # dictionary strings seed (dict columns)
    permute: bool = False     # zipf rank -> value through a seeded permutation

    @property
    def width(self) -> int:
        return TYPE_WIDTH[self.type]


@dataclasses.dataclass
class Column:
    spec: ColumnSpec
    data: torch.Tensor
    dictionary: Optional[List[bytes]] = None

    @property
    def name(self):
        return self.spec.name

    @property
    def type(self):
        return self.spec.type


@dataclasses.dataclass
class Table:
    name: str
    columns: List[Column]

    @property
    def n_rows(self) -> int:
        return 0 if not self.columns else int(self.columns[0].data.numel())

    def index(self, name: str) -> int:
        for i, c in enumerate(self.columns):
            if c.name == name:
                return i
        raise KeyError(name)

    def nbytes(self, cols: Optional[Sequence[int]] = None) -> int:
        cols = range(len(self.columns)) if cols is None else cols
        return sum(self.columns[c].spec.width * self.n_rows for c in cols)

    def to(self, device) -> "Table":
        return Table(self.name, [Column(c.spec, c.data.to(device), c.dictionary) for c in self.columns])

    def numpy(self):
        return [c.data.cpu().numpy() for c in self.columns]


# ----------------------------------------------------------------------------
# distributions
# ----------------------------------------------------------------------------

_ZIPF_CACHE = {}


_PMF_CACHE = {}


def zipf_pmf(n_values: int, s: float) -> np.ndarray:
    """P(k) proportional to k^-s for k = 1..n_values (float64), cached."""
    key = (n_values, s)
    if key not in _PMF_CACHE:
        w = np.arange(1, n_values + 1, dtype=np.float64) ** (-s)
        _PMF_CACHE[key] = w / w.sum()
    return _PMF_CACHE[key]


def zipf_cdf(n_values: int, s: float) -> np.ndarray:
    key = (n_values, s)
    if key not in _ZIPF_CACHE:
        c = np.cumsum(zipf_pmf(n_values, s))
        c /= c[-1]
        c[-1] = 1.0
        _ZIPF_CACHE[key] = c
    return _ZIPF_CACHE[key]


_RANK_CACHE = {}


def zipf_rank_values(spec: ColumnSpec) -> np.ndarray:
    """Map 0-based Zipf rank -> stored value for a zipf / dict column (cached)."""
    key = (spec.type, spec.name, spec.n_values, spec.dict_seed, spec.permute)
    if key not in _RANK_CACHE:
        _RANK_CACHE[key] = _zipf_rank_values(spec)
    return _RANK_CACHE[key]


def _zipf_rank_values(spec: ColumnSpec) -> np.ndarray:
    if spec.type == "i64":
        # int64 key domain: rank k (1-based) -> splitmix64(k) as signed int64
        ks = np.arange(1, spec.n_values + 1, dtype=np.uint64)
        z = ks + np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
        return z.view(np.int64)
    if spec.permute:
        rng = np.random.default_rng(mix_seed("perm", spec.name, spec.n_values, spec.dict_seed))
        return rng.permutation(spec.n_values).astype(np.int32)
    return np.arange(spec.n_values, dtype=np.int32)


def make_dictionary(n_entries: int, seed: int) -> List[bytes]:
    """n unique lowercase strings of 2-12 letters, sorted byte-wise."""
    rng = np.random.default_rng(mix_seed("dict", n_entries, seed))
    out = set()
    while len(out) < n_entries:
        ln = int(rng.integers(2, 13))
        letters = rng.integers(0, 26, size=ln)
        out.add(bytes(int(97 + x) for x in letters))
    return sorted(out)


def _gen_chunk(spec: ColumnSpec, n: int, g: torch.Generator, device, rank_tab, cdf_t) -> torch.Tensor:
    d = spec.dist
    if d == "uniform":
        if spec.type == "f32":
            u = torch.rand(n, generator=g, device=device, dtype=torch.float32)
            return (u * float(spec.hi - spec.lo) + float(spec.lo)).to(torch.float32)
        return torch.randint(int(spec.lo), int(spec.hi), (n,), generator=g, device=device,
                             dtype=TORCH_DTYPE[spec.type])
    if d == "date":
        return torch.randint(DATE_BASE, DATE_BASE + DATE_SPAN, (n,), generator=g, device=device,
                             dtype=torch.int32)
    if d == "normal":
        return torch.randn(n, generator=g, device=device, dtype=torch.float32)
    if d == "lognormal":
        return torch.exp(torch.randn(n, generator=g, device=device, dtype=torch.float32))
    if d == "zipf":
        u = torch.rand(n, generator=g, device=device, dtype=torch.float64)
        r = torch.searchsorted(cdf_t, u, right=True).clamp_(max=spec.n_values - 1)
        return rank_tab[r]
    raise ValueError(d)


def gen_column(spec: ColumnSpec, n: int, seed: int, device="cpu") -> Column:
    """Draw n rows of one column; identical prefixes for any n (fixed chunking)."""
    device = torch.device(device)
    dtype = TORCH_DTYPE[spec.type]
    out = torch.empty(n, dtype=dtype, device=device)
    rank_tab = cdf_t = None
    dictionary = None
    if spec.dist == "zipf":
        cdf_t = torch.from_numpy(zipf_cdf(spec.n_values, spec.s)).to(device)
        rank_tab = torch.from_numpy(zipf_rank_values(spec)).to(device=device, dtype=dtype)
    if spec.type == "dict":
        dictionary = make_dictionary(spec.n_values, spec.dict_seed)
    if spec.dist == "index":
        # a seeded bijection of the row index (used by closed-form tests)
        rng = np.random.default_rng(seed)
        out.copy_(torch.from_numpy(rng.permutation(n).astype(np.int32)))
        return Column(spec, out, dictionary)
    for c0 in range(0, n, CHUNK_ROWS):
        m = min(CHUNK_ROWS, n - c0)
        g = torch.Generator(device=device)
        g.manual_seed(mix_seed(seed, c0 // CHUNK_ROWS))
        out[c0:c0 + m] = _gen_chunk(spec, m, g, device, rank_tab, cdf_t)
    return Column(spec, out, dictionary)


def gen_table(name: str, specs: Sequence[ColumnSpec], n: int, device="cpu", cfg_label=None) -> Table:
    label = cfg_label or name
    cols = [gen_column(s, n, mix_seed(label, s.name), device) for s in specs]
    return Table(name, cols)


# ----------------------------------------------------------------------------
# the five workload shapes
# ----------------------------------------------------------------------------

def config1_specs():
    return [ColumnSpec("c0", "i32", "uniform", 0, 1_000_000),
            ColumnSpec("c1", "i32", "zipf", n_values=1000, s=1.2),
            ColumnSpec("c2", "f32", "normal"),
            ColumnSpec("c3", "date", "date")]


def config2_specs():
    return [ColumnSpec("k0", "i32", "uniform", 0, 2 ** 31),
            ColumnSpec("k1", "i32", "uniform", 0, 2 ** 31),
            ColumnSpec("k2", "i64", "zipf", n_values=1 << 24, s=1.1),
            ColumnSpec("f0", "f32", "uniform", 0.0, 1e5),
            ColumnSpec("f1", "f32", "lognormal"),
            ColumnSpec("d", "date", "date"),
            ColumnSpec("s0", "dict", "zipf", n_values=25, s=1.1, dict_seed=25, permute=True),
            ColumnSpec("s1", "dict", "zipf", n_values=10_000, s=1.1, dict_seed=10_000, permute=True)]


def config3_fact_specs():
    return [ColumnSpec("a0", "i32", "uniform", 0, 2 ** 31),
            ColumnSpec("a1", "i32", "zipf", n_values=1000, s=1.1),
            ColumnSpec("a2", "i32", "uniform", 0, 1_000_000),
            ColumnSpec("b0", "f32", "uniform", 0.0, 1.0),
            ColumnSpec("b1", "f32", "normal"),
            ColumnSpec("b2", "f32", "uniform", 0.0, 1e5)]


def config3_dim_specs(dim: int, n_rows: int):
    return [ColumnSpec(f"key{dim}", "i32", "uniform", 0, max(2, n_rows)),
            ColumnSpec(f"s25_{dim}", "dict", "zipf", n_values=25, s=1.1, dict_seed=25, permute=True),
            ColumnSpec(f"s1k_{dim}", "dict", "zipf", n_values=1000, s=1.1, dict_seed=1000, permute=True),
            ColumnSpec(f"v{dim}", "i32", "uniform", 0, 10_000)]


CONFIG3_DIM_ROWS = (2_000, 200_000, 2_400_000, 16_000_000)
CONFIG3_FACT_ROWS = 480_000_000


def config5_specs():
    return [ColumnSpec("u0", "i32", "uniform", 0, 2 ** 31),
            ColumnSpec("z1", "i32", "zipf", n_values=100_000, s=1.1),
            ColumnSpec("u2", "i32", "uniform", 0, 1_000_000),
            ColumnSpec("g0", "f32", "normal"),
            ColumnSpec("g1", "f32", "uniform", 0.0, 1.0),
            ColumnSpec("s", "dict", "zipf", n_values=1000, s=1.1, dict_seed=1000, permute=True)]


def config1_table(n=1_000_000, device="cpu"):
    return gen_table("cfg1", config1_specs(), n, device)


def config2_table(n=300_000_000, device="cpu"):
    return gen_table("cfg2", config2_specs(), n, device)


def config3_tables(fact_rows=CONFIG3_FACT_ROWS, dim_rows=CONFIG3_DIM_ROWS, device="cpu"):
    tabs = [gen_table("cfg3_fact", config3_fact_specs(), fact_rows, device)]
    for i, n in enumerate(dim_rows):
        tabs.append(gen_table(f"cfg3_dim{i}", config3_dim_specs(i, n), n, device))
    return tabs


def config5_table(n=1_200_000_000, device="cpu"):
    return gen_table("cfg5", config5_specs(), n, device)


# ----------------------------------------------------------------------------
# predicate construction helpers
# ----------------------------------------------------------------------------

def f32(x: float) -> float:
    """Round a Python float to the nearest binary32 value (returned as float)."""
    return float(np.float32(x))


def p_and(*c):
    return ("and", list(c))


def p_or(*c):
    return ("or", list(c))


def p_not(c):
    return ("not", c)


def p_cmp(col, op, v):
    return ("cmp", col, op, v)


def p_between(col, lo, hi):
    return ("between", col, lo, hi)


def p_in(col, vals):
    return ("in", col, list(vals))


def p_like(col, prefix: str):
    return ("like", col, prefix)


P_TRUE = ("true",)
P_FALSE = ("false",)


def tree_columns(t) -> List[int]:
    """Distinct column indices referenced by a tree (ascending)."""
    out = set()

    def walk(n):
        k = n[0]
        if k in ("and", "or"):
            for c in n[1]:
                walk(c)
        elif k == "not":
            walk(n[1])
        elif k in ("cmp", "between", "in", "like"):
            out.add(n[1])
    walk(t)
    return sorted(out)


def tree_leaves(t) -> int:
    k = t[0]
    if k in ("and", "or"):
        return sum(tree_leaves(c) for c in t[1])
    if k == "not":
        return tree_leaves(t[1])
    return 1


# ----------------------------------------------------------------------------
# targeted clauses (approximate per-clause selectivity p)
# ----------------------------------------------------------------------------

def _ndtri(p):
    from scipy.special import ndtri
    return float(ndtri(min(max(p, 1e-12), 1 - 1e-12)))


def _prefix_masses(spec: ColumnSpec):
    """All (prefix, probability mass) pairs of length 1..3 for a dict column."""
    d = make_dictionary(spec.n_values, spec.dict_seed)
    pmf = zipf_pmf(spec.n_values, spec.s)
    rank_of_code = np.empty(spec.n_values, dtype=np.int64)
    rank_of_code[zipf_rank_values(spec)] = np.arange(spec.n_values)
    code_mass = pmf[rank_of_code]
    acc = {}
    for code, w in enumerate(d):
        for ln in (1, 2, 3):
            if len(w) >= ln:
                acc[w[:ln]] = acc.get(w[:ln], 0.0) + code_mass[code]
    return sorted(acc.items())


_PREFIX_CACHE = {}


def clause_for(spec: ColumnSpec, col: int, p: float, rng: np.random.Generator, kind=None):
    """A clause on column ``col`` whose selectivity is about p (0 < p <= 1)."""
    p = min(max(p, 1e-9), 1.0)
    if spec.dist in ("uniform", "date") and spec.type in ("i32", "i64", "date"):
        lo, hi = (DATE_BASE, DATE_BASE + DATE_SPAN) if spec.dist == "date" else (int(spec.lo), int(spec.hi))
        span = hi - lo
        w = max(1, int(round(p * span)))
        w = min(w, span)
        a = lo + int(rng.integers(0, span - w + 1))
        return p_between(col, a, a + w - 1)
    if spec.type == "f32":
        if spec.dist == "uniform":
            w = p * (spec.hi - spec.lo)
            a = spec.lo + float(rng.random()) * (spec.hi - spec.lo - w)
            return p_between(col, f32(a), f32(a + w))
        u0 = float(rng.random()) * (1.0 - p)
        a, b = _ndtri(u0), _ndtri(u0 + p)
        if spec.dist == "lognormal":
            a, b = math.exp(a), math.exp(b)
        return p_between(col, f32(a), f32(b))
    if spec.dist == "zipf":
        if spec.type == "dict" and (kind == "like" or (kind is None and rng.random() < 0.5)):
            key = (spec.name, spec.n_values, spec.dict_seed, spec.s)
            if key not in _PREFIX_CACHE:
                _PREFIX_CACHE[key] = _prefix_masses(spec)
            cands = _PREFIX_CACHE[key]
            errs = np.array([abs(math.log(m / p)) for _, m in cands])
            best = np.argsort(errs)[: 3]
            pick = cands[int(best[int(rng.integers(0, len(best)))])][0]
            return p_like(col, pick.decode())
        vals = zipf_rank_values(spec)
        pmf = zipf_pmf(spec.n_values, spec.s)
        # ranks r..r+4 with 5 * pmf(r) ~ p (pmf is decreasing)
        target = p / 5.0
        r = int(np.searchsorted(pmf[::-1], target, side="left"))
        r = spec.n_values - r
        r = min(max(r - 2, 0), max(spec.n_values - 5, 0))
        ranks = [min(r + j, spec.n_values - 1) for j in range(5)]
        return p_in(col, [int(vals[k]) for k in ranks])
    raise ValueError(spec)


def or_of_ands(specs: Sequence[ColumnSpec], target_s: float, rng: np.random.Generator,
               n_groups=3, clauses=(2, 3), columns: Optional[Sequence[int]] = None):
    """OR of n_groups ANDs of 2-3 clauses on distinct columns, aimed at selectivity target_s."""
    columns = list(range(len(specs))) if columns is None else list(columns)
    q = 1.0 - (1.0 - target_s) ** (1.0 / n_groups)
    groups = []
    for _ in range(n_groups):
        k = int(rng.integers(clauses[0], clauses[1] + 1))
        cols = [int(c) for c in rng.choice(columns, size=k, replace=False)]
        p = q ** (1.0 / k)
        groups.append(p_and(*[clause_for(specs[c], c, p, rng) for c in sorted(cols)]))
    return p_or(*groups)


def config1_predicate(seed=0):
    """c0 BETWEEN a AND b AND c1 IN {5 values} AND c2 < t, seeded constants."""
    rng = np.random.default_rng(mix_seed("cfg1_pred", seed))
    a = int(rng.integers(0, 500_000))
    b = a + int(rng.integers(100_000, 500_000))
    vals = [int(v) for v in rng.choice(40, size=5, replace=False)]
    t = f32(float(rng.normal()))
    return p_and(p_between(0, a, b), p_in(1, vals), p_cmp(2, "<", t))


CONFIG2_TARGETS = (1e-4, 1e-3, 1e-2, 0.1, 0.5)
CONFIG2_PROJECTION = ("k0", "k2", "f0", "d")


def config2_predicate(target_s: float, seed=0):
    rng = np.random.default_rng(mix_seed("cfg2_pred", seed, int(round(-math.log10(target_s) * 1000))))
    return or_of_ands(config2_specs(), target_s, rng)


def config3_predicates(seed=0, n_fact=32, n_per_dim=8):
    """(table index, tree) pairs: 32 on the fact table, 8 per dimension table."""
    rng = np.random.default_rng(mix_seed("cfg3_pred", seed))
    out = []
    fact = config3_fact_specs()
    for _ in range(n_fact):
        s = float(10 ** rng.uniform(-4, math.log10(0.5)))
        out.append((0, or_of_ands(fact, s, rng, n_groups=int(rng.integers(1, 4)), clauses=(1, 3))))
    for d, nd in enumerate(CONFIG3_DIM_ROWS):
        specs = config3_dim_specs(d, nd)
        for _ in range(n_per_dim):
            s = float(10 ** rng.uniform(-4, math.log10(0.5)))
            out.append((d + 1, or_of_ands(specs, s, rng, n_groups=int(rng.integers(1, 3)), clauses=(1, 2))))
    return out


def config5_predicates(n=256, seed=0):
    rng = np.random.default_rng(mix_seed("cfg5_pred", seed))
    specs = config5_specs()
    targets = np.logspace(-6, math.log10(0.9), n)
    out = []
    for s in targets:
        g = int(rng.integers(1, 4))
        out.append(or_of_ands(specs, float(s), rng, n_groups=g, clauses=(1, 3)))
    return out


CONFIG5_PROJECTION = ("u0", "z1", "g1")


# ----------------------------------------------------------------------------
# small tables and random trees for brute-force style tests
# ----------------------------------------------------------------------------

def tiny_specs():
    return [ColumnSpec("i", "i32", "uniform", 0, 4),
            ColumnSpec("l", "i64", "uniform", -2, 2),
            ColumnSpec("f", "f32", "uniform", 0.0, 4.0),
            ColumnSpec("d", "date", "date"),
            ColumnSpec("s", "dict", "zipf", n_values=5, s=1.0, dict_seed=5, permute=True)]


def tiny_table(n: int, seed=0, device="cpu") -> Table:
    """Small domains so that every clause is hit often; floats on a 0.5 grid."""
    rng = np.random.default_rng(mix_seed("tiny", n, seed))
    specs = tiny_specs()
    i = rng.integers(0, 4, n).astype(np.int32)
    l = rng.integers(-2, 2, n).astype(np.int64) * (1 << 33)          # values beyond int32
    f = (rng.integers(-2, 8, n) * 0.5).astype(np.float32)             # includes -0.0? no; 0.0 and negatives
    d = (DATE_BASE + rng.integers(0, 4, n)).astype(np.int32)
    s = rng.integers(0, 5, n).astype(np.int32)
    dictionary = make_dictionary(5, 5)
    cols = []
    for spec, arr in zip(specs, (i, l, f, d, s)):
        cols.append(Column(spec, torch.from_numpy(arr).to(device),
                           dictionary if spec.type == "dict" else None))
    return Table(f"tiny{n}", cols)


def tiny_constants(table: Table, col: int):
    """Constants around and inside the tiny domains (including out-of-range ones)."""
    t = table.columns[col].type
    if t == "i32":
        return [-1, 0, 1, 2, 3, 4]
    if t == "i64":
        return [-(2 << 33), -(1 << 33), 0, 1 << 33, 3 << 33, -1]
    if t == "f32":
        return [-1.0, -0.0, 0.0, 0.5, 1.25, 3.5, 4.0]
    if t == "date":
        return [DATE_BASE - 1, DATE_BASE, DATE_BASE + 2, DATE_BASE + 3, DATE_BASE + 4]
    return [-1, 0, 2, 4, 5]


def random_leaf(table: Table, rng: np.random.Generator):
    col = int(rng.integers(0, len(table.columns)))
    t = table.columns[col].type
    consts = tiny_constants(table, col)
    kinds = ["cmp", "between", "in"] + (["like"] if t == "dict" else [])
    k = kinds[int(rng.integers(0, len(kinds)))]
    if k == "cmp":
        op = ("=", "<>", "<", "<=", ">", ">=")[int(rng.integers(0, 6))]
        return p_cmp(col, op, consts[int(rng.integers(0, len(consts)))])
    if k == "between":
        a, b = (consts[int(x)] for x in rng.integers(0, len(consts), 2))
        return p_between(col, a, b)
    if k == "in":
        m = int(rng.integers(0, 5))
        return p_in(col, [consts[int(x)] for x in rng.integers(0, len(consts), m)])
    d = table.columns[col].dictionary
    w = d[int(rng.integers(0, len(d)))]
    return p_like(col, w[: int(rng.integers(0, len(w) + 1))].decode())


def random_tree(table: Table, rng: np.random.Generator, depth=3):
    if depth == 0 or rng.random() < 0.3:
        r = rng.random()
        if r < 0.03:
            return P_TRUE
        if r < 0.06:
            return P_FALSE
        return random_leaf(table, rng)
    k = ("and", "or", "not")[int(rng.integers(0, 3))]
    if k == "not":
        return p_not(random_tree(table, rng, depth - 1))
    m = int(rng.integers(1, 4))
    return (k, [random_tree(table, rng, depth - 1) for _ in range(m)])


# ----------------------------------------------------------------------------
# predicates of the learned estimator's workload (OR of <= 3 ANDs, <= 6 leaves)
# ----------------------------------------------------------------------------

def random_dnf_predicate(specs: Sequence[ColumnSpec], rng: np.random.Generator, max_leaves=6, max_groups=3,
                         prob_not=0.1):
    """Random shape, random clause kinds and operators, per-clause selectivity
    log-uniform in [1e-4, 1]."""
    g = int(rng.integers(1, max_groups + 1))
    sizes = [1] * g
    for _ in range(int(rng.integers(0, max_leaves - g + 1))):
        sizes[int(rng.integers(0, g))] += 1
    groups = []
    for k in sizes:
        cols = [int(c) for c in rng.choice(len(specs), size=min(k, len(specs)), replace=False)]
        leaves = []
        if k >= 2 and rng.random() < 0.4:
            # two one-sided comparisons on one ordered column, as in the paper's
            # "B < y1 AND B > y2" (§1.1): correlated clauses independence gets wrong
            c = int(rng.choice([i for i, sp in enumerate(specs) if sp.type in ("i32", "i64", "f32", "date")
                                and sp.dist != "zipf"]))
            lo_leaf = clause_for(specs[c], c, float(10 ** rng.uniform(-3, math.log10(0.5))), rng)
            a, b = lo_leaf[2], lo_leaf[3]
            leaves += [p_cmp(c, ">=" if rng.random() < 0.5 else ">", a), p_cmp(c, "<=" if rng.random() < 0.5 else "<", b)]
            cols = [x for x in cols if x != c][: k - 2]
        for c in cols:
            p = float(10 ** rng.uniform(-4, 0))
            leaf = clause_for(specs[c], c, p, rng)
            if leaf[0] == "between" and rng.random() < 0.5:     # one-sided comparisons too
                op = ("<", "<=", ">", ">=")[int(rng.integers(0, 4))]
                leaf = p_cmp(c, op, leaf[2] if op in (">", ">=") else leaf[3])
            elif leaf[0] == "in" and rng.random() < 0.3:
                leaf = p_cmp(c, "=" if rng.random() < 0.7 else "<>", leaf[2][0])
            if rng.random() < prob_not:
                leaf = p_not(leaf)
            leaves.append(leaf)
        groups.append(p_and(*leaves) if len(leaves) > 1 else leaves[0])
    return p_or(*groups) if len(groups) > 1 else groups[0]
