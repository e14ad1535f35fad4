"""CPU oracle of the learned selectivity estimator.  TEST INFRASTRUCTURE ONLY
(imported by tests, smoke() and the bench's CPU leg; never by the library).

The paper has no learned component: its selectivity is always the exact
COUNT (§3.1).  This module states, plainly and in float64, what the library's
surrogate computes so that the GPU kernels can be checked against it:

* per-column empirical CDF tables from a sample of m rows whose indices come
  from SplitMix64 (Steele, Lea, Flood 2014): idx_i = splitmix64(seed +
  (col + 1) * 2^40 + i) mod n;
* predicate features: the tree is pushed to negation normal form and must be
  an OR of <= 3 ANDs of leaves, <= 6 leaves, on columns 0..7.  Each leaf
  fills a 24-float slot: column one-hot (8), operator one-hot (10: = <> < <=
  > >= BETWEEN IN LIKE, NOT), [F_lo, F_hi] from the CDF, group one-hot (3),
  and the leaf's log selectivity from the sample, ln(max(p, 1/(2m))) /
  ln(2m) in [-1, 0], where p = F_hi - F_lo, complemented for <> and for a
  negated leaf.  F values are sample counts / m in float32; the log term is
  evaluated in float64 and rounded to float32;
* an MLP 144 -> 256 -> 256 -> 256 -> 2 (ReLU) giving (mu, log sigma^2) of
  y = ln(1 + count), trained with the Gaussian negative log-likelihood and
  Adam.  BF16 rounding (round to nearest even) is applied where the GPU
  rounds: the input features, the weights fed to the matrix products, the
  post-ReLU activations and the back-propagated pre-activation gradients
  that feed the tensor-core products.  Everything else is float64 here;
* the gate of the surrogate-gated estimator (the uncertainty rule of the
  heteroscedastic head): sigma = exp(lv / 2) with lv clamped to [-8, 8]; a
  predicate without a feature form, or with sigma > tau, is answered by the
  exact COUNT of §3.1, every other one by max(0, exp(mu) - 1);
* the choice of tau on a held-out split: the largest tau for which the 95th
  percentile of the q-error of the estimates it accepts is at most 2.
"""
from __future__ import annotations

import math
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np

N_SLOTS = 6
SLOT = 24
N_FEAT = N_SLOTS * SLOT          # 144
HIDDEN = 256
LV_MIN, LV_MAX = -8.0, 8.0       # log-variance clamp
OPS = {"=": 0, "<>": 1, "<": 2, "<=": 3, ">": 4, ">=": 5}
_GOLDEN = np.uint64(0x9E3779B97F4A7C15)


# ----------------------------------------------------------------------------
# numerics helpers
# ----------------------------------------------------------------------------

def bf16_round(x) -> np.ndarray:
    """Round float32 values to bfloat16 (round to nearest, ties to even); float32 out."""
    b = np.ascontiguousarray(np.asarray(x, np.float32)).view(np.uint32).astype(np.uint64)
    lsb = (b >> np.uint64(16)) & np.uint64(1)
    r = ((b + np.uint64(0x7FFF) + lsb) >> np.uint64(16)) << np.uint64(16)
    return r.astype(np.uint32).view(np.float32).reshape(np.shape(x))


def splitmix64(z: np.ndarray) -> np.ndarray:
    """SplitMix64 output function applied to state z (uint64 array)."""
    with np.errstate(over="ignore"):
        z = z.astype(np.uint64) + _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        return z ^ (z >> np.uint64(31))


def sample_indices(seed: int, col: int, m: int, n: int) -> np.ndarray:
    base = np.uint64((seed + ((col + 1) << 40)) & 0xFFFFFFFFFFFFFFFF)
    with np.errstate(over="ignore"):
        z = base + np.arange(m, dtype=np.uint64)
    return (splitmix64(z) % np.uint64(n)).astype(np.int64)


class CDF:
    """Sorted sample of one column."""

    def __init__(self, column: np.ndarray, seed: int, col: int, m: int):
        self.m = m
        idx = sample_indices(seed, col, m, column.shape[0])
        self.s = np.sort(column[idx], kind="stable")

    @classmethod
    def from_sample(cls, values) -> "CDF":
        """A CDF over an explicit sample (hand-worked cases)."""
        c = cls.__new__(cls)
        c.s = np.sort(np.asarray(values), kind="stable")
        c.m = int(c.s.shape[0])
        return c

    def below(self, v) -> int:
        return int(np.searchsorted(self.s, v, side="left"))

    def upto(self, v) -> int:
        return int(np.searchsorted(self.s, v, side="right"))

    def frac(self, k: int) -> float:
        return float(np.float32(k) / np.float32(self.m))


# ----------------------------------------------------------------------------
# features
# ----------------------------------------------------------------------------

def _nnf(t, neg=False):
    k = t[0]
    if k == "not":
        return _nnf(t[1], not neg)
    if k in ("and", "or"):
        kk = k if not neg else ("or" if k == "and" else "and")
        return (kk, [_nnf(c, neg) for c in t[1]])
    if k in ("true", "false"):
        return ("const", (k == "true") != neg)
    return ("leaf", t, neg)


def dnf_groups(tree) -> Optional[List[List[Tuple[tuple, bool]]]]:
    """The (leaf, negated) groups of an OR of ANDs of leaves, or None."""
    t = _nnf(tree)

    def group(x):
        if x[0] == "leaf":
            return [(x[1], x[2])]
        if x[0] == "and" and x[1] and all(c[0] == "leaf" for c in x[1]):
            return [(c[1], c[2]) for c in x[1]]
        return None

    if t[0] == "or":
        gs = [group(c) for c in t[1]]
        return None if (not gs or any(g is None for g in gs)) else gs
    g = group(t)
    return None if g is None else [g]


def leaf_bounds(leaf, cdf: CDF, dictionary=None) -> Tuple[float, float]:
    """[F_lo, F_hi] of a leaf's (non-negated) value set from the column sample."""
    k = leaf[0]
    if k == "cmp":
        op, v = leaf[2], leaf[3]
        if op in ("=", "<>"):
            return cdf.frac(cdf.below(v)), cdf.frac(cdf.upto(v))
        if op == "<":
            return 0.0, cdf.frac(cdf.below(v))
        if op == "<=":
            return 0.0, cdf.frac(cdf.upto(v))
        if op == ">":
            return cdf.frac(cdf.upto(v)), 1.0
        return cdf.frac(cdf.below(v)), 1.0
    if k == "between":
        lo = cdf.below(leaf[2])
        return cdf.frac(lo), cdf.frac(max(lo, cdf.upto(leaf[3])))
    if k == "in":
        vals = sorted(set(leaf[2]))
        c = sum(cdf.upto(v) - cdf.below(v) for v in vals)
        return 0.0, cdf.frac(min(c, cdf.m))
    # like: codes whose dictionary string starts with the prefix
    pre = leaf[2].encode() if isinstance(leaf[2], str) else bytes(leaf[2])
    codes = [i for i, w in enumerate(dictionary) if w.startswith(pre)]
    c = sum(cdf.upto(i) - cdf.below(i) for i in codes)
    return 0.0, cdf.frac(min(c, cdf.m))


def log_selectivity(lo: float, hi: float, ne: bool, neg: bool, m: int) -> float:
    p = max(float(hi) - float(lo), 0.0)
    if ne:
        p = 1.0 - p
    if neg:
        p = 1.0 - p
    return float(np.float32(math.log(max(p, 0.5 / m)) / math.log(2.0 * m)))


def op_index(leaf) -> int:
    k = leaf[0]
    if k == "cmp":
        return OPS[leaf[2]]
    return {"between": 6, "in": 7, "like": 8}[k]


def featurize(tree, cdfs: Sequence[CDF], dicts) -> Tuple[np.ndarray, bool]:
    f = np.zeros(N_FEAT, np.float32)
    groups = dnf_groups(tree)
    if groups is None or len(groups) > 3 or sum(len(g) for g in groups) > N_SLOTS:
        return f, False
    s = 0
    for gi, g in enumerate(groups):
        for leaf, neg in g:
            col = int(leaf[1])
            if col >= 8:
                return np.zeros(N_FEAT, np.float32), False
            o = s * SLOT
            f[o + col] = 1.0
            f[o + 8 + op_index(leaf)] = 1.0
            if neg:
                f[o + 17] = 1.0
            lo, hi = leaf_bounds(leaf, cdfs[col], dicts[col])
            f[o + 18] = lo
            f[o + 19] = hi
            f[o + 20 + gi] = 1.0
            f[o + 23] = log_selectivity(lo, hi, leaf[0] == "cmp" and leaf[2] == "<>", neg, cdfs[col].m)
            s += 1
    return f, True


# ----------------------------------------------------------------------------
# the network
# ----------------------------------------------------------------------------

PARAM_SHAPES = [("W1", (HIDDEN, N_FEAT)), ("b1", (HIDDEN,)), ("W2", (HIDDEN, HIDDEN)), ("b2", (HIDDEN,)),
                ("W3", (HIDDEN, HIDDEN)), ("b3", (HIDDEN,)), ("W4", (2, HIDDEN)), ("b4", (2,))]


def forward(P: Dict[str, np.ndarray], X: np.ndarray, exact: bool = False) -> Dict[str, np.ndarray]:
    """exact=True drops every BF16 rounding (used by the finite-difference check)."""
    r = (lambda a: np.asarray(a, np.float64)) if exact else (lambda a: bf16_round(a).astype(np.float64))
    c = {"x": r(X)}
    a = c["x"]
    for l in (1, 2, 3):
        z = a @ r(P[f"W{l}"]).T + P[f"b{l}"].astype(np.float64)
        c[f"z{l}"] = z
        a = r(np.maximum(z, 0.0).astype(np.float64 if exact else np.float32))
        c[f"a{l}"] = a
    out = a @ r(P["W4"]).T + P["b4"].astype(np.float64)
    c["out"] = out
    c["mu"] = out[:, 0]
    c["lv"] = np.clip(out[:, 1], LV_MIN, LV_MAX)
    return c


def nll(mu, lv, y):
    """Mean Gaussian negative log-likelihood (without the constant)."""
    return float(np.mean(0.5 * (lv + (y - mu) ** 2 * np.exp(-lv))))


def loss_and_grads(P, X, y, exact: bool = False):
    c = forward(P, X, exact)
    r = (lambda a: np.asarray(a, np.float64)) if exact else (lambda a: bf16_round(a).astype(np.float64))
    B = X.shape[0]
    mu, lv, out = c["mu"], c["lv"], c["out"]
    y = np.asarray(y, np.float64)
    inv = np.exp(-lv)
    res = y - mu
    dO = np.zeros((B, 2))
    dO[:, 0] = -res * inv / B
    inside = (out[:, 1] > LV_MIN) & (out[:, 1] < LV_MAX)
    dO[:, 1] = 0.5 * (1.0 - res ** 2 * inv) / B * inside
    G = {"W4": dO.T @ c["a3"], "b4": dO.sum(0)}
    dA = dO @ r(P["W4"])
    for l in (3, 2, 1):
        dZ = dA * (c[f"a{l}"] > 0)
        dZr = dZ if exact else bf16_round(dZ.astype(np.float32)).astype(np.float64)
        prev = c[f"a{l - 1}"] if l > 1 else c["x"]
        G[f"W{l}"] = dZr.T @ prev
        G[f"b{l}"] = dZ.sum(0)
        if l > 1:
            dA = dZr @ r(P[f"W{l}"])
    return nll(mu, lv, y), G


def init_params(seed: int) -> Dict[str, np.ndarray]:
    """He-uniform weights, zero biases (float32 masters)."""
    rng = np.random.default_rng(seed)
    P = {}
    for name, shape in PARAM_SHAPES:
        if name.startswith("W"):
            bound = math.sqrt(6.0 / shape[1])
            P[name] = rng.uniform(-bound, bound, size=shape).astype(np.float32)
        else:
            P[name] = np.zeros(shape, np.float32)
    return P


def adam_step(P, G, M, V, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba 2015) of float32 masters, in float64."""
    for k in P:
        g = np.asarray(G[k], np.float64)
        M[k] = b1 * M[k] + (1 - b1) * g
        V[k] = b2 * V[k] + (1 - b2) * g * g
        mh = M[k] / (1 - b1 ** t)
        vh = V[k] / (1 - b2 ** t)
        P[k] = (P[k].astype(np.float64) - lr * mh / (np.sqrt(vh) + eps)).astype(np.float32)


def q_error(est, true) -> np.ndarray:
    """max(est, true) / min(est, true) with both clamped to >= 1."""
    e = np.maximum(np.asarray(est, np.float64), 1.0)
    t = np.maximum(np.asarray(true, np.float64), 1.0)
    return np.maximum(e / t, t / e)


# ----------------------------------------------------------------------------
# the gate (reading c15) and the choice of its threshold
# ----------------------------------------------------------------------------

def gate(mu, lv, ok, tau: float, exact):
    """The surrogate-gated estimate of each predicate.

    mu, lv: the network's two outputs (lv is clamped to [LV_MIN, LV_MAX]);
    ok: the predicate has a feature form; exact: its exact COUNT.  A
    predicate is answered exactly when it has no feature form or when
    sigma = exp(lv / 2) is not <= tau; otherwise by max(0, exp(mu) - 1).
    Returns (estimate, sigma, used_exact); sigma is +inf without a feature
    form."""
    mu = np.asarray(mu, np.float64)
    lv = np.clip(np.asarray(lv, np.float64), LV_MIN, LV_MAX)
    ok = np.asarray(ok, bool)
    exact = np.asarray(exact, np.float64)
    n = mu.shape[0]
    est = np.empty(n, np.float64)
    sigma = np.empty(n, np.float64)
    used = np.empty(n, bool)
    for i in range(n):
        sigma[i] = math.exp(0.5 * lv[i]) if ok[i] else math.inf
        used[i] = (not ok[i]) or not (sigma[i] <= tau)
        est[i] = exact[i] if used[i] else max(0.0, math.expm1(mu[i]))
    return est, sigma, used


def percentile(x, q: float) -> float:
    """The q-th percentile of x by linear interpolation between order
    statistics: h = (n - 1) q / 100, x_(floor h) + (h - floor h)(x_(floor h + 1) - x_(floor h))."""
    s = sorted(float(v) for v in x)
    h = (len(s) - 1) * (q / 100.0)
    lo = int(math.floor(h))
    if lo + 1 >= len(s):
        return s[-1]
    return s[lo] + (h - lo) * (s[lo + 1] - s[lo])


def choose_tau(sigma, est, exact, max_q: float = 2.0, q: float = 95.0) -> float:
    """The largest tau, among the held-out sigmas, whose accepted estimates
    (sigma <= tau) have a q-th percentile q-error of at most max_q; 0.0 (every
    predicate answered exactly) when no tau qualifies.  Predicates with an
    infinite sigma (no feature form) are never accepted."""
    sigma = np.asarray(sigma, np.float64)
    qe = q_error(est, exact)
    best = 0.0
    for t in sorted(set(float(v) for v in sigma if math.isfinite(v))):
        acc = [float(qe[i]) for i in range(sigma.shape[0]) if sigma[i] <= t]
        if acc and percentile(acc, q) <= max_q:
            best = t
    return best
