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
