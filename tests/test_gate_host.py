"""The gate's threshold rule in the library (sel_mlp_choose_tau, host only)
against the estimator oracle's choose_tau, CPU only.

tau is the largest held-out sigma whose accepted estimates keep the 95th
percentile q-error at or below 2 (reading of the uncertainty rule).  The
library gets the same float32 sigmas as the oracle, so the chosen tau is one
of those values and must be identical; the answered fraction follows."""
import math

import numpy as np
import pytest

from oracle import mlp as om
import paper_1806_08384_b300 as sel


def _case(seed, n):
    rng = np.random.default_rng(seed)
    sigma = rng.choice(np.exp(rng.uniform(-3, 1, 40)), n).astype(np.float32)   # ties
    sigma[rng.random(n) < 0.05] = np.inf                                       # no feature form
    exact = rng.integers(0, 10 ** 6, n).astype(np.uint64)
    exact[rng.random(n) < 0.1] = 0
    # estimates whose error grows with sigma, so that a threshold exists
    est = exact.astype(np.float64) * np.exp(rng.normal(0, 1, n) * sigma.clip(0, 5))
    est[rng.random(n) < 0.05] = 0.0
    return sigma, est, exact


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("max_q", [1.5, 2.0, 4.0])
def test_choose_tau_matches_oracle(seed, max_q):
    sigma, est, exact = _case(seed, 300)
    tau, answered = sel.choose_tau(sigma, est, exact, max_q=max_q)
    want = om.choose_tau(sigma.astype(np.float64), est, exact, max_q=max_q)
    assert tau == want
    assert answered == pytest.approx(float(np.sum(sigma.astype(np.float64) <= want)) / len(sigma) if want > 0 else 0.0)


def test_choose_tau_edge_cases():
    assert sel.choose_tau([], [], []) == (0.0, 0.0)
    assert sel.choose_tau([math.inf, math.inf], [5.0, 5.0], [5, 5]) == (0.0, 0.0)
    tau, ans = sel.choose_tau([0.5], [10.0], [10])
    assert tau == 0.5 and ans == 1.0
    with pytest.raises(sel.SelError):
        sel.choose_tau([0.5], [1.0], [1], quantile=101.0)
