"""Ch2's sampling estimator on the GPU path: the library's count of each
predicate over a row sample R' equals the oracle's count over the same
sampled rows (exact), and the estimate is that count times |R| / |R'|."""
import numpy as np
import pytest

import datagen as dg
import oracle
import paper_1806_08384_b300 as sel
from paper_1806_08384_b300 import baselines

pytestmark = pytest.mark.gpu


def test_sampling_counts_equal_the_oracle_on_the_sample(dev):
    t = dg.gen_table("cfg2", dg.config2_specs(), 2_000_003, dev)
    sample = baselines.row_sample(t.columns, 65_536, seed=17)
    TS = sel.Table(sample)
    ots = oracle.OTable([c.data.cpu().numpy() for c in sample], [c.type for c in sample],
                        [c.dictionary for c in sample])
    rng = np.random.default_rng(4)
    trees = [dg.random_dnf_predicate(dg.config2_specs(), rng) for _ in range(200)]
    trees += [dg.config2_predicate(s) for s in dg.CONFIG2_TARGETS]
    ctx = sel.Context()
    got = sel.count_many(ctx, [sel.Predicate(TS, tr) for tr in trees], TS)
    want = [oracle.count(ots, tr) for tr in trees]
    assert got == want
    est = [baselines.sampling_estimate(c, 65_536, t.n_rows) for c in got]
    assert est == [c * t.n_rows / 65_536 for c in want]
    again = baselines.row_sample(t.columns, 65_536, seed=17)   # the same seed draws the same rows
    assert all(bool((a.data == b.data).all()) for a, b in zip(sample, again))
