"""Host-side logic of bench.py (no GPU): the oracle's CPU-baseline sample.

The sample is a prefix of the workload, compared event by event with the
GPU outputs of the same workload, so it may never hold more events than the
workload itself, however fast the oracle is.
"""
import numpy as np

import bench
import oracle as O
from paper_2303_18244_gb300.inputs import process_momenta


def test_oracle_sample_capped_at_the_workload():
    v, cores, n, dt, one, ref = bench.time_oracle("e+ e- > mu+ mu-", 500.0, 1, 0, budget_s=2.0, max_events=3000)
    assert n <= 3000 and ref.shape == (n,) and cores >= 1 and v > 0 and one > 0


def test_oracle_sample_is_the_workload_prefix():
    n_max = 200
    _, _, n, _, _, ref = bench.time_oracle("g g > t t~", 1000.0, 2, 0, budget_s=0.5, one_core=False,
                                           max_events=n_max)
    assert 1 <= n <= n_max
    p = process_momenta("g g > t t~", 1000.0, n, 2)
    np.testing.assert_array_equal(ref, O.me("g g > t t~", p))
