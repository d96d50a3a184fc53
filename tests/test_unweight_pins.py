"""Pins of the oracle's hit-or-miss unweighting (paper Sect. 2) to what the
method fixes: the expected number of kept events, the distribution of the kept
sample (it must follow the weights, which also fixes the direction of the
comparison), and the special cases w >= w_max (always kept) and w <= 0 (never)."""
import numpy as np

import oracle as O
from paper_2303_18244_gb300.inputs import uniforms


def _u(seed, n, slot=0):
    return uniforms(seed, 0, n, 1)[:, 0, slot]


def test_expected_number_kept():
    n = 20000
    w = 3.0 * _u(11, n)
    r = _u(12, n)
    w_max = 2.0
    kept = O.unweight(w, r, w_max)
    p = np.minimum(w / w_max, 1.0)
    mean, sd = p.sum(), np.sqrt((p * (1 - p)).sum())
    assert abs(kept.size - mean) < 5 * sd


def test_kept_sample_follows_the_weights():
    # w = x with x uniform in [0, 1): the kept x have density 2x, mean 2/3
    # (the reversed comparison would give density 2(1 - x), mean 1/3)
    n = 40000
    x = _u(13, n)
    r = _u(14, n)
    kept = O.unweight(x, r, 1.0)
    m = x[kept].mean()
    assert abs(m - 2.0 / 3.0) < 5 * np.sqrt(1.0 / 18.0 / kept.size)


def test_special_cases_and_order():
    w = np.array([5.0, 0.0, -1.0, 1.0, 0.5, 0.5, 2.0])
    r = np.array([0.99, 0.0, 0.0, 0.999, 0.49, 0.5, 0.0])
    # w >= w_max kept whatever r; w <= 0 never; 0.49 < 0.5 kept, 0.5 < 0.5 not
    assert O.unweight(w, r, 1.0).tolist() == [0, 3, 4, 6]
    assert O.unweight(np.zeros(0), np.zeros(0), 1.0).size == 0
