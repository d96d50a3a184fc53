"""Seeded inputs: Philox4x64-10 against numpy's implementation, RAMBO flatness."""
import numpy as np
import pytest

from paper_2303_18244_gb300.inputs import philox4x64_10, process_momenta, rambo, uniforms


@pytest.mark.parametrize("key", [0, 1, 5, 12345678901234567])
@pytest.mark.parametrize("ctr", [(1, 0, 0, 0), (1, 2, 3, 4), (7, 0, 0, 0), (2**40 + 3, 9, 1, 0)])
def test_philox_block_matches_numpy(key, ctr):
    # numpy's Philox(counter=c) increments first: its first block is block(c + 1)
    c_prev = list(ctr)
    c_prev[0] -= 1
    ref = np.random.Philox(key=key, counter=np.array(c_prev, dtype=np.uint64)).random_raw(4)
    mine = philox4x64_10(np.array(ctr, dtype=np.uint64), np.array([key, 0], dtype=np.uint64))
    assert [int(a) for a in ref] == [int(b) for b in mine]


def test_uniforms_open_interval_and_cut_invariance():
    u = uniforms(3, 0, 2000, 4)
    assert np.all(u > 0.0) and np.all(u < 1.0)
    v = uniforms(3, 1000, 1000, 4)
    assert np.array_equal(u[1000:], v)
    assert abs(u.mean() - 0.5) < 0.01


@pytest.mark.parametrize("proc,sqrts,mt", [
    ("e+ e- > mu+ mu-", 500.0, 0.0), ("g g > t t~", 1000.0, 173.0),
    ("g g > t t~ g g", 1500.0, 173.0), ("g g > t t~ g g g", 2000.0, 173.0)])
def test_rambo_conservation_and_shell(proc, sqrts, mt):
    p = process_momenta(proc, sqrts, 500, 11, mt=mt)
    tot_in = p[:, :2].sum(axis=1)
    tot_out = p[:, 2:].sum(axis=1)
    # 4-momentum conserved to rounding (the imbalance of the conformal map is removed)
    assert np.allclose(tot_in, tot_out, rtol=0, atol=2e-15 * sqrts)
    m2 = p[..., 0] ** 2 - (p[..., 1:] ** 2).sum(-1)
    want = np.zeros(p.shape[1])
    if "t t~" in proc:
        want[2:4] = mt * mt
    assert np.allclose(m2, want[None, :], atol=1e-7 * sqrts * sqrts)
    assert np.all(p[..., 0] > 0)


def test_rambo_two_body_isotropic():
    # flat two-body phase space: cos(theta) uniform on [-1, 1]
    p = process_momenta("e+ e- > mu+ mu-", 500.0, 20000, 1)
    c = p[:, 3, 3] / np.linalg.norm(p[:, 3, 1:], axis=1)
    cs = np.sort(c)
    d = np.max(np.abs(cs - (np.arange(1, cs.size + 1) / cs.size * 2 - 1)) / 2)
    assert d < 1.63 / np.sqrt(cs.size) * 1.2  # KS at ~1 % level


def test_rambo_three_body_dalitz_flat():
    # flat massless three-body phase space: x = 2E/sqrt(s) has P(x < a) = a^2
    u = uniforms(5, 0, 20000, 3)
    p = rambo(100.0, [0.0, 0.0, 0.0], u)
    x = np.sort(2.0 * p[:, 0, 0] / 100.0)
    cdf = x ** 2
    emp = np.arange(1, x.size + 1) / x.size
    assert np.max(np.abs(emp - cdf)) < 1.63 / np.sqrt(x.size) * 1.2
