"""Accuracy of the split-precision colour form, derived from its arithmetic
(no GPU).

The mixed path forms sum_ij Re/Im J_i KNUM_ij Re/Im J_j on the tensor cores
(the paper's colour-algebra step in reduced precision, Sect. 3): each event's
flows are scaled by a power of two s that puts max |J| in [1, 2), split into
FP16 hi = fp16(sJ) and lo = fp16(sJ - hi), multiplied by the FP16-exact
integer numerators with FP32 accumulation, and contracted with the FP32 flows
in FP32.  This restates those steps in numpy and applies them to realistic
flows, the oracle's colour-ordered partial amplitudes of gg -> t t~ g g: the
colour form alone stays within 1e-6 of the exact FP64 quadratic form, far
inside the mixed bar of 1e-5 median, while FP16 without the lo part would not
meet it.
"""
import numpy as np
import pytest

import oracle as O
import test_oracle_pins as P
from test_tc_operands_host import _knum


def _colour_form(J, K, split=True):
    n = K.shape[0]
    fr, fi = J.real.astype(np.float32), J.imag.astype(np.float32)
    mx = max(np.abs(fr).max(), np.abs(fi).max())
    s = np.float32(2.0 ** -int(np.floor(np.log2(mx))))
    K32 = K.astype(np.float32)

    def operand(x):
        x = (s * x).astype(np.float32)
        hi = x.astype(np.float16)
        lo = (x - hi.astype(np.float32)).astype(np.float16)
        d = (hi.astype(np.float32) @ K32).astype(np.float32)
        if split:
            d = (d + (lo.astype(np.float32) @ K32).astype(np.float32)).astype(np.float32)
        return d

    dr, di = operand(fr), operand(fi)
    acc = np.float32(0)
    for k in range(n):
        acc = np.float32(acc + fr[k] * dr[k])
        acc = np.float32(acc + fi[k] * di[k])
    return float(acc) / float(s)


@pytest.fixture(scope="module")
def flows():
    """Colour-ordered amplitudes of gg -> t t~ g g for 10 events x 6 spin and
    polarisation states, with the exact FP64 colour form of each."""
    n, knum = _knum("g g > t t~ g g")
    K = np.array(knum, dtype=np.float64).reshape(n, n)
    out = []
    for seed in range(3, 13):
        for pol in range(0, 16, 3):
            p, kin, eps, ub, v = P._qline_states(4, seed, which=(seed & 1, (seed >> 1) & 1), pol=pol)
            A = O.ordered_amps(4, kin, eps, p[2], ub, p[3], v, O.Params())
            out.append((A, float(np.real(np.conj(A) @ K @ A))))
    return K, out


def test_hi_lo_split_meets_the_bar(flows):
    K, cases = flows
    r = np.array([abs(_colour_form(A, K) / exact - 1) for A, exact in cases])
    assert np.median(r) <= 1e-6 and r.max() <= 1e-6


def test_fp16_alone_would_not(flows):
    K, cases = flows
    r = np.array([abs(_colour_form(A, K, split=False) / exact - 1) for A, exact in cases])
    assert np.median(r) > 1e-5
