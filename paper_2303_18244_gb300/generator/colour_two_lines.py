"""Colour algebra of u u~ -> t t~ g: two quark lines and one gluon.

Colour indices: u i (incoming quark), u~ j (incoming antiquark), t k
(outgoing quark), t~ l (outgoing antiquark), gluon a.  Colour-flow basis
(each an invariant tensor in those indices):

    c0 = (T^a)_{k i} delta_{j l}      c1 = delta_{k i} (T^a)_{j l}
    c2 = (T^a)_{j i} delta_{k l}      c3 = delta_{j i} (T^a)_{k l}

The five diagrams' colour factors (gluon emitted at the u end, the u~ end,
the t end, the t~ end, and by the three-gluon vertex)

    D1 = sum_b (T^b T^a)_{ji} T^b_{kl}     D2 = sum_b (T^a T^b)_{ji} T^b_{kl}
    D3 = sum_b T^b_{ji} (T^a T^b)_{kl}     D4 = sum_b T^b_{ji} (T^b T^a)_{kl}
    D5 = sum_{bc} f^{bca} T^b_{ji} T^c_{kl}

decompose exactly onto the basis by the Fierz identity; this module evaluates
every tensor by explicit index sums over the Gell-Mann generators, solves for
the decomposition, checks that it is exact, and returns it with the colour
matrix C_mn = sum_{ijkla} conj(c_m) c_n as exact fractions.
"""
from __future__ import annotations

from fractions import Fraction

import numpy as np


def gell_mann_generators() -> np.ndarray:
    """T^a = lambda^a / 2, [8][3][3]."""
    lam = np.zeros((8, 3, 3), dtype=complex)
    lam[0][0, 1] = lam[0][1, 0] = 1
    lam[1][0, 1], lam[1][1, 0] = -1j, 1j
    lam[2][0, 0], lam[2][1, 1] = 1, -1
    lam[3][0, 2] = lam[3][2, 0] = 1
    lam[4][0, 2], lam[4][2, 0] = -1j, 1j
    lam[5][1, 2] = lam[5][2, 1] = 1
    lam[6][1, 2], lam[6][2, 1] = -1j, 1j
    lam[7][0, 0] = lam[7][1, 1] = 1 / np.sqrt(3)
    lam[7][2, 2] = -2 / np.sqrt(3)
    return lam / 2


def _tensors():
    T = gell_mann_generators()
    d = np.eye(3)
    # f^{abc} = -2 i Tr([T^a, T^b] T^c)
    comm = np.einsum("aij,bjk->abik", T, T) - np.einsum("bij,ajk->abik", T, T)
    f = np.real(-2j * np.einsum("abij,cji->abc", comm, T))
    basis = [
        np.einsum("aki,jl->ijkla", T, d),
        np.einsum("ki,ajl->ijkla", d, T),
        np.einsum("aji,kl->ijkla", T, d),
        np.einsum("ji,akl->ijkla", d, T),
    ]
    diagrams = [
        np.einsum("bjm,ami,bkl->ijkla", T, T, T),
        np.einsum("ajm,bmi,bkl->ijkla", T, T, T),
        np.einsum("bji,akm,bml->ijkla", T, T, T),
        np.einsum("bji,bkm,aml->ijkla", T, T, T),
        np.einsum("bca,bji,ckl->ijkla", f, T, T),
    ]
    return basis, diagrams


def _rational(x: complex, den: int = 36) -> tuple[Fraction, Fraction]:
    re, im = Fraction(round(x.real * den), den), Fraction(round(x.imag * den), den)
    assert abs(float(re) - x.real) < 1e-12 and abs(float(im) - x.imag) < 1e-12, x
    return re, im


def decomposition() -> list[list[tuple[Fraction, Fraction]]]:
    """coef[d][m] (real, imaginary parts): colour factor of diagram d equals
    sum_m coef[d][m] c_m exactly."""
    basis, diagrams = _tensors()
    B = np.stack([b.ravel() for b in basis], axis=1)
    out = []
    for D in diagrams:
        x, *_ = np.linalg.lstsq(B, D.ravel(), rcond=None)
        assert np.abs(B @ x - D.ravel()).max() < 1e-12
        out.append([_rational(v) for v in x])
    return out


def colour_matrix() -> list[list[Fraction]]:
    """C_mn = sum over all colour indices of conj(c_m) c_n (real, exact)."""
    basis, _ = _tensors()
    C = []
    for bm in basis:
        row = []
        for bn in basis:
            v = np.sum(np.conj(bm) * bn)
            re, im = _rational(v)
            assert im == 0
            row.append(re)
        C.append(row)
    return C
