"""Colour matrices pinned to hand-derived closed forms (no GPU).

The oracle evaluates colour matrices by explicit Gell-Mann index sums; the
generator, on the CUDA side, reduces the same traces symbolically with the
Fierz identity and decomposes the two-quark-line diagrams by solving on the
explicit tensors.  Both are checked here against the closed forms in
tests/golden/colour_closed_forms.txt (derived by hand, each entry with its
derivation), and against each other for 2..5 gluons.  The colour matrix is
the quadratic form of the colour-algebra step (Sect. 3).
"""
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle as O
from paper_2303_18244_gb300.generator import colour, colour_two_lines

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "colour_closed_forms.txt")


def _sections():
    out, cur = {}, None
    with open(GOLDEN) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            if line.startswith("["):
                cur = line.strip("[]")
                out[cur] = []
            else:
                out[cur].append(line.split())
    return out


def _cfrac(tok):
    re, im = tok.split(",")
    return Fraction(re), Fraction(im)


def test_fixture_is_complete():
    s = _sections()
    assert sorted(s) == ["one_line_three_gluons", "two_lines_basis_matrix", "two_lines_decomposition"]
    assert sorted(r[0] for r in s["one_line_three_gluons"]) == ["123", "132", "213", "231", "312", "321"]


def test_oracle_three_gluon_matrix_closed_form():
    """Every entry of the oracle's 6 x 6 matrix equals the closed form of its
    relative order (a swapped operand or a dropped conjugate moves entries
    between the 1/9 and 10/9 classes)."""
    table = {r[0]: Fraction(int(r[1]), 9) for r in _sections()["one_line_three_gluons"]}
    perms = O.permutations(3)
    C = O.colour_matrix(3)
    assert np.max(np.abs(C.imag)) < 1e-14
    for i, s in enumerate(perms):
        pos = {int(g): k + 1 for k, g in enumerate(s)}
        for j, t in enumerate(perms):
            key = "".join(str(pos[int(g)]) for g in t)
            assert abs(C[i, j].real - float(table[key])) < 1e-13, (s, t, key)


def test_generator_three_gluon_matrix_closed_form():
    table = {r[0]: Fraction(int(r[1]), 9) for r in _sections()["one_line_three_gluons"]}
    ws = colour.words(3)
    C = colour.colour_matrix_exact(3)
    for i, s in enumerate(ws):
        pos = {g: k + 1 for k, g in enumerate(s)}
        for j, t in enumerate(ws):
            assert C[i][j] == table["".join(str(pos[g]) for g in t)]


@pytest.mark.parametrize("n", [2, 3, 4, 5])
def test_symbolic_and_index_sum_colour_matrices_agree(n):
    """Two independent evaluations: symbolic Fierz reduction (generator) and
    explicit sums over all 8^n colour assignments (oracle), same ordering."""
    perms = O.permutations(n)
    ws = colour.words(n)
    assert [tuple(int(x) for x in p) for p in perms] == [tuple(w) for w in ws]
    exact = np.array([[float(x) for x in row] for row in colour.colour_matrix_exact(n)])
    C = O.colour_matrix(n)
    np.testing.assert_allclose(C.real, exact, rtol=0, atol=1e-12 * np.abs(exact).max())
    assert np.max(np.abs(C.imag)) < 1e-12


def test_two_line_basis_matrix_closed_form():
    want = [[Fraction(int(x)) for x in row] for row in _sections()["two_lines_basis_matrix"]]
    assert colour_two_lines.colour_matrix() == want


def test_two_line_decomposition_closed_form():
    rows = _sections()["two_lines_decomposition"]
    got = colour_two_lines.decomposition()
    assert len(got) == len(rows) == 5
    for d, row in enumerate(rows):
        assert row[0] == f"D{d + 1}"
        assert [tuple(c) for c in got[d]] == [_cfrac(t) for t in row[1:]], row[0]


@pytest.mark.parametrize("n", [2, 3, 4, 5])
def test_colour_matrix_constant_row_sums(n):
    """Relabelling the gluons permutes the orderings and leaves C invariant, so
    every row of C has the same sum (the all-ones vector is an eigenvector);
    for three gluons it is the sum of the six classes, 60/9."""
    C = O.colour_matrix(n).real
    rows = C.sum(1)
    np.testing.assert_allclose(rows, rows[0], rtol=1e-13)
    if n == 3:
        table = _sections()["one_line_three_gluons"]
        assert abs(rows[0] - sum(int(r[1]) for r in table) / 9) < 1e-13
