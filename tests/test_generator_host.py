"""Host logic of the generator (no GPU): diagram and amplitude-term counts.

Independent of the generator's tree enumeration, the counts follow from a
recursion over sets of gluons: an off-shell gluon current of a set S is a
three-gluon vertex joining currents of two disjoint subsets, or a four-gluon
vertex joining three; the top line takes an ordered sequence of currents
whose sets partition all gluons.  The four-gluon vertex has three colour
structures, each its own amplitude term in the colour-flow decomposition.
"""
from functools import lru_cache
from itertools import combinations

import pytest

from paper_2303_18244_gb300.generator import diagrams, emit


def _splits(s, k):
    """Unordered partitions of the frozenset s into k non-empty blocks."""
    items = sorted(s)
    if k == 1:
        yield (s,)
        return
    first, rest = items[0], items[1:]
    # the block holding the smallest element, then the rest split into k - 1
    for r in range(0, len(rest) - k + 2):
        for others in combinations(rest, r):
            block = frozenset((first,) + others)
            remaining = s - block
            if len(remaining) >= k - 1:
                for tail in _splits(remaining, k - 1):
                    yield (block,) + tail


@lru_cache(maxsize=None)
def _currents(s, quartic_weight):
    if len(s) == 1:
        return 1
    tot = 0
    for a, b in _splits(s, 2):
        tot += _currents(a, quartic_weight) * _currents(b, quartic_weight)
    for a, b, c in _splits(s, 3):
        tot += quartic_weight * _currents(a, quartic_weight) * _currents(b, quartic_weight) * _currents(c, quartic_weight)
    return tot


@lru_cache(maxsize=None)
def _line(s, quartic_weight):
    """Ordered sequences of currents along the top line covering s."""
    if not s:
        return 1
    tot = 0
    items = sorted(s)
    for r in range(1, len(items) + 1):
        for first in combinations(items, r):
            f = frozenset(first)
            tot += _currents(f, quartic_weight) * _line(s - f, quartic_weight)
    return tot


@pytest.mark.parametrize("n,want", [(2, 3), (3, 16), (4, 123), (5, 1240)])
def test_diagram_counts(n, want):
    """gg -> t t~ + 0..3 gluons: 3, 16, 123 and 1240 Feynman diagrams."""
    gluons = frozenset(range(n))
    assert _line(gluons, 1) == want
    assert diagrams.count_diagrams(n) == want


@pytest.mark.parametrize("proc,n", [("g g > t t~", 2), ("g g > t t~ g", 3), ("g g > t t~ g g", 4), ("g g > t t~ g g g", 5)])
def test_amplitude_terms_and_header_constants(proc, n):
    """The generated header's NDIAG and NAMP (terms: a four-gluon vertex
    counts three times) equal the recursion's counts."""
    tag, src = emit.emit(proc)
    const = {}
    for line in src.split("\n"):
        if line.startswith("static constexpr int ") and "=" in line:
            name, val = line[len("static constexpr int "):].split("=")[:2]
            const[name.strip()] = val.strip().rstrip(";").split()[0].rstrip(";")
    gluons = frozenset(range(n))
    assert int(const["NDIAG"]) == _line(gluons, 1)
    assert int(const["NAMP"]) == _line(gluons, 3)


# u u~ -> t t~ + gluons: the top line as one leaf "T" of the gluon trees on
# the light line.  The top line carries an ordered sequence of gluon currents
# over its own gluons plus the gluon joining it to the rest, which sits at any
# of the m + 1 places around m attached currents.
def _top(gs, quartic_weight):
    if not gs:
        return 1
    tot = 0
    items = sorted(gs)
    for r in range(1, len(items) + 1):
        for first in combinations(items, r):
            f = frozenset(first)
            rest = gs - f
            # sequences starting with block f; weight (m + 1) summed over the tail
            tot += _currents(f, quartic_weight) * _top_tail(rest, quartic_weight, 1)
    return tot


def _top_tail(gs, quartic_weight, m):
    """sum over ordered sequences of blocks covering gs, after m blocks, of
    (m + blocks + 1) * product of current counts."""
    if not gs:
        return m + 1
    tot = 0
    items = sorted(gs)
    for r in range(1, len(items) + 1):
        for first in combinations(items, r):
            f = frozenset(first)
            tot += _currents(f, quartic_weight) * _top_tail(gs - f, quartic_weight, m + 1)
    return tot


def _two_lines(ngluons, quartic_weight):
    gluons = frozenset(f"g{i}" for i in range(ngluons))
    tot = 0
    for r in range(len(gluons) + 1):
        for gt in combinations(sorted(gluons), r):
            tot += _top(frozenset(gt), quartic_weight) * _line((gluons - frozenset(gt)) | {"T"}, quartic_weight)
    return tot


def test_two_line_diagram_counts():
    """u u~ -> t t~ + 0, 1, 2 gluons: 1, 5 and 36 Feynman diagrams (38 terms
    with the four-gluon vertex split into its colour structures), from the
    recursion above and from the generator's enumeration rooted at the u."""
    from paper_2303_18244_gb300.generator import two_lines
    assert [_two_lines(n, 1) for n in range(3)] == [1, 5, 36]
    assert _two_lines(2, 3) == 38
    assert two_lines.count_feynman_diagrams() == 36 and len(two_lines.diagrams()) == 38
    tag, src = emit.emit("u u~ > t t~ g g")
    assert "static constexpr int NDIAG = 36;" in src and "static constexpr int NAMP = 38;" in src


def test_two_line_colour_flows():
    """The twelve colour flows of u u~ -> t t~ g g are independent, every
    diagram term decomposes onto them exactly (checked inside), and the colour
    matrix has the entries derived by hand from Tr(T^a T^b) = delta/2 and the
    Fierz identity: 16 on the diagonal (N C_F^2 N or (N C_F)^2), -2 between
    the two orders of the gluons on one chain (N C_F (C_F - N/2) N), 16/3
    between the pairings for the same generator string (N C_F^2), 0 between
    a two-gluon chain and a split in the same pairing."""
    from fractions import Fraction

    from paper_2303_18244_gb300.generator import two_lines
    names = [n for n, _ in two_lines.basis()]
    C = two_lines.colour_matrix()
    assert len(two_lines.decomposition()) == 38
    idx = {n: i for i, n in enumerate(names)}
    for i in range(12):
        assert C[i][i] == 16
        for j in range(12):
            assert C[i][j] == C[j][i]
    assert C[idx["ki_jl:ab|1"]][idx["ki_jl:ba|1"]] == -2
    assert C[idx["ki_jl:ab|1"]][idx["ji_kl:ab|1"]] == Fraction(16, 3)
    assert C[idx["ki_jl:ab|1"]][idx["ki_jl:a|b"]] == 0
