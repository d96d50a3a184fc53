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
