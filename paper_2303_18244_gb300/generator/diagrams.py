"""Tree-level Feynman diagrams of g g -> t t~ + (n-2) g and their evaluation plan.

Every tree diagram with one top line and n gluons is the top line from the
outgoing t to the outgoing t~ with k >= 1 quark-gluon vertices, the i-th of
which absorbs a gluon tree T_i over a block B_i of external gluons; the blocks
form an ordered set partition of the gluons.  Gluon trees are built from the
three-gluon vertex and the four-gluon vertex.  Counting them reproduces the
diagram counts 3, 16, 123, 1240 for 2..5 gluons (four-gluon vertices counted
once per diagram).

Colour: the diagram's colour factor is the product, along the line, of the
trees' commutator polynomials (f^{abc} T^c = -i[T^a,T^b] is absorbed into the
Lorentz part); a four-gluon vertex contributes three terms with colour
[[X,Y],Z], [[X,Z],Y], [X,[Y,Z]] and their own Lorentz structures.

Lorentz values (all gluon momenta incoming, P the momentum of a current):
  gluon leaf                 eps (incoming) or eps* (outgoing)
  three-gluon current        (-g/P^2) V3(kX,JX,kY,JY)
      V3 = (JX.JY)(kX-kY) + JY (2kY+kX).JX - JX (2kX+kY).JY
  four-gluon currents        (g^2/P^2)[(JX.JZ)JY - (JY.JZ)JX]   colour [[X,Y],Z]
                             (g^2/P^2)[(JX.JY)JZ - (JY.JZ)JX]   colour [[X,Z],Y]
                            (-g^2/P^2)[(JX.JY)JZ - (JX.JZ)JY]   colour [X,[Y,Z]]
  row current (t side)       Fbar' = (-g/D) Fbar Jslash (Qslash + m),  Q = p_t - K
  column current (t~ side)   F'    = (-g/D) (qslash + m) Jslash F,    q = -p_tbar + K
  amplitude at a top vertex  (i g) Fbar Jslash F
  amplitude at the top node of a single tree (k = 1), with
      G = (i g / P^2) ubar gamma v:   -g V3(X,Y).G   or   +-g^2 L_branch(X,Y,Z).G
with D = P^2 - m^2 + i m Gamma on every top propagator.

The plan picks, per diagram term, where the amplitude is evaluated (which top
vertex, or the tree's top node), greedily minimising the number of distinct
off-shell currents, which are shared between diagrams.
"""
from __future__ import annotations

from functools import lru_cache

from .colour import poly_comm, poly_leaf, poly_mul, words


# ---------------------------------------------------------------------------
# gluon trees over a subset (bitmask) of gluons
#   leaf: ("L", i)
#   three-gluon node: ("3", X, Y)          X, Y canonically ordered
#   four-gluon node:  ("4", X, Y, Z, br)   br in {0,1,2}
# ---------------------------------------------------------------------------

def _bits(mask: int) -> list[int]:
    return [i for i in range(mask.bit_length()) if mask >> i & 1]


def tree_mask(t) -> int:
    if t[0] == "L":
        return 1 << t[1]
    m = 0
    for c in t[1:4] if t[0] == "4" else t[1:3]:
        m |= tree_mask(c)
    return m


def _low(mask: int) -> int:
    return mask & (-mask)


@lru_cache(maxsize=None)
def trees(mask: int, branches: bool = True) -> tuple:
    """All gluon trees over the gluons in mask.  With branches=False four-gluon
    nodes are not split into their three colour terms (diagram counting)."""
    b = _bits(mask)
    if len(b) == 1:
        return (("L", b[0]),)
    out = []
    low = _low(mask)
    # three-gluon vertex: unordered {A, B}, A holds the lowest gluon
    sub = (mask - 1) & mask
    while sub:
        if sub & low:
            A, B = sub, mask ^ sub
            for ta in trees(A, branches):
                for tb in trees(B, branches):
                    out.append(("3", ta, tb))
        sub = (sub - 1) & mask
    # four-gluon vertex: unordered {A, B, C} ordered by lowest member
    sub = (mask - 1) & mask
    while sub:
        if sub & low:
            A = sub
            R = mask ^ A
            low2 = _low(R) if R else 0
            s2 = (R - 1) & R if R else 0
            while s2:
                if s2 & low2:
                    B, C = s2, R ^ s2
                    if C:
                        for ta in trees(A, branches):
                            for tb in trees(B, branches):
                                for tc in trees(C, branches):
                                    if branches:
                                        for br in range(3):
                                            out.append(("4", ta, tb, tc, br))
                                    else:
                                        out.append(("4", ta, tb, tc, -1))
                s2 = (s2 - 1) & R
        sub = (sub - 1) & mask
    return tuple(out)


def tree_poly(t) -> dict:
    """Colour polynomial of a tree (nested commutators of generators)."""
    if t[0] == "L":
        return poly_leaf(t[1])
    if t[0] == "3":
        return poly_comm(tree_poly(t[1]), tree_poly(t[2]))
    X, Y, Z, br = tree_poly(t[1]), tree_poly(t[2]), tree_poly(t[3]), t[4]
    if br == 0:
        return poly_comm(poly_comm(X, Y), Z)
    if br == 1:
        return poly_comm(poly_comm(X, Z), Y)
    return poly_comm(X, poly_comm(Y, Z))


def ordered_partitions(mask: int):
    """Ordered set partitions (B_1, ..., B_k) of the gluons in mask."""
    if mask == 0:
        yield ()
        return
    sub = mask
    while sub:
        for rest in ordered_partitions(mask ^ sub):
            yield (sub,) + rest
        sub = (sub - 1) & mask


def count_diagrams(n: int) -> int:
    full = (1 << n) - 1
    tot = 0
    for part in ordered_partitions(full):
        c = 1
        for B in part:
            c *= len(trees(B, False))
        tot += c
    return tot


def diagram_terms(n: int):
    """All amplitude terms: tuples of trees along the top line (t side first)."""
    full = (1 << n) - 1
    for part in ordered_partitions(full):
        def rec(i):
            if i == len(part):
                yield ()
                return
            for t in trees(part[i]):
                for rest in rec(i + 1):
                    yield (t,) + rest
        yield from rec(0)


def term_colour(blocks) -> dict:
    p = {(): 1}
    for t in blocks:
        p = poly_mul(p, tree_poly(t))
    return p


# ---------------------------------------------------------------------------
# evaluation plan
# ---------------------------------------------------------------------------

class Plan:
    """Ops in dependency order.

    currents: dict key -> (id, op) where op is one of
        ("ext", i)                         external gluon i
        ("3", idX, idY, mask)              three-gluon current
        ("4", idX, idY, idZ, br, mask)     four-gluon current (branch br)
        ("row", idPrev, idG, mask)         row top current, mask = gluons absorbed from t
        ("col", idG, idNext, mask)         column top current, mask = gluons absorbed from t~
        ("ubar",) / ("v",)                 external top / antitop spinors
        ("gtt",)                           G = (i g / P^2) ubar gamma v
    amps: list of (op, jamp_coeffs) with op one of
        ("f", idRow, idG, idCol)           (i g) Fbar Jslash F
        ("a3", idX, idY)                   -g V3(X,Y).G
        ("a4", idX, idY, idZ, br)          +-g^2 L_br(X,Y,Z).G
    """

    def __init__(self, n: int):
        self.n = n
        self.keys: dict = {}
        self.ops: list = []
        self.amps: list = []
        self.words = words(n)
        self.word_index = {w: i for i, w in enumerate(self.words)}

    def _add(self, key, op):
        if key in self.keys:
            return self.keys[key]
        i = len(self.ops)
        self.keys[key] = i
        self.ops.append(op)
        return i

    # current builders (keys are structural, so identical subtrees are shared)
    def gluon(self, t):
        key = ("g", t)
        if key in self.keys:
            return self.keys[key]
        if t[0] == "L":
            return self._add(key, ("ext", t[1]))
        if t[0] == "3":
            x, y = self.gluon(t[1]), self.gluon(t[2])
            return self._add(key, ("3", x, y, tree_mask(t)))
        x, y, z = self.gluon(t[1]), self.gluon(t[2]), self.gluon(t[3])
        return self._add(key, ("4", x, y, z, t[4], tree_mask(t)))

    def row(self, blocks):
        key = ("row", blocks)
        if key in self.keys:
            return self.keys[key]
        if not blocks:
            return self._add(key, ("ubar",))
        prev = self.row(blocks[:-1])
        g = self.gluon(blocks[-1])
        m = 0
        for t in blocks:
            m |= tree_mask(t)
        return self._add(key, ("row", prev, g, m))

    def col(self, blocks):
        key = ("col", blocks)
        if key in self.keys:
            return self.keys[key]
        if not blocks:
            return self._add(key, ("v",))
        nxt = self.col(blocks[1:])
        g = self.gluon(blocks[0])
        m = 0
        for t in blocks:
            m |= tree_mask(t)
        return self._add(key, ("col", g, nxt, m))

    # cost of a choice = number of currents not yet present
    def _missing_gluon(self, t, acc):
        key = ("g", t)
        if key in self.keys or key in acc:
            return
        acc.add(key)
        if t[0] == "3":
            self._missing_gluon(t[1], acc)
            self._missing_gluon(t[2], acc)
        elif t[0] == "4":
            for c in t[1:4]:
                self._missing_gluon(c, acc)

    def _missing_row(self, blocks, acc):
        key = ("row", blocks)
        if key in self.keys or key in acc:
            return
        acc.add(key)
        if blocks:
            self._missing_row(blocks[:-1], acc)
            self._missing_gluon(blocks[-1], acc)

    def _missing_col(self, blocks, acc):
        key = ("col", blocks)
        if key in self.keys or key in acc:
            return
        acc.add(key)
        if blocks:
            self._missing_col(blocks[1:], acc)
            self._missing_gluon(blocks[0], acc)

    def add_term(self, blocks):
        colour = term_colour(blocks)
        coeffs = {self.word_index[w]: c for w, c in colour.items()}
        k = len(blocks)
        if k == 1:
            t = blocks[0]
            self._add(("gtt",), ("gtt",)) if ("gtt",) not in self.keys else None
            if t[0] == "3":
                x, y = self.gluon(t[1]), self.gluon(t[2])
                self.amps.append((("a3", x, y), coeffs))
            else:
                x, y, z = self.gluon(t[1]), self.gluon(t[2]), self.gluon(t[3])
                self.amps.append((("a4", x, y, z, t[4]), coeffs))
            return
        sizes = [bin(tree_mask(t)).count("1") for t in blocks]
        best = None
        for j in range(k):
            acc = set()
            self._missing_row(blocks[:j], acc)
            self._missing_col(blocks[j + 1:], acc)
            self._missing_gluon(blocks[j], acc)
            # fewest new currents; ties go to the vertex that best balances the
            # gluons on the two sides (meet in the middle)
            cost = (len(acc), abs(sum(sizes[:j]) - sum(sizes[j + 1:])))
            if best is None or cost < best[0]:
                best = (cost, j)
        j = best[1]
        r = self.row(blocks[:j])
        c = self.col(blocks[j + 1:])
        g = self.gluon(blocks[j])
        self.amps.append((("f", r, g, c), coeffs))


def build_plan(n: int) -> Plan:
    p = Plan(n)
    # make sure ubar, v, gtt, externals come first
    p.row(())
    p.col(())
    for i in range(n):
        p.gluon(("L", i))
    terms = list(diagram_terms(n))
    # process many-block terms first (they fix the row/column currents), then
    # single-tree terms
    terms.sort(key=lambda b: -len(b))
    for b in terms:
        p.add_term(b)
    return p


def plan_stats(p: Plan) -> dict:
    kinds: dict = {}
    for op in p.ops:
        kinds[op[0]] = kinds.get(op[0], 0) + 1
    akinds: dict = {}
    nco = 0
    for op, co in p.amps:
        akinds[op[0]] = akinds.get(op[0], 0) + 1
        nco += len(co)
    return {"currents": kinds, "amps": akinds, "n_amps": len(p.amps), "jamp_updates": nco}
