"""Exact SU(3) colour algebra for one quark line plus n gluons.

Colour basis: the strings W(sigma) = (T^{a_sigma1} ... T^{a_sigman})_{i j} over
orderings sigma of the gluons, T^a the fundamental generators with
Tr(T^a T^b) = delta^{ab}/2.  Each Feynman diagram's colour factor is a nested
commutator polynomial in the T's (f^{abc} T^c = -i [T^a, T^b] absorbs every
structure constant), which expands exactly onto these strings with integer
coefficients.

Colour matrix C(sigma, tau) = sum_{a} Tr(W(sigma) W(tau)^dagger), evaluated
symbolically with exact rationals by the Fierz identity
    sum_a (T^a)_{ij} (T^a)_{kl} = 1/2 (delta_il delta_kj - 1/N delta_ij delta_kl),
i.e. Tr(X T^a Y T^a) = 1/2 [Tr X Tr Y - 1/N Tr(XY)] and
Tr(X T^a) Tr(Y T^a) = 1/2 [Tr(XY) - 1/N Tr X Tr Y], with Tr(1) = N = 3.
(The paper's "colour algebra" step, Sect. 3.)
"""
from __future__ import annotations

from fractions import Fraction
from functools import lru_cache
from itertools import permutations

NC = 3


def words(n: int) -> list[tuple[int, ...]]:
    """All orderings of gluons 0..n-1, lexicographic; index = colour-flow index."""
    return list(permutations(range(n)))


# ---------------------------------------------------------------------------
# commutator polynomials: dict word -> int
# ---------------------------------------------------------------------------

def poly_leaf(i: int) -> dict:
    return {(i,): 1}


def poly_mul(a: dict, b: dict) -> dict:
    out: dict = {}
    for wa, ca in a.items():
        for wb, cb in b.items():
            w = wa + wb
            out[w] = out.get(w, 0) + ca * cb
    return {w: c for w, c in out.items() if c != 0}


def poly_add(a: dict, b: dict, sb: int = 1) -> dict:
    out = dict(a)
    for w, c in b.items():
        out[w] = out.get(w, 0) + sb * c
    return {w: c for w, c in out.items() if c != 0}


def poly_comm(a: dict, b: dict) -> dict:
    return poly_add(poly_mul(a, b), poly_mul(b, a), -1)


# ---------------------------------------------------------------------------
# traces with every adjoint label appearing twice, reduced by Fierz
# ---------------------------------------------------------------------------

def _canon_trace(t: tuple) -> tuple:
    """Cyclic canonical form of one trace (labels are already relabelled)."""
    if not t:
        return t
    return min(t[i:] + t[:i] for i in range(len(t)))


def _relabel(traces: tuple) -> tuple:
    """Canonical form of a product of traces under relabelling of the dummy
    labels and cyclicity of each trace (used only as a memo key; the value of
    the product does not depend on dummy-label names)."""
    best = None
    # traces are short; try each rotation per trace and sort, relabel by first use
    def relabel_seq(seq_list):
        m = {}
        out = []
        for t in seq_list:
            o = []
            for x in t:
                if x not in m:
                    m[x] = len(m)
                o.append(m[x])
            out.append(tuple(o))
        return tuple(out)

    ts = [t for t in traces]
    # sort traces by length then content after independent canonicalisation
    cand = []
    for t in ts:
        cand.append(_canon_trace(t))
    order = sorted(range(len(cand)), key=lambda i: (len(cand[i]), cand[i]))
    seq = [cand[i] for i in order]
    best = relabel_seq(seq)
    return best


@lru_cache(maxsize=None)
def _trace_product(traces: tuple) -> Fraction:
    """Value of prod_k Tr(T^{l_k1} T^{l_k2} ...) summed over all labels, each
    label appearing exactly twice across the product."""
    # remove empty traces: Tr(1) = N
    val = Fraction(1)
    ts = []
    for t in traces:
        if len(t) == 0:
            val *= NC
        elif len(t) == 1:
            return Fraction(0)  # Tr T^a = 0
        else:
            ts.append(t)
    if not ts:
        return val
    key = _relabel(tuple(ts))
    if key != tuple(ts):
        return val * _trace_product(key)
    # pick the first label of the first trace
    t0 = ts[0]
    lab = t0[0]
    rest = ts[1:]
    # other occurrence in the same trace?
    if lab in t0[1:]:
        j = t0.index(lab, 1)
        B = t0[1:j]
        C = t0[j + 1:]
        # Tr(T^a B T^a C) = 1/2 [Tr(B) Tr(C) - 1/N Tr(B C)]
        r = Fraction(1, 2) * _trace_product(tuple([B, C] + rest)) \
            - Fraction(1, 2 * NC) * _trace_product(tuple([B + C] + rest))
        return val * r
    for k, t1 in enumerate(rest):
        if lab in t1:
            j = t1.index(lab)
            B = t0[1:]
            D = t1[j + 1:] + t1[:j]
            others = rest[:k] + rest[k + 1:]
            # Tr(T^a B) Tr(T^a D) = 1/2 [Tr(B D) - 1/N Tr(B) Tr(D)]
            r = Fraction(1, 2) * _trace_product(tuple([B + D] + list(others))) \
                - Fraction(1, 2 * NC) * _trace_product(tuple([B, D] + list(others)))
            return val * r
    raise ValueError("label appears once")


def colour_matrix_exact(n: int) -> list[list[Fraction]]:
    """C(sigma, tau) = sum_a Tr(T^{sigma1}..T^{sigman} T^{taun}..T^{tau1}), exact."""
    ws = words(n)
    N = len(ws)
    C = [[Fraction(0)] * N for _ in range(N)]
    for i, s in enumerate(ws):
        for j in range(i, N):
            t = ws[j]
            tr = tuple(s) + tuple(reversed(t))
            v = _trace_product((tr,))
            C[i][j] = v
            C[j][i] = v
    return C


def common_denominator(C) -> tuple[int, list[list[int]]]:
    """(d, K) with C = K / d, K integer."""
    from math import lcm
    d = 1
    for row in C:
        for x in row:
            d = lcm(d, x.denominator)
    K = [[int(x * d) for x in row] for row in C]
    return d, K
