"""Tree diagrams, colour algebra and straight-line code of u u~ -> t t~ g g.

Two quark lines (the light line from the incoming u to the incoming u~, the
top line from the outgoing t to the outgoing t~) and two outgoing gluons.
Legs: 0 u (colour i), 1 u~ (j), 2 t (k), 3 t~ (l), 4 and 5 gluons (a, b).

Diagrams.  Every tree diagram is reached once from the u leg: the vertex at
u joins an off-shell light row (the line from u~ with gluon trees attached)
and an off-shell gluon, and each off-shell object is one of

  ("ext", leg)              an external state
  ("g3", X, Y)              three-gluon vertex of two gluon objects
  ("g4", X, Y, Z, br)       four-gluon vertex, one of its three colour terms
  ("close", R, C)           the top line closed into a gluon: top row R
                            (holds t), top column C (holds t~)
  ("row", R, G)             a row (light or top) with gluon object G attached
  ("col", C, G)             the top column with gluon object G attached

over a subset of the legs 1..5.  A gluon object holds no u~ and either both
or neither of t, t~; a light row holds u~; a top row holds t but not t~; a
top column holds t~ but not t.

Feynman rules (vertex i g gamma^mu T^a, three-gluon g f^{abc} V3, four-gluon
-i g^2 f f (...), gluon propagator -i g_{mu nu}/P^2, quark propagator
i (Qslash + m)/(Q^2 - m^2 + i m Gamma), Gamma on the top only), each object
split into a colour tensor and a Lorentz value:

  g3       colour -i f^{a b c}              value (g/P^2) V3(kX, JX, kY, JY)
  g4, br   colour f^{a b e} f^{d c e}, ...  value (-g^2/P^2) L_br(X, Y, Z)
  close    colour T^c_{m n}                 value (g/P^2) Rbar gamma^mu C
  row      colour T^c_{m n} (m: old end)    value (-g/D) Rbar Jslash (Qslash + m)
  col      colour T^c_{m n} (n: old end)    value (-g/D) (Qslash + m) Jslash C
  root     colour T^c_{m i}                 value  i g  Rbar Jslash u(p1)

with Q the momentum along the fermion flow: p3 - K (top row), -p2 - K (light
row), -p4 + K (top column), K the incoming momentum of the attached legs.
The colour tensor of each diagram is evaluated by explicit index sums over
the Gell-Mann generators and decomposed exactly onto twelve colour flows:
the two pairings of the quark indices into chains, (k i)(j l) and (j i)(k l),
with the gluons' generators distributed in order over the two chains.
"""
from __future__ import annotations

from fractions import Fraction
from functools import lru_cache

import numpy as np

from .colour_two_lines import gell_mann_generators

NG = 2
NLEG = 4 + NG                 # legs 0..5
LEG_LETTER = {1: "j", 2: "k", 3: "l", 4: "a", 5: "b"}
LEG_DIM = {1: 3, 2: 3, 3: 3, 4: 8, 5: 8}


def _bit(leg: int) -> int:
    return 1 << (leg - 1)


def legs_of(mask: int) -> list[int]:
    return [leg for leg in range(1, NLEG) if mask & _bit(leg)]


def kind(mask: int) -> str | None:
    """"g" gluon object, "lrow" light row, "trow" top row, "tcol" top column."""
    h1, h2, h3 = bool(mask & _bit(1)), bool(mask & _bit(2)), bool(mask & _bit(3))
    if not h1 and h2 == h3:
        return "g"
    if h1 and h2 == h3:
        return "lrow"
    if h2 and not h3 and not h1:
        return "trow"
    if h3 and not h2 and not h1:
        return "tcol"
    return None


def node_mask(n) -> int:
    if n[0] == "ext":
        return _bit(n[1])
    if n[0] == "g4":
        return node_mask(n[1]) | node_mask(n[2]) | node_mask(n[3])
    return node_mask(n[1]) | node_mask(n[2])


def _splits(mask: int):
    sub = (mask - 1) & mask
    while sub:
        yield sub, mask ^ sub
        sub = (sub - 1) & mask


@lru_cache(maxsize=None)
def objects(mask: int) -> tuple:
    """Every off-shell object over the legs in mask (see the module docstring)."""
    k = kind(mask)
    legs = legs_of(mask)
    if k is None or not legs:
        return ()
    if len(legs) == 1:
        return (("ext", legs[0]),)
    out = []
    low = mask & (-mask)
    if k == "g":
        for A, B in _splits(mask):
            if A & low and kind(A) == "g" and kind(B) == "g":
                out += [("g3", x, y) for x in objects(A) for y in objects(B)]
        for A, R in _splits(mask):
            if not (A & low) or kind(A) != "g":
                continue
            low2 = R & (-R)
            for B, C in _splits(R):
                if B & low2 and kind(B) == "g" and kind(C) == "g":
                    out += [("g4", x, y, z, br) for x in objects(A) for y in objects(B) for z in objects(C)
                            for br in range(3)]
        for A, B in _splits(mask):
            if kind(A) == "trow" and kind(B) == "tcol":
                out += [("close", r, c) for r in objects(A) for c in objects(B)]
    else:
        end = {"lrow": 1, "trow": 2, "tcol": 3}[k]
        tag = "col" if k == "tcol" else "row"
        for A, B in _splits(mask):
            if A & _bit(end) and kind(A) == k and kind(B) == "g":
                out += [(tag, x, y) for x in objects(A) for y in objects(B)]
    return tuple(out)


def diagrams() -> list:
    """(light row, gluon object) pairs at the u vertex: one per diagram term
    (a four-gluon vertex contributes its three colour terms)."""
    full = (1 << (NLEG - 1)) - 1
    out = []
    for A, B in _splits(full):
        if A & _bit(1) and kind(A) == "lrow" and kind(B) == "g":
            out += [(r, gl) for r in objects(A) for gl in objects(B)]
    return out


def count_feynman_diagrams() -> int:
    """Diagrams with each four-gluon vertex counted once."""
    def merged(n):
        if n[0] == "g4":
            return n[4] == 0 and all(merged(c) for c in n[1:4])
        if n[0] == "ext":
            return True
        return merged(n[1]) and merged(n[2])
    return sum(1 for r, g in diagrams() if merged(r) and merged(g))


# ---------------------------------------------------------------------------
# colour
# ---------------------------------------------------------------------------

@lru_cache(maxsize=1)
def _su3():
    T = gell_mann_generators()
    comm = np.einsum("aij,bjk->abik", T, T) - np.einsum("bij,ajk->abik", T, T)
    f = np.real(-2j * np.einsum("abij,cji->abc", comm, T))
    return T, f


def colour_tensor(n):
    """(array, legs): axes [own colour] + one per leg of the object, in leg order."""
    T, f = _su3()
    if n[0] == "ext":
        leg = n[1]
        return np.eye(LEG_DIM[leg], dtype=complex), [leg]
    parts = [colour_tensor(c) for c in (n[1:4] if n[0] == "g4" else n[1:3])]
    legs = sorted(sum((p[1] for p in parts), []))
    out_letters = "".join(LEG_LETTER[x] for x in legs)

    def sub(p, own):
        return own + "".join(LEG_LETTER[x] for x in p[1])
    if n[0] == "g3":
        (X, _), (Y, _) = parts
        t = np.einsum(f"xyz,{sub(parts[0], 'x')},{sub(parts[1], 'y')}->z{out_letters}", -1j * f, X, Y)
    elif n[0] == "g4":
        br = n[4]
        ff = [np.einsum("xye,wze->xywz", f, f),   # f^{a b e} f^{d c e}: (a, b, d, c) = (x, y, w, z)
              np.einsum("xwe,yze->xywz", f, f),   # f^{a d e} f^{b c e}
              np.einsum("xze,ywe->xywz", f, f)][br]  # f^{a c e} f^{b d e}
        X, Y, Z = (p[0] for p in parts)
        t = np.einsum(f"xywz,{sub(parts[0], 'x')},{sub(parts[1], 'y')},{sub(parts[2], 'w')}->z{out_letters}",
                      ff, X, Y, Z)
    elif n[0] == "close":
        (R, _), (C, _) = parts
        t = np.einsum(f"zmn,{sub(parts[0], 'm')},{sub(parts[1], 'n')}->z{out_letters}", T, R, C)
    elif n[0] == "row":
        (R, _), (G, _) = parts
        t = np.einsum(f"cmn,{sub(parts[0], 'm')},{sub(parts[1], 'c')}->n{out_letters}", T, R, G)
    else:  # col
        (C, _), (G, _) = parts
        t = np.einsum(f"cmn,{sub(parts[0], 'n')},{sub(parts[1], 'c')}->m{out_letters}", T, C, G)
    return t, legs


def diagram_colour(d) -> np.ndarray:
    """Colour tensor [i][j][k][l][a][b] of a diagram (row, gluon object)."""
    T, _ = _su3()
    (R, rl), (G, gl) = colour_tensor(d[0]), colour_tensor(d[1])
    legs = sorted(rl + gl)
    assert legs == [1, 2, 3, 4, 5]
    r = "".join(LEG_LETTER[x] for x in rl)
    g = "".join(LEG_LETTER[x] for x in gl)
    return np.einsum(f"cmi,m{r},c{g}->ijklab", T, R, G)


def basis() -> list[tuple[str, np.ndarray]]:
    """The twelve colour flows: (name, tensor [i][j][k][l][a][b])."""
    T, _ = _su3()

    def chain(seq):
        m = np.eye(3, dtype=complex)[None, None]  # [a][b][row][col]
        m = np.broadcast_to(m, (8, 8, 3, 3)).copy()
        for g in seq:
            if g == "a":
                m = np.einsum("abrs,ast->abrt", m, T)
            else:
                m = np.einsum("abrs,bst->abrt", m, T)
        return m
    splits = [("ab", ""), ("ba", ""), ("", "ab"), ("", "ba"), ("a", "b"), ("b", "a")]
    out = []
    for pairing in ("ki_jl", "ji_kl"):
        for s1, s2 in splits:
            c1, c2 = chain(s1), chain(s2)
            if pairing == "ki_jl":   # (..)_{k i} (..)_{j l}
                t = np.einsum("abki,abjl->ijklab", c1, c2)
            else:                    # (..)_{j i} (..)_{k l}
                t = np.einsum("abji,abkl->ijklab", c1, c2)
            out.append((f"{pairing}:{s1 or '1'}|{s2 or '1'}", t))
    return out


def _rational(x: complex, den: int = 216) -> tuple[Fraction, Fraction]:
    re, im = Fraction(round(x.real * den), den), Fraction(round(x.imag * den), den)
    assert abs(float(re) - x.real) < 1e-12 and abs(float(im) - x.imag) < 1e-12, x
    return re, im


@lru_cache(maxsize=1)
def decomposition():
    """coef[d][m] (re, im) with colour(d) = sum_m coef[d][m] flow_m, exact."""
    B = np.stack([b.ravel() for _, b in basis()], axis=1)
    assert np.linalg.matrix_rank(B) == B.shape[1], "the twelve flows are independent"
    out = []
    for d in diagrams():
        D = diagram_colour(d).ravel()
        x, *_ = np.linalg.lstsq(B, D, rcond=None)
        assert np.abs(B @ x - D).max() < 1e-12
        out.append([_rational(v) for v in x])
    return out


@lru_cache(maxsize=1)
def colour_matrix() -> list[list[Fraction]]:
    """C_mn = sum over all colour indices of conj(flow_m) flow_n (real, exact)."""
    bs = [b for _, b in basis()]
    C = []
    for bm in bs:
        row = []
        for bn in bs:
            re, im = _rational(np.sum(np.conj(bm) * bn))
            assert im == 0
            row.append(re)
        C.append(row)
    return C


# ---------------------------------------------------------------------------
# code
# ---------------------------------------------------------------------------

def emit_uuttgg(tag: str) -> str:
    """Header of u u~ -> t t~ g g (struct mg::<tag>), the interface of the
    other generated processes: prepare (FP64 per-event set-up into the
    slab), amplitudes (per helicity, every object once, each diagram term's
    value added to its colour flows) and colour_quadratic."""
    from .colour import common_denominator
    from .emit import _colour_quadratic, _fmt_knum
    dec = decomposition()
    C = colour_matrix()
    cden, K = common_denominator(C)
    diags = diagrams()
    ncol = len(C)
    npar = NLEG

    # objects in dependency order, each once
    order, seen = [], set()

    def visit(n):
        if n in seen:
            return
        for c in (n[1:4] if n[0] == "g4" else n[1:3]) if n[0] != "ext" else ():
            visit(c)
        seen.add(n)
        order.append(n)
    for r, g in diags:
        visit(r)
        visit(g)

    # slab: fermion ingredients 0-19, gluon bases 20-31, then per gluon
    # subset its incoming momentum and g/P^2, -g^2/P^2, per quark object
    # subset its propagator momentum and -g/D
    slot = 32
    kslot, cslot, qslot = {}, {}, {}
    for n in order:
        m = node_mask(n)
        k = kind(m)
        if k == "g":
            if m not in kslot:
                kslot[m] = slot
                slot += 4
            if n[0] != "ext" and m not in cslot:
                cslot[m] = slot
                slot += 2
        elif n[0] != "ext" and m not in qslot:
            qslot[m] = slot
            slot += 6
    nslot = slot

    def leg_mom(leg):  # incoming momentum of a leg, as (pointer, sign)
        return (f"pd + {4 * leg}", 1 if leg in (0, 1) else -1)

    L = [f"// generated by paper_2303_18244_gb300.generator for 'u u~ > t t~ g g'",
         "#pragma once", '#include "mg_vertices.cuh"', "namespace mg {", f"struct {tag} {{",
         f"static constexpr int NPAR = {npar};", f"static constexpr int NHEL = {1 << npar};",
         f"static constexpr int NCOL = {ncol};", f"static constexpr int NDIAG = {count_feynman_diagrams()};",
         f"static constexpr int NAMP = {len(diags)};", f"static constexpr int NSLOT = {nslot};",
         f"static constexpr int NSLOT_LEAN = {nslot};", "static constexpr bool LEAN_SLAB = false;",
         "static constexpr double IDEN = 72.0;", f"static constexpr int CDEN = {cden};",
         f"static constexpr int KNUM[NCOL * NCOL] = {{{_fmt_knum(K)}}};"]
    L += ["// per-event set-up (FP64): spinor ingredients, gluon bases, the momenta of the",
          "// gluon objects and quark propagators, and their coefficients",
          "template <typename R>",
          "__device__ static __forceinline__ void prepare(const double* __restrict__ p, const double* __restrict__ kp,",
          "                                        R* __restrict__ ev, const int es) {",
          "#define EV(k) ev[(k) * es]",
          "  const double g = kp[0], mt = kp[1], wt = kp[2];",
          "  for (int i = 0; i < 4; i++) {",
          "    double f[5]; fermion_ingredients(p + 4 * i, i < 2 ? 0.0 : mt, f);",
          "    for (int j = 0; j < 5; j++) EV(5 * i + j) = R(f[j]);",
          "  }"]
    for gi in range(NG):
        L.append(f"  {{ double b[6]; vector_basis(p + {4 * (4 + gi)}, b); "
                 f"for (int j = 0; j < 6; j++) EV({20 + 6 * gi} + j) = R(b[j]); }}")
    for m, s in sorted(kslot.items(), key=lambda kv: kv[1]):
        for mu in range(4):
            expr = " ".join(f"{'+' if leg in (0, 1) else '-'} p[{4 * leg + mu}]" for leg in legs_of(m))
            L.append(f"  EV({s + mu}) = R({expr.lstrip('+ ')});")
    for m, s in sorted(cslot.items(), key=lambda kv: kv[1]):
        terms = [leg_mom(leg) for leg in legs_of(m)]
        vv = ", ".join(t[0] for t in terms)
        ss = ", ".join("double(1)" if t[1] > 0 else "double(-1)" for t in terms)
        L.append(f"  {{ const double* const vv[{len(terms)}] = {{{vv}}}; const double ss[{len(terms)}] = {{{ss}}};")
        L.append(f"    const double p2 = inv_mass2<R>(vv, ss, 0.0);")
        L.append(f"    EV({s}) = R(g / p2); EV({s + 1}) = R(-g * g / p2); }}")
    for m, s in sorted(qslot.items(), key=lambda kv: kv[1]):
        k = kind(m)
        # momentum along the fermion flow as a signed sum of leg momenta
        if k == "trow":
            terms = [("pd + 8", 1)] + [(leg_mom(x)[0], -leg_mom(x)[1]) for x in legs_of(m) if x != 2]
        elif k == "lrow":
            terms = [("pd + 4", -1)] + [(leg_mom(x)[0], -leg_mom(x)[1]) for x in legs_of(m) if x != 1]
        else:  # tcol
            terms = [("pd + 12", -1)] + [leg_mom(x) for x in legs_of(m) if x != 3]
        for mu in range(4):
            expr = " ".join(f"{'+' if sg > 0 else '-'} p[{int(ptr.split('+ ')[1]) + mu}]" for ptr, sg in terms)
            L.append(f"  EV({s + mu}) = R({expr.lstrip('+ ')});")
        vv = ", ".join(t[0] for t in terms)
        ss = ", ".join("double(1)" if t[1] > 0 else "double(-1)" for t in terms)
        top = k != "lrow"
        L.append(f"  {{ const double* const vv[{len(terms)}] = {{{vv}}}; const double ss[{len(terms)}] = {{{ss}}};")
        L.append(f"    const double dre = inv_mass2<R>(vv, ss, {'mt * mt' if top else '0.0'});"
                 f" const double dim = {'mt * wt' if top else '0.0'};")
        L.append("    const double r = -g / (dre * dre + dim * dim);")
        L.append(f"    EV({s + 4}) = R(r * dre); EV({s + 5}) = R(-r * dim); }}")
    L += ["#undef EV", "}"]

    # amplitudes
    L += ["template <typename R>",
          "__device__ static __forceinline__ void amplitudes(const R* __restrict__ ev, const int es, const int hel,",
          "                                           const double* __restrict__ kp, cx<R>* __restrict__ jamp,",
          "                                           const int js) {",
          "#define EV(k) ev[(k) * es]",
          "#define ING(i) FermIngr<R>{EV(5 * (i)), EV(5 * (i) + 1), EV(5 * (i) + 2), EV(5 * (i) + 3), EV(5 * (i) + 4)}",
          "#define MOM(k) M4<R>{{EV(k), EV((k) + 1), EV((k) + 2), EV((k) + 3)}}",
          "  const R g = R(kp[0]), mt = R(kp[1]);"]
    for i in range(npar):
        L.append(f"  const int l{i} = ((hel >> {npar - 1 - i}) & 1) ? 1 : -1;")
    L += ["  const Sp<R> w0 = ext_u<R>(ING(0), l0);"]
    names = {}
    for n in order:
        nm = f"o{len(names)}"
        names[n] = nm
        if n[0] == "ext":
            leg = n[1]
            if leg == 1:
                L.append(f"  const Sp<R> {nm} = ext_vbar<R>(ING(1), l1);")
            elif leg == 2:
                L.append(f"  const Sp<R> {nm} = ext_ubar<R>(ING(2), l2);")
            elif leg == 3:
                L.append(f"  const Sp<R> {nm} = ext_v<R>(ING(3), l3);")
            else:
                b0 = 20 + 6 * (leg - 4)
                L.append(f"  V4<R> {nm};")
                L.append(f"  {{ const R e1[3] = {{EV({b0}), EV({b0 + 1}), EV({b0 + 2})}}, "
                         f"e2[3] = {{EV({b0 + 3}), EV({b0 + 4}), EV({b0 + 5})}};")
                L.append(f"    {nm} = ext_vector<R>(e1, e2, R(l{leg}), true); }}")
            continue
        m = node_mask(n)
        if n[0] == "g3":
            x, y = n[1], n[2]
            L.append(f"  const V4<R> {nm} = vvv_cur<R>(MOM({kslot[node_mask(x)]}), {names[x]}, "
                     f"MOM({kslot[node_mask(y)]}), {names[y]}, EV({cslot[m]}));")
        elif n[0] == "g4":
            x, y, z, br = n[1:5]
            L.append(f"  const V4<R> {nm} = vvvv_cur<{br}, R>({names[x]}, {names[y]}, {names[z]}, "
                     f"EV({cslot[m] + 1}));")
        elif n[0] == "close":
            L.append(f"  const V4<R> {nm} = ffv_vcur<R>({names[n[1]]}, {names[n[2]]}, cx<R>{{EV({cslot[m]}), R(0)}});")
        elif n[0] == "row":
            mass = "R(0)" if kind(m) == "lrow" else "mt"
            s = qslot[m]
            L.append(f"  const Sp<R> {nm} = ffv_row<R>({names[n[1]]}, {names[n[2]]}, MOM({s}), {mass}, "
                     f"cx<R>{{EV({s + 4}), EV({s + 5})}});")
        else:  # col
            s = qslot[m]
            L.append(f"  const Sp<R> {nm} = ffv_col<R>({names[n[2]]}, {names[n[1]]}, MOM({s}), mt, "
                     f"cx<R>{{EV({s + 4}), EV({s + 5})}});")
    # diagram terms: i g Rbar Jslash u(p1), accumulated into the flows
    L.append(f"  cx<R> A[{len(diags)}];")
    for di, (r, gl) in enumerate(diags):
        L.append(f"  A[{di}] = ffv_amp<R>({names[r]}, {names[gl]}, w0);")
    for k in range(ncol):
        terms = []
        for di in range(len(diags)):
            re, im = dec[di][k]
            if re == 0 and im == 0:
                continue
            # times i (the vertex at u): (re + i im) i = -im + i re
            terms.append(f"cx<R>{{R({float(-im)!r}), R({float(re)!r})}} * A[{di}]")
        rhs = " + ".join(terms) if terms else "cx<R>{R(0), R(0)}"
        L.append(f"  jamp[{k} * js] = g * ({rhs});")
    L += ["#undef MOM", "#undef ING", "#undef EV", "}",
          "// sum_ij KNUM_ij (Re J_i Re J_j + Im J_i Im J_j); |M|^2 colour sum = result / CDEN",
          "template <typename R>",
          "__device__ static __forceinline__ R colour_quadratic(const cx<R>* __restrict__ jamp, const int js) {",
          "#define JAMP(k) jamp[(k) * js]"]
    L.extend(_colour_quadratic(K, ncol))
    L += ["#undef JAMP", "}", f"}};  // struct {tag}", "}  // namespace mg"]
    return "\n".join(L) + "\n"
