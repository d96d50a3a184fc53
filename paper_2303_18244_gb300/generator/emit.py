"""Emit straight-line CUDA for one process.

For every process the generated header defines, as struct mg::<tag>:

  constants   NPAR, NHEL, NCOL, NDIAG, NAMP, NSLOT, IDEN, CDEN, KNUM[NCOL*NCOL]
  prepare<R>(p, kp, ev, es)          per event, FP64 arithmetic, results stored
                                     as R in the per-thread slab ev[k*es]:
                                     external-state ingredients, propagator
                                     coefficients (-g/P^2, -g/(P^2-m^2+i m G))
  amplitudes<R>(ev, es, hel, kp, jamp, js)  per helicity: external wavefunctions,
                                     off-shell currents and amplitudes diagram
                                     by diagram, accumulated into the colour
                                     flows jamp[k * js], k < NCOL
  colour_quadratic<R>(jamp, js)          sum_ij KNUM_ij Re/Im(J_i) Re/Im(J_j)
                                     (C = KNUM / CDEN)

Helicity index convention: particle i has helicity +1 when bit (NPAR-1-i) of
the index is set, -1 otherwise (index 0 = all negative).
"""
from __future__ import annotations

import os

from .colour import colour_matrix_exact, common_denominator, words
from .diagrams import build_plan, count_diagrams

PROCESSES = {
    "e+ e- > mu+ mu-": ("eemumu", 0),
    "g g > t t~": ("ggtt", 2),
    "g g > t t~ g": ("ggttg", 3),
    "g g > t t~ g g": ("ggttgg", 4),
    "g g > t t~ g g g": ("ggttggg", 5),
}


def _fmt_knum(K) -> str:
    return ", ".join(str(x) for row in K for x in row)


class _Slots:
    def __init__(self):
        self.n = 0
        self.names = {}

    def alloc(self, name, size):
        self.names[name] = self.n
        self.n += size
        return self.names[name]


def _colour_quadratic(K, ncol) -> list[str]:
    """Straight-line sum_ij K_ij (re_i re_j + im_i im_j) using symmetry."""
    out = ["  R acc = R(0);"]
    for i in range(ncol):
        terms_r = []
        terms_i = []
        for j in range(i, ncol):
            k = K[i][j] if j == i else 2 * K[i][j]
            if k == 0:
                continue
            terms_r.append((k, f"JAMP({j}).re"))
            terms_i.append((k, f"JAMP({j}).im"))
        if not terms_r:
            continue
        k0, v0 = terms_r[0]
        out.append(f"  {{ R yr = R({k0}) * {v0}; R yi = R({k0}) * {terms_i[0][1]};")
        for (k, vr), (_, vi) in zip(terms_r[1:], terms_i[1:]):
            out.append(f"    yr = fmaf_t<R>(R({k}), {vr}, yr); yi = fmaf_t<R>(R({k}), {vi}, yi);")
        out.append(f"    acc = fmaf_t<R>(JAMP({i}).re, yr, acc); acc = fmaf_t<R>(JAMP({i}).im, yi, acc); }}")
    out.append("  return acc;")
    return out


def emit_gg(n: int, tag: str, mode: str = "straight") -> str:
    npar = n + 2
    nhel = 1 << npar
    plan = build_plan(n)
    ncol = len(plan.words)
    C = colour_matrix_exact(n)
    cden, K = common_denominator(C)
    ndiag = count_diagrams(n)
    iden = 4 * 64
    for i in range(2, n - 1):
        iden *= i
    slots = [0, 1] + list(range(4, n + 2))  # gluon index -> particle slot
    full = (1 << n) - 1

    # slab layout: momenta and propagator coefficients first (the "lean" part
    # that the FP32 path keeps), then the FP64 external-state ingredients that
    # only the FP64 path stores (FP32 recomputes them per helicity)
    S = _Slots()
    for i in range(n):
        S.alloc(f"k{i}", 4)
    S.alloc("pt", 4)
    S.alloc("ptb", 4)
    gmasks = sorted({op[-1] for op in plan.ops if op[0] in ("3", "4")})
    fmasks = set()
    for op in plan.ops:
        if op[0] == "row":
            fmasks.add(op[3])
        elif op[0] == "col":
            fmasks.add(full ^ op[3])
    fmasks = sorted(fmasks)
    for m in gmasks:
        S.alloc(f"cg{m}", 1)
    for m in fmasks:
        S.alloc(f"cf{m}", 2)
    S.alloc("cgtt", 1)
    nslot_lean = S.n
    for i in range(n):
        S.alloc(f"e{i}", 6)
    S.alloc("ft", 5)
    S.alloc("ftb", 5)
    nslot = S.n
    # table mode, FP32 path: every gluon-subset momentum sum precomputed per event
    # (off: the larger slab halves the CTAs per SM, measured slower)
    ktable = mode == "table" and os.environ.get("MG_TABLE_KSUMS", "0") == "1"
    if ktable:
        for m in range(1, full + 1):
            S.alloc(f"K{m}", 4)
    nslot_k = S.n
    sl = S.names

    L = []
    L.append(f"// generated by paper_2303_18244_gb300.generator for 'g g > t t~{' g' * (n - 2)}'")
    L.append("#pragma once")
    L.append('#include "mg_vertices.cuh"')
    L.append("namespace mg {")
    L.append(f"struct {tag} {{")
    L.append(f"static constexpr int NPAR = {npar};")
    L.append(f"static constexpr int NHEL = {nhel};")
    L.append(f"static constexpr int NCOL = {ncol};")
    L.append(f"static constexpr int NDIAG = {ndiag};")
    L.append(f"static constexpr int NAMP = {len(plan.amps)};")
    L.append(f"static constexpr int NSLOT = {nslot};")
    L.append(f"static constexpr int NSLOT_K = {nslot_k};  // + precomputed subset momenta (table mode, FP32)")
    L.append(f"static constexpr int KBASE = {sl['K1'] if ktable else 0};")
    L.append(f"static constexpr int NSLOT_LEAN = {nslot_lean};  // slots without the external-state ingredients")
    L.append("// FP32 path: recompute the external-state ingredients per helicity instead of")
    L.append("// keeping them in shared memory (measured slower while registers bound occupancy)")
    L.append("static constexpr bool LEAN_SLAB = false;")
    L.append(f"static constexpr double IDEN = {iden}.0;")
    L.append(f"static constexpr int CDEN = {cden};")
    L.append(f"static constexpr int KNUM[NCOL * NCOL] = {{{_fmt_knum(K)}}};")
    L.append("")
    # ---------------- prepare ----------------
    L.append("// per-event ingredients (FP64 arithmetic), stored as R in ev[k * es]")
    L.append("template <typename R>")
    L.append("__device__ static __forceinline__ void prepare(const double* __restrict__ p, const double* __restrict__ kp,")
    L.append("                                        R* __restrict__ ev, const int es) {")
    L.append("  const double g = kp[0], mt = kp[1], wt = kp[2];")
    L.append("#define EV(k) ev[(k) * es]")
    for i in range(n):
        s = slots[i]
        sign = "" if s < 2 else "-"
        L.append(f"  double k{i}[4] = {{{', '.join(f'{sign}p[{4 * s + mu}]' for mu in range(4))}}};")
        for mu in range(4):
            L.append(f"  EV({sl[f'k{i}'] + mu}) = R(k{i}[{mu}]);")
        L.append(f"  {{ double b[6]; vector_basis(p + {4 * s}, b);")
        for j in range(6):
            L.append(f"    EV({sl[f'e{i}'] + j}) = R(b[{j}]);")
        L.append("  }")
    for name, s in (("pt", 2), ("ptb", 3)):
        fname = "ft" if name == "pt" else "ftb"
        for mu in range(4):
            L.append(f"  EV({sl[name] + mu}) = R(p[{4 * s + mu}]);")
        L.append(f"  {{ double f[5]; fermion_ingredients(p + {4 * s}, mt, f);")
        for j in range(5):
            L.append(f"    EV({sl[fname] + j}) = R(f[{j}]);")
        L.append("  }")

    def ksum_fp64(mask):
        idx = [i for i in range(n) if mask >> i & 1]
        return [" + ".join(f"k{i}[{mu}]" for i in idx) for mu in range(4)]

    for m in gmasks:
        comps = ksum_fp64(m)
        L.append(f"  {{ const double K[4] = {{{', '.join(comps)}}};")
        L.append("    const double P2 = K[0] * K[0] - K[1] * K[1] - K[2] * K[2] - K[3] * K[3];")
        L.append(f"    EV({sl[f'cg{m}']}) = R(-g / P2); }}")
    for m in fmasks:
        comps = ksum_fp64(m) if m else ["0.0"] * 4
        L.append(f"  {{ const double K[4] = {{{', '.join(comps)}}};")
        L.append("    double Q[4]; for (int mu = 0; mu < 4; mu++) Q[mu] = p[8 + mu] - K[mu];")
        L.append("    const double dre = Q[0] * Q[0] - Q[1] * Q[1] - Q[2] * Q[2] - Q[3] * Q[3] - mt * mt;")
        L.append("    const double dim = mt * wt;")
        L.append("    const double r = -g / (dre * dre + dim * dim);")
        L.append(f"    EV({sl[f'cf{m}']}) = R(r * dre); EV({sl[f'cf{m}'] + 1}) = R(-r * dim); }}")
    comps = ksum_fp64(full)
    L.append(f"  {{ const double K[4] = {{{', '.join(comps)}}};")
    L.append("    const double P2 = K[0] * K[0] - K[1] * K[1] - K[2] * K[2] - K[3] * K[3];")
    L.append(f"    EV({sl['cgtt']}) = R(g / P2); }}")
    if ktable:
        L.append("  if constexpr (sizeof(R) == 4) {")
        for m in range(1, full + 1):
            comps = ksum_fp64(m)
            for mu in range(4):
                L.append(f"    EV({sl[f'K{m}'] + mu}) = R({comps[mu]});")
        L.append("  }")
    L.append("#undef EV")
    L.append("}")
    L.append("")
    if mode == "table":
        L.extend(_table_sections(plan, tag, n, npar, ncol, sl, slots, full, K))
        L.append(f"}};  // struct {tag}")
        L.append("}  // namespace mg")
        return "\n".join(L) + "\n"
    # ---------------- amplitudes ----------------
    L.append("// one helicity: currents and amplitudes, diagram by diagram, into the colour flows")
    L.append("template <typename R>")
    L.append("__device__ static __forceinline__ void amplitudes(const R* __restrict__ ev, const int es, const int hel,")
    L.append("                                           const double* __restrict__ kp, cx<R>* __restrict__ jamp,")
    L.append("                                           const int js) {")
    L.append("#define EV(k) ev[(k) * es]")
    L.append("#define JAMP(k) jamp[(k) * js]")
    L.append("  const R g = R(kp[0]);")
    L.append("  const R mt = R(kp[1]);")
    for i in range(npar):
        L.append(f"  const int l{i} = ((hel >> {npar - 1 - i}) & 1) ? 1 : -1;")
    L.append(f"  for (int c = 0; c < {ncol}; c++) JAMP(c) = cx<R>{{R(0), R(0)}};")
    # momenta (R) on demand
    emitted_k = set()

    def kname(mask):
        if mask in emitted_k:
            return f"K{mask}"
        idx = [i for i in range(n) if mask >> i & 1]
        comps = []
        for mu in range(4):
            comps.append(" + ".join(f"EV({sl[f'k{i}'] + mu})" for i in idx))
        L.append(f"  const R K{mask}[4] = {{{', '.join(comps)}}};")
        emitted_k.add(mask)
        return f"K{mask}"

    emitted = {}

    def cur(cid):
        """Emit current cid (and its dependencies) if not yet emitted; return its name."""
        if cid in emitted:
            return emitted[cid]
        op = plan.ops[cid]
        kind = op[0]
        name = f"w{cid}"
        if kind == "ext":
            i = op[1]
            L.extend(_ext_gluon_lines(name, i, slots[i], sl, declare=True))
        elif kind == "ubar":
            L.extend(_ext_top_lines(name, "ubar", sl, declare=True))
        elif kind == "v":
            L.extend(_ext_top_lines(name, "v", sl, declare=True))
        elif kind == "gtt":
            a = cur(plan.keys[("row", ())])
            b = cur(plan.keys[("col", ())])
            L.append(f"  const V4<R> {name} = ffv_vcur<R>({a}, {b}, cx<R>{{R(0), EV({sl['cgtt']})}});")
        elif kind == "3":
            x, y, m = op[1], op[2], op[3]
            nx, ny = cur(x), cur(y)
            kx, ky = kname(_mask_of(plan, x)), kname(_mask_of(plan, y))
            L.append(f"  const V4<R> {name} = vvv_cur<R>({kx}, {nx}, {ky}, {ny}, EV({sl[f'cg{m}']}));")
        elif kind == "4":
            x, y, z, br, m = op[1:]
            nx, ny, nz = cur(x), cur(y), cur(z)
            sign = "-" if br in (0, 1) else ""
            L.append(f"  const V4<R> {name} = vvvv_cur<{br}, R>({nx}, {ny}, {nz}, {sign}g * EV({sl[f'cg{m}']}));")
        elif kind == "row":
            prev, gid, m = op[1], op[2], op[3]
            npv, ng = cur(prev), cur(gid)
            c = sl[f"cf{m}"]
            km = kname(m)
            L.append(f"  Sp<R> {name};")
            L.append(f"  {{ const R Q[4] = {{EV({sl['pt']}) - {km}[0], EV({sl['pt'] + 1}) - {km}[1], "
                     f"EV({sl['pt'] + 2}) - {km}[2], EV({sl['pt'] + 3}) - {km}[3]}};")
            L.append(f"    {name} = ffv_row<R>({npv}, {ng}, Q, mt, cx<R>{{EV({c}), EV({c + 1})}}); }}")
        elif kind == "col":
            gid, nxt, m = op[1], op[2], op[3]
            ng, nn = cur(gid), cur(nxt)
            c = sl[f"cf{full ^ m}"]
            km = kname(m)
            L.append(f"  Sp<R> {name};")
            L.append(f"  {{ const R q[4] = {{{km}[0] - EV({sl['ptb']}), {km}[1] - EV({sl['ptb'] + 1}), "
                     f"{km}[2] - EV({sl['ptb'] + 2}), {km}[3] - EV({sl['ptb'] + 3})}};")
            L.append(f"    {name} = ffv_col<R>({ng}, {nn}, q, mt, cx<R>{{EV({c}), EV({c + 1})}}); }}")
        else:
            raise ValueError(kind)
        emitted[cid] = name
        return name

    gtt_id = plan.keys.get(("gtt",))
    for ai in schedule(plan):
        op, co = plan.amps[ai]
        if op[0] == "f":
            r, gq, c = cur(op[1]), cur(op[2]), cur(op[3])
            expr = f"mul_i(g * ffv_amp<R>({r}, {gq}, {c}))"
        elif op[0] == "a3":
            G = cur(gtt_id)
            nx, ny = cur(op[1]), cur(op[2])
            kx, ky = kname(_mask_of(plan, op[1])), kname(_mask_of(plan, op[2]))
            expr = f"vvv_amp<R>({kx}, {nx}, {ky}, {ny}, {G}, -g)"
        else:
            G = cur(gtt_id)
            nx, ny, nz = cur(op[1]), cur(op[2]), cur(op[3])
            br = op[4]
            c = "g * g" if br in (0, 1) else "-g * g"
            expr = f"vvvv_amp<{br}, R>({nx}, {ny}, {nz}, {G}, {c})"
        L.append(f"  {{ const cx<R> a = {expr};")
        parts = []
        for k, c in sorted(co.items()):
            if c == 1:
                parts.append(f"JAMP({k}) = JAMP({k}) + a;")
            elif c == -1:
                parts.append(f"JAMP({k}) = JAMP({k}) - a;")
            else:
                parts.append(f"JAMP({k}) = fma(R({c}), a, JAMP({k}));")
        L.append("    " + " ".join(parts) + " }")
    L.append("#undef JAMP")
    L.append("#undef EV")
    L.append("}")
    L.append("")
    L.append("// sum_ij KNUM_ij (Re J_i Re J_j + Im J_i Im J_j); |M|^2 colour sum = result / CDEN")
    L.append("template <typename R>")
    L.append("__device__ static __forceinline__ R colour_quadratic(const cx<R>* __restrict__ jamp, const int js) {")
    L.append("#define JAMP(k) jamp[(k) * js]")
    L.extend(_colour_quadratic(K, ncol))
    L.append("#undef JAMP")
    L.append("}")
    L.append(f"}};  // struct {tag}")
    L.append("}  // namespace mg")
    return "\n".join(L) + "\n"


def current_deps(plan, cid) -> list[int]:
    """Currents that current cid reads."""
    op = plan.ops[cid]
    k = op[0]
    if k == "3":
        return [op[1], op[2]]
    if k == "4":
        return [op[1], op[2], op[3]]
    if k == "row":
        return [op[1], op[2]]
    if k == "col":
        return [op[1], op[2]]
    if k == "gtt":
        return [plan.keys[("row", ())], plan.keys[("col", ())]]
    return []


def amp_deps(plan, op) -> list[int]:
    gtt = plan.keys.get(("gtt",))
    if op[0] == "f":
        return [op[1], op[2], op[3]]
    if op[0] == "a3":
        return [op[1], op[2], gtt]
    return [op[1], op[2], op[3], gtt]


def schedule(plan) -> list[int]:
    """Order of the amplitudes for emission (currents are emitted on first use).

    Greedy list scheduling against register pressure: at every step take the
    amplitude minimising (currents it still has to create) - (currents whose
    last use it is), preferring amplitudes that touch already-live currents.
    """
    namp = len(plan.amps)
    adeps = [amp_deps(plan, op) for op, _ in plan.amps]
    cdeps = [current_deps(plan, c) for c in range(len(plan.ops))]
    remaining = [0] * len(plan.ops)
    users = [[] for _ in plan.ops]
    for c in range(len(plan.ops)):
        for d in cdeps[c]:
            remaining[d] += 1
    for a in range(namp):
        for d in adeps[a]:
            remaining[d] += 1
            users[d].append(a)
    for c in range(len(plan.ops)):
        for d in cdeps[c]:
            users[d].append(("c", c))
    computed = [False] * len(plan.ops)
    done = [False] * namp
    order = []

    def need_of(a):
        need = []
        seen = set()

        def visit(c):
            if computed[c] or c in seen:
                return
            seen.add(c)
            for d in cdeps[c]:
                visit(d)
            need.append(c)
        for d in adeps[a]:
            visit(d)
        return need

    def score(a):
        need = need_of(a)
        use = {}
        for c in need:
            for d in cdeps[c]:
                use[d] = use.get(d, 0) + 1
        for d in adeps[a]:
            use[d] = use.get(d, 0) + 1
        freed = sum(1 for d, u in use.items() if remaining[d] - u == 0)
        return len(need) - freed, need

    live_amps = set()
    while len(order) < namp:
        cands = [a for a in live_amps if not done[a]] or [next(a for a in range(namp) if not done[a])]
        best = None
        for a in cands:
            sc, need = score(a)
            if best is None or (sc, a) < (best[0], best[1]):
                best = (sc, a, need)
        _, a, need = best
        for c in need:
            computed[c] = True
            for d in cdeps[c]:
                remaining[d] -= 1
            for u in users[c]:
                if not isinstance(u, tuple):
                    live_amps.add(u)
        for d in adeps[a]:
            remaining[d] -= 1
        done[a] = True
        live_amps.discard(a)
        order.append(a)
    return order


def _ext_gluon_lines(name, i, pslot, sl, declare):
    """External gluon i (particle slot pslot): polarisation basis from the slab
    (FP64 path) or recomputed from the stored momentum (FP32 path)."""
    e = sl[f"e{i}"]
    k = sl[f"k{i}"]
    out = "true" if pslot >= 2 else "false"
    sign = "-" if pslot >= 2 else ""  # physical momentum = +-(incoming momentum)
    L = [f"  V4<R> {name};"] if declare else []
    L.append("  {")
    L.append("    R e1[3], e2[3];")
    L.append("    if constexpr (LEAN_SLAB && sizeof(R) == 4) {")
    L.append(f"      const R pk[4] = {{{sign}EV({k}), {sign}EV({k + 1}), {sign}EV({k + 2}), {sign}EV({k + 3})}};")
    L.append("      vector_basis_r<R>(pk, e1, e2);")
    L.append("    } else {")
    L.append(f"      e1[0] = EV({e}); e1[1] = EV({e + 1}); e1[2] = EV({e + 2});")
    L.append(f"      e2[0] = EV({e + 3}); e2[1] = EV({e + 4}); e2[2] = EV({e + 5});")
    L.append("    }")
    L.append(f"    {name} = ext_vector<R>(e1, e2, R(l{pslot}), {out});")
    L.append("  }")
    return L


def _ext_top_lines(name, kind, sl, declare, wrap=False):
    """Outgoing top (ubar) or antitop (v): spinor ingredients from the slab
    (FP64 path) or recomputed from the stored momentum (FP32 path)."""
    f = sl["ft" if kind == "ubar" else "ftb"]
    pm = sl["pt" if kind == "ubar" else "ptb"]
    lam = "l2" if kind == "ubar" else "l3"
    fn = "ext_ubar" if kind == "ubar" else "ext_v"
    typ = "Sp<R>"
    L = [f"  {typ} {name};"] if declare else []
    L.append("  {")
    L.append("    FermIngr<R> fi;")
    L.append("    if constexpr (LEAN_SLAB && sizeof(R) == 4) {")
    L.append(f"      const R pp[4] = {{EV({pm}), EV({pm + 1}), EV({pm + 2}), EV({pm + 3})}};")
    L.append("      fi = fermion_ingredients_r<R>(pp, R(kp[1]));")
    L.append("    } else {")
    L.append(f"      fi = FermIngr<R>{{EV({f}), EV({f + 1}), EV({f + 2}), EV({f + 3}), EV({f + 4})}};")
    L.append("    }")
    rhs = f"{fn}<R>(fi, {lam})"
    L.append(f"    {name} = {'as_v4(' + rhs + ')' if wrap else rhs};")
    L.append("  }")
    return L


def colour_patterns(plan):
    """Group amplitude terms whose colour coefficients agree up to an overall
    sign: returns (pattern of each amp, sign of each amp relative to its
    pattern, list of canonical patterns as sorted (flow, coeff) tuples)."""
    pats, pid, sign = [], [], []
    index = {}
    for op, co in plan.amps:
        t = tuple(sorted(co.items()))
        neg = tuple(sorted((k, -c) for k, c in co.items()))
        key = min(t, neg)
        if key not in index:
            index[key] = len(pats)
            pats.append(key)
        pid.append(index[key])
        sign.append(1 if t == key else -1)
    return pid, sign, pats


def program(plan, by_pattern: bool = False) -> list[tuple[str, int]]:
    """Linear evaluation order: ("cur", id) on first use, ("amp", index) --
    the order in which the straight-line emitter writes the code.  With
    by_pattern, amplitudes sharing a colour pattern are made consecutive
    (patterns in order of first appearance in the schedule)."""
    seq = []
    done = set()
    gtt = plan.keys.get(("gtt",))
    order = schedule(plan)
    if by_pattern:
        pid, _, _ = colour_patterns(plan)
        first = {}
        for pos, ai in enumerate(order):
            first.setdefault(pid[ai], pos)
        order = sorted(order, key=lambda ai: (first[pid[ai]], order.index(ai)))

    def cur(c):
        if c in done:
            return
        op = plan.ops[c]
        k = op[0]
        if k == "gtt":
            cur(plan.keys[("row", ())])
            cur(plan.keys[("col", ())])
        elif k == "3":
            cur(op[1]); cur(op[2])
        elif k == "4":
            cur(op[1]); cur(op[2]); cur(op[3])
        elif k == "row":
            cur(op[1]); cur(op[2])
        elif k == "col":
            cur(op[1]); cur(op[2])
        done.add(c)
        seq.append(("cur", c))

    for ai in order:
        op = plan.amps[ai][0]
        if op[0] == "f":
            cur(op[1]); cur(op[2]); cur(op[3])
        elif op[0] == "a3":
            cur(gtt); cur(op[1]); cur(op[2])
        else:
            cur(gtt); cur(op[1]); cur(op[2]); cur(op[3])
        seq.append(("amp", ai))
    return seq


def _table_sections(plan, tag, n, npar, ncol, sl, slots, full, K) -> list[str]:
    """Op table + interpreter-driven amplitudes() and a looped colour form."""
    # amplitudes grouped by colour pattern (fewer colour-flow updates, a larger
    # current store); MG_TABLE_GROUP=0 keeps the register-pressure order
    by_pattern = os.environ.get("MG_TABLE_GROUP", "1") != "0"
    seq = program(plan, by_pattern=by_pattern)
    pid, psign, pats = colour_patterns(plan)
    if not by_pattern:  # every amplitude its own group
        pats = [tuple(sorted(co.items())) for op, co in plan.amps]
        pid = list(range(len(plan.amps)))
        psign = [1] * len(plan.amps)
    amp_positions = [i for kind, i in seq if kind == "amp"]
    last_of_pattern = {}
    for ai in amp_positions:
        last_of_pattern[pid[ai]] = ai
    pat_jl = {}
    gtt = plan.keys.get(("gtt",))
    # inputs of every step, for liveness
    def inputs(kind, i):
        if kind == "cur":
            return current_deps(plan, i)
        return amp_deps(plan, plan.amps[i][0])
    last = {}
    for t, (kind, i) in enumerate(seq):
        for d in inputs(kind, i):
            last[d] = t
    slot = {}
    free = []
    nstore = 0
    ops = []
    jl = []
    ext_kinds = ("ext", "ubar", "v")
    for t, (kind, i) in enumerate(seq):
        if kind == "cur":
            if free:
                free.sort()
                slot[i] = free.pop(0)
            else:
                slot[i] = nstore
                nstore += 1
            op = plan.ops[i]
            k = op[0]
            out = slot[i]
            if k == "3":
                ops.append([1, out, slot[op[1]], slot[op[2]], _mask_of(plan, op[1]), _mask_of(plan, op[2]),
                            sl[f"cg{op[3]}"], 0])
            elif k == "4":
                ops.append([2, out, slot[op[1]], slot[op[2]], slot[op[3]], op[4], sl[f"cg{op[5]}"], 0])
            elif k == "row":
                ops.append([3, out, slot[op[1]], slot[op[2]], op[3], sl[f"cf{op[3]}"], 0, 0])
            elif k == "col":
                ops.append([4, out, slot[op[1]], slot[op[2]], op[3], sl[f"cf{full ^ op[3]}"], 0, 0])
            elif k == "gtt":
                ops.append([5, out, slot[plan.keys[("row", ())]], slot[plan.keys[("col", ())]], sl["cgtt"],
                            0, 0, 0])
            else:
                assert k in ext_kinds
        else:
            op, co = plan.amps[i]
            # amplitudes of one colour pattern are consecutive: accumulate them
            # (with their sign relative to the pattern) and apply the pattern's
            # flow list once, after the last of them (njl = 0 before that)
            j0, nj = 0, 0
            if last_of_pattern[pid[i]] == i:
                j0 = len(jl)
                for f, c in pats[pid[i]]:
                    assert c in (1, -1), c
                    jl.append((f << 1) | (1 if c < 0 else 0))
                nj = len(jl) - j0
            sg = 1 if psign[i] > 0 else 0
            if op[0] == "f":
                ops.append([6, slot[op[1]], slot[op[2]], slot[op[3]], 0, 0, j0, nj])
            elif op[0] == "a3":
                ops.append([7, slot[op[1]], slot[op[2]], _mask_of(plan, op[1]), _mask_of(plan, op[2]), slot[gtt],
                            j0, nj])
            else:
                ops.append([8, slot[op[1]], slot[op[2]], slot[op[3]], op[4], slot[gtt], j0, nj])
            ops[-1][0] |= (sg << 8)  # bit 8 of the type word: +1 (set) or -1 relative sign
        for d in inputs(kind, i):
            if last[d] == t and plan.ops[d][0] not in ext_kinds:
                free.append(slot[d])
    L = []
    L.append(f"static constexpr int NG = {n};")
    chain = " : ".join(f"i == {i} ? {sl[f'k{i}']}" for i in range(n - 1)) + f" : {sl[f'k{n - 1}']}"
    L.append("// slab offset of gluon i's incoming momentum")
    L.append(f"__host__ __device__ static constexpr int koff(int i) {{ return {chain}; }}")
    L.append(f"static constexpr int PT = {sl['pt']};")
    L.append(f"static constexpr int PTB = {sl['ptb']};")
    L.append(f"static constexpr int NOPS = {len(ops)};")
    L.append(f"static constexpr int NSTORE = {nstore};")
    L.append(f"static constexpr int NJL = {len(jl)};")
    L.append("// per-helicity program: externals into the store, then the op table")
    L.append("template <typename R>")
    L.append("__device__ static __forceinline__ void amplitudes(const R* __restrict__ ev, const int es, const int hel,")
    L.append("                                           const double* __restrict__ kp, cx<R>* __restrict__ jamp,")
    L.append("                                           const int js) {")
    L.append("#define EV(k) ev[(k) * es]")
    L.append("  const R g = R(kp[0]);")
    L.append("  const R mt = R(kp[1]);")
    for i in range(npar):
        L.append(f"  const int l{i} = ((hel >> {npar - 1 - i}) & 1) ? 1 : -1;")
    L.append(f"  V4<R> W[{nstore}];")
    gl_slots = [0, 1] + list(range(4, n + 2))
    for i in range(n):
        cid = plan.keys[("g", ("L", i))]
        L.extend(_ext_gluon_lines(f"W[{slot[cid]}]", i, gl_slots[i], sl, declare=False))
    L.extend(_ext_top_lines(f"W[{slot[plan.keys[('row', ())]]}]", "ubar", sl, declare=False, wrap=True))
    L.extend(_ext_top_lines(f"W[{slot[plan.keys[('col', ())]]}]", "v", sl, declare=False, wrap=True))
    L.append(f"  for (int c = 0; c < {ncol}; c++) jamp[c * js] = cx<R>{{R(0), R(0)}};")
    L.append(f"  run_program<{tag}, R>({tag}_OPS, NOPS, {tag}_JL, ev, es, g, mt, W, jamp, js);")
    L.append("#undef EV")
    L.append("}")
    L.append("// sum_ij KNUM_ij (Re J_i Re J_j + Im J_i Im J_j), KNUM from the table knum")
    L.append("template <typename R>")
    L.append("__device__ static __forceinline__ R colour_quadratic(const cx<R>* __restrict__ jamp, const int js) {")
    L.append(f"  const short* __restrict__ knum = {tag}_KNUM;")
    L.append("  // symmetric: diagonal once, off-diagonal pairs j > i twice (knum holds 2 K_ij there)")
    L.append("  R acc = R(0);")
    L.append("#pragma unroll 1")
    L.append(f"  for (int i = 0; i < {ncol}; i++) {{")
    L.append("    const cx<R> ji = jamp[i * js];")
    L.append(f"    const short* row = knum + i * {ncol};")
    L.append("    R yr = R(__ldg(row + i)) * ji.re, yi = R(__ldg(row + i)) * ji.im;")
    L.append(f"    for (int j = i + 1; j < {ncol}; j++) {{")
    L.append("      const R k = R(__ldg(row + j));")
    L.append("      const cx<R> jj = jamp[j * js];")
    L.append("      yr = fmaf_t<R>(k, jj.re, yr);")
    L.append("      yi = fmaf_t<R>(k, jj.im, yi);")
    L.append("    }")
    L.append("    acc = fmaf_t<R>(ji.re, yr, acc);")
    L.append("    acc = fmaf_t<R>(ji.im, yi, acc);")
    L.append("  }")
    L.append("  return acc;")
    L.append("}")
    # data tables (outside the struct: emitted after it by the caller)
    table_src = []
    table_src.append(f"static __device__ const int4 {tag}_OPS[{2 * len(ops)}] = {{")
    for o in ops:
        table_src.append(f"  {{{o[0]}, {o[1]}, {o[2]}, {o[3]}}}, {{{o[4]}, {o[5]}, {o[6]}, {o[7]}}},")
    table_src.append("};")
    table_src.append(f"static __device__ const short {tag}_JL[{len(jl)}] = {{{', '.join(map(str, jl))}}};")
    # upper triangle doubled (the symmetric loop reads K_ii and 2 K_ij, j > i); |2 K| <= 8192 fits a short
    KS = [[K[i][j] if i == j else (2 * K[i][j] if j > i else 0) for j in range(ncol)] for i in range(ncol)]
    table_src.append(f"static __device__ const short {tag}_KNUM[{ncol * ncol}] = {{{_fmt_knum(KS)}}};")
    _TABLES[tag] = table_src
    return L


_TABLES: dict = {}


def _mask_of(plan, cid) -> int:
    op = plan.ops[cid]
    if op[0] == "ext":
        return 1 << op[1]
    if op[0] == "3":
        return op[3]
    if op[0] == "4":
        return op[5]
    raise ValueError(op)


def emit_eemumu(tag: str) -> str:
    """e+(0) e-(1) -> mu+(2) mu-(3): s-channel photon and Z (2 diagrams).
    kp = {e^2, gz^2, gL, gR, MZ, WZ}; amp = e^2/s Je.Jm + gz^2/(s - MZ^2 + i MZ WZ) JZe.JZm."""
    L = []
    L.append("// generated by paper_2303_18244_gb300.generator for 'e+ e- > mu+ mu-'")
    L.append("#pragma once")
    L.append('#include "mg_vertices.cuh"')
    L.append("namespace mg {")
    L.append(f"struct {tag} {{")
    L.append("static constexpr int NPAR = 4;")
    L.append("static constexpr int NHEL = 16;")
    L.append("static constexpr int NCOL = 1;")
    L.append("static constexpr int NDIAG = 2;")
    L.append("static constexpr int NAMP = 2;")
    L.append("static constexpr int NSLOT = 23;")
    L.append("static constexpr int NSLOT_K = 23;")
    L.append("static constexpr int KBASE = 0;")
    L.append("static constexpr int NSLOT_LEAN = 23;")
    L.append("static constexpr bool LEAN_SLAB = false;")
    L.append("static constexpr double IDEN = 4.0;")
    L.append("static constexpr int CDEN = 1;")
    L.append("static constexpr int KNUM[1] = {1};")
    L.append("template <typename R>")
    L.append("__device__ static __forceinline__ void prepare(const double* __restrict__ p, const double* __restrict__ kp,")
    L.append("                                        R* __restrict__ ev, const int es) {")
    L.append("#define EV(k) ev[(k) * es]")
    L.append("  for (int i = 0; i < 4; i++) {")
    L.append("    double f[5]; fermion_ingredients(p + 4 * i, 0.0, f);")
    L.append("    for (int j = 0; j < 5; j++) EV(5 * i + j) = R(f[j]);")
    L.append("  }")
    L.append("  const double P[4] = {p[0] + p[4], p[1] + p[5], p[2] + p[6], p[3] + p[7]};")
    L.append("  const double s = P[0] * P[0] - P[1] * P[1] - P[2] * P[2] - P[3] * P[3];")
    L.append("  EV(20) = R(kp[0] / s);")
    L.append("  const double dre = s - kp[4] * kp[4], dim = kp[4] * kp[5];")
    L.append("  const double r = kp[1] / (dre * dre + dim * dim);")
    L.append("  EV(21) = R(r * dre); EV(22) = R(-r * dim);")
    L.append("#undef EV")
    L.append("}")
    L.append("template <typename R>")
    L.append("__device__ static __forceinline__ void amplitudes(const R* __restrict__ ev, const int es, const int hel,")
    L.append("                                           const double* __restrict__ kp, cx<R>* __restrict__ jamp,")
    L.append("                                           const int js) {")
    L.append("#define EV(k) ev[(k) * es]")
    L.append("#define ING(i) FermIngr<R>{EV(5 * (i)), EV(5 * (i) + 1), EV(5 * (i) + 2), EV(5 * (i) + 3), EV(5 * (i) + 4)}")
    for i in range(4):
        L.append(f"  const int l{i} = ((hel >> {3 - i}) & 1) ? 1 : -1;")
    L.append("  const Sp<R> w0 = ext_vbar<R>(ING(0), l0);")
    L.append("  const Sp<R> w1 = ext_u<R>(ING(1), l1);")
    L.append("  const Sp<R> w2 = ext_v<R>(ING(2), l2);")
    L.append("  const Sp<R> w3 = ext_ubar<R>(ING(3), l3);")
    L.append("  const cx<R> one = {R(1), R(0)};")
    L.append("  const R gl = R(kp[2]), gr = R(kp[3]);")
    L.append("  const V4<R> ja = ffv_vcur<R>(w0, w1, one);")
    L.append("  const V4<R> la = ffv_vcur<R>(w3, w2, one);")
    L.append("  const V4<R> jz = ffv_vcur<R>(w0, w1, one, gl, gr);")
    L.append("  const V4<R> lz = ffv_vcur<R>(w3, w2, one, gl, gr);")
    L.append("  const cx<R> amp_a = EV(20) * dot(ja, la);")
    L.append("  const cx<R> amp_z = cx<R>{EV(21), EV(22)} * dot(jz, lz);")
    L.append("  jamp[0] = amp_a + amp_z;")
    L.append("#undef ING")
    L.append("#undef EV")
    L.append("}")
    L.append("template <typename R>")
    L.append("__device__ static __forceinline__ R colour_quadratic(const cx<R>* __restrict__ jamp, const int js) {")
    L.append("  return jamp[0].re * jamp[0].re + jamp[0].im * jamp[0].im;")
    L.append("}")
    L.append(f"}};  // struct {tag}")
    L.append("}  // namespace mg")
    return "\n".join(L) + "\n"


# processes evaluated by the table interpreter (straight-line code too large to compile)
TABLE_MODE = {"ggttggg"}


def emit(proc: str) -> tuple[str, str]:
    """(tag, header source) for a process string."""
    tag, n = PROCESSES[proc]
    if n == 0:
        return tag, emit_eemumu(tag)
    if tag in TABLE_MODE:
        src = emit_gg(n, tag, mode="table")
        tables = "\n".join(_TABLES.pop(tag))
        src = src.replace('#include "mg_vertices.cuh"', '#include "mg_vertices.cuh"\n#include "mg_interp.cuh"')
        return tag, src.replace(f"struct {tag} {{", f"{tables}\nstruct {tag} {{", 1)
    return tag, emit_gg(n, tag)


# threads per CTA: FP64 path / mixed path (shared-memory slab sizes differ)
THREADS = {
    "eemumu": (128, 128),
    "ggtt": (128, 128),
    "ggttg": (128, 128),
    "ggttgg": (64, 128),
    "ggttggg": (64, 64),
}


# processes whose mixed path contracts colour on the tensor cores (the FP16
# operand tiles of 128 events plus FP32 colour-flow accumulators must fit in
# shared memory next to the per-event slab)
TENSOR_CORE_COLOUR = {"ggttg", "ggttgg"}


def emit_kernels_tu(proc: str) -> tuple[str, str]:
    """Translation unit instantiating the kernels of one process."""
    tag, _ = PROCESSES[proc]
    nt64, nt32 = THREADS[tag]
    tc = tag in TENSOR_CORE_COLOUR
    mixed = f"launch_sigma_tc<{tag}>(a)" if tc else f"launch_sigma<{tag}, float, {nt32}>(a)"
    tck = f"tc::pad16({tag}::NCOL)" if tc else "0"
    src = f"""// generated by paper_2303_18244_gb300.generator: kernels of '{proc}'
#include "../mg_kernels.cuh"
#include "../mg_colour_tc.cuh"
#include "{tag}.cuh"

namespace mg {{
static int sigma_fp64(const LaunchArgs& a) {{ return launch_sigma<{tag}, double, {nt64}>(a); }}
static int sigma_mixed(const LaunchArgs& a) {{ return {mixed}; }}
static int helicities(const LaunchArgs& a) {{ return launch_helicities<{tag}, {nt64}>(a); }}
int select_{tag}_fp64(const LaunchArgs& a);
int select_{tag}_mixed(const LaunchArgs& a);
int paper_{tag}(const LaunchArgs& a);
static const ProcDesc desc = {{"{proc}", "{tag}", {tag}::NPAR, {tag}::NHEL, {tag}::NCOL, {tag}::NDIAG,
                              {tag}::NAMP, {tag}::IDEN, {tag}::CDEN, {tag}::KNUM,
                              sigma_fp64, sigma_mixed, helicities, {tck},
                              select_{tag}_fp64, select_{tag}_mixed, paper_{tag}}};
const ProcDesc* proc_{tag}() {{ return &desc; }}
}}  // namespace mg
"""
    return tag, src


def emit_select_tu(proc: str) -> tuple[str, str]:
    """Translation unit of the helicity/colour-choice kernels and of the
    paper-style mixed kernel (compiled in parallel with the main kernels)."""
    tag, _ = PROCESSES[proc]
    nt64, nt32 = THREADS[tag]
    src = f"""// generated by paper_2303_18244_gb300.generator: helicity/colour choice kernels of '{proc}'
#include "../mg_kernels.cuh"
#include "{tag}.cuh"

namespace mg {{
int select_{tag}_fp64(const LaunchArgs& a) {{ return launch_select<{tag}, double, {nt64}>(a); }}
int select_{tag}_mixed(const LaunchArgs& a) {{ return launch_select<{tag}, float, {nt32}>(a); }}
int paper_{tag}(const LaunchArgs& a) {{ return launch_sigma_paper<{tag}, {nt64}>(a); }}
}}  // namespace mg
"""
    return tag, src
