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

import math
import os
import re

from .colour import colour_matrix_exact, common_denominator, words
from .diagrams import build_plan, count_diagrams

PROCESSES = {
    "e+ e- > mu+ mu-": ("eemumu", 0),
    "u u~ > t t~": ("uutt", 0),
    "u u~ > t t~ g": ("uuttg", 0),
    "u u~ > t t~ g g": ("uuttgg", 0),
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


# processes whose FP32 path recomputes the external-state ingredients per
# helicity instead of keeping them in the shared-memory slab (gg -> t t~ g g:
# with the flows sharing the operand-tile space the CTA needs 66 KB instead of
# 109 KB, and the freed L1 holds more of the spilled registers; measured 5 %
# faster)
LEAN_SLAB = set(filter(None, os.environ.get("MG_LEAN_SLAB", "ggttgg").split(",")))


def emit_gg(n: int, tag: str, mode: str = "straight", chunk_order: str = "pattern") -> str:
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
    L.append(f"static constexpr int NSLOT_LEAN = {nslot_lean};  // slots without the external-state ingredients")
    L.append("// FP32 path: recompute the external-state ingredients per helicity instead of")
    L.append("// keeping them in shared memory (measured slower while registers bound occupancy)")
    L.append(f"static constexpr bool LEAN_SLAB = {'true' if tag in LEAN_SLAB else 'false'};")
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
        # the lean FP32 slab has no room for the external-state ingredients
        L.append(f"  if constexpr (!(LEAN_SLAB && sizeof(R) == 4)) {{ double b[6]; vector_basis(p + {4 * s}, b);")
        for j in range(6):
            L.append(f"    EV({sl[f'e{i}'] + j}) = R(b[{j}]);")
        L.append("  }")
    for name, s in (("pt", 2), ("ptb", 3)):
        fname = "ft" if name == "pt" else "ftb"
        for mu in range(4):
            L.append(f"  EV({sl[name] + mu}) = R(p[{4 * s + mu}]);")
        L.append(f"  if constexpr (!(LEAN_SLAB && sizeof(R) == 4)) {{ double f[5]; fermion_ingredients(p + {4 * s}, mt, f);")
        for j in range(5):
            L.append(f"    EV({sl[fname] + j}) = R(f[{j}]);")
        L.append("  }")

    # propagator invariants: (sum of the momenta)^2 [- m^2] by inv_mass2,
    # compensated (double-double) in the FP64 path, so that a nearly collinear
    # or nearly on-shell propagator keeps full relative precision
    def inv_mass2(rows, m2):
        vv = ", ".join(v for v, _ in rows)
        ss = ", ".join("double(1)" if sg > 0 else "double(-1)" for _, sg in rows)
        return (f"const double* const vv[{len(rows)}] = {{{vv}}}; const double ss[{len(rows)}] = {{{ss}}};",
                f"inv_mass2<R>(vv, ss, {m2})")

    for m in gmasks:
        decl, call = inv_mass2([(f"k{i}", 1) for i in range(n) if m >> i & 1], "0.0")
        L.append(f"  {{ {decl}")
        L.append(f"    const double P2 = {call};")
        L.append(f"    EV({sl[f'cg{m}']}) = R(-g / P2); }}")
    for m in fmasks:
        decl, call = inv_mass2([("pd + 8", 1)] + [(f"k{i}", -1) for i in range(n) if m >> i & 1], "mt * mt")
        L.append(f"  {{ {decl}")
        L.append(f"    const double dre = {call};")
        L.append("    const double dim = mt * wt;")
        L.append("    const double r = -g / (dre * dre + dim * dim);")
        L.append(f"    EV({sl[f'cf{m}']}) = R(r * dre); EV({sl[f'cf{m}'] + 1}) = R(-r * dim); }}")
    decl, call = inv_mass2([(f"k{i}", 1) for i in range(n)], "0.0")
    L.append(f"  {{ {decl}")
    L.append(f"    const double P2 = {call};")
    L.append(f"    EV({sl['cgtt']}) = R(g / P2); }}")
    L.append("#undef EV")
    L.append("}")
    L.append("")
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
        L.append(f"  const M4<R> K{mask} = {{{{{', '.join(comps)}}}}};")
        emitted_k.add(mask)
        return f"K{mask}"

    emitted = {}
    imports = {}  # chunked mode: currents produced by an earlier chunk -> store slot

    def cur(cid):
        """Emit current cid (and its dependencies) if not yet emitted; return its name."""
        if cid in emitted:
            return emitted[cid]
        op = plan.ops[cid]
        kind = op[0]
        name = f"w{cid}"
        if cid in imports:
            if kind in ("row", "col", "ubar", "v"):
                L.append(f"  const Sp<R> {name} = as_sp(W[{imports[cid]}]);")
            else:
                L.append(f"  const V4<R> {name} = W[{imports[cid]}];")
            emitted[cid] = name
            return name
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
            L.append(f"  {{ const M4<R> Q = {{{{EV({sl['pt']}) - {km}[0], EV({sl['pt'] + 1}) - {km}[1], "
                     f"EV({sl['pt'] + 2}) - {km}[2], EV({sl['pt'] + 3}) - {km}[3]}}}};")
            L.append(f"    {name} = ffv_row<R>({npv}, {ng}, Q, mt, cx<R>{{EV({c}), EV({c + 1})}}); }}")
        elif kind == "col":
            gid, nxt, m = op[1], op[2], op[3]
            ng, nn = cur(gid), cur(nxt)
            c = sl[f"cf{full ^ m}"]
            km = kname(m)
            L.append(f"  Sp<R> {name};")
            L.append(f"  {{ const M4<R> q = {{{{{km}[0] - EV({sl['ptb']}), {km}[1] - EV({sl['ptb'] + 1}), "
                     f"{km}[2] - EV({sl['ptb'] + 2}), {km}[3] - EV({sl['ptb'] + 3})}}}};")
            L.append(f"    {name} = ffv_col<R>({ng}, {nn}, q, mt, cx<R>{{EV({c}), EV({c + 1})}}); }}")
        else:
            raise ValueError(kind)
        emitted[cid] = name
        return name

    gtt_id = plan.keys.get(("gtt",))
    # MG_LINE_GROUP=1: amplitudes sharing a colour pattern are made consecutive
    # and summed in a register before the colour flows are updated (always on
    # in chunked mode)
    group = mode == "chunked" or os.environ.get("MG_LINE_GROUP", "0") == "1"
    amp_order = [i for kind, i in program(plan, by_pattern=True) if kind == "amp"] if group else schedule(plan)
    if mode == "chunked" and chunk_order == "shared":
        amp_order = shared_current_order(plan, amp_order)
    pid, psign, pats = colour_patterns(plan)
    last_of = {}
    for ai in amp_order:
        last_of[pid[ai]] = ai

    # a (row, column) spinor pair used by several top-line amplitudes (of the
    # program, or of one chunk in chunked mode) is contracted once into
    # V = rbar gamma^mu c, and each of its amplitudes becomes the Minkowski
    # product V.J (gg -> t t~ g g: 74 pairs for 114 amplitudes, measured 6 %
    # faster in FP32, 11 % in FP64; MG_PAIR_V=0 turns it off)
    pair_v = os.environ.get("MG_PAIR_V", "1") == "1"
    # chunked mode, MG_FLUSH_CALL=1: a colour pattern's flows are updated by one
    # non-inlined call over its entry in a device table of (flow << 1 | minus)
    # instead of inline code per pattern (gg -> t t~ g g g: measured 2.5x
    # slower in FP32, 15 % in FP64)
    flush_calls = os.environ.get("MG_FLUSH_CALL", "0") == "1"
    flow_list: list = []
    flow_list_off: dict = {}
    pair_uses: dict = {}
    for ai in amp_order:
        op = plan.amps[ai][0]
        if op[0] == "f":
            pair_uses[(op[1], op[3])] = pair_uses.get((op[1], op[3]), 0) + 1
    pair_names: dict = {}

    def emit_amp(ai):
        op, co = plan.amps[ai]
        if op[0] == "f":
            r, gq, c = cur(op[1]), cur(op[2]), cur(op[3])
            key = (op[1], op[3])
            if pair_v and pair_uses[key] > 1:
                if key not in pair_names:
                    pair_names[key] = f"vp{op[1]}_{op[3]}"
                    L.append(f"  const V4<R> {pair_names[key]} = ffv_vcur<R>({r}, {c}, cx<R>{{R(1), R(0)}});")
                expr = f"mul_i(g * dot({pair_names[key]}, {gq}))"
            else:
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
        if group:
            L.append(f"    pacc = pacc {'+' if psign[ai] > 0 else '-'} a;")
            if last_of[pid[ai]] == ai:
                pat = pats[pid[ai]]
                if mode == "chunked" and flush_calls:
                    # the pattern's flow list in the device table; one call
                    off = flow_list_off.setdefault(pid[ai], len(flow_list))
                    if off == len(flow_list):
                        flow_list.extend((k << 1) | (1 if c < 0 else 0) for k, c in pat)
                    L.append(f"    jamp.flush({tag}_FLOWLIST + {off}, {len(pat)}, pacc);")
                    L.append("    pacc = cx<R>{R(0), R(0)};")
                elif mode == "chunked":
                    kk = ", ".join(str(k) for k, _ in pat)
                    sg = ", ".join("1" if c > 0 else "-1" for _, c in pat)
                    L.append(f"    {{ constexpr int kk[{len(pat)}] = {{{kk}}}; constexpr int sg[{len(pat)}] = {{{sg}}};")
                    L.append(f"      jamp.template update<{len(pat)}>(kk, sg, pacc); }}")
                    L.append("    pacc = cx<R>{R(0), R(0)};")
                else:
                    parts = []
                    for k, c in pat:
                        parts.append(f"JAMP({k}) = JAMP({k}) {'+' if c > 0 else '-'} pacc;")
                    parts.append("pacc = cx<R>{R(0), R(0)};")
                    L.append("    " + " ".join(parts))
            L.append("  }")
            return
        parts = []
        for k, c in sorted(co.items()):
            if c == 1:
                parts.append(f"JAMP({k}) = JAMP({k}) + a;")
            elif c == -1:
                parts.append(f"JAMP({k}) = JAMP({k}) - a;")
            else:
                parts.append(f"JAMP({k}) = fma(R({c}), a, JAMP({k}));")
        L.append("    " + " ".join(parts) + " }")

    if mode == "chunked":
        main_L = L
        chunk_size = CHUNK_AMPS
        chunks, curc = [], []
        for ai in amp_order:  # cut only at the end of a colour-pattern group
            curc.append(ai)
            if len(curc) >= chunk_size and last_of[pid[ai]] == ai:
                chunks.append(curc)
                curc = []
        if curc:
            chunks.append(curc)
        # pass 1: where each current is produced and which later chunks read it.
        # Local currents are recomputed in every chunk that uses them instead
        # of passing through the store: the external states, and with
        # MG_REMAT=1 also the currents built from external states only
        # (gg -> t t~ g g g: measured 6 % slower in FP32, 17 % in FP64).
        remat = os.environ.get("MG_REMAT", "0") == "1"
        ext_kinds = ("ext", "ubar", "v")

        def is_local(c):
            if plan.ops[c][0] in ext_kinds:
                return True
            return remat and all(plan.ops[d][0] in ext_kinds for d in current_deps(plan, c))
        produced, readers = {}, {}
        for j, ch in enumerate(chunks):
            seen = set()

            def visit(c, j=j, seen=seen):
                if c in seen:
                    return
                seen.add(c)
                if not is_local(c) and c in produced:
                    readers.setdefault(c, set()).add(j)
                    return
                for d in current_deps(plan, c):
                    visit(d)
                if not is_local(c):
                    produced[c] = j
            for ai in ch:
                for d in amp_deps(plan, plan.amps[ai][0]):
                    visit(d)
        cross = {c for c in readers}
        # store slots by interval colouring over chunk indices
        intervals = sorted((produced[c], max(readers[c]), c) for c in cross)
        slot_of, free_at = {}, []
        for a0, a1, c in intervals:
            for si, end in enumerate(free_at):
                if end < a0:
                    slot_of[c] = si
                    free_at[si] = a1
                    break
            else:
                slot_of[c] = len(free_at)
                free_at.append(a1)
        nstore = max(1, len(free_at))
        chunk_funcs = []
        for j, ch in enumerate(chunks):
            L = []
            emitted = {}
            emitted_k = set()
            imports = {c: slot_of[c] for c in cross if produced[c] < j and j in readers[c]}
            L.append("template <typename R, typename J>")
            L.append(f"__device__ static __noinline__ void chunk{j}(const R* __restrict__ ev, const int es, "
                     "const int hel, const double* __restrict__ kp, V4<R>* __restrict__ W, const J jamp) {")
            L.append("  [[maybe_unused]] const R g = R(kp[0]);")
            L.append("  [[maybe_unused]] const R mt = R(kp[1]);")
            for i in range(npar):
                L.append(f"  [[maybe_unused]] const int l{i} = ((hel >> {npar - 1 - i}) & 1) ? 1 : -1;")
            L.append("  cx<R> pacc = {R(0), R(0)};")
            pair_names.clear()
            pair_uses.clear()
            for ai in ch:
                op = plan.amps[ai][0]
                if op[0] == "f":
                    pair_uses[(op[1], op[3])] = pair_uses.get((op[1], op[3]), 0) + 1
            for ai in ch:
                emit_amp(ai)
            for c in sorted(cross):
                if produced[c] == j:
                    nm = emitted[c]
                    conv = f"as_v4({nm})" if plan.ops[c][0] in ("row", "col") else nm
                    L.append(f"  W[{slot_of[c]}] = {conv};")
            L.append("}")
            chunk_funcs.append(L)
        L = main_L
        # the chunk-calling amplitudes function replaces the straight-line body begun above
        head = L.index("// one helicity: currents and amplitudes, diagram by diagram, into the colour flows")
        del L[head:]
        L.append("#define EV(k) ev[(k) * es]")
        for f in chunk_funcs:
            L.extend(f)
        L.append("#undef EV")
        L.append(f"static constexpr int NCHUNK = {len(chunks)};")
        L.append(f"static constexpr int NSTORE = {nstore};")
        L.append("// one helicity: the chunks in order, the colour flows in the store J")
        L.append("// (FlowsSmem: shared memory; FlowsTmem: tensor memory)")
        L.append("template <typename R, typename J>")
        L.append("__device__ static __forceinline__ void amplitudes_store(const R* __restrict__ ev, const int es, "
                 "const int hel, const double* __restrict__ kp, const J jamp) {")
        L.append(f"  V4<R> W[{nstore}];  // currents passed between chunks")
        L.append("  jamp.zero(NCOL);")
        for j in range(len(chunks)):
            L.append(f"  chunk{j}<R, J>(ev, es, hel, kp, W, jamp);")
            if j + 1 < len(chunks):
                L.append("  jamp.chunk_done();")
        L.append("}")
        L.append("template <typename R>")
        L.append("__device__ static __forceinline__ void amplitudes(const R* __restrict__ ev, const int es, const int hel,")
        L.append("                                           const double* __restrict__ kp, cx<R>* __restrict__ jamp,")
        L.append("                                           const int js) {")
        L.append("  amplitudes_store<R>(ev, es, hel, kp, FlowsSmem<R>{jamp, js});")
        L.append("}")
        L.append("")
        L.extend(_colour_quadratic_looped(tag, ncol))
        L.append(f"}};  // struct {tag}")
        L.append("}  // namespace mg")
        src = "\n".join(L) + "\n"
        src = src.replace('#include "mg_vertices.cuh"', '#include "mg_vertices.cuh"\n#include "mg_flowstore.cuh"', 1)
        tables = _knum_table(tag, K)
        if flush_calls:
            tables += (f"\nstatic __device__ const short {tag}_FLOWLIST[{max(1, len(flow_list))}] = {{"
                       + ", ".join(str(v) for v in flow_list) + "};")
        return src.replace(f"struct {tag} {{", tables + f"\nstruct {tag} {{", 1)

    if group:
        L.append("  cx<R> pacc = {R(0), R(0)};")
    for ai in amp_order:
        emit_amp(ai)
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


def shared_current_order(plan, order, window: int = 2) -> list[int]:
    """Chunked mode, chunk order "shared": the colour-pattern groups of
    `order` (each kept contiguous) reordered greedily so that each group
    follows the ones whose currents it shares most (over the last `window`
    groups), which shortens the life of currents that cross chunk boundaries
    (gg -> t t~ g g g, chunks of 40: store 241 -> 87 slots, crossing
    currents 363 -> 183)."""
    pid, _, _ = colour_patterns(plan)
    ext = ("ext", "ubar", "v")
    groups: dict = {}
    for ai in order:
        groups.setdefault(pid[ai], []).append(ai)

    def needs(ai):
        out, stack = set(), list(amp_deps(plan, plan.amps[ai][0]))
        while stack:
            c = stack.pop()
            if c in out or plan.ops[c][0] in ext:
                continue
            out.add(c)
            stack.extend(current_deps(plan, c))
        return out
    uses = {g: set().union(*[needs(a) for a in amps]) for g, amps in groups.items()}
    remaining = list(groups)
    chosen = [remaining.pop(0)]
    while remaining:
        recent = set().union(*[uses[g] for g in chosen[-window:]])
        best = max(remaining, key=lambda g: (len(uses[g] & recent), -len(uses[g] - recent)))
        remaining.remove(best)
        chosen.append(best)
    return [a for g in chosen for a in groups[g]]


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


def _knum_table(tag, K) -> str:
    """Colour numerators as a device table: row i holds K_ii on the diagonal and
    2 K_ij for j > i (the form is symmetric); the lower triangle is unused."""
    ncol = len(K)
    vals = []
    for i in range(ncol):
        for j in range(ncol):
            vals.append(K[i][j] if j == i else (2 * K[i][j] if j > i else 0))
    assert max(abs(v) for v in vals) < 32768
    rows = [", ".join(str(v) for v in vals[i * ncol:(i + 1) * ncol]) for i in range(ncol)]
    return (f"static __device__ const short {tag}_KNUM[{ncol * ncol}] = {{\n  " + ",\n  ".join(rows) + "};")


def _colour_quadratic_looped(tag, ncol) -> list[str]:
    """sum_ij KNUM_ij (Re J_i Re J_j + Im J_i Im J_j) as a loop over the device
    table (the straight-line form of a 120-flow process is too much code)."""
    L = []
    L.append("// colour numerators in device memory: K_ii on the diagonal, 2 K_ij for j > i")
    L.append(f"__device__ static const short* knum_dev() {{ return {tag}_KNUM; }}")
    L.append("// sum_ij KNUM_ij (Re J_i Re J_j + Im J_i Im J_j); |M|^2 colour sum = result / CDEN")
    L.append("template <typename R>")
    L.append("__device__ static __forceinline__ R colour_quadratic(const cx<R>* __restrict__ jamp, const int js) {")
    L.append(f"  const short* __restrict__ knum = {tag}_KNUM;")
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
    return L



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


def emit_uutt(tag: str) -> str:
    """u(0) u~(1) -> t(2) t~(3): the s-channel gluon diagram.  One colour
    structure T^a_{i_t j_tbar} T^a_{i_u j_ubar}, whose colour sum is 2 (KNUM
    {2}, CDEN 1).  kp = {g_s, mt}; amp = (g^2 / s) (vbar gamma u).(ubar gamma v)."""
    L = []
    L.append("// generated by paper_2303_18244_gb300.generator for 'u u~ > t t~'")
    L.append("#pragma once")
    L.append('#include "mg_vertices.cuh"')
    L.append("namespace mg {")
    L.append(f"struct {tag} {{")
    L.append("static constexpr int NPAR = 4;")
    L.append("static constexpr int NHEL = 16;")
    L.append("static constexpr int NCOL = 1;")
    L.append("static constexpr int NDIAG = 1;")
    L.append("static constexpr int NAMP = 1;")
    L.append("static constexpr int NSLOT = 21;")
    L.append("static constexpr int NSLOT_LEAN = 21;")
    L.append("static constexpr bool LEAN_SLAB = false;")
    L.append("static constexpr double IDEN = 36.0;")
    L.append("static constexpr int CDEN = 1;")
    L.append("static constexpr int KNUM[1] = {2};")
    L.append("// per-event ingredients (FP64): spinor ingredients of the four fermions, g^2 / s")
    L.append("template <typename R>")
    L.append("__device__ static __forceinline__ void prepare(const double* __restrict__ p, const double* __restrict__ kp,")
    L.append("                                        R* __restrict__ ev, const int es) {")
    L.append("#define EV(k) ev[(k) * es]")
    L.append("  for (int i = 0; i < 4; i++) {")
    L.append("    double f[5]; fermion_ingredients(p + 4 * i, i < 2 ? 0.0 : kp[1], f);")
    L.append("    for (int j = 0; j < 5; j++) EV(5 * i + j) = R(f[j]);")
    L.append("  }")
    L.append("  const double P[4] = {p[0] + p[4], p[1] + p[5], p[2] + p[6], p[3] + p[7]};")
    L.append("  const double s = P[0] * P[0] - P[1] * P[1] - P[2] * P[2] - P[3] * P[3];")
    L.append("  EV(20) = R(kp[0] * kp[0] / s);")
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
    L.append("  const Sp<R> w0 = ext_u<R>(ING(0), l0);")
    L.append("  const Sp<R> w1 = ext_vbar<R>(ING(1), l1);")
    L.append("  const Sp<R> w2 = ext_ubar<R>(ING(2), l2);")
    L.append("  const Sp<R> w3 = ext_v<R>(ING(3), l3);")
    L.append("  const cx<R> one = {R(1), R(0)};")
    L.append("  const V4<R> jl = ffv_vcur<R>(w1, w0, one);")
    L.append("  const V4<R> jh = ffv_vcur<R>(w2, w3, one);")
    L.append("  jamp[0] = EV(20) * dot(jl, jh);")
    L.append("#undef ING")
    L.append("#undef EV")
    L.append("}")
    L.append("template <typename R>")
    L.append("__device__ static __forceinline__ R colour_quadratic(const cx<R>* __restrict__ jamp, const int js) {")
    L.append("  return R(2) * (jamp[0].re * jamp[0].re + jamp[0].im * jamp[0].im);")
    L.append("}")
    L.append(f"}};  // struct {tag}")
    L.append("}  // namespace mg")
    return "\n".join(L) + "\n"


def emit_uuttg(tag: str) -> str:
    """u(0) u~(1) -> t(2) t~(3) g(4): five diagrams (gluon off the u end, the
    u~ end, the t end, the t~ end, three-gluon vertex on the s-channel gluon),
    Feynman rules with vertices i g gamma^mu T^a and g f^{abc} V3, gluon
    propagator -i g_{mu nu}/k^2, quark propagator i (qslash + m)/(q^2 - m^2
    + i m Gamma).  Colour: four flows (generator.colour_two_lines) with the
    decomposition and colour matrix computed there.  kp = {g_s, mt, Gamma_t}.
    Slab (per event, FP64 set-up): spinor ingredients of the four fermions,
    the gluon's transverse basis, the propagator momenta and coefficients."""
    from .colour_two_lines import colour_matrix, decomposition
    dec = decomposition()
    C = colour_matrix()
    cden, K = common_denominator(C)
    L = []
    L.append("// generated by paper_2303_18244_gb300.generator for 'u u~ > t t~ g'")
    L.append("#pragma once")
    L.append('#include "mg_vertices.cuh"')
    L.append("namespace mg {")
    L.append(f"struct {tag} {{")
    L.append("static constexpr int NPAR = 5;")
    L.append("static constexpr int NHEL = 32;")
    L.append("static constexpr int NCOL = 4;")
    L.append("static constexpr int NDIAG = 5;")
    L.append("static constexpr int NAMP = 5;")
    L.append("static constexpr int NSLOT = 60;")
    L.append("static constexpr int NSLOT_LEAN = 60;")
    L.append("static constexpr bool LEAN_SLAB = false;")
    L.append("static constexpr double IDEN = 36.0;")
    L.append(f"static constexpr int CDEN = {cden};")
    L.append(f"static constexpr int KNUM[NCOL * NCOL] = {{{_fmt_knum(K)}}};")
    # slab: 0-19 fermion ingredients, 20-25 gluon basis, 26-29 qA = p1 - p5,
    # 30-33 qB = p5 - p2, 34-37 qC = p3 + p5, 38-41 qD = -p4 - p5, 42-45 P = p1 + p2,
    # 46-49 -q34, 50 cA, 51 cB, 52-53 cC, 54-55 cD, 56 1/q34^2, 57 1/s
    L.append("// per-event set-up (FP64): spinor ingredients, gluon basis, propagator momenta")
    L.append("// and coefficients (i g)(i / denominator)")
    L.append("template <typename R>")
    L.append("__device__ static __forceinline__ void prepare(const double* __restrict__ p, const double* __restrict__ kp,")
    L.append("                                        R* __restrict__ ev, const int es) {")
    L.append("#define EV(k) ev[(k) * es]")
    L.append("  const double g = kp[0], mt = kp[1], wt = kp[2];")
    L.append("  for (int i = 0; i < 4; i++) {")
    L.append("    double f[5]; fermion_ingredients(p + 4 * i, i < 2 ? 0.0 : mt, f);")
    L.append("    for (int j = 0; j < 5; j++) EV(5 * i + j) = R(f[j]);")
    L.append("  }")
    L.append("  { double b[6]; vector_basis(p + 16, b); for (int j = 0; j < 6; j++) EV(20 + j) = R(b[j]); }")
    L.append("  double q[6][4];")
    L.append("  for (int mu = 0; mu < 4; mu++) {")
    L.append("    q[0][mu] = p[mu] - p[16 + mu];")
    L.append("    q[1][mu] = p[16 + mu] - p[4 + mu];")
    L.append("    q[2][mu] = p[8 + mu] + p[16 + mu];")
    L.append("    q[3][mu] = -p[12 + mu] - p[16 + mu];")
    L.append("    q[4][mu] = p[mu] + p[4 + mu];")
    L.append("    q[5][mu] = -p[8 + mu] - p[12 + mu];")
    L.append("  }")
    L.append("  for (int k = 0; k < 6; k++)")
    L.append("    for (int mu = 0; mu < 4; mu++) EV(26 + 4 * k + mu) = R(q[k][mu]);")
    L.append("  // invariants compensated in the FP64 path (inv_mass2): collinear emissions")
    L.append("  double m2[6];")
    rows = [[("pd + 0", 1), ("pd + 16", -1)], [("pd + 16", 1), ("pd + 4", -1)], [("pd + 8", 1), ("pd + 16", 1)],
            [("pd + 12", -1), ("pd + 16", -1)], [("pd + 0", 1), ("pd + 4", 1)], [("pd + 8", -1), ("pd + 12", -1)]]
    for k, rr in enumerate(rows):
        vv = ", ".join(v for v, _ in rr)
        ss = ", ".join("double(1)" if sg > 0 else "double(-1)" for _, sg in rr)
        L.append(f"  {{ const double* const vv[2] = {{{vv}}}; const double ss[2] = {{{ss}}};")
        L.append(f"    m2[{k}] = inv_mass2<R>(vv, ss, {'mt * mt' if k in (2, 3) else '0.0'}); }}")
    L.append("  EV(50) = R(-g / m2[0]);")
    L.append("  EV(51) = R(-g / m2[1]);")
    L.append("  for (int k = 2; k < 4; k++) {")
    L.append("    const double dre = m2[k], dim = mt * wt, r = -g / (dre * dre + dim * dim);  // m2[2], m2[3]: q^2 - mt^2")
    L.append("    EV(52 + 2 * (k - 2)) = R(r * dre); EV(53 + 2 * (k - 2)) = R(-r * dim);")
    L.append("  }")
    L.append("  EV(56) = R(1.0 / m2[5]);")
    L.append("  EV(57) = R(1.0 / m2[4]);")
    L.append("#undef EV")
    L.append("}")
    L.append("template <typename R>")
    L.append("__device__ static __forceinline__ void amplitudes(const R* __restrict__ ev, const int es, const int hel,")
    L.append("                                           const double* __restrict__ kp, cx<R>* __restrict__ jamp,")
    L.append("                                           const int js) {")
    L.append("#define EV(k) ev[(k) * es]")
    L.append("#define ING(i) FermIngr<R>{EV(5 * (i)), EV(5 * (i) + 1), EV(5 * (i) + 2), EV(5 * (i) + 3), EV(5 * (i) + 4)}")
    L.append("#define MOM(k) M4<R>{{EV(k), EV((k) + 1), EV((k) + 2), EV((k) + 3)}}")
    L.append("  const R g = R(kp[0]), mt = R(kp[1]);")
    for i in range(5):
        L.append(f"  const int l{i} = ((hel >> {4 - i}) & 1) ? 1 : -1;")
    L.append("  const Sp<R> w0 = ext_u<R>(ING(0), l0);")
    L.append("  const Sp<R> w1 = ext_vbar<R>(ING(1), l1);")
    L.append("  const Sp<R> w2 = ext_ubar<R>(ING(2), l2);")
    L.append("  const Sp<R> w3 = ext_v<R>(ING(3), l3);")
    L.append("  const R e1[3] = {EV(20), EV(21), EV(22)}, e2[3] = {EV(23), EV(24), EV(25)};")
    L.append("  const V4<R> eps = ext_vector<R>(e1, e2, R(l4), true);")
    L.append("  const cx<R> ig = {R(0), g};")
    L.append("  const cx<R> mi_q2 = {R(0), -EV(56)}, mi_s = {R(0), -EV(57)};  // -i/q34^2, -i/s")
    L.append("  const V4<R> Lc = ffv_vcur<R>(w1, w0, ig);  // vbar2 (i g gamma) u1")
    L.append("  const V4<R> Hc = ffv_vcur<R>(w2, w3, ig);  // ubar3 (i g gamma) v4")
    L.append("  const Sp<R> sA = ffv_col<R>(eps, w0, MOM(26), R(0), cx<R>{EV(50), R(0)});")
    L.append("  const Sp<R> sB = ffv_row<R>(w1, eps, MOM(30), R(0), cx<R>{EV(51), R(0)});")
    L.append("  const Sp<R> sC = ffv_row<R>(w2, eps, MOM(34), mt, cx<R>{EV(52), EV(53)});")
    L.append("  const Sp<R> sD = ffv_col<R>(eps, w3, MOM(38), mt, cx<R>{EV(54), EV(55)});")
    L.append("  cx<R> A[5];")
    L.append("  A[0] = mi_q2 * dot(ffv_vcur<R>(w1, sA, ig), Hc);")
    L.append("  A[1] = mi_q2 * dot(ffv_vcur<R>(sB, w0, ig), Hc);")
    L.append("  A[2] = mi_s * dot(Lc, ffv_vcur<R>(sC, w3, ig));")
    L.append("  A[3] = mi_s * dot(Lc, ffv_vcur<R>(w2, sD, ig));")
    L.append("  V4<R> GL, GH;")
    L.append("  for (int mu = 0; mu < 4; mu++) {")
    L.append("    GL.c[mu] = mi_s * Lc.c[mu];")
    L.append("    GH.c[mu] = mi_q2 * Hc.c[mu];")
    L.append("  }")
    L.append("  A[4] = vvv_amp<R>(MOM(42), GL, MOM(46), GH, eps, g);")
    for m in range(4):
        terms = []
        for d in range(5):
            re, im = dec[d][m]
            if re == 0 and im == 0:
                continue
            terms.append(f"cx<R>{{R({float(re)!r}), R({float(im)!r})}} * A[{d}]")
        L.append(f"  jamp[{m} * js] = " + " + ".join(terms) + ";")
    L.append("#undef MOM")
    L.append("#undef ING")
    L.append("#undef EV")
    L.append("}")
    L.append("// sum_ij KNUM_ij (Re J_i Re J_j + Im J_i Im J_j); |M|^2 colour sum = result / CDEN")
    L.append("template <typename R>")
    L.append("__device__ static __forceinline__ R colour_quadratic(const cx<R>* __restrict__ jamp, const int js) {")
    L.append("#define JAMP(k) jamp[(k) * js]")
    L.extend(_colour_quadratic(K, 4))
    L.append("#undef JAMP")
    L.append("}")
    L.append(f"}};  // struct {tag}")
    L.append("}  // namespace mg")
    return "\n".join(L) + "\n"


# processes emitted as straight-line code cut into separately compiled chunk
# functions of about CHUNK_AMPS amplitudes (one straight-line function of this
# size does not compile in reasonable time); currents that cross a chunk
# boundary are passed through a per-thread store
CHUNKED = {"ggttggg"}
CHUNK_AMPS = int(os.environ.get("MG_CHUNK_AMPS", "40"))
# order of the amplitudes over the chunks, per precision: "pattern" (colour-
# pattern groups in generation order) or "shared" (groups ordered by the
# currents they share, shared_current_order: cross-chunk store 241 -> 87
# slots).  Measured on gg -> t t~ g g g, 65536 events (A/B on one GB300):
# mixed 2.80e5 -> 2.91e5 MEs/s with "shared", FP64 1.92e4 -> 1.87e4; each
# precision takes its faster order.  MG_CHUNK_ORDER overrides both.
CHUNK_ORDER = {"f64": "pattern", "f32": "shared"}


def chunk_order(prec: str) -> str:
    return os.environ.get("MG_CHUNK_ORDER") or CHUNK_ORDER[prec]


def header_name(proc: str, prec: str) -> str:
    """Generated header a precision's translation unit includes: one per
    process, or one per precision where the chunk orders differ."""
    tag, _ = PROCESSES[proc]
    if tag in CHUNKED and chunk_order(prec) != chunk_order("f64"):
        return f"{tag}_{prec}.cuh"
    return f"{tag}.cuh"


def emit(proc: str, prec: str = "f64") -> tuple[str, str]:
    """(tag, header source) for a process string; prec selects the chunk
    order of a chunked process (the header of the other processes does not
    depend on it).  A header that differs from the FP64 one puts its struct in
    an inline namespace of its own, so that its kernels never share a mangled
    name with those built from the FP64 header."""
    tag, n = PROCESSES[proc]
    if tag == "eemumu":
        src = emit_eemumu(tag)
    elif tag == "uutt":
        src = emit_uutt(tag)
    elif tag == "uuttg":
        src = emit_uuttg(tag)
    elif tag == "uuttgg":
        from .two_lines import emit_uuttgg
        src = emit_uuttgg(tag)
    else:
        src = emit_gg(n, tag, mode="chunked" if tag in CHUNKED else "straight", chunk_order=chunk_order(prec))
    src = _prepare_in_D(src)
    if header_name(proc, prec) != f"{tag}.cuh":
        ns = f"chunk_order_{chunk_order(prec)}"
        assert src.count("namespace mg {\n") == 1 and src.rstrip().endswith("}  // namespace mg")
        src = src.replace("namespace mg {\n", f"namespace mg {{\ninline namespace {ns} {{\n", 1)
        src = src.rstrip()[: -len("}  // namespace mg")] + f"}}  // namespace {ns}\n}}  // namespace mg\n"
    return tag, src


def _prepare_in_D(src: str) -> str:
    """Give prepare() a second template parameter D, the arithmetic type of the
    per-event set-up (double by default; float for the all-FP32 mode): the
    emitted FP64 set-up is rewritten with D for double, the event's momenta
    converted to D once."""
    head = "template <typename R>\n__device__ static __forceinline__ void prepare("
    assert src.count(head) == 1
    src = src.replace(head, "template <typename R, typename D = double>\n"
                            "__device__ static __forceinline__ void prepare(", 1)
    lines = src.split("\n")
    i0 = next(i for i, l in enumerate(lines) if "void prepare(" in l)
    i1 = next(i for i in range(i0, len(lines)) if lines[i].rstrip().endswith("const int es) {"))
    i2 = next(i for i in range(i1, len(lines)) if lines[i] == "}")
    # E: arithmetic type of the external-state ingredients (spinor and
    # polarisation set-up), FP32 whenever the amplitudes are FP32; the
    # propagator denominators keep D
    body = ["  D pd[NPAR * 4];", "  for (int i = 0; i < NPAR * 4; i++) pd[i] = D(p[i]);",
            "  using E = typename std::conditional<sizeof(R) == 4, float, D>::type;",
            "  E pe[NPAR * 4];", "  for (int i = 0; i < NPAR * 4; i++) pe[i] = E(p[i]);"]
    for l in lines[i1 + 1:i2]:
        if not l.startswith("#"):
            l = re.sub(r"\bdouble\b", "D", l)
            l = re.sub(r"(?<![\w.])p\[", "pd[", l)
            l = l.replace("(p + ", "(pd + ")
            l = re.sub(r"\bkp\[(\d)\]", r"D(kp[\1])", l)
            l = re.sub(r"(?<![\w.\[])(\d+\.\d+)(?![\w.])", r"D(\1)", l)
            if "vector_basis(" in l:
                l = l.replace("D b[6]", "E b[6]").replace("vector_basis(pd", "vector_basis(pe")
            if "fermion_ingredients(" in l:
                l = l.replace("D f[5]", "E f[5]")
                l = re.sub(r"fermion_ingredients\(pd( \+ [^,]+), ([^;]+), f\);",
                           r"fermion_ingredients(pe\1, E(\2), f);", l)
        body.append(l)
    return "\n".join(lines[:i1 + 1] + body + lines[i2:])


# threads per CTA: FP64 path / mixed path (shared-memory slab sizes differ)
THREADS = {
    "eemumu": (128, 128),
    "uutt": (128, 128),
    "uuttg": (128, 128),
    "uuttgg": (64, 128),
    "ggtt": (128, 128),
    "ggttg": (128, 128),
    "ggttgg": (64, 128),
    "ggttggg": (64, 64),
}


# processes whose mixed path contracts colour on the tensor cores (the FP16
# operand tiles of 128 events plus FP32 colour-flow accumulators must fit in
# shared memory next to the per-event slab)
TENSOR_CORE_COLOUR = {"ggttg", "ggttgg"}
# tensor-core processes whose colour flows share the operand tiles' space
TC_ALIAS = {"ggttgg"}
# processes whose FP64 |M|^2 keeps the colour flows in tensor memory (120
# complex FP64 flows per event do not fit in shared memory beside the slab)
TMEM_FP64 = set(filter(None, os.environ.get("MG_TMEM_FP64", "ggttggg").split(",")))
# processes whose mixed path writes the colour flows of every (helicity, event)
# row to HBM and contracts them on the tensor cores in a second kernel
# (120 flows: the operand tiles do not fit beside the per-event state)
TENSOR_CORE_ROWS = set(filter(None, os.environ.get("MG_TC_ROWS", "ggttggg").split(",")))


# processes whose vertex routines are called rather than inlined, per
# precision: the straight-line helicity program then shrinks to a sequence of
# calls to a few small routines that stay in the instruction cache.  Measured:
# faster for the FP32 path of the larger processes, whose inlined program
# streams from L2 on every helicity; the FP64 paths (bound by the FP64 pipe;
# gg -> t t~ g g g 1.05e4 inlined against 8.4e3 called) and the smaller
# processes keep the inlined code
VERTEX_CALLS = {"f32": {"ggttgg", "ggttggg"}, "f64": set()}


# colour-flow counts of the processes written by hand (gg processes: n!)
FIXED_NCOL = {"eemumu": 1, "uutt": 1, "uuttg": 4, "uuttgg": 12}


def emit_tu(proc: str, prec: str) -> tuple[str, str]:
    """Translation unit instantiating the kernels of one process in one
    precision ("f64": FP64 |M|^2, helicity scan, FP64 helicity/colour choice,
    the paper's mixed mode, and the process descriptor; "f32": the mixed
    |M|^2 and the mixed helicity/colour choice)."""
    tag, n = PROCESSES[proc]
    nt64, nt32 = THREADS[tag]
    calls = "#define MG_VERTEX __noinline__\n" if tag in VERTEX_CALLS[prec] else ""
    if prec == "f32" and tag in TC_ALIAS:
        calls += "#define MG_TC_ALIAS 1\n"
    head = f"// generated by paper_2303_18244_gb300.generator: {prec} kernels of '{proc}'\n{calls}"
    tc = tag in TENSOR_CORE_COLOUR or tag in TENSOR_CORE_ROWS
    if prec == "f32":
        if tag in TENSOR_CORE_ROWS:
            mixed = f"launch_sigma_rows<{tag}, {nt32}>(a)"
        elif tc:
            mixed = f"launch_sigma_tc<{tag}>(a)"
        else:
            mixed = f"launch_sigma<{tag}, float, {nt32}>(a)"
        inc = '#include "../mg_colour_tc.cuh"\n' if tc else ""
        src = f"""{head}#include "../mg_kernels.cuh"
{inc}#include "{header_name(proc, "f32")}"

namespace mg {{
int sigma_{tag}_mixed(const LaunchArgs& a) {{ return {mixed}; }}
int select_{tag}_mixed(const LaunchArgs& a) {{ return launch_select<{tag}, float, {nt32}>(a); }}
int sigma_{tag}_float(const LaunchArgs& a) {{ return launch_sigma<{tag}, float, {nt32}, float, float>(a); }}
}}  // namespace mg
"""
        return tag, src
    ncol = FIXED_NCOL.get(tag) or math.factorial(n)
    tck = ((ncol + 15) // 16) * 16 if tc else 0
    if tag in TMEM_FP64:
        inc64 = '#include "../mg_colour_tc.cuh"\n'
        fp64 = f"launch_sigma_tmem64<{tag}>(a)"
    else:
        inc64 = ""
        fp64 = f"launch_sigma<{tag}, double, {nt64}>(a)"
    src = f"""{head}#include "../mg_kernels.cuh"
{inc64}#include "{header_name(proc, "f64")}"

namespace mg {{
static int sigma_fp64(const LaunchArgs& a) {{ return {fp64}; }}
static int helicities(const LaunchArgs& a) {{ return launch_helicities<{tag}, {nt64}>(a); }}
static int select_fp64(const LaunchArgs& a) {{ return launch_select<{tag}, double, {nt64}>(a); }}
static int paper(const LaunchArgs& a) {{ return launch_sigma_paper<{tag}, {nt64}>(a); }}
int sigma_{tag}_mixed(const LaunchArgs& a);
int select_{tag}_mixed(const LaunchArgs& a);
int sigma_{tag}_float(const LaunchArgs& a);
static_assert({tag}::NCOL == {ncol}, "colour-flow count");
static const ProcDesc desc = {{"{proc}", "{tag}", {tag}::NPAR, {tag}::NHEL, {tag}::NCOL, {tag}::NDIAG,
                              {tag}::NAMP, {tag}::IDEN, {tag}::CDEN, {tag}::KNUM,
                              sigma_fp64, sigma_{tag}_mixed, helicities, {tck},
                              select_fp64, select_{tag}_mixed, paper, sigma_{tag}_float,
                              {1 if tag in TENSOR_CORE_ROWS else 0}}};
const ProcDesc* proc_{tag}() {{ return &desc; }}
}}  // namespace mg
"""
    return tag, src
