"""Pins of the FP64 CPU oracle to facts outside itself.

Each test ties one part of the oracle to a closed form, an identity of the
algebra, a symmetry, or an independent brute-force evaluation, so that a
dropped term, a wrong sign, a wrong index or a transposed operand anywhere in
mg_oracle.c fails at least one of them:

* e+e- -> mu+mu-: photon-only e^4 (1 + cos^2 theta); photon+Z helicity closed form.
* g g -> t t~: the analytic LO result (Gamma_t = 0), and its threshold and
  massless limits.
* Dirac algebra, spinor and polarisation completeness (external states).
* SU(3): Tr(T^a T^b) = delta/2, Casimir, structure constants, colour matrix
  of g g -> t t~ exact, colour matrices real symmetric.
* Partial amplitudes: gauge invariance (Ward identity) for every ordering and
  every gluon with 2..5 gluons -- fixes the three- and four-gluon vertices
  relative to the quark-gluon vertex.
* Colour decomposition: colour-dressed recursion with explicit f^{abc},
  summed over all colour assignments, equals A^dagger C A (2..4 gluons).
* Full ME: Bose symmetry and Lorentz invariance; the spin and colour sum
  rebuilt over every spin state of a helicity basis built in the test, with
  the identical-particle factor counted from Bose symmetry (3..5 gluons).
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2303_18244_gb300.inputs import process_momenta

PROC_N = {2: "g g > t t~", 3: "g g > t t~ g", 4: "g g > t t~ g g", 5: "g g > t t~ g g g"}
SQRTS = {2: 1000.0, 3: 1200.0, 4: 1500.0, 5: 2000.0}


def mdot(a, b):
    return a[..., 0] * b[..., 0] - (a[..., 1:] * b[..., 1:]).sum(-1)


# --------------------------------------------------------------------------
# e+ e- -> mu+ mu-
# --------------------------------------------------------------------------

def _cos_e_mu(p):
    # angle between e- (slot 1) and mu- (slot 3)
    a, b = p[:, 1, 1:], p[:, 3, 1:]
    return (a * b).sum(-1) / np.linalg.norm(a, axis=1) / np.linalg.norm(b, axis=1)


def test_eemumu_photon_only_closed_form():
    """QED: spin-averaged |M|^2 = e^4 (1 + cos^2 theta) for massless fermions."""
    p = process_momenta("e+ e- > mu+ mu-", 500.0, 200, 1)
    par = O.Params(photon_only=1.0)
    me = O.me("e+ e- > mu+ mu-", p, par)
    e2 = 4 * math.pi / par.alpha_em_inv
    c = _cos_e_mu(p)
    np.testing.assert_allclose(me, e2 ** 2 * (1 + c ** 2), rtol=1e-13)


def test_eemumu_gamma_z_helicity_closed_form():
    """gamma+Z: (e^4/4)[(|A_LL|^2+|A_RR|^2)(1+c)^2 + (|A_LR|^2+|A_RL|^2)(1-c)^2],
    A_ij = Q_e Q_mu + g_i g_j s / (sw^2 cw^2 (s - MZ^2 + i MZ GZ)), G_F scheme."""
    p = process_momenta("e+ e- > mu+ mu-", 500.0, 200, 1)
    par = O.Params()
    me = O.me("e+ e- > mu+ mu-", p, par)
    alpha = 1.0 / par.alpha_em_inv
    mz2 = par.mz ** 2
    mw2 = mz2 / 2 + math.sqrt(mz2 ** 2 / 4 - math.pi * alpha * mz2 / (math.sqrt(2) * par.gf))
    sw2 = 1 - mw2 / mz2
    cw2 = 1 - sw2
    g = {"L": -0.5 + sw2, "R": sw2}
    s = 500.0 ** 2
    bw = s / (s - mz2 + 1j * par.mz * par.wz)
    A = {i + j: 1.0 + g[i] * g[j] / (sw2 * cw2) * bw for i in "LR" for j in "LR"}
    c = _cos_e_mu(p)
    e4 = (4 * math.pi * alpha) ** 2
    want = e4 / 4 * ((abs(A["LL"]) ** 2 + abs(A["RR"]) ** 2) * (1 + c) ** 2
                     + (abs(A["LR"]) ** 2 + abs(A["RL"]) ** 2) * (1 - c) ** 2)
    np.testing.assert_allclose(me, want, rtol=1e-13)


# --------------------------------------------------------------------------
# g g -> t t~ analytic
# --------------------------------------------------------------------------

def ggtt_analytic(p, mt, alpha_s):
    """Spin- and colour-averaged LO g g -> Q Qbar (Combridge 1979; e.g. Ellis,
    Stirling, Webber, 'QCD and collider physics'):
    g^4 (1/(6 t1 t2) - 3/8)(t1^2 + t2^2 + rho - rho^2/(4 t1 t2)),
    t1 = 2 p1.p3 / s, t2 = 2 p2.p3 / s, rho = 4 m^2 / s."""
    s = mdot(p[:, 0] + p[:, 1], p[:, 0] + p[:, 1])
    t1 = 2 * mdot(p[:, 0], p[:, 2]) / s
    t2 = 2 * mdot(p[:, 1], p[:, 2]) / s
    rho = 4 * mt * mt / s
    g4 = (4 * math.pi * alpha_s) ** 2
    return g4 * (1 / (6 * t1 * t2) - 3 / 8) * (t1 ** 2 + t2 ** 2 + rho - rho ** 2 / (4 * t1 * t2))


def test_ggtt_analytic_formula_limits():
    """Self-checks of the closed form: threshold 7/48 g^4; massless gg -> qq~."""
    g4 = (4 * math.pi * 0.118) ** 2
    s = 1.0
    # threshold: t1 = t2 = 1/2, rho = 1
    t1 = t2 = 0.5
    rho = 1.0
    thr = g4 * (1 / (6 * t1 * t2) - 3 / 8) * (t1 ** 2 + t2 ** 2 + rho - rho ** 2 / (4 * t1 * t2))
    assert abs(thr / g4 - 7 / 48) < 1e-15
    # massless: (t^2+u^2)/(6tu) - 3(t^2+u^2)/(8 s^2)
    t, u = -0.3, -0.7
    t1, t2 = -t / s, -u / s
    lhs = (1 / (6 * t1 * t2) - 3 / 8) * (t1 ** 2 + t2 ** 2)
    rhs = (t * t + u * u) / (6 * t * u) - 3 * (t * t + u * u) / (8 * s * s)
    assert abs(lhs - rhs) < 1e-15


@pytest.mark.parametrize("mt", [173.0, 0.0])
def test_ggtt_matches_analytic(mt):
    p = process_momenta("g g > t t~", 1000.0, 300, 2, mt=mt)
    par = O.Params(mt=mt, wt=0.0)
    me = O.me("g g > t t~", p, par)
    np.testing.assert_allclose(me, ggtt_analytic(p, mt, par.alpha_s), rtol=1e-12)


def uutt_analytic(p, mt, alpha_s):
    """q q~ -> Q Q~ at LO, averaged over initial spins and colours:
    (4/9) g^4 [(m^2 - t)^2 + (m^2 - u)^2 + 2 m^2 s] / s^2 (textbook result)."""
    g4 = (4 * math.pi * alpha_s) ** 2

    def m2(a):
        return a[..., 0] ** 2 - a[..., 1] ** 2 - a[..., 2] ** 2 - a[..., 3] ** 2

    s = m2(p[:, 0] + p[:, 1])
    t = m2(p[:, 0] - p[:, 2])
    u = m2(p[:, 0] - p[:, 3])
    m = mt * mt
    return 4.0 / 9.0 * g4 * ((m - t) ** 2 + (m - u) ** 2 + 2 * m * s) / s ** 2


@pytest.mark.parametrize("mt", [173.0, 0.0])
def test_uutt_matches_analytic(mt):
    p = process_momenta("u u~ > t t~", 1000.0, 300, 7, mt=mt)
    par = O.Params(mt=mt)
    me = O.me("u u~ > t t~", p, par)
    np.testing.assert_allclose(me, uutt_analytic(p, mt, par.alpha_s), rtol=1e-12)


def test_uutt_analytic_formula_massless_limit():
    """Self-check of the closed form: m = 0 gives (4/9) g^4 (t^2 + u^2) / s^2."""
    g4 = (4 * math.pi * 0.118) ** 2
    E = 50.0
    c = 0.3
    p = np.array([[[E, 0, 0, E], [E, 0, 0, -E], [E, E * math.sqrt(1 - c * c), 0, E * c],
                   [E, -E * math.sqrt(1 - c * c), 0, -E * c]]])
    s, t, u = 4 * E * E, -2 * E * E * (1 - c), -2 * E * E * (1 + c)
    assert abs(uutt_analytic(p, 0.0, 0.118)[0] / (4 / 9 * g4 * (t * t + u * u) / (s * s)) - 1) < 1e-14


def test_ggtt_width_is_small_effect():
    """With Gamma_t in the t-channel propagators the result moves by O(1e-4) only."""
    p = process_momenta("g g > t t~", 1000.0, 100, 2)
    me = O.me("g g > t t~", p, O.Params())
    r = me / ggtt_analytic(p, 173.0, 0.118)
    assert np.all(np.abs(r - 1) < 1e-3)
    assert np.any(np.abs(r - 1) > 1e-9)


# --------------------------------------------------------------------------
# Dirac algebra and external states
# --------------------------------------------------------------------------

G = np.diag([1.0, -1.0, -1.0, -1.0])


def test_clifford_algebra():
    gam = O.gamma()
    for mu in range(4):
        for nu in range(4):
            ac = gam[mu] @ gam[nu] + gam[nu] @ gam[mu]
            np.testing.assert_allclose(ac, 2 * G[mu, nu] * np.eye(4), atol=1e-15)
        np.testing.assert_allclose(gam[4] @ gam[mu] + gam[mu] @ gam[4], 0, atol=1e-15)
    np.testing.assert_allclose(gam[4] @ gam[4], np.eye(4), atol=1e-15)


def _slash(p):
    gam = O.gamma()
    return sum(G[mu, mu] * gam[mu] * p[mu] for mu in range(4))


@pytest.mark.parametrize("m", [173.0, 0.0])
def test_spinor_completeness_and_dirac_equation(m):
    rng = np.random.default_rng(1)
    for _ in range(5):
        k = rng.normal(size=3) * 300
        p = np.array([math.sqrt(m * m + k @ k), *k])
        su = sum(np.outer(O.spinor("u", p, m, s), O.spinor("ubar", p, m, s)) for s in range(2))
        sv = sum(np.outer(O.spinor("v", p, m, s), O.spinor("vbar", p, m, s)) for s in range(2))
        ps = _slash(p)
        np.testing.assert_allclose(su, ps + m * np.eye(4), atol=1e-11 * p[0])
        np.testing.assert_allclose(sv, ps - m * np.eye(4), atol=1e-11 * p[0])
        for s in range(2):
            np.testing.assert_allclose((ps - m * np.eye(4)) @ O.spinor("u", p, m, s), 0, atol=1e-10 * p[0])
            np.testing.assert_allclose((ps + m * np.eye(4)) @ O.spinor("v", p, m, s), 0, atol=1e-10 * p[0])


def test_polarisation_transverse_complete():
    rng = np.random.default_rng(2)
    dirs = [rng.normal(size=3) for _ in range(5)] + [np.array([0, 0, 1.0]), np.array([0, 0, -1.0])]
    for d in dirs:
        k = np.array([np.linalg.norm(d), *d]) * 100
        e = np.array([O.polarisation(k, w) for w in range(2)])
        assert np.allclose(e[:, 0], 0)
        np.testing.assert_allclose(e[:, 1:] @ k[1:], 0, atol=1e-12)
        np.testing.assert_allclose(e[:, 1:] @ e[:, 1:].T, np.eye(2), atol=1e-14)
        kh = k[1:] / np.linalg.norm(k[1:])
        np.testing.assert_allclose(e[:, 1:].T @ e[:, 1:], np.eye(3) - np.outer(kh, kh), atol=1e-14)


# --------------------------------------------------------------------------
# SU(3) colour algebra
# --------------------------------------------------------------------------

def test_gell_mann_algebra():
    T = O.generators()
    tr = np.einsum("aij,bji->ab", T, T)
    np.testing.assert_allclose(tr, 0.5 * np.eye(8), atol=1e-15)
    np.testing.assert_allclose(np.einsum("aij,ajk->ik", T, T), 4 / 3 * np.eye(3), atol=1e-15)
    for a in range(8):
        np.testing.assert_allclose(T[a], T[a].conj().T, atol=0)
        assert abs(np.trace(T[a])) < 1e-15
    f = O.fabc()
    assert abs(f[0, 1, 2] - 1.0) < 1e-14                  # f^{123} = 1
    assert abs(f[3, 4, 7] - math.sqrt(3) / 2) < 1e-14      # f^{458} = sqrt(3)/2
    np.testing.assert_allclose(f, -np.transpose(f, (1, 0, 2)), atol=1e-15)
    np.testing.assert_allclose(f, np.transpose(f, (1, 2, 0)), atol=1e-15)
    # [T^a, T^b] = i f^{abc} T^c
    comm = np.einsum("aij,bjk->abik", T, T) - np.einsum("bij,ajk->abik", T, T)
    np.testing.assert_allclose(comm, 1j * np.einsum("abc,cik->abik", f, T), atol=1e-15)
    # adjoint Casimir: f^{acd} f^{bcd} = 3 delta^{ab}
    np.testing.assert_allclose(np.einsum("acd,bcd->ab", f, f), 3 * np.eye(8), atol=1e-13)


def test_colour_matrix_ggtt_exact():
    C = O.colour_matrix(2)
    np.testing.assert_allclose(C, [[16 / 3, -2 / 3], [-2 / 3, 16 / 3]], atol=1e-14)


@pytest.mark.parametrize("n", [2, 3, 4, 5])
def test_colour_matrix_real_symmetric(n):
    C = O.colour_matrix(n)
    assert np.max(np.abs(C.imag)) < 1e-13
    np.testing.assert_allclose(C.real, C.real.T, atol=1e-13)
    # diagonal: sum over a of Tr(T^a1..T^an T^an..T^a1) = N C_F^n
    np.testing.assert_allclose(np.diag(C.real), 3 * (4 / 3) ** n, rtol=1e-12)
    # positive semi-definite (a sum of |.|^2)
    assert np.linalg.eigvalsh(C.real).min() > -1e-10


# --------------------------------------------------------------------------
# Partial amplitudes: Ward identities, colour decomposition
# --------------------------------------------------------------------------

def _qline_states(n, seed, which=(0, 0), pol=0):
    p = process_momenta(PROC_N[n], SQRTS[n], 1, seed)[0]
    slots = [0, 1] + list(range(4, n + 2))
    kin = np.array([p[s] if s < 2 else -p[s] for s in slots])
    eps = np.array([O.polarisation(p[s], (pol >> i) & 1) for i, s in enumerate(slots)], dtype=complex)
    ub = O.spinor("ubar", p[2], 173.0, which[0])
    v = O.spinor("v", p[3], 173.0, which[1])
    return p, kin, eps, ub, v


@pytest.mark.parametrize("n", [2, 3, 4, 5])
@pytest.mark.parametrize("seed", [7, 8])
def test_ward_identity_every_ordering(n, seed):
    """eps_i -> k_i annihilates every colour-ordered amplitude (Gamma_t = 0)."""
    par = O.Params(wt=0.0)
    p, kin, eps, ub, v = _qline_states(n, seed, which=(seed & 1, 1), pol=seed)
    A = O.ordered_amps(n, kin, eps, p[2], ub, p[3], v, par)
    scale = np.max(np.abs(A))
    for i in range(n):
        e2 = eps.copy()
        e2[i] = kin[i]
        W = O.ordered_amps(n, kin, e2, p[2], ub, p[3], v, par)
        # k_i carries the scale of an energy: normalise by it
        assert np.max(np.abs(W)) / kin[i][0] < 1e-10 * scale


@pytest.mark.parametrize("n", [2, 3, 4])
def test_colour_dressed_recursion_equals_colour_ordered(n):
    """Explicit-colour recursion (P&S vertices with f^{abc}) summed over every
    colour assignment equals A^dagger C A from the colour-ordered recursion."""
    par = O.Params()
    for seed, pol in ((3, 0), (4, 5)):
        p, kin, eps, ub, v = _qline_states(n, seed, which=(0, 1), pol=pol)
        d = O.dressed_colour_sum(n, kin, eps, p[2], ub, p[3], v, par)
        o = O.ordered_colour_sum(n, kin, eps, p[2], ub, p[3], v, par)
        assert abs(d / o - 1) < 1e-12


# --------------------------------------------------------------------------
# Full ME: symmetries
# --------------------------------------------------------------------------

@pytest.mark.parametrize("n,nevt", [(2, 20), (3, 10), (4, 6), (5, 1)])
def test_bose_symmetry(n, nevt):
    proc = PROC_N[n]
    p = process_momenta(proc, SQRTS[n], nevt, 21)
    me = O.me(proc, p)
    # swap the two initial gluons
    q = p.copy()
    q[:, [0, 1]] = q[:, [1, 0]]
    np.testing.assert_allclose(O.me(proc, q), me, rtol=1e-12)
    if n >= 4:
        q = p.copy()
        q[:, [4, n + 1]] = q[:, [n + 1, 4]]
        np.testing.assert_allclose(O.me(proc, q), me, rtol=1e-12)


def _boost_rotate(p, beta, axis, angle):
    b = np.asarray(beta, dtype=float)
    b2 = b @ b
    gam = 1 / math.sqrt(1 - b2)
    L = np.eye(4)
    L[0, 0] = gam
    L[0, 1:] = L[1:, 0] = gam * b
    L[1:, 1:] += (gam - 1) * np.outer(b, b) / b2
    ax = np.asarray(axis, dtype=float) / np.linalg.norm(axis)
    K = np.array([[0, -ax[2], ax[1]], [ax[2], 0, -ax[0]], [-ax[1], ax[0], 0]])
    R = np.eye(4)
    R[1:, 1:] = np.eye(3) + math.sin(angle) * K + (1 - math.cos(angle)) * K @ K
    return p @ (L @ R).T


@pytest.mark.parametrize("n,nevt", [(2, 20), (3, 8), (4, 4), (5, 1)])
def test_lorentz_invariance(n, nevt):
    """Boost + rotation of every momentum leaves the spin/colour sum unchanged
    (Gamma_t = 0, so the amplitudes are gauge invariant)."""
    proc = PROC_N[n]
    par = O.Params(wt=0.0)
    p = process_momenta(proc, SQRTS[n], nevt, 31)
    me = O.me(proc, p, par)
    q = _boost_rotate(p, [0.3, -0.2, 0.5], [1, 2, 3], 0.7)
    np.testing.assert_allclose(O.me(proc, q, par), me, rtol=1e-11)


def test_eemumu_lorentz_invariance_with_z_width():
    p = process_momenta("e+ e- > mu+ mu-", 500.0, 20, 41)
    me = O.me("e+ e- > mu+ mu-", p)
    q = _boost_rotate(p, [0.1, 0.4, -0.3], [0, 1, 1], 1.1)
    np.testing.assert_allclose(O.me("e+ e- > mu+ mu-", q), me, rtol=1e-12)


# --------------------------------------------------------------------------
# u u~ -> t t~ g: five diagrams with explicit colour factors
# --------------------------------------------------------------------------

def test_uuttg_ward_identity():
    """eps(gluon) -> k(gluon) annihilates the colour-dressed amplitude of every
    colour assignment and spin state (Gamma_t = 0): fixes the relative signs
    and phases of the quark-line emissions and the three-gluon diagram."""
    par = O.Params(wt=0.0)
    p = process_momenta("u u~ > t t~ g", 1200.0, 3, 41)
    e = np.array([0.0, 0.6, 0.8, 0.0], dtype=complex)
    for ev in range(p.shape[0]):
        all_spins = [tuple((s >> (3 - i)) & 1 for i in range(4)) for s in range(16)]
        ref = max(np.abs(O.uuttg_amps(p[ev], sp, e, par)).max() for sp in all_spins)
        assert ref > 0
        for spins in all_spins:
            ward = np.abs(O.uuttg_amps(p[ev], spins, p[ev, 4].astype(complex), par)).max()
            assert ward <= 1e-12 * ref * p[ev, 4, 0]


def test_uuttg_width_breaks_ward_identity_only_slightly():
    p = process_momenta("u u~ > t t~ g", 1200.0, 1, 41)
    e = np.array([0.0, 0.6, 0.8, 0.0], dtype=complex)
    ref = np.abs(O.uuttg_amps(p[0], (0, 1, 0, 1), e)).max()
    ward = np.abs(O.uuttg_amps(p[0], (0, 1, 0, 1), p[0, 4].astype(complex))).max()
    assert 1e-9 * ref * p[0, 4, 0] < ward < 1e-1 * ref * p[0, 4, 0]


def test_uuttg_me_is_the_sum_of_the_dressed_amplitudes():
    p = process_momenta("u u~ > t t~ g", 1200.0, 2, 42)
    me = O.me("u u~ > t t~ g", p)
    for ev in range(2):
        tot = 0.0
        for s in range(16):
            spins = tuple((s >> (3 - i)) & 1 for i in range(4))
            for w in range(2):
                eps = O.polarisation(p[ev, 4], w).astype(complex)
                tot += np.sum(np.abs(O.uuttg_amps(p[ev], spins, eps)) ** 2)
        assert abs(tot / 36.0 / me[ev] - 1) < 1e-12


def test_uuttg_lorentz_invariance():
    par = O.Params(wt=0.0)
    p = process_momenta("u u~ > t t~ g", 1200.0, 20, 43)
    me = O.me("u u~ > t t~ g", p, par)
    q = _boost_rotate(p, [0.3, -0.2, 0.5], [1, 2, 3], 0.7)
    np.testing.assert_allclose(O.me("u u~ > t t~ g", q, par), me, rtol=1e-11)


# --------------------------------------------------------------------------
# Colour-flow weights sum_spins |A(sigma)|^2 (the colour-flow choice)
# --------------------------------------------------------------------------

def _relabelled(perms, a, b):
    """Index of each ordering with gluon labels a and b exchanged."""
    index = {tuple(int(x) for x in s): i for i, s in enumerate(perms)}
    swap = {a: b, b: a}
    return np.array([index[tuple(swap.get(int(x), int(x)) for x in s)] for s in perms])


@pytest.mark.parametrize("n,nevt", [(2, 10), (3, 6), (4, 3)])
def test_flow_weights_bose_relabelling(n, nevt):
    """Exchanging the momenta of two gluons maps the weight of each ordering
    onto the ordering with those two labels exchanged (a wrong index between
    orderings and flows fails this)."""
    proc = PROC_N[n]
    p = process_momenta(proc, SQRTS[n], nevt, 51)
    w = O.flow_weights(proc, p)
    perms = O.permutations(n)
    assert w.shape == (nevt, len(perms)) and np.all(w >= 0)
    slots = [0, 1] + list(range(4, n + 2))  # gluon label -> particle slot
    pairs = [(0, 1)] + ([(2, n - 1)] if n >= 4 else [])
    for a, b in pairs:
        q = p.copy()
        q[:, [slots[a], slots[b]]] = q[:, [slots[b], slots[a]]]
        np.testing.assert_allclose(O.flow_weights(proc, q), w[:, _relabelled(perms, a, b)], rtol=1e-11)


@pytest.mark.parametrize("n,nevt", [(2, 10), (3, 6), (4, 3)])
def test_flow_weights_lorentz_invariant(n, nevt):
    """Each ordering's spin-summed |A(sigma)|^2 is Lorentz invariant (Gamma_t = 0)."""
    proc = PROC_N[n]
    par = O.Params(wt=0.0)
    p = process_momenta(proc, SQRTS[n], nevt, 52)
    w = O.flow_weights(proc, p, par)
    q = _boost_rotate(p, [0.3, -0.2, 0.5], [1, 2, 3], 0.7)
    np.testing.assert_allclose(O.flow_weights(proc, q, par), w, rtol=1e-10, atol=1e-12 * w.max())


# --------------------------------------------------------------------------
# The full spin- and colour-summed ME and its normalisation
# --------------------------------------------------------------------------

def _helicity_spinors(p, m):
    """Massive Dirac-representation spinors in the helicity basis, built here
    from the eigenvectors of sigma.p_hat (a basis other than the oracle's
    spin-z one, with arbitrary phases): u = [sqrt(E+m) chi; s sqrt(E-m) chi],
    v = [s sqrt(E-m) eta; sqrt(E+m) eta], s = +-1 the helicity sign."""
    k = p[1:] / np.linalg.norm(p[1:])
    sp = np.array([[k[2], k[0] - 1j * k[1]], [k[0] + 1j * k[1], -k[2]]])
    val, vec = np.linalg.eigh(sp)
    a, b = math.sqrt(p[0] + m), math.sqrt(max(p[0] - m, 0.0))
    us, vs = [], []
    for j, phase in enumerate((np.exp(0.3j), np.exp(-1.1j))):
        chi = vec[:, j] * phase
        s = round(val[j])
        us.append(np.concatenate([a * chi, s * b * chi]))
        vs.append(np.concatenate([s * b * chi, a * chi]))
    return us, vs


def _circular_polarisations(p, outgoing):
    """eps+- = (e1 +- i e2)/sqrt(2) with e1 from a fixed oblique reference
    direction (not the oracle's coordinate-axis construction); conjugated for
    an outgoing gluon."""
    k = p[1:] / np.linalg.norm(p[1:])
    ref = np.array([0.36, -0.48, 0.8])
    e1 = np.cross(ref, k)
    e1 /= np.linalg.norm(e1)
    e2 = np.cross(k, e1)
    out = []
    for sgn in (1, -1):
        e = np.concatenate([[0.0], (e1 + sgn * 1j * e2) / math.sqrt(2)])
        out.append(e.conj() if outgoing else e)
    return out


def _final_gluon_symmetry(proc, p, n):
    """How many permutations of the final-state gluons' momenta leave |M|^2
    unchanged (Bose symmetry: all of them, for generic momenta).  The top and
    antitop are distinct particles and are not permuted (their exchange is a
    charge conjugation, which also leaves the summed |M|^2 unchanged)."""
    import itertools
    me0 = O.me(proc, p[None])[0]
    final = list(range(4, n + 2))
    count = 0
    for perm in itertools.permutations(final):
        q = p.copy()
        q[final] = p[list(perm)]
        if abs(O.me(proc, q[None])[0] / me0 - 1) < 1e-12:
            count += 1
    return count


@pytest.mark.parametrize("n,seed", [(3, 61), (4, 62), (5, 63)])
def test_spin_colour_summed_me_and_normalisation(n, seed):
    """The per-event ME (paper Sect. 1: the LO |M|^2 averaged over initial
    spins and colours) rebuilt outside mgo_me: every one of the 2^(n+2) spin
    states in a helicity basis built here (circular gluon polarisations, top
    helicity spinors), the colour sum by the colour-dressed recursion summed
    over every colour assignment (n <= 4; for n = 5, A^dagger C A, which that
    recursion pins at n <= 4), divided by 2*2 initial gluon polarisations,
    8*8 initial gluon colours and the final-state symmetry factor counted from
    Bose symmetry.  Catches a spin state dropped or counted twice and a wrong
    identical-particle factor in the oracle's helicity loop."""
    from concurrent.futures import ThreadPoolExecutor
    proc = PROC_N[n]
    par = O.Params()
    p = process_momenta(proc, SQRTS[n], 1, seed)[0]
    gam = O.gamma()
    us = _helicity_spinors(p[2], par.mt)[0]
    vs = _helicity_spinors(p[3], par.mt)[1]
    for s in range(2):  # valid, complete spinors of the oracle's representation
        ps_t, ps_tb = _slash(p[2]), _slash(p[3])
        np.testing.assert_allclose((ps_t - par.mt * np.eye(4)) @ us[s], 0, atol=1e-10 * p[2, 0])
        np.testing.assert_allclose((ps_tb + par.mt * np.eye(4)) @ vs[s], 0, atol=1e-10 * p[3, 0])
    ubars = [u.conj() @ gam[0] for u in us]
    np.testing.assert_allclose(sum(np.outer(us[s], ubars[s]) for s in range(2)),
                               _slash(p[2]) + par.mt * np.eye(4), atol=1e-11 * p[2, 0])
    slots = [0, 1] + list(range(4, n + 2))
    kin = np.array([p[s] if s < 2 else -p[s] for s in slots])
    pols = [_circular_polarisations(p[s], outgoing=s >= 2) for s in slots]
    summed = O.dressed_colour_sum if n <= 4 else O.ordered_colour_sum

    def one_state(h):
        eps = np.array([pols[i][(h >> i) & 1] for i in range(n)])
        st, stb = (h >> n) & 1, (h >> (n + 1)) & 1
        return summed(n, kin, eps, p[2], ubars[st], p[3], vs[stb], par)

    with ThreadPoolExecutor(8) as ex:
        total = sum(ex.map(one_state, range(1 << (n + 2))))
    sym = _final_gluon_symmetry(proc, p, n)
    assert sym == math.factorial(n - 2)  # identical final gluons only
    iden = 2 * 2 * O.generators().shape[0] ** 2 * sym
    assert iden == {3: 256, 4: 512, 5: 1536}[n]  # the normalisation of the matrix element definition
    assert abs(total / iden / O.me(proc, p[None])[0] - 1) < 1e-12


# --------------------------------------------------------------------------
# u u~ -> t t~ g g: colour-dressed recursion over both quark lines
# --------------------------------------------------------------------------

def test_two_line_recursion_reproduces_uutt_and_uuttg():
    """The same recursion with no gluon and with one gluon gives the
    independently pinned u u~ -> t t~ (analytic LO result) and u u~ -> t t~ g
    (five explicit diagrams, Ward identity) values: the quark lines, their
    propagators, the closing of the top line into a gluon and the three-gluon
    vertex on the s-channel gluon are those of the tested evaluations."""
    p0 = process_momenta("u u~ > t t~", 1000.0, 12, 71)
    np.testing.assert_allclose(O.uutt_ng(0, p0), O.me("u u~ > t t~", p0), rtol=1e-13)
    p1 = process_momenta("u u~ > t t~ g", 1200.0, 4, 72)
    np.testing.assert_allclose(O.uutt_ng(1, p1), O.me("u u~ > t t~ g", p1), rtol=1e-12)


@pytest.mark.parametrize("ev", [0, 1])
def test_uuttgg_ward_identity(ev):
    """eps_i -> k_i of either gluon annihilates the colour-dressed amplitude,
    summed over every colour and quark spin (Gamma_t = 0): fixes the
    four-gluon vertex and the two-gluon currents relative to the rest."""
    par = O.Params(wt=0.0)
    p = process_momenta("u u~ > t t~ g g", 1500.0, 2, 73)[ev]
    e5 = (O.polarisation(p[4], 0) + 0.3j * O.polarisation(p[4], 1)).astype(complex)
    e6 = (O.polarisation(p[5], 1) - 0.7j * O.polarisation(p[5], 0)).astype(complex)
    ref = O.uutt_ng_fixed_pol(2, p, [e5, e6], par)
    assert ref > 0
    w5 = O.uutt_ng_fixed_pol(2, p, [p[4].astype(complex), e6], par)
    w6 = O.uutt_ng_fixed_pol(2, p, [e5, p[5].astype(complex)], par)
    # |M|^2 is quadratic in the amplitude: 1e-11 of it at the amplitude level
    assert w5 <= 1e-22 * ref * p[4, 0] ** 2
    assert w6 <= 1e-22 * ref * p[5, 0] ** 2


def test_uuttgg_bose_symmetry_and_lorentz_invariance():
    par = O.Params(wt=0.0)
    p = process_momenta("u u~ > t t~ g g", 1500.0, 2, 74)
    me = O.me("u u~ > t t~ g g", p)
    q = p.copy()
    q[:, [4, 5]] = q[:, [5, 4]]
    np.testing.assert_allclose(O.me("u u~ > t t~ g g", q), me, rtol=1e-12)
    me0 = O.me("u u~ > t t~ g g", p, par)
    r = _boost_rotate(p, [0.3, -0.2, 0.5], [1, 2, 3], 0.7)
    np.testing.assert_allclose(O.me("u u~ > t t~ g g", r, par), me0, rtol=1e-11)


def test_uuttgg_gluon_spin_sum_and_normalisation():
    """The ME rebuilt from the fixed-polarisation hook: the gluon spins summed
    over circular polarisations built here (a basis other than the oracle's
    linear one), divided by 2*2 initial quark spins, 3*3 initial colours and
    the final-state symmetry factor counted from Bose symmetry (2 for two
    gluons): 72."""
    proc = "u u~ > t t~ g g"
    p = process_momenta(proc, 1500.0, 1, 75)[0]
    pols = [_circular_polarisations(p[s], outgoing=True) for s in (4, 5)]
    total = sum(O.uutt_ng_fixed_pol(2, p, [pols[0][a], pols[1][b]]) for a in range(2) for b in range(2))
    sym = _final_gluon_symmetry(proc, p, 4)
    assert sym == 2
    iden = 2 * 2 * 3 * 3 * sym
    assert iden == 72
    assert abs(total / iden / O.me(proc, p[None])[0] - 1) < 1e-12
