"""The pins catch plausible mistakes in the oracle (no GPU).

Each case plants one typical mistake (a flipped sign, a transposed operand, a
dropped conjugate, a wrong factor or index) into a temporary copy of
oracle/mg_oracle.c, builds that copy with the oracle's own flags, points the
oracle binding at it, and checks that the pin named beside it fails, after
checking that the same pin passes on the real oracle.  The oracle's source
is never modified.
"""
import ctypes
import subprocess

import pytest

import oracle as O
import test_colour_pins as CP
import test_oracle_pins as P

# (what is wrong, text in mg_oracle.c, planted text, the pin that must fail)
MUTANTS = [
    ("four-gluon contact term with the wrong sign",
     "acc[mu] += q->g * q->g * t[mu];", "acc[mu] -= q->g * q->g * t[mu];",
     lambda: P.test_ward_identity_every_ordering(4, 7)),
    ("quartic terms of the longest range dropped",
     "for (int m2 = m1 + 1; m2 < j; m2++) {", "for (int m2 = m1 + 1; m2 < j - 1; m2++) {",
     lambda: P.test_ward_identity_every_ordering(4, 8)),
    ("three-gluon vertex with its legs' momenta exchanged",
     "out[mu] = jab * (ka[mu] - kb[mu]) + jb[mu] * xa - ja[mu] * yb;",
     "out[mu] = jab * (kb[mu] - ka[mu]) + jb[mu] * xa - ja[mu] * yb;",
     lambda: P.test_ggtt_matches_analytic(173.0)),
    ("top propagator numerator p-slash - m instead of + m",
     "for (int c = 0; c < 4; c++) P[c][c] += q->mt;", "for (int c = 0; c < 4; c++) P[c][c] -= q->mt;",
     lambda: P.test_ggtt_matches_analytic(173.0)),
    ("last quark-gluon vertex off by sqrt(2)",
     "amp += (I * q->g) * rowcol(Psi[m], t);", "amp += (I * q->g) * sqrt(2.0) * rowcol(Psi[m], t);",
     lambda: P.test_ggtt_matches_analytic(173.0)),
    ("colour matrix without the complex conjugate",
     "sum += W[s][i][j] * conj(W[t][i][j]);", "sum += W[s][i][j] * W[t][i][j];",
     CP.test_oracle_three_gluon_matrix_closed_form),
    ("left-handed Z coupling with the wrong sign of T3",
     "const real gl = -0.5 + sw2, gr = sw2;", "const real gl = 0.5 + sw2, gr = sw2;",
     P.test_eemumu_gamma_z_helicity_closed_form),
    ("v spinor with a sign flipped in its lower components",
     "v[2] = a * eta[0];", "v[2] = -a * eta[0];",
     lambda: P.test_spinor_completeness_and_dirac_equation(173.0)),
    ("polarisation vector with a time component",
     "eps[0] = 0.0;", "eps[0] = 0.1;",
     P.test_polarisation_transverse_complete),
    ("u u~ -> t t~ without the spin average",
     "return sum * colour / 36.0;", "return sum * colour / 9.0;",
     lambda: P.test_uutt_matches_analytic(173.0)),
    ("u u~ -> t t~ g: emission at the u~ end with the wrong sign",
     "A[1] = dot_cc(L2, H) * (-I / q2);", "A[1] = -dot_cc(L2, H) * (-I / q2);",
     P.test_uuttg_ward_identity),
    ("u u~ -> t t~ g: three-gluon vertex momentum term reversed",
     "y[mu] = p5[mu] - q34[mu];", "y[mu] = q34[mu] - p5[mu];",
     P.test_uuttg_ward_identity),
    ("identical-particle factor loop off by one",
     "for (int i = 2; i <= n - 2; i++) iden *= i;", "for (int i = 2; i <= n - 1; i++) iden *= i;",
     lambda: P.test_spin_colour_summed_me_and_normalisation(3, 61)),
    ("top and antitop spin states read from the same helicity bit",
     "const int st = (h >> n) & 1, stb = (h >> (n + 1)) & 1;", "const int st = (h >> n) & 1, stb = (h >> n) & 1;",
     lambda: P.test_spin_colour_summed_me_and_normalisation(3, 61)),
    ("a gluon's polarisation state read from its neighbour's helicity bit",
     "q.eps[i][mu] = pol[i][(h >> i) & 1][mu];", "q.eps[i][mu] = pol[i][(h >> (i + 1)) & 1][mu];",
     lambda: P.test_spin_colour_summed_me_and_normalisation(3, 61)),
    ("two-line recursion: four-gluon term with the wrong sign",
     "acc[c][x][mu] += -g * g * lor; /* (-i/P^2) (-i g^2) */", "acc[c][x][mu] += g * g * lor;",
     lambda: P.test_uuttgg_ward_identity(0)),
    ("two-line recursion: light-quark propagator with the attached momenta reversed",
     "Q[mu] = (kind == 4) ? (kend[mu] + attached) : (-kend[mu] - attached);",
     "Q[mu] = (kind == 4) ? (kend[mu] + attached) : (-kend[mu] + attached);",
     P.test_two_line_recursion_reproduces_uutt_and_uuttg),
    ("two-line recursion: top line closed with the colour generator transposed",
     "if (tc != 0) acc[c][x][mu] += g * tc * rv; /* (-i/P^2) (i g) */",
     "if (tc != 0) acc[c][x][mu] += g * TGEN[c][n][m] * rv;",
     P.test_two_line_recursion_reproduces_uutt_and_uuttg),
]


@pytest.mark.parametrize("what,old,new,pin", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pin_catches_planted_mistake(what, old, new, pin, tmp_path, monkeypatch):
    with open(O._SRC) as f:
        src = f.read()
    assert src.count(old) == 1, f"the text to replace must occur once: {old}"
    pin()  # holds on the real oracle
    c = tmp_path / "mutant.c"
    c.write_text(src.replace(old, new))
    so = tmp_path / "libmutant.so"
    subprocess.run(["gcc", *O.CFLAGS, "-o", str(so), str(c), "-lm", "-lpthread"], check=True)
    monkeypatch.setattr(O, "_lib", O._declare(ctypes.CDLL(str(so))))
    with pytest.raises(AssertionError):
        pin()
