"""The parity comparison catches plausible mistakes in the CUDA-side code
(no GPU).

Each case plants one typical mistake into a copy of the vertex routines or of
a generated header (a flipped sign, a wrong momentum order, a wrong colour
coefficient or colour-form entry), compiles the process for the host as in
test_generated_code_host.py, and checks that its |M|^2 leaves the oracle by
far more than the 1e-12 the FP64 parity tests allow.  The sources in the
repository are never modified.
"""
import os

import numpy as np
import pytest

import oracle as O
from test_generated_code_host import CSRC, host_me
from paper_2303_18244_gb300.generator import emit

# (what is wrong, process, "vertices" or "header", text, planted text)
MUTANTS = [
    ("three-gluon current: momentum difference reversed", "g g > t t~ g", "vertices",
     "cx<R> t = (kx[mu] - ky[mu]) * xy;", "cx<R> t = (ky[mu] - kx[mu]) * xy;"),
    ("four-gluon amplitude: relative sign of its two terms", "g g > t t~ g g", "vertices",
     "if (BR == 0) t = dot(X, Z) * dot(Y, G) - dot(Y, Z) * dot(X, G);",
     "if (BR == 0) t = dot(X, Z) * dot(Y, G) + dot(Y, Z) * dot(X, G);"),
    ("top row current: mass term sign in one component", "g g > t t~ g", "vertices",
     "  o.c[0] = coef * fma(m, rL0, s0);", "  o.c[0] = coef * fma(-m, rL0, s0);"),
    ("fermion vector current: sign of one component", "e+ e- > mu+ mu-", "vertices",
     "g.c[2] = cR * mul_i(u12 - u03) + cL * mul_i(l21 - l30);",
     "g.c[2] = cR * mul_i(u03 - u12) + cL * mul_i(l21 - l30);"),
    ("colour flow: one amplitude added with the wrong sign", "g g > t t~ g", "header",
     "JAMP(0) = JAMP(0) + a;", "JAMP(0) = JAMP(0) - a;"),
    ("colour form: one off-diagonal numerator off by one", "g g > t t~ g", "header",
     "yr = fmaf_t<R>(R(20), JAMP(5).re, yr);", "yr = fmaf_t<R>(R(19), JAMP(5).re, yr);"),
]


@pytest.mark.parametrize("what,proc,where,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_parity_catches_planted_mistake(what, proc, where, old, new, tmp_path):
    if where == "vertices":
        with open(os.path.join(CSRC, "mg_vertices.cuh")) as f:
            src = f.read()
        assert src.count(old) == 1, old
        p, got = host_me(proc, "double", tmp_path, vertices=src.replace(old, new))
    else:
        _, src = emit.emit(proc)
        assert src.count(old) >= 1, old
        p, got = host_me(proc, "double", tmp_path, header=src.replace(old, new, 1))
    ref = O.me(proc, p)
    r = np.abs(got - ref) / np.abs(ref)
    assert not np.all(r <= 1e-12)  # the FP64 parity bar fails
    assert np.max(r) > 1e-6
