"""The generated per-process code, compiled for the host, against the oracle
(no GPU).

The kernels run the generator's straight-line code (per-event set-up, the
amplitudes of one helicity into the colour flows, the colour quadratic form)
written against the vertex routines of csrc/mg_vertices.cuh.  Compiled here
with g++ in FP64 (the CUDA qualifiers defined away), summed over every
helicity and normalised like the FP64 kernel, it must give the oracle's |M|^2
to 1e-12 per event; compiled with FP32 amplitudes (the mixed kernels' code
but for the tensor-core colour form), within the mixed bounds.  A regression
in the generator or the vertex routines thus fails on the CPU before any GPU
run.  This is a test harness only; the library never runs this code on the
host.
"""
import math
import os
import subprocess

import numpy as np
import pytest

import oracle as O
from paper_2303_18244_gb300.generator import emit
from paper_2303_18244_gb300.inputs import process_momenta

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2303_18244_gb300", "csrc")

PROGRAM = r"""
#include <cmath>
#include <cstdio>
#define __device__
#define __host__
#define __forceinline__ inline
#define __noinline__
#define __restrict__
template <typename T> inline T __ldg(const T* p) { return *p; }
#include "mg_vertices.cuh"
#include "TAG.cuh"
using namespace mg;
int main() {
  double kp[8];
  for (int i = 0; i < 8; i++)
    if (scanf("%lf", &kp[i]) != 1) return 1;
  int nevt;
  if (scanf("%d", &nevt) != 1) return 1;
  for (int e = 0; e < nevt; e++) {
    double p[TAG::NPAR * 4];
    for (int i = 0; i < TAG::NPAR * 4; i++)
      if (scanf("%lf", &p[i]) != 1) return 1;
    REAL slab[TAG::NSLOT];
    TAG::prepare<REAL, double>(p, kp, slab, 1);
    cx<REAL> jamp[TAG::NCOL];
    double acc = 0.0;
    for (int h = 0; h < TAG::NHEL; h++) {
      TAG::amplitudes<REAL>(slab, 1, h, kp, jamp, 1);
      acc += (double)TAG::colour_quadratic<REAL>(jamp, 1);
    }
    printf("%.17g\n", acc / (TAG::IDEN * TAG::CDEN));
  }
  return 0;
}
"""

# process -> (sqrt(s), events)
CASES = {
    "e+ e- > mu+ mu-": (500.0, 50),
    "g g > t t~": (1000.0, 50),
    "g g > t t~ g": (1200.0, 20),
    "g g > t t~ g g": (1500.0, 10),
    "g g > t t~ g g g": (2000.0, 2),
    "u u~ > t t~": (1000.0, 50),
    "u u~ > t t~ g": (1200.0, 20),
    "u u~ > t t~ g g": (1500.0, 6),
}


def _couplings(proc):
    """The kernels' parameter block for the default inputs: g_s, m_t, Gamma_t
    for QCD processes; e^2, (e / (s_W c_W))^2, g_L, g_R, M_Z, Gamma_Z for
    e+e- -> mu+mu- (G_F scheme)."""
    par = O.Params()
    if proc == "e+ e- > mu+ mu-":
        alpha = 1.0 / par.alpha_em_inv
        e2 = 4.0 * math.pi * alpha
        mz2 = par.mz ** 2
        mw2 = 0.5 * mz2 + math.sqrt(0.25 * mz2 * mz2 - math.pi * alpha * mz2 / (math.sqrt(2.0) * par.gf))
        sw2 = 1.0 - mw2 / mz2
        return [e2, e2 / (sw2 * (1.0 - sw2)), -0.5 + sw2, sw2, par.mz, par.wz, 0.0, 0.0]
    return [math.sqrt(4.0 * math.pi * par.alpha_s), par.mt, par.wt, 0.0, 0.0, 0.0, 0.0, 0.0]


def host_me(proc, real, workdir, header=None, vertices=None):
    """(momenta, |M|^2) of the generated code of proc compiled for the host
    in workdir; header / vertices replace the generated header or the text of
    mg_vertices.cuh (a copy in workdir is found before the original)."""
    tag, generated = emit.emit(proc, "f32" if real == "float" else "f64")
    (workdir / f"{tag}.cuh").write_text(generated if header is None else header)
    if vertices is not None:
        (workdir / "mg_vertices.cuh").write_text(vertices)
    src = workdir / "main.cpp"
    src.write_text(PROGRAM.replace("TAG", tag))
    exe = workdir / "main"
    subprocess.run(["g++", "-O0", "-std=c++17", f"-DREAL={real}", f"-I{workdir}", f"-I{CSRC}", "-o", str(exe),
                    str(src)], check=True)
    sqrts, n = CASES[proc]
    p = process_momenta(proc, sqrts, n, 91)
    lines = [" ".join(repr(float(x)) for x in _couplings(proc)), str(n)]
    lines += [" ".join(repr(float(x)) for x in ev.ravel()) for ev in p]
    out = subprocess.run([str(exe)], input="\n".join(lines) + "\n", capture_output=True, text=True, check=True)
    return p, np.array([float(x) for x in out.stdout.split()])


@pytest.mark.parametrize("real", ["double", "float"], ids=["fp64", "fp32"])
@pytest.mark.parametrize("proc", list(CASES), ids=lambda p: emit.PROCESSES[p][0])
def test_generated_code_on_the_host_matches_the_oracle(proc, real, tmp_path):
    """FP64: within 1e-12 per event.  FP32 amplitudes with the FP64 set-up
    and helicity sum (what the mixed kernels run, with the colour form on
    CUDA cores in place of the tensor cores): the mixed bounds of the GPU
    parity tests."""
    p, got = host_me(proc, real, tmp_path)
    n = CASES[proc][1]
    assert got.shape == (n,) and np.all(np.isfinite(got))
    ref = O.me(proc, p)
    r = np.abs(got - ref) / np.abs(ref)
    if real == "float":
        assert np.median(r) <= 1e-5 and r.max() <= 1e-2
        return
    bad = np.nonzero(r > 1e-12)[0]
    if bad.size:  # the long-double oracle decides, as for the GPU's FP64 path
        ext = O.me(proc, p[bad], extended=True)
        assert np.max(np.abs(got[bad] - ext) / np.abs(ext)) <= 1e-12


def test_shared_current_chunk_order(tmp_path, monkeypatch):
    """gg -> t t~ g g g: the FP32 header orders its chunks by shared currents
    (a store of 87 crossing currents instead of the FP64 header's 241, its
    struct in an inline namespace of its own), with the same |M|^2 (compiled
    in FP64 here: within 1e-12 of the oracle)."""
    import re
    monkeypatch.delenv("MG_CHUNK_ORDER", raising=False)
    proc = "g g > t t~ g g g"
    assert emit.header_name(proc, "f64") == "ggttggg.cuh" and emit.header_name(proc, "f32") == "ggttggg_f32.cuh"
    _, default = emit.emit(proc, "f64")
    _, shared = emit.emit(proc, "f32")
    store = [int(re.search(r"NSTORE = (\d+)", src).group(1)) for src in (default, shared)]
    assert store == [241, 87]
    assert "inline namespace chunk_order_shared {" in shared and "inline namespace" not in default
    p, got = host_me(proc, "double", tmp_path, header=shared)
    ref = O.me(proc, p)
    assert np.max(np.abs(got - ref) / np.abs(ref)) <= 1e-12
