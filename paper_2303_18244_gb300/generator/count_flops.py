"""Algorithmic FLOP counts of the generated per-helicity code.

Compiles the generated process code for the host with a real type that counts
every add, subtract and multiply as written (an FMA is counted as its multiply
plus its add), runs one helicity of one event, and writes
paper_2303_18244_gb300/flops.json:

  {tag: {"amp_flops_per_hel": ..., "colour_flops_per_hel": ...,
         "colour_dense_flops_per_hel": 4 * ncol^2, "nhel": ..., "ncol": ...}}

The counts are those of the source as generated (before any compiler
simplification), i.e. the algorithmic work of steps A2-A5 per helicity.
Run: python -m paper_2303_18244_gb300.generator.count_flops
"""
from __future__ import annotations

import json
import os
import subprocess
import sys
import tempfile

HERE = os.path.dirname(os.path.abspath(__file__))
PKG = os.path.dirname(HERE)
CSRC = os.path.join(PKG, "csrc")
OUT = os.path.join(PKG, "flops.json")

PROGRAM = r"""
#include <cmath>
#include <cstdio>
#define __device__
#define __host__
#define __forceinline__ inline
#define __noinline__
#define __restrict__
struct int4 { int x, y, z, w; };
template <typename T> inline T __ldg(const T* p) { return *p; }
static long long n_add = 0, n_mul = 0;
struct Cnt {
  double v;
  Cnt() : v(0) {}
  Cnt(double x) : v(x) {}
};
inline Cnt operator+(Cnt a, Cnt b) { n_add++; return Cnt(a.v + b.v); }
inline Cnt operator-(Cnt a, Cnt b) { n_add++; return Cnt(a.v - b.v); }
inline Cnt operator*(Cnt a, Cnt b) { n_mul++; return Cnt(a.v * b.v); }
inline Cnt operator-(Cnt a) { return Cnt(-a.v); }
inline bool operator>(Cnt a, Cnt b) { return a.v > b.v; }
inline Cnt operator+(Cnt a, double b) { return a + Cnt(b); }
#include "mg_vertices.cuh"
#include "gen/TAG.cuh"
using namespace mg;
int main() {
  Cnt ev[TAG::NSLOT];
  for (int k = 0; k < TAG::NSLOT; k++) ev[k] = Cnt(0.1 + 0.01 * k);
  double kp[8] = {1.2, 173.0, 1.5, 0.5, 0.2, 0.3, 91.0, 2.4};
  cx<Cnt> jamp[TAG::NCOL];
  n_add = n_mul = 0;
  TAG::amplitudes<Cnt>(ev, 1, 5, kp, jamp, 1);
  long long amp = n_add + n_mul;
  n_add = n_mul = 0;
  volatile double s = TAG::colour_quadratic<Cnt>(jamp, 1).v;
  (void)s;
  long long col = n_add + n_mul;
  printf("%lld %lld %d %d\n", amp, col, TAG::NHEL, TAG::NCOL);
  return 0;
}
"""


def count(tag: str) -> dict:
    with tempfile.TemporaryDirectory() as d:
        src = os.path.join(d, "c.cpp")
        exe = os.path.join(d, "c")
        with open(src, "w") as f:
            f.write(PROGRAM.replace("TAG", tag))
        subprocess.run(["g++", "-O0", "-std=c++17", f"-I{CSRC}", "-o", exe, src], check=True)
        out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout.split()
    amp, col, nhel, ncol = (int(x) for x in out)
    return {"amp_flops_per_hel": amp, "colour_flops_per_hel": col,
            "colour_dense_flops_per_hel": 4 * ncol * ncol, "nhel": nhel, "ncol": ncol}


def main(tags=None):
    sys.path.insert(0, os.path.dirname(PKG))
    from paper_2303_18244_gb300 import build as B
    B.generate()
    from paper_2303_18244_gb300.generator.emit import PROCESSES
    tags = tags or [t for t, _ in PROCESSES.values()]
    res = {}
    if os.path.exists(OUT):
        with open(OUT) as f:
            res = json.load(f)
    for t in tags:
        res[t] = count(t)
        print(t, res[t])
    with open(OUT, "w") as f:
        json.dump(res, f, indent=1, sort_keys=True)


if __name__ == "__main__":
    main(sys.argv[1:] or None)
