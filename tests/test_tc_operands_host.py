"""Host-side construction of the tensor-core colour operands (no GPU).

The mixed path contracts the colour flows with the colour-matrix numerators
KNUM on the tensor cores (kind::f16).  The numerators go in as an FP16 B tile
built on the host by colour_tile_host, in the K-major no-swizzle layout the
shared-memory descriptors describe: element (row r, column k) at byte
(r / 8) * SBO + (k / 8) * LBO + (r % 8) * 16 + (k % 8) * 2, LBO = 128 bytes,
SBO = (K / 8) * 128 bytes.  Compiled with nvcc into a host-only program (it
runs without a GPU), the encoding is checked against numpy's IEEE binary16
and the layout against that formula, for every numerator of the processes
whose mixed path uses the tensor cores.
"""
import os
import shutil
import subprocess

import numpy as np
import pytest

from paper_2303_18244_gb300.generator import emit

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2303_18244_gb300", "csrc")

PROGRAM = r"""
#include <cstdio>
#include <vector>
#include "mg_colour_tc.cuh"
int main() {
  int lo, hi;
  if (scanf("%d %d", &lo, &hi) != 2) return 1;
  for (int v = lo; v <= hi; v++) printf("%d\n", mg::fp16_bits_of_int(v));
  int ncol;
  while (scanf("%d", &ncol) == 1) {
    std::vector<int> knum((size_t)ncol * ncol);
    for (auto& x : knum)
      if (scanf("%d", &x) != 1) return 1;
    const int K = mg::tc::pad16(ncol);
    std::vector<unsigned short> tile((size_t)K * K);
    printf("ok %d\n", mg::colour_tile_host(knum.data(), ncol, tile.data()) ? 1 : 0);
    for (auto x : tile) printf("%u\n", (unsigned)x);
  }
  return 0;
}
"""


@pytest.fixture(scope="module")
def program(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not found")
    d = tmp_path_factory.mktemp("tc")
    (d / "t.cu").write_text(PROGRAM)
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-std=c++17", "--expt-relaxed-constexpr",
                    f"-I{os.path.join(ROOT, 'include')}", f"-I{CSRC}", "-o", str(d / "t"), str(d / "t.cu")],
                   check=True)
    return d / "t"


def _knum(proc):
    _, src = emit.emit(proc)
    i = src.index("KNUM[NCOL * NCOL] = {") + len("KNUM[NCOL * NCOL] = {")
    vals = [int(x) for x in src[i:src.index("}", i)].split(",")]
    n = int(round(len(vals) ** 0.5))
    assert n * n == len(vals)
    return n, vals


def _fp16_bits(v):
    """binary16 bits of the integer v, or -1 if v is not exact in binary16."""
    with np.errstate(over="ignore"):
        h = np.float16(v)
    if not np.isfinite(h) or float(h) != v:
        return -1
    return int(np.array(h).view(np.uint16))


def test_fp16_encoding_of_integers(program):
    lo, hi = -70000, 70000
    out = subprocess.run([str(program)], input=f"{lo} {hi}\n", capture_output=True, text=True, check=True)
    got = [int(x) for x in out.stdout.split()]
    want = [_fp16_bits(v) for v in range(lo, hi + 1)]
    assert got == want


@pytest.mark.parametrize("proc", ["g g > t t~ g", "g g > t t~ g g", "g g > t t~ g g g"])
def test_colour_tile_layout(program, proc):
    n, knum = _knum(proc)
    out = subprocess.run([str(program)], input=f"1 0\n{n} " + " ".join(map(str, knum)) + "\n",
                         capture_output=True, text=True, check=True).stdout.split()
    assert out[:2] == ["ok", "1"]  # every numerator is exact in FP16
    K = ((n + 15) // 16) * 16
    tile = np.array([int(x) for x in out[2:]], dtype=np.int64)
    assert tile.size == K * K
    want = np.zeros(K * K, dtype=np.int64)
    for r in range(n):          # B-operand row = output column n of D
        for k in range(n):
            byte = (r // 8) * (K // 8) * 128 + (k // 8) * 128 + (r % 8) * 16 + (k % 8) * 2
            want[byte // 2] = _fp16_bits(knum[r * n + k])
    np.testing.assert_array_equal(tile, want)
