"""The unweighting kernels' build-time variants compile for sm_103a (no GPU):
the default, the FP64 decision for every event, other events-per-thread
counts, and the count pass with TMA-staged tiles.  Each was measured on a
GB300 against the default; this keeps the measured alternatives buildable."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2303_18244_gb300", "csrc")


@pytest.mark.parametrize("flags", [[], ["-DMG_UW_FP32_FIRST=0"], ["-DMG_UW_PER_THREAD=4"],
                                   ["-DMG_UW_PER_THREAD=32"], ["-DMG_UW_TMA=1"]],
                         ids=["default", "fp64-decision", "4-per-thread", "32-per-thread", "tma"])
def test_unweight_variant_compiles(flags, tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not found")
    r = subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17",
                        "--expt-relaxed-constexpr", f"-I{os.path.join(ROOT, 'include')}", f"-I{CSRC}", *flags,
                        "-c", os.path.join(CSRC, "mg_unweight.cu"), "-o", str(tmp_path / "uw.o")],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-2000:]
