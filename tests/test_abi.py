"""The C-ABI library loads and exports every function declared in include/*.h
(no compute call is made: this runs without a GPU)."""
import ctypes
import glob
import os
import re
import subprocess

import pytest

from paper_2303_18244_gb300 import mg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(mg_\w+)\s*\(", src, flags=re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def libmg():
    if not os.path.exists(mg.LIB_PATH):
        from paper_2303_18244_gb300 import build as B
        B.build(verbose=False)
    return mg.lib()


def test_headers_declare_the_boundary():
    names = declared_functions()
    for n in ("mg_process_create", "mg_good_helicities", "mg_sigma", "mg_server_submit", "mg_server_poll"):
        assert n in names


def test_every_declared_symbol_is_exported(libmg):
    names = declared_functions()
    missing = [n for n in sorted(names) if not hasattr(libmg, n)]
    assert not missing, f"declared but not exported: {missing}"
    # and the Python binding marshals each of them
    assert set(mg.EXPORTS) == names


def test_exported_symbols_are_c_linkage(libmg):
    out = subprocess.run(["nm", "-D", "--defined-only", mg.LIB_PATH], capture_output=True, text=True).stdout
    exported = {ln.split()[-1] for ln in out.splitlines() if " T " in ln}
    for n in declared_functions():
        assert n in exported, n


def test_host_only_calls(libmg):
    # calls that touch no device: defaults, error strings, argument checks
    p = mg.mg_params()
    assert libmg.mg_params_default(ctypes.byref(p)) == 0
    assert p.mt == 173.0 and p.alpha_s == 0.118 and p.precision == 0
    c = mg.mg_server_cfg()
    assert libmg.mg_server_cfg_default(ctypes.byref(c)) == 0
    assert c.n_streams == 4 and c.max_bucket == 65536
    assert mg.strerror(-1) == "unknown process"
    assert libmg.mg_params_default(None) == -2
    h = ctypes.c_void_p()
    assert libmg.mg_process_create(b"g g > t t~", None, ctypes.byref(h)) == -2
    assert libmg.mg_process_info(None, None, None, None, None, None) == -2


def test_no_cpu_fallback_without_a_gpu(libmg):
    """The product path has no CPU fallback: without a CUDA device a process
    handle cannot be created (a CUDA error, not a silent CPU result), and the
    binding refuses host tensors where device buffers are required."""
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("checks the behaviour on a machine without a GPU")
    with pytest.raises(mg.MGError) as ei:
        mg.Process("g g > t t~")
    assert ei.value.code in (-3, -4)  # MG_ERR_NOMEM / MG_ERR_CUDA
    with pytest.raises(TypeError):
        mg._dev_check(torch.zeros((8, 4, 4), dtype=torch.float64))
