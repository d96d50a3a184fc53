"""Build libmg.so: run the generator, compile every translation unit with nvcc
for sm_103a in parallel, link one shared library (in-tree, _build/)."""
from __future__ import annotations

import hashlib
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
GEN = os.path.join(CSRC, "gen")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libmg.so")
INCLUDE = os.path.join(ROOT, "include")

NVCC = os.environ.get("NVCC", shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
         "--expt-relaxed-constexpr", f"-I{INCLUDE}", f"-I{CSRC}"]

# extra nvcc flags (e.g. -DMG_TC_MINB=3 for a launch-shape sweep)
FLAGS += os.environ.get("MG_NVCC_EXTRA", "").split()

HAND = ["mg_runtime.cu", "mg_server.cu", "mg_diag.cu", "mg_static.cu", "mg_phasespace.cu", "mg_unweight.cu"]


def _write_if_changed(path: str, text: str) -> None:
    if os.path.exists(path):
        with open(path) as f:
            if f.read() == text:
                return
    tmp = path + f".{os.getpid()}.tmp"
    with open(tmp, "w") as f:
        f.write(text)
    os.replace(tmp, path)


def processes() -> list[str]:
    """Process strings to build (MG_PROCESSES: comma-separated tags to restrict)."""
    sys.path.insert(0, ROOT)
    from paper_2303_18244_gb300.generator.emit import PROCESSES
    only = os.environ.get("MG_PROCESSES")
    if not only:
        return list(PROCESSES)
    tags = set(only.split(","))
    return [p for p, (t, _) in PROCESSES.items() if t in tags]


def generate() -> list[str]:
    """Write csrc/gen/<tag>.cuh, <tag>_f64.cu, <tag>_f32.cu and registry.cu; return the TUs."""
    sys.path.insert(0, ROOT)
    from paper_2303_18244_gb300.generator.emit import PROCESSES, emit, emit_tu, header_name
    os.makedirs(GEN, exist_ok=True)
    tus = []
    procs = processes()
    tags = [PROCESSES[p][0] for p in procs]
    reg = ['// generated: registry of the compiled processes', '#include "../mg_kernels.cuh"', "namespace mg {"]
    reg += [f"const ProcDesc* proc_{t}();" for t in tags]
    reg += ["const ProcDesc* const* registry(int* n) {",
            f"  static const ProcDesc* all[] = {{{', '.join(f'proc_{t}()' for t in tags)}}};",
            f"  *n = {len(tags)};", "  return all;", "}", "}  // namespace mg", ""]
    path = os.path.join(GEN, "registry.cu")
    _write_if_changed(path, "\n".join(reg))
    tus.append(path)
    for proc in procs:
        for prec in ("f64", "f32"):
            name = header_name(proc, prec)
            if prec == "f64" or name != header_name(proc, "f64"):
                tag, hdr = emit(proc, prec)
                _write_if_changed(os.path.join(GEN, name), hdr)
        for prec in ("f64", "f32"):
            _, tu = emit_tu(proc, prec)
            path = os.path.join(GEN, f"{tag}_{prec}.cu")
            _write_if_changed(path, tu)
            tus.append(path)
    return tus


def _deps_hash(src: str) -> str:
    h = hashlib.sha256()
    for p in [src] + sorted(
            os.path.join(d, f) for d in (CSRC, GEN, INCLUDE) for f in os.listdir(d)
            if f.endswith((".cuh", ".h"))):
        with open(p, "rb") as f:
            h.update(f.read())
    h.update(" ".join([NVCC] + ARCH + FLAGS).encode())
    return h.hexdigest()


def _compile(src: str) -> str:
    obj = os.path.join(BUILD, os.path.basename(src).replace(".cu", ".o"))
    stamp = obj + ".hash"
    digest = _deps_hash(src)
    if os.path.exists(obj) and os.path.exists(stamp) and open(stamp).read() == digest:
        return obj
    cmd = [NVCC] + ARCH + FLAGS + ["-c", src, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stderr[-4000:]}")
    with open(stamp, "w") as f:
        f.write(digest)
    return obj


def build(verbose: bool = True) -> str:
    os.makedirs(BUILD, exist_ok=True)
    tus = generate() + [os.path.join(CSRC, f) for f in HAND]
    # largest units first so that they start early
    def weight(p):
        for suf in ("_f64.cu", "_f32.cu"):
            if p.endswith(suf):
                return -os.path.getsize(p.replace(suf, ".cuh"))
        return 0
    tus.sort(key=weight)
    jobs = max(1, min(len(tus), os.cpu_count() or 1))
    with ThreadPoolExecutor(jobs) as ex:
        objs = list(ex.map(_compile, tus))  # only the objects of these sources are linked
    tmp = LIB + f".{os.getpid()}.tmp"
    cmd = [NVCC] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart_static", "-lrt", "-lpthread", "-ldl"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr[-4000:]}")
    os.replace(tmp, LIB)
    if verbose:
        print(f"built {LIB}")
    return LIB


if __name__ == "__main__":
    build()
