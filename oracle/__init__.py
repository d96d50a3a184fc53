"""FP64 CPU oracle for the per-event LO |M|^2 (ctypes binding of mg_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by tests/, __graft_entry__.smoke() and the
CPU legs of bench.py, never by the product path.  It shares no code with the
CUDA path; the only thing both sides consume in common is the momenta made by
paper_2303_18244_gb300.inputs.

Every function cites the passage it restates in mg_oracle.c; the physics
inputs below are this oracle's own copy of the workload parameters.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass, astuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mg_oracle.c")
_LIBDIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_LIBDIR, "libmgoracle.so")
_LIB_EXT = os.path.join(_LIBDIR, "libmgoracle_ext.so")

PROCS = {
    "e+ e- > mu+ mu-": 0,
    "g g > t t~": 1,
    "g g > t t~ g": 2,
    "g g > t t~ g g": 3,
    "g g > t t~ g g g": 4,
    "u u~ > t t~": 5,
    "u u~ > t t~ g": 6,
    "u u~ > t t~ g g": 7,
}


@dataclass
class Params:
    """Physics inputs: top mass/width, fixed alpha_s, EW inputs (G_F scheme)."""
    mt: float = 173.0
    wt: float = 1.4915
    alpha_s: float = 0.118
    mz: float = 91.188
    wz: float = 2.441404
    alpha_em_inv: float = 132.507
    gf: float = 1.16639e-5
    photon_only: float = 0.0

    def array(self) -> np.ndarray:
        return np.array(astuple(self), dtype=np.float64)


# plain C11; no contraction into FMAs, so that every product and sum is
# rounded as written
CFLAGS = ["-std=gnu11", "-O2", "-fPIC", "-shared", "-fcx-limited-range", "-ffp-contract=off"]


def build(force: bool = False) -> str:
    """Compile mg_oracle.c with gcc (plain C11): the FP64 oracle and its
    extended-precision twin (same source, long double arithmetic)."""
    os.makedirs(_LIBDIR, exist_ok=True)
    for lib_path, extra in ((_LIB, []), (_LIB_EXT, ["-DORACLE_REAL=long double"])):
        if (not force and os.path.exists(lib_path)
                and os.path.getmtime(lib_path) >= os.path.getmtime(_SRC)):
            continue
        tmp = lib_path + f".{os.getpid()}.tmp"
        cmd = ["gcc", *CFLAGS, *extra, "-o", tmp, _SRC, "-lm", "-lpthread"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, lib_path)
    return _LIB


_lib = None
_lib_ext = None
_lib_lock = threading.Lock()

_D = ctypes.POINTER(ctypes.c_double)
_I = ctypes.POINTER(ctypes.c_int)


def _declare(L):
    L.mgo_me.argtypes = [ctypes.c_int, _D, _D, ctypes.c_int64, _D]
    for name in ("mgo_ordered_amps", "mgo_ordered_colour_sum", "mgo_dressed_colour_sum"):
        getattr(L, name).argtypes = [ctypes.c_int, _D, _D, _D, _D, _D, _D, _D, _D]
    L.mgo_colour_matrix.argtypes = [ctypes.c_int, _D]
    L.mgo_permutations.argtypes = [ctypes.c_int, _I]
    L.mgo_generators.argtypes = [_D]
    L.mgo_fabc.argtypes = [_D]
    L.mgo_spinor.argtypes = [ctypes.c_int, _D, ctypes.c_double, ctypes.c_int, _D]
    L.mgo_polarisation.argtypes = [_D, ctypes.c_int, _D]
    L.mgo_gamma.argtypes = [_D]
    L.mgo_npar.argtypes = [ctypes.c_int]
    L.mgo_flow_weights.argtypes = [ctypes.c_int, _D, _D, ctypes.c_int64, _D]
    L.mgo_uuttg_amps.argtypes = [_D, _D, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, _D, _D]
    L.mgo_uutt_ng.argtypes = [ctypes.c_int, _D, _D, ctypes.c_int64, _D]
    L.mgo_uutt_ng_fixed_pol.argtypes = [ctypes.c_int, _D, _D, _D, _D]
    return L


def lib_ext():
    """The extended-precision (long double) build of the same oracle source."""
    global _lib_ext
    with _lib_lock:
        if _lib_ext is None:
            build()
            _lib_ext = _declare(ctypes.CDLL(_LIB_EXT))
    return _lib_ext


def lib():
    global _lib
    with _lib_lock:
        if _lib is None:
            _lib = _declare(ctypes.CDLL(build()))
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(_D)


def _check(rc: int):
    if rc != 0:
        raise RuntimeError(f"oracle call failed with code {rc}")


def me(proc: str, momenta: np.ndarray, params: Params | None = None,
       threads: int | None = None, extended: bool = False) -> np.ndarray:
    """Per-event ME (mg_oracle.c: mgo_me), events split over host threads.
    extended=True evaluates in long double (the adjudicator at the 1e-12 level)."""
    params = params or Params()
    pid = PROCS[proc]
    mom = np.ascontiguousarray(momenta, dtype=np.float64)
    nevt = mom.shape[0]
    out = np.empty(nevt, dtype=np.float64)
    pa = params.array()
    L = lib_ext() if extended else lib()
    if proc.startswith("g g"):
        colour_matrix(pid + 1)  # fill the colour-matrix cache once, outside the pool
    threads = threads or os.cpu_count() or 1
    threads = max(1, min(threads, nevt))
    if threads == 1 or nevt < 2:
        _check(L.mgo_me(pid, _p(pa), _p(mom), nevt, _p(out)))
        return out
    bounds = np.linspace(0, nevt, threads + 1).astype(np.int64)

    def run(i):
        a, b = int(bounds[i]), int(bounds[i + 1])
        if b > a:
            sub_m = mom[a:b]
            sub_o = np.empty(b - a, dtype=np.float64)
            _check(L.mgo_me(pid, _p(pa), _p(sub_m), b - a, _p(sub_o)))
            out[a:b] = sub_o

    with ThreadPoolExecutor(threads) as ex:
        list(ex.map(run, range(threads)))
    return out


def flow_weights(proc: str, momenta: np.ndarray, params: Params | None = None) -> np.ndarray:
    """Per-event colour-flow weights sum_spins |A(sigma)|^2 (mgo_flow_weights)."""
    import math
    params = params or Params()
    mom = np.ascontiguousarray(momenta, dtype=np.float64)
    n = PROCS[proc] + 1
    out = np.empty((mom.shape[0], math.factorial(n)), dtype=np.float64)
    _check(lib().mgo_flow_weights(PROCS[proc], _p(params.array()), _p(mom), mom.shape[0], _p(out)))
    return out


def colour_matrix(n: int) -> np.ndarray:
    """C(sigma, tau) by explicit Gell-Mann index sums (orderings lexicographic)."""
    import math
    np_ = math.factorial(n)
    out = np.empty((np_, np_), dtype=np.complex128)
    _check(lib().mgo_colour_matrix(n, out.ctypes.data_as(_D)))
    return out


def permutations(n: int) -> np.ndarray:
    import math
    out = np.empty((math.factorial(n), n), dtype=np.int32)
    _check(lib().mgo_permutations(n, out.ctypes.data_as(_I)))
    return out


def generators() -> np.ndarray:
    out = np.empty((8, 3, 3), dtype=np.complex128)
    _check(lib().mgo_generators(out.ctypes.data_as(_D)))
    return out


def fabc() -> np.ndarray:
    out = np.empty((8, 8, 8), dtype=np.float64)
    _check(lib().mgo_fabc(_p(out)))
    return out


def gamma() -> np.ndarray:
    out = np.empty((5, 4, 4), dtype=np.complex128)
    _check(lib().mgo_gamma(out.ctypes.data_as(_D)))
    return out


def spinor(kind: str, p, m: float, s: int) -> np.ndarray:
    k = {"u": 0, "v": 1, "ubar": 2, "vbar": 3}[kind]
    p = np.ascontiguousarray(p, dtype=np.float64)
    out = np.empty(4, dtype=np.complex128)
    _check(lib().mgo_spinor(k, _p(p), m, s, out.ctypes.data_as(_D)))
    return out


def polarisation(k, which: int) -> np.ndarray:
    k = np.ascontiguousarray(k, dtype=np.float64)
    out = np.empty(4, dtype=np.float64)
    _check(lib().mgo_polarisation(_p(k), which, _p(out)))
    return out


def _qline_call(fn, n, params, kin, eps, pt, ubar, ptb, v, out):
    params = params or Params()
    args = [np.ascontiguousarray(x, dtype=dt) for x, dt in (
        (params.array(), np.float64), (kin, np.float64), (eps, np.complex128),
        (pt, np.float64), (ubar, np.complex128), (ptb, np.float64), (v, np.complex128))]
    _check(fn(n, *[a.ctypes.data_as(_D) for a in args], out.ctypes.data_as(_D)))
    return out


def ordered_amps(n, kin, eps, pt, ubar, ptb, v, params: Params | None = None) -> np.ndarray:
    """Colour-ordered partial amplitudes A(sigma) for explicit external states."""
    import math
    out = np.empty(math.factorial(n), dtype=np.complex128)
    return _qline_call(lib().mgo_ordered_amps, n, params, kin, eps, pt, ubar, ptb, v, out)


def ordered_colour_sum(n, kin, eps, pt, ubar, ptb, v, params: Params | None = None) -> float:
    out = np.empty(1, dtype=np.float64)
    return float(_qline_call(lib().mgo_ordered_colour_sum, n, params, kin, eps, pt, ubar, ptb, v, out)[0])


def dressed_colour_sum(n, kin, eps, pt, ubar, ptb, v, params: Params | None = None) -> float:
    out = np.empty(1, dtype=np.float64)
    return float(_qline_call(lib().mgo_dressed_colour_sum, n, params, kin, eps, pt, ubar, ptb, v, out)[0])


def unweight(w: np.ndarray, r: np.ndarray, w_max: float) -> np.ndarray:
    """Hit-or-miss unweighting (paper Sect. 2, a serial step after the ME):
    the indices i, in increasing order, of the events with r_i * w_max < w_i,
    r_i uniform in [0, 1).  Written as the definition, one event at a time."""
    w = np.asarray(w, dtype=np.float64)
    r = np.asarray(r, dtype=np.float64)
    kept = [i for i in range(w.shape[0]) if r[i] * w_max < w[i]]
    return np.array(kept, dtype=np.int64)


def uuttg_amps(mom: np.ndarray, spins, eps5, params: Params | None = None) -> np.ndarray:
    """Colour-dressed amplitudes of u u~ -> t t~ g for one event, spins
    (s1, s2, s3, s4) in {0, 1} and a complex gluon polarisation vector eps5[4]
    (mgo_uuttg_amps): complex [3 (u)][3 (u~)][3 (t)][3 (t~)][8 (gluon)]."""
    params = params or Params()
    m = np.ascontiguousarray(mom, dtype=np.float64).reshape(20)
    e = np.ascontiguousarray(np.asarray(eps5, dtype=np.complex128).view(np.float64))
    out = np.empty(648 * 2, dtype=np.float64)
    _check(lib().mgo_uuttg_amps(_p(params.array()), _p(m), *[int(x) for x in spins], _p(e), _p(out)))
    return out.view(np.complex128).reshape(3, 3, 3, 3, 8)


def uutt_ng(ng: int, momenta: np.ndarray, params: Params | None = None, threads: int | None = None,
            extended: bool = False) -> np.ndarray:
    """u u~ -> t t~ + ng gluons (0..2) by the colour-dressed recursion over
    both quark lines (mgo_uutt_ng), events split over host threads."""
    params = params or Params()
    mom = np.ascontiguousarray(momenta, dtype=np.float64)
    nevt = mom.shape[0]
    out = np.empty(nevt, dtype=np.float64)
    pa = params.array()
    L = lib_ext() if extended else lib()
    threads = max(1, min(threads or os.cpu_count() or 1, nevt))
    bounds = np.linspace(0, nevt, threads + 1).astype(np.int64)

    def run(i):
        a, b = int(bounds[i]), int(bounds[i + 1])
        if b > a:
            sub_m = np.ascontiguousarray(mom[a:b])
            sub_o = np.empty(b - a, dtype=np.float64)
            _check(L.mgo_uutt_ng(ng, _p(pa), _p(sub_m), b - a, _p(sub_o)))
            out[a:b] = sub_o

    if threads == 1:
        run(0)
    else:
        with ThreadPoolExecutor(threads) as ex:
            list(ex.map(run, range(threads)))
    return out


def uutt_ng_fixed_pol(ng: int, mom: np.ndarray, eps, params: Params | None = None) -> float:
    """|M|^2 of u u~ -> t t~ + ng gluons summed over quark spins and colours,
    for given complex gluon polarisation vectors eps[ng][4] (eps = k: Ward)."""
    params = params or Params()
    m = np.ascontiguousarray(mom, dtype=np.float64).reshape(-1)
    e = np.ascontiguousarray(np.asarray(eps, dtype=np.complex128).reshape(ng, 4).view(np.float64))
    out = np.empty(1, dtype=np.float64)
    _check(lib().mgo_uutt_ng_fixed_pol(ng, _p(params.array()), _p(m), _p(e), _p(out)))
    return float(out[0])
