"""Python binding of the C ABI in include/mg.h (argument marshalling only).

Every computation runs in libmg.so's CUDA kernels.  Device buffers are torch
CUDA tensors (float64, contiguous); streams are torch CUDA streams.  If the
library has not been built this module raises at import of the library -- there
is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libmg.so")

MG_OK = 0
MG_PENDING = 1
MG_FP64 = 0
MG_MIXED = 1
MG_MIXED_PAPER = 2
MG_FLOAT = 3
MG_NO_TOP_WIDTH = 1
MG_PHOTON_ONLY = 2

# every symbol declared in include/mg.h
EXPORTS = (
    "mg_params_default", "mg_process_create", "mg_process_destroy", "mg_process_info",
    "mg_good_helicities", "mg_sigma", "mg_sigma_workspace_bytes", "mg_sigma_host", "mg_process_status",
    "mg_sigma_helicities",
    "mg_good_helicities_static", "mg_rambo", "mg_sigma_select", "mg_unweight",
    "mg_server_cfg_default", "mg_server_create", "mg_server_submit", "mg_server_poll",
    "mg_server_destroy", "mg_strerror",
    # include/mg_diag.h
    "mg_diag_fma_peak", "mg_diag_mma_peak", "mg_diag_sigma_phases", "mg_diag_set_wait_polls",
)


class mg_params(ctypes.Structure):
    _fields_ = [("mt", ctypes.c_double), ("wt", ctypes.c_double), ("alpha_s", ctypes.c_double),
                ("mz", ctypes.c_double), ("wz", ctypes.c_double), ("alpha_em_inv", ctypes.c_double),
                ("gf", ctypes.c_double), ("precision", ctypes.c_int), ("flags", ctypes.c_int)]


class mg_server_cfg(ctypes.Structure):
    _fields_ = [("n_streams", ctypes.c_int), ("mem_budget_bytes", ctypes.c_int64),
                ("min_bucket", ctypes.c_int64), ("max_bucket", ctypes.c_int64), ("use_graphs", ctypes.c_int)]


class mg_req_stats(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("submit_us", ctypes.c_double), ("start_us", ctypes.c_double),
                ("done_us", ctypes.c_double), ("latency_us", ctypes.c_double), ("nevt", ctypes.c_int64),
                ("padded_nevt", ctypes.c_int64)]


class MGError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        super().__init__(f"{what}: {strerror(code)} ({code})")


_lib = None


def lib() -> ctypes.CDLL:
    """Load libmg.so (raises if it has not been built: no fallback path exists)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with "
                              "`python -c 'import __graft_entry__ as g; g.build()'`")
        L = ctypes.CDLL(LIB_PATH)
        vp, i64, dp = ctypes.c_void_p, ctypes.c_int64, ctypes.POINTER(ctypes.c_double)
        L.mg_params_default.argtypes = [ctypes.POINTER(mg_params)]
        L.mg_process_create.argtypes = [ctypes.c_char_p, ctypes.POINTER(mg_params), ctypes.POINTER(vp)]
        L.mg_process_destroy.argtypes = [vp]
        L.mg_process_destroy.restype = None
        ip = ctypes.POINTER(ctypes.c_int)
        L.mg_process_info.argtypes = [vp, ip, ip, ip, ip, dp]
        L.mg_good_helicities.argtypes = [vp, vp, i64, ip, ctypes.POINTER(ctypes.c_uint8)]
        L.mg_good_helicities_static.argtypes = [vp, vp, i64, ip, ctypes.POINTER(ctypes.c_uint8)]
        L.mg_sigma.argtypes = [vp, vp, i64, vp, vp]
        L.mg_sigma_workspace_bytes.argtypes = [vp, i64, ctypes.POINTER(i64)]
        L.mg_rambo.argtypes = [vp, ctypes.c_double, ctypes.c_uint64, i64, i64, vp, vp]
        L.mg_unweight.argtypes = [vp, vp, i64, ctypes.c_double, vp, vp, vp]
        L.mg_sigma_select.argtypes = [vp, vp, i64, vp, vp, vp, vp, vp, vp]
        L.mg_sigma_host.argtypes = [vp, vp, i64, vp, vp]
        L.mg_process_status.argtypes = [vp]
        L.mg_sigma_helicities.argtypes = [vp, vp, i64, vp, vp]
        L.mg_server_cfg_default.argtypes = [ctypes.POINTER(mg_server_cfg)]
        L.mg_server_create.argtypes = [ctypes.POINTER(mg_server_cfg), ctypes.POINTER(vp)]
        L.mg_server_submit.argtypes = [vp, vp, vp, i64, vp, ctypes.POINTER(ctypes.c_uint64)]
        L.mg_server_poll.argtypes = [vp, ctypes.c_uint64, i64, ctypes.POINTER(mg_req_stats)]
        L.mg_server_destroy.argtypes = [vp]
        L.mg_server_destroy.restype = None
        L.mg_diag_fma_peak.argtypes = [ctypes.c_int, dp]
        L.mg_diag_mma_peak.argtypes = [dp]
        fp = ctypes.POINTER(ctypes.c_float)
        L.mg_diag_sigma_phases.argtypes = [vp, vp, i64, vp, vp, fp, fp, ip]
        L.mg_diag_set_wait_polls.argtypes = [vp, ctypes.c_uint32]
        L.mg_strerror.argtypes = [ctypes.c_int]
        L.mg_strerror.restype = ctypes.c_char_p
        _lib = L
    return _lib


def strerror(code: int) -> str:
    try:
        return lib().mg_strerror(code).decode()
    except ImportError:
        return "libmg.so not loaded"


def _check(rc: int, what: str) -> int:
    if rc < 0:
        raise MGError(rc, what)
    return rc


def _stream_ptr(stream) -> int | None:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return getattr(stream, "cuda_stream", stream)


def params_default(**over) -> mg_params:
    p = mg_params()
    _check(lib().mg_params_default(ctypes.byref(p)), "mg_params_default")
    for k, v in over.items():
        setattr(p, k, v)
    return p


@dataclass
class Info:
    npar: int
    n_hel: int
    n_col: int
    n_diag: int
    iden: float


class Process:
    """Owning wrapper of an mg_process handle."""

    def __init__(self, proc: str, params: mg_params | None = None, **over):
        self.params = params if params is not None else params_default(**over)
        h = ctypes.c_void_p()
        _check(lib().mg_process_create(proc.encode(), ctypes.byref(self.params), ctypes.byref(h)),
               f"mg_process_create({proc!r})")
        self.handle = h
        self.proc = proc
        self.info = process_info(self)

    def close(self):
        if self.handle:
            lib().mg_process_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def process_create(proc: str, params: mg_params | None = None, **over) -> Process:
    return Process(proc, params, **over)


def process_info(h: Process) -> Info:
    a, b, c, d = (ctypes.c_int() for _ in range(4))
    e = ctypes.c_double()
    _check(lib().mg_process_info(h.handle, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c), ctypes.byref(d),
                                 ctypes.byref(e)), "mg_process_info")
    return Info(a.value, b.value, c.value, d.value, e.value)


def _dev_check(t, npar=None):
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise TypeError("expected a contiguous float64 CUDA tensor")
    return t.data_ptr()


def good_helicities(h: Process, momenta_dev, nevt: int | None = None):
    """(n_good, mask[n_hel] uint8) -- mg_good_helicities."""
    nevt = momenta_dev.shape[0] if nevt is None else nevt
    ptr = _dev_check(momenta_dev) if nevt else None
    n = ctypes.c_int()
    mask = np.zeros(h.info.n_hel, dtype=np.uint8)
    _check(lib().mg_good_helicities(h.handle, ptr, nevt, ctypes.byref(n),
                                    mask.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))), "mg_good_helicities")
    return n.value, mask


def good_helicities_static(h: Process, momenta_dev, nevt: int | None = None):
    """(n_good, mask) -- mg_good_helicities_static: the helicity filter for
    callers that cannot allocate device memory (scratch in a fixed device array)."""
    nevt = momenta_dev.shape[0] if nevt is None else nevt
    ptr = _dev_check(momenta_dev) if nevt else None
    n = ctypes.c_int()
    mask = np.zeros(h.info.n_hel, dtype=np.uint8)
    _check(lib().mg_good_helicities_static(h.handle, ptr, nevt, ctypes.byref(n),
                                           mask.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))),
           "mg_good_helicities_static")
    return n.value, mask


def sigma(h: Process, momenta_dev, me_out_dev, stream=None, nevt: int | None = None):
    """mg_sigma: stream-ordered ME of momenta_dev[nevt][npar][4] into me_out_dev[nevt]."""
    nevt = momenta_dev.shape[0] if nevt is None else nevt
    _check(lib().mg_sigma(h.handle, _dev_check(momenta_dev), nevt, _dev_check(me_out_dev), _stream_ptr(stream)),
           "mg_sigma")


def sigma_workspace_bytes(h: Process, nevt: int) -> int:
    """mg_sigma_workspace_bytes: stream-ordered device bytes one mg_sigma call of nevt events takes."""
    b = ctypes.c_int64()
    _check(lib().mg_sigma_workspace_bytes(h.handle, nevt, ctypes.byref(b)), "mg_sigma_workspace_bytes")
    return b.value


def rambo(h: Process, sqrt_s: float, seed: int, first_event: int, momenta_dev, stream=None):
    """mg_rambo: fill momenta_dev[nevt][npar][4] with device-generated phase space."""
    nevt = momenta_dev.shape[0]
    _check(lib().mg_rambo(h.handle, sqrt_s, seed, first_event, nevt, _dev_check(momenta_dev),
                          _stream_ptr(stream)), "mg_rambo")


def unweight(w_dev, r_dev, w_max: float, idx_out_dev, n_acc_dev, stream=None):
    """mg_unweight: kept indices (r * w_max < w) in increasing order into
    idx_out_dev (int64 [n]); their number into n_acc_dev (int64 [1]). All CUDA."""
    import torch
    n = w_dev.shape[0]
    for t in (idx_out_dev, n_acc_dev):
        if not (t.is_cuda and t.dtype == torch.int64 and t.is_contiguous()):
            raise TypeError("expected contiguous int64 CUDA tensors for the outputs")
    if r_dev.shape[0] != n or idx_out_dev.shape[0] < n:
        raise ValueError("w, r and idx_out must hold n events")
    _check(lib().mg_unweight(_dev_check(w_dev), _dev_check(r_dev), n, w_max, idx_out_dev.data_ptr(),
                             n_acc_dev.data_ptr(), _stream_ptr(stream)), "mg_unweight")


def sigma_select(h: Process, momenta_dev, rnd_dev, me_out_dev, hel_out_dev, col_out_dev, colw_out_dev=None,
                 stream=None):
    """mg_sigma_select: ME plus the per-event helicity and colour-flow choice.
    rnd_dev: float64 [nevt][2]; hel/col outputs: int32 [nevt]; colw: float64 [nevt][n_col] or None."""
    import torch
    nevt = momenta_dev.shape[0]
    for t in (hel_out_dev, col_out_dev):
        if not (t.is_cuda and t.dtype == torch.int32 and t.is_contiguous()):
            raise TypeError("expected contiguous int32 CUDA tensors for the choices")
    _check(lib().mg_sigma_select(h.handle, _dev_check(momenta_dev), nevt, _dev_check(rnd_dev), _dev_check(me_out_dev),
                                 hel_out_dev.data_ptr(), col_out_dev.data_ptr(),
                                 _dev_check(colw_out_dev) if colw_out_dev is not None else None,
                                 _stream_ptr(stream)), "mg_sigma_select")


def sigma_helicities(h: Process, momenta_dev, out_dev, stream=None):
    nevt = momenta_dev.shape[0]
    _check(lib().mg_sigma_helicities(h.handle, _dev_check(momenta_dev), nevt, _dev_check(out_dev),
                                     _stream_ptr(stream)), "mg_sigma_helicities")


def sigma_host(h: Process, momenta_host, me_out_host, stream=None):
    """mg_sigma_host on host arrays (numpy or pinned CPU tensors), synchronous."""
    mp = _host_ptr(momenta_host)
    op = _host_ptr(me_out_host)
    nevt = momenta_host.shape[0]
    _check(lib().mg_sigma_host(h.handle, mp, nevt, op, _stream_ptr(stream)), "mg_sigma_host")


def process_status(h: Process) -> int:
    return lib().mg_process_status(h.handle)


def _host_ptr(a) -> int:
    if isinstance(a, np.ndarray):
        if not (a.flags.c_contiguous and a.dtype == np.float64):
            raise TypeError("expected a contiguous float64 array")
        return a.ctypes.data
    import torch
    if isinstance(a, torch.Tensor) and not a.is_cuda and a.dtype == torch.float64 and a.is_contiguous():
        return a.data_ptr()
    raise TypeError("expected a contiguous float64 host array")


def _any_ptr(a) -> int:
    if isinstance(a, np.ndarray):
        return _host_ptr(a)
    return _dev_check(a) if getattr(a, "is_cuda", False) else _host_ptr(a)


class Server:
    """Owning wrapper of an mg_server (continuous-batching request loop)."""

    def __init__(self, **cfg):
        c = mg_server_cfg()
        _check(lib().mg_server_cfg_default(ctypes.byref(c)), "mg_server_cfg_default")
        for k, v in cfg.items():
            setattr(c, k, v)
        self.cfg = c
        s = ctypes.c_void_p()
        _check(lib().mg_server_create(ctypes.byref(c), ctypes.byref(s)), "mg_server_create")
        self.handle = s

    def submit(self, h: Process, momenta, me_out) -> int:
        """Queue a request; momenta and me_out are host arrays (numpy or CPU
        tensors) or float64 CUDA tensors, each on its own."""
        rid = ctypes.c_uint64()
        _check(lib().mg_server_submit(self.handle, h.handle, _any_ptr(momenta), momenta.shape[0],
                                      _any_ptr(me_out), ctypes.byref(rid)), "mg_server_submit")
        return rid.value

    def poll(self, req_id: int, timeout_us: int = 0):
        """(status, stats) with status MG_OK or MG_PENDING; errors raise."""
        st = mg_req_stats()
        rc = lib().mg_server_poll(self.handle, req_id, timeout_us, ctypes.byref(st))
        _check(rc, "mg_server_poll")
        return rc, st

    def close(self):
        if self.handle:
            lib().mg_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def diag_fma_peak(kind: int) -> float:
    """Measured FMA peak in GFLOP/s (0 = FP32, 1 = FP64), include/mg_diag.h."""
    g = ctypes.c_double()
    _check(lib().mg_diag_fma_peak(kind, ctypes.byref(g)), "mg_diag_fma_peak")
    return g.value


def diag_sigma_phases(h: Process, momenta_dev, me_out_dev, stream=None):
    """(ms of the first kernels, ms of the second kernels, slices) of one
    two-phase mg_sigma call, timed kernel by kernel (include/mg_diag.h)."""
    a, b, n = ctypes.c_float(), ctypes.c_float(), ctypes.c_int()
    _check(lib().mg_diag_sigma_phases(h.handle, _dev_check(momenta_dev), momenta_dev.shape[0], _dev_check(me_out_dev),
                                      _stream_ptr(stream), ctypes.byref(a), ctypes.byref(b), ctypes.byref(n)),
           "mg_diag_sigma_phases")
    return a.value, b.value, n.value


DIAG_WAIT_POLLS = 1 << 22


def diag_set_wait_polls(h: Process, polls: int):
    """Bound of the first wait on each device barrier of h's kernels (include/mg_diag.h)."""
    _check(lib().mg_diag_set_wait_polls(h.handle, polls), "mg_diag_set_wait_polls")


def diag_mma_peak() -> float:
    """Measured dense FP16 tcgen05 MMA throughput in TFLOP/s (include/mg_diag.h)."""
    t = ctypes.c_double()
    _check(lib().mg_diag_mma_peak(ctypes.byref(t)), "mg_diag_mma_peak")
    return t.value
