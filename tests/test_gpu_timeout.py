"""The bounded-wait failure path, taken on healthy inputs.

Every device wait (the bulk copy of a CTA's momenta tile, each tensor-core
MMA) gives up after a bound of polls, sets a bit in the handle's status word
and leaves the kernel's outputs unwritten.  With the bound set to 0 through
mg_diag_set_wait_polls every such wait gives up at once: the call must report
MG_ERR_TIMEOUT, leave the outputs as they were, and the next call with the
default bound must be correct again (the GPU context stays usable).  No
kernel is broken and no wait is removed: after giving up, a kernel still
waits with the full bound for the copy or MMA it started."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
from paper_2303_18244_gb300 import mg  # noqa: E402
from paper_2303_18244_gb300.inputs import process_momenta  # noqa: E402
from mixed_bounds import check_mixed  # noqa: E402

pytestmark = pytest.mark.gpu

MG_ERR_TIMEOUT = -5

# (process, sqrt(s), precision, events): the waits each case reaches
CASES = [
    ("g g > t t~", 1000.0, mg.MG_FP64, 300),         # bulk copy (CUDA-core kernel)
    ("g g > t t~ g g", 1500.0, mg.MG_MIXED, 300),    # bulk copy (tensor-core kernel)
    ("g g > t t~ g g g", 2000.0, mg.MG_MIXED, 200),  # bulk copy (flow kernel), MMA (colour kernel)
    ("g g > t t~ g g g", 2000.0, mg.MG_FP64, 200),   # bulk copy (tensor-memory FP64 kernel)
]


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.mark.parametrize("proc,sqrts,precision,n", CASES, ids=["ggtt-fp64", "ggttgg-mixed", "ggttggg-mixed",
                                                                 "ggttggg-fp64"])
def test_timeout_path_reports_and_recovers(proc, sqrts, precision, n):
    assert mg.lib().mg_strerror(MG_ERR_TIMEOUT) == b"bounded wait timed out"
    p = process_momenta(proc, sqrts, n, 17)
    mom = torch.from_numpy(p).cuda()
    h = mg.Process(proc, precision=precision)
    assert mg.process_status(h) == 0
    sentinel = -12345.0
    out = torch.full((n,), sentinel, dtype=torch.float64, device="cuda")
    mg.diag_set_wait_polls(h, 0)
    mg.sigma(h, mom, out)
    torch.cuda.synchronize()
    assert mg.process_status(h) == MG_ERR_TIMEOUT
    assert mg.process_status(h) == 0  # reading the status clears it
    assert bool((out == sentinel).all()), "a kernel that gave up wrote its outputs"
    mg.diag_set_wait_polls(h, mg.DIAG_WAIT_POLLS)
    mg.sigma(h, mom, out)
    torch.cuda.synchronize()
    assert mg.process_status(h) == 0
    got = out.cpu().numpy()
    ref = O.me(proc, p)
    r = np.abs(got / ref - 1)
    if precision == mg.MG_FP64:
        bad = np.nonzero(r > 1e-12)[0]
        if bad.size:
            r[bad] = np.abs(got[bad] / O.me(proc, p[bad], extended=True) - 1)
        assert r.max() <= 1e-12
    else:
        check_mixed(proc, r)
