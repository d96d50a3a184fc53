"""Device phase-space generation (mg_rambo) against the host input module."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
from paper_2303_18244_gb300 import mg  # noqa: E402
from paper_2303_18244_gb300.inputs import process_momenta  # noqa: E402

pytestmark = pytest.mark.gpu

CASES = [("e+ e- > mu+ mu-", 500.0, 1), ("g g > t t~", 1000.0, 2), ("g g > t t~ g", 1200.0, 6),
         ("g g > t t~ g g", 1500.0, 3), ("g g > t t~ g g g", 2000.0, 4), ("u u~ > t t~", 1000.0, 7),
         ("u u~ > t t~ g", 1200.0, 8), ("u u~ > t t~ g g", 1500.0, 9)]


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.mark.parametrize("proc,sqrts,seed", CASES, ids=["eemumu", "ggtt", "ggttg", "ggttgg", "ggttggg", "uutt", "uuttg", "uuttgg"])
def test_device_stream_matches_host(proc, sqrts, seed):
    h = mg.Process(proc)
    n, first = 5000, 123456
    dev = torch.empty((n, h.info.npar, 4), dtype=torch.float64, device="cuda")
    mg.rambo(h, sqrts, seed, first, dev)
    torch.cuda.synchronize()
    got = dev.cpu().numpy()
    want = process_momenta(proc, sqrts, n, seed, first_event=first)
    # Same Philox integers; CUDA's and the host's log/sin/cos may differ in the
    # last ulp, which the conformal map amplifies when the generated total
    # momentum is nearly lightlike (a few 2-body events reach ~1e-11 relative).
    d = np.abs(got - want)
    assert np.mean(d <= 1e-12 * sqrts) >= 0.999
    assert d.max() <= 1e-8 * sqrts
    # exact kinematics of the device output itself
    tot = got[:, 2:].sum(1) - got[:, :2].sum(1)
    assert np.abs(tot).max() <= 4e-15 * sqrts
    m2 = got[..., 0] ** 2 - (got[..., 1:] ** 2).sum(-1)
    mt2 = 173.0 ** 2 if "t t~" in proc else 0.0
    assert np.abs(m2[:, 2:4] - mt2).max() <= 1e-10 * sqrts ** 2


def test_device_momenta_give_the_oracle_me():
    proc = "g g > t t~ g g"
    h = mg.Process(proc)
    dev = torch.empty((64, 6, 4), dtype=torch.float64, device="cuda")
    mg.rambo(h, 1500.0, 3, 0, dev)
    out = torch.empty(64, dtype=torch.float64, device="cuda")
    mg.sigma(h, dev, out)
    torch.cuda.synchronize()
    ref = O.me(proc, dev.cpu().numpy())
    np.testing.assert_allclose(out.cpu().numpy(), ref, rtol=1e-12)


def test_bad_arguments():
    h = mg.Process("g g > t t~")
    dev = torch.empty((4, 4, 4), dtype=torch.float64, device="cuda")
    L = mg.lib()
    assert L.mg_rambo(h.handle, 300.0, 1, 0, 4, dev.data_ptr(), None) == -2  # below 2 mt
    assert L.mg_rambo(h.handle, 1000.0, 1, -1, 4, dev.data_ptr(), None) == -2
    assert L.mg_rambo(h.handle, 1000.0, 1, 0, -4, dev.data_ptr(), None) == -2
    assert L.mg_rambo(h.handle, 1000.0, 1, 0, 0, None, None) == 0
