"""mg_good_helicities_static: the helicity filter for callers that cannot
allocate device memory (a fixed device-memory budget, an own pool allocator,
or a set-up path that must not pay for cudaMalloc/cudaFree).  Its scratch is a
fixed 8 MiB device array inside libmg.so, so it is checked here against the
allocating mg_good_helicities on the same calibration events, call after call.

This file is collected last on purpose: it must pass both alone in a fresh
process and after every other GPU test has used the library."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2303_18244_gb300 import mg  # noqa: E402
from paper_2303_18244_gb300.inputs import process_momenta  # noqa: E402

pytestmark = pytest.mark.gpu

SCRATCH_DOUBLES = 1 << 20  # MG_STATIC_SCRATCH_DOUBLES in include/mg.h
MAX_HEL = 128              # MG_STATIC_MAX_HEL

CASES = [("e+ e- > mu+ mu-", 500.0, 1001), ("g g > t t~ g", 1200.0, 1006), ("g g > t t~ g g", 1500.0, 1003)]


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("proc,sqrts,seed", CASES, ids=["eemumu", "ggttg", "ggttgg"])
def test_matches_allocating_filter_two_calls(proc, sqrts, seed):
    h_alloc = mg.Process(proc)
    h_static = mg.Process(proc)
    fresh = _dev(process_momenta(proc, sqrts, 300, seed + 50))
    for call in range(2):
        calib = _dev(process_momenta(proc, sqrts, 1024, seed + 10 * call))
        n_a, m_a = mg.good_helicities(h_alloc, calib)
        n_s, m_s = mg.good_helicities_static(h_static, calib)
        assert n_s == n_a
        assert np.array_equal(m_s, m_a)
        # the matrix elements with the two helicity lists agree (FP64 bar)
        a = torch.empty(300, dtype=torch.float64, device="cuda")
        b = torch.empty(300, dtype=torch.float64, device="cuda")
        mg.sigma(h_alloc, fresh, a)
        mg.sigma(h_static, fresh, b)
        torch.cuda.synchronize()
        np.testing.assert_allclose(b.cpu().numpy(), a.cpu().numpy(), rtol=1e-12)
        assert mg.process_status(h_static) == 0


def test_rejects_sizes_beyond_the_array():
    proc = "g g > t t~ g g"  # 64 helicities
    h = mg.Process(proc)
    nmax = (SCRATCH_DOUBLES - MAX_HEL) // 64
    p = _dev(process_momenta(proc, 1500.0, nmax + 1, 3))
    n = np.zeros(1, dtype=np.int32)
    rc = mg.lib().mg_good_helicities_static(h.handle, p.data_ptr(), nmax + 1, None, None)
    assert rc == -2  # MG_ERR_ARG, nothing launched
    # the largest accepted size works
    n, mask = mg.good_helicities_static(h, p[:nmax])
    assert 1 <= n <= 64 and mask.sum() == n


def test_largest_helicity_count_at_the_size_limit():
    """g g > t t~ g g g has MG_STATIC_MAX_HEL = 128 helicities: 8191 events
    fill the array up to its reduction slots and match the allocating filter;
    8192 events are refused with MG_ERR_ARG before anything runs."""
    proc = "g g > t t~ g g g"
    nmax = (SCRATCH_DOUBLES - MAX_HEL) // MAX_HEL
    assert nmax == 8191
    p = _dev(process_momenta(proc, 2000.0, nmax + 1, 1004))
    h_alloc = mg.Process(proc)
    h_static = mg.Process(proc)
    assert mg.lib().mg_good_helicities_static(h_static.handle, p.data_ptr(), nmax + 1, None, None) == -2
    for _ in range(2):
        n_a, m_a = mg.good_helicities(h_alloc, p[:nmax])
        n_s, m_s = mg.good_helicities_static(h_static, p[:nmax])
        assert n_s == n_a and np.array_equal(m_s, m_a)


def test_no_information_keeps_every_helicity():
    """Calibration events without a positive finite |M|^2 (here NaN momenta,
    which stay in their own lanes) say nothing about the helicities: both
    filters keep all of them, and the count equals the mask's sum."""
    proc = "e+ e- > mu+ mu-"
    bad = _dev(np.full((64, 4, 4), np.nan))
    for fn in (mg.good_helicities, mg.good_helicities_static):
        h = mg.Process(proc)
        n0, _ = fn(h, _dev(process_momenta(proc, 500.0, 256, 1001)))  # a filtered list first
        assert n0 == 4
        n, mask = fn(h, bad)
        assert n == 16 and mask.sum() == 16
        assert mg.process_status(h) == 0
