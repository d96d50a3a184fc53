"""Event-by-event helicity and colour-flow choice (mg_sigma_select)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
from paper_2303_18244_gb300 import mg  # noqa: E402
from paper_2303_18244_gb300.inputs import process_momenta, uniforms  # noqa: E402

pytestmark = pytest.mark.gpu

# process, sqrt(s), seed, events
CASES = [("g g > t t~", 1000.0, 2, 300), ("g g > t t~ g", 1200.0, 6, 300), ("g g > t t~ g g", 1500.0, 3, 300),
         ("g g > t t~ g g g", 2000.0, 4, 130)]


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _run(h, p, r):
    n = p.shape[0]
    me = torch.empty(n, dtype=torch.float64, device="cuda")
    hel = torch.empty(n, dtype=torch.int32, device="cuda")
    col = torch.empty(n, dtype=torch.int32, device="cuda")
    w = torch.empty((n, h.info.n_col), dtype=torch.float64, device="cuda")
    mg.sigma_select(h, _dev(p), _dev(r), me, hel, col, w)
    torch.cuda.synchronize()
    assert mg.process_status(h) == 0
    return me.cpu().numpy(), hel.cpu().numpy(), col.cpu().numpy(), w.cpu().numpy()


def _expected_choice(weights, r):
    """smallest index whose cumulative weight exceeds r * total; the margin to
    the nearest boundary tells whether rounding could flip the choice."""
    cum = np.cumsum(weights)
    th = r * cum[-1]
    k = int(np.argmax((cum > th) & (weights > 0)))
    margin = np.min(np.abs(cum - th)) / cum[-1]
    return k, margin


@pytest.mark.parametrize("proc,sqrts,seed,n", CASES, ids=["ggtt", "ggttg", "ggttgg", "ggttggg"])
def test_fp64_choices_are_consistent(proc, sqrts, seed, n):
    """FP64 choices against the per-helicity values and flow weights, and the
    flow weights against the oracle's; for g g > t t~ g g g (128 helicities,
    120 flows per event kept per thread) over two CTAs and a tail."""
    p = process_momenta(proc, sqrts, n, seed + 40)
    r = uniforms(77, 0, n, 1)[:, 0, :2]
    h = mg.Process(proc)
    ngood, mask = mg.good_helicities(h, _dev(process_momenta(proc, sqrts, 1024, seed + 1000)))
    good = np.nonzero(mask)[0]
    me, hel, col, w = _run(h, p, r)
    # the ME is mg_sigma's
    ref = torch.empty(n, dtype=torch.float64, device="cuda")
    mg.sigma(h, _dev(p), ref)
    torch.cuda.synchronize()
    np.testing.assert_allclose(me, ref.cpu().numpy(), rtol=1e-14)
    # helicity choice from the per-helicity values of the good list
    per = torch.empty((n, h.info.n_hel), dtype=torch.float64, device="cuda")
    mg.sigma_helicities(h, _dev(p), per)
    torch.cuda.synchronize()
    per = per.cpu().numpy()[:, good]
    for e in range(n):
        k, margin = _expected_choice(per[e], r[e, 0])
        if margin > 1e-12:
            assert hel[e] == good[k]
        k, margin = _expected_choice(w[e], r[e, 1])
        if margin > 1e-12:
            assert col[e] == k
    # colour-flow weights: the oracle's spin-summed |A(sigma)|^2, up to one
    # flow-independent normalisation
    ow = O.flow_weights(proc, p)
    np.testing.assert_allclose(w / w.sum(1, keepdims=True), ow / ow.sum(1, keepdims=True), rtol=1e-10, atol=1e-14)


def test_mixed_choices_valid():
    proc = "g g > t t~ g g"
    n = 2000
    p = process_momenta(proc, 1500.0, n, 9)
    r = uniforms(78, 0, n, 1)[:, 0, :2]
    h64 = mg.Process(proc)
    hmx = mg.Process(proc, precision=mg.MG_MIXED)
    cal = _dev(process_momenta(proc, 1500.0, 1024, 1003))
    _, mask = mg.good_helicities(h64, cal)
    mg.good_helicities(hmx, cal)
    me64, hel64, col64, w64 = _run(h64, p, r)
    me, hel, col, w = _run(hmx, p, r)
    rel = np.abs(me / me64 - 1)
    assert np.median(rel) <= 1e-5
    assert np.all(mask[hel] == 1) and np.all((col >= 0) & (col < 24))
    # the same choices except where FP32 rounding crosses a boundary
    assert np.mean(hel == hel64) > 0.99 and np.mean(col == col64) > 0.99


def test_eemumu_single_flow():
    proc = "e+ e- > mu+ mu-"
    p = process_momenta(proc, 500.0, 500, 1)
    r = uniforms(79, 0, 500, 1)[:, 0, :2]
    h = mg.Process(proc)
    _, mask = mg.good_helicities(h, _dev(process_momenta(proc, 500.0, 1024, 1001)))
    me, hel, col, w = _run(h, p, r)
    assert np.all(col == 0) and np.all(mask[hel] == 1)
    np.testing.assert_allclose(me, O.me(proc, p), rtol=1e-12)


def test_mixed_choices_valid_ggttggg():
    """The mixed selection of g g > t t~ g g g: its ME within the mixed bounds
    of the FP64 one, every chosen helicity good, every flow index in range,
    the choices equal to the FP64 ones except where rounding crosses a
    boundary."""
    proc = "g g > t t~ g g g"
    n = 256
    p = process_momenta(proc, 2000.0, n, 10)
    r = uniforms(80, 0, n, 1)[:, 0, :2]
    h64 = mg.Process(proc)
    hmx = mg.Process(proc, precision=mg.MG_MIXED)
    cal = _dev(process_momenta(proc, 2000.0, 1024, 1004))
    _, mask = mg.good_helicities(h64, cal)
    mg.good_helicities(hmx, cal)
    me64, hel64, col64, _ = _run(h64, p, r)
    me, hel, col, _ = _run(hmx, p, r)
    rel = np.abs(me / me64 - 1)
    assert np.median(rel) <= 1e-5 and rel.max() <= 1e-3
    assert np.all(mask[hel] == 1) and np.all((col >= 0) & (col < 120))
    assert np.mean(hel == hel64) > 0.98 and np.mean(col == col64) > 0.98
