"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle.

FP64 path: relative error <= 1e-12 per event (the FP64 bar of the workload).
Mixed path: per-process bounds on the median, p99 and max relative error
(tests/mixed_bounds.py, about ten times the measured values).
Small cases span several CTAs plus a ragged tail; the full workload sizes are
checked on sampled events in the launch configuration bench.py times.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
from paper_2303_18244_gb300 import mg  # noqa: E402
from paper_2303_18244_gb300.inputs import process_momenta  # noqa: E402
from mixed_bounds import MIXED_BOUNDS, check_mixed  # noqa: E402

pytestmark = pytest.mark.gpu

# process -> (sqrt(s), seed, small-case size, full workload size)
WORKLOADS = {
    "e+ e- > mu+ mu-": (500.0, 1, 1000, 16384),
    "g g > t t~": (1000.0, 2, 1000, 524288),
    "g g > t t~ g": (1200.0, 6, 300, 65536),
    "g g > t t~ g g": (1500.0, 3, 300, 524288),
    "g g > t t~ g g g": (2000.0, 4, 130, 65536),
    "u u~ > t t~": (1000.0, 7, 1000, 524288),
    "u u~ > t t~ g": (1200.0, 8, 500, 524288),
    "u u~ > t t~ g g": (1500.0, 9, 130, 524288),
}
PROCS = list(WORKLOADS)
TAGS = {"e+ e- > mu+ mu-": "eemumu", "g g > t t~": "ggtt", "g g > t t~ g": "ggttg",
        "g g > t t~ g g": "ggttgg", "g g > t t~ g g g": "ggttggg", "u u~ > t t~": "uutt",
        "u u~ > t t~ g": "uuttg", "u u~ > t t~ g g": "uuttgg"}


def _ids(p):
    return TAGS.get(p, str(p))


def _have(proc):
    try:
        mg.Process(proc).close()
        return True
    except mg.MGError as e:
        if e.code == -1:
            return False
        raise


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _gpu_me(h, p, stream=None):
    mom = _dev(p)
    out = torch.full((p.shape[0],), float("nan"), dtype=torch.float64, device="cuda")
    if stream is not None:
        stream.wait_stream(torch.cuda.current_stream())
    mg.sigma(h, mom, out, stream=stream)
    torch.cuda.synchronize()
    assert mg.process_status(h) == 0
    return out.cpu().numpy()


def _rel(x, y):
    return np.abs(x - y) / np.abs(y)


def _assert_fp64(proc, p, got, ref, tol=1e-12, params=None):
    """Per-event relative error <= tol against the FP64 oracle; where the two
    disagree by more, the long-double build of the oracle decides: the CUDA
    result must then be within tol of the extended-precision value."""
    r = _rel(got, ref)
    bad = np.nonzero(r > tol)[0]
    if bad.size:
        ext = O.me(proc, p[bad], params, extended=True)
        r_ext = _rel(got[bad], ext)
        assert r_ext.max() <= tol, (
            f"{bad.size} events beyond {tol:g}; vs extended precision max {r_ext.max():.3e} "
            f"at event {int(bad[r_ext.argmax()])}")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.mark.parametrize("proc", PROCS, ids=_ids)
def test_fp64_parity_small(proc):
    if not _have(proc):
        pytest.fail(f"{proc} is not compiled into libmg.so")
    rs, seed, n, _ = WORKLOADS[proc]
    p = process_momenta(proc, rs, n, seed)
    h = mg.Process(proc)
    got = _gpu_me(h, p)
    ref = O.me(proc, p)
    assert np.all(np.isfinite(got))
    _assert_fp64(proc, p, got, ref)


@pytest.mark.parametrize("proc", PROCS, ids=_ids)
def test_mixed_parity_small(proc):
    if not _have(proc):
        pytest.fail(f"{proc} is not compiled into libmg.so")
    rs, seed, n, _ = WORKLOADS[proc]
    p = process_momenta(proc, rs, n, seed)
    h = mg.Process(proc, precision=mg.MG_MIXED)
    got = _gpu_me(h, p)
    ref = O.me(proc, p)
    r = _rel(got, ref)
    print(f"{proc}: mixed rel err median {np.median(r):.2e} p99 {np.quantile(r, 0.99):.2e} max {r.max():.2e}")
    check_mixed(proc, r)


@pytest.mark.parametrize("proc", PROCS, ids=_ids)
@pytest.mark.parametrize("precision", [mg.MG_FP64, mg.MG_MIXED], ids=["fp64", "mixed"])
def test_full_size_sampled(proc, precision):
    """Full workload size, bench launch configuration, sampled events vs oracle."""
    if not _have(proc):
        pytest.fail(f"{proc} is not compiled into libmg.so")
    rs, seed, _, nfull = WORKLOADS[proc]
    p = process_momenta(proc, rs, nfull, seed)
    h = mg.Process(proc, precision=precision)
    calib = process_momenta(proc, rs, 1024, seed + 1000)
    mg.good_helicities(h, _dev(calib))
    got = _gpu_me(h, p)
    assert np.all(np.isfinite(got)) and np.all(got > 0)
    rng = np.random.default_rng(seed)
    # the oracle's slowest processes get fewer random samples (gg -> t t~ g g g:
    # 120 orderings x 128 helicities; u u~ -> t t~ g g: colour-dressed recursion)
    nsamp = {"g g > t t~ g g g": 300, "u u~ > t t~ g g": 64}.get(proc, 200)
    # CTA edges (64- and 128-event blocks), the last full block and the tail
    edges = [0, 63, 64, 127, 128, 255, 256, nfull - 129, nfull - 128, nfull - 2, nfull - 1]
    idx = np.unique(np.concatenate([edges, rng.integers(0, nfull, nsamp)]))
    ref = O.me(proc, p[idx])
    r = _rel(got[idx], ref)
    print(f"{proc} {precision}: sampled rel err median {np.median(r):.2e} max {r.max():.2e}")
    if precision == mg.MG_FP64:
        _assert_fp64(proc, p[idx], got[idx], ref)
    else:
        check_mixed(proc, r)


def test_two_phase_mixed_across_slices():
    """gg -> t t~ g g g mixed runs in two phases (colour flows of every
    helicity-event row to HBM, then the tensor-core colour form) over slices
    of the helicities sized to a 1 GiB workspace: 16514 events take two
    slices, 300 events one.  The batch agrees with the FP64 path, and every
    event's value is bit-identical in both batches."""
    proc = "g g > t t~ g g g"
    if not _have(proc):
        pytest.fail(f"{proc} is not compiled into libmg.so")
    rs, seed, _, _ = WORKLOADS[proc]
    p = process_momenta(proc, rs, 16384 + 130, seed)
    calib = _dev(process_momenta(proc, rs, 1024, seed + 1000))
    h = mg.Process(proc, precision=mg.MG_MIXED)
    h64 = mg.Process(proc)
    mg.good_helicities(h, calib)
    mg.good_helicities(h64, calib)
    got = _gpu_me(h, p)
    ref = _gpu_me(h64, p)
    r = _rel(got, ref)
    assert np.all(np.isfinite(got))
    check_mixed(proc, r)
    sub = _gpu_me(h, p[8000:8300])
    assert np.array_equal(sub, got[8000:8300])


def test_good_helicities_eemumu():
    """Massless e+e- -> mu+mu-: exactly the 4 chirality-conserving combinations survive."""
    proc = "e+ e- > mu+ mu-"
    h = mg.Process(proc)
    calib = process_momenta(proc, 500.0, 1024, 1001)
    n, mask = mg.good_helicities(h, _dev(calib))
    assert n == 4
    # helicity index bits: particle i <-> bit (3 - i), 1 = +; e+ e- mu+ mu-
    good = {i for i in range(16) if mask[i]}
    want = set()
    for i in range(16):
        l = [1 if (i >> (3 - k)) & 1 else -1 for k in range(4)]
        if l[0] == -l[1] and l[2] == -l[3]:
            want.add(i)
    assert good == want


@pytest.mark.parametrize("proc", ["u u~ > t t~", "u u~ > t t~ g", "u u~ > t t~ g g"], ids=["uutt", "uuttg", "uuttgg"])
def test_good_helicities_light_quark_chirality(proc):
    """The massless u u~ pair couples through a vector current: exactly the
    helicity states with opposite u and u~ helicities survive (every top and
    gluon helicity does)."""
    rs, seed, _, _ = WORKLOADS[proc]
    h = mg.Process(proc)
    npar = h.info.npar
    n, mask = mg.good_helicities(h, _dev(process_momenta(proc, rs, 1024, seed + 1000)))
    good = {i for i in range(1 << npar) if mask[i]}
    want = {i for i in range(1 << npar) if ((i >> (npar - 1)) & 1) != ((i >> (npar - 2)) & 1)}
    assert good == want and n == len(want)


@pytest.mark.parametrize("proc", PROCS, ids=_ids)
def test_good_helicities_masked_sum_equals_full(proc):
    if not _have(proc):
        pytest.fail(f"{proc} is not compiled into libmg.so")
    rs, seed, n, _ = WORKLOADS[proc]
    h = mg.Process(proc)
    fresh = process_momenta(proc, rs, min(n, 256), seed + 7)
    full = _gpu_me(h, fresh)
    calib = process_momenta(proc, rs, 1024, seed + 1000)
    ngood, mask = mg.good_helicities(h, _dev(calib))
    assert 1 <= ngood <= h.info.n_hel and mask.sum() == ngood
    masked = _gpu_me(h, fresh)
    assert np.max(_rel(masked, full)) <= 1e-14 * 10
    # per-helicity values sum to the ME
    out = torch.empty((fresh.shape[0], h.info.n_hel), dtype=torch.float64, device="cuda")
    mg.sigma_helicities(h, _dev(fresh), out)
    torch.cuda.synchronize()
    np.testing.assert_allclose(out.sum(1).cpu().numpy(), full, rtol=1e-13)


@pytest.mark.parametrize("n", [1, 2, 31, 127, 128, 129, 257])
def test_ragged_sizes(n):
    proc = "g g > t t~ g"
    p = process_momenta(proc, 1200.0, n, 17)
    h = mg.Process(proc)
    got = _gpu_me(h, p)
    _assert_fp64(proc, p, got, O.me(proc, p))


def test_zero_events_and_bad_arguments():
    h = mg.Process("g g > t t~")
    mom = torch.zeros((0, 4, 4), dtype=torch.float64, device="cuda")
    out = torch.zeros((0,), dtype=torch.float64, device="cuda")
    assert mg.lib().mg_sigma(h.handle, None, 0, None, None) == 0
    mg.sigma(h, mom, out)
    p = _dev(process_momenta("g g > t t~", 1000.0, 8, 2))
    o = torch.empty(8, dtype=torch.float64, device="cuda")
    assert mg.lib().mg_sigma(h.handle, p.data_ptr(), -1, o.data_ptr(), None) == -2
    assert mg.lib().mg_sigma(h.handle, p.data_ptr() + 8, 4, o.data_ptr(), None) == -2  # misaligned
    assert mg.lib().mg_sigma(None, p.data_ptr(), 8, o.data_ptr(), None) == -2
    with pytest.raises(mg.MGError) as ei:
        mg.Process("d d~ > t t~ g")  # not a compiled process
    assert ei.value.code == -1
    with pytest.raises(mg.MGError):
        mg.Process("g g > t t~", precision=7)


def test_sigma_host_matches_device_and_stream():
    proc = "g g > t t~ g g"
    p = process_momenta(proc, 1500.0, 300, 23)
    h = mg.Process(proc, precision=mg.MG_MIXED)
    s = torch.cuda.Stream()
    dev = _gpu_me(h, p, stream=s)
    out = np.empty(p.shape[0])
    mg.sigma_host(h, p, out)
    np.testing.assert_array_equal(out, dev)


def test_no_top_width_flag_matches_oracle():
    proc = "g g > t t~ g"
    p = process_momenta(proc, 1200.0, 200, 29)
    h = mg.Process(proc, flags=mg.MG_NO_TOP_WIDTH)
    par = O.Params(wt=0.0)
    _assert_fp64(proc, p, _gpu_me(h, p), O.me(proc, p, par), params=par)


def test_photon_only_closed_form():
    proc = "e+ e- > mu+ mu-"
    p = process_momenta(proc, 500.0, 1000, 1)
    h = mg.Process(proc, flags=mg.MG_PHOTON_ONLY)
    got = _gpu_me(h, p)
    e2 = 4 * np.pi / 132.507
    a, b = p[:, 1, 1:], p[:, 3, 1:]
    c = (a * b).sum(-1) / np.linalg.norm(a, axis=1) / np.linalg.norm(b, axis=1)
    np.testing.assert_allclose(got, e2 ** 2 * (1 + c ** 2), rtol=1e-12)


@pytest.mark.parametrize("proc", PROCS, ids=_ids)
def test_paper_mixed_parity_small(proc):
    """The paper's mixed mode: FP64 diagrams, FP32 colour algebra."""
    if not _have(proc):
        pytest.fail(f"{proc} is not compiled into libmg.so")
    rs, seed, n, _ = WORKLOADS[proc]
    p = process_momenta(proc, rs, n, seed)
    h = mg.Process(proc, precision=mg.MG_MIXED_PAPER)
    got = _gpu_me(h, p)
    r = _rel(got, O.me(proc, p))
    assert np.median(r) <= 1e-6 and r.max() <= 1e-4


@pytest.mark.parametrize("proc", PROCS, ids=_ids)
def test_float_parity_small(proc):
    """The paper's float mode: every step in FP32, including the per-event
    set-up and the propagator denominators.  Bounds: FP32 rounding (6e-8)
    grows with the number of terms (up to ~1e5 per helicity) and with the
    cancellation in P^2 - m^2 near the top mass shell (|P^2| / |P^2 - m^2| up
    to ~1e3 for soft gluons off a top), so single events can lose several
    digits; the typical event keeps about six."""
    if not _have(proc):
        pytest.fail(f"{proc} is not compiled into libmg.so")
    rs, seed, n, _ = WORKLOADS[proc]
    p = process_momenta(proc, rs, n, seed)
    h = mg.Process(proc, precision=mg.MG_FLOAT)
    got = _gpu_me(h, p)
    r = _rel(got, O.me(proc, p))
    print(f"{proc}: float rel err median {np.median(r):.2e} p99 {np.quantile(r, 0.99):.2e} max {r.max():.2e}")
    assert np.all(np.isfinite(got))
    assert np.median(r) <= 1e-5 and np.quantile(r, 0.99) <= 1e-3 and r.max() <= 5e-2


def test_fp64_ill_conditioned_event_against_extended_oracle():
    """Event 29039 of the gg -> t t~ g g workload has an initial and a final
    gluon 0.33 GeV^2 from collinear: a t-channel invariant that cancels to six
    digits in FP64 components.  The FP64 oracle loses them (5e-10 from its
    long-double build); the FP64 path, whose propagator invariants are
    compensated, must stay within 1e-12 of the long-double value on it and its
    neighbours."""
    proc = "g g > t t~ g g"
    p = process_momenta(proc, 1500.0, 29040, 3)[29030:29040].copy()
    h = mg.Process(proc)
    got = _gpu_me(h, p)
    ext = O.me(proc, p, extended=True)
    assert _rel(got, ext).max() <= 1e-12
    assert _rel(O.me(proc, p), ext).max() > 1e-10  # the FP64 oracle itself does not


# (process, precision, batch size): batch * npar * 4 > 2^31 momentum elements
LARGE = [
    ("g g > t t~", mg.MG_FP64, (1 << 27) + (1 << 20) + 77),
    ("g g > t t~", mg.MG_MIXED, (1 << 27) + (1 << 20) + 77),
    ("g g > t t~ g g", mg.MG_MIXED, 89_478_485 + 65536 + 45),
]


@pytest.mark.parametrize("proc,precision,nevt", LARGE, ids=["ggtt-fp64", "ggtt-mixed", "ggttgg-mixed"])
def test_element_offsets_beyond_32_bits(proc, precision, nevt):
    """Maximum sizes: more than 2^31 momentum elements (17 GB on the device),
    so every offset past 2^31 must be 64-bit.  The batch repeats a block of
    4099 (prime) events: an offset that wrapped at 2^31 elements, or a result
    written to the wrong slot, would pair an event with another event's
    value.  Every copy of an event must give the block's value (a property of
    the whole 1e8-event output), and events on both sides of the
    2^31-element boundary, in the ragged tail and at the start are compared
    with the oracle."""
    rs, seed, _, _ = WORKLOADS[proc]
    h = mg.Process(proc, precision=precision)
    npar = h.info.npar
    need = nevt * (npar * 4 * 8 + 8 + 1) + (1 << 30)
    free, _ = torch.cuda.mem_get_info()
    if free < need:
        pytest.skip(f"needs {need / 1e9:.1f} GB of free device memory, {free / 1e9:.1f} GB free")
    B = 4099
    block = process_momenta(proc, rs, B, seed + 2000)
    blk = _dev(block)
    mom = torch.empty((nevt, npar, 4), dtype=torch.float64, device="cuda")
    reps = nevt // B
    mom[: reps * B].view(reps, B, npar, 4).copy_(blk.unsqueeze(0).expand(reps, B, npar, 4))
    mom[reps * B:].copy_(blk[: nevt - reps * B])
    out = torch.full((nevt,), float("nan"), dtype=torch.float64, device="cuda")
    mg.good_helicities(h, _dev(process_momenta(proc, rs, 1024, seed + 1000)))
    mg.sigma(h, mom, out)
    torch.cuda.synchronize()
    assert mg.process_status(h) == 0
    del mom
    head = out[:B]
    assert bool(torch.isfinite(out).all()) and bool((out > 0).all())
    dev = (out[: reps * B].view(reps, B) - head).abs() / head
    tail = (out[reps * B:] - head[: nevt - reps * B]).abs() / head[: nevt - reps * B]
    worst = max(float(dev.max()), float(tail.max()) if tail.numel() else 0.0)
    print(f"{proc} nevt {nevt}: largest deviation between copies of an event {worst:.2e}")
    # FP64: one thread per event, the same instructions wherever the event
    # sits; mixed: the same, bar any dependence of the tensor-core rows on
    # their TMEM lane
    assert worst <= (0.0 if precision == mg.MG_FP64 else 1e-6)
    cross = -(-(1 << 31) // (npar * 4))  # first event at element offset >= 2^31
    rng = np.random.default_rng(seed)
    idx = np.unique(np.concatenate([
        [0, 1, 127, 128, cross - 129, cross - 1, cross, cross + 1, cross + 127, cross + 128,
         nevt - 130, nevt - 2, nevt - 1], rng.integers(0, nevt, 16)]))
    got = out[torch.from_numpy(idx).cuda()].cpu().numpy()
    p = block[idx % B]
    ref = O.me(proc, p)
    if precision == mg.MG_FP64:
        _assert_fp64(proc, p, got, ref)
    else:
        med, _, mx = MIXED_BOUNDS[proc]
        r = _rel(got, ref)
        assert np.median(r) <= med and r.max() <= mx


def _rotate_onto_axis(p, slot, sign):
    """Rotate every final-state momentum of each event so that particle `slot`
    points along sign * z, then set its transverse components to exactly 0
    (and, for two-body final states, its partner's to the exact opposite)."""
    q = p.copy()
    target = np.array([0.0, 0.0, float(sign)])
    for e in range(q.shape[0]):
        t = q[e, slot, 1:] / np.linalg.norm(q[e, slot, 1:])
        axis = np.cross(t, target)
        s, c = np.linalg.norm(axis), float(t @ target)
        if s > 0:
            k = axis / s
            K = np.array([[0, -k[2], k[1]], [k[2], 0, -k[0]], [-k[1], k[0], 0]])
            R = np.eye(3) + s * K + (1 - c) * K @ K
            q[e, 2:, 1:] = q[e, 2:, 1:] @ R.T
        P = np.linalg.norm(q[e, slot, 1:])
        q[e, slot, 1:] = [0.0, 0.0, sign * P]
        if q.shape[1] == 4:
            q[e, 5 - slot, 1:] = [0.0, 0.0, -sign * P]
    return q


@pytest.mark.parametrize("proc", PROCS, ids=_ids)
def test_final_state_along_the_beam_axis(proc):
    """Special kinematics: the top (mu- for e+e- -> mu+mu-) exactly along +z
    and along -z (p_T = 0), where the spinor set-up takes its degenerate
    branch (p along -z) and the azimuth is undefined; FP64 within 1e-12 of the
    oracle, mixed within its bounds, no NaN.  (Gluons are never put on the
    axis: that is the collinear singularity with a beam gluon.)"""
    if not _have(proc):
        pytest.fail(f"{proc} is not compiled into libmg.so")
    rs, seed, _, _ = WORKLOADS[proc]
    slot = 3 if proc == "e+ e- > mu+ mu-" else 2
    base = process_momenta(proc, rs, 8, seed + 3000)
    p = np.concatenate([_rotate_onto_axis(base, slot, +1), _rotate_onto_axis(base, slot, -1)])
    assert np.all(p[:, slot, 1:3] == 0.0)
    ref = O.me(proc, p)
    assert np.all(np.isfinite(ref)) and np.all(ref > 0)
    got = _gpu_me(mg.Process(proc), p)
    assert np.all(np.isfinite(got))
    _assert_fp64(proc, p, got, ref)
    mixed = _gpu_me(mg.Process(proc, precision=mg.MG_MIXED), p)
    r = _rel(mixed, ref)
    med, _, mx = MIXED_BOUNDS[proc]
    assert np.all(np.isfinite(mixed)) and np.median(r) <= med and r.max() <= mx


@pytest.mark.parametrize("proc,precision", [
    ("e+ e- > mu+ mu-", mg.MG_FP64), ("g g > t t~", mg.MG_MIXED),
    ("g g > t t~ g g", mg.MG_FP64), ("g g > t t~ g g", mg.MG_MIXED),
], ids=["eemumu-fp64", "ggtt-mixed", "ggttgg-fp64", "ggttgg-mixed"])
def test_nan_event_stays_in_its_lane(proc, precision):
    """Bad input is not an error of the call: an event with NaN momenta gets a
    NaN |M|^2 and every other event of the batch (the same CTA included, and
    the tensor-core colour form, whose rows are independent) is bit-identical
    to the clean batch; the handle reports no error."""
    if not _have(proc):
        pytest.fail(f"{proc} is not compiled into libmg.so")
    rs, seed, _, _ = WORKLOADS[proc]
    p = process_momenta(proc, rs, 300, seed + 4000)
    h = mg.Process(proc, precision=precision)
    clean = _gpu_me(h, p)
    bad = p.copy()
    bad[5, 2, 1] = np.nan
    bad[200] = np.nan
    got = _gpu_me(h, bad)
    assert np.isnan(got[5]) and np.isnan(got[200])
    keep = np.setdiff1d(np.arange(300), [5, 200])
    np.testing.assert_array_equal(got[keep], clean[keep])
