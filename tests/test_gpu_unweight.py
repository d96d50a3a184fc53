"""Device hit-or-miss unweighting (mg_unweight) against the oracle's
definition: the kept index list must be identical (integer work: bit-exact)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
from paper_2303_18244_gb300 import mg  # noqa: E402
from paper_2303_18244_gb300.inputs import process_momenta, uniforms  # noqa: E402

pytestmark = pytest.mark.gpu

TILE = 4096  # events per tile of the device kernels (256 threads x 16)


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _run(w, r, w_max):
    n = w.shape[0]
    wd = torch.from_numpy(np.ascontiguousarray(w)).cuda()
    rd = torch.from_numpy(np.ascontiguousarray(r)).cuda()
    idx = torch.full((max(n, 1),), -7, dtype=torch.int64, device="cuda")
    cnt = torch.full((1,), -7, dtype=torch.int64, device="cuda")
    mg.unweight(wd, rd, w_max, idx, cnt)
    torch.cuda.synchronize()
    k = int(cnt.item())
    return idx.cpu().numpy()[:k], k, idx.cpu().numpy()


@pytest.mark.parametrize("n", [1, 31, 257, TILE // 2 + 1, TILE - 1, TILE, TILE + 1, 5 * TILE + 333, 1 << 20, (1 << 23) + 77])
def test_matches_oracle(n):
    u = uniforms(21, 0, n, 1)[:, 0, :]
    w = 4.0 * u[:, 0] ** 2
    r = u[:, 1]
    got, k, raw = _run(w, r, 1.5)
    want = O.unweight(w, r, 1.5)
    assert k == want.size
    assert np.array_equal(got, want)
    assert np.all(raw[k:n] == -7)  # nothing written past the kept events


@pytest.mark.parametrize("n", [16384 * TILE - 3, 16392 * TILE + 5])
def test_tile_scan_at_67m_events_and_beyond(n):
    """At 67 M events (16384 tiles: the scan of the tile counts keeps 16 per
    thread in registers) and past it (17 per thread: batched loads).  Events
    with w >= w_max are always kept and w <= 0 never, so a kept set chosen in
    advance, with a pseudo-random density per tile, is the exact answer."""
    rng = np.random.default_rng(n)
    tile_p = rng.random(n // TILE + 1) ** 3  # per-tile density, many tiles nearly empty
    keep = rng.random(n) < np.repeat(tile_p, TILE)[:n]
    w = np.where(keep, 2.0, 0.0)
    r = rng.random(n)
    got, k, _ = _run(w, r, 1.0)
    want = np.flatnonzero(keep)
    assert k == want.size and np.array_equal(got, want)


@pytest.mark.parametrize("tiles", [(0,), (5,), (0, 5), (2, 3), (1, 4, 5)])
def test_kept_events_in_some_tiles_only(tiles):
    """Tiles without kept events are skipped by the write pass (their offset
    equals the next tile's, or the total for the last one): kept events in
    chosen tiles only, the last (partial) one included; w >= w_max is always
    kept and w <= 0 never."""
    n = 5 * TILE + 333
    rng = np.random.default_rng(len(tiles))
    keep = np.zeros(n, dtype=bool)
    for t in tiles:
        seg = slice(t * TILE, min(n, (t + 1) * TILE))
        keep[seg] = rng.random(keep[seg].size) < 0.3
    w = np.where(keep, 2.0, -1.0)
    got, k, raw = _run(w, rng.random(n), 1.0)
    want = np.flatnonzero(keep)
    assert k == want.size and np.array_equal(got, want)
    assert np.all(raw[k:n] == -7)


def test_all_and_none_kept():
    n = 3 * TILE + 5
    u = uniforms(22, 0, n, 1)[:, 0, 0]
    got, k, _ = _run(np.full(n, 2.0), u, 1.0)
    assert k == n and np.array_equal(got, np.arange(n))
    got, k, _ = _run(np.zeros(n), u, 1.0)
    assert k == 0


def test_empty_and_bad_args():
    cnt = torch.full((1,), -7, dtype=torch.int64, device="cuda")
    e = torch.empty(0, dtype=torch.float64, device="cuda")
    ei = torch.empty(0, dtype=torch.int64, device="cuda")
    mg.unweight(e, e, 1.0, ei, cnt)
    torch.cuda.synchronize()
    assert int(cnt.item()) == 0
    w = torch.ones(10, dtype=torch.float64, device="cuda")
    idx = torch.empty(10, dtype=torch.int64, device="cuda")
    for bad in (0.0, -1.0, float("nan")):
        with pytest.raises(mg.MGError):
            mg.unweight(w, w, bad, idx, cnt)


def test_unweighted_events_from_matrix_elements():
    # the full chain on the device: phase space, |M|^2, unweighting against
    # the largest weight of the batch; the kept set equals the oracle's on
    # the same device weights
    proc, sqrts, n = "g g > t t~", 1000.0, 200000
    h = mg.Process(proc)
    mg.good_helicities(h, torch.from_numpy(process_momenta(proc, sqrts, 1024, 1002)).cuda())
    mom = torch.empty((n, 4, 4), dtype=torch.float64, device="cuda")
    mg.rambo(h, sqrts, 2, 0, mom)
    me = torch.empty(n, dtype=torch.float64, device="cuda")
    mg.sigma(h, mom, me)
    r = torch.from_numpy(uniforms(23, 0, n, 1)[:, 0, 0].copy()).cuda()
    w_max = float(me.max().item())
    idx = torch.empty(n, dtype=torch.int64, device="cuda")
    cnt = torch.empty(1, dtype=torch.int64, device="cuda")
    mg.unweight(me, r, w_max, idx, cnt)
    torch.cuda.synchronize()
    k = int(cnt.item())
    want = O.unweight(me.cpu().numpy(), r.cpu().numpy(), w_max)
    assert np.array_equal(idx[:k].cpu().numpy(), want)
    # efficiency <w>/w_max within 5 sigma
    p = me.cpu().numpy() / w_max
    assert abs(k - p.sum()) < 5 * np.sqrt((p * (1 - p)).sum())


@pytest.mark.parametrize("w_max", [1.7, 3e38, 1e39, 2e-38])
def test_decisions_at_the_rounding_edge_and_outside_fp32(w_max):
    """Weights exactly at the FP64 product r * w_max and one ulp on either
    side (decided by the last bit: the FP64 comparison), and values outside
    the FP32 normal range (0, FP32-subnormal, beyond FP32, infinite, NaN,
    negative; w_max itself beyond FP32 or near its bottom): the kept set
    equals the oracle's definition bit for bit."""
    rng = np.random.default_rng(5)
    n = 3 * TILE + 17
    r = rng.random(n)
    p = r * w_max
    k3 = np.arange(n) % 3
    w = np.where(k3 == 0, p, np.where(k3 == 1, np.nextafter(p, np.inf), np.nextafter(p, -np.inf)))
    # far from the edge too: decided in FP32
    w[10::11] = p[10::11] * (1 + 1e-5 * (1 - 2 * (np.arange(10, n, 11) % 2)))
    for off, v in enumerate((0.0, 1e-40, 1e39, np.inf, np.nan, -1.0, 5e-39, -0.0)):
        w[off::97] = v
    r[8::97] = 0.0
    got, k, _ = _run(w, r, w_max)
    want = O.unweight(w, r, w_max)
    assert k == want.size and np.array_equal(got, want)
    assert 0 < k < n


def test_unaligned_inputs_match():
    """w and r starting 8 bytes past a 16-byte boundary (views one element
    into their buffers) take the 8-byte loads; odd lengths end on a half
    pair.  The kept set equals the oracle's either way."""
    for n in (TILE + 1, 5 * TILE + 333):
        u = uniforms(23, 0, n + 1, 1)[:, 0, :]
        w = 4.0 * u[:, 0] ** 2
        r = u[:, 1]
        wd = torch.from_numpy(w).cuda()[1:]
        rd = torch.from_numpy(r).cuda()[1:]
        assert wd.data_ptr() % 16 == 8
        idx = torch.full((n,), -7, dtype=torch.int64, device="cuda")
        cnt = torch.full((1,), -7, dtype=torch.int64, device="cuda")
        mg.unweight(wd, rd, 1.5, idx, cnt)
        torch.cuda.synchronize()
        k = int(cnt.item())
        want = O.unweight(w[1:], r[1:], 1.5)
        assert k == want.size and np.array_equal(idx.cpu().numpy()[:k], want)
