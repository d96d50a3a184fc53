"""Serving loop: continuous batching of requests of several processes and
sizes; each result is the same alone and in the mix and matches the oracle;
memory admission counts the two-phase workspace; host and device buffers."""
import numpy as np
import pytest

import oracle as O

torch = pytest.importorskip("torch")

from paper_2303_18244_gb300 import mg  # noqa: E402
from paper_2303_18244_gb300.inputs import process_momenta, uniforms  # noqa: E402
from mixed_bounds import MIXED_BOUNDS  # noqa: E402

pytestmark = pytest.mark.gpu

PROCS = {"e+ e- > mu+ mu-": 500.0, "g g > t t~": 1000.0, "g g > t t~ g": 1200.0, "g g > t t~ g g": 1500.0,
         "g g > t t~ g g g": 2000.0, "u u~ > t t~ g g": 1500.0}


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _alone(h, mom):
    # the test's own stream only: a device-wide synchronisation is not
    # permitted while the server thread captures a graph
    s = torch.cuda.current_stream()
    d = torch.from_numpy(mom).cuda()
    out = torch.empty(mom.shape[0], dtype=torch.float64, device="cuda")
    mg.sigma(h, d, out, s)
    s.synchronize()
    return out.cpu().numpy()


def _requests(n, seed):
    u = uniforms(seed, 0, n, 1)[:, 0, :]
    reqs = []
    for i in range(n):
        proc = list(PROCS)[int(u[i, 0] * len(PROCS))]
        nevt = int(np.exp(np.log(100) + u[i, 1] * (np.log(9000) - np.log(100))))
        reqs.append((proc, process_momenta(proc, PROCS[proc], nevt, seed, first_event=1000 * i)))
    return reqs


@pytest.mark.parametrize("precision", [mg.MG_MIXED, mg.MG_FP64], ids=["mixed", "fp64"])
@pytest.mark.parametrize("graphs", [1, 0], ids=["graphs", "plain"])
def test_results_same_alone_and_in_the_mix(precision, graphs):
    handles = {p: mg.Process(p, precision=precision) for p in PROCS}
    reqs = _requests(24, 5)
    srv = mg.Server(n_streams=4, use_graphs=graphs, min_bucket=256, max_bucket=4096)
    outs, ids = [], []
    for proc, mom in reqs:  # all submitted at once: they overlap on the device
        o = np.full(mom.shape[0], np.nan)
        outs.append(o)
        ids.append(srv.submit(handles[proc], mom, o))
    for rid, (proc, mom), o in zip(ids, reqs, outs):
        rc, st = srv.poll(rid, 60_000_000)
        assert rc == mg.MG_OK and st.status == 0
        assert st.nevt == mom.shape[0] and st.padded_nevt >= st.nevt
        assert st.latency_us > 0 and st.done_us >= st.start_us >= st.submit_us
        np.testing.assert_array_equal(o, _alone(handles[proc], mom))
    srv.close()


def test_memory_admission_and_errors():
    h = mg.Process("g g > t t~ g g", precision=mg.MG_MIXED)
    # budget for one 4096-event chunk of this process at a time: requests queue
    per_evt = 6 * 32 + 8
    srv = mg.Server(n_streams=4, mem_budget_bytes=4096 * per_evt, min_bucket=256, max_bucket=4096)
    moms = [process_momenta("g g > t t~ g g", 1500.0, n, 7, first_event=20000 * i)
            for i, n in enumerate((5000, 300, 4096))]
    outs = [np.empty(m.shape[0]) for m in moms]
    ids = [srv.submit(h, m, o) for m, o in zip(moms, outs)]
    for rid, m, o in zip(ids, moms, outs):
        rc, st = srv.poll(rid, 60_000_000)
        assert rc == mg.MG_OK
        np.testing.assert_array_equal(o, _alone(h, m))
    with pytest.raises(mg.MGError) as ei:
        srv.poll(ids[0], 0)  # already collected
    assert ei.value.code == -7
    srv.close()
    # a chunk that can never fit the budget is refused at submit
    srv = mg.Server(mem_budget_bytes=1000, min_bucket=256, max_bucket=4096)
    m = process_momenta("g g > t t~ g g", 1500.0, 10, 7)
    with pytest.raises(mg.MGError) as ei:
        srv.submit(h, m, np.empty(10))
    assert ei.value.code == -3
    srv.close()


def test_shutdown_with_requests_in_flight():
    h = mg.Process("g g > t t~ g g", precision=mg.MG_FP64)
    srv = mg.Server(n_streams=2, min_bucket=256, max_bucket=8192)
    moms = [process_momenta("g g > t t~ g g", 1500.0, 8192, 11, first_event=8192 * i) for i in range(6)]
    outs = [np.empty(8192) for _ in moms]
    for m, o in zip(moms, outs):
        srv.submit(h, m, o)
    srv.close()  # waits for in-flight work, fails what is still queued; must not hang


def test_zero_event_request():
    h = mg.Process("g g > t t~")
    srv = mg.Server()
    m = np.zeros((0, 4, 4))
    rid = srv.submit(h, m, np.empty(0))
    rc, st = srv.poll(rid, 1_000_000)
    assert rc == mg.MG_OK and st.nevt == 0
    srv.close()


def test_new_handles_after_destroyed_ones():
    """Handles destroyed once their requests completed, and new ones created
    (the allocator often hands out the freed address again): each request
    runs its own handle's process and constants, never a graph the server
    captured for an earlier handle."""
    srv = mg.Server(n_streams=1, min_bucket=256, max_bucket=1024)
    cases = [("g g > t t~", process_momenta("g g > t t~", 1000.0, 300, 5)),
             ("g g > t t~ g", process_momenta("g g > t t~ g", 1200.0, 300, 6))]
    for _ in range(3):
        for proc, mom in cases:
            h = mg.Process(proc)
            o = np.full(mom.shape[0], np.nan)
            rc, st = srv.poll(srv.submit(h, mom, o), 60_000_000)
            assert rc == mg.MG_OK and st.status == 0
            np.testing.assert_array_equal(o, _alone(h, mom))
            h.close()
    srv.close()


def _oracle_check(proc, mom, got, precision, idx):
    ref = O.me(proc, mom[idx])
    r = np.abs(got[idx] / ref - 1)
    if precision == mg.MG_FP64:
        bad = np.nonzero(r > 1e-12)[0]
        if bad.size:  # the oracle's long-double build decides
            r[bad] = np.abs(got[idx][bad] / O.me(proc, mom[idx][bad], extended=True) - 1)
        assert r.max() <= 1e-12, (proc, r.max())
    else:
        assert r.max() <= MIXED_BOUNDS[proc][2], (proc, r.max())


@pytest.mark.parametrize("precision", [mg.MG_MIXED, mg.MG_FP64], ids=["mixed", "fp64"])
def test_served_results_match_the_oracle(precision):
    """A stream of requests of every process, host and device buffers mixed,
    all in flight together: sampled events of every request (its first and
    last event, the edges of every 4096-event piece, random ones) against the
    FP64 oracle -- the padding, the piece offsets, the staging copies and the
    graph replays are checked against an independent evaluation."""
    handles = {p: mg.Process(p, precision=precision) for p in PROCS}
    for p, hh in handles.items():
        mg.good_helicities(hh, torch.from_numpy(process_momenta(p, PROCS[p], 1024, 1000 + len(p))).cuda())
    reqs = _requests(15, 9)
    srv = mg.Server(n_streams=3, min_bucket=256, max_bucket=4096)
    outs, ids = [], []
    for i, (proc, mom) in enumerate(reqs):
        if i % 3 == 1:  # device-resident momenta and results
            d_in = torch.from_numpy(mom).cuda()
            o = torch.full((mom.shape[0],), float("nan"), dtype=torch.float64, device="cuda")
            outs.append(o)
            ids.append(srv.submit(handles[proc], d_in, o))
            outs[-1] = (o, d_in)
        else:
            o = np.full(mom.shape[0], np.nan)
            outs.append(o)
            ids.append(srv.submit(handles[proc], mom, o))
    rng = np.random.default_rng(3)
    for rid, (proc, mom), o in zip(ids, reqs, outs):
        rc, st = srv.poll(rid, 120_000_000)
        assert rc == mg.MG_OK and st.status == 0
        got = o[0].cpu().numpy() if isinstance(o, tuple) else o
        assert np.all(np.isfinite(got))
        n = mom.shape[0]
        edges = [0, n - 1] + [k for b in range(4096, n, 4096) for k in (b - 1, b)]
        idx = np.unique(np.concatenate([edges, rng.integers(0, n, 6)]))
        _oracle_check(proc, mom, got, precision, idx)
    srv.close()


def test_workspace_bytes():
    """mg_sigma_workspace_bytes: the two-phase mixed g g > t t~ g g g path takes
    as many helicities of 120 complex FP32 flows per event (events padded to
    128) as fit 1 GiB; every other path takes nothing."""
    h = mg.Process("g g > t t~ g g g", precision=mg.MG_MIXED)
    for nevt in (1, 300, 65536):
        ld = (nevt + 127) // 128 * 128
        per_hel = 120 * ld * 8
        hs = max(1, min(128, (1 << 30) // per_hel))
        assert mg.sigma_workspace_bytes(h, nevt) == hs * per_hel
    assert mg.sigma_workspace_bytes(h, 0) == 0
    for proc, prec in (("g g > t t~ g g g", mg.MG_FP64), ("g g > t t~ g g", mg.MG_MIXED),
                       ("g g > t t~ g g g", mg.MG_MIXED_PAPER)):
        assert mg.sigma_workspace_bytes(mg.Process(proc, precision=prec), 65536) == 0


def test_two_phase_chunk_waits_for_its_workspace():
    """A budget with room for one g g > t t~ g g g mixed piece and its
    workspace: the second request starts only after the first is done, and
    both are correct."""
    proc = "g g > t t~ g g g"
    h = mg.Process(proc, precision=mg.MG_MIXED)
    n = 2048
    one = n * (7 * 32 + 8) + mg.sigma_workspace_bytes(h, n)
    srv = mg.Server(n_streams=4, mem_budget_bytes=one + 1000, min_bucket=256, max_bucket=n)
    moms = [process_momenta(proc, 2000.0, n, 13, first_event=n * i) for i in range(2)]
    outs = [np.full(n, np.nan) for _ in moms]
    ids = [srv.submit(h, m, o) for m, o in zip(moms, outs)]
    sts = []
    for rid in ids:
        rc, st = srv.poll(rid, 120_000_000)
        assert rc == mg.MG_OK
        sts.append(st)
    assert sts[1].start_us >= sts[0].done_us
    for m, o in zip(moms, outs):
        np.testing.assert_array_equal(o, _alone(h, m))
    srv.close()
