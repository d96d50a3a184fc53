"""Serving loop: continuous batching of requests of several processes and
sizes; each result is the same alone and in the mix; memory admission."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2303_18244_gb300 import mg  # noqa: E402
from paper_2303_18244_gb300.inputs import process_momenta, uniforms  # noqa: E402

pytestmark = pytest.mark.gpu

PROCS = {"e+ e- > mu+ mu-": 500.0, "g g > t t~": 1000.0, "g g > t t~ g": 1200.0, "g g > t t~ g g": 1500.0}


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _alone(h, mom):
    d = torch.from_numpy(mom).cuda()
    out = torch.empty(mom.shape[0], dtype=torch.float64, device="cuda")
    mg.sigma(h, d, out)
    torch.cuda.synchronize()
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
