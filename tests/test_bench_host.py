"""Host-side logic of bench.py (no GPU): the oracle's CPU-baseline sample,
and the reference arm launched on two ranks.

The sample is a prefix of the workload, compared event by event with the
GPU outputs of the same workload, so it may never hold more events than the
workload itself, however fast the oracle is.
"""
import numpy as np

import bench
import oracle as O
from paper_2303_18244_gb300.inputs import process_momenta


def test_oracle_sample_capped_at_the_workload():
    v, cores, n, dt, one, ref = bench.time_oracle("e+ e- > mu+ mu-", 500.0, 1, 0, budget_s=2.0, max_events=3000)
    assert n <= 3000 and ref.shape == (n,) and cores >= 1 and v > 0 and one > 0


def test_oracle_sample_is_the_workload_prefix():
    n_max = 200
    _, _, n, _, _, ref = bench.time_oracle("g g > t t~", 1000.0, 2, 0, budget_s=0.5, one_core=False,
                                           max_events=n_max)
    assert 1 <= n <= n_max
    p = process_momenta("g g > t t~", 1000.0, n, 2)
    np.testing.assert_array_equal(ref, O.me("g g > t t~", p))


def test_reference_arm_under_torchrun_prints_one_line_from_rank_zero():
    """`bench.py --impl reference` launched like the multi-GPU bench (two
    ranks under torch.distributed.run): rank 0 times the oracle and prints
    the one JSON line, the other rank exits 0 without work."""
    import json
    import os
    import socket
    import subprocess
    import sys

    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
                        "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--impl",
                        "reference", "--gpus", "2", "--steps", "1", "--warmup", "0"],
                       cwd=root, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [json.loads(x) for x in r.stdout.splitlines() if x.startswith("{")]
    assert len(lines) == 1
    d = lines[0]
    assert d["impl"] == "reference" and d["value"] > 0 and d["unit"] == "MEs/s" and d["steps"] == 1
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["value"] == d["value"] and d["e2e"]["h2d_bytes_per_step"] == 0
