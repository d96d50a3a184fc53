"""Multi-rank host logic (event sharding, barrier, max-over-ranks timing) on
CPU with the gloo backend, world size 2."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_2303_18244_gb300.inputs import process_momenta  # noqa: E402
from paper_2303_18244_gb300.shard import event_block, max_over_ranks  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        first, n = event_block(rank, world, 64)
        p = process_momenta("g g > t t~ g", 1200.0, n, 9, first_event=first)
        np.save(os.path.join(out_dir, f"mom{rank}.npy"), p)
        # each rank reports a different "time"; every rank must see the maximum
        t = max_over_ranks([1.0 + rank, 5.0 - rank])
        np.save(os.path.join(out_dir, f"max{rank}.npy"), np.array(t))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_rank_sharding_and_max(tmp_path):
    world = 2
    mp.start_processes(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, start_method="spawn")
    whole = process_momenta("g g > t t~ g", 1200.0, 128, 9)
    parts = [np.load(tmp_path / f"mom{r}.npy") for r in range(world)]
    # the two blocks are disjoint and together equal the single-process stream
    np.testing.assert_array_equal(np.concatenate(parts), whole)
    for r in range(world):
        np.testing.assert_array_equal(np.load(tmp_path / f"max{r}.npy"), [2.0, 5.0])


def test_event_block_bounds():
    assert event_block(0, 1, 10) == (0, 10)
    assert event_block(3, 4, 10) == (30, 10)
    with pytest.raises(ValueError):
        event_block(4, 4, 10)
