"""The N > 1 path of bench.py on CPU with two gloo ranks (no GPU).

Cells are independent, so ranks take contiguous, disjoint blocks of one
global batch (weak scaling) and the only communication is the barrier and the
max-over-ranks of the timings. Two processes check that the blocks cover the
global batch exactly once, that every rank gets the slowest rank's time, and
that the whole-job value counts every rank's cells.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    import sys
    import torch.distributed as dist
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from paper_2511_10558_gb300 import synth
    per = 8
    glob = synth.cells(per * world)
    mine = bench.shard_cells(glob, rank, per)
    blocks = [None] * world
    dist.all_gather_object(blocks, mine.tolist())
    t_max = bench.max_over_ranks(1.5 + rank, torch.device("cpu"))
    value = bench.weak_value(world, per, 3, t_max)
    dist.barrier()
    dist.destroy_process_group()
    np.save(os.path.join(out_dir, f"r{rank}.npy"),
            np.array([t_max, value] + list(np.concatenate([np.array(b).ravel() for b in blocks]))))


def test_two_gloo_ranks_shard_and_reduce(tmp_path):
    import torch.multiprocessing as mp
    world = 2
    mp.start_processes(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, start_method="spawn")
    from paper_2511_10558_gb300 import synth
    glob = synth.cells(8 * world).ravel()
    for r in range(world):
        res = np.load(tmp_path / f"r{r}.npy")
        assert res[0] == 2.5                       # slowest rank's time, on every rank
        assert res[1] == pytest.approx(world * 8 * 3 / 2.5)
        np.testing.assert_array_equal(res[2:], glob)  # blocks in rank order = the global batch
