"""The multi-rank path of the benchmark on CPU: two gloo ranks, each with its
own seeded problem, combined into whole-job figures (slowest rank's time,
states summed over ranks) with no collective on the data path."""
import os
import socket
import sys

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        assert bench.dist_env() == (ws, rank, rank)
        w = bench.workload("tiny", rank)
        # per-rank figures: rank r took (1 + r) s and converged 8 + r states
        got = bench.combine_ranks(dist, torch.device("cpu"), 1.0 + rank, 8 + rank, 2.0 + rank, 8 + rank)
        np.save(os.path.join(out, f"rank{rank}.npy"),
                np.array([*got, w.seed, float(np.sum(w.vloc))], dtype=np.float64))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_combine_whole_job(tmp_path):
    ws = 2
    mp.start_processes(_rank_main, args=(ws, _free_port(), str(tmp_path)), nprocs=ws, start_method="spawn")
    r = [np.load(tmp_path / f"rank{i}.npy") for i in range(ws)]
    for x in r:
        assert x[0] == pytest.approx(2.0)        # slowest rank's device time
        assert x[1] == 8 + 9                     # states of both ranks
        assert x[2] == pytest.approx(3.0)        # slowest rank's end-to-end time
        assert x[3] == 8 + 9
    # independent problems: the ranks' instances differ (seed and potential)
    assert r[0][4] != r[1][4]
    assert r[0][5] != pytest.approx(r[1][5])


def test_single_rank_needs_no_collective():
    import bench
    assert bench.combine_ranks(None, None, 1.5, 7, 2.5, 7) == (1.5, 7, 2.5, 7)
