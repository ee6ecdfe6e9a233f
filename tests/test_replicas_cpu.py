"""The N > 1 path of bench.py on CPU: two gloo ranks run as replicas; the
job time is the maximum over ranks and the job rate counts every rank's units."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, out):
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(ws), "LOCAL_RANK": str(rank)})
    assert bench.dist_setup() == (ws, rank, rank)
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    # per-rank step times (ms): rank 1 is slower on the first, rank 0 on the second
    mine = [10.0 + 5.0 * rank, 20.0 - 3.0 * rank, 0.0]
    got = bench.max_over_ranks(mine, ws, torch.device("cpu"))
    dist.barrier()
    out[rank] = got
    dist.destroy_process_group()


def test_two_gloo_replicas_take_the_slowest_rank():
    port = _free_port()
    ws = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(ws, port, out), nprocs=ws, join=True)
        res = dict(out)
    assert res[0] == res[1] == [15.0, 20.0, 0.0]
    sys.path.insert(0, ROOT)
    import bench
    # 2244 subdomains per rank, 20 steps in 15 ms of job time on 2 replicas
    assert abs(bench.job_rate(2244, 20, ws, 15.0) - 2244 * 20 * 2 / 0.015) < 1e-6
