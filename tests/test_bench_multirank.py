"""The N > 1 path of bench.py on CPU: world_size 2 over gloo.  The bench runs
independent replicas (no data-path collective); the only collective is the
max over ranks of the timed interval, and the job value counts every rank's
work over the slowest rank's time."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, out):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    ms = 10.0 + 5.0 * rank
    m = bench.max_over_ranks(ms, ws)
    v = bench.job_value(1000, 5, m, ws)
    out[rank] = (m, v)
    dist.destroy_process_group()


def test_max_over_ranks_and_job_value_world_size_2():
    ws, port = 2, _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_worker, args=(ws, port, out), nprocs=ws, join=True)
        res = dict(out)
    for r in range(ws):
        m, v = res[r]
        assert m == 15.0
        assert v == pytest.approx(2 * 1000 * 5 / 15e-3)


def test_single_rank_is_identity():
    import bench
    assert bench.max_over_ranks(3.0, 1) == 3.0
    assert bench.job_value(10, 5, 2.0, 1) == pytest.approx(10 * 5 / 2e-3)
