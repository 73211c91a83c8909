"""Multi-rank host logic of bench.py on CPU (gloo, world size 2): each rank
solves its own column, the job's time is the slowest rank's, and its rate is
world_size steps per that time."""
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


def _worker(rank, ws, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        assert bench._dist() == (ws, rank, rank)
        ms_local = 100.0 + 50.0 * rank                   # rank 1 is the slower one
        rate, ms = bench.whole_job_rate(ms_local, ws, "cpu")
        bench._barrier(ws)
        out[rank] = (rate, ms, bench.replica_seed(rank))
    finally:
        dist.destroy_process_group()


def test_whole_job_rate_two_ranks():
    ws = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(ws, port, out), nprocs=ws, join=True)
        res = dict(out)
    assert set(res) == {0, 1}
    for rank in (0, 1):
        rate, ms, _ = res[rank]
        assert ms == pytest.approx(150.0)                # max over ranks
        assert rate == pytest.approx(ws * 1e3 / 150.0)   # whole-job steps/s
    assert res[0][2] != res[1][2]                        # each rank its own column


def test_single_rank_is_local():
    sys.path.insert(0, ROOT)
    import bench
    rate, ms = bench.whole_job_rate(40.0, 1, "cpu")
    assert ms == 40.0 and rate == pytest.approx(25.0)
