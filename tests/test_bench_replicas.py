"""Multi-GPU runs are independent replicas: each rank runs the whole
workload and the job's throughput is all ranks' units over the slowest
rank's time.  Two gloo ranks on the CPU check the max-over-ranks
reduction and the aggregate."""

import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        import bench

        assert bench._dist() == (ws, rank, rank)
        # rank r took 100 (r + 1) ms for 4 steps of 3e9 units each
        out[rank] = bench.replica_throughput(100.0 * (rank + 1), 3e9, 4, ws)
    finally:
        dist.destroy_process_group()


def test_replicas_take_max_over_ranks():
    ws = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(ws, _free_port(), out), nprocs=ws, join=True)
        res = dict(out)
    assert res[0] == res[1]
    ms_step, value = res[0]
    assert ms_step == pytest.approx(200.0 / 4)
    assert value == pytest.approx(3e9 * ws / 0.05)


def test_single_rank_needs_no_process_group():
    import bench

    assert bench.replica_throughput(80.0, 1e6, 4, 1) == (20.0, pytest.approx(1e6 / 0.02))
