"""bench.py's multi-GPU path runs independent replicas (the contraction of one batch never spans
GPUs); its only cross-rank logic is the timing aggregation, checked here with two gloo ranks."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE="2")
    dist.init_process_group("gloo", rank=rank, world_size=2)
    import bench
    local = [2.0, 3.0][rank]
    value, t = bench.replica_throughput(units_per_rank=12.0, local_seconds=local, ws=2, device="cpu")
    out[rank] = (value, t)
    dist.barrier()
    dist.destroy_process_group()


def test_replica_throughput_gloo_two_ranks():
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(port, out), nprocs=2, join=True)
        res = dict(out)
    for rank in (0, 1):
        value, t = res[rank]
        assert t == 3.0                      # the slowest rank's time
        assert value == 2 * 12.0 / 3.0       # all ranks' units over that time


def test_single_rank_is_identity():
    import bench
    assert bench.replica_throughput(5.0, 2.0, 1) == (2.5, 2.0)
