"""bench.py's multi-GPU path runs independent replicas (the contraction of one batch never spans
GPUs); its only cross-rank logic is the timing aggregation, checked here with two gloo ranks."""
import json
import os
import socket
import subprocess
import sys

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


def test_reference_arm_runs_on_rank_zero_only():
    """`--impl reference` launched as two ranks: rank 1 exits 0 without work or output; rank 0
    times the oracle and prints one line with impl "reference", its cpu_baseline and an e2e
    object with no host-device bytes."""
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    cmd = [sys.executable, "bench.py", "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0"]
    out = {}
    for rank in (1, 0):
        env = dict(os.environ, RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE="2",
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(_free_port()))
        r = subprocess.run(cmd, cwd=root, env=env, capture_output=True, text=True, timeout=600)
        assert r.returncode == 0, r.stderr[-2000:]
        out[rank] = r.stdout.strip()
    assert out[1] == ""
    lines = out[0].splitlines()
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["steps"] == 1
    assert line["value"] > 0 and line["unit"] == "TFLOP/s" and line["higher_is_better"] is True
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"] == {"value": line["value"], "unit": "TFLOP/s", "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
