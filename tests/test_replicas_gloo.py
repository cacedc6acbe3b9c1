"""Multi-GPU host logic of bench.py on CPU: world-size-2 gloo ranks as independent replicas.

The path does not shard (each rank evolves its own instances), so the only collective is the
max-over-ranks of the timed region; this checks it and the whole-job throughput on two CPU ranks."""
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


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_ms = 100.0 * (rank + 1)                 # rank 1 is the slow replica
    mx = bench.reduce_max_ms(local_ms, dist, "cpu")
    value = bench.replica_throughput(15, world, mx)
    out[rank] = (mx, value)
    dist.barrier()
    dist.destroy_process_group()


def test_replica_timing_is_max_over_ranks():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0] == res[1]
    mx, value = res[0]
    assert mx == 200.0
    assert abs(value - 15 * 2 / 0.2) < 1e-9
