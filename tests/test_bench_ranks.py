"""The multi-rank path of bench.py (replicas, weak scaling) on the CPU: two
gloo ranks aggregate the slowest rank's time and the sum of the updates."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    ms = [12.5, 20.0][rank]
    upd = [1.0e9, 3.0e9][rank]
    out[rank] = bench.aggregate(ms, upd, ws)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_aggregation_gloo():
    ws = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(ws, _free_port(), out), nprocs=ws, join=True)
        res = dict(out)
    for r in range(ws):
        t, u = res[r]
        assert t == 20.0 and u == 4.0e9


def test_single_rank_is_identity():
    import bench
    assert bench.aggregate(7.0, 5.0, 1) == (7.0, 5.0)
