"""bench.py on the CPU: the multi-rank path (replicas, weak scaling), where
two gloo ranks aggregate the slowest rank's time and the sum of the updates,
and the reference arm's JSON line."""
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


def test_reference_arm_prints_its_json_line():
    """`bench.py --impl reference` (the CPU oracle, timed as it stands) prints
    one JSON line with the contract's keys; the cavity keeps it to a second."""
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--workload", "cavity", "--steps", "1",
                        "--warmup", "0"], cwd=root, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == "cell-velocity-node updates/s"
    assert d["value"] > 0 and d["higher_is_better"] is True and d["n_gpus"] == 1
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["config"]["workload"].startswith("cavity")
