"""The multi-rank host path of bench.py on CPU: two gloo ranks (replicas) agree on the
slowest rank's time and on a throughput that counts both ranks' primitives."""
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
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    assert bench.dist_env()[:2] == (ws, rank)
    local_ms = [120.0, 150.0][rank]
    t = bench.max_over_ranks(local_ms, ws, torch.device("cpu"))
    out[rank] = (t, bench.replica_throughput(ws, 768000, 5, t))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_replicas_take_the_slowest_rank():
    ws = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        procs = [ctx.Process(target=_rank, args=(r, ws, port, out)) for r in range(ws)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    assert res[0] == res[1]
    t, v = res[0]
    assert t == 150.0
    assert v == pytest.approx(2 * 768000 * 5 / 0.150)


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(42.0, 1, None) == 42.0
    assert bench.replica_throughput(1, 1000, 2, 500.0) == pytest.approx(4000.0)
