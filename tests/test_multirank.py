"""The N > 1 timing path of bench.py (replicas only, no data-path
collective): barrier and max over ranks, on world_size 2 with gloo on CPU."""
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
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench

    assert bench.dist_env() == (ws, rank, rank)
    bench.barrier(ws)
    t = bench.max_over_ranks(10.0 + rank, ws)      # per-rank elapsed times
    out[rank] = t
    dist.destroy_process_group()


def test_max_over_ranks_world_size_2():
    ws = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    procs = [ctx.Process(target=_worker, args=(r, ws, port, out)) for r in range(ws)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(60)
        assert p.exitcode == 0
    assert dict(out) == {0: 11.0, 1: 11.0}
