"""The N>1 bench path (one replica per rank, barrier, max-over-ranks timing) on gloo, CPU only."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, ws, port, q):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws))
    sys.path.insert(0, ROOT)
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench

    ms = 100.0 + 10.0 * rank                     # each replica's own time
    worst = bench.max_over_ranks(ms, dist, None)
    bench.barrier(dist)
    v = bench.whole_job_mflups(1_000_000, ws, 50, worst)
    q.put((rank, worst, v))
    dist.destroy_process_group()


@pytest.mark.parametrize("ws", [2])
def test_replicas_max_over_ranks_gloo(ws):
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, ws, port, q)) for r in range(ws)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(ws)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    worst = 100.0 + 10.0 * (ws - 1)
    for rank, w, v in out:
        assert w == worst
        assert abs(v - 1_000_000 * ws * 50 / (worst / 1e3) / 1e6) < 1e-9
