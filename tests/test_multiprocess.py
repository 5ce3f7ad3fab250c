"""The N > 1 path of bench.py on CPU: replicas with a barrier and
max-over-ranks timing, world size 2 over gloo (no GPU, no data-path
collective: the solver does not shard)."""
import os
import socket

import pytest
import torch
import torch.distributed as td
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    td.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms_local = 100.0 * (rank + 1)       # rank 1 is the slow replica
    ms, value = bench.aggregate(ms_local, 64, 3, world, td, "cpu")
    td.barrier()
    out.put((rank, ms, value))
    td.destroy_process_group()


def test_replicas_max_over_ranks_gloo():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, value in res:
        assert ms == 200.0                      # slowest rank
        assert value == pytest.approx(2 * 64 * 3 / 0.2)
