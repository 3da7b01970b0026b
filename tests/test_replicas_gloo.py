"""Host logic of the N-replica benchmark (one process per GPU, no collective on the
data path): max-over-ranks timing and the whole-job aggregate, on 2 gloo ranks."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    ms = 10.0 + 5.0 * rank                      # rank 1 is slower
    value, mx = bench.aggregate_value(1e9, ms, ws)
    bench.barrier(ws)
    q.put((rank, value, mx))
    dist.destroy_process_group()


def test_two_rank_aggregate():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    out = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, value, mx in out:
        assert mx == 15.0                        # the slowest rank's time
        assert value == pytest.approx(2 * 1e9 / 15e-3 / 1e9)
