"""Host logic of the N > 1 bench path on CPU: world_size-2 gloo ranks (replicas only, so the only
cross-rank step is the max over ranks of the timed region and the whole-job rate)."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_ms = [120.0, 150.0][rank]
    t = bench.reduce_max_time(local_ms, device="cpu")
    rate = bench.whole_job_rate(world, 4096, 24, 10, t)
    out.put((rank, t, rate))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_max_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [150.0, 150.0]
    want = 2 * 4096 * 24 * 10 / 0.150
    assert all(abs(r[2] - want) < 1e-6 * want for r in res)


def test_single_rank_is_identity():
    import bench
    assert bench.reduce_max_time(12.5) == 12.5
    assert bench.whole_job_rate(1, 4096, 24, 1, 1000.0) == 4096 * 24
