"""The multi-rank path of bench.py on CPU: two gloo ranks (weak scaling,
no data-path collective; the only collectives are the barrier and the
max-over-ranks reduction of the timed region)."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, _ = bench.dist_env()
    dist.barrier()
    local_ms = 10.0 + 5.0 * r          # rank 1 is the slow one
    mx = bench.reduce_max(local_ms, w)
    out[r] = (mx, bench.whole_job_rate(64 * 20, w, mx))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_reduce_max_and_weak_scaling_value():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    assert out[0] == out[1]
    mx, rate = out[0]
    assert mx == 15.0
    assert rate == pytest.approx(2 * 64 * 20 / 0.015)
