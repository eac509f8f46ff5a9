"""The N > 1 path of the benchmark on CPU: two gloo ranks shard frames
disjointly and agree on the max-over-ranks time."""
import os
import socket

import pytest
import torch.multiprocessing as mp

from paper_2601_19901_gb300 import multigpu


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    frames = multigpu.rank_frames(rank, world, 5, start=3)
    mine = 1.5 + rank          # a rank's timed total
    mx = multigpu.max_over_ranks(mine)
    out.put((rank, frames, mx))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_frames_and_reduce_max():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    frames = [set(f) for _, f, _ in res]
    assert not (frames[0] & frames[1])
    assert all(len(f) == 5 for f in frames)
    assert [mx for _, _, mx in res] == [2.5, 2.5]
    assert multigpu.job_rate(world, 10, 2.5) == 8.0


def test_single_process_is_identity():
    assert multigpu.max_over_ranks(3.25) == 3.25
    assert multigpu.rank_frames(0, 1, 3) == [0, 1, 2]
    with pytest.raises(ValueError):
        multigpu.rank_frames(2, 2, 1)
