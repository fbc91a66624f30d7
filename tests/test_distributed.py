"""Multi-rank path on CPU (gloo, world size 2): the chain shards and the final
exchange of the best cost and assignment."""
import os
import socket

import numpy as np
import pytest

from paper_2311_02101_gb300 import distributed as dd


def test_shard_offsets_cover_the_ensemble():
    shards = [dd.shard_of(r, 4, 1024) for r in range(4)]
    assert shards == [(0, 4096), (1024, 4096), (2048, 4096), (3072, 4096)]
    with pytest.raises(ValueError):
        dd.shard_of(0, 2, 100)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, case, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    cost, chain, assign = case[rank]
    got = dd.reduce_best(cost, chain, np.array(assign, np.uint8))
    out.put((rank, got[0], got[1], got[2].tolist()))
    dist.destroy_process_group()


@pytest.mark.parametrize("case,expect", [
    # rank 1 holds the lower cost
    ({0: (17, 5, [1, 0, 1]), 1: (12, 1030, [0, 0, 1])}, (12, 1030, [0, 0, 1])),
    # equal costs: the lower global chain index wins
    ({0: (9, 700, [1, 1, 1]), 1: (9, 1024, [0, 1, 0])}, (9, 700, [1, 1, 1])),
])
def test_reduce_best_two_ranks(case, expect):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, case, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, c, ch, a in res:
        assert (c, ch, a) == expect, rank


def _rank_dies(rank, world, port, out):
    """Rank 1 leaves between rounds, before the final exchange (as a rank
    whose host fails); rank 0's exchange must then fail with an error within
    the process group's timeout instead of waiting forever."""
    import datetime
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world,
                            timeout=datetime.timedelta(seconds=10))
    if rank == 1:
        os._exit(3)
    try:
        dd.reduce_best(5, 0, np.zeros(4, np.uint8))
        out.put((rank, "returned"))
    except Exception as e:  # the collective reports the lost peer
        out.put((rank, "error: " + type(e).__name__))


def test_reduce_best_reports_a_lost_rank():
    import time
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_dies, args=(r, 2, port, q)) for r in range(2)]
    t0 = time.monotonic()
    for p in procs:
        p.start()
    rank, status = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
    assert rank == 0 and status.startswith("error"), status
    assert procs[1].exitcode == 3
    assert time.monotonic() - t0 < 100
