"""Multi-rank host logic of bench.py on CPU (gloo, world size 2): templates
are independent problems sharded round-robin with no data-path collective;
the step time is the max over ranks and the throughput sums all ranks."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    items = list(range(11))
    mine = bench.shard(items, *bench.dist_env()[:2])
    # per-rank step time and locations, reduced the way bench.py reduces them
    ms = torch.tensor([10.0 + 5.0 * rank])
    dist.all_reduce(ms, op=dist.ReduceOp.MAX)
    loc = torch.tensor([float(100 * len(mine))], dtype=torch.float64)
    dist.all_reduce(loc)
    gathered = [None] * world
    dist.all_gather_object(gathered, mine)
    q.put((rank, mine, float(ms.item()), float(loc.item()), gathered))
    dist.destroy_process_group()


def test_template_sharding_two_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    (_, a, ms0, loc0, g0), (_, b, ms1, loc1, _) = out
    assert sorted(a + b) == list(range(11)) and not set(a) & set(b)
    assert a == list(range(0, 11, 2)) and b == list(range(1, 11, 2))
    assert ms0 == ms1 == 15.0
    assert loc0 == loc1 == 1100.0
    assert g0 == [a, b]
