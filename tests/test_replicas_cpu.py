"""Multi-GPU replica path, exercised with two gloo ranks on the CPU: the work split is
disjoint and complete, and the timing aggregation takes the slowest rank and the total."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_1706_07263_gb300 import replicas  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = list(replicas.shard(37, rank, world))
        ms, units = replicas.aggregate(10.0 + 5.0 * rank, len(mine))
        gathered = [None] * world
        dist.all_gather_object(gathered, mine)
        q.put((rank, ms, units, gathered))
    finally:
        dist.destroy_process_group()


def test_two_ranks_split_and_aggregate():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, units, gathered in res:
        assert ms == 15.0                      # the slowest rank's time
        assert units == 37                     # every frame counted once
        flat = sorted(u for part in gathered for u in part)
        assert flat == list(range(37))         # disjoint and complete


def test_single_process_is_identity():
    assert replicas.aggregate(3.5, 7) == (3.5, 7)
    assert list(replicas.shard(5, 0, 1)) == [0, 1, 2, 3, 4]
    with pytest.raises(ValueError):
        replicas.shard(5, 2, 2)
