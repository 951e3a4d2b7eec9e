"""Multi-process paths on CPU (gloo, world size 2): the job sharding used for
batches and served streams is a partition with no data exchange, and the
slowest-rank timing reduction of the bench works over gloo."""
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


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2606_16959_gb300 import serve
    mine = serve.shard_jobs(list(range(23)), rank, world)
    got = [None] * world
    dist.all_gather_object(got, mine)
    t = torch.tensor([float(rank + 1)], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    if rank == 0:
        q.put((got, float(t.item())))
    dist.destroy_process_group()


def test_shard_jobs_partition_two_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got, tmax = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    flat = sorted(x for part in got for x in part)
    assert flat == list(range(23))
    assert not set(got[0]) & set(got[1])
    assert tmax == 2.0


def test_shard_jobs_single_and_errors():
    from paper_2606_16959_gb300 import serve
    assert serve.shard_jobs([1, 2, 3], 0, 1) == [1, 2, 3]
    with pytest.raises(ValueError):
        serve.shard_jobs([1], 2, 2)
