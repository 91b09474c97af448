"""The N>1 host logic of bench.py on CPU with two gloo ranks: every rank gets
its own block-aligned slice of the binade (weak scaling, no data-path
collective) and the step time is the maximum over ranks."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    import workloads as wl
    job = bench.rank_job(wl.plain_job(), rank)
    t = torch.tensor([float(rank + 1) * 1.5], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    out.put((rank, job.start, job.count, float(t.item())))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_get_disjoint_slices_and_max_time():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, s0, c0, t0), (r1, s1, c1, t1) = res
    assert c0 == c1 == 1 << 36
    assert s0 % (1 << 24) == 0 and s1 % (1 << 24) == 0
    assert s0 + c0 <= s1 or s1 + c1 <= s0           # disjoint slices
    assert max(s0, s1) + c0 <= 1 << 52               # inside the binade
    assert t0 == t1 == 3.0                           # max over ranks
