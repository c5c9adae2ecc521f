"""The multi-rank plumbing of bench.py on CPU: two gloo ranks (127.0.0.1)
agree on the barrier and take the maximum of their step times; the whole-job
value aggregates every rank's units (weak scaling, independent replicas); a
slowdown seen by one rank makes every rank measure again."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    bench.barrier(world)
    ms = bench.allreduce_max(100.0 + 50.0 * rank, world)
    flops = bench.step_flops(1024, 1)
    value = world * flops * 2 / (ms / 1e3) / 1e9  # 2 steps, as bench computes it
    # the re-measure decision is collective: rank 1 alone saw a slowdown
    clocks = {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["hw_slowdown"] if rank == 1 else []}
    again = bench.allreduce_max(1.0 if bench.clocks_rejected(clocks) else 0.0, world) > 0
    q.put((rank, ms, value, again))
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_max_time():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    times = {r: ms for r, ms, _, _ in out}
    assert times == {0: 150.0, 1: 150.0}
    vals = {v for _, _, v, _ in out}
    assert len(vals) == 1
    assert all(again for _, _, _, again in out)   # both ranks measure again
