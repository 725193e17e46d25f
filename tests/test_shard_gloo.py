"""The multi-rank path on CPU with the gloo backend (world size 2): ranks
simulate disjoint path ranges and all-reduce their level sums; the result
equals the single-process sums over the whole range.  The per-rank sums are
computed with the CPU oracle (same counters as the GPU kernels)."""
import os
import socket

import pytest
import torch.multiprocessing as mp

from paper_2012_09739_gb300.shard import shard_range


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, l, N, q):
    import torch.distributed as dist
    import oracle as O
    from paper_2012_09739_gb300.shard import allreduce_sums, max_over_ranks, shard_range
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    off, cnt = shard_range(N, rank, world)
    sde = O.gbm(payoff=O.PAYOFF_CALL)
    s1, s2 = O.level_sums(l, cnt, off, O.variant(), sde, 1234, O.make_tag(O.KIND_STD, l))
    tot = allreduce_sums(s1, s2, cnt)
    t = max_over_ranks(float(rank + 1))
    if rank == 0:
        q.put((tot, t))
    dist.barrier()
    dist.destroy_process_group()


def test_shard_range_partitions():
    for n in (0, 1, 7, 1000, 1001):
        for w in (1, 2, 3, 8):
            parts = [shard_range(n, r, w, offset=5) for r in range(w)]
            assert sum(c for _, c in parts) == n
            starts = [o for o, _ in parts]
            assert starts[0] == 5
            for (o0, c0), (o1, _) in zip(parts, parts[1:]):
                assert o0 + c0 == o1


def test_two_rank_gloo_sums_equal_single_process():
    import oracle as O
    l, N, world = 4, 20001, 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, l, N, q)) for r in range(world)]
    for p in procs:
        p.start()
    (s1, s2, n), tmax = q.get(timeout=120)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    sde = O.gbm(payoff=O.PAYOFF_CALL)
    r1, r2 = O.level_sums(l, N, 0, O.variant(), sde, 1234, O.make_tag(O.KIND_STD, l))
    assert n == N
    assert abs(s1 - r1) <= 1e-12 * abs(r1) and abs(s2 - r2) <= 1e-12 * r2
    assert tmax == 2.0
