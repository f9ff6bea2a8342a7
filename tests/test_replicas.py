"""Host logic of the multi-GPU path on CPU: two gloo ranks shard independent lattices
with no data-path collective and reduce only their timings."""
import os

import numpy as np
import pytest

from paper_1610_07114_gb300 import replicas
from paper_1610_07114_gb300 import workloads as W


def test_shard_is_a_balanced_partition():
    rng = np.random.default_rng(3)
    work = [int(x) for x in rng.integers(1, 10_000, size=257)]
    for world in (1, 2, 3, 8):
        shares = [replicas.shard(work, world, r) for r in range(world)]
        flat = sorted(i for s in shares for i in s)
        assert flat == list(range(len(work)))
        loads = [sum(work[i] for i in s) for s in shares]
        assert max(loads) <= sum(work) / world + max(work)


def test_shard_of_the_batched_sweep_by_nodes():
    cases = W.batched_rb_sweep(count=64, storage="fp16")
    nodes = [c["nx"] * c["ny"] for c, _ in cases]
    a, b = replicas.shard(nodes, 2, 0), replicas.shard(nodes, 2, 1)
    assert not set(a) & set(b) and len(a) + len(b) == 64
    la, lb = sum(nodes[i] for i in a), sum(nodes[i] for i in b)
    assert abs(la - lb) <= max(nodes)


def test_shard_rejects_bad_rank():
    with pytest.raises(ValueError):
        replicas.shard([1, 2], 2, 2)


def _rank_main(rank, world, port, out):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w, r, _ = replicas.dist_env()
    cases = W.batched_rb_sweep(count=32, storage="fp16")
    nodes = [c["nx"] * c["ny"] for c, _ in cases]
    mine = replicas.shard(nodes, w, r)
    replicas.barrier(w)
    t = 1.0 + r  # stands in for a rank's timed region
    tmax = replicas.max_over_ranks(t, w)
    total = replicas.sum_over_ranks(float(sum(nodes[i] for i in mine)), w)
    out.put((r, mine, tmax, total, sum(nodes)))
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_reduce_timings():
    import socket

    import torch.multiprocessing as mp

    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, m0, t0, s0, n0), (r1, m1, t1, s1, n1) = res
    assert t0 == t1 == 2.0  # the max over ranks, on both ranks
    assert s0 == s1 == n0 == n1  # the shares cover every node once
    assert not set(m0) & set(m1)
