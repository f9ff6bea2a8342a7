"""Slab decomposition along y without a GPU: the split and exchange plan of
paper_1610_07114_gb300.slabs, driven by the FP64 oracle, must reproduce the undivided
lattice bit for bit -- in one process, and with two gloo ranks that each hold one slab
and swap their ghost rows by point-to-point messages.

The oracle's state is the populations at each node after streaming and the wall
schemes (its step collides, pushes, then rebuilds wall rows), so a ghost-row copy here
moves node states; the CUDA path copies stored post-collision rows instead.  Either
way a row's next state depends on the two rows on each side, which is what the plan
rests on.
"""
import os
import socket

import numpy as np
import pytest

import oracle
from paper_1610_07114_gb300 import slabs as S
from paper_1610_07114_gb300 import workloads as W


def test_plan_partitions_the_rows_and_places_ghosts():
    for ny, parts, ghost, per in [(32, 2, 2, False), (33, 3, 4, True), (128, 4, 8, False), (10, 2, 2, True)]:
        sl = S.plan(ny, parts, ghost, per)
        assert [s.lo for s in sl] == sorted(s.lo for s in sl)
        assert sum(s.own for s in sl) == ny and sl[0].lo == 0 and sl[-1].hi == ny
        for a, b in zip(sl, sl[1:]):
            assert a.hi == b.lo
        for k, s in enumerate(sl):
            assert s.below == (ghost if per or k > 0 else 0)
            assert s.above == (ghost if per or k < parts - 1 else 0)
            rows = s.rows(ny)
            assert list(rows[s.below:s.below + s.own]) == list(range(s.lo, s.hi))
            if not per:
                assert rows.min() >= 0 and rows.max() < ny and np.all(np.diff(rows) == 1)


def test_exchanges_copy_each_ghost_row_from_its_owner():
    for ny, parts, ghost, per in [(40, 2, 2, False), (40, 2, 4, True), (45, 3, 2, True), (96, 4, 6, False)]:
        sl = S.plan(ny, parts, ghost, per)
        filled = [np.zeros(s.ny, bool) for s in sl]
        for d, dr, s, sr, n in S.exchanges(sl, per):
            src_rows = sl[s].rows(ny)[sr:sr + n]
            dst_rows = sl[d].rows(ny)[dr:dr + n]
            assert list(src_rows) == list(dst_rows)  # the same rows of the whole lattice
            assert sr >= sl[s].below and sr + n <= sl[s].below + sl[s].own  # read from owned rows only
            assert not filled[d][dr:dr + n].any()
            filled[d][dr:dr + n] = True
        for s, f in zip(sl, filled):  # every ghost row and no owned row is written
            assert f[:s.below].all() and f[s.below + s.own:].all() and not f[s.below:s.below + s.own].any()


def test_plan_rejects_thin_slabs_and_odd_ghosts():
    with pytest.raises(ValueError):
        S.plan(12, 4, 4, True)  # 3 rows per slab < 4 ghost rows
    with pytest.raises(ValueError):
        S.plan(64, 2, 3, False)
    with pytest.raises(ValueError):
        S.plan(64, 1, 2, False)
    tg = W.random_periodic(32, 32, seed=1, force="taylor_green")[0]
    with pytest.raises(ValueError):
        S.check_case(tg)
    sr = dict(W.random_periodic(32, 32, seed=1)[0], storage="fp16", rounding="stochastic")
    with pytest.raises(ValueError):
        S.check_case(sr)


class OracleSlabs:
    """The plan driven by the oracle in one process (test scaffolding)."""

    def __init__(self, case, fields, parts, every):
        self.ny = case["ny"]
        self.every = every
        per = S.y_periodic(case)
        self.sl = S.plan(case["ny"], parts, 2 * every, per)
        self.copies = S.exchanges(self.sl, per)
        self.o = [oracle.Oracle(S.slab_case(case, s), S.slab_fields(fields, s, self.ny)) for s in self.sl]
        self.exchange()

    def exchange(self):
        for d, dr, s, sr, n in self.copies:
            self.o[d].f[:, dr:dr + n] = self.o[s].f[:, sr:sr + n]
            self.o[d].h[:, dr:dr + n] = self.o[s].h[:, sr:sr + n]

    def step(self, n):
        while n > 0:
            k = min(self.every, n)
            for o in self.o:
                o.step(k)
            self.exchange()
            n -= k

    def owned(self, a):
        return np.concatenate([getattr(o, a)[:, s.below:s.below + s.own] for s, o in zip(self.sl, self.o)], axis=1)


CASES = [
    ("rb_walls_48x30", lambda: W.rayleigh_benard(48, 30, Ra=2e4, seed=3)),
    ("periodic_40x33", lambda: W.random_periodic(40, 33, seed=4, force="accel")),
    ("x_walls_24x16", lambda: W.with_walls(*W.random_periodic(24, 16, seed=5, force="none"), axis="x",
                                            kind="equilibrium")),
    ("zouhe_nee_couette_8x40", lambda: W.couette(ny=40)),
]


@pytest.mark.parametrize("name,make", CASES)
@pytest.mark.parametrize("parts,every", [(2, 1), (3, 2), (2, 3)])
def test_oracle_slabs_equal_the_undivided_lattice(name, make, parts, every):
    case, fields = make()
    whole = oracle.Oracle(case, fields)
    split = OracleSlabs(case, fields, parts, every)
    steps = 13
    whole.step(steps)
    split.step(steps)
    assert np.array_equal(split.owned("f"), whole.f), name
    assert np.array_equal(split.owned("h"), whole.h), name


def test_too_few_ghost_rows_break_the_equality():
    # exchange every 2 steps with the ghost rows of 1: the plan's bound is tight
    case, fields = W.random_periodic(40, 32, seed=6, force="accel")
    whole = oracle.Oracle(case, fields)
    split = OracleSlabs(case, fields, 2, 1)
    split.every = 2
    whole.step(4)
    split.step(4)
    assert not np.array_equal(split.owned("f"), whole.f)


def _rank_main(rank, world, port, out):
    import torch
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    case, fields = W.rayleigh_benard(40, 24, Ra=2e4, seed=7)
    every, steps = 2, 9
    sl = S.plan(case["ny"], world, 2 * every, S.y_periodic(case))
    copies = S.exchanges(sl, S.y_periodic(case))
    me = sl[rank]
    o = oracle.Oracle(S.slab_case(case, me), S.slab_fields(fields, me, case["ny"]))

    def exchange():
        # every copy crosses ranks here: the source rank sends, the destination receives
        reqs, recvs = [], []
        for tag, (d, dr, s, sr, n) in enumerate(copies):
            if s == rank:
                buf = torch.from_numpy(np.ascontiguousarray(np.stack([o.f[:, sr:sr + n], o.h[:, sr:sr + n]])))
                reqs.append((dist.isend(buf, dst=d, tag=tag), buf))
            if d == rank:
                buf = torch.zeros((2, 9, n, case["nx"]), dtype=torch.float64)
                recvs.append((dist.irecv(buf, src=s, tag=tag), buf, dr, n))
        for r, buf, dr, n in recvs:
            r.wait()
            o.f[:, dr:dr + n] = buf[0].numpy()
            o.h[:, dr:dr + n] = buf[1].numpy()
        for r, _ in reqs:
            r.wait()

    exchange()
    left = steps
    while left > 0:
        k = min(every, left)
        o.step(k)
        exchange()
        left -= k
    out.put((rank, me.lo, me.hi, o.f[:, me.below:me.below + me.own].copy(), o.h[:, me.below:me.below + me.own].copy()))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_exchange_ghost_rows_and_match_the_whole_lattice():
    import torch.multiprocessing as mp

    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=180) for _ in range(2)), key=lambda t: t[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    case, fields = W.rayleigh_benard(40, 24, Ra=2e4, seed=7)
    whole = oracle.Oracle(case, fields)
    whole.step(9)
    for rank, lo, hi, f, h in res:
        assert np.array_equal(f, whole.f[:, lo:hi]), rank
        assert np.array_equal(h, whole.h[:, lo:hi]), rank
