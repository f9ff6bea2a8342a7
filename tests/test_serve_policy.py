"""Host-side scheduling policy of the serving loop, without a GPU: the lattices stepped in
a chunk are the ones with the least remaining work (nodes x steps left), taken in that
order until the node budget is reached, and the first one is always taken."""
import numpy as np
import pytest

from paper_1610_07114_gb300 import workloads as W


@pytest.fixture(scope="module")
def serve():
    from paper_1610_07114_gb300 import build

    build.build()  # the serving module imports the library binding
    from paper_1610_07114_gb300 import serve

    return serve


def _server(serve, node_budget):
    s = object.__new__(serve.Server)  # the policy needs no streams or device memory
    s.node_budget = node_budget
    s.active = []
    return s


def _active(serve, rid, nx, ny, steps=None, residual=None, max_steps=1000, done=0):
    case, fields = W.random_periodic(nx, ny, seed=rid)
    req = serve.Request(rid, case, fields, steps=steps, residual=residual, max_steps=max_steps)
    req.steps_done = done
    return serve._Active(req, None, 0, 0)


def test_least_remaining_work_first_up_to_the_node_budget(serve):
    rng = np.random.default_rng(5)
    s = _server(serve, node_budget=40_000)
    for rid in range(30):
        nx, ny = [(16, 8), (64, 32), (128, 64), (256, 128)][int(rng.integers(4))]
        steps = int(rng.integers(100, 5000))
        s.active.append(_active(serve, rid, nx, ny, steps=steps, done=int(rng.integers(0, steps))))
    chosen = s._select()
    work = [s._work_left(a) for a in chosen]
    assert work == sorted(work)
    assert sum(a.req.nodes for a in chosen) <= s.node_budget
    rest = [a for a in s.active if all(a is not c for c in chosen)]
    # every lattice left out has at least the remaining work of the last one chosen
    assert all(s._work_left(a) >= work[-1] for a in rest)
    # and the first one left out would have broken the budget
    nxt = min(rest, key=s._work_left)
    assert sum(a.req.nodes for a in chosen) + nxt.req.nodes > s.node_budget


def test_a_lattice_above_the_budget_is_still_stepped(serve):
    s = _server(serve, node_budget=1000)
    s.active = [_active(serve, 1, 256, 128, steps=10)]
    assert [a.req.rid for a in s._select()] == [1]


def test_steady_state_requests_count_their_step_cap_as_work(serve):
    s = _server(serve, node_budget=10**9)
    a = _active(serve, 1, 64, 32, residual=1e-8, max_steps=20_000, done=5_000)
    b = _active(serve, 2, 64, 32, steps=20_000, done=4_000)
    s.active = [b, a]
    assert s._work_left(a) == 64 * 32 * 15_000
    assert [x.req.rid for x in s._select()] == [1, 2]
