"""The serving loop's host bookkeeping on the CPU.

The Server's scheduling -- admission in arrival order by free slots and device
memory, rounds of the batched members, hand-off to the single-problem path,
retirement and the latency report -- is plain host code.  Here it drives fake
problems whose "solve" is a counter (each fake LP needs a set number of
attempts), so the rules can be checked without a GPU; the real library path
is covered by tests/test_gpu_serving.py.
"""
import itertools

import pytest

import paper_2506_17650_gb300.serving as serving

LP_OPTIMAL, LP_ITERATION_LIMIT = 1, 2


class FakeLP:
    def __init__(self, needed, nnz=1000, m=10, n=20):
        self.needed, self.nnz, self.m, self.n = needed, nnz, m, n


class FakeProblem:
    live = 0

    def __init__(self, lp, **opts):
        self.lp, self.done, self.status, self.closed = lp, 0, 0, False
        self.solo = False
        FakeProblem.live += 1

    def advance(self, attempts, limit):
        step = min(attempts, self.lp.needed - self.done, limit - self.done)
        self.done += max(step, 0)
        if self.done >= self.lp.needed:
            self.status = LP_OPTIMAL
        elif self.done >= limit:
            self.status = LP_ITERATION_LIMIT

    def solve(self, tol, limit):  # the single-problem path: to the end
        self.solo = True
        self.advance(limit, limit)

    def result(self, want_x=True, want_y=True):
        return None, None, {"status": self.status, "iterations": self.done}

    def close(self):
        assert not self.closed
        self.closed = True
        FakeProblem.live -= 1


class FakeBatch:
    def __init__(self, members, cluster=1, wide=0):
        self.members = list(members)

    def set_members(self, members):
        self.members = list(members)

    def round(self, tol, attempts, limit):
        for p in self.members:
            assert p.status == 0 and not p.solo  # only open, batched problems are members
            p.advance(attempts, limit)

    def status(self):
        return [p.status for p in self.members], [p.done for p in self.members]

    def close(self):
        pass


@pytest.fixture
def fake(monkeypatch):
    monkeypatch.setattr(serving, "Problem", FakeProblem)
    monkeypatch.setattr(serving, "Batch", FakeBatch)
    monkeypatch.setattr(serving, "lp_memory_bytes", lambda m, n, nnz, opts: 100 * nnz)
    monkeypatch.setattr(serving, "lp_options_default", lambda **kw: None)
    FakeProblem.live = 0
    ticks = itertools.count()
    return lambda: float(next(ticks))


def test_every_request_finishes_with_its_own_attempt_count(fake):
    srv = serving.Server(round_attempts=64, memory_budget=10 ** 9, clock=fake)
    needs = [10, 64, 65, 300, 1, 129]
    ids = [srv.submit(FakeLP(k)) for k in needs]
    srv.drain()
    assert sorted(srv.done) == ids
    for rid, k in zip(ids, needs):
        assert srv.done[rid].status == LP_OPTIMAL and srv.done[rid].iterations == k
    assert srv.used == 0 and FakeProblem.live == 0
    # rounds: the slowest request needs ceil(300 / 64) of them
    assert srv.rounds == 5


def test_attempt_limit_retires_an_unsolved_request(fake):
    srv = serving.Server(round_attempts=50, iter_limit=120, memory_budget=10 ** 9, clock=fake)
    rid = srv.submit(FakeLP(1000))
    srv.drain()
    assert srv.done[rid].status == LP_ITERATION_LIMIT and srv.done[rid].iterations == 120


def test_memory_budget_and_arrival_order(fake):
    # budget for two 1000-nonzero problems; a 3000-nonzero request at the head
    # waits until everything ahead of it has left, and nothing behind it jumps ahead
    srv = serving.Server(round_attempts=10, memory_budget=200_000, clock=fake)
    order = []
    real_init = FakeProblem.__init__

    def init(self, lp, **opts):
        order.append(lp)
        real_init(self, lp, **opts)

    FakeProblem.__init__ = init
    try:
        lps = [FakeLP(30), FakeLP(30), FakeLP(20, nnz=3000), FakeLP(5), FakeLP(5)]
        for lp in lps:
            srv.submit(lp)
        while srv.step():
            # within the budget, except one request larger than it that runs alone
            assert srv.used <= 200_000 or len(srv.active) + len(srv.solo) == 1
        assert order == lps  # admitted in arrival order
    finally:
        FakeProblem.__init__ = real_init
    assert len(srv.done) == 5 and srv.used == 0


def test_a_request_larger_than_the_budget_runs_alone(fake):
    srv = serving.Server(round_attempts=10, memory_budget=50_000, clock=fake)
    big = srv.submit(FakeLP(15, nnz=1000))  # 100,000 bytes > budget: admitted only when nothing else holds memory
    small = srv.submit(FakeLP(5, nnz=100))
    srv.step()
    assert [r.rid for r, _ in srv.active] == [big]  # the small one waits behind it
    srv.drain()
    assert srv.done[big].status == LP_OPTIMAL and srv.done[small].status == LP_OPTIMAL


def test_slots_limit_the_batch(fake):
    srv = serving.Server(round_attempts=1, max_slots=3, memory_budget=10 ** 9, clock=fake)
    for _ in range(7):
        srv.submit(FakeLP(4))
    while srv.step():
        assert len(srv.active) <= 3
    assert len(srv.done) == 7


def test_handoff_and_large_problems_take_the_single_problem_path(fake):
    srv = serving.Server(round_attempts=100, handoff=200, solo_nnz=50_000, memory_budget=10 ** 9, clock=fake)
    long_one = srv.submit(FakeLP(1000))         # still open after 200 attempts: handed off
    short_one = srv.submit(FakeLP(150))         # finishes in the batch
    large_one = srv.submit(FakeLP(70, nnz=60_000))  # single-problem path from the start
    probs = {}
    real_init = FakeProblem.__init__

    def init(self, lp, **opts):
        probs[id(lp)] = self
        real_init(self, lp, **opts)

    FakeProblem.__init__ = init
    try:
        lps = {rid: r.lp for rid, r in ((r.rid, r) for r in srv.queue)}
        srv.drain()
    finally:
        FakeProblem.__init__ = real_init
    for rid, need in ((long_one, 1000), (short_one, 150), (large_one, 70)):
        assert srv.done[rid].status == LP_OPTIMAL and srv.done[rid].iterations == need
    assert probs[id(lps[long_one])].solo and probs[id(lps[large_one])].solo
    assert not probs[id(lps[short_one])].solo
    assert FakeProblem.live == 0 and srv.used == 0


def test_latency_report(fake):
    srv = serving.Server(round_attempts=10, memory_budget=10 ** 9, clock=fake)
    for k in (5, 15, 25):
        srv.submit(FakeLP(k), arrival=0.0)
    srv.drain()
    rep = srv.latency_report()
    times = sorted(r.time_to_tol for r in srv.done.values())
    assert rep["finished"] == 3 and rep["reached_tol"] == 3 and rep["rounds"] == 3
    assert rep["stopped_before_tol"] == 0 and "stopped_p50_s" not in rep
    assert times[0] < times[1] < times[2]  # retired after 1, 2 and 3 rounds
    assert rep["p50_s"] == times[1] and rep["mean_s"] == pytest.approx(sum(times) / 3)


def test_latency_report_keeps_capped_requests_apart(fake):
    """Percentiles of time to tolerance cover only the requests that reached
    it; a request stopped by the attempt limit is counted and timed apart."""
    srv = serving.Server(round_attempts=10, iter_limit=40, memory_budget=10 ** 9, clock=fake)
    for k in (5, 15, 1000):
        srv.submit(FakeLP(k), arrival=0.0)
    srv.drain()
    rep = srv.latency_report()
    solved = sorted(r.time_to_tol for r in srv.done.values() if r.status == LP_OPTIMAL)
    capped = [r.time_to_tol for r in srv.done.values() if r.status != LP_OPTIMAL]
    assert rep["finished"] == 3 and rep["reached_tol"] == 2 and rep["stopped_before_tol"] == 1
    assert len(capped) == 1 and capped[0] > solved[-1]  # stopped after 4 rounds
    assert rep["p99_s"] <= solved[-1] and rep["mean_s"] == pytest.approx(sum(solved) / 2)
    assert rep["stopped_p50_s"] == capped[0]
