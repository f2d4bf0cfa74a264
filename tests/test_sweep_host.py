"""The learning-rate sweep's host logic on the CPU, with fake problems.

alpha_sweep solves one LP per grid value as members of one batch and keeps
the value that reached the tolerance in the fewest attempts (ties: the
smaller rate); the real library path is covered by tests/test_gpu_sweep.py.
"""
import pytest

import paper_2506_17650_gb300.sweep as sweep

LP_OPTIMAL, LP_ITERATION_LIMIT = 1, 2


class FakeProblem:
    closed = []

    def __init__(self, lp, alpha, **opts):
        self.alpha = alpha
        self.need = lp[alpha]  # attempts this rate needs (None: never converges)

    def result(self, want_x=True, want_y=True):
        return None, None, {"pobj": 10.0 * self.alpha}

    def close(self):
        FakeProblem.closed.append(self.alpha)


class FakeBatch:
    fail = False

    def __init__(self, members, cluster=1, wide=0):
        self.members = members

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        return False

    def solve(self, tol, limit, round_attempts):
        if FakeBatch.fail:
            raise RuntimeError("device error")
        self.limit = limit

    def status(self):
        st, it = [], []
        for p in self.members:
            done = p.need is not None and p.need <= self.limit
            st.append(LP_OPTIMAL if done else LP_ITERATION_LIMIT)
            it.append(p.need if done else self.limit)
        return st, it


@pytest.fixture
def fake(monkeypatch):
    monkeypatch.setattr(sweep, "Problem", FakeProblem)
    monkeypatch.setattr(sweep, "Batch", FakeBatch)
    FakeProblem.closed = []
    FakeBatch.fail = False


def test_fewest_attempts_wins(fake):
    lp = {1e-5: 900, 1e-6: 640, 1e-7: 1200}
    best, rows = sweep.alpha_sweep(lp)
    assert best == 1e-6
    assert [r["alpha"] for r in rows] == [1e-5, 1e-6, 1e-7]
    assert [r["iterations"] for r in rows] == [900, 640, 1200]
    assert all(r["status"] == LP_OPTIMAL for r in rows)
    assert sorted(FakeProblem.closed) == sorted(lp)


def test_ties_go_to_the_smaller_rate_and_unsolved_values_are_ignored(fake):
    lp = {1e-1: None, 1e-2: 500, 1e-3: 500}
    best, rows = sweep.alpha_sweep(lp, alphas=(1e-1, 1e-2, 1e-3), iter_limit=1000)
    assert best == 1e-3
    assert rows[0]["status"] == LP_ITERATION_LIMIT and rows[0]["iterations"] == 1000


def test_no_value_converges(fake):
    lp = {1e-5: None, 1e-6: 5000, 1e-7: None}
    best, rows = sweep.alpha_sweep(lp, iter_limit=1000)
    assert best is None and all(r["status"] == LP_ITERATION_LIMIT for r in rows)


def test_problems_are_released_when_the_batch_fails(fake):
    FakeBatch.fail = True
    with pytest.raises(RuntimeError):
        sweep.alpha_sweep({1e-5: 1, 1e-6: 2, 1e-7: 3})
    assert sorted(FakeProblem.closed) == [1e-7, 1e-6, 1e-5]
