"""Continuous-batching serving loop for LPs.

Requests (LPs given as host arrays) arrive over time.  The server admits a
waiting request when a slot is free and the device memory its problem needs
(lp_memory_bytes) fits in the memory budget; admission creates the problem on
the device (lp_create: copy, preprocessing, initial state).  Every admitted
problem keeps its whole iteration state on the device -- iterates,
preconditioners, step size, primal weight, restart state -- and all of them
advance together: one round is a single batched kernel launch in which every
admitted problem runs up to ``round_attempts`` step attempts.  After a round
the server retires the problems that reached the tolerance (or the iteration
limit), copies their results to the host and frees their memory, and admits
waiting requests into the freed slots.  A problem's arithmetic depends only on
its own state and team size, so its result is the same alone and in any mix.

The scheduling here is host bookkeeping; every step of the method runs in the
library's kernels (``Batch.round``).
"""
from __future__ import annotations

import collections
import time
from dataclasses import dataclass, field

import numpy as np

from . import LP_OPTIMAL, LP_PREC_MIXED, Batch, Problem, lp_memory_bytes, lp_options_default


@dataclass
class Request:
    rid: int
    lp: object
    arrival: float
    bytes: int
    admitted: float | None = None
    finished: float | None = None
    status: int = 0
    iterations: int = 0
    stats: dict = field(default_factory=dict)
    x: np.ndarray | None = None
    y: np.ndarray | None = None

    @property
    def time_to_tol(self):
        return None if self.finished is None else self.finished - self.arrival


class Server:
    """Admission by slots and device memory, device-resident state, one batched launch per round.

    memory_budget: device bytes the admitted problems may hold (default: 90% of
    the free device memory when the server starts).  schedule: (cluster_size,
    wide_nnz) of the batched kernel.  Other keyword arguments are lp_options
    fields for every problem (precision defaults to mixed)."""

    def __init__(self, tol=1e-4, iter_limit=200_000, round_attempts=128, max_slots=512, memory_budget=None,
                 schedule=(1, 1 << 62), keep_solution=True, clock=time.perf_counter, **options):
        import torch

        options.setdefault("precision", LP_PREC_MIXED)
        self.options = options
        self.tol = tol
        self.iter_limit = iter_limit
        self.round_attempts = round_attempts
        self.max_slots = max_slots
        self.keep_solution = keep_solution
        self.clock = clock
        if memory_budget is None:
            free, _ = torch.cuda.mem_get_info()
            memory_budget = int(0.9 * free)
        self.memory_budget = memory_budget
        self.used = 0
        self.queue: collections.deque[Request] = collections.deque()
        self.active: list[tuple[Request, Problem]] = []
        self.done: dict[int, Request] = {}
        self.rounds = 0
        self._next = 0
        self._opts = lp_options_default(**options)
        self.batch = Batch([], *schedule)

    def submit(self, lp, arrival=None) -> int:
        rid = self._next
        self._next += 1
        nbytes = lp_memory_bytes(lp.m, lp.n, lp.nnz, self._opts)
        self.queue.append(Request(rid, lp, self.clock() if arrival is None else arrival, nbytes))
        return rid

    def _admit(self):
        while self.queue and len(self.active) < self.max_slots:
            req = self.queue[0]
            if self.active and self.used + req.bytes > self.memory_budget:
                break  # first come, first served: wait until enough memory is free
            self.queue.popleft()
            prob = Problem(req.lp, **self.options)
            req.admitted = self.clock()
            self.used += req.bytes
            self.active.append((req, prob))

    def _retire(self):
        status, iters = self.batch.status()
        keep = []
        now = self.clock()
        for (req, prob), st, it in zip(self.active, status, iters):
            if st != 0 or it >= self.iter_limit:
                x, y, stats = prob.result(self.keep_solution, self.keep_solution)
                req.finished = now
                req.status = stats["status"]
                req.iterations = int(it)
                req.stats = stats
                req.x, req.y = x, y
                prob.close()
                self.used -= req.bytes
                self.done[req.rid] = req
            else:
                keep.append((req, prob))
        self.active = keep

    def step(self) -> int:
        """Admit, run one round, retire.  Returns the number of problems still admitted or waiting."""
        self._admit()
        if self.active:
            self.batch.set_members([p for _, p in self.active])
            self.batch.round(self.tol, self.round_attempts, self.iter_limit)
            self.rounds += 1
            self._retire()
        return len(self.active) + len(self.queue)

    def drain(self):
        while self.step():
            pass

    def close(self):
        for _, prob in self.active:
            prob.close()
        self.active = []
        self.batch.close()

    def latency_report(self):
        t = np.array([r.time_to_tol for r in self.done.values() if r.time_to_tol is not None])
        ok = sum(1 for r in self.done.values() if r.status == LP_OPTIMAL)
        if t.size == 0:
            return {"solved": 0}
        return {"solved": int(t.size), "optimal": ok, "p50_s": float(np.percentile(t, 50)),
                "p99_s": float(np.percentile(t, 99)), "mean_s": float(t.mean()), "rounds": self.rounds}
