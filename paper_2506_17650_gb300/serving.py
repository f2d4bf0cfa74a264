"""Continuous-batching serving loop for LPs.

Requests (LPs given as host arrays) arrive over time.  The server admits a
waiting request when a slot is free and the device memory its problem needs
(lp_memory_bytes) fits in the memory budget; admission creates the problem on
the device (lp_create: copy, preprocessing, initial state).  Every admitted
problem keeps its whole iteration state on the device -- iterates,
preconditioners, step size, primal weight, restart state.  Small problems
advance together: one round is a single batched kernel launch in which every
batched problem runs up to ``round_attempts`` step attempts.  A problem with
at least ``solo_nnz`` nonzeros, or one still open after ``handoff`` attempts,
runs instead on the single-problem kernels (the whole GPU's grid, its own
stream) from a worker thread, concurrently with the rounds.  After a round the
server retires the problems that reached the tolerance (or the attempt
limit), copies their results to the host and frees their memory, and admits
waiting requests into the freed slots.  Both rules depend only on the problem
itself, so a problem's result is the same alone and in any mix.

The scheduling here is host bookkeeping; every step of the method runs in the
library's kernels (``Batch.round`` and ``Problem.solve``).
"""
from __future__ import annotations

import collections
import threading
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
    wide_nnz) of the batched kernel.  solo_nnz: problems with at least this
    many nonzeros run on the single-problem kernels (None: never).  handoff:
    a batched problem still open after this many attempts moves there too
    (0: never).  Other keyword arguments are lp_options fields for every
    problem (precision defaults to mixed)."""

    def __init__(self, tol=1e-4, iter_limit=200_000, round_attempts=128, max_slots=512, memory_budget=None,
                 schedule=(1, 1 << 62), keep_solution=True, clock=time.perf_counter, solo_nnz=None,
                 handoff=0, **options):
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
        self.solo_nnz = solo_nnz
        self.handoff = handoff
        self.solo: list[tuple[Request, Problem, threading.Thread]] = []
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
            if (self.active or self.solo) and self.used + req.bytes > self.memory_budget:
                break  # first come, first served: wait until enough memory is free
            self.queue.popleft()
            prob = Problem(req.lp, **self.options)
            req.admitted = self.clock()
            self.used += req.bytes
            if self.solo_nnz is not None and req.lp.nnz >= self.solo_nnz:
                self._go_solo(req, prob)
            else:
                self.active.append((req, prob))

    def _go_solo(self, req, prob):
        # the ctypes call releases the GIL: the solve runs while the rounds go on
        t = threading.Thread(target=prob.solve, args=(self.tol, self.iter_limit), daemon=True)
        t.start()
        self.solo.append((req, prob, t))

    def _finish(self, req, prob, now):
        x, y, stats = prob.result(self.keep_solution, self.keep_solution)
        req.finished = now
        req.status = stats["status"]
        req.iterations = int(stats["iterations"])
        req.stats = stats
        req.x, req.y = x, y
        prob.close()
        self.used -= req.bytes
        self.done[req.rid] = req

    def _retire(self):
        now = self.clock()
        if self.active:
            status, iters = self.batch.status()
            keep = []
            for (req, prob), st, it in zip(self.active, status, iters):
                if st != 0 or it >= self.iter_limit:
                    self._finish(req, prob, now)
                elif self.handoff and it >= self.handoff:
                    self._go_solo(req, prob)
                else:
                    keep.append((req, prob))
            self.active = keep
        running = []
        for req, prob, t in self.solo:
            if t.is_alive():
                running.append((req, prob, t))
            else:
                t.join()
                self._finish(req, prob, now)
        self.solo = running

    def step(self) -> int:
        """Admit, run one round, retire.  Returns the number of problems still admitted or waiting."""
        self._admit()
        if self.active:
            self.batch.set_members([p for _, p in self.active])
            self.batch.round(self.tol, self.round_attempts, self.iter_limit)
            self.rounds += 1
        elif self.solo:
            time.sleep(0.0005)  # only solo problems running: wait for one to finish
        self._retire()
        return len(self.active) + len(self.queue) + len(self.solo)

    def drain(self):
        while self.step():
            pass

    def close(self):
        for _, prob, t in self.solo:
            t.join()
            prob.close()
        self.solo = []
        for _, prob in self.active:
            prob.close()
        self.active = []
        self.batch.close()

    def latency_report(self):
        """Time to tolerance (finish - arrival) over the requests that reached
        the tolerance, with their count; requests that stopped at the attempt
        limit (or failed) are reported apart, with their time to that stop."""
        done = [r for r in self.done.values() if r.time_to_tol is not None]
        if not done:
            return {"finished": 0}
        solved = np.array([r.time_to_tol for r in done if r.status == LP_OPTIMAL])
        capped = np.array([r.time_to_tol for r in done if r.status != LP_OPTIMAL])
        out = {"finished": len(done), "reached_tol": int(solved.size), "stopped_before_tol": int(capped.size),
               "rounds": self.rounds}
        if solved.size:
            out.update(p50_s=float(np.percentile(solved, 50)), p99_s=float(np.percentile(solved, 99)),
                       mean_s=float(solved.mean()))
        if capped.size:
            out.update(stopped_p50_s=float(np.percentile(capped, 50)), stopped_p99_s=float(np.percentile(capped, 99)))
        return out
