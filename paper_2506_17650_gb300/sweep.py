"""Per-instance learning-rate selection as one batch.

The online learning rate is chosen per instance from a small grid by
iteration count (Section 4.1: {1e-1, 1e-2, 1e-3} for vanilla PDHG,
{1e-5, 1e-6, 1e-7} for the PDLP integration; the Remark after Table 1).
``alpha_sweep`` solves the same LP once per grid value, all as members of one
batch, so every round of the whole sweep is a single kernel launch, and
returns the value that reached the tolerance in the fewest iterations.
"""
from __future__ import annotations

from . import LP_OPTIMAL, Batch, Problem

PAPER_GRID_VANILLA = (1e-1, 1e-2, 1e-3)
PAPER_GRID_PDLP = (1e-5, 1e-6, 1e-7)


def alpha_sweep(lp, alphas=PAPER_GRID_PDLP, tol=1e-4, iter_limit=200_000, round_attempts=256, schedule=(1, 1 << 62),
                **options):
    """Returns (best_alpha or None, [dict(alpha, status, iterations, pobj) per grid value])."""
    probs = [Problem(lp, alpha=a, **options) for a in alphas]
    try:
        with Batch(probs, *schedule) as b:
            b.solve(tol, iter_limit, round_attempts)
            status, iters = b.status()
        rows = []
        for a, p, s, it in zip(alphas, probs, status, iters):
            _, _, st = p.result(False, False)
            rows.append(dict(alpha=a, status=int(s), iterations=int(it), pobj=st["pobj"]))
    finally:
        for p in probs:
            p.close()
    ok = [r for r in rows if r["status"] == LP_OPTIMAL]
    best = min(ok, key=lambda r: (r["iterations"], r["alpha"]))["alpha"] if ok else None
    return best, rows
