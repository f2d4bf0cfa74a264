"""Brute-force LP optimum by vertex enumeration, for tiny instances.

TEST INFRASTRUCTURE ONLY.  Used to pin the oracle's converged objective on LPs
small enough that every vertex can be listed (a few thousand linear solves).

A vertex of {x : A_i x (sense) b_i, l <= x <= u} is a feasible point where n
linearly independent constraints hold with equality.  When every variable has
finite bounds the feasible set is a polytope, so if it is non-empty the
minimum of c^T x is attained at a vertex; the minimum over all feasible
vertices is therefore the LP optimum.
"""
from __future__ import annotations

import itertools

import numpy as np

SENSE_E = ord("E")
SENSE_L = ord("L")
SENSE_G = ord("G")


def enumerate_vertices(A, b, c, lb, ub, sense, feas_tol=1e-9):
    """Return (best objective, best x) over all vertices; (inf, None) if none is feasible.

    ``A`` is a dense (m, n) array; every bound must be finite."""
    A = np.asarray(A, dtype=np.float64)
    m, n = A.shape
    if not (np.all(np.isfinite(lb)) and np.all(np.isfinite(ub))):
        raise ValueError("vertex enumeration needs finite bounds")
    rows = []  # (coefficients, rhs)
    for i in range(m):
        rows.append((A[i], b[i]))
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        rows.append((e, lb[j]))
        rows.append((e, ub[j]))
    eq_rows = [i for i in range(m) if sense[i] == SENSE_E]
    other = [i for i in range(len(rows)) if i not in eq_rows]

    def feasible(x):
        ax = A @ x
        for i in range(m):
            s = sense[i]
            if s == SENSE_E and abs(ax[i] - b[i]) > feas_tol * (1 + abs(b[i])):
                return False
            if s == SENSE_L and ax[i] - b[i] > feas_tol * (1 + abs(b[i])):
                return False
            if s == SENSE_G and b[i] - ax[i] > feas_tol * (1 + abs(b[i])):
                return False
        return bool(np.all(x >= lb - feas_tol) and np.all(x <= ub + feas_tol))

    best = np.inf
    best_x = None
    need = n - len(eq_rows)
    if need < 0:
        # more equalities than variables: try every n-subset of them instead
        need = 0
    for extra in itertools.combinations(other, need):
        idx = list(eq_rows) + list(extra)
        if len(idx) > n:
            # over-determined: use a least-squares solve of the square subsets
            subsets = itertools.combinations(idx, n)
        else:
            subsets = [idx]
        for sub in subsets:
            M = np.array([rows[i][0] for i in sub])
            r = np.array([rows[i][1] for i in sub])
            if abs(np.linalg.det(M)) < 1e-12:
                continue
            x = np.linalg.solve(M, r)
            if feasible(x):
                v = float(c @ x)
                if v < best:
                    best = v
                    best_x = x
    return best, best_x
