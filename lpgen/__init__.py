"""Seeded synthetic LP generators.

This module is the only code shared by the CUDA path's tests/benchmarks and the
CPU oracle.  It builds problem data (CSR matrix, right-hand side, costs, bounds,
row senses) and, where the construction allows it, a primal-dual optimal pair
(x0, y0) that is optimal by construction (complementary slackness holds
entry-wise).  It holds none of the PDHG method's arithmetic.

Problem form used throughout::

    min  c^T x   s.t.  A_i x  (=, <=, >=)  b_i   for each row i,   lb <= x <= ub

Row senses are stored as ASCII codes (``E``, ``L`` for <=, ``G`` for >=) in a
uint8 array; infinite bounds are IEEE +-inf.

Generators
----------
* :func:`tiny_random` -- m=200, n=500, 5 nonzeros per column, N(0,1) values,
  equality rows, 0 <= x <= 10.  Half of x0 sits at the lower bound so that the
  cost vector is not in the row space of A (otherwise every feasible point would
  be optimal).
* :func:`transport` -- supply (<=) and demand (=) rows, arcs with two unit
  nonzeros, costs U(1, 100), x >= 0.
* :func:`powerlaw` -- m=2M, n=5M, ~30M nonzeros; power-law column degrees
  (exponent 2.1), log-uniform magnitudes on [1e-3, 1e3] with random signs,
  30% equality / 70% <= rows, 80% boxed / 20% free variables.
* :func:`from_pattern` -- any sparsity pattern, with the same optimal-by-
  construction recipe; used for row-length edge cases.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp

SENSE_E = ord("E")
SENSE_L = ord("L")
SENSE_G = ord("G")


@dataclass
class LP:
    """One LP instance in CSR form (host arrays)."""

    m: int
    n: int
    row_ptr: np.ndarray  # int64 [m+1]
    col_idx: np.ndarray  # int32 [nnz]
    val: np.ndarray  # float64 [nnz]
    b: np.ndarray  # float64 [m]
    c: np.ndarray  # float64 [n]
    lb: np.ndarray  # float64 [n], -inf allowed
    ub: np.ndarray  # float64 [n], +inf allowed
    sense: np.ndarray  # uint8 [m], ASCII E/L/G
    name: str = ""
    x_opt: np.ndarray | None = None  # optimal primal point, if known by construction
    y_opt: np.ndarray | None = None  # optimal dual point, if known by construction
    obj_opt: float | None = None
    meta: dict = field(default_factory=dict)

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    def csr(self) -> sp.csr_matrix:
        return sp.csr_matrix((self.val, self.col_idx, self.row_ptr), shape=(self.m, self.n))


def _sorted_unique(a):
    """np.unique(a) for an integer array, by one sort and a neighbour test (the
    hash-based path of np.unique is many times slower on tens of millions of keys)."""
    a = np.sort(a)
    if a.size > 1:
        keep = np.empty(a.size, dtype=bool)
        keep[0] = True
        np.not_equal(a[1:], a[:-1], out=keep[1:])
        a = a[keep]
    return a


def _csr_from_coo(m, n, rows, cols, vals):
    """Sorted, duplicate-free CSR arrays from coordinate triplets (no summing: callers pass distinct pairs)."""
    key = np.asarray(rows, dtype=np.int64) * max(int(n), 1) + np.asarray(cols, dtype=np.int64)
    order = np.argsort(key)  # keys are distinct, so this is the (row, col) order
    ks = key[order]
    if ks.size > 1 and np.any(ks[1:] == ks[:-1]):
        raise ValueError("repeated (row, column) pair")
    rows = rows[order]
    cols = cols[order]
    vals = vals[order]
    counts = np.bincount(rows, minlength=m)
    row_ptr = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    return row_ptr, cols.astype(np.int32), vals.astype(np.float64)


def _distinct_rows_per_column(rng, m, degrees):
    """For column j pick ``degrees[j]`` distinct rows uniformly at random.

    Draws with replacement and then removes repeated (row, col) pairs, so a
    column can end with slightly fewer entries than asked when its degree is a
    sizeable fraction of m; the returned arrays are the realised pattern.
    """
    degrees = np.asarray(degrees, dtype=np.int64)
    cols = np.repeat(np.arange(degrees.size, dtype=np.int64), degrees)
    rows = rng.integers(0, m, size=cols.size, dtype=np.int64)
    key = _sorted_unique(cols * m + rows)
    return (key % m), (key // m)


def from_pattern(
    m,
    n,
    rows,
    cols,
    vals,
    rng,
    *,
    sense_probs=(1.0, 0.0, 0.0),
    var_probs=(1.0, 0.0, 0.0),
    box_upper=10.0,
    p_at_lower=0.3,
    p_at_upper=0.1,
    tight_frac=0.5,
    name="pattern",
):
    """Build an LP with a known optimum on a given sparsity pattern.

    ``sense_probs`` = probabilities of (E, L, G) rows; ``var_probs`` = of
    (boxed [0, box_upper], lower-bounded [0, inf), free) variables.

    Recipe: x0 in bounds (boxed: ``p_at_lower`` at 0, ``p_at_upper`` at the
    upper bound, else uniform; lower-bounded: ``p_at_lower`` at 0, else
    U(0, box_upper); free: N(0, 1)).  Equality rows: b = A x0, y0 ~ N(0,1).
    Inequality rows: a ``tight_frac`` share is tight (b = A x0, y0 of the
    row's sign: <= 0 for L, >= 0 for G), the rest slack by U(0,1) with y0 = 0.
    Reduced cost z = c - A^T y0 is U(0,1) at a lower bound, -U(0,1) at an upper
    bound, 0 elsewhere; c = A^T y0 + z.  Complementary slackness then holds
    entry-wise, so (x0, y0) is optimal and c^T x0 is the optimal value.
    """
    rows = np.asarray(rows, dtype=np.int64)
    cols = np.asarray(cols, dtype=np.int64)
    vals = np.asarray(vals, dtype=np.float64)
    row_ptr, col_idx, val = _csr_from_coo(m, n, rows, cols, vals)
    A = sp.csr_matrix((val, col_idx, row_ptr), shape=(m, n))

    kind = rng.choice(3, size=n, p=np.asarray(var_probs, dtype=np.float64))
    lb = np.where(kind == 2, -np.inf, 0.0)
    ub = np.where(kind == 0, box_upper, np.inf)

    u01 = rng.random(n)
    x0 = box_upper * rng.random(n)
    at_lower = (kind != 2) & (u01 < p_at_lower)
    at_upper = (kind == 0) & (u01 >= p_at_lower) & (u01 < p_at_lower + p_at_upper)
    x0[at_lower] = 0.0
    x0[at_upper] = box_upper
    free = kind == 2
    x0[free] = rng.standard_normal(int(free.sum()))

    sense_pick = rng.choice(3, size=m, p=np.asarray(sense_probs, dtype=np.float64))
    sense = np.array([SENSE_E, SENSE_L, SENSE_G], dtype=np.uint8)[sense_pick]
    ax0 = A @ x0
    y0 = rng.standard_normal(m)
    tight = rng.random(m) < tight_frac
    slack = rng.random(m)
    b = ax0.copy()
    is_l = sense == SENSE_L
    is_g = sense == SENSE_G
    y0[is_l] = -np.abs(y0[is_l])
    y0[is_g] = np.abs(y0[is_g])
    loose_l = is_l & ~tight
    loose_g = is_g & ~tight
    y0[loose_l | loose_g] = 0.0
    b[loose_l] += slack[loose_l]
    b[loose_g] -= slack[loose_g]

    z = np.zeros(n)
    z[at_lower] = rng.random(int(at_lower.sum()))
    z[at_upper] = -rng.random(int(at_upper.sum()))
    c = A.T @ y0 + z

    return LP(
        m=m,
        n=n,
        row_ptr=row_ptr,
        col_idx=col_idx,
        val=val,
        b=b,
        c=c,
        lb=lb,
        ub=ub,
        sense=sense,
        name=name,
        x_opt=x0,
        y_opt=y0,
        obj_opt=float(c @ x0),
    )


def tiny_random(seed=0, m=200, n=500, col_nnz=5):
    """Tiny random equality-form LP (5 nonzeros per column, N(0,1) values, 0 <= x <= 10)."""
    rng = np.random.default_rng(seed)
    if col_nnz > m:
        raise ValueError("col_nnz must not exceed m")
    # distinct rows per column: a permutation prefix per column
    rows = np.argsort(rng.random((n, m)), axis=1)[:, :col_nnz].reshape(-1)
    cols = np.repeat(np.arange(n), col_nnz)
    vals = rng.standard_normal(rows.size)
    lp = from_pattern(
        m, n, rows, cols, vals, rng,
        sense_probs=(1.0, 0.0, 0.0), var_probs=(1.0, 0.0, 0.0),
        p_at_lower=0.5, p_at_upper=0.0, name=f"tiny_random_m{m}_n{n}",
    )
    return lp


def transport(seed=0, n_supply=25_000, n_demand=25_000, n_arcs=200_000):
    """Transportation-style LP.

    Rows 0..S-1 are supply rows (sum of outgoing arcs <= s_i), rows S..S+D-1
    demand rows (sum of incoming arcs = d_k).  Each arc (column) has a +1 in
    its supply row and a +1 in its demand row.  The first S + D arcs touch every
    node, the rest join uniform random pairs.  A random flow x0 ~ U(0, 10)
    fixes d = in-flow(x0) and s = 1.2 out-flow(x0), so the LP is feasible; costs
    U(1, 100) with x >= 0 make it bounded.
    """
    rng = np.random.default_rng(seed)
    S, D = n_supply, n_demand
    if n_arcs < S + D:
        raise ValueError("need at least n_supply + n_demand arcs")
    src = np.empty(n_arcs, dtype=np.int64)
    dst = np.empty(n_arcs, dtype=np.int64)
    src[:S] = np.arange(S)
    dst[:S] = rng.integers(0, D, size=S)
    src[S:S + D] = rng.integers(0, S, size=D)
    dst[S:S + D] = np.arange(D)
    rest = n_arcs - S - D
    src[S + D:] = rng.integers(0, S, size=rest)
    dst[S + D:] = rng.integers(0, D, size=rest)
    rows = np.concatenate([src, S + dst])
    cols = np.concatenate([np.arange(n_arcs), np.arange(n_arcs)])
    vals = np.ones(rows.size)
    row_ptr, col_idx, val = _csr_from_coo(S + D, n_arcs, rows, cols, vals)

    x0 = 10.0 * rng.random(n_arcs)
    out_flow = np.bincount(src, weights=x0, minlength=S)
    in_flow = np.bincount(dst, weights=x0, minlength=D)
    b = np.concatenate([1.2 * out_flow, in_flow])
    sense = np.concatenate([np.full(S, SENSE_L, np.uint8), np.full(D, SENSE_E, np.uint8)])
    c = rng.uniform(1.0, 100.0, size=n_arcs)
    return LP(
        m=S + D,
        n=n_arcs,
        row_ptr=row_ptr,
        col_idx=col_idx,
        val=val,
        b=b,
        c=c,
        lb=np.zeros(n_arcs),
        ub=np.full(n_arcs, np.inf),
        sense=sense,
        name=f"transport_m{S + D}_n{n_arcs}",
        meta={"x_feasible": x0},
    )


def powerlaw_degrees(rng, n, nnz_target, exponent=2.1, dmax=100_000):
    """Column degrees d_j = min(ceil(x_min * U^(-1/(exponent-1))), dmax), with x_min
    set by bisection so that sum(d) is close to ``nnz_target``."""
    u = rng.random(n)
    tail = u ** (-1.0 / (exponent - 1.0))

    def total(xmin):
        return np.minimum(np.ceil(xmin * tail), dmax).sum()

    lo, hi = 1e-6, float(nnz_target) / n
    for _ in range(80):
        mid = 0.5 * (lo + hi)
        if total(mid) < nnz_target:
            lo = mid
        else:
            hi = mid
    return np.minimum(np.ceil(hi * tail), dmax).astype(np.int64)


def powerlaw(seed=0, m=2_000_000, n=5_000_000, nnz_target=30_000_000, exponent=2.1, dmax=100_000):
    """Large sparse LP with power-law column degrees (see module docstring)."""
    rng = np.random.default_rng(seed)
    deg = powerlaw_degrees(rng, n, nnz_target, exponent, min(dmax, m))
    rows, cols = _distinct_rows_per_column(rng, m, deg)
    mag = 10.0 ** rng.uniform(-3.0, 3.0, size=rows.size)
    vals = np.where(rng.random(rows.size) < 0.5, -mag, mag)
    return from_pattern(
        m, n, rows, cols, vals, rng,
        sense_probs=(0.3, 0.7, 0.0), var_probs=(0.8, 0.0, 0.2),
        p_at_lower=0.3, p_at_upper=0.1, name=f"powerlaw_m{m}_n{n}",
    )


def mixed_small(seed=0, m=60, n=150, col_nnz=(1, 6)):
    """Small LP with every row sense and every bound kind (box, lower-only,
    free), ragged column degrees and a few empty rows and columns."""
    rng = np.random.default_rng(seed)
    deg = rng.integers(col_nnz[0], col_nnz[1] + 1, size=n)
    deg[rng.random(n) < 0.05] = 0  # some empty columns
    rows, cols = _distinct_rows_per_column(rng, m - 3, deg)  # last 3 rows stay empty
    vals = rng.standard_normal(rows.size)
    return from_pattern(
        m, n, rows, cols, vals, rng,
        sense_probs=(0.4, 0.3, 0.3), var_probs=(0.5, 0.3, 0.2),
        p_at_lower=0.3, p_at_upper=0.15, name=f"mixed_small_m{m}_n{n}",
    )


def row_length_mix(seed=0, lengths=(0, 1, 2, 3, 5, 8, 9, 16, 17, 31, 32, 33, 64, 200, 1100, 3000), n=4000, reps=3):
    """LP whose rows of A have the given lengths (each repeated ``reps`` times,
    shuffled) and whose columns (rows of A^T) get ragged lengths as a result,
    including a few very long columns.  For covering every row-length bin of a
    sparse product, including the empty row and the ragged tail."""
    rng = np.random.default_rng(seed)
    lens = np.repeat(np.asarray(lengths, dtype=np.int64), reps)
    rng.shuffle(lens)
    m = lens.size
    rows_l, cols_l = [], []
    hot = rng.choice(n, size=4, replace=False)  # a few columns shared by many rows
    for i, L in enumerate(lens):
        if L == 0:
            continue
        L = min(int(L), n)
        cs = rng.choice(n, size=L, replace=False)
        if L > 4:
            cs[:2] = hot[:2]
            cs = np.unique(cs)
        rows_l.append(np.full(cs.size, i))
        cols_l.append(cs)
    rows = np.concatenate(rows_l)
    cols = np.concatenate(cols_l)
    vals = rng.standard_normal(rows.size)
    return from_pattern(
        m, n, rows, cols, vals, rng,
        sense_probs=(0.5, 0.25, 0.25), var_probs=(0.6, 0.2, 0.2),
        p_at_lower=0.3, p_at_upper=0.1, name=f"row_length_mix_m{m}_n{n}",
    )


def long_rows(seed=0, m=9000, n=12000, row_lengths=(4097, 8192, 11000), col_lengths=(4097, 6000, 8192),
              background=(2, 4)):
    """Sparse LP with a few rows of A and a few columns (rows of A^T) far longer
    than the rest: the given lengths exactly, on a background of 2-4 nonzeros
    per column.  For the products that cut very long rows into segments reduced
    by several blocks (lengths just above, at and between segment multiples)."""
    rng = np.random.default_rng(seed)
    deg = rng.integers(background[0], background[1] + 1, size=n)
    br, bc = _distinct_rows_per_column(rng, m, deg)
    long_r = rng.choice(m, size=len(row_lengths), replace=False)
    long_c = rng.choice(n, size=len(col_lengths), replace=False)
    keys = [bc * m + br]
    for r, L in zip(long_r, row_lengths):
        keys.append(rng.choice(n, size=L, replace=False) * m + r)
    for c, L in zip(long_c, col_lengths):
        keys.append(c * m + rng.choice(m, size=L, replace=False))
    key = _sorted_unique(np.concatenate(keys))
    rows, cols = key % m, key // m
    # the long rows / columns hold exactly their lengths, except for entries
    # shared with another long line or the background; trim those from the background
    keep = np.ones(key.size, dtype=bool)
    for r, L in zip(long_r, row_lengths):
        idx = np.flatnonzero(rows == r)
        extra = idx.size - L
        if extra > 0:
            bg = idx[~np.isin(cols[idx], long_c)]
            keep[bg[:extra]] = False
    for c, L in zip(long_c, col_lengths):
        idx = np.flatnonzero((cols == c) & keep)
        extra = idx.size - L
        if extra > 0:
            bg = idx[~np.isin(rows[idx], long_r)]
            keep[bg[:extra]] = False
    rows, cols = rows[keep], cols[keep]
    vals = rng.standard_normal(rows.size)
    return from_pattern(
        m, n, rows, cols, vals, rng,
        sense_probs=(0.4, 0.3, 0.3), var_probs=(0.6, 0.2, 0.2),
        p_at_lower=0.3, p_at_upper=0.1, name=f"long_rows_m{m}_n{n}",
    )


def batch_sizes(seed=0, count=512, m_lo=100, m_hi=20_000):
    """Sizes m = floor(10^U(log10 m_lo, log10 m_hi)) for a batch of small LPs (n = 2.5 m)."""
    rng = np.random.default_rng(seed)
    ms = np.floor(10.0 ** rng.uniform(np.log10(m_lo), np.log10(m_hi), size=count)).astype(np.int64)
    return ms, (2.5 * ms).astype(np.int64)


def batch_member(seed, m, n, nnz_lo=4, nnz_hi=8):
    """One member of a batch of small LPs: the tiny_random recipe with 4-8 nonzeros per column."""
    rng = np.random.default_rng(seed)
    deg = rng.integers(nnz_lo, nnz_hi + 1, size=n)
    deg = np.minimum(deg, m)
    rows, cols = _distinct_rows_per_column(rng, m, deg)
    vals = rng.standard_normal(rows.size)
    return from_pattern(
        m, n, rows, cols, vals, rng,
        sense_probs=(1.0, 0.0, 0.0), var_probs=(1.0, 0.0, 0.0),
        p_at_lower=0.5, p_at_upper=0.0, name=f"batch_member_m{m}_n{n}_s{seed}",
    )
