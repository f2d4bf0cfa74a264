"""Online-preconditioned PDHG for LP, written out step by step in numpy float64.

TEST INFRASTRUCTURE ONLY (see the package docstring): the CUDA library never
imports this module.

Source: H. Lu and W. Zhang, "Enhanced PDHG for Linear Programming with Online
Preconditioning" (arXiv 2506.17650).  Equation numbers below follow the
paper's numbering: Eq. (1) standard-form LP, Eq. (2) saddle point, Eq. (3)
preconditioned PDHG, Eq. (5) online losses, Eq. (6) PDHG with adaptive step
and primal weight, Eq. (7) online gradients; Algorithm 1 is the one-step
iteration with online preconditioning.  The paper's dual variable lambda is
called ``y`` here.

Problem form (Eq. (1) generalised to row senses and variable bounds)::

    min c^T x   s.t.  A_i x (= | <= | >=) b_i,   l <= x <= u

with Lagrangian L(x, y) = c^T x - y^T A x + b^T y (Eq. (2)), y_i free for
equality rows, y_i >= 0 for >= rows and y_i <= 0 for <= rows.

Readings of points the paper leaves open (each is a decision, not a quote):

* R1 dual loss at x^k: the dual online gradient uses b - A x^k (Eq. (5), Eq. (7)).
* R2 the primal indicator I(x^{k+1/2} >= 0) becomes I(l <= x^{k+1/2} <= u).
* R3 inequality rows project y onto its sign cone; the dual gradient carries the
  projection's derivative I(y^{k+1/2} inside the cone).
* R4 the eta/omega and eta*omega factors of Eq. (7) are kept.
* R5 proj onto the candidate preconditioners = entry-wise max(P, floor), floor 1e-6.
* R6 AdaGrad (Section 4.1) = diagonal AdaGrad: G_j += grad_j^2,
  P_j -= alpha grad_j / sqrt(G_j) (no step where G_j = 0).  Alternatives:
  "adagrad_norm" (one accumulator per side, G += ||grad||^2) and "const".
* R7 k in "k mod phi" counts accepted steps since the start of the solve, from 0;
  phi <= 0 never updates.
* R8 adaptive step (PDLP prior art): eta_max = (omega ||dx||^2_{T^-1} +
  ||dy||^2_{Sigma^-1} / omega) / (2 |dy^T A dx|); accept iff eta <= eta_max;
  next eta = min((1 - (t+1)^-0.3) eta_max, (1 + (t+1)^-0.6) eta), t = attempts so far.
  An interaction of exactly 0 gives eta_max = inf; a non-finite step that
  makes eta_max NaN rejects the attempt, and the next eta is then the growth
  term (1 + (t+1)^-0.6) eta alone.
* R9 restarts (PDLP prior art): every ``check_every`` attempts, candidate =
  current or eta-weighted average, whichever has the smaller weighted KKT
  K_w = sqrt(w^2 ||pres||^2 + ||dres||^2 / w^2 + gap^2) (scaled space);
  restart if K <= 0.2 K_last, or K <= 0.8 K_last and K > K_previous_check, or
  attempts since the last restart >= 0.36 attempts in total.  On restart the
  primal weight becomes exp(0.5 log(||dy|| / ||dx||) + 0.5 log w) (changes
  measured from the last restart point, skipped below 1e-10) and T, Sigma are
  kept (Section 3.2).
* R10 termination: relative KKT on the unscaled problem (2-norms):
  ||pres|| <= eps (1 + ||b||), ||dres|| <= eps (1 + ||c||),
  |pobj - dobj| <= eps (1 + |pobj| + |dobj|); checked on the current iterate
  and (pdlp mode) on the average, current first.
* R11 Ruiz: each round divides rows and columns by the square root of their
  infinity norms, from the current scaled matrix (Section 2).
* R12 L2 rescaling (Section 4.2): rows and columns divided by the square root
  of their 2-norms.
* R13 plain (vanilla) mode: T_0 = Sigma_0 = 1 with eta = 0.9 / ||A~||_2 fixed,
  omega = ||c~|| / ||b~||, no restarts or averages.  ||A~||_2 by power iteration
  from the all-ones direction, restarted from a fixed +-1 vector (SplitMix64
  signs of the column index) when A~ 1 = 0.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp

SENSE_E = ord("E")
SENSE_L = ord("L")
SENSE_G = ord("G")

OPTIMAL = 1
ITERATION_LIMIT = 2
TIME_LIMIT = 3
NUMERICAL_ERROR = 4


@dataclass
class Options:
    mode: str = "pdlp"  # "pdlp": Eq. (6) with adaptive step, restarts, primal weight; "plain": vanilla PDHG
    alpha: float = 0.0  # online learning rate
    phi: int = 20  # update period (Section 3.2, infrequent update); <= 0 means never
    normalize: bool = True  # normalised online loss (Section 3.2)
    scheduler: str = "adagrad"  # "adagrad" | "adagrad_norm" | "const"
    precond_floor: float = 1e-6
    ruiz_iters: int = 10
    pc_beta: float = 1.0  # Pock-Chambolle exponent (pdlp mode)
    check_every: int = 64
    restart: bool = True
    power_iters: int = 200  # for ||A~||_2 in plain mode
    plain_step_factor: float = 0.9


@dataclass
class Scaled:
    """The preprocessed LP: A~ = diag(dr) A diag(dc), b~ = dr b, c~ = dc c,
    l~ = l / dc, u~ = u / dc.  Unscaled x = dc * x~, y = dr * y~."""

    A: sp.csr_matrix
    At: sp.csr_matrix
    b: np.ndarray
    c: np.ndarray
    l: np.ndarray
    u: np.ndarray
    sense: np.ndarray
    dr: np.ndarray
    dc: np.ndarray
    b_norm: float  # ||b||_2 of the unscaled problem
    c_norm: float  # ||c||_2 of the unscaled problem


@dataclass
class State:
    x: np.ndarray
    y: np.ndarray
    ax: np.ndarray  # A~ x, kept with x
    T: np.ndarray
    Sigma: np.ndarray
    GT: np.ndarray  # AdaGrad accumulators
    GS: np.ndarray
    GT_norm: float
    GS_norm: float
    eta: float
    omega: float
    k: int = 0  # accepted steps
    attempts: int = 0  # all step attempts (accepted or not)
    xbar: np.ndarray | None = None  # eta-weighted sums since the last restart
    ybar: np.ndarray | None = None
    wsum: float = 0.0
    x_last: np.ndarray | None = None  # last restart point
    y_last: np.ndarray | None = None
    K_last_parts: tuple = (0.0, 0.0, 0.0)
    K_prev: float = math.inf
    last_restart_attempt: int = 0
    restarts: int = 0
    checked0: bool = False  # the check before the first attempt has run
    status: int | None = None
    stats: dict = field(default_factory=dict)


@dataclass
class Result:
    x: np.ndarray
    y: np.ndarray
    status: int
    pobj: float
    dobj: float
    rel_pres: float
    rel_dres: float
    rel_gap: float
    iterations: int
    accepted: int
    restarts: int


# --------------------------------------------------------------------------
# Preprocessing (Section 2: Ruiz and Pock-Chambolle; Section 4.2: L2 rescaling)
# --------------------------------------------------------------------------

def _apply(A, fr, fc):
    return (sp.diags(fr) @ A @ sp.diags(fc)).tocsr()


def ruiz_equilibrate(A, iters):
    """Ruiz equilibration (Section 2, Ruiz preconditioning; reading R11).

    Each round computes the infinity norm of every row and column of the
    current scaled matrix and divides rows and columns by their square roots
    (empty rows/columns keep factor 1).  Returns (A~, dr, dc).
    Pinned by: row/column infinity norms tend to 1 (tests).
    """
    A = A.tocsr(copy=True)
    m, n = A.shape
    dr = np.ones(m)
    dc = np.ones(n)
    for _ in range(iters):
        absA = abs(A)
        if A.nnz:
            r = np.asarray(absA.max(axis=1).todense()).ravel()
            c = np.asarray(absA.max(axis=0).todense()).ravel()
        else:  # no entries (e.g. m = 0): every factor stays 1
            r, c = np.zeros(m), np.zeros(n)
        r[r == 0] = 1.0
        c[c == 0] = 1.0
        fr = 1.0 / np.sqrt(r)
        fc = 1.0 / np.sqrt(c)
        A = _apply(A, fr, fc)
        dr *= fr
        dc *= fc
    return A, dr, dc


def pock_chambolle_rescale(A, beta=1.0):
    """Pock-Chambolle diagonal rescaling (Section 2): rows divided by
    sqrt(sum_j |A_ij|^beta), columns by sqrt(sum_i |A_ij|^(2-beta)).
    Pinned by: ||A~||_2 <= 1 for beta = 1 (tests)."""
    absA = abs(A)
    r = np.asarray(absA.power(beta).sum(axis=1)).ravel()
    c = np.asarray(absA.power(2.0 - beta).sum(axis=0)).ravel()
    r[r == 0] = 1.0
    c[c == 0] = 1.0
    fr = 1.0 / np.sqrt(r)
    fc = 1.0 / np.sqrt(c)
    return _apply(A, fr, fc), fr, fc


def l2_norm_rescale(A):
    """L2-norm rescaling (Section 4.2; reading R12): rows and columns divided
    by the square roots of their 2-norms.
    Pinned by: every row and column 2-norm is sqrt-equilibrated on a rank-one
    pattern (tests)."""
    A2 = A.multiply(A)
    r = np.sqrt(np.asarray(A2.sum(axis=1)).ravel())
    c = np.sqrt(np.asarray(A2.sum(axis=0)).ravel())
    r[r == 0] = 1.0
    c[c == 0] = 1.0
    fr = 1.0 / np.sqrt(r)
    fc = 1.0 / np.sqrt(c)
    return _apply(A, fr, fc), fr, fc


def splitmix_signs(n):
    """+1 or -1 for each index j < n: the top bit of SplitMix64 of j (the
    generator of G. Steele, D. Lea and C. Flood, "Fast splittable pseudorandom
    number generators", OOPSLA 2014: state j * 0x9E3779B97F4A7C15 after one
    increment, then the two xor-shift-multiply rounds and a final xor-shift);
    a set top bit gives -1.  Pinned by: hand values of the published mixer (tests)."""
    with np.errstate(over="ignore"):
        z = (np.arange(n, dtype=np.uint64) + np.uint64(1)) * np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return np.where((z >> np.uint64(63)) != 0, -1.0, 1.0)


def power_spectral_norm(A, iters):
    """||A||_2 by power iteration on A^T A from the all-ones direction:
    v <- w / ||w||, w = A^T A v, for ``iters`` rounds; returns sqrt(||w||) of the
    last round.  If the first product is exactly zero (every row of A sums to
    zero, so the all-ones direction is in its null space), the iteration
    starts again from the SplitMix64 sign vector (reading R13).  Pinned by:
    agreement with the SVD norm, also on a matrix whose rows sum to zero (tests)."""
    n = A.shape[1]
    if n == 0 or A.nnz == 0:
        return 0.0
    for start in (np.ones(n), splitmix_signs(n)):
        v = start / math.sqrt(n)
        nw = 0.0
        for it in range(iters):
            w = A.T @ (A @ v)
            nw = float(np.linalg.norm(w))
            if nw == 0.0:
                break
            v = w / nw
        if nw > 0.0:
            return math.sqrt(nw)
        if it > 0:  # only a zero first product restarts
            return 0.0
    return 0.0


def scale_problem(lp, opts: Options) -> Scaled:
    """Preprocess: Ruiz (``ruiz_iters`` rounds), then Pock-Chambolle (pdlp
    mode, Section 4.3 uses cuPDLP.jl defaults) or L2 rescaling (plain mode,
    Section 4.2).  Bounds, costs and right-hand side are rescaled with the
    same diagonal factors.  Pinned by: the closed forms of its stages (below)
    and the optimum it preserves (HiGHS on the original and the scaled LP)."""
    A = sp.csr_matrix((lp.val, lp.col_idx, lp.row_ptr), shape=(lp.m, lp.n))
    A.sum_duplicates()
    A.sort_indices()
    As, dr, dc = ruiz_equilibrate(A, opts.ruiz_iters)
    if opts.mode == "pdlp":
        As, fr, fc = pock_chambolle_rescale(As, opts.pc_beta)
    else:
        As, fr, fc = l2_norm_rescale(As)
    dr = dr * fr
    dc = dc * fc
    with np.errstate(invalid="ignore"):
        l = lp.lb / dc
        u = lp.ub / dc
    return Scaled(
        A=As,
        At=As.T.tocsr(),
        b=dr * lp.b,
        c=dc * lp.c,
        l=l,
        u=u,
        sense=np.asarray(lp.sense, dtype=np.uint8),
        dr=dr,
        dc=dc,
        b_norm=float(np.linalg.norm(lp.b)),
        c_norm=float(np.linalg.norm(lp.c)),
    )


# --------------------------------------------------------------------------
# The iteration
# --------------------------------------------------------------------------

def lagrangian(P: Scaled, x, y):
    """L(x, y) = c^T x - y^T A x + b^T y (Eq. (2)).  Pinned by: L(x*, y*) =
    c^T x* at constructed optima, and a value worked by hand."""
    return float(P.c @ x - y @ (P.A @ x) + P.b @ y)


def initial_state(P: Scaled, opts: Options) -> State:
    """x_0 = proj_[l,u](0), y_0 = 0, T_0 = I, Sigma_0 = I (Section 3.2);
    omega_0 = ||c~|| / ||b~|| (1 if either is 0); eta_0 = 1 / max|A~_ij| in pdlp
    mode, 0.9 / ||A~||_2 in plain mode (reading R13).  Pinned by: special
    cases (box positions of 0, b = 0) and the SVD norm (tests)."""
    m, n = P.A.shape
    x = np.minimum(np.maximum(np.zeros(n), P.l), P.u)
    y = np.zeros(m)
    bn = float(np.linalg.norm(P.b))
    cn = float(np.linalg.norm(P.c))
    omega = cn / bn if (bn > 0 and cn > 0) else 1.0
    if opts.mode == "pdlp":
        amax = float(abs(P.A).max()) if P.A.nnz else 0.0
        eta = 1.0 / amax if amax > 0 else 1.0
    else:
        nrm = power_spectral_norm(P.A, opts.power_iters)
        eta = opts.plain_step_factor / nrm if nrm > 0 else 1.0
    return State(
        x=x, y=y, ax=P.A @ x,
        T=np.ones(n), Sigma=np.ones(m), GT=np.zeros(n), GS=np.zeros(m),
        GT_norm=0.0, GS_norm=0.0, eta=eta, omega=omega,
        xbar=np.zeros(n), ybar=np.zeros(m),
    )


def primal_half_step(P: Scaled, x, y, T, eta, omega):
    """x^{k+1} = proj_[l,u](x^k - (eta/omega) T (c - A^T y^k)) (Eq. (6), first line).
    Returns (x^{k+1}, g = c - A^T y^k, x^{k+1/2}).  Pinned by: the
    hand-derived steps of tests/golden/one_step_1x2.json."""
    g = P.c - P.At @ y
    x_half = x - (eta / omega) * T * g
    x_new = np.minimum(np.maximum(x_half, P.l), P.u)
    return x_new, g, x_half


def project_dual(P: Scaled, y_half):
    """Projection of y onto its sign cone per row sense (reading R3).
    Pinned by: hand values for each sense (tests)."""
    y = y_half.copy()
    g = P.sense == SENSE_G
    l = P.sense == SENSE_L
    y[g] = np.maximum(y[g], 0.0)
    y[l] = np.minimum(y[l], 0.0)
    return y


def dual_feasible_mask(P: Scaled, y_half):
    """I(y^{k+1/2} inside the sign cone of its row), inclusive at 0 (reading R3).
    Pinned by: hand values for each sense (tests)."""
    return np.where(P.sense == SENSE_G, y_half >= 0.0,
                    np.where(P.sense == SENSE_L, y_half <= 0.0, True))


def dual_half_step(P: Scaled, x_new, y, ax, Sigma, eta, omega):
    """y^{k+1} = proj(y^k + eta omega Sigma (b - A(2 x^{k+1} - x^k))) (Eq. (6), second line).
    Returns (y^{k+1}, A x^{k+1}, r = b - A(2x^{k+1} - x^k), y^{k+1/2}).
    Pinned by: the hand-derived steps of tests/golden/one_step_1x2.json."""
    ax_new = P.A @ x_new
    r = P.b - (2.0 * ax_new - ax)
    y_half = y + (eta * omega) * Sigma * r
    return project_dual(P, y_half), ax_new, r, y_half


def online_gradients(P: Scaled, g, x_half, ax, r, y_half, eta, omega, normalize):
    """Diagonals of the online gradients (Eq. (7), readings R1-R4):

        grad_T_j     = -(eta/omega) g_j^2 I(l_j <= x^{k+1/2}_j <= u_j)
        grad_Sigma_i = -(eta omega) (b - A x^k)_i r_i I(y^{k+1/2}_i in cone)

    With ``normalize`` they are divided by ||g||^2 and ||b - A x^k||^2
    (Algorithm 1, normalised loss); a side whose norm is 0 returns None (no
    update).  Pinned by: central finite differences of the losses Eq. (5)
    evaluated from the Lagrangian (tests)."""
    ind_p = (x_half >= P.l) & (x_half <= P.u)
    grad_T = -(eta / omega) * (g * ind_p) * g
    res = P.b - ax
    ind_d = dual_feasible_mask(P, y_half)
    grad_S = -(eta * omega) * res * r * ind_d
    if normalize:
        gn = float(g @ g)
        rn = float(res @ res)
        grad_T = grad_T / gn if gn > 0 else None
        grad_S = grad_S / rn if rn > 0 else None
    return grad_T, grad_S


def ogd_update(Pvec, Gacc, Gnorm, grad, opts: Options):
    """One projected online-gradient step P <- proj[P - alpha grad] with the
    AdaGrad learning-rate rule (Section 3.1 OGD, Section 4.1 AdaGrad;
    readings R5, R6).  Returns (P, G, Gnorm).  Pinned by: hand values of one
    step of each rule (diagonal AdaGrad in tests/golden/one_step_1x2.json,
    scalar AdaGrad and the constant rate in tests/golden/step_rules_1x1.json,
    floor included); T never decreases, Sigma stays >= floor, alpha = 0
    leaves P unchanged bit for bit (tests)."""
    if grad is None:
        return Pvec, Gacc, Gnorm
    a = opts.alpha
    if opts.scheduler == "adagrad":
        Gacc = Gacc + grad * grad
        step = np.zeros_like(grad)
        nz = Gacc > 0
        step[nz] = grad[nz] / np.sqrt(Gacc[nz])
        Pvec = Pvec - a * step
    elif opts.scheduler == "adagrad_norm":
        Gnorm = Gnorm + float(grad @ grad)
        if Gnorm > 0:
            Pvec = Pvec - a * (grad / math.sqrt(Gnorm))
    elif opts.scheduler == "const":
        Pvec = Pvec - a * grad
    else:
        raise ValueError(opts.scheduler)
    return np.maximum(Pvec, opts.precond_floor), Gacc, Gnorm


def step_size_limit(dx, dy, dax, T, Sigma, omega):
    """Largest step the adaptive rule accepts (reading R8):
    (omega ||dx||^2_{T^-1} + ||dy||^2_{Sigma^-1} / omega) / (2 |dy^T A dx|).
    Pinned by: it is >= 1 / ||Sigma^1/2 A T^1/2||_2 for every (dx, dy) (tests)."""
    movement = omega * float(np.sum(dx * dx / T)) + float(np.sum(dy * dy / Sigma)) / omega
    interaction = abs(float(np.sum(dy * dax)))
    if interaction == 0.0:
        return math.inf
    return movement / (2.0 * interaction)


def attempt(P: Scaled, S: State, opts: Options) -> bool:
    """One step attempt of Algorithm 1 with Eq. (6).  Returns True if accepted.

    pdlp mode: the step is accepted iff eta <= eta_max (reading R8); a rejected
    attempt leaves (x, y, T, Sigma) unchanged and retries with the new eta.
    On acceptance: if k mod phi = 0 the preconditioners take one online step
    (Algorithm 1), the eta-weighted averages are updated, and k increases.

    Pinned by: the hand-derived steps and the rejected attempt of
    tests/golden/one_step_1x2.json (half-steps, gradients, eta_max), and the
    attempts worked by hand in tests/golden/step_rules_1x1.json: the next
    step size at attempt 1023, where the factors are exactly 7/8 and 65/64
    (both terms of the min), the averages weighted by the step each accepted
    attempt used, and the update points k = 0, phi, 2 phi counted in accepted
    steps across a rejected attempt (and, in a test, across restarts).  The
    step-size rule itself (exponents 0.3 / 0.6) is a prior-art reading the
    paper does not fix."""
    eta, omega = S.eta, S.omega
    update_now = opts.phi > 0 and (S.k % opts.phi == 0)
    x_new, g, x_half = primal_half_step(P, S.x, S.y, S.T, eta, omega)
    y_new, ax_new, r, y_half = dual_half_step(P, x_new, S.y, S.ax, S.Sigma, eta, omega)
    S.attempts += 1
    if opts.mode == "pdlp":
        eta_max = step_size_limit(x_new - S.x, y_new - S.y, ax_new - S.ax, S.T, S.Sigma, omega)
        accept = eta <= eta_max
        t = S.attempts
        if math.isnan(eta_max):  # no limit could be formed (non-finite step): grow from eta
            eta_next = (1.0 + (t + 1) ** -0.6) * eta
        else:
            eta_next = min((1.0 - (t + 1) ** -0.3) * eta_max, (1.0 + (t + 1) ** -0.6) * eta)
    else:
        accept = True
        eta_next = eta
    if accept:
        if update_now:
            gT, gS = online_gradients(P, g, x_half, S.ax, r, y_half, eta, omega, opts.normalize)
            S.T, S.GT, S.GT_norm = ogd_update(S.T, S.GT, S.GT_norm, gT, opts)
            S.Sigma, S.GS, S.GS_norm = ogd_update(S.Sigma, S.GS, S.GS_norm, gS, opts)
        if opts.mode == "pdlp":
            S.xbar = S.xbar + eta * x_new
            S.ybar = S.ybar + eta * y_new
            S.wsum = S.wsum + eta
        S.x, S.y, S.ax = x_new, y_new, ax_new
        S.k += 1
    S.eta = eta_next
    return accept


# --------------------------------------------------------------------------
# KKT, restarts, termination
# --------------------------------------------------------------------------

def kkt(P: Scaled, x, y, ax, aty):
    """Relative KKT quantities of (x, y) (reading R10), given A~ x and A~^T y.

    Primal residual (user units): (A x - b)_i for = rows, max(b_i - A_i x, 0)
    for >= rows, max(A_i x - b_i, 0) for <= rows.  Reduced cost rc = c - A^T y
    is split per variable: both bounds finite -> all of it is a bound
    multiplier; only l finite -> multiplier max(rc, 0), residual min(rc, 0);
    only u finite -> multiplier min(rc, 0), residual max(rc, 0); free ->
    residual rc.  Dual objective = b^T y + sum l_j max(lam_j, 0) - sum u_j
    max(-lam_j, 0).  Pinned by: a hand-computed example, and ~0 at an optimal
    pair known by construction (tests)."""
    rs = ax - P.b
    pres_s = np.where(P.sense == SENSE_E, rs,
                      np.where(P.sense == SENSE_G, np.maximum(-rs, 0.0), np.maximum(rs, 0.0)))
    pres = pres_s / P.dr
    rc = P.c - aty
    lf = np.isfinite(P.l)
    uf = np.isfinite(P.u)
    lam = np.where(lf & uf, rc, np.where(lf, np.maximum(rc, 0.0), np.where(uf, np.minimum(rc, 0.0), 0.0)))
    dres_s = rc - lam
    dres = dres_s / P.dc
    pobj = float(P.c @ x)
    lo_term = np.where(lf, P.l, 0.0) * np.maximum(lam, 0.0)
    up_term = np.where(uf, P.u, 0.0) * np.maximum(-lam, 0.0)
    dobj = float(P.b @ y) + float(lo_term.sum()) - float(up_term.sum())
    gap = pobj - dobj
    pn = float(np.linalg.norm(pres))
    dn = float(np.linalg.norm(dres))
    return dict(
        pobj=pobj,
        dobj=dobj,
        pres_norm=pn,
        dres_norm=dn,
        rel_pres=pn / (1.0 + P.b_norm),
        rel_dres=dn / (1.0 + P.c_norm),
        rel_gap=abs(gap) / (1.0 + abs(pobj) + abs(dobj)),
        parts=(float(pres_s @ pres_s), float(dres_s @ dres_s), gap * gap),
    )


def _kw(parts, omega):
    p2, d2, g2 = parts
    return math.sqrt(omega * omega * p2 + d2 / (omega * omega) + g2)


def _converged(kk, tol):
    return kk["rel_pres"] <= tol and kk["rel_dres"] <= tol and kk["rel_gap"] <= tol


def check(P: Scaled, S: State, opts: Options, tol: float, eval_only: bool = False):
    """KKT check, termination and (pdlp mode) restart decision (readings R9, R10).

    ``eval_only`` only refreshes ``S.stats`` for the current iterate.

    Pinned by: the KKT quantities (``kkt``, hand-computed example),
    convergence to the vertex / HiGHS optimum, and restart decisions worked by
    hand on a 1x1 LP for each condition of the restart reading (sufficient
    decay, decay without progress, long period, candidate choice, primal
    weight).  The reading itself (PDLP prior art, constants 0.2 / 0.8 /
    0.36) is not fixed by the paper."""
    aty = P.At @ S.y
    cur = kkt(P, S.x, S.y, S.ax, aty)
    if eval_only:
        S.stats = cur
        return
    cands = [("current", S.x, S.y, S.ax, cur)]
    if opts.mode == "pdlp" and S.wsum > 0:
        xa = S.xbar / S.wsum
        ya = S.ybar / S.wsum
        axa = P.A @ xa
        avg = kkt(P, xa, ya, axa, P.At @ ya)
        cands.append(("average", xa, ya, axa, avg))
    S.stats = cur
    vals = [v for c in cands for v in (c[4]["rel_pres"], c[4]["rel_dres"], c[4]["rel_gap"])]
    if not all(math.isfinite(v) for v in vals):
        S.status = NUMERICAL_ERROR
        return
    for name, xx, yy, aa, kk in cands:
        if _converged(kk, tol):
            S.x, S.y, S.ax = xx.copy(), yy.copy(), aa.copy()
            S.stats = kk
            S.status = OPTIMAL
            return
    if opts.mode != "pdlp":
        return
    if S.x_last is None:
        # first check that does not terminate: the current point is the first restart reference
        S.x_last, S.y_last = S.x.copy(), S.y.copy()
        S.K_last_parts = cur["parts"]
        S.K_prev = _kw(cur["parts"], S.omega)
        S.last_restart_attempt = S.attempts
        return
    if not opts.restart:
        return
    kc = [_kw(c[4]["parts"], S.omega) for c in cands]
    pick = 1 if (len(cands) > 1 and kc[1] < kc[0]) else 0
    K = kc[pick]
    K_last = _kw(S.K_last_parts, S.omega)
    since = S.attempts - S.last_restart_attempt
    do_restart = (K <= 0.2 * K_last) or (K <= 0.8 * K_last and K > S.K_prev) or (since >= 0.36 * S.attempts)
    S.K_prev = K
    if not do_restart:
        return
    _, xx, yy, aa, kk = cands[pick]
    dx = float(np.linalg.norm(xx - S.x_last))
    dy = float(np.linalg.norm(yy - S.y_last))
    if dx > 1e-10 and dy > 1e-10:
        S.omega = math.exp(0.5 * math.log(dy / dx) + 0.5 * math.log(S.omega))
    S.x, S.y, S.ax = xx.copy(), yy.copy(), aa.copy()
    S.x_last, S.y_last = S.x.copy(), S.y.copy()
    S.xbar = np.zeros_like(S.xbar)
    S.ybar = np.zeros_like(S.ybar)
    S.wsum = 0.0
    S.K_last_parts = kk["parts"]
    S.last_restart_attempt = S.attempts
    S.restarts += 1


def unscale(P: Scaled, S: State):
    """User-unit primal and dual: x = dc x~, y = dr y~.  Pinned by: the
    unscaled optimum against HiGHS and the constructed optima (tests)."""
    return P.dc * S.x, P.dr * S.y


def solve(lp, opts: Options, tol=1e-4, iter_limit=50_000, trace=None, P=None, S=None):
    """Run attempts until a check finds the relative KKT tolerance met or
    ``iter_limit`` attempts (counted since the start) are done.  A check runs
    before the first attempt and after every ``check_every``-th attempt; at the
    iteration limit off a check boundary only the current iterate's KKT is
    re-evaluated.  ``trace(P, S)`` is called after every attempt (after that
    attempt's check, if any).  Returns (Result, P, S).  Pinned by: optima from
    vertex enumeration and HiGHS, and the generators' constructed optima."""
    if P is None:
        P = scale_problem(lp, opts)
    if S is None:
        S = initial_state(P, opts)
    S.status = None
    if not S.checked0:
        check(P, S, opts, tol)
        S.checked0 = True
    while S.status is None and S.attempts < iter_limit:
        attempt(P, S, opts)
        if S.attempts % opts.check_every == 0:
            check(P, S, opts, tol)
        if trace is not None:
            trace(P, S)
    if S.status is None:
        S.status = ITERATION_LIMIT
        if S.attempts % opts.check_every != 0:
            check(P, S, opts, tol, eval_only=True)
    x, y = unscale(P, S)
    st = S.stats
    res = Result(
        x=x, y=y, status=S.status, pobj=st["pobj"], dobj=st["dobj"],
        rel_pres=st["rel_pres"], rel_dres=st["rel_dres"], rel_gap=st["rel_gap"],
        iterations=S.attempts, accepted=S.k, restarts=S.restarts,
    )
    return res, P, S
