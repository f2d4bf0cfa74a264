"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

Nothing here compares the oracle with itself: each check uses a hand-derived
fixture, a closed form, an invariant, a library routine the oracle does not
call for that step (SVD norm, HiGHS), or brute force on tiny inputs.
"""
import math

import numpy as np
import pytest
import scipy.sparse as sp
from scipy.optimize import linprog

import lpgen
import oracle
from oracle.pdhg import Scaled, State
from tests.conftest import arr, load_golden

SENSE = {"E": ord("E"), "L": ord("L"), "G": ord("G")}


def _scaled_from_dense(A, b, c, l, u, sense, dr=None, dc=None):
    """Build the oracle's preprocessed-problem object for a given (A, b, c, l, u)
    and explicit diagonal factors (identity by default)."""
    A = np.asarray(A, dtype=np.float64)
    m, n = A.shape
    dr = np.ones(m) if dr is None else np.asarray(dr, dtype=np.float64)
    dc = np.ones(n) if dc is None else np.asarray(dc, dtype=np.float64)
    As = sp.csr_matrix(np.diag(dr) @ A @ np.diag(dc))
    with np.errstate(invalid="ignore"):
        return Scaled(
            A=As, At=As.T.tocsr(), b=dr * np.asarray(b, float), c=dc * np.asarray(c, float),
            l=np.asarray(l, float) / dc, u=np.asarray(u, float) / dc,
            sense=np.array([SENSE[s] for s in sense], dtype=np.uint8), dr=dr, dc=dc,
            b_norm=float(np.linalg.norm(b)), c_norm=float(np.linalg.norm(c)),
        )


def _highs(lp):
    """Optimal objective of an lpgen.LP by HiGHS (scipy)."""
    A = lp.csr().toarray()
    ub_rows, ub_rhs, eq_rows, eq_rhs = [], [], [], []
    for i in range(lp.m):
        s = lp.sense[i]
        if s == SENSE["E"]:
            eq_rows.append(A[i]); eq_rhs.append(lp.b[i])
        elif s == SENSE["L"]:
            ub_rows.append(A[i]); ub_rhs.append(lp.b[i])
        else:
            ub_rows.append(-A[i]); ub_rhs.append(-lp.b[i])
    bounds = [(None if not np.isfinite(lo) else lo, None if not np.isfinite(hi) else hi)
              for lo, hi in zip(lp.lb, lp.ub)]
    res = linprog(lp.c, A_ub=np.array(ub_rows) if ub_rows else None, b_ub=ub_rhs or None,
                  A_eq=np.array(eq_rows) if eq_rows else None, b_eq=eq_rhs or None,
                  bounds=bounds, method="highs")
    assert res.status == 0, res.message
    return res.fun


# ---------------------------------------------------------------------------
# Hand-derived one-step example (tests/golden/one_step_1x2.json)
# ---------------------------------------------------------------------------

def test_golden_two_steps_by_hand():
    g = load_golden("one_step_1x2.json")
    L = g["lp"]
    P = _scaled_from_dense(L["A"], L["b"], L["c"], arr(L["l"]), arr(L["u"]), L["sense"])
    eta, omega = g["start"]["eta"], g["start"]["omega"]
    x = arr(g["start"]["x"]); y = arr(g["start"]["y"]); ax = P.A @ x
    T = np.ones(2); Sig = np.ones(1)
    for key in ("step1", "step2"):
        e = g[key]
        x1, gg, xh = oracle.primal_half_step(P, x, y, T, eta, omega)
        y1, ax1, r, yh = oracle.dual_half_step(P, x1, y, ax, Sig, eta, omega)
        np.testing.assert_allclose(gg, e["g"], rtol=0, atol=1e-15)
        np.testing.assert_allclose(xh, e["x_half"], rtol=0, atol=1e-15)
        np.testing.assert_allclose(x1, e["x"], rtol=0, atol=1e-15)
        np.testing.assert_allclose(ax1, e["ax"], rtol=0, atol=1e-15)
        np.testing.assert_allclose(r, e["r"], rtol=0, atol=1e-15)
        np.testing.assert_allclose(yh, e["y_half"], rtol=0, atol=1e-15)
        np.testing.assert_allclose(y1, e["y"], rtol=0, atol=1e-15)
        gT, gS = oracle.online_gradients(P, gg, xh, ax, r, yh, eta, omega, normalize=False)
        np.testing.assert_allclose(gT, e["grad_T"], rtol=0, atol=1e-15)
        np.testing.assert_allclose(gS, e["grad_Sigma"], rtol=0, atol=1e-15)
        lim = oracle.step_size_limit(x1 - x, y1 - y, ax1 - ax, T, Sig, omega)
        if e["eta_max"] == "inf":
            assert lim == math.inf
        else:
            assert lim == pytest.approx(e["eta_max"], rel=1e-15)
        if key == "step2":
            gTn, gSn = oracle.online_gradients(P, gg, xh, ax, r, yh, eta, omega, normalize=True)
            np.testing.assert_allclose(gTn, e["grad_T_normalized"], rtol=1e-15)
            np.testing.assert_allclose(gSn, e["grad_Sigma_normalized"], rtol=1e-15)
            o = oracle.Options(alpha=e["adagrad_alpha"], scheduler="adagrad")
            Tn, _, _ = oracle.ogd_update(T, np.zeros(2), 0.0, gT, o)
            Sn, _, _ = oracle.ogd_update(Sig, np.zeros(1), 0.0, gS, o)
            np.testing.assert_allclose(Tn, e["T_after"], rtol=1e-15)
            np.testing.assert_allclose(Sn, e["Sigma_after"], rtol=1e-15)
        x, y, ax = x1, y1, ax1


def test_golden_plain_attempts_match_hand_steps():
    """Two plain-mode attempts from the hand example's start reproduce its iterates."""
    g = load_golden("one_step_1x2.json")
    L = g["lp"]
    P = _scaled_from_dense(L["A"], L["b"], L["c"], arr(L["l"]), arr(L["u"]), L["sense"])
    S = State(x=np.zeros(2), y=np.zeros(1), ax=np.zeros(1), T=np.ones(2), Sigma=np.ones(1),
              GT=np.zeros(2), GS=np.zeros(1), GT_norm=0.0, GS_norm=0.0, eta=0.5, omega=1.0,
              xbar=np.zeros(2), ybar=np.zeros(1))
    o = oracle.Options(mode="plain", alpha=0.0, phi=0)
    for key in ("step1", "step2"):
        assert oracle.attempt(P, S, o)
        np.testing.assert_allclose(S.x, g[key]["x"], atol=1e-15)
        np.testing.assert_allclose(S.y, g[key]["y"], atol=1e-15)
    # pdlp mode rejects the second step at eta = 0.5 (limit 13/27)
    S2 = State(x=np.zeros(2), y=np.array([1.5]), ax=np.zeros(1), T=np.ones(2), Sigma=np.ones(1),
               GT=np.zeros(2), GS=np.zeros(1), GT_norm=0.0, GS_norm=0.0, eta=0.5, omega=1.0,
               xbar=np.zeros(2), ybar=np.zeros(1), k=1, attempts=1)
    assert not oracle.attempt(P, S2, oracle.Options(mode="pdlp", phi=0))
    np.testing.assert_array_equal(S2.x, [0.0, 0.0])
    assert S2.k == 1 and S2.attempts == 2
    # the next step stays below the rejected attempt's limit 13/27 (the step
    # size's exact values are pinned in tests/golden/step_rules_1x1.json)
    assert 0.0 < S2.eta < 13 / 27


# ---------------------------------------------------------------------------
# KKT definition (tests/golden/kkt_2x3.json)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("scaled", [False, True])
def test_golden_kkt_by_hand(scaled):
    g = load_golden("kkt_2x3.json")
    dr = np.array([0.5, 3.0]) if scaled else None
    dc = np.array([2.0, 0.25, 7.0]) if scaled else None
    P = _scaled_from_dense(g["A"], g["b"], g["c"], arr(g["l"]), arr(g["u"]), g["sense"], dr, dc)
    x = arr(g["x"]) / P.dc  # the point in scaled coordinates
    y = arr(g["y"]) / P.dr
    k = oracle.kkt(P, x, y, P.A @ x, P.At @ y)
    e = g["expect"]
    for key in ("pobj", "dobj", "pres_norm", "dres_norm", "rel_pres", "rel_dres", "rel_gap"):
        assert k[key] == pytest.approx(e[key], rel=1e-14, abs=1e-15), key
    if not scaled:
        np.testing.assert_allclose(k["parts"], e["parts"], rtol=1e-14)


def test_kkt_zero_at_constructed_optimum():
    for lp in (lpgen.tiny_random(3), lpgen.mixed_small(2)):
        o = oracle.Options()
        P = oracle.scale_problem(lp, o)
        x = lp.x_opt / P.dc
        y = lp.y_opt / P.dr
        k = oracle.kkt(P, x, y, P.A @ x, P.At @ y)
        assert k["rel_pres"] < 1e-12 and k["rel_dres"] < 1e-12 and k["rel_gap"] < 1e-12
        # a perturbed point is not optimal
        k2 = oracle.kkt(P, x * 1.01, y, P.A @ (x * 1.01), P.At @ y)
        assert max(k2["rel_pres"], k2["rel_gap"]) > 1e-6


def test_lagrangian_at_constructed_optimum_is_the_objective():
    """Complementary slackness makes y*^T (b - A x*) = 0 at a primal-dual
    optimum, so L(x*, y*) of Eq. (2) equals c^T x* -- in the scaled space as
    in the caller's; plus one value worked by hand."""
    for lp in (lpgen.tiny_random(3), lpgen.mixed_small(2)):
        P = oracle.scale_problem(lp, oracle.Options())
        x, y = lp.x_opt / P.dc, lp.y_opt / P.dr
        assert oracle.pdhg.lagrangian(P, x, y) == pytest.approx(lp.obj_opt, rel=1e-12)
    # A = [1 1], b = 4, c = (1, -1), x = (1, 2), y = 3: (1 - 2) - 3 * 3 + 4 * 3 = 2
    P = _scaled_from_dense([[1.0, 1.0]], [4.0], [1.0, -1.0], [0.0, 0.0], [10.0, 10.0], "E")
    assert oracle.pdhg.lagrangian(P, arr([1.0, 2.0]), arr([3.0])) == 2.0


def test_initial_state_special_cases():
    """x_0 is the point of the box nearest 0, y_0 = 0, T_0 = Sigma_0 = I
    (Section 3.2); eta_0 ||A~||_2 = 0.9 in plain mode with the norm from an
    SVD; hand values of eta_0 and omega_0 in pdlp mode; omega_0 = 1 for b = 0."""
    A = [[3.0, 4.0, 0.0], [0.0, 0.0, 1.0]]  # singular values 5 and 1; largest |a_ij| 4
    P = _scaled_from_dense(A, [1.0, 2.0], [1.0, 1.0, 1.0], [-1.0, 2.0, -np.inf], [1.0, 5.0, -3.0], "EE")
    S = oracle.initial_state(P, oracle.Options(mode="plain"))
    np.testing.assert_array_equal(S.x, [0.0, 2.0, -3.0])
    assert np.all(S.y == 0) and np.all(S.T == 1) and np.all(S.Sigma == 1)
    assert S.eta * np.linalg.svd(np.array(A), compute_uv=False)[0] == pytest.approx(0.9, rel=1e-12)
    Sp = oracle.initial_state(P, oracle.Options(mode="pdlp"))
    assert Sp.eta == 0.25 and Sp.omega == pytest.approx(math.sqrt(3.0 / 5.0), rel=1e-15)
    P0 = _scaled_from_dense(A, [0.0, 0.0], [1.0, 1.0, 1.0], [0.0] * 3, [1.0] * 3, "EE")
    assert oracle.initial_state(P0, oracle.Options(mode="pdlp")).omega == 1.0


def test_dual_projection_and_mask_per_sense():
    """Sign cone per row sense (reading R3): equality rows free, >= rows
    y >= 0, <= rows y <= 0; the mask is membership, inclusive at 0."""
    P = _scaled_from_dense(np.ones((9, 1)), [0.0] * 9, [0.0], [0.0], [1.0], "EEEGGGLLL")
    yh = arr([-2.0, 0.0, 3.0] * 3)
    np.testing.assert_array_equal(oracle.pdhg.project_dual(P, yh), [-2, 0, 3, 0, 0, 3, -2, 0, 0])
    np.testing.assert_array_equal(oracle.pdhg.dual_feasible_mask(P, yh),
                                  [True, True, True, False, True, True, True, True, False])


# ---------------------------------------------------------------------------
# Restart decisions worked by hand (the restart reading: KKT-based restarts
# with sufficient decay 0.2, necessary decay 0.8 without progress, and an
# artificial restart once the period holds 0.36 of all attempts)
# ---------------------------------------------------------------------------
# LP: min x  s.t.  x = 1, x >= 0 (no scaling).  At (x, y) = (2, 0.5): primal
# residual 1, reduced cost 0.5 absorbed by the bound (dual residual 0),
# pobj 2, dobj 0.5, gap 1.5, so K_1 = sqrt(1 + 2.25) = sqrt(3.25).  At the
# average (1.5, 0.75): residual 0.5, gap 0.75, K_1 = sqrt(0.8125).

def _restart_state(x_last=(0.0,), k_last_parts=(36.0, 0.0, 144.0), k_prev=100.0, last=90, with_avg=False):
    S = State(x=arr([2.0]), y=arr([0.5]), ax=arr([2.0]), T=np.ones(1), Sigma=np.ones(1), GT=np.zeros(1),
              GS=np.zeros(1), GT_norm=0.0, GS_norm=0.0, eta=0.5, omega=1.0, attempts=100,
              xbar=arr([1.5]) if with_avg else np.zeros(1), ybar=arr([0.75]) if with_avg else np.zeros(1),
              wsum=1.0 if with_avg else 0.0)
    S.x_last = None if x_last is None else arr(list(x_last))
    S.y_last = None if x_last is None else np.zeros(1)
    S.K_last_parts, S.K_prev, S.last_restart_attempt = k_last_parts, k_prev, last
    return S


_P1 = _scaled_from_dense([[1.0]], [1.0], [1.0], [0.0], [np.inf], "E")


@pytest.mark.parametrize("case,parts,k_prev,last,restart", [
    ("sufficient decay", (36.0, 0.0, 144.0), 100.0, 90, True),   # K / K_last = sqrt(3.25 / 180) < 0.2
    ("decay without progress", (4.0, 0.0, 4.0), 1.0, 90, True),  # ratio sqrt(3.25 / 8) ~ 0.64 <= 0.8, K > K_prev
    ("decay with progress", (4.0, 0.0, 4.0), 5.0, 90, False),    # same ratio, K < K_prev
    ("long period", (1.0, 0.0, 2.25), 1.0, 60, True),            # ratio 1, 40 of 100 attempts >= 0.36
    ("short period", (1.0, 0.0, 2.25), 1.0, 70, False),          # ratio 1, 30 of 100 attempts
])
def test_restart_decisions_by_hand(case, parts, k_prev, last, restart):
    S = _restart_state(k_last_parts=parts, k_prev=k_prev, last=last)
    oracle.pdhg.check(_P1, S, oracle.Options(mode="pdlp"), tol=1e-9)
    assert S.status is None
    assert S.restarts == (1 if restart else 0), case
    assert S.K_prev == pytest.approx(math.sqrt(3.25), rel=1e-15)
    if restart:
        # restart point (2, 0.5) from (0, 0): omega <- sqrt(omega ||dy|| / ||dx||) = sqrt(0.5 / 2)
        np.testing.assert_array_equal(S.x_last, [2.0])
        assert S.omega == pytest.approx(0.5, rel=1e-15)
        assert S.last_restart_attempt == 100 and S.wsum == 0.0
        assert S.K_last_parts == pytest.approx((1.0, 0.0, 2.25), rel=1e-15)
    else:
        assert S.omega == 1.0 and S.last_restart_attempt == last


def test_restart_to_the_better_average_by_hand():
    S = _restart_state(with_avg=True)
    oracle.pdhg.check(_P1, S, oracle.Options(mode="pdlp"), tol=1e-9)
    assert S.restarts == 1
    np.testing.assert_array_equal(S.x, [1.5])
    np.testing.assert_array_equal(S.y, [0.75])
    assert S.K_prev == pytest.approx(math.sqrt(0.8125), rel=1e-15)
    assert S.omega == pytest.approx(math.sqrt(0.5), rel=1e-15)  # ||dy|| / ||dx|| = 0.75 / 1.5


def test_first_check_records_the_reference_and_restarts_can_be_off():
    S = _restart_state(x_last=None)
    oracle.pdhg.check(_P1, S, oracle.Options(mode="pdlp"), tol=1e-9)
    assert S.restarts == 0 and S.last_restart_attempt == 100
    np.testing.assert_array_equal(S.x_last, [2.0])
    S = _restart_state()
    oracle.pdhg.check(_P1, S, oracle.Options(mode="pdlp", restart=False), tol=1e-9)
    assert S.restarts == 0


# ---------------------------------------------------------------------------
# Online gradients: finite differences of the losses of Eq. (5)
# ---------------------------------------------------------------------------

def _random_state(P, rng):
    m, n = P.A.shape
    lo = np.where(np.isfinite(P.l), P.l, -5.0)
    hi = np.where(np.isfinite(P.u), P.u, 5.0)
    x = lo + (hi - lo) * rng.random(n)
    y = oracle.pdhg.project_dual(P, rng.standard_normal(m))
    return x, y


def test_online_gradients_match_finite_differences():
    rng = np.random.default_rng(7)
    lp = lpgen.mixed_small(5, m=20, n=40)
    P = oracle.scale_problem(lp, oracle.Options())
    x, y = _random_state(P, rng)
    ax = P.A @ x
    T = 0.5 + rng.random(P.A.shape[1])
    Sig = 0.5 + rng.random(P.A.shape[0])
    eta, omega = 0.7, 1.3

    def x_next(Tv):
        return oracle.primal_half_step(P, x, y, Tv, eta, omega)[0]

    def y_next(Sv, xn):
        return oracle.dual_half_step(P, xn, y, ax, Sv, eta, omega)[0]

    x1, g, xh = oracle.primal_half_step(P, x, y, T, eta, omega)
    y1, ax1, r, yh = oracle.dual_half_step(P, x1, y, ax, Sig, eta, omega)
    gT, gS = oracle.online_gradients(P, g, xh, ax, r, yh, eta, omega, normalize=False)
    gTn, gSn = oracle.online_gradients(P, g, xh, ax, r, yh, eta, omega, normalize=True)
    L0 = oracle.lagrangian(P, x, y)
    h = 1e-6
    checked_p = checked_d = 0
    for j in range(P.A.shape[1]):
        # skip coordinates within h of a projection kink
        step = (eta / omega) * g[j]
        if np.isfinite(P.l[j]) and abs(xh[j] - P.l[j]) < 2 * h * abs(step) + 1e-9:
            continue
        if np.isfinite(P.u[j]) and abs(xh[j] - P.u[j]) < 2 * h * abs(step) + 1e-9:
            continue
        Tp = T.copy(); Tp[j] += h
        Tm = T.copy(); Tm[j] -= h
        lp_ = oracle.lagrangian(P, x_next(Tp), y) - L0
        lm_ = oracle.lagrangian(P, x_next(Tm), y) - L0
        fd = (lp_ - lm_) / (2 * h)
        assert fd == pytest.approx(gT[j], rel=1e-5, abs=1e-8)
        checked_p += 1
    for i in range(P.A.shape[0]):
        step = eta * omega * r[i]
        if P.sense[i] != ord("E") and abs(yh[i]) < 2 * h * abs(step) + 1e-9:
            continue
        Sp = Sig.copy(); Sp[i] += h
        Sm = Sig.copy(); Sm[i] -= h
        # l^d(Sigma) = L(x^k, y^k) - L(x^k, y^{k+1}(Sigma))
        lp_ = L0 - oracle.lagrangian(P, x, y_next(Sp, x1))
        lm_ = L0 - oracle.lagrangian(P, x, y_next(Sm, x1))
        fd = (lp_ - lm_) / (2 * h)
        assert fd == pytest.approx(gS[i], rel=1e-5, abs=1e-8)
        checked_d += 1
    assert checked_p > 20 and checked_d > 10
    np.testing.assert_allclose(gTn, gT / float(g @ g), rtol=1e-14)
    res = P.b - ax
    np.testing.assert_allclose(gSn, gS / float(res @ res), rtol=1e-14)


# ---------------------------------------------------------------------------
# Invariants of the preconditioner update
# ---------------------------------------------------------------------------

def test_alpha_zero_is_vanilla_bitwise():
    """A zero learning rate reproduces the run without any update, bit for bit."""
    lp = lpgen.mixed_small(3)
    for mode in ("pdlp", "plain"):
        runs = []
        for phi in (1, 0):
            trace = []
            o = oracle.Options(mode=mode, alpha=0.0, phi=phi, normalize=True)
            oracle.solve(lp, o, tol=1e-12, iter_limit=300,
                         trace=lambda P, S: trace.append((S.x.copy(), S.y.copy(), S.T.copy(), S.Sigma.copy(), S.eta)))
            runs.append(trace)
        for a, b in zip(*runs):
            for u, v in zip(a[:4], b[:4]):
                assert np.array_equal(u, v)
            assert a[4] == b[4]
            assert np.all(a[2] == 1.0) and np.all(a[3] == 1.0)


@pytest.mark.parametrize("scheduler", ["adagrad", "adagrad_norm", "const"])
def test_T_monotone_and_sigma_floor(scheduler):
    lp = lpgen.mixed_small(4)
    prev = {}
    floor = 1e-6
    seen_floor = [False]

    def tr(P, S):
        if "T" in prev:
            assert np.all(S.T >= prev["T"])
        assert np.all(S.Sigma >= floor) and np.all(S.T >= floor)
        if np.any(S.Sigma == floor):
            seen_floor[0] = True
        prev["T"] = S.T.copy()

    alpha = 0.5 if scheduler == "const" else 5.0
    o = oracle.Options(alpha=alpha, phi=1, scheduler=scheduler, normalize=True)
    oracle.solve(lp, o, tol=1e-12, iter_limit=400, trace=tr)
    assert np.all(np.isfinite(prev["T"]))
    if scheduler != "const":
        assert seen_floor[0], "a large learning rate should drive some Sigma_i to the floor"


def test_step_limit_lower_bound():
    """eta_max >= 1 / ||Sigma^1/2 A T^1/2||_2 for any (dx, dy): Cauchy-Schwarz
    plus the AM-GM inequality, for every positive T, Sigma and omega."""
    rng = np.random.default_rng(11)
    A = sp.random(30, 50, density=0.2, random_state=3, format="csr")
    for _ in range(200):
        T = np.exp(rng.normal(size=50))
        Sig = np.exp(rng.normal(size=30))
        omega = float(np.exp(rng.normal()))
        dx = rng.normal(size=50)
        dy = rng.normal(size=30)
        lim = oracle.step_size_limit(dx, dy, A @ dx, T, Sig, omega)
        M = np.diag(np.sqrt(Sig)) @ A.toarray() @ np.diag(np.sqrt(T))
        assert lim * np.linalg.norm(M, 2) >= 1.0 - 1e-12


# ---------------------------------------------------------------------------
# Preprocessing
# ---------------------------------------------------------------------------

def test_ruiz_equilibrates_infinity_norms():
    rng = np.random.default_rng(0)
    A = sp.random(80, 120, density=0.1, random_state=1, format="csr")
    A.data = 10.0 ** rng.uniform(-3, 3, size=A.nnz) * np.sign(rng.normal(size=A.nnz))
    keep_r = np.diff(A.indptr) > 0
    keep_c = np.bincount(A.indices, minlength=120) > 0
    As, dr, dc = oracle.ruiz_equilibrate(A, 40)
    rmax = abs(As).max(axis=1).toarray().ravel()
    cmax = abs(As).max(axis=0).toarray().ravel()
    np.testing.assert_allclose(rmax[keep_r], 1.0, atol=1e-6)
    np.testing.assert_allclose(cmax[keep_c], 1.0, atol=1e-6)
    np.testing.assert_allclose(As.toarray(), np.diag(dr) @ A.toarray() @ np.diag(dc), rtol=1e-12, atol=0)


def test_pock_chambolle_norm_at_most_one():
    rng = np.random.default_rng(1)
    for s in range(5):
        A = sp.random(40, 60, density=0.15, random_state=s, format="csr")
        A.data = rng.normal(size=A.nnz)
        As, fr, fc = oracle.pock_chambolle_rescale(A, 1.0)
        assert np.linalg.norm(As.toarray(), 2) <= 1.0 + 1e-12
        np.testing.assert_allclose(As.toarray(), np.diag(fr) @ A.toarray() @ np.diag(fc), rtol=1e-13)


def test_l2_rescale_closed_forms():
    # a diagonal matrix becomes the identity up to sign
    d = np.array([4.0, -9.0, 0.25])
    As, fr, fc = oracle.l2_norm_rescale(sp.csr_matrix(np.diag(d)))
    np.testing.assert_allclose(As.toarray(), np.diag(np.sign(d)), rtol=1e-15)
    # a rank-one positive matrix u v^T maps to sqrt(u_i v_j) / sqrt(||u|| ||v||)
    u = np.array([1.0, 2.0, 3.0]); v = np.array([4.0, 1.0])
    As, _, _ = oracle.l2_norm_rescale(sp.csr_matrix(np.outer(u, v)))
    expect = np.sqrt(np.outer(u, v)) / math.sqrt(np.linalg.norm(u) * np.linalg.norm(v))
    np.testing.assert_allclose(As.toarray(), expect, rtol=1e-14)


def test_power_iteration_matches_svd():
    rng = np.random.default_rng(2)
    A = sp.random(50, 70, density=0.2, random_state=4, format="csr")
    A.data = rng.normal(size=A.nnz)
    est = oracle.power_spectral_norm(A, 200)
    assert est == pytest.approx(np.linalg.norm(A.toarray(), 2), rel=1e-8)


def _cycle_differences(n, seed=0):
    """Rows w_i (x_i - x_{i+1 mod n}) with weights w_i ~ U(0.5, 2): every row
    sums to zero, so the all-ones direction is in the null space."""
    w = np.random.default_rng(seed).uniform(0.5, 2.0, size=n)
    rows = np.repeat(np.arange(n), 2)
    cols = np.stack([np.arange(n), (np.arange(n) + 1) % n], axis=1).ravel()
    vals = np.stack([w, -w], axis=1).ravel()
    return sp.csr_matrix((vals, (rows, cols)), shape=(n, n))


def test_splitmix_signs_follow_the_published_generator():
    g = load_golden("splitmix64.json")
    want = [-1.0 if int(h, 16) >> 63 else 1.0 for h in g["outputs"]]
    np.testing.assert_array_equal(oracle.pdhg.splitmix_signs(len(want)), want)


def test_power_iteration_restarts_when_rows_sum_to_zero():
    A = _cycle_differences(40)
    assert np.all(np.asarray(A.sum(axis=1)).ravel() == 0.0)
    assert np.all(A @ np.ones(40) == 0.0)
    est = oracle.power_spectral_norm(A, 200)
    assert est == pytest.approx(np.linalg.norm(A.toarray(), 2), rel=1e-8)


def test_scaling_preserves_the_optimum():
    """The rescaled LP (mapped back) has the same optimum: HiGHS on both."""
    lp = lpgen.mixed_small(6, m=25, n=50)
    for mode in ("pdlp", "plain"):
        P = oracle.scale_problem(lp, oracle.Options(mode=mode))
        scaled = lpgen.LP(
            m=lp.m, n=lp.n, row_ptr=P.A.indptr.astype(np.int64), col_idx=P.A.indices.astype(np.int32),
            val=P.A.data, b=P.b, c=P.c, lb=P.l, ub=P.u, sense=lp.sense)
        assert _highs(scaled) == pytest.approx(_highs(lp), rel=1e-9, abs=1e-9)


# ---------------------------------------------------------------------------
# Converged solutions: brute force, constructed optimum, HiGHS
# ---------------------------------------------------------------------------

def test_vertex_enumeration_agrees_with_highs():
    rng = np.random.default_rng(5)
    for trial in range(10):
        m, n = int(rng.integers(1, 4)), int(rng.integers(2, 6))
        lp = _tiny_box_lp(rng, m, n)
        v, _ = oracle.enumerate_vertices(lp.csr().toarray(), lp.b, lp.c, lp.lb, lp.ub, lp.sense)
        assert v == pytest.approx(_highs(lp), rel=1e-9, abs=1e-9)


def _tiny_box_lp(rng, m, n):
    """A tiny feasible LP with finite boxes and random senses (feasible at a random point)."""
    A = rng.normal(size=(m, n))
    x0 = rng.uniform(0, 3, size=n)
    senses = rng.choice([ord("E"), ord("L"), ord("G")], size=m).astype(np.uint8)
    b = A @ x0 + np.where(senses == ord("L"), 0.5, np.where(senses == ord("G"), -0.5, 0.0))
    Asp = sp.csr_matrix(A)
    return lpgen.LP(m=m, n=n, row_ptr=Asp.indptr.astype(np.int64), col_idx=Asp.indices.astype(np.int32),
                    val=Asp.data.astype(float), b=b, c=rng.normal(size=n), lb=np.zeros(n),
                    ub=np.full(n, 3.0), sense=senses)


@pytest.mark.parametrize("mode", ["pdlp", "plain"])
def test_oracle_reaches_vertex_optimum(mode):
    rng = np.random.default_rng(9)
    for trial in range(8):
        m, n = int(rng.integers(1, 5)), int(rng.integers(2, 7))
        lp = _tiny_box_lp(rng, m, n)
        v, _ = oracle.enumerate_vertices(lp.csr().toarray(), lp.b, lp.c, lp.lb, lp.ub, lp.sense)
        res, _, _ = oracle.solve(lp, oracle.Options(mode=mode, alpha=1e-2, phi=1), tol=1e-9, iter_limit=400_000)
        assert res.status == oracle.pdhg.OPTIMAL
        assert res.pobj == pytest.approx(v, rel=1e-6, abs=1e-6)


def test_golden_two_variable_lp():
    g = load_golden("lp_2var.json")
    Asp = sp.csr_matrix(np.array(g["A"]))
    lp = lpgen.LP(m=2, n=2, row_ptr=Asp.indptr.astype(np.int64), col_idx=Asp.indices.astype(np.int32),
                  val=Asp.data, b=arr(g["b"]), c=arr(g["c"]), lb=arr(g["l"]), ub=arr(g["u"]),
                  sense=np.array([SENSE[s] for s in g["sense"]], dtype=np.uint8))
    for mode in ("pdlp", "plain"):
        res, _, _ = oracle.solve(lp, oracle.Options(mode=mode, alpha=1e-2, phi=1), tol=1e-10, iter_limit=200_000)
        assert res.status == oracle.pdhg.OPTIMAL
        assert res.pobj == pytest.approx(g["obj_opt"], rel=1e-8)
        np.testing.assert_allclose(res.x, g["x_opt"], atol=1e-7)
        np.testing.assert_allclose(res.y, g["y_opt"], atol=1e-7)


@pytest.mark.parametrize("mode,alpha,phi", [("plain", 0.0, 1), ("plain", 1e-2, 1), ("pdlp", 0.0, 20), ("pdlp", 1e-3, 20)])
def test_tiny_random_reaches_constructed_optimum(mode, alpha, phi):
    lp = lpgen.tiny_random(0)
    res, _, _ = oracle.solve(lp, oracle.Options(mode=mode, alpha=alpha, phi=phi), tol=1e-8, iter_limit=200_000)
    assert res.status == oracle.pdhg.OPTIMAL
    assert res.pobj == pytest.approx(lp.obj_opt, rel=1e-7)
    assert res.dobj == pytest.approx(lp.obj_opt, rel=1e-7)


def test_mixed_senses_and_bounds_match_highs():
    for seed in range(3):
        lp = lpgen.mixed_small(seed)
        ref = _highs(lp)
        assert ref == pytest.approx(lp.obj_opt, rel=1e-7, abs=1e-7)
        res, _, _ = oracle.solve(lp, oracle.Options(alpha=1e-3), tol=1e-8, iter_limit=200_000)
        assert res.status == oracle.pdhg.OPTIMAL
        assert res.pobj == pytest.approx(ref, rel=1e-6, abs=1e-6)


def test_small_transport_matches_highs():
    lp = lpgen.transport(1, n_supply=150, n_demand=150, n_arcs=1500)
    ref = _highs(lp)
    res, _, _ = oracle.solve(lp, oracle.Options(alpha=1e-4), tol=1e-8, iter_limit=200_000)
    assert res.status == oracle.pdhg.OPTIMAL
    assert res.pobj == pytest.approx(ref, rel=1e-6)
    # strong duality at the returned point
    assert res.dobj == pytest.approx(ref, rel=1e-6)


# ---------------------------------------------------------------------------
# Step-size rule, average weights, update points and the other schedulers
# (tests/golden/step_rules_1x1.json, worked by hand)
# ---------------------------------------------------------------------------

def _rules_problem(g):
    L = g["lp"]
    return _scaled_from_dense(L["A"], L["b"], L["c"], arr(L["l"]), arr(L["u"]), L["sense"])


def _rules_state(eta, attempts=0, k=0):
    return State(x=np.zeros(1), y=np.zeros(1), ax=np.zeros(1), T=np.ones(1), Sigma=np.ones(1),
                 GT=np.zeros(1), GS=np.zeros(1), GT_norm=0.0, GS_norm=0.0, eta=eta, omega=1.0,
                 xbar=np.zeros(1), ybar=np.zeros(1), k=k, attempts=attempts)


@pytest.mark.parametrize("case", ["accept_then_grow", "reject_then_shrink"])
def test_golden_next_step_size_and_average_weights(case):
    """Two pdlp attempts from a hand-worked state at attempt 1023, where the
    step-size factors are exactly 7/8 and 65/64: the accept test, the next
    step size (either term of the min), and the averages weighted by the
    step size each accepted attempt used."""
    g = load_golden("step_rules_1x1.json")
    e = g[case]
    P = _rules_problem(g)
    S = _rules_state(e["eta"], attempts=e["attempts_before"])
    o = oracle.Options(mode="pdlp", alpha=0.0, phi=0)
    for key in ("step1", "step2"):
        s = e[key]
        x0, y0, ax0 = S.x.copy(), S.y.copy(), S.ax.copy()
        eta_used = S.eta
        acc = oracle.attempt(P, S, o)
        assert acc == s["accepted"]
        np.testing.assert_allclose(S.x, s["x"], rtol=0, atol=1e-15)
        np.testing.assert_allclose(S.y, s["y"], rtol=0, atol=1e-15)
        np.testing.assert_allclose(S.xbar, s["xbar"], rtol=1e-15, atol=0)
        np.testing.assert_allclose(S.ybar, s["ybar"], rtol=1e-15, atol=0)
        assert S.wsum == pytest.approx(s["wsum"], rel=1e-15, abs=0)
        # the limit of this attempt, from the same point and step
        x1, _, _ = oracle.primal_half_step(P, x0, y0, np.ones(1), eta_used, 1.0)
        y1, ax1, _, _ = oracle.dual_half_step(P, x1, y0, ax0, np.ones(1), eta_used, 1.0)
        lim = oracle.step_size_limit(x1 - x0, y1 - y0, ax1 - ax0, np.ones(1), np.ones(1), 1.0)
        assert lim == pytest.approx(s["eta_max"], rel=1e-15)
        if "eta_next" in s:
            assert S.eta == pytest.approx(s["eta_next"], rel=1e-15, abs=0)
        if not acc:
            assert S.k == 0 and S.attempts == e["attempts_before"] + 1


def test_golden_update_points_count_accepted_steps():
    """The online update fires on accepted attempts whose count of earlier
    accepted steps is 0, phi, 2 phi, ... (Algorithm 1, reading R7), with a
    rejected attempt in between."""
    g = load_golden("step_rules_1x1.json")
    e = g["update_points"]
    P = _rules_problem(g)
    S = _rules_state(e["eta"])
    o = oracle.Options(mode="pdlp", alpha=e["alpha"], phi=e["phi"], normalize=False, scheduler="const")
    forced = {int(k): v for k, v in e["eta_forced"].items()}
    for i, (acc_e, k_e, move_e) in enumerate(zip(e["accepted"], e["k_after"], e["preconditioner_moves"])):
        S.eta = forced.get(i, e["eta"])
        T0, S0 = S.T.copy(), S.Sigma.copy()
        acc = oracle.attempt(P, S, o)
        assert acc == acc_e, i
        assert S.k == k_e, i
        moved = bool(np.any(S.T != T0) or np.any(S.Sigma != S0))
        assert moved == move_e, i


def test_update_points_follow_accepted_steps_across_restarts():
    """Over a restarted pdlp solve, the preconditioners move exactly on the
    accepted attempts whose number of earlier accepted attempts (counted here,
    not read from the oracle's k) is a multiple of phi: k is not reset by a
    restart and rejected attempts do not count (reading R7)."""
    lp = lpgen.tiny_random(3, m=30, n=70, col_nnz=4)
    phi = 3
    o = oracle.Options(mode="pdlp", alpha=1e-2, phi=phi, normalize=True, check_every=8)
    P = oracle.scale_problem(lp, o)
    S = oracle.initial_state(P, o)
    oracle.check(P, S, o, 0.0)
    S.checked0 = True
    accepted = rejected = 0
    restarts_seen = 0
    for i in range(400):
        if i % 37 == 36:
            S.eta *= 50.0  # far beyond the step limit: a rejected attempt
        T0, S0 = S.T.copy(), S.Sigma.copy()
        before = accepted
        acc = oracle.attempt(P, S, o)
        moved = bool(np.any(S.T != T0) or np.any(S.Sigma != S0))
        expect = acc and before % phi == 0
        assert moved == expect, (S.attempts, acc, before)
        accepted += acc
        rejected += not acc
        if S.attempts % o.check_every == 0:
            r0 = S.restarts
            oracle.check(P, S, o, 0.0)
            restarts_seen += S.restarts - r0
    assert restarts_seen >= 2 and rejected >= 5


def test_golden_scheduler_steps():
    """One step of each learning-rate rule worked by hand (reading R6):
    scalar AdaGrad over the whole gradient and a constant rate, each followed
    by the floor."""
    g = load_golden("step_rules_1x1.json")["schedulers"]
    for s in g["adagrad_norm"]:
        o = oracle.Options(alpha=s["alpha"], scheduler="adagrad_norm", precond_floor=1e-6)
        P, G, Gn = oracle.ogd_update(arr(s["P"]), np.zeros(len(s["P"])), s["G"], arr(s["grad"]), o)
        np.testing.assert_allclose(P, s["P_after"], rtol=1e-15, atol=0)
        assert Gn == s["G_after"]
    for s in g["const"]:
        o = oracle.Options(alpha=s["alpha"], scheduler="const", precond_floor=1e-6)
        P, _, _ = oracle.ogd_update(arr(s["P"]), np.zeros(len(s["P"])), 0.0, arr(s["grad"]), o)
        np.testing.assert_allclose(P, s["P_after"], rtol=1e-15, atol=0)
