"""GPU parity: the CUDA library (through the C ABI) against the CPU oracle.

Floating point is FP64 on both sides.  The bars:

* One step from an identical state (the oracle's state after attempt k-1 is
  loaded into the library, one attempt -- and the check when k is a multiple
  of 64 -- runs on each side): every vector of the state within 1e-12
  relative, the step scalars within 1e-10, counters identical.  This pins the
  arithmetic of each of the first 100 attempts, including restarts.
* Free-running trajectories: iterates and preconditioners within 1e-10
  relative for all of the first 100 attempts in plain mode, and for the first
  60 attempts in pdlp mode.  The adaptive step size makes pdlp mode sensitive
  to rounding: in the oracle itself a 1e-15 relative perturbation at attempt
  10 grows to 1e-12..1e-10 by attempt 63 and to 1e-10..3e-8 by attempt 100
  (measured on these cases), so two correct FP64 implementations that sum in
  different orders agree to 1e-10 only over that horizon.
* Step scalars of the free-running runs (eta, omega, average weight): 1e-8
  relative; they come from step differences (eta_max = ||dz||^2 /
  (2 |dy^T A dx|)) whose relative rounding error exceeds the iterates' by
  about ||z|| / ||dz||.
* Full solves: same status; iteration count at 1e-4 within +-2% (the
  full-size transport LP: one check period) of the range the oracle itself
  spans under 1e-15 relative perturbations of c (the count is
  rounding-sensitive in pdlp mode; where that range is one value this is
  plain +-2%); final
  objective within 1e-6 relative when both sides solve to 1e-8 (at 1e-4 the
  objective itself is only determined to about the tolerance).
"""
import copy
import math

import numpy as np
import pytest

import lpgen
import oracle
import paper_2506_17650_gb300 as lpop
from paper_2506_17650_gb300 import build as lpbuild

pytestmark = pytest.mark.gpu

SCHED = {"adagrad": lpop.LP_SCHED_ADAGRAD, "adagrad_norm": lpop.LP_SCHED_ADAGRAD_NORM, "const": lpop.LP_SCHED_CONST}
MODE = {"plain": lpop.LP_MODE_PLAIN, "pdlp": lpop.LP_MODE_PDLP}

REL = 1e-10
REL_SCALAR = 1e-8


@pytest.fixture(scope="module", autouse=True)
def _built():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lpbuild.build()
    lpop.load_library()


def gpu_options(o: oracle.Options, **extra):
    return dict(mode=MODE[o.mode], scheduler=SCHED[o.scheduler], alpha=o.alpha, phi=o.phi,
                normalize=int(o.normalize), precond_floor=o.precond_floor, ruiz_iters=o.ruiz_iters,
                pc_beta=o.pc_beta, check_every=o.check_every, restart=int(o.restart), power_iters=o.power_iters,
                plain_step_factor=o.plain_step_factor, **extra)


def close(a, b, rel=REL):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    err = float(np.linalg.norm(a - b))
    return err <= rel * float(np.linalg.norm(b)) + 1e-14 * math.sqrt(max(b.size, 1)), err


def oracle_trace(lp, o, attempts, tol=0.0):
    """Oracle states (scaled space) after each attempt in ``attempts``."""
    want = set(attempts)
    rec = {}

    def tr(P, S):
        if S.attempts in want:
            rec[S.attempts] = dict(x=S.x.copy(), y=S.y.copy(), T=S.T.copy(), Sigma=S.Sigma.copy(), eta=S.eta,
                                   omega=S.omega, k=S.k, restarts=S.restarts, wsum=S.wsum)

    res, P, S = oracle.solve(lp, o, tol=tol, iter_limit=max(attempts), trace=tr)
    return rec, P, S


def compare_state(g, r, where):
    for key in ("x", "y", "T", "Sigma"):
        ok, err = close(g[key], r[key])
        assert ok, f"{where}: {key} differs by {err:.3e} (norm {np.linalg.norm(r[key]):.3e})"
    for key in ("eta", "omega", "wsum"):
        ok, err = close([g[key]], [r[key]], REL_SCALAR)
        assert ok, f"{where}: {key} gpu {g[key]!r} oracle {r[key]!r}"
    assert g["k"] == r["k"], f"{where}: accepted steps {g['k']} vs {r['k']}"
    assert g["restarts"] == r["restarts"], f"{where}: restarts {g['restarts']} vs {r['restarts']}"


CASES = {
    "tiny_plain_norm_freq": (lambda: lpgen.tiny_random(0), oracle.Options(mode="plain", alpha=1e-2, phi=1)),
    "tiny_pdlp_freq": (lambda: lpgen.tiny_random(1), oracle.Options(mode="pdlp", alpha=1e-3, phi=1)),
    "mixed_pdlp_adagrad": (lambda: lpgen.mixed_small(0), oracle.Options(alpha=1e-2, phi=1)),
    "mixed_pdlp_adagrad_norm": (lambda: lpgen.mixed_small(1),
                                oracle.Options(alpha=1e-1, phi=3, scheduler="adagrad_norm", normalize=False)),
    "mixed_plain_const": (lambda: lpgen.mixed_small(2), oracle.Options(mode="plain", alpha=1e-3, phi=2,
                                                                       scheduler="const")),
    "rowmix_pdlp": (lambda: lpgen.row_length_mix(0), oracle.Options(alpha=1e-3, phi=20)),
    "transport_small_pdlp": (lambda: lpgen.transport(0, 1500, 1500, 12000), oracle.Options(alpha=1e-4, phi=20)),
    "alpha0_pdlp": (lambda: lpgen.mixed_small(3), oracle.Options(alpha=0.0, phi=1)),
    # rows of A and of A^T longer than a segment (4096 entries here): reduced by several blocks
    "long_rows_pdlp": (lambda: lpgen.long_rows(0), oracle.Options(alpha=1e-3, phi=1)),
    # the large power-law LP's recipe at 1% of its size (m 20k, n 50k, ~300k nonzeros): column
    # degrees up to 20k (segmented rows of A^T), |a| over six decades, free and boxed variables,
    # = and <= rows; the bench's online-preconditioning settings
    "powerlaw_small_pdlp": (lambda: lpgen.powerlaw(0, 20_000, 50_000, 300_000), oracle.Options(alpha=1e-6, phi=20)),
    # the same recipe at 0.05% (m 1000, n 2500, ~13k nonzeros): small enough to solve to 1e-4
    "powerlaw_tiny_pdlp": (lambda: lpgen.powerlaw(0, 1_000, 2_500, 15_000), oracle.Options(alpha=1e-6, phi=20)),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_scaling_matches_oracle(case):
    make, o = CASES[case]
    lp = make()
    P = oracle.scale_problem(lp, o)
    S0 = oracle.initial_state(P, o)
    with lpop.Problem(lp, **gpu_options(o)) as p:
        dr, dc, sc = p.scaling()
    assert close(dr, P.dr, 1e-13)[0] and close(dc, P.dc, 1e-13)[0]
    assert sc["eta0"] == pytest.approx(S0.eta, rel=1e-12)
    assert sc["omega0"] == pytest.approx(S0.omega, rel=1e-12)


def oracle_steps(lp, o, count):
    """Oracle states before the first attempt (after the initial check) and after each of ``count`` attempts."""
    P = oracle.scale_problem(lp, o)
    S = oracle.initial_state(P, o)
    oracle.check(P, S, o, 0.0)
    S.checked0 = True
    states = [copy.deepcopy(S)]
    for _ in range(count):
        oracle.attempt(P, S, o)
        if S.attempts % o.check_every == 0:
            oracle.check(P, S, o, 0.0)
        states.append(copy.deepcopy(S))
    return P, states


def to_lib_state(S):
    n, m = S.x.size, S.y.size
    refs = S.x_last is not None
    return dict(
        x=S.x, xbar=S.xbar, T=S.T, GT=S.GT, x_last=S.x_last if refs else np.zeros(n),
        y=S.y, ybar=S.ybar, ax=S.ax, Sigma=S.Sigma, GS=S.GS, y_last=S.y_last if refs else np.zeros(m),
        eta=S.eta, omega=S.omega, wsum=S.wsum, gp_norm=S.GT_norm, gd_norm=S.GS_norm,
        klast_p2=S.K_last_parts[0], klast_d2=S.K_last_parts[1], klast_g2=S.K_last_parts[2],
        k_prev=S.K_prev, k=S.k, attempts=S.attempts, last_restart_attempt=S.last_restart_attempt,
        restarts=S.restarts, refs_set=int(refs), initial_check_done=int(S.checked0))


def compare_full_state(g, S, where, rel_vec=1e-12, rel_scal=1e-10, prev=None):
    """Compare the library's state after one step with the oracle's.

    The next step size comes from eta_max = ||dz||^2 / (2 |dy^T A dx|), formed
    from the step dz itself, so its relative rounding error is about
    eps ||z|| / ||dz||: it is compared at max(1e-10, 1e-13 ||z|| / ||dz||)
    (1e-13 ~ 500 eps covers the sums), and skipped when the step is at
    rounding level (||dz|| < 1e-9 ||z||)."""
    r = to_lib_state(S)
    keys = ["x", "xbar", "T", "GT", "y", "ybar", "ax", "Sigma", "GS"]
    if r["refs_set"]:
        keys += ["x_last", "y_last"]
    for key in keys:
        ok, err = close(g[key], r[key], rel_vec)
        assert ok, f"{where}: {key} differs by {err:.3e} (norm {np.linalg.norm(r[key]):.3e})"
    scalars = {"eta": rel_scal, "omega": rel_scal, "wsum": rel_scal, "gp_norm": rel_scal, "gd_norm": rel_scal}
    if prev is not None:
        move = np.linalg.norm(S.x - prev.x) + np.linalg.norm(S.y - prev.y)
        size = np.linalg.norm(S.x) + np.linalg.norm(S.y) + 1e-300
        if move < 1e-9 * size:
            del scalars["eta"]
        else:
            scalars["eta"] = max(rel_scal, 1e-13 * size / move)
    for key, tol in scalars.items():
        ok, err = close([g[key]], [r[key]], tol)
        assert ok, f"{where}: {key} gpu {g[key]!r} oracle {r[key]!r} (tolerance {tol:.1e})"
    for key in ("k", "attempts", "restarts", "refs_set", "last_restart_attempt"):
        assert g[key] == r[key], f"{where}: {key} gpu {g[key]} oracle {r[key]}"


@pytest.mark.parametrize("case", sorted(CASES))
def test_each_of_first_100_steps_from_oracle_state(case):
    make, o = CASES[case]
    lp = make()
    P, states = oracle_steps(lp, o, 100)
    with lpop.Problem(lp, **gpu_options(o)) as p:
        for k in range(1, 101):
            p.set_state(to_lib_state(states[k - 1]))
            p.solve(0.0, k)
            compare_full_state(p.get_state(), states[k], f"{case} step {k}", prev=states[k - 1])


@pytest.mark.parametrize("case", sorted(CASES))
def test_free_running_trajectory_matches_oracle(case):
    make, o = CASES[case]
    lp = make()
    horizon = 100 if o.mode == "plain" else 60
    steps = list(range(1, horizon + 1))
    ref, P, _ = oracle_trace(lp, o, steps)
    with lpop.Problem(lp, **gpu_options(o)) as p:
        for k in steps:
            p.solve(0.0, k)
            g = p.iterate()
            assert g["attempts"] == k
            compare_state(g, ref[k], f"{case} attempt {k}")


def test_full_size_transport_sampled_attempts():
    """The bench workload (25k supply + 25k demand rows, 200k arcs): one-step
    parity from the oracle's state at sampled attempts (including the checks at
    64, 128 and 192), and the free-running trajectory over the first 60."""
    lp = lpgen.transport(0)
    o = oracle.Options(alpha=1e-6, phi=20)
    P, states = oracle_steps(lp, o, 192)
    with lpop.Problem(lp, **gpu_options(o)) as p:
        for k in (1, 2, 3, 20, 21, 41, 63, 64, 65, 100, 127, 128, 129, 191, 192):
            p.set_state(to_lib_state(states[k - 1]))
            p.solve(0.0, k)
            compare_full_state(p.get_state(), states[k], f"transport step {k}", prev=states[k - 1])
        p.reset()
        for k in (1, 2, 5, 10, 20, 21, 40, 60):
            p.solve(0.0, k)
            compare_state(p.iterate(), _as_trace(states[k]), f"transport attempt {k}")


def _as_trace(S):
    return dict(x=S.x, y=S.y, T=S.T, Sigma=S.Sigma, eta=S.eta, omega=S.omega, k=S.k, restarts=S.restarts,
                wsum=S.wsum)


def oracle_count_range(lp, o, tol, seeds=5, iter_limit=100_000):
    """Iteration counts of the oracle to ``tol`` on the LP and on copies whose
    cost vector is perturbed by 1e-15 relative (one per seed): the count the
    method lands on is itself sensitive to rounding (on the transport LP these
    perturbations move it between 576 and 1088), so a second correct FP64
    implementation is held to this range, widened by 2% or, where the count
    is only tested every check period, by one period."""
    counts = []
    for seed in range(seeds + 1):
        P = oracle.scale_problem(lp, o)
        if seed:
            rng = np.random.default_rng(seed)
            P.c = P.c * (1.0 + 1e-15 * rng.standard_normal(P.c.size))
        S = oracle.initial_state(P, o)
        r, _, _ = oracle.solve(lp, o, tol=tol, iter_limit=iter_limit, P=P, S=S)
        counts.append(r.iterations)
    return min(counts), max(counts)


# The tight solve (1e-8) pins the final objective to 1e-6.  The power-law
# recipe does not reach 1e-8 (nor 1e-7) within 400,000 attempts even at 0.05%
# of its size (the oracle stalls there too), so for it the 1e-4 solve's
# objective is held to the distance two points at that tolerance can have.
FULL_SOLVE_CASES = {"tiny_plain_norm_freq": True, "tiny_pdlp_freq": True, "mixed_pdlp_adagrad": True,
                    "rowmix_pdlp": True, "transport_small_pdlp": True, "powerlaw_tiny_pdlp": False}
# Perturbed oracle solves that sample the count's spread: on the small power-law
# LP the oracle's own count moves between 3,648 and 8,000 attempts over 101
# perturbations of c at 1e-15 (median ~4,600; 6,016 or more in 7 of them), so
# five samples, or thirty (3,968 to 5,888), do not cover it.
COUNT_SEEDS = {"powerlaw_tiny_pdlp": 100}


@pytest.mark.parametrize("case", sorted(FULL_SOLVE_CASES))
def test_full_solve_matches_oracle(case):
    make, o = CASES[case]
    lp = make()
    res, P, S = oracle.solve(lp, o, tol=1e-4, iter_limit=100_000)
    with lpop.Problem(lp, **gpu_options(o)) as p:
        status = p.solve(1e-4, 100_000)
        x, y, st = p.result()
        if FULL_SOLVE_CASES[case]:
            tight, _, _ = oracle.solve(lp, o, tol=1e-8, iter_limit=400_000)
            p.reset()
            status_tight = p.solve(1e-8, 400_000)
            _, _, st_tight = p.result(want_x=False, want_y=False)
    assert status == res.status == lpop.LP_OPTIMAL
    lo, hi = oracle_count_range(lp, o, 1e-4, seeds=COUNT_SEEDS.get(case, 5))
    assert 0.98 * lo <= st["iterations"] <= 1.02 * hi, (st["iterations"], lo, hi, res.iterations)
    assert max(st["rel_pres"], st["rel_dres"], st["rel_gap"]) <= 1e-4
    if FULL_SOLVE_CASES[case]:
        assert status_tight == tight.status == lpop.LP_OPTIMAL
        assert st_tight["pobj"] == pytest.approx(tight.pobj, rel=1e-6, abs=1e-9)
        if lp.obj_opt is not None:
            assert st_tight["pobj"] == pytest.approx(lp.obj_opt, rel=1e-6, abs=1e-9)
    else:
        assert st["pobj"] == pytest.approx(res.pobj, rel=4e-4)
        assert st["pobj"] == pytest.approx(lp.obj_opt, rel=4e-4)
    # the returned point, re-evaluated by the oracle's KKT in user units
    kk = oracle.kkt(P, x / P.dc, y / P.dr, P.A @ (x / P.dc), P.At @ (y / P.dr))
    assert max(kk["rel_pres"], kk["rel_dres"], kk["rel_gap"]) <= 1.0001e-4
    assert kk["pobj"] == pytest.approx(st["pobj"], rel=1e-9, abs=1e-9)


def test_full_size_transport_solve():
    lp = lpgen.transport(0)
    o = oracle.Options(alpha=1e-4, phi=20)
    res, _, _ = oracle.solve(lp, o, tol=1e-4, iter_limit=20_000)
    with lpop.Problem(lp, **gpu_options(o)) as p:
        status = p.solve(1e-4, 20_000)
        _, _, st = p.result(want_x=False, want_y=False)
    assert status == res.status == lpop.LP_OPTIMAL
    lo, hi = oracle_count_range(lp, o, 1e-4, seeds=6)
    # termination is tested every check_every attempts, so counts move in whole check periods
    assert lo - o.check_every <= st["iterations"] <= hi + o.check_every, (st["iterations"], lo, hi, res.iterations)
    # both points satisfy the 1e-4 relative KKT tolerance, which bounds their objectives' distance
    assert st["pobj"] == pytest.approx(res.pobj, rel=4e-4)


def test_graph_and_direct_launches_agree_bitwise():
    lp = lpgen.row_length_mix(1)
    o = oracle.Options(alpha=1e-3, phi=5)
    out = []
    for use_graph in (1, 0):
        with lpop.Problem(lp, **gpu_options(o, use_graph=use_graph)) as p:
            p.solve(0.0, 200)
            out.append(p.iterate())
    for key in ("x", "y", "T", "Sigma"):
        assert np.array_equal(out[0][key], out[1][key]), key
    assert out[0]["eta"] == out[1]["eta"] and out[0]["omega"] == out[1]["omega"]


def test_runs_are_deterministic_and_reset_restores_the_start():
    lp = lpgen.transport(2, 800, 800, 6000)
    o = oracle.Options(alpha=1e-3, phi=20)
    with lpop.Problem(lp, **gpu_options(o)) as p:
        start = p.iterate()
        p.solve(1e-4, 5000)
        a = p.iterate()
        p.reset()
        again = p.iterate()
        p.solve(1e-4, 5000)
        b = p.iterate()
    for key in ("x", "y", "T", "Sigma"):
        assert np.array_equal(a[key], b[key])
        assert np.array_equal(start[key], again[key])


def test_unsorted_rows_and_repeated_entries_give_the_same_solve():
    """lp_create sorts each row by column and sums repeated entries: an LP whose
    rows are shuffled and whose entries are partly split into two exact halves
    is the same LP, so its solve is bitwise the same."""
    lp = lpgen.row_length_mix(2)
    rng = np.random.default_rng(5)
    rows_ci, rows_v, rp = [], [], [0]
    for i in range(lp.m):
        a, b = lp.row_ptr[i], lp.row_ptr[i + 1]
        ci, v = list(lp.col_idx[a:b]), list(lp.val[a:b])
        for k in rng.choice(len(ci), size=min(len(ci), 2), replace=False) if len(ci) else []:
            v[k] = v[k] / 2  # exact: the two halves add back to the value
            ci.append(ci[k])
            v.append(v[k])
        perm = rng.permutation(len(ci))
        rows_ci += [ci[t] for t in perm]
        rows_v += [v[t] for t in perm]
        rp.append(len(rows_ci))
    messy = copy.copy(lp)
    messy.row_ptr = np.asarray(rp, dtype=np.int64)
    messy.col_idx = np.asarray(rows_ci, dtype=np.int32)
    messy.val = np.asarray(rows_v, dtype=np.float64)
    assert messy.nnz > lp.nnz
    o = oracle.Options(alpha=1e-3, phi=5)
    out = []
    for q in (lp, messy):
        with lpop.Problem(q, **gpu_options(o)) as p:
            p.solve(0.0, 300)
            out.append(p.iterate())
    for key in ("x", "y", "T", "Sigma"):
        assert np.array_equal(out[0][key], out[1][key]), key
    assert out[0]["eta"] == out[1]["eta"] and out[0]["omega"] == out[1]["omega"]


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_device_memory_of_a_problem_within_lp_memory_bytes(precision):
    """lp_create takes its device buffers from one allocation of the
    lp_memory_bytes bound: the device's free memory drops by about that much
    (whole 2 MiB pages, plus the stream and graph) and no more."""
    torch = pytest.importorskip("torch")
    prec = lpop.LP_PREC_FP64 if precision == "fp64" else lpop.LP_PREC_MIXED
    lp = lpgen.transport(0, 5000, 5000, 80000)
    with lpop.Problem(lp, precision=prec) as warm:  # library, kernels and per-device tables loaded
        warm.solve(1e-4, 2000)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    bound = lpop.lp_memory_bytes(lp.m, lp.n, lp.nnz, lpop.lp_options_default(precision=prec))
    p = lpop.Problem(lp, precision=prec)
    try:
        p.solve(1e-4, 2000)
        torch.cuda.synchronize()
        free1, _ = torch.cuda.mem_get_info()
        used = free0 - free1
        assert used <= bound + (8 << 20), (used, bound)
        assert used >= bound - (4 << 20), (used, bound)
    finally:
        p.close()


def test_device_buffers_from_the_caller_allocator():
    """With device_alloc / device_free (here PyTorch's caching allocator) a
    problem's buffers come from the caller's pool -- one block of
    lp_memory_bytes -- and go back to it on destroy; the solve is bitwise the
    same as with the library's own allocation."""
    torch = pytest.importorskip("torch")
    lp = lpgen.transport(0, 2000, 2000, 16000)
    o = oracle.Options(alpha=1e-4, phi=20)
    with lpop.Problem(lp, **gpu_options(o)) as p:
        p.solve(1e-4, 5000)
        want = p.iterate()
    alloc = lpop.TorchDeviceAllocator()
    torch.cuda.synchronize()
    before = torch.cuda.memory_allocated()
    bound = lpop.lp_memory_bytes(lp.m, lp.n, lp.nnz, lpop.lp_options_default())
    with lpop.Problem(lp, allocator=alloc, **gpu_options(o)) as p:
        assert torch.cuda.memory_allocated() - before >= bound
        p.solve(1e-4, 5000)
        got = p.iterate()
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated() == before
    for key in ("x", "y", "T", "Sigma"):
        assert np.array_equal(got[key], want[key]), key


def test_plain_step_when_rows_sum_to_zero():
    """Plain mode on rows x_i - x_{i+1} = 0 (a cycle; Ruiz and L2 rescaling
    keep every row's sum at zero): the power iteration for ||A~||_2 restarts
    from the SplitMix64 sign direction, on both sides, so eta_0 matches the
    oracle's (instead of the fallback step 1 that a zero estimate gave)."""
    n = 40
    rows = np.repeat(np.arange(n), 2)
    cols = np.stack([np.arange(n), (np.arange(n) + 1) % n], axis=1).ravel()
    rng = np.random.default_rng(7)
    lp = lpgen.from_pattern(n, n, rows, cols, np.tile([1.0, -1.0], n), rng, sense_probs=(1.0, 0.0, 0.0),
                            var_probs=(1.0, 0.0, 0.0))
    o = oracle.Options(mode="plain", alpha=0.0, phi=0)
    P = oracle.scale_problem(lp, o)
    assert np.all(P.A @ np.ones(n) == 0.0)
    S0 = oracle.initial_state(P, o)
    with lpop.Problem(lp, **gpu_options(o)) as p:
        _, _, sc = p.scaling()
    assert sc["norm_est"] > 1.0
    assert sc["eta0"] == pytest.approx(S0.eta, rel=1e-12)


def test_alpha_zero_keeps_identity_preconditioners():
    lp = lpgen.mixed_small(4)
    o = oracle.Options(alpha=0.0, phi=1)
    with lpop.Problem(lp, **gpu_options(o)) as p:
        p.solve(0.0, 300)
        g = p.iterate()
    assert np.all(g["T"] == 1.0) and np.all(g["Sigma"] == 1.0)


def test_no_constraints():
    lp = lpgen.LP(m=0, n=3, row_ptr=np.zeros(1, np.int64), col_idx=np.zeros(0, np.int32), val=np.zeros(0),
                  b=np.zeros(0), c=np.array([1.0, -2.0, -0.5]), lb=np.array([0.0, -1.0, -np.inf]),
                  ub=np.array([4.0, 3.0, 2.0]), sense=np.zeros(0, np.uint8))
    for mode in ("pdlp", "plain"):
        o = oracle.Options(mode=mode, alpha=1e-2, phi=1)
        res, _, _ = oracle.solve(lp, o, tol=1e-8, iter_limit=10_000)
        with lpop.Problem(lp, **gpu_options(o)) as p:
            assert p.solve(1e-8, 10_000) == lpop.LP_OPTIMAL
            x, y, st = p.result()
        np.testing.assert_allclose(x, res.x, atol=1e-12)
        assert st["pobj"] == pytest.approx(-7.0)
        assert st["iterations"] == res.iterations


def test_single_variable_and_free_variables():
    rng = np.random.default_rng(3)
    m, n = 5, 1
    rows = np.arange(m)
    lp = lpgen.from_pattern(m, n, rows, np.zeros(m, dtype=np.int64), rng.standard_normal(m), rng,
                            sense_probs=(0.2, 0.4, 0.4), var_probs=(0.0, 0.0, 1.0))
    o = oracle.Options(alpha=1e-2, phi=1)
    P, states = oracle_steps(lp, o, 130)

    def moving(k):  # this instance converges to rounding level within ~60 steps; compare only steps that move
        S, Q = states[k], states[k - 1]
        move = np.linalg.norm(S.x - Q.x) + np.linalg.norm(S.y - Q.y)
        return move > 1e-9 * (np.linalg.norm(S.x) + np.linalg.norm(S.y))

    ks = [k for k in range(1, 131) if moving(k)]
    assert len(ks) >= 20
    with lpop.Problem(lp, **gpu_options(o)) as p:
        for k in ks:
            p.set_state(to_lib_state(states[k - 1]))
            p.solve(0.0, k)
            compare_full_state(p.get_state(), states[k], f"single variable step {k}", prev=states[k - 1])


def test_kernel_timing_and_launch_count():
    lp = lpgen.transport(0, 2000, 2000, 16000)
    o = oracle.Options(alpha=1e-4, phi=20)
    with lpop.Problem(lp, **gpu_options(o, kernel_timing=1)) as p:
        p.solve(0.0, 256)
        ms, samples, launches = p.kernel_times()
    assert samples[0] > 0 and samples[1] > 0
    assert ms[0] > 0 and ms[1] > 0
    # initial check (3 launches) + 4 graph replays of 64 attempts (2 kernels each) and a check (3)
    assert launches == 3 + 4 * (2 * 64 + 3)
    assert samples[0] == samples[1] == 4 * 64 // 8  # one attempt in 8 of each replay
    with lpop.Problem(lp, **gpu_options(o, kernel_timing=32)) as p:
        p.solve(0.0, 256)
        ms32, samples32, _ = p.kernel_times()
    assert samples32[0] == samples32[1] == 4 * 64 // 32
    assert ms32[0] > 0 and ms32[1] > 0


def test_invalid_input_rejected_before_device_work():
    lp = lpgen.mixed_small(0)
    b = lp.b.copy()
    b[0] = math.nan
    with pytest.raises(lpop.LpError) as ei:
        lpop.lp_create(lp.m, lp.n, lp.row_ptr, lp.col_idx, lp.val, b, lp.c, lp.lb, lp.ub, lp.sense)
    assert ei.value.code == lpop.LP_ERR_INVALID_INPUT


def test_log_every_writes_one_line_per_check(capfd):
    """log_every = k: lp_solve writes a line after every k-th KKT check (the
    initial check counts), holding that check's figures."""
    lp = lpgen.tiny_random(0)
    for every in (1, 3):
        with lpop.Problem(lp, alpha=1e-3, phi=20, log_every=every) as p:
            assert p.solve(1e-4, 100_000) == lpop.LP_OPTIMAL
            _, _, s = p.result(want_x=False, want_y=False)
        lines = [l.split() for l in capfd.readouterr().err.splitlines() if l.startswith("lpop: ")]
        checks = 1 + s["iterations"] // 64
        assert len(lines) == checks // every
        for k, l in enumerate(lines):
            assert int(l[l.index("attempts") + 1]) == 64 * (every * (k + 1) - 1)
            assert l[-1] == "fp64"
        if every == 1:
            last = lines[-1]
            assert int(last[last.index("accepted") + 1]) == s["accepted"]
            for key in ("rel_pres", "rel_dres", "rel_gap"):
                assert float(last[last.index(key) + 1]) == pytest.approx(s[key], rel=1e-3, abs=1e-300)
    with lpop.Problem(lp, alpha=1e-3, phi=20) as p:  # silent by default
        p.solve(1e-4, 100_000)
    assert "lpop: " not in capfd.readouterr().err
