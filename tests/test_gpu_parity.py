"""GPU parity: the CUDA library (through the C ABI) against the CPU oracle.

Bars (floating point, FP64 on both sides):
  * iterates, preconditioners and step scalars of the first 100 step attempts:
    ||gpu - oracle|| <= 1e-10 ||oracle|| + 1e-14 sqrt(len) (the sqrt(len) floor
    covers vectors that are still exactly zero on the oracle side);
  * discrete state (accepted steps k, attempts, restarts) identical;
  * a full solve: same status, final objective within 1e-6 relative, and
    iteration count within +-2% (at most one check period apart when smaller).
"""
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
        ok, err = close([g[key]], [r[key]])
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


@pytest.mark.parametrize("case", sorted(CASES))
def test_first_100_attempts_match_oracle(case):
    make, o = CASES[case]
    lp = make()
    steps = list(range(1, 101))
    ref, P, _ = oracle_trace(lp, o, steps)
    with lpop.Problem(lp, **gpu_options(o)) as p:
        for k in steps:
            p.solve(0.0, k)
            g = p.iterate()
            assert g["attempts"] == k
            compare_state(g, ref[k], f"{case} attempt {k}")


def test_full_size_transport_sampled_attempts():
    """The bench workload (25k supply + 25k demand rows, 200k arcs) in the launch
    configuration the bench times (graph replay of whole check periods)."""
    lp = lpgen.transport(0)
    o = oracle.Options(alpha=1e-4, phi=20)
    marks = [1, 2, 3, 5, 10, 20, 21, 40, 63, 64, 65, 100, 128, 129, 192]
    ref, P, _ = oracle_trace(lp, o, marks)
    with lpop.Problem(lp, **gpu_options(o)) as p:
        done = 0
        for k in marks:
            p.solve(0.0, k)
            done = k
            compare_state(p.iterate(), ref[k], f"transport attempt {k}")
        assert done == marks[-1]


@pytest.mark.parametrize("case", ["tiny_plain_norm_freq", "tiny_pdlp_freq", "mixed_pdlp_adagrad",
                                  "rowmix_pdlp", "transport_small_pdlp"])
def test_full_solve_matches_oracle(case):
    make, o = CASES[case]
    lp = make()
    res, P, S = oracle.solve(lp, o, tol=1e-4, iter_limit=100_000)
    with lpop.Problem(lp, **gpu_options(o)) as p:
        status = p.solve(1e-4, 100_000)
        x, y, st = p.result()
    assert status == res.status == lpop.LP_OPTIMAL
    assert st["pobj"] == pytest.approx(res.pobj, rel=1e-6, abs=1e-9)
    n_gpu, n_cpu = st["iterations"], res.iterations
    assert abs(n_gpu - n_cpu) <= max(0.02 * n_cpu, 0), (n_gpu, n_cpu)
    if lp.obj_opt is not None:
        assert st["pobj"] == pytest.approx(lp.obj_opt, rel=1e-3, abs=1e-6)
    # the returned point in user units
    assert close(x, res.x, 1e-6)[0] and close(y, res.y, 1e-6)[0]


def test_full_size_transport_solve():
    lp = lpgen.transport(0)
    o = oracle.Options(alpha=1e-4, phi=20)
    res, _, _ = oracle.solve(lp, o, tol=1e-4, iter_limit=20_000)
    with lpop.Problem(lp, **gpu_options(o)) as p:
        status = p.solve(1e-4, 20_000)
        _, _, st = p.result(want_x=False, want_y=False)
    assert status == res.status == lpop.LP_OPTIMAL
    assert st["pobj"] == pytest.approx(res.pobj, rel=1e-6)
    assert abs(st["iterations"] - res.iterations) <= 0.02 * res.iterations


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
    ref, _, _ = oracle_trace(lp, o, list(range(1, 80)))
    with lpop.Problem(lp, **gpu_options(o)) as p:
        for k in (1, 2, 10, 64, 79):
            p.solve(0.0, k)
            compare_state(p.iterate(), ref[k], f"single variable attempt {k}")


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


def test_invalid_input_rejected_before_device_work():
    lp = lpgen.mixed_small(0)
    b = lp.b.copy()
    b[0] = math.nan
    with pytest.raises(lpop.LpError) as ei:
        lpop.lp_create(lp.m, lp.n, lp.row_ptr, lp.col_idx, lp.val, b, lp.c, lp.lb, lp.ub, lp.sense)
    assert ei.value.code == lpop.LP_ERR_INVALID_INPUT
