"""The large power-law LP at full size (m = 2M, n = 5M, ~30M nonzeros), in
the launch configuration the benchmark times (same grids, sliced and
segmented bins, segments of ~16k entries), against the CPU oracle.

The oracle needs about a second per attempt at this size, so parity is
checked on sampled outputs it can compute: the initial KKT check, then one
attempt at a time from the oracle's own state for the first attempts (with
check_every = 2, so that attempts 2 and 4 also run the KKT check and the
restart logic, attempt 1 records the online gradient and attempt 2 applies
the preconditioner update), each vector within 1e-12 relative as in the
small cases.  The free-running GPU trajectory over the same attempts is
held to 1e-10.  After one benchmark step (640 free-running attempts, plus
one, so that the final report is the evaluation of the returned point and
not a check that may then restart) the KKT figures the GPU reports are
re-evaluated by the oracle's KKT at the point the GPU returns, and the
invariants of the method hold (T >= 1, Sigma >= floor, all finite).
"""
import numpy as np
import pytest

import lpgen
import oracle
import paper_2506_17650_gb300 as lpop
from paper_2506_17650_gb300 import build as lpbuild
from tests.test_gpu_parity import close, compare_full_state, gpu_options, to_lib_state

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def full():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lpbuild.build()
    lpop.load_library()
    lp = lpgen.powerlaw(0)
    o = oracle.Options(alpha=1e-6, phi=20, check_every=2)
    P = oracle.scale_problem(lp, o)
    return lp, o, P


def test_full_size_powerlaw_sampled_attempts(full):
    lp, o, P = full
    import copy

    S = oracle.initial_state(P, o)
    oracle.check(P, S, o, 0.0)
    S.checked0 = True
    with lpop.Problem(lp, **gpu_options(o)) as p:
        dr, dc, sc = p.scaling()
        assert close(dr, P.dr, 1e-13)[0] and close(dc, P.dc, 1e-13)[0]
        assert sc["eta0"] == pytest.approx(1.0 / abs(P.A).max(), rel=1e-12)
        # the initial check: KKT of the starting point
        p.solve(0.0, 0)
        _, _, st0 = p.result(want_x=False, want_y=False)
        for key in ("rel_pres", "rel_dres", "rel_gap", "pobj", "dobj"):
            assert st0[key] == pytest.approx(S.stats[key], rel=1e-11, abs=1e-300), key
        states = [copy.deepcopy(S)]
        for k in range(1, 5):
            oracle.attempt(P, S, o)
            if S.attempts % o.check_every == 0:
                oracle.check(P, S, o, 0.0)
            p.set_state(to_lib_state(states[-1]))
            p.solve(0.0, k)
            compare_full_state(p.get_state(), S, f"power-law full size step {k}", prev=states[-1])
            states.append(copy.deepcopy(S))
            if len(states) > 2:
                states.pop(0)
        # free-running from the start over the same attempts
        p.reset()
        p.solve(0.0, 4)
        g = p.iterate()
        for key in ("x", "y", "T", "Sigma"):
            ok, err = close(g[key], getattr(S, key), 1e-10)
            assert ok, f"free-running attempt 4: {key} differs by {err:.3e}"
        assert g["k"] == S.k and g["restarts"] == S.restarts


def test_full_size_powerlaw_bench_step_certified(full):
    lp, o, P = full
    bench = oracle.Options(alpha=1e-6, phi=20)  # the benchmark's check period of 64
    with lpop.Problem(lp, **gpu_options(bench)) as p:
        assert p.solve(0.0, 641) == lpop.LP_ITERATION_LIMIT
        x, y, st = p.result()
        it = p.iterate()
    assert st["iterations"] == 641
    kk = oracle.kkt(P, x / P.dc, y / P.dr, P.A @ (x / P.dc), P.At @ (y / P.dr))
    for key in ("rel_pres", "rel_dres", "rel_gap", "pobj", "dobj"):
        assert st[key] == pytest.approx(kk[key], rel=1e-9), key
    assert np.all(it["T"] >= 1.0) and np.all(np.isfinite(it["T"]))
    assert np.all(it["Sigma"] >= 1e-6) and np.all(np.isfinite(it["Sigma"]))
