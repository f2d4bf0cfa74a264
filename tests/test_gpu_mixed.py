"""Mixed precision (LP_PREC_MIXED) against the FP64 oracle.

The FP32 phase runs the sparse products, vector updates and projections in
FP32 (FP32 matrix values, FP32 vectors); the KKT, step-size and normalisation
reductions and the solver scalars stay FP64, and a final FP64 phase takes over
from the FP32 iterate.  Its error against the FP64 oracle is stated per test:

* one step from the oracle's state (rounded to FP32): every vector within
  1e-5 relative of the oracle's next state (FP32 rounding of ~30 operations
  per entry, with cancellation in c - A^T y and b - A x);
* a solve to 1e-4: status optimal with the tolerance certified by the FP64
  check; objective within 4e-4 relative of the oracle's (the distance two
  points that both meet a 1e-4 relative KKT tolerance can have);
* a solve to 1e-8 must pass through the FP64 refinement phase and reach the
  oracle's tight objective within 1e-6 relative.
"""
import copy

import numpy as np
import pytest

import lpgen
import oracle
import paper_2506_17650_gb300 as lpop
from paper_2506_17650_gb300 import build as lpbuild
from tests.test_gpu_parity import CASES, close, gpu_options, oracle_steps, to_lib_state

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lpbuild.build()
    lpop.load_library()


def mixed(o, **extra):
    return gpu_options(o, precision=lpop.LP_PREC_MIXED, **extra)


@pytest.mark.parametrize("case", ["tiny_plain_norm_freq", "tiny_pdlp_freq", "mixed_pdlp_adagrad", "rowmix_pdlp",
                                  "transport_small_pdlp", "powerlaw_small_pdlp"])
def test_mixed_one_step_from_oracle_state(case):
    make, o = CASES[case]
    lp = make()
    P, states = oracle_steps(lp, o, 70)
    with lpop.Problem(lp, **mixed(o)) as p:
        for k in (1, 2, 5, 20, 21, 40, 63, 64, 65, 70):
            p.set_state(to_lib_state(states[k - 1]))
            p.solve(0.0, k)
            g = p.get_state()
            r = to_lib_state(states[k])
            for key in ("x", "y", "ax", "T", "Sigma", "xbar", "ybar"):
                ok, err = close(g[key], r[key], 1e-5)
                assert ok, f"{case} step {k}: {key} differs by {err:.3e} (norm {np.linalg.norm(r[key]):.3e})"
            assert g["k"] == r["k"] and g["attempts"] == r["attempts"] and g["restarts"] == r["restarts"]


@pytest.mark.parametrize("case", ["tiny_plain_norm_freq", "tiny_pdlp_freq", "mixed_pdlp_adagrad", "rowmix_pdlp",
                                  "transport_small_pdlp", "powerlaw_tiny_pdlp"])
def test_mixed_solve_to_1e4_is_certified(case):
    make, o = CASES[case]
    lp = make()
    res, P, _ = oracle.solve(lp, o, tol=1e-4, iter_limit=100_000)
    with lpop.Problem(lp, **mixed(o)) as p:
        status = p.solve(1e-4, 100_000)
        x, y, st = p.result()
    assert status == lpop.LP_OPTIMAL
    assert max(st["rel_pres"], st["rel_dres"], st["rel_gap"]) <= 1e-4
    # the oracle's own KKT of the returned point (FP64, user units)
    kk = oracle.kkt(P, x / P.dc, y / P.dr, P.A @ (x / P.dc), P.At @ (y / P.dr))
    assert max(kk["rel_pres"], kk["rel_dres"], kk["rel_gap"]) <= 1.01e-4
    assert st["pobj"] == pytest.approx(res.pobj, rel=4e-4, abs=1e-6)


@pytest.mark.parametrize("case", ["tiny_pdlp_freq", "mixed_pdlp_adagrad", "transport_small_pdlp"])
def test_mixed_refinement_reaches_tight_tolerance(case):
    make, o = CASES[case]
    lp = make()
    tight, _, _ = oracle.solve(lp, o, tol=1e-8, iter_limit=400_000)
    with lpop.Problem(lp, **mixed(o)) as p:
        status = p.solve(1e-8, 400_000)
        _, _, st = p.result(want_x=False, want_y=False)
    assert status == tight.status == lpop.LP_OPTIMAL
    assert max(st["rel_pres"], st["rel_dres"], st["rel_gap"]) <= 1e-8
    assert st["pobj"] == pytest.approx(tight.pobj, rel=1e-6, abs=1e-9)


def test_mixed_full_size_transport():
    lp = lpgen.transport(0)
    o = oracle.Options(alpha=1e-6, phi=20)
    res, P, _ = oracle.solve(lp, o, tol=1e-4, iter_limit=20_000)
    with lpop.Problem(lp, **mixed(o)) as p:
        status = p.solve(1e-4, 20_000)
        x, y, st = p.result()
    assert status == lpop.LP_OPTIMAL
    kk = oracle.kkt(P, x / P.dc, y / P.dr, P.A @ (x / P.dc), P.At @ (y / P.dr))
    assert max(kk["rel_pres"], kk["rel_dres"], kk["rel_gap"]) <= 1.01e-4
    assert st["pobj"] == pytest.approx(res.pobj, rel=4e-4)
