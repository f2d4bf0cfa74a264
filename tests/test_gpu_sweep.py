"""Learning-rate sweep as one batch: every grid value's solve equals the same
solve run alone (bitwise), the choice is the fewest-iterations value, the
alpha = 0 member keeps T = Sigma = I (vanilla PDHG), and each grid value's
solve is held to the oracle's solve at that learning rate: the same status,
an iteration count within the spread of the oracle's own count under 1e-15
perturbations of c, and an objective within the distance two points at the
1e-4 tolerance can have."""
import numpy as np
import pytest

import lpgen
import oracle
import paper_2506_17650_gb300 as lpop
from paper_2506_17650_gb300 import build as lpbuild

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lpbuild.build()
    lpop.load_library()


def test_alpha_sweep_matches_single_runs():
    from paper_2506_17650_gb300.sweep import alpha_sweep

    lp = lpgen.tiny_random(0)
    grid = (0.0, 1e-1, 1e-2, 1e-3)
    opts = dict(mode=lpop.LP_MODE_PLAIN, phi=1)
    best, rows = alpha_sweep(lp, grid, tol=1e-4, **opts)
    assert all(r["status"] == lpop.LP_OPTIMAL for r in rows)
    assert best == min(rows, key=lambda r: (r["iterations"], r["alpha"]))["alpha"]
    for r in rows:
        with lpop.Problem(lp, alpha=r["alpha"], **opts) as p:
            with lpop.Batch([p]) as b:
                b.solve(1e-4, 200_000, 256)
            st = p.get_state()
            assert st["attempts"] == r["iterations"]
            if r["alpha"] == 0.0:
                assert np.all(st["T"] == 1.0) and np.all(st["Sigma"] == 1.0)


def test_alpha_sweep_against_the_oracle():
    from paper_2506_17650_gb300.sweep import alpha_sweep
    from tests.test_gpu_parity import oracle_count_range

    lp = lpgen.tiny_random(0)
    grid = (0.0, 1e-1, 1e-2, 1e-3)
    best, rows = alpha_sweep(lp, grid, tol=1e-4, mode=lpop.LP_MODE_PLAIN, phi=1)
    for r in rows:
        o = oracle.Options(mode="plain", alpha=r["alpha"], phi=1)
        res, P, _ = oracle.solve(lp, o, tol=1e-4, iter_limit=200_000)
        assert r["status"] == res.status == lpop.LP_OPTIMAL
        lo, hi = oracle_count_range(lp, o, 1e-4)
        assert 0.98 * lo <= r["iterations"] <= 1.02 * hi, (r["alpha"], r["iterations"], lo, hi)
        assert r["pobj"] == pytest.approx(res.pobj, rel=4e-4)
        assert r["pobj"] == pytest.approx(lp.obj_opt, rel=4e-4)
    # the oracle's own choice over the grid (fewest attempts, ties to the smaller
    # rate): here 1e-1, with 1,152 attempts against 1,856 and more for the others
    counts = {a: oracle.solve(lp, oracle.Options(mode="plain", alpha=a, phi=1), tol=1e-4, iter_limit=200_000)[0].iterations
              for a in grid}
    assert best == min(grid, key=lambda a: (counts[a], a)), (best, counts)
