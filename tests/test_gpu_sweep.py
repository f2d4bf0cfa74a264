"""Learning-rate sweep as one batch: every grid value's solve equals the same
solve run alone (bitwise), the choice is the fewest-iterations value, and the
alpha = 0 member keeps T = Sigma = I (vanilla PDHG)."""
import numpy as np
import pytest

import lpgen
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
