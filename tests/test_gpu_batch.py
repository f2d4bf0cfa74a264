"""Batched solves (lp_batch_*): many LPs in one persistent launch per round.

* One step from the oracle's state through a batch round of one attempt, for
  single-CTA teams and for cluster-wide teams (rows split over the CTAs of a
  thread-block cluster): vectors within 1e-12 relative, as for the
  single-problem kernels.
* A batch solve of LPs of mixed sizes in mixed precision to 1e-6 (so the
  FP32 phase hands over to FP64 inside the batched kernel): every member
  optimal, its tolerance certified by the oracle's own KKT evaluation of the
  returned point, and its objective within 2e-4 relative of the constructed
  optimum (a relative KKT error bounds the objective error only up to the
  problem's conditioning: at 1e-4 one of these instances is 1.4e-3 off).
* A member's result does not depend on the rest of the batch: solved alone or
  in a mix, with the same team size, it is bitwise identical -- also when slow
  members are handed to the single-problem kernels.
"""
import numpy as np
import pytest

import lpgen
import oracle
import paper_2506_17650_gb300 as lpop
from paper_2506_17650_gb300 import build as lpbuild
from tests.test_gpu_parity import compare_full_state, gpu_options, oracle_steps, to_lib_state

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lpbuild.build()
    lpop.load_library()


def _members(seeds, m_values):
    lps = []
    for s, m in zip(seeds, m_values):
        lps.append(lpgen.batch_member(s, int(m), int(2.5 * m)))
    return lps


@pytest.mark.parametrize("cluster", [1, 4])
def test_batch_one_step_from_oracle_state(cluster):
    cases = [(lpgen.mixed_small(0), oracle.Options(alpha=1e-2, phi=1)),
             (lpgen.row_length_mix(0), oracle.Options(alpha=1e-3, phi=20)),
             (lpgen.tiny_random(0), oracle.Options(mode="plain", alpha=1e-2, phi=1))]
    traj = [oracle_steps(lp, o, 66)[1] for lp, o in cases]
    probs = [lpop.Problem(lp, **gpu_options(o)) for lp, o in cases]
    try:
        with lpop.Batch(probs, cluster_size=cluster, wide_nnz=0 if cluster > 1 else 1 << 62) as b:
            for k in (1, 2, 20, 63, 64, 65):
                for p, states in zip(probs, traj):
                    p.set_state(to_lib_state(states[k - 1]))
                b.round(0.0, 1, 1_000_000)
                for (lp, o), p, states in zip(cases, probs, traj):
                    compare_full_state(p.get_state(), states[k], f"{lp.name} batch step {k}", prev=states[k - 1])
    finally:
        for p in probs:
            p.close()


@pytest.mark.parametrize("cluster,wide_nnz", [(1, 1 << 62), (4, 6000)])
def test_batch_solve_mixed_sizes(cluster, wide_nnz):
    rng = np.random.default_rng(5)
    ms = np.floor(10 ** rng.uniform(2, np.log10(3000), size=12)).astype(int)
    lps = _members(range(100, 112), ms)
    probs = [lpop.Problem(lp, alpha=1e-3, phi=20, precision=lpop.LP_PREC_MIXED) for lp in lps]
    try:
        with lpop.Batch(probs, cluster_size=cluster, wide_nnz=wide_nnz) as b:
            n_opt = b.solve(1e-6, 400_000, 256)
            status, iters = b.status()
        assert n_opt == len(lps)
        assert np.all(status == lpop.LP_OPTIMAL)
        for lp, p in zip(lps, probs):
            x, y, st = p.result()
            assert st["status"] == lpop.LP_OPTIMAL
            P = oracle.scale_problem(lp, oracle.Options())
            kk = oracle.kkt(P, x / P.dc, y / P.dr, P.A @ (x / P.dc), P.At @ (y / P.dr))
            assert max(kk["rel_pres"], kk["rel_dres"], kk["rel_gap"]) <= 1.01e-6, lp.name
            assert st["pobj"] == pytest.approx(lp.obj_opt, rel=2e-4, abs=1e-6), lp.name
    finally:
        for p in probs:
            p.close()


def test_member_result_independent_of_the_mix():
    lps = _members(range(200, 208), [150, 400, 900, 120, 2000, 300, 700, 1500])
    target = 2
    alone = lpop.Problem(lps[target], alpha=1e-3, phi=20, precision=lpop.LP_PREC_MIXED)
    mix = [lpop.Problem(lp, alpha=1e-3, phi=20, precision=lpop.LP_PREC_MIXED) for lp in lps]
    try:
        with lpop.Batch([alone]) as b1:
            b1.solve(1e-4, 100_000, 128)
        with lpop.Batch(mix) as b2:
            b2.solve(1e-4, 100_000, 128)
        a = alone.get_state()
        m = mix[target].get_state()
        for key in ("x", "y", "T", "Sigma", "ax"):
            assert np.array_equal(a[key], m[key]), key
        assert a["attempts"] == m["attempts"] and a["eta"] == m["eta"]
    finally:
        alone.close()
        for p in mix:
            p.close()


def test_batch_and_single_path_agree_on_the_solution():
    lp = lpgen.batch_member(7, 800, 2000)
    single = lpop.Problem(lp, alpha=1e-3, phi=20)
    batched = lpop.Problem(lp, alpha=1e-3, phi=20)
    try:
        single.solve(1e-6, 200_000)
        _, _, s1 = single.result(False, False)
        with lpop.Batch([batched]) as b:
            b.solve(1e-6, 200_000, 256)
        _, _, s2 = batched.result(False, False)
        assert s1["status"] == s2["status"] == lpop.LP_OPTIMAL
        assert s2["pobj"] == pytest.approx(s1["pobj"], rel=2e-4)
        assert s2["pobj"] == pytest.approx(lp.obj_opt, rel=2e-4)
    finally:
        single.close()
        batched.close()


def test_handoff_to_single_problem_path():
    """Members still open after 256 attempts finish on the single-problem
    kernels (lp_batch_set_handoff); every member optimal and certified, and a
    member's result is the same alone and in the mix (the rule depends only on
    its own attempts)."""
    lps = _members(range(300, 308), [150, 400, 900, 120, 2000, 300, 700, 1500])
    target = 4
    mix = [lpop.Problem(lp, alpha=1e-3, phi=20, precision=lpop.LP_PREC_MIXED) for lp in lps]
    alone = lpop.Problem(lps[target], alpha=1e-3, phi=20, precision=lpop.LP_PREC_MIXED)
    try:
        with lpop.Batch(mix) as b:
            b.set_handoff(256)
            n_opt = b.solve(1e-4, 100_000, 128)
            status, iters = b.status()
        assert n_opt == len(lps) and np.all(status == lpop.LP_OPTIMAL)
        assert np.any(iters > 256)  # some member did leave the batch
        for lp, p in zip(lps, mix):
            x, y, st = p.result()
            P = oracle.scale_problem(lp, oracle.Options())
            kk = oracle.kkt(P, x / P.dc, y / P.dr, P.A @ (x / P.dc), P.At @ (y / P.dr))
            assert max(kk["rel_pres"], kk["rel_dres"], kk["rel_gap"]) <= 1.01e-4, lp.name
        with lpop.Batch([alone]) as b1:
            b1.set_handoff(256)
            b1.solve(1e-4, 100_000, 128)
        a, m = alone.get_state(), mix[target].get_state()
        for key in ("x", "y", "T", "Sigma"):
            assert np.array_equal(a[key], m[key]), key
        assert a["attempts"] == m["attempts"]
    finally:
        alone.close()
        for p in mix:
            p.close()
