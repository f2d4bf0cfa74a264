"""The no-allocation entry point lp_power_norm_noalloc.

Callers that cannot allocate device memory (their framework owns all of it,
or they must not allocate inside a latency-critical loop) pass their matrix
in device memory they already own; the entry point works in the library's
fixed scratch array.  Its estimate of ||A~||_2 must equal the one lp_create
computes for the same preprocessed matrix (reported by lp_get_scaling in
plain mode) within 1e-10 relative, on two calls in a row (the second call
reuses the scratch the first one left behind).

This file is collected last on purpose, so that a run stopping at its first
failure has run every other test before it.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import lpgen
import paper_2506_17650_gb300 as lpop
from paper_2506_17650_gb300 import build as lpbuild

pytestmark = pytest.mark.gpu


def _device_csr(torch, M):
    M = M.tocsr()
    M.sort_indices()
    return (torch.tensor(M.indptr.astype(np.int32), device="cuda"),
            torch.tensor(M.indices.astype(np.int32), device="cuda"),
            torch.tensor(M.data.astype(np.float64), device="cuda"))


def test_noalloc_power_norm_matches_lp_create():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lpbuild.build()
    lpop.load_library()
    lp = lpgen.tiny_random(0)
    with lpop.Problem(lp, mode=lpop.LP_MODE_PLAIN, power_iters=200) as p:
        dr, dc, sc = p.scaling()
    ref = sc["norm_est"]
    assert ref > 0
    A = sp.diags(dr) @ lp.csr() @ sp.diags(dc)
    a = _device_csr(torch, A)
    at = _device_csr(torch, A.T)
    ptrs = [t.data_ptr() for t in a] + [t.data_ptr() for t in at]
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        est = lpop.lp_power_norm_noalloc(lp.m, lp.n, *ptrs, iters=200, stream=stream)
        assert est == pytest.approx(ref, rel=1e-10), f"call {call}: {est!r} vs {ref!r}"
    # sizes beyond the fixed scratch are refused before any device work
    with pytest.raises(lpop.LpError) as ei:
        lpop.lp_power_norm_noalloc(lp.m, 1 << 20, *ptrs, iters=10, stream=stream)
    assert ei.value.code == lpop.LP_ERR_INVALID_ARG
    assert "scratch" in lpop.lp_last_error(None)


def test_noalloc_power_norm_restarts_when_rows_sum_to_zero():
    """Rows w_i (x_i - x_{i+1}) sum to zero, so the all-ones start direction is
    in the null space of A; the entry point starts again from the SplitMix64
    sign direction (as lp_create does) and finds the SVD norm."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lpbuild.build()
    n = 40
    w = np.random.default_rng(0).uniform(0.5, 2.0, size=n)
    rows = np.repeat(np.arange(n), 2)
    cols = np.stack([np.arange(n), (np.arange(n) + 1) % n], axis=1).ravel()
    A = sp.csr_matrix((np.stack([w, -w], axis=1).ravel(), (rows, cols)), shape=(n, n))
    a = _device_csr(torch, A)
    at = _device_csr(torch, A.T)
    ptrs = [t.data_ptr() for t in a] + [t.data_ptr() for t in at]
    stream = torch.cuda.current_stream().cuda_stream
    ref = np.linalg.norm(A.toarray(), 2)
    for call in range(2):
        est = lpop.lp_power_norm_noalloc(n, n, *ptrs, iters=200, stream=stream)
        assert est == pytest.approx(ref, rel=1e-8), f"call {call}: {est!r} vs {ref!r}"

