"""Failure detection through the C ABI, with every failure made on the host.

Nothing here faults, traps or hangs the GPU: the failures are a time limit
that has already run out, a caller allocator that returns NULL or a
misaligned block, and a checkpoint whose finite but huge step size drives
the iterate to infinity, which the next KKT check reports as a numerical
error.  After each failure the library must still work (a fresh problem
solves normally) and must not leak a caller-allocated block.
"""
import ctypes

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


class FakeAllocator:
    """device_alloc / device_free that count blocks and fail on request:
    ``mode`` "null" returns NULL, "misaligned" returns a real block offset by
    8 bytes (the library must hand it straight back), "ok" passes through to
    PyTorch's caching allocator."""

    def __init__(self, mode):
        import torch

        self.torch = torch
        self.mode = mode
        self.live = {}  # address handed out -> (torch address, bytes)
        self.calls = 0
        self.frees = 0
        self._alloc = lpop._DEVICE_ALLOC_FN(self._do_alloc)
        self._free = lpop._DEVICE_FREE_FN(self._do_free)

    def _do_alloc(self, nbytes, ctx):
        self.calls += 1
        if self.mode == "null":
            return None
        base = self.torch.cuda.caching_allocator_alloc(int(nbytes) + 256, self.torch.cuda.current_device())
        addr = base + 8 if self.mode == "misaligned" else base
        self.live[addr] = (base, int(nbytes))
        return addr

    def _do_free(self, ptr, nbytes, ctx):
        self.frees += 1
        base, size = self.live.pop(ptr)
        assert size == nbytes
        self.torch.cuda.caching_allocator_delete(base)

    def options(self):
        return dict(device_alloc=ctypes.cast(self._alloc, ctypes.c_void_p).value,
                    device_free=ctypes.cast(self._free, ctypes.c_void_p).value)


def _solves_normally(lp):
    with lpop.Problem(lp, alpha=1e-3, phi=20) as p:
        st = p.solve(1e-4, 50_000)
        _, _, s = p.result(want_x=False, want_y=False)
    assert st == lpop.LP_OPTIMAL
    assert abs(s["pobj"] - lp.obj_opt) <= 1e-3 * (1 + abs(lp.obj_opt))


def test_time_limit_reached():
    lp = lpgen.transport(0, 2_000, 2_000, 16_000)
    with lpop.Problem(lp, alpha=1e-6, phi=20, time_limit=1e-9) as p:
        st = p.solve(1e-12, 1_000_000)
        _, _, s = p.result(want_x=False, want_y=False)
        assert st == lpop.LP_TIME_LIMIT
        assert s["status"] == lpop.LP_TIME_LIMIT
        # the limit is tested after each check period: one period ran
        assert 1 <= s["iterations"] <= 64
        assert np.isfinite(s["pobj"])
        # a later call continues from where the limit stopped it
        st2 = p.solve(1e-12, 1_000_000)
        _, _, s2 = p.result(want_x=False, want_y=False)
        assert st2 == lpop.LP_TIME_LIMIT and s2["iterations"] > s["iterations"]
    _solves_normally(lpgen.tiny_random(1))


def test_caller_allocator_returning_null_is_out_of_memory():
    lp = lpgen.tiny_random(2)
    fa = FakeAllocator("null")
    with pytest.raises(lpop.LpError) as ei:
        lpop.Problem(lp, allocator=fa, alpha=1e-3)
    assert ei.value.code == lpop.LP_ERR_OOM
    assert "NULL" in lpop.lp_last_error(None)
    assert fa.calls >= 1 and not fa.live
    _solves_normally(lp)


def test_caller_allocator_misaligned_block_is_rejected_and_returned():
    lp = lpgen.tiny_random(3)
    fa = FakeAllocator("misaligned")
    with pytest.raises(lpop.LpError) as ei:
        lpop.Problem(lp, allocator=fa, alpha=1e-3)
    assert ei.value.code == lpop.LP_ERR_INVALID_ARG
    assert "aligned" in lpop.lp_last_error(None)
    assert fa.calls == 1 and fa.frees == 1 and not fa.live


def test_caller_allocator_blocks_all_returned():
    lp = lpgen.tiny_random(4)
    fa = FakeAllocator("ok")
    with lpop.Problem(lp, allocator=fa, alpha=1e-3, phi=20) as p:
        assert p.solve(1e-4, 50_000) == lpop.LP_OPTIMAL
        assert fa.live
    assert not fa.live and fa.frees == fa.calls


@pytest.mark.parametrize("precision", [lpop.LP_PREC_FP64, lpop.LP_PREC_MIXED])
def test_huge_step_from_checkpoint_is_a_numerical_error(precision):
    """Plain mode (fixed step): a checkpoint with a finite step size of 1e300
    passes lp_set_state's checks (finite, positive); the next attempts
    overflow the free variables to infinity and then NaN, and the next KKT
    check reports LP_NUMERICAL_ERROR (the oracle does the same at attempt 64)."""
    lp = lpgen.mixed_small(5)
    assert np.any(~np.isfinite(lp.lb) & ~np.isfinite(lp.ub))  # free variables
    with lpop.Problem(lp, mode=lpop.LP_MODE_PLAIN, alpha=1e-3, phi=20, precision=precision, use_graph=0) as p:
        assert p.solve(0.0, 10) == lpop.LP_ITERATION_LIMIT
        st = p.get_state()
        st["eta"] = 1e300
        p.set_state(st)
        status = p.solve(1e-4, 640)
        _, _, s = p.result(want_x=False, want_y=False)
        assert status == lpop.LP_NUMERICAL_ERROR
        assert s["status"] == lpop.LP_NUMERICAL_ERROR
        assert s["iterations"] == 64
    _solves_normally(lpgen.tiny_random(6))


def test_huge_step_is_rejected_by_the_adaptive_rule():
    """pdlp mode: the same checkpoint makes every attempt's step limit NaN, so
    every attempt is rejected (no accepted step: k stays, as in the oracle);
    the checks still restart to the finite averages, and the solve ends at
    its iteration limit with a finite KKT error."""
    lp = lpgen.mixed_small(5)
    with lpop.Problem(lp, alpha=1e-3, phi=20, use_graph=0) as p:
        p.solve(0.0, 10)
        st = p.get_state()
        st["eta"] = 1e300
        p.set_state(st)
        status = p.solve(1e-4, 640)
        it = p.iterate()
        _, _, s = p.result(want_x=False, want_y=False)
    assert status == lpop.LP_ITERATION_LIMIT
    assert it["k"] == st["k"] and not it["accepted"]
    assert np.all(np.isfinite(it["x"])) and np.all(np.isfinite(it["y"]))
    assert np.isfinite(s["rel_pres"]) and np.isfinite(s["rel_dres"]) and np.isfinite(s["rel_gap"])
