"""The C-ABI library builds for sm_103a, loads, and exports what include/lpop.h
declares; host-side argument and data validation runs without a GPU."""
import ctypes
import math
import os
import re
import subprocess

import numpy as np
import pytest

import lpgen
import paper_2506_17650_gb300 as lpop
from paper_2506_17650_gb300 import build as lpbuild
from tests.conftest import ROOT

HEADER = os.path.join(ROOT, "include", "lpop.h")


@pytest.fixture(scope="module")
def lib():
    lpbuild.build()
    return lpop.load_library()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lp_[a-z_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("lp_options_default", "lp_create", "lp_solve", "lp_result", "lp_get_iterate",
                     "lp_destroy", "lp_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", lpbuild.LIB], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r" T (lp_[a-z_]+)$", out, flags=re.M))
    for name in declared_functions():
        assert name in exported, name
        assert hasattr(lib, name)


def test_options_default(lib):
    o = lpop.lp_options_default()
    assert o.mode == lpop.LP_MODE_PDLP
    assert o.scheduler == lpop.LP_SCHED_ADAGRAD
    assert o.phi == 20 and o.normalize == 1 and o.check_every == 64
    assert o.ruiz_iters == 10 and o.pc_beta == 1.0 and o.precond_floor == 1e-6
    assert o.alpha == 0.0 and o.use_graph == 1 and o.restart == 1
    assert o.refine_stall == 16 and o.log_every == 0
    assert ctypes.sizeof(lpop.LpOptions) == ctypes.sizeof(o)


def _args(lp):
    return (lp.m, lp.n, lp.row_ptr, lp.col_idx, lp.val, lp.b, lp.c, lp.lb, lp.ub, lp.sense)


def _expect(code, lp, opts=None):
    with pytest.raises(lpop.LpError) as ei:
        lpop.lp_create(*_args(lp), opts)
    assert ei.value.code == code, str(ei.value)
    return str(ei.value)


@pytest.mark.parametrize("what", ["b_nan", "c_inf", "val_nan", "col_range", "rowptr_order", "sense",
                                  "lb_gt_ub", "lb_plus_inf", "ub_minus_inf", "rowptr_end"])
def test_invalid_input_is_rejected_on_the_host(lib, what):
    lp = lpgen.mixed_small(0, m=12, n=20)
    lp.b = lp.b.copy(); lp.c = lp.c.copy(); lp.val = lp.val.copy(); lp.col_idx = lp.col_idx.copy()
    lp.row_ptr = lp.row_ptr.copy(); lp.sense = lp.sense.copy(); lp.lb = lp.lb.copy(); lp.ub = lp.ub.copy()
    if what == "b_nan":
        lp.b[3] = math.nan
    elif what == "c_inf":
        lp.c[0] = math.inf
    elif what == "val_nan":
        lp.val[1] = math.nan
    elif what == "col_range":
        lp.col_idx[2] = lp.n
    elif what == "rowptr_order":
        i = int(np.argmax(np.diff(lp.row_ptr) > 0))
        lp.row_ptr[i + 1] = lp.row_ptr[i] - 1 if lp.row_ptr[i] > 0 else lp.row_ptr[i + 2] + 1
    elif what == "sense":
        lp.sense[0] = ord("X")
    elif what == "lb_gt_ub":
        lp.lb[0], lp.ub[0] = 2.0, 1.0
    elif what == "lb_plus_inf":
        lp.lb[1] = math.inf
    elif what == "ub_minus_inf":
        lp.ub[1] = -math.inf
    elif what == "rowptr_end":
        lp.row_ptr[-1] -= 1
        lp.col_idx = lp.col_idx[:-1]
        lp.val = lp.val[:-1]
    _expect(lpop.LP_ERR_INVALID_INPUT, lp)
    assert lpop.lp_last_error(None)


@pytest.mark.parametrize("field,value", [("mode", 7), ("scheduler", 5), ("alpha", -1.0), ("check_every", 0),
                                         ("check_every", (1 << 16) + 1),
                                         ("precond_floor", 0.0), ("pc_beta", 3.0), ("ruiz_iters", -1),
                                         ("kernel_timing", -1), ("device_alloc", 4096), ("device_free", 4096),
                                         ("refine_stall", 0), ("log_every", -1)])
def test_invalid_options_are_rejected(lib, field, value):
    lp = lpgen.mixed_small(0, m=12, n=20)
    opts = lpop.lp_options_default()
    setattr(opts, field, value)
    _expect(lpop.LP_ERR_INVALID_ARG, lp, opts)


def test_null_handle_calls_fail_cleanly(lib):
    assert lib.lp_solve(None, 1e-4, 10, None) == lpop.LP_ERR_INVALID_ARG
    assert lib.lp_result(None, None, None, None) == lpop.LP_ERR_INVALID_ARG
    assert lib.lp_reset(None) == lpop.LP_ERR_INVALID_ARG
    lib.lp_destroy(None)
    assert lib.lp_create(1, 1, 0, None, None, None, None, None, None, None, None, None, None) == lpop.LP_ERR_INVALID_ARG


def test_no_gpu_reports_cuda_error():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    lpbuild.build()
    lp = lpgen.mixed_small(0, m=12, n=20)
    _expect(lpop.LP_ERR_CUDA, lp)


@pytest.mark.parametrize("what", ["b_inf_two", "sense_two", "c_nan_then_bounds", "bounds_two"])
def test_large_vectors_name_the_first_offending_entry(lib, what):
    """The vector checks run over ranges on host threads (n = 200,000 here):
    with two offending entries in different ranges the first one is named."""
    lp = lpgen.transport(0)
    lp.b = lp.b.copy(); lp.c = lp.c.copy(); lp.sense = lp.sense.copy(); lp.lb = lp.lb.copy(); lp.ub = lp.ub.copy()
    m, n = lp.m, lp.n
    if what == "b_inf_two":
        lp.b[m - 3] = -math.inf
        lp.b[m // 2 + 1] = math.inf
        want = "b[%d] is not finite" % (m // 2 + 1)
    elif what == "sense_two":
        lp.sense[m - 1] = ord("x")
        lp.sense[7 * m // 8] = ord("l")
        want = "sense[%d] must be 'E', 'L' or 'G'" % (7 * m // 8)
    elif what == "c_nan_then_bounds":
        lp.c[3 * n // 4] = math.nan
        lp.lb[n // 3], lp.ub[n // 3] = 5.0, 4.0
        want = "bounds of variable %d are invalid" % (n // 3)
    else:
        lp.ub[n - 2] = -math.inf
        lp.lb[n // 5 + 3] = math.nan
        want = "bounds of variable %d are invalid" % (n // 5 + 3)
    msg = _expect(lpop.LP_ERR_INVALID_INPUT, lp)
    assert want in msg, msg


def test_large_valid_input_passes_the_host_checks():
    """A valid LP large enough for the threaded checks gets past every host
    check: without a GPU lp_create then fails at the device, not on input."""
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    lpbuild.build()
    lp = lpgen.transport(0)
    assert lp.n > 1 << 16
    _expect(lpop.LP_ERR_CUDA, lp)
