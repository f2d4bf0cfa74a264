"""The layout lp_create builds on the device (csrc/device_layout.cu) against the
host's build_layout (csrc/host_layout.cpp, checked against scipy on the CPU
by tests/test_host_layout.py).

tests/device_layout_runner.cu and tests/host_layout_runner.cpp run the two
on the same CSR input; their outputs must be identical byte for byte: both
permutations, both permuted CSR copies, the bin tables and the segmentation.
Inputs: the generators' shapes (power-law columns longer than the counting
range, whole-block and segmented rows included), shuffled rows with repeated
entries, empty rows, no constraints, and the widened layouts.  The device
runner also reports the first rows of at most 32 entries, the device copies
of the permutations and the permuted copies of b, c, lb, ub and the senses,
checked here against the host layout.
"""
import os
import shutil
import subprocess

import numpy as np
import pytest

import lpgen
from tests.conftest import ROOT
from tests.test_host_layout import CASES, _Reader, check_layout, messy

pytestmark = pytest.mark.gpu

CSRC = os.path.join(ROOT, "paper_2506_17650_gb300", "csrc")
INCLUDE = os.path.join(ROOT, "include")


@pytest.fixture(scope="module")
def runners(tmp_path_factory):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    gxx, nvcc = shutil.which("g++"), shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if gxx is None or not os.path.exists(nvcc):
        pytest.skip("g++ or nvcc not available")
    d = tmp_path_factory.mktemp("device_layout")
    host, dev = str(d / "host_layout_runner"), str(d / "device_layout_runner")
    subprocess.run([gxx, "-O1", "-std=c++17", "-pthread", "-I", CSRC, os.path.join(ROOT, "tests", "host_layout_runner.cpp"),
                    os.path.join(CSRC, "host_layout.cpp"), "-o", host], check=True, capture_output=True)
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O2", "-std=c++17", "--expt-relaxed-constexpr",
                    "-Xcompiler", "-pthread", "-I", CSRC, "-I", INCLUDE, os.path.join(ROOT, "tests", "device_layout_runner.cu"),
                    os.path.join(CSRC, "device_layout.cu"), os.path.join(CSRC, "host_layout.cpp"), "-o", dev],
                   check=True, capture_output=True)
    return host, dev


def run_both(runners, tmp_path, m, n, rp, ci, v, target=0, seg_len=0):
    pre = str(tmp_path / "in_")
    np.asarray(rp, np.int64).tofile(pre + "rp.bin")
    np.asarray(ci, np.int32).tofile(pre + "ci.bin")
    np.asarray(v, np.float64).tofile(pre + "v.bin")
    outs = []
    for runner, name in zip(runners, ("host.bin", "device.bin")):
        out = str(tmp_path / name)
        subprocess.run([runner, str(m), str(n), str(len(ci)), pre, out, str(target), str(seg_len)], check=True)
        outs.append(open(out, "rb").read())
    host, dev = outs
    assert len(dev) > len(host) and dev[:len(host)] == host, "device layout differs from the host layout"
    r = _Reader(host)
    rc = r.take("<i")
    n_err = r.take("<i")
    r.o += n_err
    lay = dict(rc=rc, err="", nnz=r.take("<q"), prow=r.vec(np.int32), pcol=r.vec(np.int32),
               A_rp=r.vec(np.int32), A_ci=r.vec(np.int32), A_v=r.vec(np.float64),
               At_rp=r.vec(np.int32), At_ci=r.vec(np.int32), At_v=r.vec(np.float64))
    lay["binsA"], lay["binsAt"] = r.bins(), r.bins()
    lay["segA"], lay["segAt"] = r.vec(np.int32), r.vec(np.int32)
    assert r.o == len(host)
    x = _Reader(dev)
    x.o = len(host)
    extra = dict(split=(x.take("<i"), x.take("<i")), prow=x.vec(np.int32), pcol=x.vec(np.int32), b=x.vec(np.float64),
                 sense=x.vec(np.uint8), c=x.vec(np.float64), l=x.vec(np.float64), u=x.vec(np.float64))
    return lay, extra


def check_extra(lay, extra, m, n):
    for which, (rp, rows) in enumerate(((lay["A_rp"], m), (lay["At_rp"], n))):
        short = np.flatnonzero(np.diff(rp) <= 32)
        assert extra["split"][which] == (short[0] if len(short) else rows)
    i, j = lay["prow"], lay["pcol"]
    assert np.array_equal(extra["prow"], i) and np.array_equal(extra["pcol"], j)  # the device copies kept
    assert np.array_equal(extra["b"], i + 0.5)
    assert np.array_equal(extra["sense"], i % 3)  # E, L, G -> 0, 1, 2
    assert np.array_equal(extra["c"], -1.0 - j)
    assert np.array_equal(extra["l"], 2.0 * j) and np.array_equal(extra["u"], 2.0 * j + 1.0)


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("target", [0, 1 << 20])
def test_device_layout_equals_host_layout(runners, tmp_path, case, target):
    lp = CASES[case]()
    seg_len = 4096 if case == "long_rows" else 0
    lay, extra = run_both(runners, tmp_path, lp.m, lp.n, lp.row_ptr, lp.col_idx, lp.val, target=target, seg_len=seg_len)
    check_layout(lay, lp.m, lp.n, lp.csr())
    check_extra(lay, extra, lp.m, lp.n)


@pytest.mark.parametrize("scale", [0.01, 0.1])
def test_device_layout_of_the_power_law_lp(runners, tmp_path, scale):
    """Columns of up to ~1e5 entries: order keys beyond the counting range,
    whole-block and segmented rows of A^T."""
    lp = lpgen.powerlaw(0, int(2_000_000 * scale), int(5_000_000 * scale), int(30_000_000 * scale))
    lay, extra = run_both(runners, tmp_path, lp.m, lp.n, lp.row_ptr, lp.col_idx, lp.val, seg_len=8192)
    assert lay["rc"] == 0 and lay["nnz"] == lp.nnz
    assert lay["binsAt"]["bins"][0]["width"] in (0, -1)  # the heaviest columns take whole blocks
    if scale == 0.1:
        assert np.diff(lay["At_rp"]).max() > 4096 and lay["binsAt"]["seg_rows"] > 0
    check_extra(lay, extra, lp.m, lp.n)


@pytest.mark.parametrize("case", ["transport", "rowmix", "long_rows"])
def test_device_layout_of_shuffled_rows_with_repeated_entries(runners, tmp_path, case):
    lp = CASES[case]()
    rp, ci, v = messy(lp, 3)
    lay, extra = run_both(runners, tmp_path, lp.m, lp.n, rp, ci, v)
    assert lay["rc"] == 0 and lay["nnz"] == lp.nnz
    check_extra(lay, extra, lp.m, lp.n)


def test_device_layout_of_empty_rows_and_no_constraints(runners, tmp_path):
    lay, extra = run_both(runners, tmp_path, 0, 5, [0], [], [])
    assert lay["rc"] == 0 and lay["nnz"] == 0
    check_extra(lay, extra, 0, 5)
    lay, extra = run_both(runners, tmp_path, 4, 3, [0, 0, 2, 2, 3], [2, 0, 1], [1.0, 2.0, 3.0])
    assert lay["rc"] == 0 and lay["nnz"] == 3
    check_extra(lay, extra, 4, 3)
    # one column, every row the same length (a single class: the sort is a stable copy)
    m = 3000
    lay, extra = run_both(runners, tmp_path, m, 1, np.arange(m + 1), np.zeros(m, np.int32), np.arange(m) + 1.0)
    assert list(lay["prow"]) == list(range(m)) and list(lay["At_ci"]) == list(range(m))
    check_extra(lay, extra, m, 1)
