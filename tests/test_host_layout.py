"""Host-side layout of a problem (csrc/host_layout.cpp), checked on the CPU.

tests/host_layout_runner.cpp runs the library's build_layout (and
segment_long_rows) on a CSR matrix; these tests check what it produced
against scipy.sparse and against the layout's own definition:

* prow / pcol are permutations, and the permuted CSR of A is exactly
  A[prow][:, pcol] with repeated entries summed and every row in increasing
  column order;
* the CSR of A^T is exactly the transpose of that matrix;
* the bins cover the rows contiguously, longest rows first, with the unit
  numbering and the sliced-copy offsets their rows imply;
* invalid input is rejected with the first offending index;
* segmentation cuts exactly the rows longer than the segment length;
* smaller sliced units renumber the units and change nothing else.
"""
import os
import shutil
import struct
import subprocess

import numpy as np
import pytest
import scipy.sparse as sp

import lpgen
from tests.conftest import ROOT

CSRC = os.path.join(ROOT, "paper_2506_17650_gb300", "csrc")
K_SEGMENTED, K_SELL, K_BLOCK = -1, -2, 256
K_SELL_MAX = 48  # rows of at most this many entries are sliced (kSellMaxLen of the layout)
K_PAIR_MAX = 2  # sliced rows of at most this many entries: units of two rows per thread (kPairMaxLen)


@pytest.fixture(scope="module")
def runner(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    out = str(tmp_path_factory.mktemp("layout") / "host_layout_runner")
    subprocess.run([gxx, "-O1", "-std=c++17", "-pthread", "-I", CSRC, os.path.join(ROOT, "tests", "host_layout_runner.cpp"),
                    os.path.join(CSRC, "host_layout.cpp"), "-o", out], check=True, capture_output=True)
    return out


class _Reader:
    def __init__(self, data):
        self.d, self.o = data, 0

    def take(self, fmt):
        v = struct.unpack_from(fmt, self.d, self.o)
        self.o += struct.calcsize(fmt)
        return v[0] if len(v) == 1 else v

    def vec(self, dtype):
        n = self.take("<q")
        a = np.frombuffer(self.d, dtype=dtype, count=n, offset=self.o).copy()
        self.o += n * np.dtype(dtype).itemsize
        return a

    def bins(self):
        nb, nu, seg_len, seg_rows = self.take("<iiii")
        rows = [self.take("<qqqqqq") for _ in range(nb)]
        return dict(nunits=nu, seg_len=seg_len, seg_rows=seg_rows, sliced=self.take("<q"),
                    bins=[dict(zip(("row_begin", "row_end", "width", "unit_begin", "len", "base"), r)) for r in rows])


def run_layout(runner, tmp_path, m, n, rp, ci, v, target=0, seg_len=0, sliced_rows=0):
    pre = str(tmp_path / "in_")
    np.asarray(rp, np.int64).tofile(pre + "rp.bin")
    np.asarray(ci, np.int32).tofile(pre + "ci.bin")
    np.asarray(v, np.float64).tofile(pre + "v.bin")
    out = str(tmp_path / "out.bin")
    extra = [str(sliced_rows)] if sliced_rows else []
    subprocess.run([runner, str(m), str(n), str(len(ci)), pre, out, str(target), str(seg_len), *extra], check=True)
    r = _Reader(open(out, "rb").read())
    rc = r.take("<i")
    n_err = r.take("<i")
    err = r.d[r.o:r.o + n_err].decode()
    r.o += n_err
    lay = dict(rc=rc, err=err, nnz=r.take("<q"), prow=r.vec(np.int32), pcol=r.vec(np.int32),
               A_rp=r.vec(np.int32), A_ci=r.vec(np.int32), A_v=r.vec(np.float64),
               At_rp=r.vec(np.int32), At_ci=r.vec(np.int32), At_v=r.vec(np.float64))
    lay["binsA"], lay["binsAt"] = r.bins(), r.bins()
    lay["segA"], lay["segAt"] = r.vec(np.int32), r.vec(np.int32)
    return lay


def rows_per_unit(width, length=None, sliced_rows=K_BLOCK):
    if width in (0, K_SEGMENTED):
        return 1
    if width == K_SELL and length is not None and length <= K_PAIR_MAX:
        return 2 * sliced_rows
    if width == K_SELL:
        return sliced_rows
    return K_BLOCK // width


def check_bins(bt, rp, rows, sliced_rows=K_BLOCK):
    lens = np.diff(rp)
    assert np.all(np.diff(lens) <= 0), "rows are not in non-increasing length order"
    at, unit, sliced = 0, 0, 0
    for b in bt["bins"]:
        assert b["row_begin"] == at and b["row_end"] > b["row_begin"]
        assert b["unit_begin"] == unit
        seg = lens[b["row_begin"]:b["row_end"]]
        w = b["width"]
        if w == K_SEGMENTED:
            nseg = int(np.sum((seg + bt["seg_len"] - 1) // bt["seg_len"]))
            unit += nseg
        else:
            unit += -(-(b["row_end"] - b["row_begin"]) // rows_per_unit(w, b["len"], sliced_rows))
        if w == K_SELL:
            assert np.all(seg == b["len"]) and 0 <= b["len"] <= K_SELL_MAX  # empty rows form a bin of length 0
            assert b["base"] == sliced
            sliced += -(-(b["row_end"] - b["row_begin"]) // 32) * 32 * b["len"]
        elif w == 0:
            assert np.all(seg > 2048)
        elif w != K_SEGMENTED:
            assert w in (1, 2, 4, 8, 16, 32)
        at = b["row_end"]
    assert at == rows and unit == bt["nunits"] and sliced == bt["sliced"]


def check_layout(lay, lp_m, lp_n, ref):
    """ref: the caller's matrix with repeated entries summed (scipy CSR)."""
    assert lay["rc"] == 0, lay["err"]
    m, n = lp_m, lp_n
    assert sorted(lay["prow"]) == list(range(m)) and sorted(lay["pcol"]) == list(range(n))
    A = sp.csr_matrix((lay["A_v"], lay["A_ci"], lay["A_rp"]), shape=(m, n))
    want = ref[lay["prow"]][:, lay["pcol"]].tocsr()
    want.sort_indices()
    assert lay["nnz"] == want.nnz == A.nnz
    assert np.array_equal(A.indptr, want.indptr) and np.array_equal(A.indices, want.indices)
    assert np.array_equal(A.data, want.data)
    for i in range(m):  # strictly increasing columns in every row
        assert np.all(np.diff(A.indices[A.indptr[i]:A.indptr[i + 1]]) > 0)
    At = sp.csr_matrix((lay["At_v"], lay["At_ci"], lay["At_rp"]), shape=(n, m))
    T = A.T.tocsr()
    T.sort_indices()
    assert np.array_equal(At.indptr, T.indptr) and np.array_equal(At.indices, T.indices)
    assert np.array_equal(At.data, T.data)
    check_bins(lay["binsA"], lay["A_rp"], m)
    check_bins(lay["binsAt"], lay["At_rp"], n)


def messy(lp, seed):
    """The same matrix with every row shuffled and some entries split into two
    exact halves (repeated entries that must be summed back)."""
    rng = np.random.default_rng(seed)
    ci, v, rp = [], [], [0]
    for i in range(lp.m):
        a, b = lp.row_ptr[i], lp.row_ptr[i + 1]
        c, x = list(lp.col_idx[a:b]), list(lp.val[a:b])
        if c:
            k = int(rng.integers(len(c)))
            x[k] = x[k] / 2
            c.append(c[k])
            x.append(x[k])
        p = rng.permutation(len(c))
        ci += [c[t] for t in p]
        v += [x[t] for t in p]
        rp.append(len(ci))
    return np.asarray(rp, np.int64), np.asarray(ci, np.int32), np.asarray(v, np.float64)


CASES = {
    "transport": lambda: lpgen.transport(0, 1500, 1500, 12000),
    "tiny": lambda: lpgen.tiny_random(0),
    "mixed": lambda: lpgen.mixed_small(1),
    "rowmix": lambda: lpgen.row_length_mix(0),
    "long_rows": lambda: lpgen.long_rows(0),
}


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("target", [0, 1 << 20])
def test_layout_is_the_permuted_matrix_and_its_transpose(runner, tmp_path, case, target):
    lp = CASES[case]()
    lay = run_layout(runner, tmp_path, lp.m, lp.n, lp.row_ptr, lp.col_idx, lp.val, target=target)
    check_layout(lay, lp.m, lp.n, lp.csr())


@pytest.mark.parametrize("case", ["transport", "rowmix", "long_rows"])
def test_shuffled_rows_and_repeated_entries_give_the_same_layout(runner, tmp_path, case):
    lp = CASES[case]()
    clean = run_layout(runner, tmp_path, lp.m, lp.n, lp.row_ptr, lp.col_idx, lp.val)
    rp, ci, v = messy(lp, 3)
    lay = run_layout(runner, tmp_path, lp.m, lp.n, rp, ci, v)
    ref = sp.csr_matrix((v, ci, rp), shape=(lp.m, lp.n))
    ref.sum_duplicates()
    check_layout(lay, lp.m, lp.n, ref)
    for key in ("prow", "pcol", "A_rp", "A_ci", "A_v", "At_rp", "At_ci", "At_v"):
        assert np.array_equal(lay[key], clean[key]), key


def test_segmentation_cuts_exactly_the_long_rows(runner, tmp_path):
    lp = lpgen.long_rows(0)
    seg_len = 4096
    lay = run_layout(runner, tmp_path, lp.m, lp.n, lp.row_ptr, lp.col_idx, lp.val, seg_len=seg_len)
    for rp_key, bt_key, seg_key in (("A_rp", "binsA", "segA"), ("At_rp", "binsAt", "segAt")):
        rp, bt, units = lay[rp_key], lay[bt_key], lay[seg_key].reshape(-1, 2)
        lens = np.diff(rp)
        long_rows = np.flatnonzero(lens > seg_len)
        assert bt["seg_rows"] == len(long_rows)
        if len(long_rows) == 0:
            assert len(units) == 0
            continue
        assert bt["bins"][0]["width"] == K_SEGMENTED and bt["seg_len"] == seg_len
        assert list(long_rows) == list(range(len(long_rows)))  # longest rows come first
        want = [(r, s) for r in long_rows for s in range(-(-lens[r] // seg_len))]
        assert [tuple(u) for u in units] == want
        check_bins(bt, rp, len(lens))


@pytest.mark.parametrize("what,expect", [
    ("col_high", "col_idx[7] out of range"),
    ("col_neg", "col_idx[7] out of range"),
    ("val_nan", "val[7] is not finite"),
    ("val_inf_then_col", "val[3] is not finite"),
    ("rowptr_dec", "row_ptr must be non-decreasing (row 2)"),
    ("rowptr_end", "row_ptr[0] must be 0 and row_ptr[m] must equal nnz"),
])
def test_invalid_input_names_the_first_offending_entry(runner, tmp_path, what, expect):
    lp = lpgen.mixed_small(0, m=12, n=20)
    rp, ci, v = lp.row_ptr.copy(), lp.col_idx.copy(), lp.val.copy()
    if what == "col_high":
        ci[7] = lp.n
        ci[9] = lp.n + 4
    elif what == "col_neg":
        ci[7] = -1
    elif what == "val_nan":
        v[7] = np.nan
        v[8] = np.inf
    elif what == "val_inf_then_col":
        v[3] = np.inf
        ci[5] = lp.n
    elif what == "rowptr_dec":
        rp[3] = rp[2] - 1
    elif what == "rowptr_end":
        rp[-1] += 1  # one more entry than the arrays hold
    lay = run_layout(runner, tmp_path, lp.m, lp.n, rp, ci, v)
    assert lay["rc"] < 0 and lay["err"] == expect


def run_validate(runner, tmp_path, m, n, rp, ci, v):
    pre = str(tmp_path / "val_")
    np.asarray(rp, np.int64).tofile(pre + "rp.bin")
    np.asarray(ci, np.int32).tofile(pre + "ci.bin")
    np.asarray(v, np.float64).tofile(pre + "v.bin")
    out = str(tmp_path / "val_out.bin")
    subprocess.run([runner, str(m), str(n), str(len(ci)), pre, out, "0", "0", "-1"], check=True)
    d = open(out, "rb").read()
    rc, n_err = np.frombuffer(d[:8], "<i4")
    err = d[8:8 + n_err].decode()
    return int(rc), err, bool(np.frombuffer(d[8 + n_err:12 + n_err], "<i4")[0])


def test_validation_on_host_threads_matches_its_definition(runner, tmp_path):
    """validate_csr on a matrix large enough to be split over host threads
    (>= 2^16 entries, many empty rows): the first entry with a column out of
    range or a non-finite value is the one named, the first decreasing row
    pointer is the one named, and the canonical flag (every row strictly
    increasing in column) is decided by the rows alone, whatever the columns
    on either side of a row start."""
    rng = np.random.default_rng(11)
    m, n = 60000, 5000
    lens = rng.integers(0, 9, m) * (rng.random(m) < 0.7)
    rows = [np.sort(rng.choice(n, size=k, replace=False)) for k in lens]
    rp = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    ci = np.concatenate(rows).astype(np.int32)
    v = rng.standard_normal(len(ci))
    nnz = len(ci)
    assert nnz >= 1 << 17
    starts = rp[1:-1][(rp[1:-1] > 0) & (rp[1:-1] < nnz)]
    assert np.any(ci[starts - 1] >= ci[starts])  # descents across row starts exist
    assert run_validate(runner, tmp_path, m, n, rp, ci, v) == (0, "", True)

    multi = np.flatnonzero(lens >= 2)
    for r in (multi[0], multi[len(multi) // 2], multi[-1]):  # one descent or one repeat in one row
        for kind in ("swap", "repeat"):
            c = ci.copy()
            k = rp[r]
            if kind == "swap":
                c[k], c[k + 1] = c[k + 1], c[k]
            else:
                c[k + 1] = c[k]
            assert run_validate(runner, tmp_path, m, n, rp, c, v) == (0, "", False), (r, kind)

    for ks, kv, want in (((nnz - 5, nnz // 2), (), "col_idx[%d] out of range" % (nnz // 2)),
                         ((nnz // 4 + 1,), (3 * nnz // 4,), "col_idx[%d] out of range" % (nnz // 4 + 1)),
                         ((nnz - 1,), (nnz // 3, nnz - 2), "val[%d] is not finite" % (nnz // 3))):
        c, w = ci.copy(), v.copy()
        for k in ks:
            c[k] = n if k % 2 else -7
        for k in kv:
            w[k] = np.inf if k % 2 else np.nan
        rc, err, _ = run_validate(runner, tmp_path, m, n, rp, c, w)
        assert rc < 0 and err == want

    p = rp.copy()
    nz = np.flatnonzero(lens > 0)
    r1, r2 = nz[len(nz) // 2], nz[-3]
    p[r1 + 1] = p[r1] - 1
    p[r2 + 1] = p[r2] - 1
    rc, err, _ = run_validate(runner, tmp_path, m, n, p, ci, v)
    assert rc < 0 and err == "row_ptr must be non-decreasing (row %d)" % r1


def test_empty_rows_and_no_constraints(runner, tmp_path):
    lay = run_layout(runner, tmp_path, 0, 5, [0], [], [])
    assert lay["rc"] == 0 and lay["nnz"] == 0 and sorted(lay["pcol"]) == list(range(5))
    lay = run_layout(runner, tmp_path, 4, 3, [0, 0, 2, 2, 3], [2, 0, 1], [1.0, 2.0, 3.0])
    check_layout(lay, 4, 3, sp.csr_matrix(([1.0, 2.0, 3.0], [2, 0, 1], [0, 0, 2, 2, 3]), shape=(4, 3)))


@pytest.mark.parametrize("case", ["long_rows", "transport"])
@pytest.mark.parametrize("rows", [224, 192, 128])
def test_smaller_sliced_units_renumber_only_the_units(runner, tmp_path, case, rows):
    """set_sliced_unit_rows: units of `rows` rows (of twice that for the bins
    of at most two entries per row, two rows per thread), a segmented bin
    keeping its units; every other field of the tables is unchanged, and
    back at 256 rows the tables are the default ones again."""
    lp = CASES[case]()
    args = (lp.m, lp.n, lp.row_ptr, lp.col_idx, lp.val)
    base = run_layout(runner, tmp_path, *args, seg_len=4096)
    lay = run_layout(runner, tmp_path, *args, seg_len=4096, sliced_rows=rows)
    back = run_layout(runner, tmp_path, *args, seg_len=4096, sliced_rows=K_BLOCK)
    sliced = 0
    for bt_key, rp_key in (("binsA", "A_rp"), ("binsAt", "At_rp")):
        check_bins(lay[bt_key], lay[rp_key], len(lay[rp_key]) - 1, sliced_rows=rows)
        assert back[bt_key] == base[bt_key]
        for b0, b1 in zip(base[bt_key]["bins"], lay[bt_key]["bins"]):
            assert {k: v for k, v in b0.items() if k != "unit_begin"} == {k: v for k, v in b1.items() if k != "unit_begin"}
            sliced += b0["width"] == K_SELL
        assert lay[bt_key]["nunits"] >= base[bt_key]["nunits"]
        assert lay[bt_key]["sliced"] == base[bt_key]["sliced"]
    assert sliced > 0
    for key in ("segA", "segAt"):
        assert np.array_equal(lay[key], base[key])
