"""A debug build with every gather's index checked (liblpop_checked.so,
built with LPOP_CHECK_BOUNDS: an index outside the gathered vector is counted
and read as 0 instead of memory) runs the solves of the parity cases' shapes
-- sliced, paired, lane and whole-block rows, segmented rows, the power-law
columns, mixed precision -- and the batched kernel: no index falls outside
its vector, and every result equals the regular build's bit for bit (the
checks change no arithmetic).  Each build runs in a process of its own."""
import subprocess
import sys

import numpy as np
import pytest

from paper_2506_17650_gb300 import build as lpbuild
from tests.conftest import ROOT

pytestmark = pytest.mark.gpu

SCRIPT = r'''
import ctypes, sys
import numpy as np
root, lib, out = sys.argv[1:4]
sys.path.insert(0, root)
import lpgen
import paper_2506_17650_gb300 as lpop
lpop.load_library(lib)
raw = ctypes.CDLL(lib)
checked = hasattr(raw, "lpop_bad_gathers")
bad = 0

def count(p):
    if not checked:
        return 0
    c = ctypes.c_ulonglong(0)
    assert raw.lpop_bad_gathers(p.handle, ctypes.byref(c)) == 0
    return c.value

cases = {
    "tiny": (lpgen.tiny_random(0), dict(alpha=1e-3, phi=20)),
    "rowmix": (lpgen.row_length_mix(0), dict(alpha=1e-3, phi=20)),
    "long_rows": (lpgen.long_rows(0), dict(alpha=1e-3, phi=20)),
    "transport": (lpgen.transport(0, 2000, 2000, 16000), dict(alpha=1e-6, phi=20)),
    "powerlaw": (lpgen.powerlaw(0, 20000, 50000, 300000), dict(alpha=1e-6, phi=20)),
    "plain": (lpgen.tiny_random(2), dict(mode=lpop.LP_MODE_PLAIN, alpha=1e-3, phi=1)),
    "mixed": (lpgen.mixed_small(1), dict(alpha=1e-3, phi=20, precision=lpop.LP_PREC_MIXED)),
}
res = {}
for name, (lp, opts) in cases.items():
    with lpop.Problem(lp, **opts) as p:
        p.solve(0.0, 320)
        x, y, _ = p.result()
        bad += count(p)
    res[name + "_x"], res[name + "_y"] = x, y
probs = [lpop.Problem(lp, alpha=1e-3, phi=20) for lp in (lpgen.tiny_random(1), lpgen.row_length_mix(1))]
with lpop.Batch(probs) as b:
    b.solve(0.0, 320, 64)
for i, p in enumerate(probs):
    x, y, _ = p.result()
    res["batch%d_x" % i], res["batch%d_y" % i] = x, y
    bad += count(p)
    p.close()
np.savez(out, bad=np.int64(bad), checked=np.int64(checked), **res)
'''


def test_checked_build_reads_no_index_out_of_range_and_matches(tmp_path):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    libs = {"regular": lpbuild.build(), "checked": lpbuild.build(checked=True)}
    out = {}
    for name, lib in libs.items():
        path = str(tmp_path / f"{name}.npz")
        subprocess.run([sys.executable, "-c", SCRIPT, ROOT, lib, path], check=True, timeout=1800)
        out[name] = dict(np.load(path))
    assert int(out["checked"]["checked"]) == 1 and int(out["regular"]["checked"]) == 0
    assert int(out["checked"]["bad"]) == 0
    keys = [k for k in out["regular"] if k not in ("bad", "checked")]
    assert len(keys) == 18
    for k in keys:
        assert np.array_equal(out["regular"][k], out["checked"][k]), k
