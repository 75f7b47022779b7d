"""The bounds-checked build (-DWF_DEBUG_BOUNDS, libwf_dbg.so): every shared
tile index of the FFT stages, their global spectrum, pixel and scratch
indices and the streaming kernels' vector indices are checked against their
buffers; a bad index is counted and redirected inside its buffer, so nothing
traps.  The checker's self-test must count its planted index, and tiny maps
(one and two channels, FP64 and mixed) through every operator entry point
and short solves under a covering set of FFT-stage variants must count none,
on square maps (n = 8..128) and rectangular ones of both aspects down to
8 x 1024 and 1024 x 8 strips.  The library is built here (a few minutes) and
run in a child process."""
import json
import os
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1810_00503_gb300 import build, wf  # noqa: E402
from tests.helpers import ensure_lib  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    ensure_lib()


def test_normal_build_has_no_bounds_checks():
    with pytest.raises(wf.WfError, match="not built with bounds checks"):
        wf.debug_bounds()


def test_bounds_checked_build_counts_nothing_on_every_variant():
    lib = build.build(debug_bounds=True)
    env = dict(os.environ, WF_LIB_PATH=lib)
    res = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "bounds_driver.py")], capture_output=True,
                         text=True, timeout=1800, cwd=ROOT, env=env)
    assert res.returncode == 0, res.stdout[-2000:] + res.stderr[-4000:]
    out = json.loads(res.stdout.strip().splitlines()[-1])
    assert out["lib"] == lib
    assert out["selftest"] == 1 and out["selftest_first"][3] == 4096, out
    assert out["violations"] == 0, out
    assert not out.get("solve_errors"), out["solve_errors"][:5]
    assert out["worst_grad_rel"] < 2e-5, out
    assert out["solves"] >= 36 * 44
