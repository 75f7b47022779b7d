"""The C-ABI library loads on a machine without a GPU and exports every entry
point declared in include/wf.h; host-only calls behave as documented."""
import ctypes
import os
import re

from paper_1810_00503_gb300 import wf
from tests.helpers import ensure_lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "wf.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b((?:wf|bandpower)_[a-z_0-9]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    L = ensure_lib()
    names = declared_symbols()
    assert names, "no declarations found"
    for name in names:
        assert hasattr(L, name), f"{name} declared in wf.h but not exported"
    assert sorted(wf.EXPORTS) == names


def test_opts_default_and_last_error_need_no_gpu():
    L = ensure_lib()
    o = wf.WfOpts()
    L.wf_opts_default(ctypes.byref(o))
    assert (o.lbfgs_m, o.max_iter, o.gtol_rel, o.check_every, o.use_graphs) == (10, 10000, 1e-6, 16, 1)
    assert isinstance(L.wf_last_error(), bytes)


def test_null_arguments_are_rejected_without_touching_the_device():
    L = ensure_lib()
    assert L.wf_create(None) == 1
    assert b"null" in L.wf_last_error()
    out = ctypes.c_void_p()
    # null handle is rejected before any CUDA call
    assert L.wf_problem_create(None, None, 1, 32, 1, 1, 0, 10, None, ctypes.byref(out)) == 1
    assert L.wf_eval(None, None, None, None, None) == 1
