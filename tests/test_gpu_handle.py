"""The handle's workspace: every device allocation of its problems and solvers
is charged to it, released on destroy, and refused beyond workspace_limit."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1810_00503_gb300 import synth, wf  # noqa: E402
from tests.helpers import ensure_lib, to_dev  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    ensure_lib()


def _inputs(n, B=1):
    inp = synth.density_small(n, seed=2)
    dt = torch.float32
    d = to_dev(np.stack([inp.noise] * B), dt)
    N = to_dev(np.stack([inp.Ninv] * B), dt)
    M = to_dev(inp.mask, torch.uint8)
    P = to_dev(inp.P[..., : n // 2 + 1], dt)
    return d, M, N, P


def test_workspace_is_charged_and_released():
    h = wf.Handle()
    base = h.workspace_used()
    assert base >= 264 * 1024  # twiddle tables in FP64 and FP32
    prob = wf.Problem(*_inputs(64, B=2), precision="mixed", handle=h)
    with_problem = h.workspace_used()
    assert with_problem - base >= 3 * 2 * 64 * 64 * 4  # data, weights, scratch
    prob.solve(max_iter=3, gtol_rel=0.0)
    # the solver's state, gradient and 2m history vectors are charged too
    assert h.workspace_used() - with_problem >= (2 + 2 * 10) * 2 * 64 * 32 * 8
    prob.close()
    assert h.workspace_used() == base
    h.close()


def test_workspace_limit_refuses_and_leaves_no_trace():
    h0 = wf.Handle()
    base = h0.workspace_used()
    h0.close()
    h = wf.Handle(workspace_limit=base + 256 * 1024)
    small = wf.Problem(*_inputs(32), precision="mixed", handle=h)
    used = h.workspace_used()
    with pytest.raises(wf.WfError, match="ENOMEM"):
        wf.Problem(*_inputs(256), precision="mixed", handle=h)
    assert h.workspace_used() == used
    with pytest.raises(wf.WfError, match="ENOMEM"):
        small.solve(max_iter=2, gtol_rel=0.0, lbfgs_m=32)  # history does not fit
    small.close()
    assert h.workspace_used() == base
    h.close()
