"""The convergence ring (wf_opts.history, wf_solver_history): per iteration k the
solver's chi^2 and |g|/|g0| as tracked on the device, the step and the
evaluation count.  On this quadratic objective with the exact line search
chi^2 decreases every iteration, the records are consecutive, and the last
one matches the solve's closing statistics."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1810_00503_gb300 import synth, wf  # noqa: E402
from tests.helpers import ensure_lib, make_problem  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    ensure_lib()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_history_records_every_iteration(precision):
    maps = [synth.density_small(64, seed=s) for s in (3, 4)]
    prob, _ = make_problem(maps, precision)
    cap = 4000
    res = prob.solve(gtol_rel=1e-8 if precision == "fp64" else 1e-5, max_iter=3000, history=cap)
    hist = prob.history(cap)
    for b in range(2):
        h, st = hist[b], res.stats[b]
        assert st["status"] == "WF_OK", st
        assert len(h) == st["iters"]
        assert np.array_equal(h[:, 0], np.arange(1, st["iters"] + 1))
        chi2 = h[:, 1]
        assert np.all(np.isfinite(chi2))
        # exact line search on a quadratic: chi2 never rises (to rounding of the line model)
        assert np.all(np.diff(chi2) <= 1e-9 * np.abs(chi2[:-1]))
        assert np.all(h[:, 3] > 0.0)                     # steps
        assert np.all(np.diff(h[:, 4]) >= 1)             # one evaluation per iteration at least
        # the tracked |g|/|g0| and chi2 of the last iteration agree with the closing true
        # evaluation; in the mixed path the tracked norm comes from dot products of FP32
        # vectors, so 1e-5 below |g0| it carries a relative error near FP32 eps |g0|^2 / |g|^2
        tol_g, tol_c = (1e-3, 1e-6) if precision == "fp64" else (2e-2, 1e-4)
        assert abs(h[-1, 2] - st["gnorm_rel"]) <= tol_g * st["gnorm_rel"] + 1e-12, (h[-1], st)
        assert abs(h[-1, 1] - st["chi2"]) <= tol_c * abs(st["chi2"]), (h[-1], st)


def test_history_ring_keeps_the_last_iterations():
    prob, _ = make_problem([synth.density_small(64, seed=5)], "fp64")
    cap = 10
    res = prob.solve(gtol_rel=1e-8, max_iter=3000, history=cap)
    k = res.stats[0]["iters"]
    assert k > cap
    h = prob.history(cap)[0]
    assert np.array_equal(h[:, 0], np.arange(k - cap + 1, k + 1))
    # a second solve on the same problem starts a new trace
    prob.solve(gtol_rel=1e-3, max_iter=3000, history=cap)
    h2 = prob.history(cap)[0]
    assert h2[0, 0] == max(1, h2[-1, 0] - cap + 1) and len(h2) <= cap


def test_history_options_checked():
    prob, _ = make_problem([synth.density_small(32, seed=1)], "fp64")
    with pytest.raises(wf.WfError, match="EINVAL"):
        prob.solve(max_iter=3, history=-1)
    prob2, _ = make_problem([synth.density_small(32, seed=2)], "fp64")
    prob2.solve(max_iter=3)
    with pytest.raises(wf.WfError, match="EINVAL"):  # no history was asked for
        prob2.history(4)
