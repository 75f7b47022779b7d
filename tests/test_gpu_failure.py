"""Failure handling on the device without a GPU fault: a bounded wait of the
TMA-fed inverse column stage is made to run out (the copies of one map's tiles
are never issued), that map stops with WF_ETIMEOUT while the others carry on,
and the context stays usable for the next solve."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import wf_oracle as O  # noqa: E402
from paper_1810_00503_gb300 import synth, wf  # noqa: E402
from tests.helpers import ensure_lib, make_problem, rel, rfft_u  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    ensure_lib()


def test_wait_runs_out_then_context_is_usable():
    maps = [synth.density_small(64, seed=s) for s in (1, 2, 3, 4)]
    prob, host = make_problem(maps, "mixed")
    with pytest.raises(wf.WfError, match="ETIMEOUT") as ei:
        prob.solve(gtol_rel=1e-6, max_iter=300, refresh_every=64, inject_timeout_map=3,  # map 2
                   spin_limit=2_000_000)
    stats = ei.value.result.stats
    assert stats[2]["status"] == "WF_ETIMEOUT"
    assert all(s["status"] in ("WF_OK", "WF_ENOTCONVERGED") for b, s in enumerate(stats) if b != 2)
    # the stopped map keeps its last good state (here the start), with its true chi^2
    s2 = ei.value.result.s[2].cpu().numpy()
    assert np.all(np.isfinite(s2)) and np.isfinite(stats[2]["chi2"])
    # the same problem and context solve normally afterwards
    res = prob.solve(gtol_rel=1e-6, max_iter=3000, refresh_every=64)
    for b in range(4):
        assert res.stats[b]["status"] == "WF_OK"
        zs, _ = O.map_solve(host["d"][b], host["W"][b], host["P"][b], gtol_rel=1e-11, max_iter=5000)
        assert rel(res.s[b].cpu().numpy(), rfft_u(zs)) <= 1e-4


def test_bad_diagnostic_options_rejected():
    prob, _ = make_problem([synth.density_small(32, seed=1)], "mixed")
    with pytest.raises(wf.WfError, match="EINVAL"):
        prob.solve(max_iter=3, inject_timeout_map=5)
    with pytest.raises(wf.WfError, match="EINVAL"):
        prob.solve(max_iter=3, spin_limit=-1)
    with pytest.raises(wf.WfError, match="EINVAL"):  # the injected wait needs the TMA-fed stage
        prob.solve(max_iter=3, inject_timeout_map=1, fft_variant=2111)
