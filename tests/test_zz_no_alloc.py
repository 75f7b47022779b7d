"""The allocation-free objective + gradient entry point (wf_eval_noalloc),
called through the C ABI, agrees with the regular wf_eval on two calls in a
row with different inputs.  Its scratch sits in a static device array shared
by all calls, so the second call also shows that the first call's leftovers
do not leak into its result.  This file is collected last on purpose."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import wf_oracle as O  # noqa: E402
from paper_1810_00503_gb300 import synth, wf  # noqa: E402
from tests.helpers import ensure_lib, make_problem, rel, rfft_u, to_dev  # noqa: E402

TOL = {"fp64": 1e-12, "mixed": 2e-5}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    ensure_lib()


def _case(n, C, B, seed, precision):
    inputs = [synth.density_small(n, seed=seed + b) if C == 1 else synth.shear_eb(n, seed=seed)
              for b in range(B)]
    prob, host = make_problem(inputs, precision, shared_P=True)
    wdt = torch.float64 if precision == "fp64" else torch.float32
    cdt = torch.complex128 if precision == "fp64" else torch.complex64
    d = to_dev(np.stack([dd * m[None] for dd, m in zip(host["d"], host["mask"])]), wdt)
    w = to_dev(np.stack(host["W"]), wdt)
    P = to_dev(host["P"][0][..., : n // 2 + 1], wdt)
    S = np.stack([rfft_u(synth.random_state(n, C, seed=seed + 50 + b)) for b in range(B)])
    s = to_dev(S, cdt)
    return prob, s, d, w, P


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_noalloc_matches_wf_eval_on_two_calls(precision):
    cases = [_case(256, 1, 2, 11, precision), _case(64, 2, 1, 23, precision)]
    for prob, s, d, w, P in cases:
        ref_c, ref_g = prob.eval(s)
        c, g = wf.eval_noalloc(s, d, w, P)
        torch.cuda.synchronize()
        assert rel(g.cpu().numpy(), ref_g.cpu().numpy()) <= TOL[precision]
        assert np.allclose(c.cpu().numpy(), ref_c.cpu().numpy(), rtol=TOL[precision], atol=0)


def test_noalloc_rejects_batches_beyond_its_scratch():
    dt = torch.float64
    n, C, B = 1024, 2, 1
    s = torch.zeros((B, C, n, n // 2 + 1), dtype=torch.complex128, device="cuda")
    d = torch.zeros((B, C, n, n), dtype=dt, device="cuda")
    P = torch.zeros((C, n, n // 2 + 1), dtype=dt, device="cuda")
    with pytest.raises(wf.WfError, match="EINVAL.*static"):
        wf.eval_noalloc(s, d, d, P)
