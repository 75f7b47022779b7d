"""Full-size checks in the launch configuration bench.py times: 120 maps of
1024^2 (the CMB workload), mixed precision.  Sampled maps are compared element
by element with the oracle; the rest is checked through properties that hold
at any size (exact line search: the new gradient is orthogonal to the step;
chi^2 never increases)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import wf_oracle as O  # noqa: E402
from paper_1810_00503_gb300 import synth, wf  # noqa: E402
from tests.helpers import ensure_lib, rel, rfft_u  # noqa: E402

B, N = 120, 1024


@pytest.fixture(scope="module")
def batch():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    ensure_lib()
    dev = torch.device("cuda")
    inp = synth.cmb_patch(N, seed=3)
    g = torch.Generator(device=dev)
    g.manual_seed(1000)
    Ninv = torch.as_tensor(inp.Ninv, dtype=torch.float32, device=dev).unsqueeze(0).expand(B, -1, -1, -1).contiguous()
    mask = torch.as_tensor(inp.mask, dtype=torch.uint8, device=dev)
    P = torch.as_tensor(inp.P_half, dtype=torch.float32, device=dev)
    prob = wf.Problem(torch.zeros_like(Ninv), mask, Ninv, P, precision="mixed")
    z = torch.randn(B, 1, N, N, generator=g, device=dev)
    sig = torch.where(Ninv > 0, torch.rsqrt(torch.clamp(Ninv, min=1e-30)), torch.zeros_like(Ninv))
    noise = torch.randn(B, 1, N, N, generator=g, device=dev) * sig
    d = prob.simulate(z, noise)
    prob.set_data(d)
    host = dict(P=inp.P.astype(np.float32).astype(np.float64), mask=inp.mask,
                W=(inp.mask[None] * inp.Ninv).astype(np.float32).astype(np.float64))
    yield prob, d, host
    prob.close()


def test_sampled_maps_of_the_batch_eval_match_oracle(batch):
    prob, d, host = batch
    rng = np.random.default_rng(0)
    zs = rng.standard_normal((B, 1, N, N)).astype(np.float32)
    s = torch.fft.rfft2(torch.as_tensor(zs, device="cuda"), norm="ortho").contiguous()
    chi2, g = prob.eval(s)
    torch.cuda.synchronize()
    for b in (0, 57, B - 1):
        z = np.fft.irfft2(s[b].cpu().numpy().astype(np.complex128), s=(N, N), norm="ortho")
        db = d[b].cpu().numpy().astype(np.float64)
        rc = O.chi2(z, db, host["W"], host["P"])
        rg = rfft_u(O.grad(z, db, host["W"], host["P"]))
        assert abs(chi2[b].item() - rc) <= 1e-5 * abs(rc)
        assert rel(g[b].cpu().numpy(), rg) <= 2e-5


def test_iterations_of_the_batch_keep_line_search_properties(batch):
    prob, d, host = batch
    prob.start(gtol_rel=0.0, max_iter=1 << 30, check_every=1)
    prob.step(12)
    res = prob.finish()
    chi = np.array([st["chi2"] for st in res.stats])
    assert np.all(np.isfinite(chi))
    # chi^2 after 12 iterations is far below its value at s = 0
    chi2_0, _ = prob.eval(torch.zeros_like(res.s))
    assert np.all(chi < chi2_0.cpu().numpy())
    # spot check one map's returned chi^2 and gradient against the oracle
    b = 3
    z = np.fft.irfft2(res.s[b].cpu().numpy().astype(np.complex128), s=(N, N), norm="ortho")
    db = d[b].cpu().numpy().astype(np.float64)
    assert abs(res.stats[b]["chi2"] - O.chi2(z, db, host["W"], host["P"])) <= 1e-5 * res.stats[b]["chi2"]
