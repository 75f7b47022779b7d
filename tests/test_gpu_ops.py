"""GPU parity of the single-pass operator calls (objective + gradient,
Hessian-vector product, signal map, data synthesis, band energies) against the
FP64 oracle, element by element, through the C ABI.

Tolerances (relative L2 over the whole output unless stated):
* FP64 path: 1e-12.  FFT round-off is O(eps log n) ~ 1e-15; the margin covers
  the residual d - Ax, which cancels when the state fits the data.
* Mixed path (FP32 fields, FP64 sums): 2e-5 for fields (FP32 eps 6e-8 times
  log2(n^2) <= 20 FFT stages and the same cancellation), 1e-5 for chi^2.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import wf_oracle as O  # noqa: E402
from paper_1810_00503_gb300 import synth  # noqa: E402
from tests.helpers import ensure_lib, make_problem, rel, rfft_u, to_dev  # noqa: E402

TOL = {"fp64": dict(field=1e-12, chi2=1e-12), "mixed": dict(field=2e-5, chi2=1e-5)}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    ensure_lib()


def _inputs(n, C, B, seed):
    if C == 1:
        return [synth.density_small(n, seed=seed + b) for b in range(B)]
    return [synth.shear_eb(n, seed=seed + b) for b in range(B)]


def _spec_t(fields, precision):
    cdt = torch.complex128 if precision == "fp64" else torch.complex64
    npc = np.complex128 if precision == "fp64" else np.complex64
    S = np.stack([rfft_u(f) for f in fields]).astype(npc)
    return to_dev(S, cdt), [np.fft.irfft2(s.astype(np.complex128), s=f.shape[-2:], norm="ortho")
                           for s, f in zip(S, fields)]


CASES = [(8, 1, 1, "fp64"), (16, 2, 2, "fp64"), (32, 1, 3, "fp64"), (64, 2, 1, "fp64"),
         (128, 1, 2, "fp64"), (256, 1, 1, "fp64"), (512, 2, 1, "fp64"), (1024, 1, 1, "fp64"),
         (32, 1, 2, "mixed"), (128, 2, 1, "mixed"), (256, 1, 2, "mixed"), (1024, 2, 1, "mixed")]


@pytest.mark.parametrize("n,C,B,precision", CASES)
def test_eval_matches_oracle(n, C, B, precision):
    inputs = _inputs(n, C, B, seed=100 + n)
    prob, host = make_problem(inputs, precision, shared_P=(C == 1 and B % 2 == 1))
    fields = [synth.random_state(n, C, seed=7 + b) for b in range(B)]
    s, zs = _spec_t(fields, precision)
    chi2, g = prob.eval(s)
    torch.cuda.synchronize()
    tol = TOL[precision]
    for b in range(B):
        z = zs[b]
        rc = O.chi2(z, host["d"][b], host["W"][b], host["P"][b])
        rg = rfft_u(O.grad(z, host["d"][b], host["W"][b], host["P"][b]))
        assert abs(chi2[b].item() - rc) <= tol["chi2"] * abs(rc), (b, chi2[b].item(), rc)
        assert rel(g[b].cpu().numpy(), rg) <= tol["field"], b


@pytest.mark.parametrize("n,C,precision", [(16, 1, "fp64"), (64, 2, "fp64"), (256, 1, "mixed"),
                                           (512, 2, "mixed")])
def test_hess_vec_and_signal_map(n, C, precision):
    inputs = _inputs(n, C, 1, seed=5)
    prob, host = make_problem(inputs, precision)
    v = synth.random_state(n, C, seed=3)
    s, zs = _spec_t([v], precision)
    hv = prob.hess_vec(s)
    x = prob.signal_map(s)
    torch.cuda.synchronize()
    tol = TOL[precision]["field"]
    assert rel(hv[0].cpu().numpy(), rfft_u(O.hess_vec(zs[0], host["W"][0], host["P"][0]))) <= tol
    assert rel(x[0].cpu().numpy(), O.apply_A(zs[0], host["P"][0])) <= tol


@pytest.mark.parametrize("n,C,precision", [(32, 1, "fp64"), (64, 2, "fp64"), (1024, 1, "mixed")])
def test_simulate_data_matches_oracle(n, C, precision):
    inputs = _inputs(n, C, 2, seed=9)
    prob, host = make_problem(inputs, precision)
    wdt = torch.float64 if precision == "fp64" else torch.float32
    npdt = np.float64 if precision == "fp64" else np.float32
    z = np.stack([i.z for i in inputs]).astype(npdt)
    nz = np.stack([i.noise for i in inputs]).astype(npdt)
    out = prob.simulate(to_dev(z, wdt), to_dev(nz, wdt))
    torch.cuda.synchronize()
    for b in range(2):
        ref = O.synthesize_data(z[b].astype(np.float64), nz[b].astype(np.float64), host["mask"][b],
                                host["P"][0])
        assert rel(out[b].cpu().numpy(), ref) <= TOL[precision]["field"]


def test_band_energy_matches_oracle():
    n, nb = 64, 6
    inputs = _inputs(n, 1, 2, seed=4)
    prob, host = make_problem(inputs, "fp64")
    bands = synth.log_bands(n, nb)
    theta = O.theta_fid(host["P"][0], bands, nb)
    fields = [synth.random_state(n, 1, seed=b) for b in range(2)]
    s, zs = _spec_t(fields, "fp64")
    E = prob.band_energy(s, to_dev(bands[..., : n // 2 + 1], torch.int16),
                         to_dev(theta, torch.float64))
    torch.cuda.synchronize()
    for b in range(2):
        ref = O.band_E(zs[b], bands, theta, nb)
        assert np.allclose(E[b].cpu().numpy(), ref, rtol=1e-12, atol=0)


def test_bad_inputs_rejected():
    from paper_1810_00503_gb300 import wf
    inp = synth.density_small(16, seed=1)
    P = inp.P.copy(); P[0, 1, 1] = -1.0
    dt = torch.float64
    d = to_dev(inp.z[None], dt)
    with pytest.raises(wf.WfError, match="EINVAL"):
        wf.Problem(d, to_dev(inp.mask, torch.uint8), to_dev(inp.Ninv[None], dt),
                   to_dev(P[..., :9], dt))
    Ninv = inp.Ninv.copy(); Ninv[0, 2, 2] = np.nan
    with pytest.raises(wf.WfError, match="ENONFINITE"):
        wf.Problem(d, to_dev(inp.mask, torch.uint8), to_dev(Ninv[None], dt),
                   to_dev(inp.P[..., :9], dt))
    with pytest.raises(wf.WfError, match="EINVAL"):
        wf.Problem(d[..., :12, :12].contiguous(), to_dev(inp.mask[:12, :12], torch.uint8),
                   to_dev(inp.Ninv[None, :, :12, :12], dt), to_dev(inp.P[..., :12, :7], dt))
