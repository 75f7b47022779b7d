"""Band-amplitude derivatives from the adjoint stage (wf_eval_bands) against
the oracle, and the torch.autograd.Function against central finite
differences on random directions (Hermitian-consistent for s)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import wf_oracle as O  # noqa: E402
from paper_1810_00503_gb300 import synth  # noqa: E402
from tests.helpers import ensure_lib, make_problem, rel, rfft_u, to_dev  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    ensure_lib()


@pytest.mark.parametrize("n,C", [(32, 1), (64, 2), (256, 1)])
def test_eval_bands_matches_oracle(n, C):
    nb = 4
    inp = synth.density_small(n, seed=12) if C == 1 else synth.shear_eb(n, seed=12)
    prob, host = make_problem([inp], "fp64")
    bands = synth.log_bands(n, nb, C=C)
    nbt = nb * C
    band_t = to_dev(bands[..., : n // 2 + 1], torch.int16)
    rng = np.random.default_rng(1)
    q = rng.uniform(0.5, 2.0, size=nbt)
    prob.set_band_scale(band_t, to_dev(q, torch.float64))
    Pq = host["P"][0] * np.where(bands >= 0, q[np.maximum(bands, 0)], 1.0)
    z = synth.random_state(n, C, seed=2)
    s = to_dev(rfft_u(z)[None], torch.complex128)
    chi2, g, dq = prob.eval_bands(s, band_t, nbt)
    torch.cuda.synchronize()
    ref = O.chi2_dlogq(z, host["d"][0], host["W"][0], Pq, bands, nbt)
    assert np.allclose(dq[0].cpu().numpy(), ref, rtol=1e-10, atol=1e-10 * np.abs(ref).max())
    assert abs(chi2[0].item() - O.chi2(z, host["d"][0], host["W"][0], Pq)) <= 1e-12 * chi2[0].item()
    assert rel(g[0].cpu().numpy(), rfft_u(O.grad(z, host["d"][0], host["W"][0], Pq))) <= 1e-12


def test_autograd_function_matches_finite_differences():
    from paper_1810_00503_gb300.autograd import chi2 as wf_chi2
    n, nb = 64, 5
    inp = synth.density_small(n, seed=3)
    prob, host = make_problem([inp], "fp64")
    bands = synth.log_bands(n, nb)
    band_t = to_dev(bands[..., : n // 2 + 1], torch.int16)
    rng = np.random.default_rng(9)
    s = to_dev(rfft_u(synth.random_state(n, 1, seed=5))[None], torch.complex128).requires_grad_(True)
    q = to_dev(rng.uniform(0.5, 1.5, size=nb), torch.float64).requires_grad_(True)
    f = wf_chi2(s, q, prob, band_t).sum()
    f.backward()
    gs, gq = s.grad.clone(), q.grad.clone()
    h = 1e-4
    with torch.no_grad():
        for k in range(20):
            dirs = to_dev(rfft_u(np.random.default_rng(100 + k).standard_normal((1, n, n)))[None],
                          torch.complex128)
            dq = to_dev(np.random.default_rng(200 + k).standard_normal(nb), torch.float64)
            fp = wf_chi2(s + h * dirs, q + h * dq, prob, band_t).sum().item()
            fm = wf_chi2(s - h * dirs, q - h * dq, prob, band_t).sum().item()
            fd = (fp - fm) / (2 * h)
            an = float((gs.real * dirs.real + gs.imag * dirs.imag).sum() + (gq * dq).sum())
            assert abs(fd - an) <= 1e-6 * abs(f.item()) / 1e3 + 1e-6 * abs(an), (k, fd, an)


def test_autograd_eb_512_on_1000_random_directions():
    """Joint E/B shear at 512^2: the adjoint stage behind the autograd Function
    against central differences along 1000 random directions in (s, q), the s
    part Hermitian-consistent (spectra of real fields).  chi^2 is quadratic in
    s, so along s the differences are exact up to rounding; along q they carry
    an O(h^2) term."""
    from paper_1810_00503_gb300.autograd import chi2 as wf_chi2
    n, nb = 512, 4
    inp = synth.shear_eb(n, seed=21)
    prob, _ = make_problem([inp], "fp64")
    bands = synth.log_bands(n, nb, C=2)
    band_t = to_dev(bands[..., : n // 2 + 1], torch.int16)
    g = torch.Generator(device="cuda")
    g.manual_seed(5)
    s0 = torch.fft.rfft2(torch.randn(1, 2, n, n, generator=g, device="cuda", dtype=torch.float64), norm="ortho")
    s = s0.clone().requires_grad_(True)
    q = (0.5 + torch.rand(2 * nb, generator=g, device="cuda", dtype=torch.float64)).requires_grad_(True)
    f = wf_chi2(s, q, prob, band_t).sum()
    f.backward()
    gs, gq = s.grad.clone(), q.grad.clone()
    h, worst = 1e-4, 0.0
    with torch.no_grad():
        for k in range(1000):
            dirs = torch.fft.rfft2(torch.randn(1, 2, n, n, generator=g, device="cuda", dtype=torch.float64),
                                   norm="ortho")
            dq = torch.randn(2 * nb, generator=g, device="cuda", dtype=torch.float64)
            fp = wf_chi2(s0 + h * dirs, q + h * dq, prob, band_t).sum().item()
            fm = wf_chi2(s0 - h * dirs, q - h * dq, prob, band_t).sum().item()
            fd = (fp - fm) / (2 * h)
            an = float((gs.real * dirs.real + gs.imag * dirs.imag).sum() + (gq * dq).sum())
            err = abs(fd - an) / (1e-6 * abs(f.item()) / 1e3 + 1e-6 * abs(an))
            worst = max(worst, err)
    assert worst <= 1.0, worst


def _fd_check(prob, band_t, nbt, s0, q0, n_dir, g, h_s, h_q):
    """Central differences of the autograd Function along random directions:
    s-directions (Hermitian-consistent) with step h_s, where chi^2 is exactly
    quadratic, and q-directions with step h_q.  Returns the worst error in
    units of the FP32-field tolerance 1e-6 |chi2| / h (plus 1e-5 of the
    directional derivative)."""
    from paper_1810_00503_gb300.autograd import chi2 as wf_chi2
    B, C, n = s0.shape[0], s0.shape[1], s0.shape[2]
    s = s0.clone().requires_grad_(True)
    q = q0.clone().requires_grad_(True)
    f = wf_chi2(s, q, prob, band_t).sum()
    f.backward()
    gs, gq = s.grad.clone(), q.grad.clone()
    fv = abs(f.item())
    worst = 0.0
    with torch.no_grad():
        for k in range(n_dir):
            if k % 2 == 0:
                h = h_s
                dirs = torch.fft.rfft2(torch.randn(B, C, n, n, generator=g, device="cuda", dtype=torch.float32),
                                       norm="ortho")
                dq = torch.zeros_like(q0)
            else:
                h = h_q
                dirs = torch.zeros_like(s0)
                dq = torch.randn(nbt, generator=g, device="cuda", dtype=torch.float64)
            fp = wf_chi2(s0 + h * dirs, q0 + h * dq, prob, band_t).sum().item()
            fm = wf_chi2(s0 - h * dirs, q0 - h * dq, prob, band_t).sum().item()
            fd = (fp - fm) / (2 * h)
            an = float((gs.real.double() * dirs.real.double() + gs.imag.double() * dirs.imag.double()).sum()
                       + (gq * dq).sum())
            worst = max(worst, abs(fd - an) / (1e-6 * fv / h + 1e-5 * abs(an)))
    return worst


def test_autograd_mixed_eb_512_on_1000_random_directions():
    """The FP32-field path (mixed precision) of the joint E/B 512^2 workload:
    the adjoint behind the autograd Function against central differences on
    1000 random directions, at the FP32 tolerance 1e-6 |chi2| / h."""
    n, nb = 512, 4
    inp = synth.shear_eb(n, seed=21)
    prob, _ = make_problem([inp], "mixed")
    bands = synth.log_bands(n, nb, C=2)
    band_t = to_dev(bands[..., : n // 2 + 1], torch.int16)
    g = torch.Generator(device="cuda")
    g.manual_seed(6)
    s0 = torch.fft.rfft2(torch.randn(1, 2, n, n, generator=g, device="cuda"), norm="ortho")
    q0 = 0.5 + torch.rand(2 * nb, generator=g, device="cuda", dtype=torch.float64)
    worst = _fd_check(prob, band_t, 2 * nb, s0, q0, 1000, g, h_s=0.5, h_q=1e-3)
    assert worst <= 1.0, worst


def test_autograd_mixed_cmb_1024_recomputes_and_matches_oracle():
    """One 1024^2 CMB map in mixed precision: the forward pass keeps only the
    gradient and the band derivatives (no stored intermediates; every
    backward input is recomputed by one fused pass).  Its band derivatives and
    gradient match the oracle's, and the autograd Function matches central
    differences on 200 random directions."""
    n, nb = 1024, 10
    inp = synth.cmb_patch(n, seed=3)
    prob, host = make_problem([inp], "mixed")
    bands = synth.log_bands(n, nb)
    band_t = to_dev(bands[..., : n // 2 + 1], torch.int16)
    rng = np.random.default_rng(4)
    q = rng.uniform(0.7, 1.4, size=nb)
    prob.set_band_scale(band_t, to_dev(q, torch.float64))
    sp32 = (np.sqrt(host["P"][0]) / n).astype(np.float32).astype(np.float64)
    Pq = (n * sp32) ** 2 * np.where(bands >= 0, q[np.maximum(bands, 0)], 1.0)
    z = synth.random_state(n, 1, seed=7).astype(np.float32).astype(np.float64)
    s = to_dev(rfft_u(z)[None], torch.complex64)
    chi2, gr, dq = prob.eval_bands(s, band_t, nb)
    torch.cuda.synchronize()
    zz = np.fft.irfft2(s[0].cpu().numpy().astype(np.complex128), s=(n, n), norm="ortho")
    ref = O.chi2_dlogq(zz, host["d"][0], host["W"][0], Pq, bands, nb)
    assert np.abs(dq[0].cpu().numpy() - ref).max() <= 2e-5 * np.abs(ref).max(), (dq, ref)
    assert abs(chi2[0].item() - O.chi2(zz, host["d"][0], host["W"][0], Pq)) <= 1e-5 * chi2[0].item()
    assert rel(gr[0].cpu().numpy(), rfft_u(O.grad(zz, host["d"][0], host["W"][0], Pq))) <= 2e-5
    g = torch.Generator(device="cuda")
    g.manual_seed(8)
    worst = _fd_check(prob, band_t, nb, s, to_dev(q, torch.float64), 200, g, h_s=0.5, h_q=1e-3)
    assert worst <= 1.0, worst
