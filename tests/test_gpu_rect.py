"""Rectangular maps (ny x nx, both powers of two, square pixels) on the GPU
against the FP64 oracle's rectangular grids: the objective + gradient pass,
the Hessian-vector product, the signal map, data synthesis and band energies
element by element; MAP solves against the dense Wiener filter; the certified
mixed solve judged by the oracle's gradient; checkpoint and resume; batches of
several shapes in one call; and a band-power estimate.  The joint E/B cases
test the rotation at the wavevector (mx / nx, my / ny) of App. C, which is
where a rectangular map differs from a square one beyond its indexing.

Tolerances as the square tests: FP64 fields and chi^2 1e-12 (relative L2),
mixed fields 2e-5 and chi^2 1e-5; MAP 1e-10 (FP64); band powers 1e-7 (FP64)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import wf_oracle as O  # noqa: E402
from paper_1810_00503_gb300 import synth, wf  # noqa: E402
from tests.helpers import ensure_lib, make_problem, rel, rfft_u, to_dev  # noqa: E402

TOL = {"fp64": dict(field=1e-12, chi2=1e-12), "mixed": dict(field=2e-5, chi2=1e-5)}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    ensure_lib()


def _inputs(ny, nx, C, B, seed):
    if C == 1:
        return [synth.density_small(ny, seed=seed + b, nx=nx) for b in range(B)]
    return [synth.shear_eb(ny, seed=seed + b, nx=nx) for b in range(B)]


def _spec_t(fields, precision):
    cdt = torch.complex128 if precision == "fp64" else torch.complex64
    npc = np.complex128 if precision == "fp64" else np.complex64
    S = np.stack([rfft_u(f) for f in fields]).astype(npc)
    return to_dev(S, cdt), [np.fft.irfft2(s.astype(np.complex128), s=f.shape[-2:], norm="ortho")
                           for s, f in zip(S, fields)]


# shapes spanning both aspect directions, narrow strips at both extremes
# (8 or 16 pixels on one side, 1024 on the other: column tiles as wide as the
# block, one row block) and several tiles with a ragged last trip in the
# per-mode loop
CASES = [(8, 64, 1, 1, "fp64"), (64, 8, 2, 1, "fp64"), (16, 128, 2, 2, "fp64"), (128, 32, 1, 3, "fp64"),
         (32, 1024, 1, 1, "fp64"), (1024, 16, 2, 1, "fp64"), (256, 512, 2, 1, "fp64"),
         (512, 128, 1, 2, "fp64"), (1024, 8, 1, 1, "fp64"), (8, 1024, 1, 1, "fp64"), (8, 1024, 2, 2, "fp64"),
         (16, 1024, 1, 1, "fp64"),
         (32, 256, 2, 2, "mixed"), (512, 64, 1, 3, "mixed"), (256, 1024, 2, 1, "mixed"),
         (1024, 512, 1, 1, "mixed")]


@pytest.mark.parametrize("ny,nx,C,B,precision", CASES)
def test_eval_rect_matches_oracle(ny, nx, C, B, precision):
    inputs = _inputs(ny, nx, C, B, seed=300 + ny + nx)
    prob, host = make_problem(inputs, precision, shared_P=(B % 2 == 1))
    fields = [synth.random_state(ny, C, seed=17 + b, nx=nx) for b in range(B)]
    s, zs = _spec_t(fields, precision)
    chi2, g = prob.eval(s)
    torch.cuda.synchronize()
    tol = TOL[precision]
    for b in range(B):
        P = host["P"][0] if B % 2 == 1 else host["P"][b]
        rc = O.chi2(zs[b], host["d"][b], host["W"][b], P)
        rg = rfft_u(O.grad(zs[b], host["d"][b], host["W"][b], P))
        assert abs(chi2[b].item() - rc) <= tol["chi2"] * abs(rc), (b, chi2[b].item(), rc)
        assert rel(g[b].cpu().numpy(), rg) <= tol["field"], b


@pytest.mark.parametrize("ny,nx,C,precision", [(16, 64, 2, "fp64"), (128, 16, 2, "fp64"), (64, 256, 1, "fp64"),
                                               (512, 256, 2, "mixed"), (128, 1024, 1, "mixed")])
def test_hess_vec_signal_and_simulate_rect(ny, nx, C, precision):
    inputs = _inputs(ny, nx, C, 2, seed=5)
    prob, host = make_problem(inputs, precision)
    v = synth.random_state(ny, C, seed=3, nx=nx)
    s, zs = _spec_t([v, v], precision)
    hv = prob.hess_vec(s)
    x = prob.signal_map(s)
    wdt = torch.float64 if precision == "fp64" else torch.float32
    npdt = np.float64 if precision == "fp64" else np.float32
    z = np.stack([i.z for i in inputs]).astype(npdt)
    nz = np.stack([i.noise for i in inputs]).astype(npdt)
    dsim = prob.simulate(to_dev(z, wdt), to_dev(nz, wdt))
    torch.cuda.synchronize()
    tol = TOL[precision]["field"]
    for b in range(2):
        assert rel(hv[b].cpu().numpy(), rfft_u(O.hess_vec(zs[b], host["W"][b], host["P"][0]))) <= tol
        assert rel(x[b].cpu().numpy(), O.apply_A(zs[b], host["P"][0])) <= tol
        ref = O.synthesize_data(z[b].astype(np.float64), nz[b].astype(np.float64), host["mask"][b], host["P"][0])
        assert rel(dsim[b].cpu().numpy(), ref) <= tol


def test_eb_rect_rotation_is_the_physical_one():
    """An unmasked E/B map with no noise weight on B: the gradient of a pure-E
    state on a 32 x 128 grid differs from the one the mode-number rotation
    would give, and the GPU follows the wavevector form of the oracle."""
    ny, nx = 32, 128
    inp = synth.shear_eb(ny, seed=9, nx=nx)
    prob, host = make_problem([inp], "fp64")
    f = synth.random_state(ny, 2, seed=4, nx=nx)
    f[1] = 0.0
    s, zs = _spec_t([f], "fp64")
    _, g = prob.eval(s)
    x = prob.signal_map(s)
    torch.cuda.synchronize()
    want = O.apply_A(zs[0], host["P"][0])
    assert rel(x[0].cpu().numpy(), want) <= 1e-12
    # the integer-mode-number rotation (wrong for rectangular pixels' grids)
    my, mx = O.signed_modes(ny, nx)
    k2 = mx * mx + my * my
    c = np.where(k2 > 0, (mx * mx - my * my) / np.where(k2 > 0, k2, 1), 1.0)
    Z = O.fft2u(zs[0]) * np.sqrt(host["P"][0])
    wrong = O.ifft2u(np.stack([c * Z[0], Z[0] * 0])).real
    assert rel(x[0].cpu().numpy()[0], wrong[0]) > 1e-2
    assert rel(g[0].cpu().numpy(), rfft_u(O.grad(zs[0], host["d"][0], host["W"][0], host["P"][0]))) <= 1e-12


def test_band_energy_rect():
    ny, nx, nb = 64, 256, 6
    inputs = _inputs(ny, nx, 2, 2, seed=4)
    prob, host = make_problem(inputs, "fp64")
    bands = synth.log_bands(ny, nb, C=2, nx=nx)
    theta = O.theta_fid(host["P"][0], bands, 2 * nb)
    fields = [synth.random_state(ny, 2, seed=b, nx=nx) for b in range(2)]
    s, zs = _spec_t(fields, "fp64")
    E = prob.band_energy(s, to_dev(bands[..., : nx // 2 + 1], torch.int16), to_dev(theta, torch.float64))
    torch.cuda.synchronize()
    for b in range(2):
        assert np.allclose(E[b].cpu().numpy(), O.band_E(zs[b], bands, theta, 2 * nb), rtol=1e-12, atol=0)


@pytest.mark.parametrize("ny,nx,C", [(16, 32, 1), (32, 8, 1), (8, 32, 2), (16, 16, 2)])
def test_fp64_rect_solve_matches_dense_wiener_filter(ny, nx, C):
    inp = _inputs(ny, nx, C, 1, seed=21)[0]
    prob, host = make_problem([inp], "fp64")
    res = prob.solve(gtol_rel=1e-12, max_iter=20000, x_out=True)
    assert res.stats[0]["status"] == "WF_OK", res.stats
    zs = O.dense_wf_whitened(host["d"][0], host["W"][0], host["P"][0])
    assert rel(res.s[0].cpu().numpy(), rfft_u(zs)) <= 1e-10
    assert rel(res.x[0].cpu().numpy(), O.apply_A(zs, host["P"][0])) <= 1e-10


@pytest.mark.parametrize("ny,nx,C", [(8, 1024, 1), (1024, 8, 2), (16, 512, 2)])
def test_fp64_strip_solve_certified_by_the_oracle(ny, nx, C):
    """Strips too large for the dense filter: the FP64 solve stops at
    |g| / |g0| < 1e-12, and the oracle's gradient at the state it returns
    agrees (within 2x; the MAP error is then at most |g| / 2)."""
    inp = _inputs(ny, nx, C, 1, seed=23)[0]
    prob, host = make_problem([inp], "fp64")
    res = prob.solve(gtol_rel=1e-12, max_iter=50000)
    assert res.stats[0]["status"] == "WF_OK", res.stats
    z = np.fft.irfft2(res.s[0].cpu().numpy(), s=(ny, nx), norm="ortho")
    g = O.grad(z, host["d"][0], host["W"][0], host["P"][0])
    g0 = O.grad(np.zeros_like(z), host["d"][0], host["W"][0], host["P"][0])
    assert np.linalg.norm(g) <= 2e-12 * np.linalg.norm(g0), (np.linalg.norm(g), np.linalg.norm(g0))


def _p_eff(P32, ny, nx):
    """Per-mode power whose FP64 sqrt(P / (ny nx)) equals the library's FP32 table."""
    sp = np.sqrt(P32.astype(np.float64) / (ny * nx)).astype(np.float32).astype(np.float64)
    return sp * sp * (ny * nx)


@pytest.mark.parametrize("ny,nx", [(128, 512), (512, 64)])
def test_mixed_rect_refined_solve_certified_by_the_oracle(ny, nx):
    """E/B shear on a rectangular patch in mixed precision with FP64
    refinement to the 1e-4 certificate; the oracle's FP64 gradient at the
    returned state (on the FP32-rounded problem the library solves) confirms
    |grad| / 2 <= 1e-4 |s|, which bounds the relative error of the MAP."""
    inp = synth.shear_eb(ny, seed=12, nx=nx)
    prob, host = make_problem([inp], "mixed")
    res, cert = prob.solve_refined(cert_tol=1e-4, max_rounds=8, gtol_rel=1e-5, max_iter=50000)
    assert res.stats[0]["status"] == "WF_OK", res.stats
    s = res.s[0].cpu().numpy()
    z = np.fft.irfft2(s, s=(ny, nx), norm="ortho")
    W = (inp.mask[None] * inp.Ninv.astype(np.float32)).astype(np.float64)
    g = O.grad(z, host["d"][0], W, _p_eff(inp.P.astype(np.float32), ny, nx))
    oc = 0.5 * np.linalg.norm(g) / np.linalg.norm(z)
    assert oc <= 1e-4, oc
    assert cert[0] <= 1e-4 and abs(cert[0] - oc) <= 0.05 * oc + 1e-9, (cert[0], oc)


def test_rect_checkpoint_resume_equals_uninterrupted():
    ny, nx = 64, 256
    inputs = _inputs(ny, nx, 2, 2, seed=40)

    def problem():
        return make_problem(inputs, "mixed", shared_P=False)[0]

    opts = dict(gtol_rel=1e-9, max_iter=5000, refresh_every=50, check_every=8)
    pa = problem()
    pa.start(**opts)
    pa.step(29)
    ck = pa.export_state()
    pa.step(40)
    ra = pa.finish()
    pb = problem()
    pb.import_state(ck)
    pb.step(40)
    rb = pb.finish()
    assert torch.equal(ra.s, rb.s)
    assert [s["iters"] for s in ra.stats] == [s["iters"] for s in rb.stats]
    # a checkpoint of the transposed shape is refused
    pt = make_problem(_inputs(nx, ny, 2, 2, seed=40), "mixed", shared_P=False)[0]
    with pytest.raises(wf.WfError, match="EINVAL"):
        pt.import_state(ck)
    for p in (pa, pb, pt):
        p.close()


def test_solve_many_mixes_rect_and_square_shapes():
    """One wf_map_solve_many call over problems of shapes 64 x 256, 256 x 64 and
    128 x 128 ends with the same states as solving each problem alone."""
    shapes = [(64, 256), (256, 64), (128, 128)]
    opts = dict(gtol_rel=1e-8, max_iter=20000, autotune=0)
    probs = [make_problem(_inputs(ny, nx, 1, 2, seed=ny + 3 * nx), "fp64")[0] for ny, nx in shapes]
    together = wf.solve_many(probs, **opts)
    for p, r in zip(probs, together):
        alone = p.solve(**opts)
        assert all(s["status"] == "WF_OK" for s in r.stats)
        assert rel(r.s.cpu().numpy(), alone.s.cpu().numpy()) <= 1e-12
        p.close()


def test_bandpower_rect_fp64_matches_oracle():
    ny, nx, nb, J, nfd, seed = 16, 32, 3, 8, 4, 31
    inp = synth.density_small(ny, seed=seed, masked_frac=0.25, nx=nx)
    d = O.synthesize_data(inp.z, inp.noise, inp.mask, inp.P)
    bands = synth.log_bands(ny, nb, nx=nx)
    rng = np.random.default_rng(seed + 100)
    sig = np.where(inp.Ninv > 0, 1.0 / np.sqrt(np.where(inp.Ninv > 0, inp.Ninv, 1.0)), 0.0)
    z = rng.standard_normal((J, 1, ny, nx))
    nz = rng.standard_normal((J, 1, ny, nx)) * sig
    u = rng.standard_normal((nb, nfd, 1, ny, nx))
    dt = torch.float64
    h1 = nx // 2 + 1
    res, stats = wf.bandpower_estimate(
        to_dev(d, dt), to_dev(inp.mask, torch.uint8), to_dev(inp.Ninv, dt), to_dev(inp.P[..., :h1], dt),
        to_dev(bands[..., :h1], torch.int16), nb, to_dev(z, dt), to_dev(nz, dt), to_dev(u, dt),
        precision="fp64", gtol_rel=1e-12, max_iter=20000, refresh_every=0)
    assert all(s["status"] == "WF_OK" for s in stats)
    ref = O.bandpower_sims(d, inp.mask, inp.Ninv, inp.P, bands, nb, z, nz, u, gtol_rel=1e-12, max_iter=20000)
    for k in ("theta_fid", "E", "b", "F", "cov_E", "theta_hat", "cov"):
        kk = {"b": "bias", "F": "fisher"}.get(k, k)
        a, b = np.asarray(res[kk]), np.asarray(ref[k])
        assert np.abs(a - b).max() <= 1e-7 * np.abs(b).max(), (k, a, b)


def test_rect_shapes_refused():
    inp = synth.density_small(16, seed=1, nx=32)
    dt = torch.float64
    for ny, nx in ((16, 12), (4, 32), (16, 2048), (24, 32)):
        N = torch.ones((1, 1, ny, nx), dtype=dt, device="cuda")
        with pytest.raises(wf.WfError, match="EINVAL"):
            wf.Problem(N * 0, torch.ones((ny, nx), dtype=torch.uint8, device="cuda"), N,
                       torch.ones((1, ny, nx // 2 + 1), dtype=dt, device="cuda"))
    del inp


def test_bandpower_rect_mixed_matches_oracle_to_1e3():
    """Mixed precision (FP32 fields, FP64 sums) on a 64 x 128 map with the
    stated band-power tolerance of 1e-3."""
    ny, nx, nb, J, nfd, seed = 64, 128, 4, 8, 3, 17
    inp = synth.density_small(ny, seed=seed, masked_frac=0.25, nx=nx)
    P = inp.P.astype(np.float32).astype(np.float64)
    Ninv = inp.Ninv.astype(np.float32).astype(np.float64)
    d = O.synthesize_data(inp.z, inp.noise, inp.mask, P).astype(np.float32).astype(np.float64)
    bands = synth.log_bands(ny, nb, nx=nx)
    rng = np.random.default_rng(seed + 100)
    sig = np.where(Ninv > 0, 1.0 / np.sqrt(np.where(Ninv > 0, Ninv, 1.0)), 0.0)
    z = rng.standard_normal((J, 1, ny, nx)).astype(np.float32).astype(np.float64)
    nz = (rng.standard_normal((J, 1, ny, nx)) * sig).astype(np.float32).astype(np.float64)
    u = rng.standard_normal((nb, nfd, 1, ny, nx)).astype(np.float32).astype(np.float64)
    dt, h1 = torch.float32, nx // 2 + 1
    res, stats = wf.bandpower_estimate(
        to_dev(d, dt), to_dev(inp.mask, torch.uint8), to_dev(Ninv, dt), to_dev(P[..., :h1], dt),
        to_dev(bands[..., :h1], torch.int16), nb, to_dev(z, dt), to_dev(nz, dt), to_dev(u, dt),
        precision="mixed", gtol_rel=1e-7, max_iter=20000, refresh_every=50)
    ref = O.bandpower_sims(d, inp.mask, Ninv, P, bands, nb, z, nz, u, gtol_rel=1e-12, max_iter=20000)
    for k in ("E", "b", "F", "theta_hat"):
        kk = {"b": "bias", "F": "fisher"}.get(k, k)
        a, b = np.asarray(res[kk]), np.asarray(ref[k])
        assert np.abs(a - b).max() <= 1e-3 * np.abs(b).max(), (k, a, b)
