"""Device normal deviates (wf_normal_draw) against the oracle's own
Philox4x32-10 + Box-Muller implementation (oracle/philox.py, pinned to the
generator's published known-answer vectors), and band powers computed from
fields the library draws itself against the oracle fed the same deviates."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import philox as PH  # noqa: E402
from oracle import wf_oracle as O  # noqa: E402
from paper_1810_00503_gb300 import synth, wf  # noqa: E402
from tests.helpers import ensure_lib, to_dev  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    ensure_lib()


@pytest.mark.parametrize("offset", [0, 13, 2 ** 33 + 1])
def test_normal_draw_fp64_matches_oracle(offset):
    dev = wf.normal_draw(7, 100001, stream_id=2, offset=offset).cpu().numpy()
    ref = PH.normals(7, 2, 100001, offset=offset)
    # same generator words; cos, sin, log, sqrt rounding may differ by an ulp
    assert np.max(np.abs(dev - ref)) <= 1e-14 * np.max(np.abs(ref))


def test_normal_draw_fp32_and_empty():
    dev = wf.normal_draw(123, 4097, stream_id=0, dtype=torch.float32).cpu().numpy()
    ref = PH.normals(123, 0, 4097).astype(np.float32)
    assert np.max(np.abs(dev - ref)) <= 2e-7 * np.max(np.abs(ref))
    assert wf.normal_draw(1, 0).numel() == 0


def test_bandpower_with_device_draws_matches_oracle():
    n, nb, J, nfd, seed = 16, 3, 8, 4, 21
    inp = synth.density_small(n, seed=31, masked_frac=0.25)
    d = O.synthesize_data(inp.z, inp.noise, inp.mask, inp.P)
    bands = synth.log_bands(n, nb)
    dt = torch.float64
    res, stats = wf.bandpower_estimate(
        to_dev(d, dt), to_dev(inp.mask, torch.uint8), to_dev(inp.Ninv, dt), to_dev(inp.P[..., : n // 2 + 1], dt),
        to_dev(bands[..., : n // 2 + 1], torch.int16), nb, None, None, None, n_sim=J, n_fd=nfd,
        precision="fp64", gtol_rel=1e-12, max_iter=20000, seed=seed)
    assert all(s["status"] == "WF_OK" for s in stats)
    npix = n * n
    w = inp.mask * inp.Ninv
    sig = np.where(w > 0, 1.0 / np.sqrt(np.where(w > 0, w, 1.0)), 0.0)
    z = PH.normals(seed, PH.STREAM_Z, J * npix).reshape(J, 1, n, n)
    nz = PH.normals(seed, PH.STREAM_NOISE, J * npix).reshape(J, 1, n, n) * sig
    u = np.zeros((nb, nfd, 1, n, n))
    for j in range(nfd):  # Fisher map (l, j) reuses simulation j: deviates (j nb + l) npix ..
        for lb in range(nb):
            u[lb, j] = PH.normals(seed, PH.STREAM_U, npix, offset=(j * nb + lb) * npix).reshape(1, n, n)
    ref = O.bandpower_sims(d, inp.mask, inp.Ninv, inp.P, bands, nb, z, nz, u, gtol_rel=1e-12, max_iter=20000)
    for k in ("E", "b", "F", "theta_hat", "cov_E"):
        kk = {"b": "bias", "F": "fisher"}.get(k, k)
        a, b = np.asarray(res[kk]), np.asarray(ref[k])
        assert np.abs(a - b).max() <= 1e-7 * np.abs(b).max(), (k, a, b)


def test_partial_random_fields_rejected():
    n = 16
    dt = torch.float64
    z = torch.zeros((2, 1, n, n), dtype=dt, device="cuda")
    with pytest.raises(wf.WfError, match="EINVAL"):
        wf.bandpower_estimate(z[0], torch.ones((n, n), dtype=torch.uint8, device="cuda"), z[0] + 1,
                              torch.ones((1, n, n // 2 + 1), dtype=dt, device="cuda"),
                              torch.zeros((1, n, n // 2 + 1), dtype=torch.int16, device="cuda"), 1,
                              z, None, None, n_sim=2, n_fd=1)


def test_split_simulations_give_the_single_run_estimate():
    """Simulations split over calls as over GPUs (dist.assignment), each call
    drawing its own fields by global simulation index: the summed partials
    equal one call over all simulations, for one, two and three ranks."""
    from paper_1810_00503_gb300 import dist as D
    n, nb, J, nfd, seed = 16, 3, 7, 3, 9
    inp = synth.density_small(n, seed=5, masked_frac=0.2)
    d = O.synthesize_data(inp.z, inp.noise, inp.mask, inp.P)
    bands = synth.log_bands(n, nb)
    dt = torch.float64
    args = (to_dev(d, dt), to_dev(inp.mask, torch.uint8), to_dev(inp.Ninv, dt), to_dev(inp.P[..., : n // 2 + 1], dt),
            to_dev(bands[..., : n // 2 + 1], torch.int16), nb)
    kw = dict(precision="fp64", gtol_rel=1e-12, max_iter=20000, seed=seed)
    full, _ = wf.bandpower_estimate(*args, None, None, None, n_sim=J, n_fd=nfd, **kw)
    for world in (1, 2, 3):
        total = np.zeros(2 + nb + 2 * nb * nb)
        for rank in range(world):
            sims, (lo, hi) = D.assignment(J, nfd, world, rank)
            res, _ = wf.bandpower_estimate(*args, None, None, None, n_sim=len(sims), n_fd=hi - lo,
                                           sim_index=sims, **kw)
            total += D.local_sums(res["E_maps"], len(sims), nb, hi - lo)
        red = D.combine(total, full["E"], full["theta_fid"])
        for k in ("bias", "fisher", "cov_E", "theta_hat"):
            assert np.abs(red[k] - full[k]).max() <= 1e-9 * np.abs(full[k]).max(), (world, k)
    # estimate_on_rank without a process group is the single-process estimate
    est, _ = D.estimate_on_rank(*args, J, nfd, 1, 0, seed, precision="fp64", gtol_rel=1e-12, max_iter=20000)
    assert np.abs(est["theta_hat"] - full["theta_hat"]).max() <= 1e-9 * np.abs(full["theta_hat"]).max()
