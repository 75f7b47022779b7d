"""GPU band-power estimator (bandpower_estimate) against the oracle's
simulation band powers (Sec. 2.4-2.5) on the same seeded random fields.

Both sides solve every map to a tight gradient tolerance, so the comparison is
a numerics check.  Tolerances: FP64 1e-7 relative (the MAP error of 1e-10 is
squared into E and differenced in F), mixed 1e-3 (the stated band-power
tolerance)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import wf_oracle as O  # noqa: E402
from paper_1810_00503_gb300 import synth, wf  # noqa: E402
from tests.helpers import ensure_lib, to_dev  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    ensure_lib()


def _run(n, nb, J, nfd, precision, seed, masked_frac=0.25):
    inp = synth.density_small(n, seed=seed, masked_frac=masked_frac)
    npdt = np.float64 if precision == "fp64" else np.float32
    wdt = torch.float64 if precision == "fp64" else torch.float32
    P = inp.P.astype(npdt).astype(np.float64)
    Ninv = inp.Ninv.astype(npdt).astype(np.float64)
    d = O.synthesize_data(inp.z, inp.noise, inp.mask, P).astype(npdt).astype(np.float64)
    bands = synth.log_bands(n, nb)
    rng = np.random.default_rng(seed + 100)
    sig = np.where(Ninv > 0, 1.0 / np.sqrt(np.where(Ninv > 0, Ninv, 1.0)), 0.0)
    z = rng.standard_normal((J, 1, n, n)).astype(npdt).astype(np.float64)
    nz = (rng.standard_normal((J, 1, n, n)) * sig).astype(npdt).astype(np.float64)
    u = rng.standard_normal((nb, nfd, 1, n, n)).astype(npdt).astype(np.float64)
    res, stats = wf.bandpower_estimate(
        to_dev(d, wdt), to_dev(inp.mask, torch.uint8), to_dev(Ninv, wdt), to_dev(P[..., : n // 2 + 1], wdt),
        to_dev(bands[..., : n // 2 + 1], torch.int16), nb, to_dev(z, wdt), to_dev(nz, wdt), to_dev(u, wdt),
        precision=precision, gtol_rel=1e-12 if precision == "fp64" else 1e-7, max_iter=20000,
        refresh_every=0 if precision == "fp64" else 50)
    ref = O.bandpower_sims(d, inp.mask, Ninv, P, bands, nb, z, nz, u, gtol_rel=1e-12, max_iter=20000)
    return res, ref, stats


def _close(a, b, tol):
    a = np.asarray(a); b = np.asarray(b)
    return np.abs(a - b).max() <= tol * np.abs(b).max()


def test_bandpower_fp64_matches_oracle():
    res, ref, stats = _run(16, 3, 8, 4, "fp64", seed=31)
    assert all(s["status"] == "WF_OK" for s in stats)
    for k in ("theta_fid", "E", "b", "F", "cov_E", "theta_hat", "cov"):
        kk = {"b": "bias", "F": "fisher"}.get(k, k)
        assert _close(res[kk], ref[k], 1e-7), (k, res[kk], ref[k])


def test_bandpower_mixed_matches_oracle_to_1e3():
    res, ref, stats = _run(64, 4, 12, 3, "mixed", seed=5)
    for k in ("E", "b", "F", "theta_hat"):
        kk = {"b": "bias", "F": "fisher"}.get(k, k)
        assert _close(res[kk], ref[k], 1e-3), (k, res[kk], ref[k])


def test_bandpower_rejects_bad_counts():
    n = 16
    dt = torch.float64
    z = torch.zeros((1, 1, n, n), dtype=dt, device="cuda")
    with pytest.raises(wf.WfError, match="EINVAL"):
        wf.bandpower_estimate(z[0], torch.ones((n, n), dtype=torch.uint8, device="cuda"), z[0] + 1,
                              torch.ones((1, n, n // 2 + 1), dtype=dt, device="cuda"),
                              torch.zeros((1, n, n // 2 + 1), dtype=torch.int16, device="cuda"), 2,
                              z, z, torch.zeros((2, 2, 1, n, n), dtype=dt, device="cuda"))  # n_fd > n_sim


def test_sharded_calls_reduce_to_the_single_call():
    """The multi-GPU split run as two sequential shards on one GPU: shard 0 owns
    every Fisher map, shard 1 none (n_fd = 0); their summed partial sums give
    the single call's estimate (the maps are solved independently)."""
    from paper_1810_00503_gb300 import dist as D
    n, nb, J, nfd, seed = 16, 3, 8, 4, 31
    inp = synth.density_small(n, seed=seed, masked_frac=0.25)
    d = O.synthesize_data(inp.z, inp.noise, inp.mask, inp.P)
    bands = synth.log_bands(n, nb)
    rng = np.random.default_rng(seed + 100)
    sig = np.where(inp.Ninv > 0, 1.0 / np.sqrt(np.where(inp.Ninv > 0, inp.Ninv, 1.0)), 0.0)
    z = rng.standard_normal((J, 1, n, n))
    nz = rng.standard_normal((J, 1, n, n)) * sig
    u = rng.standard_normal((nb, nfd, 1, n, n))
    dt = torch.float64
    common = (to_dev(d, dt), to_dev(inp.mask, torch.uint8), to_dev(inp.Ninv, dt), to_dev(inp.P[..., : n // 2 + 1], dt),
              to_dev(bands[..., : n // 2 + 1], torch.int16), nb)
    kw = dict(precision="fp64", gtol_rel=1e-12, max_iter=20000, refresh_every=0)
    full, _ = wf.bandpower_estimate(*common, to_dev(z, dt), to_dev(nz, dt), to_dev(u, dt), **kw)
    total = np.zeros(2 + nb + 2 * nb * nb)
    for sims, (lo, hi) in ((list(range(0, 5)), (0, 4)), (list(range(5, 8)), (4, 4))):
        res, stats = wf.bandpower_estimate(*common, to_dev(z[sims], dt), to_dev(nz[sims], dt),
                                           to_dev(u[:, lo:hi], dt), **kw)
        assert all(s["status"] == "WF_OK" for s in stats)
        assert np.allclose(res["E_maps"][0], full["E"], rtol=1e-9)
        if hi == lo:
            assert np.isnan(res["theta_hat"]).all() and np.isnan(res["fisher"]).all()
        total += D.local_sums(res["E_maps"], len(sims), nb, hi - lo)
    red = D.combine(total, full["E"], full["theta_fid"])
    for k in ("bias", "fisher", "cov_E", "theta_hat", "cov"):
        assert _close(red[k], full[k], 1e-9), (k, red[k], full[k])
    assert np.allclose(full["E_maps"][1:1 + J].mean(axis=0), full["bias"], rtol=1e-12)


def test_device_outputs_equal_host_outputs():
    # in->out_on_device: the same estimate written to device arrays, single and
    # iterated (whose fiducial moves on the host between estimates)
    n, nb = 16, 3
    inp = synth.density_small(n, seed=41)
    dt = torch.float64
    d = O.synthesize_data(inp.z, inp.noise, inp.mask, inp.P)
    args = (to_dev(d, dt), to_dev(inp.mask, torch.uint8), to_dev(inp.Ninv, dt),
            to_dev(inp.P[..., : n // 2 + 1], dt), to_dev(synth.log_bands(n, nb)[..., : n // 2 + 1], torch.int16),
            nb, None, None, None)
    kw = dict(precision="fp64", n_sim=4, n_fd=2, seed=9, gtol_rel=1e-12, max_iter=20000)
    host, _ = wf.bandpower_estimate(*args, **kw)
    dev, _ = wf.bandpower_estimate(*args, out_on_device=True, **kw)
    # two runs agree to rounding (the band sums are accumulated with atomics,
    # so their last bits depend on the order)
    same = lambda a, b: np.allclose(a, b, rtol=1e-9, atol=1e-12 * np.abs(b).max(), equal_nan=True)
    for k, v in host.items():
        assert isinstance(dev[k], torch.Tensor) and dev[k].is_cuda
        assert same(dev[k].cpu().numpy(), v), k
    host_i, _, hist_h, _ = wf.bandpower_iterate(*args, n_iter=2, **kw)
    dev_i, _, hist_d, _ = wf.bandpower_iterate(*args, n_iter=2, out_on_device=True, **kw)
    assert same(hist_d, hist_h)
    for k, v in host_i.items():
        assert same(dev_i[k].cpu().numpy(), v), k


def test_sharded_leakage_bias_calls_reduce_to_the_single_call():
    """Joint E/B in the leakage-bias form with the EE block truncated, split
    over two sequential shards as over two GPUs (dist.assignment, device draws
    keyed by global simulation index): the summed partial sums give the single
    call's estimate."""
    from paper_1810_00503_gb300 import dist as D
    n, nb, J, nfd, seed = 16, 3, 6, 4, 33
    inp = synth.shear_eb(n, seed=10)
    d = O.synthesize_data(inp.z, inp.noise, inp.mask, inp.P)
    bands = synth.log_bands(n, nb, C=2)
    nbt = 2 * nb
    dt = torch.float64
    common = (to_dev(d, dt), to_dev(inp.mask, torch.uint8), to_dev(inp.Ninv, dt), to_dev(inp.P[..., : n // 2 + 1], dt),
              to_dev(bands[..., : n // 2 + 1], torch.int16), nbt)
    kw = dict(precision="fp64", gtol_rel=1e-12, max_iter=20000, seed=seed, leak_split=nb, trunc=(nb, 1))
    full, _ = wf.bandpower_estimate(*common, None, None, None, n_sim=J, n_fd=nfd, **kw)
    F = np.asarray(full["fisher"])
    assert F[0, 2] == 0.0 and F[0, 1] != 0.0 and not F[:nb, nb:].any()
    total = None
    for rank in range(2):
        sims, (lo, hi) = D.assignment(J, nfd, 2, rank)
        res, stats = wf.bandpower_estimate(*common, None, None, None, n_sim=len(sims), n_fd=hi - lo,
                                           sim_index=sims, **kw)
        assert all(s["status"] == "WF_OK" for s in stats)
        part = D.local_sums(res["E_maps"], len(sims), nbt, hi - lo, leak_split=nb)
        total = part if total is None else total + part
    red = D.combine(total, full["E"], full["theta_fid"], leak_split=nb, trunc=(nb, 1))
    for k in ("bias", "fisher", "cov_E", "theta_hat", "cov"):
        assert _close(red[k], full[k], 1e-9), (k, red[k], full[k])


def _fields32(inp, J, rows, nfd, C, seed):
    """FP32-rounded white fields and noise (as float64 arrays) for both sides."""
    rng = np.random.default_rng(seed)
    n = inp.n
    N32 = inp.Ninv.astype(np.float32).astype(np.float64)
    sig = np.where(N32 > 0, 1.0 / np.sqrt(np.where(N32 > 0, N32, 1.0)), 0.0)
    r32 = lambda a: a.astype(np.float32).astype(np.float64)
    return (r32(rng.standard_normal((J, C, n, n))), r32(rng.standard_normal((J, C, n, n)) * sig),
            r32(rng.standard_normal((rows, nfd, C, n, n))))


def test_bandpower_mixed_256_full_tiles_matches_oracle_to_1e3():
    """Mixed precision at 256^2, where every FFT stage runs its full-tile fast
    path: 6 log bands, 4 noise-bias simulations, 2 Fisher simulations per band,
    against the oracle's simulation estimate on the same FP32 inputs.  (A
    projected-density spectrum: the kernels do not depend on the spectrum's
    shape, and the oracle's textbook L-BFGS needs ~3000 iterations per map on
    the CMB-like one at this size.)"""
    n, nb, J, nfd = 256, 6, 4, 2
    inp = synth.density_projected(n, seed=1)
    r32 = lambda a: a.astype(np.float32).astype(np.float64)
    P, Ninv = r32(inp.P), r32(inp.Ninv)
    d = r32(O.synthesize_data(inp.z, inp.noise, inp.mask, P))
    bands = synth.log_bands(n, nb)
    z, nz, u = _fields32(inp, J, nb, nfd, 1, 41)
    f32 = torch.float32
    res, stats = wf.bandpower_estimate(
        to_dev(d, f32), to_dev(inp.mask, torch.uint8), to_dev(Ninv, f32), to_dev(P[..., : n // 2 + 1], f32),
        to_dev(bands[..., : n // 2 + 1], torch.int16), nb, to_dev(z, f32), to_dev(nz, f32), to_dev(u, f32),
        precision="mixed", gtol_rel=1e-7, max_iter=20000, refresh_every=50)
    assert all(s["status"] == "WF_OK" for s in stats), stats
    ref = O.bandpower_sims(d, inp.mask, Ninv, P, bands, nb, z, nz, u, gtol_rel=1e-9, max_iter=20000)
    for k in ("theta_fid", "E", "b", "F", "theta_hat"):
        kk = {"b": "bias", "F": "fisher"}.get(k, k)
        assert _close(res[kk], ref[k], 1e-3), (k, res[kk], ref[k])


def test_bandpower_mixed_eb_128_leakage_bias_matches_oracle_to_1e3():
    """Joint E/B at 128^2 in mixed precision, the leakage-bias form of App. C
    (per-band Fisher maps for the 4 E bands, one joint B map per Fisher
    simulation), 4 noise-bias simulations, 2 Fisher simulations per row."""
    n, nb, J, nfd = 128, 4, 4, 2
    inp = synth.shear_eb(n, seed=2)
    r32 = lambda a: a.astype(np.float32).astype(np.float64)
    P, Ninv = r32(inp.P), r32(inp.Ninv)
    d = r32(O.synthesize_data(inp.z, inp.noise, inp.mask, P))
    bands = synth.log_bands(n, nb, C=2)
    z, nz, u = _fields32(inp, J, nb + 1, nfd, 2, 43)
    f32 = torch.float32
    res, stats = wf.bandpower_estimate(
        to_dev(d, f32), to_dev(inp.mask, torch.uint8), to_dev(Ninv, f32), to_dev(P[..., : n // 2 + 1], f32),
        to_dev(bands[..., : n // 2 + 1], torch.int16), 2 * nb, to_dev(z, f32), to_dev(nz, f32), to_dev(u, f32),
        precision="mixed", gtol_rel=1e-7, max_iter=20000, refresh_every=50, leak_split=nb)
    assert all(s["status"] == "WF_OK" for s in stats), stats
    ref = O.bandpower_sims(d, inp.mask, Ninv, P, bands, 2 * nb, z, nz, u, gtol_rel=1e-10, max_iter=20000,
                           leak_split=nb)
    F = np.asarray(res["fisher"])
    assert not F[:nb, nb:].any() and not F[nb:, :nb].any()
    for k in ("E", "b", "F", "theta_hat"):
        kk = {"b": "bias", "F": "fisher"}.get(k, k)
        assert _close(res[kk], ref[k], 1e-3), (k, res[kk], ref[k])
