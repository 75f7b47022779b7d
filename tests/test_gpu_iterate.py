"""Iterated fiducial (bandpower_iterate) and the joint E/B band powers (C = 2)
against the oracle, and the iteration's behaviour from a distorted start."""
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


def _fields(inp, J, nb, nfd, C, seed):
    rng = np.random.default_rng(seed)
    n = inp.n
    sig = np.where(inp.Ninv > 0, 1.0 / np.sqrt(np.where(inp.Ninv > 0, inp.Ninv, 1.0)), 0.0)
    z = rng.standard_normal((J, C, n, n))
    nz = rng.standard_normal((J, C, n, n)) * sig
    u = rng.standard_normal((nb, nfd, C, n, n))
    return z, nz, u


def _dev(inp, d, P, bands, dt=torch.float64):
    n = inp.n
    return (to_dev(d, dt), to_dev(inp.mask, torch.uint8), to_dev(inp.Ninv, dt), to_dev(P[..., : n // 2 + 1], dt),
            to_dev(bands[..., : n // 2 + 1], torch.int16))


def test_iterate_matches_oracle_iteration():
    n, nb, J, nfd, n_iter = 16, 3, 6, 3, 3
    inp = synth.density_small(n, seed=12, masked_frac=0.2)
    d = O.synthesize_data(inp.z, inp.noise, inp.mask, inp.P)
    bands = synth.log_bands(n, nb)
    r = np.array([0.2, 1.0, 3.0])
    P0 = inp.P.copy()
    for lb in range(nb):
        P0[bands == lb] *= r[lb]
    z, nz, u = _fields(inp, J, nb, nfd, 1, 5)
    dd, mk, Nv, Pv, bv = _dev(inp, d, P0, bands)
    res, stats, hist, Pf = wf.bandpower_iterate(dd, mk, Nv, Pv, bv, nb, to_dev(z, torch.float64),
                                                to_dev(nz, torch.float64), to_dev(u, torch.float64),
                                                n_iter=n_iter, q_min=0.05, q_max=20.0, precision="fp64",
                                                gtol_rel=1e-12, max_iter=20000)
    ref, Pref = O.bandpower_iterate(d, inp.mask, inp.Ninv, P0, bands, nb, z, nz, u, n_iter, q_min=0.05, q_max=20.0,
                                    gtol_rel=1e-12, max_iter=20000)
    for it in range(n_iter):
        th = ref[it]["theta_hat"]
        assert np.abs(hist[it] - th).max() <= 1e-7 * np.abs(th).max(), (it, hist[it], th)
    assert np.abs(res["theta_fid"] - ref[-1]["theta_fid"]).max() <= 1e-7 * np.abs(ref[-1]["theta_fid"]).max()
    Ph = Pf.cpu().numpy()
    assert np.abs(Ph - Pref[..., : n // 2 + 1]).max() <= 1e-7 * np.abs(Pref).max()
    assert all(s["status"] == "WF_OK" for s in stats)


def test_iteration_from_a_distorted_start_reaches_the_truth():
    """The paper's scheme: the true spectrum with every band scaled by a random
    factor in [0.01, 1], then re-estimation.  The re-estimated band powers lie
    near the truth although the start was off by up to 100x."""
    n, nb, J, nfd = 64, 4, 24, 6
    inp = synth.density_small(n, seed=21, masked_frac=0.15)
    d = O.synthesize_data(inp.z, inp.noise, inp.mask, inp.P)
    bands = synth.log_bands(n, nb, kmin=2.0)
    th_true = O.theta_fid(inp.P, bands, nb)
    r = np.random.default_rng(3).uniform(0.01, 1.0, nb)
    P0 = inp.P.copy()
    for lb in range(nb):
        P0[bands == lb] *= r[lb]
    dd, mk, Nv, Pv, bv = _dev(inp, d, P0, bands)
    res, stats, hist, Pf = wf.bandpower_iterate(dd, mk, Nv, Pv, bv, nb, None, None, None, n_sim=J, n_fd=nfd,
                                                n_iter=3, q_min=0.01, q_max=100.0, precision="fp64",
                                                gtol_rel=1e-10, max_iter=20000, seed=8)
    err0 = np.abs(np.log(r))
    err = np.abs(np.log(np.clip(hist[-1], 1e-30, None) / th_true))
    assert np.all(err < 0.35), (r, hist / th_true)
    assert err.mean() < 0.2 * err0.mean(), (err, err0)


def test_joint_eb_bandpowers_match_oracle():
    n, nb, J, nfd = 16, 2, 5, 2
    inp = synth.shear_eb(n, seed=6)
    d = O.synthesize_data(inp.z, inp.noise, inp.mask, inp.P)
    bands = synth.log_bands(n, nb, C=2)  # E bands 0, 1; B bands 2, 3
    z, nz, u = _fields(inp, J, 2 * nb, nfd, 2, 17)
    dd, mk, Nv, Pv, bv = _dev(inp, d, inp.P, bands)
    res, stats = wf.bandpower_estimate(dd, mk, Nv, Pv, bv, 2 * nb, to_dev(z, torch.float64),
                                       to_dev(nz, torch.float64), to_dev(u, torch.float64), precision="fp64",
                                       gtol_rel=1e-12, max_iter=20000)
    ref = O.bandpower_sims(d, inp.mask, inp.Ninv, inp.P, bands, 2 * nb, z, nz, u, gtol_rel=1e-12, max_iter=20000)
    for k in ("E", "b", "F", "theta_hat"):
        kk = {"b": "bias", "F": "fisher"}.get(k, k)
        a, b = np.asarray(res[kk]), np.asarray(ref[k])
        assert np.abs(a - b).max() <= 1e-7 * np.abs(b).max(), (k, a, b)
    # the leakage blocks EB / BE of the Fisher matrix are non-zero under the mask
    F = np.asarray(res["fisher"])
    assert np.abs(F[:nb, nb:]).max() > 1e-6 * np.abs(F).max()


def test_sampled_fisher_columns_match_oracle():
    """Fisher maps for bands 0, 2, 3 only; column 1 interpolated (Sec. 3.1)."""
    n, nb, J, nfd = 16, 4, 6, 3
    inp = synth.density_small(n, seed=14, masked_frac=0.2)
    d = O.synthesize_data(inp.z, inp.noise, inp.mask, inp.P)
    bands = synth.log_bands(n, nb)
    fdb = [0, 2, 3]
    z, nz, u = _fields(inp, J, len(fdb), nfd, 1, 23)
    dd, mk, Nv, Pv, bv = _dev(inp, d, inp.P, bands)
    res, stats = wf.bandpower_estimate(dd, mk, Nv, Pv, bv, nb, to_dev(z, torch.float64), to_dev(nz, torch.float64),
                                       to_dev(u, torch.float64), precision="fp64", gtol_rel=1e-12, max_iter=20000,
                                       fd_bands=fdb)
    assert len(stats) == 1 + J + len(fdb) * nfd
    ref = O.bandpower_sims(d, inp.mask, inp.Ninv, inp.P, bands, nb, z, nz, u, gtol_rel=1e-12, max_iter=20000,
                           fd_bands=fdb)
    for k in ("F", "theta_hat", "b"):
        kk = {"b": "bias", "F": "fisher"}.get(k, k)
        a, b = np.asarray(res[kk]), np.asarray(ref[k])
        assert np.abs(a - b).max() <= 1e-7 * np.abs(b).max(), (k, a, b)


def test_truncated_eb_fisher_matches_oracle():
    """Joint E/B with 3 + 3 bands and the EE block truncated beyond one band
    off the diagonal (App. C)."""
    n, nb, J, nfd = 16, 3, 5, 2
    inp = synth.shear_eb(n, seed=9)
    d = O.synthesize_data(inp.z, inp.noise, inp.mask, inp.P)
    bands = synth.log_bands(n, nb, C=2)
    z, nz, u = _fields(inp, J, 2 * nb, nfd, 2, 29)
    dd, mk, Nv, Pv, bv = _dev(inp, d, inp.P, bands)
    res, _ = wf.bandpower_estimate(dd, mk, Nv, Pv, bv, 2 * nb, to_dev(z, torch.float64), to_dev(nz, torch.float64),
                                   to_dev(u, torch.float64), precision="fp64", gtol_rel=1e-12, max_iter=20000,
                                   trunc=(nb, 1))
    ref = O.bandpower_sims(d, inp.mask, inp.Ninv, inp.P, bands, 2 * nb, z, nz, u, gtol_rel=1e-12, max_iter=20000,
                           trunc=(nb, 1))
    F = np.asarray(res["fisher"])
    assert F[0, 2] == 0.0 and F[2, 0] == 0.0 and F[0, 1] != 0.0 and F[0, 5] != 0.0
    for k in ("F", "theta_hat"):
        kk = {"F": "fisher"}.get(k, k)
        a, b = np.asarray(res[kk]), np.asarray(ref[k])
        assert np.abs(a - b).max() <= 1e-7 * np.abs(b).max(), (k, a, b)


def test_device_draws_of_sampled_bands_agree_with_the_full_run():
    """Fisher fields drawn on the device are keyed by band id, so the sampled
    bands' Fisher columns equal those of the run over every band."""
    n, nb, J, nfd = 16, 4, 5, 2
    inp = synth.density_small(n, seed=15, masked_frac=0.2)
    d = O.synthesize_data(inp.z, inp.noise, inp.mask, inp.P)
    bands = synth.log_bands(n, nb)
    args = _dev(inp, d, inp.P, bands)
    kw = dict(n_sim=J, n_fd=nfd, precision="fp64", gtol_rel=1e-12, max_iter=20000, seed=4)
    full, _ = wf.bandpower_estimate(*args, nb, None, None, None, **kw)
    part, _ = wf.bandpower_estimate(*args, nb, None, None, None, fd_bands=[1, 3], **kw)
    F, G = np.asarray(full["fisher"]), np.asarray(part["fisher"])
    for lp in (1, 3):
        assert np.abs(F[:, lp] - G[:, lp]).max() <= 1e-9 * np.abs(F).max()
    assert np.allclose(full["bias"], part["bias"], rtol=1e-12)


def test_leakage_bias_eb_matches_oracle():
    """Leakage-bias form of App. C: E bands 0, 1 with per-band Fisher maps, B
    bands 2, 3 from one joint map per Fisher simulation, no E-B cross terms."""
    n, nb, J, nfd = 16, 2, 5, 2
    inp = synth.shear_eb(n, seed=6)
    d = O.synthesize_data(inp.z, inp.noise, inp.mask, inp.P)
    bands = synth.log_bands(n, nb, C=2)
    z, nz, u = _fields(inp, J, nb + 1, nfd, 2, 19)
    dd, mk, Nv, Pv, bv = _dev(inp, d, inp.P, bands)
    res, stats = wf.bandpower_estimate(dd, mk, Nv, Pv, bv, 2 * nb, to_dev(z, torch.float64),
                                       to_dev(nz, torch.float64), to_dev(u, torch.float64), precision="fp64",
                                       gtol_rel=1e-12, max_iter=20000, leak_split=nb)
    assert len(stats) == 1 + J + (nb + 1) * nfd
    assert all(s["status"] == "WF_OK" for s in stats)
    ref = O.bandpower_sims(d, inp.mask, inp.Ninv, inp.P, bands, 2 * nb, z, nz, u, gtol_rel=1e-12,
                           max_iter=20000, leak_split=nb)
    F = np.asarray(res["fisher"])
    assert not F[:nb, nb:].any() and not F[nb:, :nb].any() and F[2, 3] == 0.0 and F[3, 2] == 0.0
    for k in ("E", "b", "F", "theta_hat"):
        kk = {"b": "bias", "F": "fisher"}.get(k, k)
        a, b = np.asarray(res[kk]), np.asarray(ref[k])
        assert np.abs(a - b).max() <= 1e-7 * np.abs(b).max(), (k, a, b)


def test_leakage_bias_with_device_draws_and_sampled_e_bands():
    """Device-drawn fields (the joint B maps draw band L's row), Fisher maps for
    E bands 0 and 2 only, column 1 interpolated inside the E block."""
    from oracle import philox as PH
    n, nb, J, nfd, seed = 16, 3, 4, 2, 12
    inp = synth.shear_eb(n, seed=7)
    d = O.synthesize_data(inp.z, inp.noise, inp.mask, inp.P)
    bands = synth.log_bands(n, nb, C=2)
    nbt, fdb = 2 * nb, [0, 2]
    args = _dev(inp, d, inp.P, bands)
    res, stats = wf.bandpower_estimate(*args, nbt, None, None, None, n_sim=J, n_fd=nfd, precision="fp64",
                                       gtol_rel=1e-12, max_iter=20000, seed=seed, fd_bands=fdb, leak_split=nb)
    assert len(stats) == 1 + J + (len(fdb) + 1) * nfd
    npix = 2 * n * n
    w = inp.mask[None] * inp.Ninv
    sig = np.where(w > 0, 1.0 / np.sqrt(np.where(w > 0, w, 1.0)), 0.0)
    z = PH.normals(seed, PH.STREAM_Z, J * npix).reshape(J, 2, n, n)
    nz = PH.normals(seed, PH.STREAM_NOISE, J * npix).reshape(J, 2, n, n) * sig
    rows = fdb + [nb]  # the joint B row draws as band L = nb
    u = np.zeros((len(rows), nfd, 2, n, n))
    for k, lb in enumerate(rows):
        for j in range(nfd):
            u[k, j] = PH.normals(seed, PH.STREAM_U, npix, offset=(j * nbt + lb) * npix).reshape(2, n, n)
    ref = O.bandpower_sims(d, inp.mask, inp.Ninv, inp.P, bands, nbt, z, nz, u, gtol_rel=1e-12, max_iter=20000,
                           fd_bands=fdb, leak_split=nb)
    F = np.asarray(res["fisher"])
    assert F[0, 1] != 0.0 and not F[:nb, nb:].any()
    for k in ("E", "b", "F", "theta_hat"):
        kk = {"b": "bias", "F": "fisher"}.get(k, k)
        a, b = np.asarray(res[kk]), np.asarray(ref[k])
        assert np.abs(a - b).max() <= 1e-7 * np.abs(b).max(), (k, a, b)


def test_leakage_bias_arguments_checked():
    n, nb = 16, 2
    inp = synth.shear_eb(n, seed=8)
    bands = synth.log_bands(n, nb, C=2)
    args = _dev(inp, inp.z, inp.P, bands)
    kw = dict(n_sim=2, n_fd=1, precision="fp64", max_iter=5)
    for bad in (dict(leak_split=2 * nb), dict(leak_split=-1), dict(leak_split=nb, fd_bands=[0, nb]),
                dict(leak_split=1, trunc=(2, 0))):
        with pytest.raises(wf.WfError, match="EINVAL"):
            wf.bandpower_estimate(*args, 2 * nb, None, None, None, **kw, **bad)
    one = synth.density_small(n, seed=2)
    b1 = synth.log_bands(n, 3)
    with pytest.raises(wf.WfError, match="EINVAL"):  # one channel: no E/B split
        wf.bandpower_estimate(*_dev(one, one.z, one.P, b1), 3, None, None, None, leak_split=1, **kw)
    with pytest.raises(ValueError, match="Fisher rows"):
        z = torch.zeros((2, 2, n, n), dtype=torch.float64, device="cuda")
        u = torch.zeros((2 * nb, 1, 2, n, n), dtype=torch.float64, device="cuda")
        wf.bandpower_estimate(*args, 2 * nb, z, z, u, leak_split=nb, precision="fp64", max_iter=5)


def test_iterate_on_a_rectangular_map_matches_oracle_iteration():
    """bandpower_iterate_rect on a 16 x 32 map: every estimate's Theta_hat and
    the final fiducial as the oracle's iteration on the same grid."""
    ny, nx, nb, J, nfd, n_iter = 16, 32, 3, 6, 3, 2
    inp = synth.density_small(ny, seed=14, masked_frac=0.2, nx=nx)
    d = O.synthesize_data(inp.z, inp.noise, inp.mask, inp.P)
    bands = synth.log_bands(ny, nb, nx=nx)
    P0 = inp.P.copy()
    for lb, f in enumerate((0.3, 1.0, 2.5)):
        P0[bands == lb] *= f
    rng = np.random.default_rng(6)
    sig = np.where(inp.Ninv > 0, 1.0 / np.sqrt(np.where(inp.Ninv > 0, inp.Ninv, 1.0)), 0.0)
    z = rng.standard_normal((J, 1, ny, nx))
    nz = rng.standard_normal((J, 1, ny, nx)) * sig
    u = rng.standard_normal((nb, nfd, 1, ny, nx))
    dt, h1 = torch.float64, nx // 2 + 1
    res, stats, hist, Pf = wf.bandpower_iterate(
        to_dev(d, dt), to_dev(inp.mask, torch.uint8), to_dev(inp.Ninv, dt), to_dev(P0[..., :h1], dt),
        to_dev(bands[..., :h1], torch.int16), nb, to_dev(z, dt), to_dev(nz, dt), to_dev(u, dt), n_iter=n_iter,
        q_min=0.05, q_max=20.0, precision="fp64", gtol_rel=1e-12, max_iter=20000)
    ref, Pref = O.bandpower_iterate(d, inp.mask, inp.Ninv, P0, bands, nb, z, nz, u, n_iter, q_min=0.05, q_max=20.0,
                                    gtol_rel=1e-12, max_iter=20000)
    for it in range(n_iter):
        th = ref[it]["theta_hat"]
        assert np.abs(hist[it] - th).max() <= 1e-7 * np.abs(th).max(), (it, hist[it], th)
    assert np.abs(Pf.cpu().numpy() - Pref[..., :h1]).max() <= 1e-7 * np.abs(Pref).max()
    assert all(s["status"] == "WF_OK" for s in stats)
