"""Pins of the FP64 oracle against facts that do not come from the oracle itself:
textbook DFT definitions and closed forms, exact identities of a quadratic,
Woodbury agreement of two independent dense Wiener-filter forms, and analytic
band terms for an unmasked map with homogeneous noise."""
import os

import numpy as np
import pytest

from oracle import wf_oracle as O
from paper_1810_00503_gb300 import synth


def test_naive_dft_plane_wave_and_delta():
    # Unitary DFT of a delta is 1/n everywhere; of exp(+2 pi i (a y + b x)/n) it is n at (a, b).
    n = 8
    x = np.zeros((n, n)); x[0, 0] = 1.0
    assert np.allclose(O.dft2_naive(x), 1.0 / n, atol=1e-15)
    yy, xx = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    a, b = 3, 5
    w = np.exp(2j * np.pi * (a * yy + b * xx) / n)
    X = O.dft2_naive(w)
    ref = np.zeros((n, n), complex); ref[a, b] = n
    assert np.allclose(X, ref, atol=1e-12)


@pytest.mark.parametrize("n", [2, 4, 8])
def test_fft_matches_naive_dft(n):
    rng = np.random.default_rng(n)
    x = rng.standard_normal((2, n, n)) + 1j * rng.standard_normal((2, n, n))
    assert np.allclose(O.fft2u(x), O.dft2_naive(x), atol=1e-13, rtol=0)


def test_parseval_and_roundtrip():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((1, 32, 32))
    X = O.fft2u(x)
    assert np.isclose(np.sum(np.abs(X) ** 2), np.sum(x * x), rtol=1e-14)
    assert np.allclose(O.ifft2u(X).real, x, atol=1e-14)


def test_operator_identity_and_adjoint():
    n = 16
    rng = np.random.default_rng(2)
    z = rng.standard_normal((1, n, n))
    assert np.allclose(O.apply_A(z, np.ones((1, n, n))), z, atol=1e-14)
    for C in (1, 2):
        P = rng.uniform(0.1, 2.0, size=(C, n, n))
        P = 0.5 * (P + P[:, (-np.arange(n)) % n][:, :, (-np.arange(n)) % n])  # even in k
        a = rng.standard_normal((C, n, n)); b = rng.standard_normal((C, n, n))
        lhs = np.sum(O.apply_A(a, P) * b)
        rhs = np.sum(a * O.apply_At(b, P))
        assert np.isclose(lhs, rhs, rtol=1e-12)
        # a real field stays real: the imaginary part before .real is round-off only
        Z = O.fft2u(a) * np.sqrt(P)
        assert np.abs(O.ifft2u(Z).imag).max() < 1e-12


def test_ks_rotation_plane_wave_closed_form():
    # Pure E-mode cosine wave with unit power on one mode pair: gamma1 = c phi,
    # gamma2 = s phi with c = (kx^2-ky^2)/k^2, s = 2 kx ky / k^2 (App. C operator
    # divided by -k^2).  Pins orientation (x = last axis) and sign.
    n = 16
    ky, kx = 2, 3
    yy, xx = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    phi = np.cos(2 * np.pi * (ky * yy + kx * xx) / n)
    z = np.stack([phi, np.zeros_like(phi)])
    g = O.apply_A(z, np.ones((2, n, n)))
    k2 = kx * kx + ky * ky
    assert np.allclose(g[0], (kx * kx - ky * ky) / k2 * phi, atol=1e-13)
    assert np.allclose(g[1], 2 * kx * ky / k2 * phi, atol=1e-13)
    # and a pure B mode rotates the other way
    zb = np.stack([np.zeros_like(phi), phi])
    gb = O.apply_A(zb, np.ones((2, n, n)))
    assert np.allclose(gb[0], -2 * kx * ky / k2 * phi, atol=1e-13)
    assert np.allclose(gb[1], (kx * kx - ky * ky) / k2 * phi, atol=1e-13)


def test_ks_rotation_orthogonal_off_nyquist():
    n = 16
    c, s = O.ks_rotation(n)
    my, mx = O.signed_modes(n)
    off = (np.abs(mx) != n // 2) & (np.abs(my) != n // 2)
    assert np.allclose((c * c + s * s)[off], 1.0, atol=1e-15)
    assert np.all(s[~off] == 0)


@pytest.mark.parametrize("C", [1, 2])
def test_gradient_is_exact_central_difference(C):
    # chi^2 is quadratic, so (f(z+hv) - f(z-hv)) / 2h equals g.v up to round-off.
    n = 16
    inp = synth.density_small(n, seed=5) if C == 1 else synth.shear_eb(n, seed=5)
    W = inp.mask[None] * inp.Ninv
    d = O.synthesize_data(inp.z, inp.noise, inp.mask, inp.P)
    rng = np.random.default_rng(7)
    z = rng.standard_normal(d.shape)
    g = O.grad(z, d, W, inp.P)
    f0 = O.chi2(z, d, W, inp.P)
    h = 1e-3
    for _ in range(20):
        v = rng.standard_normal(d.shape)
        fd = (O.chi2(z + h * v, d, W, inp.P) - O.chi2(z - h * v, d, W, inp.P)) / (2 * h)
        assert abs(fd - np.sum(g * v)) <= 1e-13 * abs(f0) / h + 1e-9 * abs(fd)


def test_hessian_vector_is_gradient_difference():
    n = 16
    inp = synth.density_small(n, seed=3)
    W = inp.mask[None] * inp.Ninv
    d = O.synthesize_data(inp.z, inp.noise, inp.mask, inp.P)
    rng = np.random.default_rng(3)
    z = rng.standard_normal(d.shape); v = rng.standard_normal(d.shape)
    lhs = O.grad(z + v, d, W, inp.P) - O.grad(z, d, W, inp.P)
    assert np.allclose(lhs, O.hess_vec(v, W, inp.P), rtol=1e-11, atol=1e-9)


def test_unmasked_homogeneous_closed_form():
    # No mask, constant noise sigma^2: z*_m = sqrt(P_m) d_m / (P_m + sigma^2) per mode
    # (the S / (S + N) filter of App. A in whitened variables).
    n, sig2 = 32, 0.3
    inp = synth.density_small(n, seed=11)
    mask = np.ones((n, n), np.uint8)
    W = np.full((1, n, n), 1.0 / sig2)
    d = O.synthesize_data(inp.z, np.sqrt(sig2) * inp.z[::-1], mask, inp.P)
    D = O.fft2u(d)
    zstar = O.ifft2u(np.sqrt(inp.P) * D / (inp.P + sig2)).real
    z_dense = O.dense_wf_whitened(d, W, inp.P)
    assert np.linalg.norm(z_dense - zstar) <= 1e-12 * np.linalg.norm(zstar)
    z_lb, info = O.map_solve(d, W, inp.P, gtol_rel=1e-12)
    assert info["status"] == "converged"
    assert np.linalg.norm(z_lb - zstar) <= 1e-10 * np.linalg.norm(zstar)


def test_dense_forms_agree_woodbury_and_lbfgs():
    inp = synth.density_small(32, seed=0)
    W = inp.mask[None] * inp.Ninv
    d = O.synthesize_data(inp.z, inp.noise, inp.mask, inp.P)
    A = O.dense_operator(inp.P)
    z1 = O.dense_wf_whitened(d, W, inp.P, A=A)
    x2, z2 = O.dense_wf_covariance(d, inp.mask, inp.Ninv, inp.P, A=A)
    assert np.linalg.norm(z1 - z2) <= 1e-11 * np.linalg.norm(z1)
    assert np.allclose(O.apply_A(z1, inp.P), x2, rtol=0, atol=1e-10 * np.abs(x2).max())
    # chi^2 at the minimiser equals d_o^T C^-1 d_o
    assert np.isclose(O.chi2(z1, d, W, inp.P), O.chi2_min_dense(d, inp.mask, inp.Ninv, inp.P, A=A),
                      rtol=1e-11)
    # textbook L-BFGS reaches the same point; certificate ||z - z*|| <= ||grad|| / 2
    zl, info = O.map_solve(d, W, inp.P, m=10, gtol_rel=1e-12, max_iter=5000)
    gl = O.grad(zl, d, W, inp.P)
    err = np.linalg.norm(zl - z1)
    assert err <= 0.5 * np.linalg.norm(gl) * (1 + 1e-6) + 1e-13 * np.linalg.norm(z1)
    assert err <= 1e-10 * np.linalg.norm(z1)


def test_certificate_bound_is_tight_enough_and_valid():
    # lambda_min of the half-Hessian I + A^T W A is >= 1, so ||z - z*|| <= ||g|| / 2
    inp = synth.density_small(16, seed=4)
    W = inp.mask[None] * inp.Ninv
    d = O.synthesize_data(inp.z, inp.noise, inp.mask, inp.P)
    zs = O.dense_wf_whitened(d, W, inp.P)
    rng = np.random.default_rng(0)
    for _ in range(5):
        z = zs + 1e-3 * rng.standard_normal(zs.shape)
        g = O.grad(z, d, W, inp.P)
        assert np.linalg.norm(z - zs) <= 0.5 * np.linalg.norm(g) * (1 + 1e-12)


def test_exact_step_minimises_along_line():
    inp = synth.density_small(16, seed=6)
    W = inp.mask[None] * inp.Ninv
    d = O.synthesize_data(inp.z, inp.noise, inp.mask, inp.P)
    rng = np.random.default_rng(1)
    z = rng.standard_normal(d.shape); p = rng.standard_normal(d.shape)
    g = O.grad(z, d, W, inp.P)
    a = O.exact_step(g, p, W, inp.P)
    g_new = O.grad(z + a * p, d, W, inp.P)
    assert abs(np.sum(g_new * p)) <= 1e-10 * np.linalg.norm(g) * np.linalg.norm(p)


def test_exact_band_terms_unmasked_closed_form():
    # No mask, homogeneous noise: C is diagonal in Fourier with P_m + sigma^2, so
    # b_l = (1/2 Theta_l) sum_{m in l} P_m / (P_m + s2),
    # F_ll' = delta_ll' (1/2 Theta_l^2) sum_{m in l} P_m^2 / (P_m + s2)^2.
    n, s2, nb = 8, 0.5, 3
    inp = synth.density_small(n, seed=2)
    mask = np.ones((n, n), np.uint8)
    Ninv = np.full((1, n, n), 1.0 / s2)
    bands = synth.log_bands(n, nb)
    b, F, th = O.exact_band_terms(mask, Ninv, inp.P, bands, nb)
    P = inp.P
    for l in range(nb):
        sel = bands == l
        assert np.isclose(b[l], 0.5 / th[l] * np.sum(P[sel] / (P[sel] + s2)), rtol=1e-11)
        assert np.isclose(F[l, l], 0.5 / th[l] ** 2 * np.sum(P[sel] ** 2 / (P[sel] + s2) ** 2),
                          rtol=1e-11)
    off = F - np.diag(np.diag(F))
    assert np.abs(off).max() <= 1e-12 * np.abs(F).max()


@pytest.mark.slow
def test_simulated_band_terms_match_exact_traces():
    # b from simulations (eq. blmv) and F by finite differences (eq. fisher) agree with
    # the exact traces of eq:wf_exact_f within Monte-Carlo error; the sample covariance
    # of E over the simulations agrees with F (Fisher identity).
    n, nb, J = 8, 3, 400
    inp = synth.density_small(n, seed=9, masked_frac=0.25)
    bands = synth.log_bands(n, nb)
    rng = np.random.default_rng(21)
    z_s = rng.standard_normal((J, 1, n, n))
    n_s = rng.standard_normal((J, 1, n, n)) / np.sqrt(np.where(inp.Ninv > 0, inp.Ninv, 1.0))
    u_fd = rng.standard_normal((nb, J, 1, n, n))
    d = O.synthesize_data(inp.z, inp.noise, inp.mask, inp.P)
    res = O.bandpower_sims(d, inp.mask, inp.Ninv, inp.P, bands, nb, z_s, n_s, u_fd,
                           gtol_rel=1e-9)
    b_ex, F_ex, th = O.exact_band_terms(inp.mask, inp.Ninv, inp.P, bands, nb)
    # MC standard error of b_l is sqrt(F_ll / J) (Var E_l = F_ll at the fiducial)
    se_b = np.sqrt(np.diag(F_ex) / J)
    assert np.all(np.abs(res["b"] - b_ex) <= 5 * se_b)
    # finite-difference F: each entry is a mean of J cross terms; loose 5-sigma-ish bound
    assert np.allclose(res["F"], F_ex, rtol=0.25, atol=0.1 * np.abs(F_ex).max())
    assert np.allclose(res["cov_E"], F_ex, rtol=0.3, atol=0.1 * np.abs(F_ex).max())


@pytest.mark.parametrize("C", [1, 2])
def test_band_amplitude_derivative_matches_finite_differences(C):
    # chi^2(log q) is smooth; central differences with step 1e-4 agree to O(h^2).
    n, nb = 16, 3
    inp = synth.density_small(n, seed=8) if C == 1 else synth.shear_eb(n, seed=8)
    W = inp.mask[None] * inp.Ninv
    d = O.synthesize_data(inp.z, inp.noise, inp.mask, inp.P)
    bands = synth.log_bands(n, nb, C=C)
    rng = np.random.default_rng(4)
    z = rng.standard_normal(d.shape)
    an = O.chi2_dlogq(z, d, W, inp.P, bands, nb * C)
    h = 1e-4
    for l in range(nb * C):
        up = np.where(bands == l, np.exp(h), 1.0) * inp.P
        dn = np.where(bands == l, np.exp(-h), 1.0) * inp.P
        fd = (O.chi2(z, d, W, up) - O.chi2(z, d, W, dn)) / (2 * h)
        assert abs(fd - an[l]) <= 1e-6 * max(abs(an).max(), 1.0), (l, fd, an[l])


# ---------------------------------------------------------------------------
# Counter-based normal deviates (oracle/philox.py)
# ---------------------------------------------------------------------------
def _kat_rows():
    path = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")
    rows = []
    for line in open(path):
        line = line.strip()
        if line and not line.startswith("#"):
            rows.append([int(w, 16) for w in line.split()])
    return rows


def test_philox_known_answer_vectors():
    from oracle.philox import philox4x32_10
    rows = _kat_rows()
    assert len(rows) == 3
    for r in rows:
        out = philox4x32_10([np.array([c]) for c in r[:4]], r[4:6])
        assert [int(o[0]) for o in out] == r[6:10]


def test_philox_normals_box_muller_pairs_and_moments():
    from oracle.philox import MASK32, normals, philox4x32_10
    z = normals(11, 3, 400000)
    # moments of N(0, 1) within 6 sigma of their sampling error
    n = z.size
    assert abs(z.mean()) < 6 / np.sqrt(n)
    assert abs(z.var() - 1) < 6 * np.sqrt(2 / n)
    assert abs(np.mean(z ** 4) - 3) < 6 * np.sqrt(96 / n)
    # a pair (2j, 2j+1) lies on the circle of radius sqrt(-2 ln u1) of block j
    j = 12345
    x = philox4x32_10((np.array([j]), np.array([0]), np.array([3]), np.array([0])), (11, 0))
    u1 = ((int(x[0][0]) >> 5) * 67108864.0 + (int(x[1][0]) >> 6) + 0.5) * 2.0 ** -53
    assert abs(z[2 * j] ** 2 + z[2 * j + 1] ** 2 + 2 * np.log(u1)) < 1e-12
    # offsets address the same stream; streams and seeds differ
    assert np.array_equal(normals(11, 3, 10, offset=2 * j), z[2 * j: 2 * j + 10])
    assert not np.allclose(normals(11, 4, 10), z[:10])
    assert not np.allclose(normals(12, 3, 10), z[:10])
    assert MASK32 == 2 ** 32 - 1


def test_exact_band_terms_unmasked_closed_form_eb():
    """Joint E/B (C = 2) with separate E and B band ids, no mask, isotropic
    noise: the rotation R(k) is orthogonal off the Nyquist lines and c I on them,
    so each channel is filtered on its own with effective power P_eff = P (c^2 P
    on the Nyquist lines) and the band terms take the C = 1 closed forms."""
    n, s2, nb = 8, 0.5, 2
    inp = synth.shear_eb(n, seed=4)
    mask = np.ones((n, n), np.uint8)
    Ninv = np.full((2, n, n), 1.0 / s2)
    b1 = synth.log_bands(n, nb)[0]
    bands = np.stack([b1, np.where(b1 >= 0, b1 + nb, -1)])
    b, F, th = O.exact_band_terms(mask, Ninv, inp.P, bands, 2 * nb)
    c, _ = O.ks_rotation(n)
    my, mx = O.signed_modes(n)
    nyq = (np.abs(mx) == n // 2) | (np.abs(my) == n // 2)
    Peff = inp.P * np.where(nyq, c * c, 1.0)[None]
    for l in range(2 * nb):
        sel = bands == l
        assert np.isclose(th[l], inp.P[sel].mean(), rtol=1e-12)
        assert np.isclose(b[l], 0.5 / th[l] * np.sum(Peff[sel] / (Peff[sel] + s2)), rtol=1e-10)
        assert np.isclose(F[l, l], 0.5 / th[l] ** 2 * np.sum(Peff[sel] ** 2 / (Peff[sel] + s2) ** 2), rtol=1e-10)
    off = F - np.diag(np.diag(F))
    assert np.abs(off).max() <= 1e-11 * np.abs(F).max()


def test_iterated_fiducial_update_rule():
    """Each re-estimate starts from the previous fiducial times the clamped ratio
    of estimate to fiducial on every band's modes; modes outside the bands keep
    their power."""
    n, nb, J, nfd = 8, 2, 3, 2
    inp = synth.density_small(n, seed=3)
    bands = synth.log_bands(n, nb)
    rng = np.random.default_rng(4)
    sig = np.where(inp.Ninv > 0, 1.0 / np.sqrt(np.where(inp.Ninv > 0, inp.Ninv, 1.0)), 0.0)
    z = rng.standard_normal((J, 1, n, n))
    nz = rng.standard_normal((J, 1, n, n)) * sig
    u = rng.standard_normal((nb, nfd, 1, n, n))
    d = O.synthesize_data(inp.z, inp.noise, inp.mask, inp.P)
    P0 = inp.P * 0.3
    res, Pf = O.bandpower_iterate(d, inp.mask, inp.Ninv, P0, bands, nb, z, nz, u, 2, q_min=0.5, q_max=2.0,
                                  gtol_rel=1e-12)
    assert len(res) == 2
    q = np.clip(res[0]["theta_hat"] / res[0]["theta_fid"], 0.5, 2.0)
    want = P0.copy()
    for l in range(nb):
        want[bands == l] *= q[l]
    assert np.array_equal(Pf, want)
    assert np.allclose(res[1]["theta_fid"], res[0]["theta_fid"] * q, rtol=1e-12)
    outside = bands < 0
    assert np.array_equal(Pf[outside], P0[outside])


def test_fisher_column_interpolation_rule():
    """fisher_fill_columns: sampled columns are kept; on a matrix that is exactly
    translation invariant with a factor linear in the column, F[l][l'] =
    f(l - l') (a + b l'), interpolated columns are exact where both shifted rows
    exist; with every band sampled nothing changes."""
    nb = 9
    f = lambda o: np.exp(-abs(o) / 1.5) * (1.0 if o >= 0 else 0.7)
    F = np.array([[f(l - lp) * (2.0 + 0.3 * lp) for lp in range(nb)] for l in range(nb)])
    S = [0, 2, 5, 8]
    G = O.fisher_fill_columns(F * np.isin(np.arange(nb), S)[None, :], S)
    for lp in S:
        assert np.array_equal(G[:, lp], F[:, lp])
    for lp in (1, 3, 4, 6, 7):
        s0 = max(s for s in S if s < lp)
        s1 = min(s for s in S if s > lp)
        for l in range(nb):
            o = l - lp
            if 0 <= s0 + o < nb and 0 <= s1 + o < nb:
                assert np.isclose(G[l, lp], F[l, lp], rtol=1e-12), (l, lp)
    assert np.array_equal(O.fisher_fill_columns(F, list(range(nb))), F)
    # outside the sampled range the nearest column is shifted
    G2 = O.fisher_fill_columns(F * np.isin(np.arange(nb), [2, 5])[None, :], [2, 5])
    assert np.isclose(G2[1, 0], F[3, 2]) and np.isclose(G2[8, 7], F[6, 5])


def test_fisher_truncation_rule():
    F = np.arange(1.0, 37.0).reshape(6, 6)
    G = O.fisher_truncate(F, 4, 1)
    for l in range(6):
        for lp in range(6):
            zeroed = l < 4 and lp < 4 and abs(l - lp) > 1
            assert G[l, lp] == (0.0 if zeroed else F[l, lp])


def _eb_leak_case(n, nb, J, nfd, seed, full_sky):
    """E/B inputs with E bands 0..nb-1 and B bands nb..2nb-1, fields for the
    full Fisher run (one row per band, every B band given the same field u_B)
    and for the leakage-bias run (the E rows, then u_B)."""
    inp = synth.shear_eb(n, seed=seed)
    rng = np.random.default_rng(seed + 100)
    if full_sky:
        mask = np.ones((n, n), np.uint8)
        Ninv = np.full((2, n, n), 2.0)
    else:
        mask, Ninv = inp.mask, inp.Ninv
    sig = np.where(Ninv > 0, 1.0 / np.sqrt(np.where(Ninv > 0, Ninv, 1.0)), 0.0)
    d = O.synthesize_data(inp.z, rng.standard_normal((2, n, n)) * sig, mask, inp.P)
    b1 = synth.log_bands(n, nb)[0]
    bands = np.stack([b1, np.where(b1 >= 0, b1 + nb, -1)])
    z = rng.standard_normal((J, 2, n, n))
    nz = rng.standard_normal((J, 2, n, n)) * sig
    uE = rng.standard_normal((nb, nfd, 2, n, n))
    uB = rng.standard_normal((1, nfd, 2, n, n))
    u_full = np.concatenate([uE] + [uB] * nb)
    u_leak = np.concatenate([uE, uB])
    return d, mask, Ninv, inp.P, bands, z, nz, u_full, u_leak


def test_leakage_bias_equals_full_fisher_when_nothing_leaks():
    """App. C leakage-bias alternative.  Without a mask and with isotropic
    noise, E and B do not mix (R(k) orthogonal, c I on the Nyquist lines) and
    the Hessian is diagonal per mode, so a B injection moves only its own
    band's modes: the joint B map's response in band l equals the per-band
    map's when both use the same field, and the full Fisher matrix is diagonal
    in its B block with empty cross blocks.  Both estimates must then agree."""
    n, nb, J, nfd = 8, 2, 3, 2
    d, mask, Ninv, P, bands, z, nz, u_full, u_leak = _eb_leak_case(n, nb, J, nfd, 31, True)
    kw = dict(gtol_rel=1e-12, max_iter=20000)
    full = O.bandpower_sims(d, mask, Ninv, P, bands, 2 * nb, z, nz, u_full, **kw)
    leak = O.bandpower_sims(d, mask, Ninv, P, bands, 2 * nb, z, nz, u_leak, leak_split=nb, **kw)
    F, G = full["F"], leak["F"]
    scale = np.abs(F).max()
    assert np.abs(F - G).max() <= 1e-8 * scale, (F, G)
    assert np.all(np.diag(G)[nb:] > 0.0)
    assert np.allclose(leak["theta_hat"], full["theta_hat"], rtol=1e-7, atol=0.0)
    assert np.array_equal(leak["b"], full["b"])


def test_leakage_bias_blocks_under_a_mask():
    """Under a mask the full Fisher matrix has E-B cross terms; the
    leakage-bias form keeps the full EE block, drops the cross blocks and the
    BB off-diagonal, so the E estimates do not depend on the B fields."""
    n, nb, J, nfd = 8, 2, 3, 2
    d, mask, Ninv, P, bands, z, nz, u_full, u_leak = _eb_leak_case(n, nb, J, nfd, 32, False)
    kw = dict(gtol_rel=1e-12, max_iter=20000)
    full = O.bandpower_sims(d, mask, Ninv, P, bands, 2 * nb, z, nz, u_full, **kw)
    leak = O.bandpower_sims(d, mask, Ninv, P, bands, 2 * nb, z, nz, u_leak, leak_split=nb, **kw)
    F, G = full["F"], leak["F"]
    assert np.abs(F[:nb, nb:]).max() > 1e-6 * np.abs(F).max()      # the mask mixes E and B
    assert np.abs(F[nb:, :nb]).max() > 1e-6 * np.abs(F).max()
    assert np.array_equal(G[:nb, :nb], F[:nb, :nb])
    assert not G[:nb, nb:].any() and not G[nb:, :nb].any()
    assert np.array_equal(G[nb:, nb:], np.diag(np.diag(G)[nb:]))
    u2 = u_leak.copy()
    u2[nb] = np.random.default_rng(5).standard_normal(u2[nb].shape)
    leak2 = O.bandpower_sims(d, mask, Ninv, P, bands, 2 * nb, z, nz, u2, leak_split=nb, **kw)
    assert np.array_equal(leak2["theta_hat"][:nb], leak["theta_hat"][:nb])
    assert not np.allclose(leak2["theta_hat"][nb:], leak["theta_hat"][nb:], rtol=1e-6)


# ---------------------------------------------------------------------------
# Textbook L-BFGS pieces (Nocedal & Wright): two-loop recursion against the
# dense inverse-Hessian update, and the strong-Wolfe conditions of the search
# ---------------------------------------------------------------------------


def test_two_loop_equals_dense_bfgs_inverse_update():
    """-two_loop(g) = H g with H built densely by the BFGS inverse update
    H <- V^T H V + rho s s^T, V = I - rho y s^T (N&W eq. 6.17), from
    H0 = gamma I, gamma = s^T y / y^T y of the newest pair (N&W eq. 7.20);
    and H satisfies the secant condition H y = s for the newest pair."""
    rng = np.random.default_rng(12)
    dim, m = 9, 4
    A = rng.standard_normal((dim, dim))
    Hs = A @ A.T + dim * np.eye(dim)            # SPD, so s^T y > 0
    S = [rng.standard_normal(dim) for _ in range(m)]
    Y = [Hs @ s for s in S]
    g = rng.standard_normal(dim)
    gamma = S[-1] @ Y[-1] / (Y[-1] @ Y[-1])
    H = gamma * np.eye(dim)
    for s, y in zip(S, Y):
        rho = 1.0 / (y @ s)
        V = np.eye(dim) - rho * np.outer(y, s)
        H = V.T @ H @ V + rho * np.outer(s, s)
    p = O._two_loop(g, S, Y)
    assert np.allclose(-p, H @ g, rtol=1e-12, atol=1e-12 * np.abs(H @ g).max())
    assert np.allclose(H @ Y[-1], S[-1], rtol=1e-10)
    assert np.allclose(O._two_loop(g, [], []), -g)    # no pairs: steepest descent


@pytest.mark.parametrize("case", ["accept_unit", "expand", "zoom"])
def test_line_search_returns_a_strong_wolfe_step(case):
    """On phi(a) = f(x + a p) for a quadratic f, the returned step satisfies
    f(a) <= f(0) + c1 a phi'(0) and |phi'(a)| <= c2 |phi'(0)| (N&W eq. 3.7);
    a unit step that already does is returned unchanged (Alg. 3.5 tries 1 first)."""
    c1, c2 = 1e-4, {"accept_unit": 0.9, "expand": 0.1, "zoom": 0.1}[case]
    a_star = {"accept_unit": 1.2, "expand": 9.0, "zoom": 0.3}[case]  # minimiser along p
    dim = 5
    rng = np.random.default_rng(4)
    Q = np.diag(rng.uniform(1.0, 3.0, dim))
    x = rng.standard_normal(dim)
    g0 = Q @ x
    p = -g0 * (1.0 / a_star) * (g0 @ g0) / (g0 @ Q @ g0)  # exact minimiser at a = a_star

    def fg(v):
        return 0.5 * v @ Q @ v, Q @ v

    f0 = fg(x)[0]
    a, f, g = O._line_search(fg, x, f0, g0, p, c1, c2)
    d0 = g0 @ p
    fa, ga = fg(x + a * p)
    assert fa <= f0 + c1 * a * d0 + 1e-14 * abs(f0)
    assert abs(ga @ p) <= c2 * abs(d0) * (1 + 1e-12)
    assert np.isclose(f, fa, rtol=1e-14)
    if case == "accept_unit":
        assert a == 1.0
    else:
        assert abs(a - a_star) <= 0.1 * a_star         # c2 = 0.1 pins the step near the minimiser


@pytest.mark.parametrize("C", [1, 2])
def test_envelope_identity_at_the_map(C):
    """At the MAP the gradient vanishes, z = A^T W r, so the band derivative
    d chi^2 / d log q_l = -r^T W A Pi_l z reduces to -z^T Pi_l z =
    -2 Theta_fid,l E_l(z_MAP): the adjoint band derivative and the band energy
    of eq. el agree at the solution, up to O(||g||), and not elsewhere."""
    n, nb = 16, 3
    inp = synth.density_small(n, seed=17) if C == 1 else synth.shear_eb(n, seed=17)
    W = inp.mask[None] * inp.Ninv
    d = O.synthesize_data(inp.z, inp.noise, inp.mask, inp.P)
    bands = synth.log_bands(n, nb, C=C)
    nbt = nb * C
    z, _ = O.map_solve(d, W, inp.P, m=10, gtol_rel=1e-13, max_iter=20000)
    theta = O.theta_fid(inp.P, bands, nbt)
    lhs = O.chi2_dlogq(z, d, W, inp.P, bands, nbt)
    rhs = -2.0 * theta * O.band_E(z, bands, theta, nbt)
    assert np.allclose(lhs, rhs, rtol=1e-8, atol=1e-10 * np.abs(rhs).max()), (lhs, rhs)
    z2 = z + 0.1 * np.random.default_rng(1).standard_normal(z.shape)
    assert not np.allclose(O.chi2_dlogq(z2, d, W, inp.P, bands, nbt),
                           -2.0 * theta * O.band_E(z2, bands, theta, nbt), rtol=1e-3)


def test_chi2_minimum_is_chi_square_distributed():
    """For data drawn from the model, d = M (A z + n) with z ~ N(0, I) and
    n ~ N(0, N), the observed pixels have covariance C = A_o A_o^T + N_o, so
    chi^2_min = d_o^T C^-1 d_o is chi-square with N_obs degrees of freedom:
    mean N_obs, variance 2 N_obs (checked within 4 and 5 standard errors).  A
    white signal spectrum at the mean noise level gives signal and noise about
    half of the degrees of freedom each, so a mis-scaled signal or noise term
    moves the mean by many standard errors."""
    n, K = 16, 300
    inp = synth.density_small(n, seed=23, masked_frac=0.25)
    obs = inp.mask == 1
    P = np.full((1, n, n), float(np.mean(1.0 / inp.Ninv[0][obs])))
    P[0, 0, 0] = 0.0
    A = O.dense_operator(P)
    nobs = int(obs.sum())
    rng = np.random.default_rng(7)
    sig = np.where(inp.Ninv > 0, 1.0 / np.sqrt(np.where(inp.Ninv > 0, inp.Ninv, 1.0)), 0.0)
    vals = np.array([O.chi2_min_dense(O.synthesize_data(rng.standard_normal((1, n, n)),
                                                        rng.standard_normal((1, n, n)) * sig, inp.mask, P),
                                      inp.mask, inp.Ninv, P, A=A) for _ in range(K)])
    assert abs(vals.mean() - nobs) <= 4.0 * np.sqrt(2.0 * nobs / K), (vals.mean(), nobs)
    assert abs(vals.var(ddof=1) - 2.0 * nobs) <= 5.0 * np.sqrt(2.0 / K) * 2.0 * nobs, (vals.var(ddof=1), nobs)


def test_estimator_is_unbiased_for_a_rescaled_true_spectrum():
    """With the exact b and F, <E_l> over data drawn with any band powers is
    b_l + sum_l' F_ll' (Theta_true,l' - Theta_fid,l'), because E is quadratic in
    the data and C is linear in the band powers; so Theta_hat = Theta_fid +
    F^-1 (E - b) (eq. eq:wfmv) averages to Theta_true.  Data drawn with each
    band of the fiducial rescaled; mean of Theta_hat within 5 standard errors."""
    n, nb, K = 8, 3, 4000
    inp = synth.density_small(n, seed=29, masked_frac=0.25)
    bands = synth.log_bands(n, nb)
    q = np.array([1.6, 0.6, 1.3])
    P_true = inp.P * np.where(bands >= 0, q[np.maximum(bands, 0)], 1.0)
    b, F, theta = O.exact_band_terms(inp.mask, inp.Ninv, inp.P, bands, nb)
    W = inp.mask[None] * inp.Ninv
    A = O.dense_operator(inp.P)
    sig = np.where(inp.Ninv > 0, 1.0 / np.sqrt(np.where(inp.Ninv > 0, inp.Ninv, 1.0)), 0.0)
    rng = np.random.default_rng(31)
    est = np.empty((K, nb))
    for k in range(K):
        d = O.synthesize_data(rng.standard_normal((1, n, n)), rng.standard_normal((1, n, n)) * sig, inp.mask,
                              P_true)
        z = O.dense_wf_whitened(d, W, inp.P, A=A)
        est[k] = theta + np.linalg.solve(F, O.band_E(z, bands, theta, nb) - b)
    se = est.std(axis=0, ddof=1) / np.sqrt(K)
    assert np.all(np.abs(est.mean(axis=0) - theta * q) <= 5.0 * se), (est.mean(axis=0), theta * q, se)
    assert np.any(np.abs(est.mean(axis=0) - theta) > 5.0 * se)     # distinguishable from the fiducial


# ---------------------------------------------------------------------------
# Rectangular and non-power-of-two grids (the oracle side of such maps)
# ---------------------------------------------------------------------------

RECT = [(4, 6), (5, 3), (6, 10), (7, 7), (9, 12)]


@pytest.mark.parametrize("shape", RECT)
def test_dft_rectangular_plane_wave_and_fft(shape):
    """The naive DFT maps a plane wave exp(2 pi i (a y / ny + b x / nx)) to
    sqrt(ny nx) at mode (a, b) and zero elsewhere; the FFT path agrees with it."""
    ny, nx = shape
    a, b = 1 % ny, (nx - 2) % nx
    y, x = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    wave = np.exp(2j * np.pi * (a * y / ny + b * x / nx))[None]
    X = O.dft2_naive(wave)
    want = np.zeros((1, ny, nx), complex)
    want[0, a, b] = np.sqrt(ny * nx)
    assert np.allclose(X, want, atol=1e-12)
    r = np.random.default_rng(sum(shape)).standard_normal((2, ny, nx))
    assert np.allclose(O.fft2u(r), O.dft2_naive(r), atol=1e-12)


@pytest.mark.parametrize("shape", [(6, 10), (5, 7), (8, 16), (16, 8), (9, 12)])
def test_ks_rotation_rectangular_shears_a_plane_wave_potential(shape):
    """On a grid of square pixels, a lensing potential psi = cos(kx x + ky y)
    with (kx, ky) = 2 pi (b / nx, a / ny) per pixel has convergence
    kappa = (psi_xx + psi_yy) / 2 and shear gamma1 = (psi_xx - psi_yy) / 2,
    gamma2 = psi_xy (App. C), all from the derivatives of the wave itself.  An
    E field equal to kappa must come out of the operator as that shear; a B
    field rotates the other way.  Pins the wavevector of a mode on a
    rectangular grid, not only its mode numbers."""
    ny, nx = shape
    a, b = 1, 2  # off both Nyquist lines
    y, x = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    kx, ky = 2 * np.pi * b / nx, 2 * np.pi * a / ny
    psi = np.cos(kx * x + ky * y)
    kappa = -0.5 * (kx * kx + ky * ky) * psi
    g1, g2 = -0.5 * (kx * kx - ky * ky) * psi, -kx * ky * psi
    zero = np.zeros_like(psi)
    out = O.apply_A(np.stack([kappa, zero]), np.ones((2, ny, nx)))
    assert np.allclose(out[0], g1, atol=1e-12) and np.allclose(out[1], g2, atol=1e-12)
    outb = O.apply_A(np.stack([zero, kappa]), np.ones((2, ny, nx)))
    assert np.allclose(outb[0], -g2, atol=1e-12) and np.allclose(outb[1], g1, atol=1e-12)


@pytest.mark.parametrize("shape", RECT)
def test_ks_rotation_rectangular_symmetry_and_nyquist(shape):
    """c and s are even under k -> -k on the grid, which is what keeps A z
    real; s = 0 on a Nyquist line (a Nyquist mode is its own negative, where s
    is odd), and an odd side has none, so there c^2 + s^2 = 1 everywhere but
    k = 0."""
    ny, nx = shape
    c, s = O.ks_rotation(ny, nx)
    my, mx = O.signed_modes(ny, nx)
    k2 = mx ** 2 + my ** 2
    nyq = ((nx % 2 == 0) & (np.abs(mx) == nx / 2)) | ((ny % 2 == 0) & (np.abs(my) == ny / 2))
    assert np.all(s[nyq] == 0)
    off = (k2 > 0) & ~nyq
    assert np.allclose(c[off] ** 2 + s[off] ** 2, 1.0, atol=1e-15)
    neg = (-np.arange(ny)) % ny, (-np.arange(nx)) % nx
    assert np.array_equal(c, c[neg[0]][:, neg[1]]) and np.array_equal(s, s[neg[0]][:, neg[1]])


def test_ks_rotation_square_grid_is_the_mode_number_form():
    """On a square grid the wavevector is proportional to the mode numbers, so
    the rotation is c = (mx^2 - my^2)/m^2, s = 2 mx my / m^2 bit for bit."""
    n = 16
    c, s = O.ks_rotation(n)
    my, mx = O.signed_modes(n)
    k2 = mx ** 2 + my ** 2
    nyq = (np.abs(mx) == n / 2) | (np.abs(my) == n / 2)
    off = (k2 > 0) & ~nyq
    assert np.array_equal(c[off], (mx[off] ** 2 - my[off] ** 2) / k2[off])
    assert np.array_equal(s[off], 2 * mx[off] * my[off] / k2[off])


@pytest.mark.parametrize("shape", [(6, 10), (5, 7), (9, 12)])
def test_unmasked_rectangular_map_is_s_over_s_plus_n(shape):
    """No mask, noise variance sigma^2 everywhere: the MAP is diagonal in
    Fourier space, z_hat = sqrt(P) d_hat / (P + sigma^2) (S/(S+N) for the
    signal), on rectangular and odd grids alike."""
    ny, nx = shape
    rng = np.random.default_rng(ny * nx)
    my, mx = O.signed_modes(ny, nx)
    P = (1.0 + np.hypot(my, mx))[None] ** -2.0 * 5.0
    s2 = 0.3
    mask = np.ones((ny, nx), np.uint8)
    Ninv = np.full((1, ny, nx), 1.0 / s2)
    d = O.synthesize_data(rng.standard_normal((1, ny, nx)), rng.standard_normal((1, ny, nx)) * np.sqrt(s2), mask, P)
    z = O.dense_wf_whitened(d, mask[None] * Ninv, P)
    want = O.ifft2u(np.sqrt(P) * O.fft2u(d) / (P + s2)).real
    assert np.allclose(z, want, rtol=0, atol=1e-12 * np.abs(want).max())


@pytest.mark.parametrize("shape", [(6, 10), (5, 7)])
def test_gradient_rectangular_eb_is_exact_central_difference(shape):
    """chi^2 is quadratic, so central differences equal g^T v up to rounding,
    here for the two-channel E/B operator on rectangular and odd grids."""
    ny, nx = shape
    rng = np.random.default_rng(3)
    my, mx = O.signed_modes(ny, nx)
    P = np.stack([(1.0 + np.hypot(my, mx)) ** -1.5, 0.1 * (1.0 + np.hypot(my, mx)) ** -1.5])
    W = (rng.uniform(size=(ny, nx)) > 0.3)[None] * rng.uniform(0.5, 2.0, size=(2, ny, nx))
    d = rng.standard_normal((2, ny, nx))
    z, v = rng.standard_normal((2, ny, nx)), rng.standard_normal((2, ny, nx))
    h = 1e-3
    fd = (O.chi2(z + h * v, d, W, P) - O.chi2(z - h * v, d, W, P)) / (2 * h)
    assert abs(fd - np.sum(O.grad(z, d, W, P) * v)) <= 1e-9 * abs(O.chi2(z, d, W, P))


@pytest.mark.parametrize("shape", [(6, 10), (5, 7)])
def test_exact_band_terms_rectangular_unmasked_closed_form(shape):
    """The band terms on rectangular and odd grids: no mask and homogeneous
    noise make C diagonal in Fourier space with P_m + sigma^2, so b_l and F_ll
    take the per-mode closed forms and F is diagonal, as on square maps."""
    ny, nx = shape
    s2, nb = 0.4, 3
    my, mx = O.signed_modes(ny, nx)
    k = np.hypot(my, mx)
    P = (2.0 * (1.0 + k) ** -1.7)[None]
    edges = np.array([0.5, 1.6, 2.6, k.max() + 1.0])
    bands = (np.searchsorted(edges, k, side="right") - 1)[None]
    bands[(k < edges[0]) | (bands >= nb)] = -1
    mask = np.ones((ny, nx), np.uint8)
    Ninv = np.full((1, ny, nx), 1.0 / s2)
    b, F, th = O.exact_band_terms(mask, Ninv, P, bands, nb)
    for l in range(nb):
        sel = bands == l
        assert sel.any()
        assert np.isclose(th[l], P[sel].mean(), rtol=1e-12)
        assert np.isclose(b[l], 0.5 / th[l] * np.sum(P[sel] / (P[sel] + s2)), rtol=1e-11)
        assert np.isclose(F[l, l], 0.5 / th[l] ** 2 * np.sum(P[sel] ** 2 / (P[sel] + s2) ** 2), rtol=1e-11)
    assert np.abs(F - np.diag(np.diag(F))).max() <= 1e-12 * np.abs(F).max()
