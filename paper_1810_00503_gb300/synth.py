"""Seeded synthetic inputs shaped like the paper's workloads (density, shear, CMB).

This module only draws random numbers and tabulates power-spectrum formulas: it
returns masks, inverse-noise maps, power tables P per Fourier mode, white-noise
fields z and noise realisations.  It does none of the method's arithmetic: the
data map d = M (A z + noise) is formed by whoever consumes these inputs (the
oracle on the CPU, or the library's own data-synthesis call on the GPU), so a
mistake here changes the test data, never the expected answer.

Conventions
-----------
* Maps are n x n periodic pixels (ny x nx where a generator takes nx: square
  pixels, so mode (my, mx) has wavevector 2 pi (mx / nx, my / ny) per pixel);
  C channels (1 = density/CMB, 2 = E/B shear).
* Fourier index m = (my, mx) in signed form, my, mx in [-n/2, n/2).
* P[c, my, mx] is the variance of the unitary DFT coefficient of channel c at
  mode m (full plane).  For a continuous spectrum P(k) on an L-sided box this
  is P(k) n^2 / L^2 with k in units of the fundamental 2 pi / L; P at m = 0 is 0.
* ``P_half`` is the real-FFT half plane P[..., : nx // 2 + 1].
* mask is uint8, 1 = observed; Ninv = 1 / noise variance on observed pixels,
  0 on masked ones.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


@dataclass
class MapInputs:
    n: int
    C: int
    mask: np.ndarray          # (n, n) uint8, 1 = observed
    Ninv: np.ndarray          # (C, n, n) float64, 0 where masked
    P: np.ndarray             # (C, n, n) float64, full-plane per-mode variance
    z: np.ndarray             # (C, n, n) float64 white signal field, N(0, 1)
    noise: np.ndarray         # (C, n, n) float64 noise realisation, var = 1/Ninv
    meta: dict = field(default_factory=dict)

    @property
    def P_half(self) -> np.ndarray:
        return np.ascontiguousarray(self.P[..., : self.P.shape[-1] // 2 + 1])


def signed_freqs(n: int):
    """Integer mode numbers (my, mx), both (n, n), signed in [-n/2, n/2)."""
    f = np.fft.fftfreq(n, d=1.0 / n).astype(np.int64)
    return np.meshgrid(f, f, indexing="ij")


def mode_modulus(n: int, nx: int | None = None) -> np.ndarray:
    """|k| per mode in units of the fundamental of the longer side (square
    pixels): sqrt((mx N / nx)^2 + (my N / n)^2), N = max(n, nx); for a square
    map the modulus of the mode numbers."""
    if nx is None or nx == n:
        my, mx = signed_freqs(n)
        return np.sqrt(my.astype(np.float64) ** 2 + mx.astype(np.float64) ** 2)
    N = max(n, nx)
    fy = np.fft.fftfreq(n, d=1.0 / n) * (N / n)
    fx = np.fft.fftfreq(nx, d=1.0 / nx) * (N / nx)
    my, mx = np.meshgrid(fy, fx, indexing="ij")
    return np.sqrt(my ** 2 + mx ** 2)


def _disk_mask(n: int, rng, count: int, radius: float, nx: int | None = None) -> np.ndarray:
    """Boolean map of `count` periodic disks of the given radius (True = hole)."""
    nx = n if nx is None else nx
    holes = np.zeros((n, nx), dtype=bool)
    cy = rng.integers(0, n, size=count)
    cx = rng.integers(0, nx, size=count)
    r = int(np.ceil(radius))
    off = np.arange(-r, r + 1)
    oy, ox = np.meshgrid(off, off, indexing="ij")
    inside = (oy * oy + ox * ox) <= radius * radius
    oy, ox = oy[inside], ox[inside]
    for y0, x0 in zip(cy, cx):
        holes[(y0 + oy) % n, (x0 + ox) % nx] = True
    return holes


def _normalise_to_snr1(P: np.ndarray, noise_var_obs_mean: float) -> np.ndarray:
    """Scale P so the mean pixel signal variance, sum_m P_m / n^2, equals the
    mean observed noise variance (signal-to-noise 1 per pixel on average)."""
    npix = P.shape[-2] * P.shape[-1]
    pix_var = P.reshape(P.shape[0], -1).sum(axis=1).mean() / npix
    return P * (noise_var_obs_mean / pix_var)


def _finish(n, C, mask_bool_obs, var, P, rng, meta) -> MapInputs:
    """Common tail: white field, noise, Ninv with zeros on masked pixels."""
    mask = mask_bool_obs.astype(np.uint8)
    shape = (C,) + mask.shape
    var = np.broadcast_to(var, shape).astype(np.float64)
    Ninv = np.where(mask[None] == 1, 1.0 / var, 0.0)
    z = rng.standard_normal(shape)
    noise = rng.standard_normal(shape) * np.sqrt(var)
    return MapInputs(n=n, C=C, mask=mask, Ninv=np.ascontiguousarray(Ninv),
                     P=np.ascontiguousarray(P), z=z, noise=noise, meta=meta)


def density_small(n: int = 32, seed: int = 0, masked_frac: float = 0.2,
                  sigma2: float = 0.1, nx: int | None = None) -> MapInputs:
    """Plain FP64 density case: P(k) = k^-2 (A = 1, box L = 1), Bernoulli mask
    with ``masked_frac`` of pixels removed, per-pixel noise variance
    sigma2 * U[0.5, 1.5].  nx: a rectangular n x nx map."""
    rng = np.random.default_rng(seed)
    nx = n if nx is None else nx
    k = mode_modulus(n, nx)
    P = np.zeros((1, n, nx))
    nz = k > 0
    P[0][nz] = k[nz] ** -2.0 * n * nx
    observed = rng.random((n, nx)) >= masked_frac
    var = sigma2 * rng.uniform(0.5, 1.5, size=(n, nx))
    return _finish(n, 1, observed, var, P, rng,
                   dict(kind="density", spectrum="k^-2", masked_frac=masked_frac))


def density_projected(n: int = 256, seed: int = 1) -> MapInputs:
    """Projected density: P(k) ~ k^-1.5 exp(-(2k/k_Nyq)^2), two 10-px stripes
    plus 200 disks of radius 3 px, n_gal ~ Poisson(20) per pixel, noise
    variance 1/n_gal (n_gal = 0 pixels are masked); S/N = 1 normalisation."""
    rng = np.random.default_rng(seed)
    k = mode_modulus(n)
    kny = n / 2
    P = np.zeros((1, n, n))
    nz = k > 0
    P[0][nz] = k[nz] ** -1.5 * np.exp(-((2.0 * k[nz] / kny) ** 2))
    holes = _disk_mask(n, rng, 200, 3.0)
    y0, x0 = rng.integers(0, n, size=2)
    rows = (np.arange(n)[:, None] - y0) % n < 10
    cols = (np.arange(n)[None, :] - x0) % n < 10
    holes |= rows | cols
    ngal = rng.poisson(20.0, size=(n, n))
    observed = (~holes) & (ngal > 0)
    var = np.where(ngal > 0, 1.0 / np.maximum(ngal, 1), 1.0)
    P = _normalise_to_snr1(P, float(var[observed].mean()))
    return _finish(n, 1, observed, var, P, rng,
                   dict(kind="density", spectrum="k^-1.5 exp(-(2k/kNyq)^2)"))


def shear_eb(n: int = 512, seed: int = 2, b_frac: float = 0.01, nx: int | None = None) -> MapInputs:
    """Joint E/B shear: P_E ~ k^-1.2, P_B = b_frac P_E; shape noise
    0.09 / n_gal per component with n_gal ~ Poisson(10); mask = Gaussian-smoothed
    white noise (sigma 8 px) above its 70th percentile (30% masked).  nx: a
    rectangular n x nx patch (k in units of the longer side's fundamental)."""
    rng = np.random.default_rng(seed)
    nx = n if nx is None else nx
    k = mode_modulus(n, nx)
    PE = np.zeros((n, nx))
    nz = k > 0
    PE[nz] = k[nz] ** -1.2
    P = np.stack([PE, b_frac * PE])
    # Smoothing is done in Fourier space with a Gaussian kernel (numpy FFT).
    white = rng.standard_normal((n, nx))
    N = max(n, nx)
    my, mx = np.meshgrid(np.fft.fftfreq(n, d=1.0 / n) * (N / n), np.fft.fftfreq(nx, d=1.0 / nx) * (N / nx),
                         indexing="ij")
    kern = np.exp(-0.5 * (2 * np.pi * 8.0 / N) ** 2 * (my ** 2 + mx ** 2))
    smooth = np.fft.ifft2(np.fft.fft2(white) * kern).real
    thr = np.quantile(smooth, 0.70)
    ngal = rng.poisson(10.0, size=(n, nx))
    observed = (smooth <= thr) & (ngal > 0)
    var = np.where(ngal > 0, 0.09 / np.maximum(ngal, 1), 1.0)
    P = _normalise_to_snr1(P, float(var[observed].mean()))
    return _finish(n, 2, observed, var, P, rng,
                   dict(kind="shear_eb", spectrum="k^-1.2", b_frac=b_frac, nx=nx))


def cmb_cl(ell: np.ndarray) -> np.ndarray:
    """Analytic CMB-like angular spectrum
    C_l = 1e3 / (l (l + 1)) (1 + 0.3 cos(pi l / 300)) exp(-(l / 1500)^2)."""
    ell = np.asarray(ell, dtype=np.float64)
    out = np.zeros_like(ell)
    nz = ell > 0
    l = ell[nz]
    out[nz] = 1e3 / (l * (l + 1.0)) * (1.0 + 0.3 * np.cos(np.pi * l / 300.0)) \
        * np.exp(-((l / 1500.0) ** 2))
    return out


def cmb_patch(n: int = 1024, seed: int = 3, pix_arcmin: float = 2.0,
              noise_uk_arcmin: float = 6.0, band_frac: float = 0.15,
              holes: int = 500) -> MapInputs:
    """CMB temperature on a flat patch of n x n pixels of ``pix_arcmin``.
    P_m = C_l / Omega_pix with l = 2 pi |m| / Theta_patch; noise variance
    (noise_uk_arcmin / pix_arcmin)^2 times a scan-like stripe modulation in
    [0.5, 3] with a +-5% per-row jitter; a contiguous galactic band of
    ``band_frac`` of the rows plus ``holes`` point-source holes of radius 3 px."""
    rng = np.random.default_rng(seed)
    pix = pix_arcmin / 60.0 * np.pi / 180.0
    theta = n * pix
    ell = 2.0 * np.pi * mode_modulus(n) / theta
    P = (cmb_cl(ell) / (pix * pix))[None]
    y = np.arange(n, dtype=np.float64)
    v = 0.5 + 2.5 * 0.5 * (1.0 + np.sin(2.0 * np.pi * 8.0 * y / n))
    v = v * (1.0 + 0.05 * rng.uniform(-1.0, 1.0, size=n))
    var = (noise_uk_arcmin / pix_arcmin) ** 2 * np.repeat(v[:, None], n, axis=1)
    nb = int(round(band_frac * n))
    y0 = int(rng.integers(0, n))
    band = ((np.arange(n) - y0) % n) < nb
    hole = _disk_mask(n, rng, holes, 3.0) if holes else np.zeros((n, n), bool)
    observed = ~(band[:, None] | hole)
    return _finish(n, 1, observed, var, P, rng,
                   dict(kind="cmb", pix_arcmin=pix_arcmin, theta_rad=theta))


def log_bands(n: int, n_bands: int, kmin: float = 1.0, kmax: float | None = None,
              C: int = 1, nx: int | None = None) -> np.ndarray:
    """Band id per full-plane mode: log-spaced shells in |m| between kmin and
    kmax (default the Nyquist n/2); -1 for modes outside every band (m = 0 and
    corners beyond kmax).  Shape (C, n, n), int16; channel c uses ids offset by
    c * n_bands.  nx: an n x nx map, |k| as mode_modulus(n, nx) and kmax
    defaulting to max(n, nx)/2."""
    kmax = max(n, n if nx is None else nx) / 2 if kmax is None else kmax
    k = mode_modulus(n, nx)
    edges = np.geomspace(kmin, kmax, n_bands + 1)
    edges[-1] = kmax * (1 + 1e-12)
    ids = np.searchsorted(edges, k, side="right") - 1
    ids[(k < kmin) | (k > edges[-1])] = -1
    ids = ids.astype(np.int16)
    out = np.stack([np.where(ids >= 0, ids + c * n_bands, -1) for c in range(C)])
    return out.astype(np.int16)


def hetero_batch(count: int = 256, seed: int = 4,
                 sizes=(64, 128, 256, 512)) -> list[MapInputs]:
    """Independent maps of uneven size: n uniform over ``sizes``, masked fraction
    U[0.1, 0.4] (half Bernoulli pixels, half disks of radius 3 px), noise
    variance log-uniform in [0.01, 1], P = |m|^slope n^2 with slope U[-2.5, -1]."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        n = int(rng.choice(sizes))
        sub = np.random.default_rng(rng.integers(0, 2 ** 63))
        frac = sub.uniform(0.1, 0.4)
        slope = sub.uniform(-2.5, -1.0)
        sig2 = float(np.exp(sub.uniform(np.log(0.01), np.log(1.0))))
        k = mode_modulus(n)
        P = np.zeros((1, n, n))
        nz = k > 0
        P[0][nz] = k[nz] ** slope * n * n
        observed = sub.random((n, n)) >= frac / 2
        ndisk = int(frac / 2 * n * n / (math.pi * 9.0))
        if ndisk:
            observed &= ~_disk_mask(n, sub, ndisk, 3.0)
        out.append(_finish(n, 1, observed, np.full((n, n), sig2), P, sub,
                           dict(kind="hetero", slope=slope, sigma2=sig2, masked_frac=frac)))
    return out


def random_state(n: int, C: int, seed: int, nx: int | None = None) -> np.ndarray:
    """A random real pixel field (C, n, n), or (C, n, nx), used as an evaluation point."""
    return np.random.default_rng(seed).standard_normal((C, n, n if nx is None else nx))


def white_noise_batch(count: int, C: int, n: int, seed: int) -> np.ndarray:
    """`count` independent N(0, 1) pixel fields, shape (count, C, n, n)."""
    return np.random.default_rng(seed).standard_normal((count, C, n, n))


WORKLOADS = {
    "density_32_fp64": lambda: density_small(32, 0),
    "density_256_mixed": lambda: density_projected(256, 1),
    "shear_eb_512": lambda: shear_eb(512, 2),
    "cmb_1024": lambda: cmb_patch(1024, 3),
}
