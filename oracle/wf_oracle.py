"""FP64 CPU oracle for the Wiener-filter MAP objective, its solution and the
simulation-based band powers of Horowitz, Seljak & Aslanyan (arXiv:1810.00503).

TEST INFRASTRUCTURE ONLY.  Only the tests, the package smoke check and the
benchmark's CPU-baseline leg may import or run this module.  The GPU library
never calls it and shares no code with it: this file uses full-plane complex
numpy FFTs, a pixel-basis real state vector and dense linear algebra, written
to be read against the paper, not to be fast.

Variables
---------
The paper minimises chi^2(s) = s^T S^-1 s + (d - R s)^T N^-1 (d - R s) (Sec. 2.2,
eq. eq_chi).  Here S is diagonal in Fourier space with per-mode variance P_m and
R = M (mask).  We use the whitened real pixel field z, s = A z with
A = U^-1 diag(sqrt P) U (U the unitary 2-D DFT), which turns the prior into
z^T z.  With W = M N^-1 (diagonal, zero on masked pixels):

    chi^2(z) = z^T z + (d - A z)^T W (d - A z)
    grad     = 2 (z - A^T W (d - A z))       (twice eq. eq_cost)

For the joint E/B shear case (App. C) the operator is two-channel:
A = U^-1 R(k) diag(sqrt P_E, sqrt P_B) U with the per-mode Kaiser-Squires
rotation R(k) = [[c, -s], [s, c]], c = (kx^2 - ky^2)/k^2, s = 2 kx ky / k^2.
The paper's derivative operator equals this up to -k^2, absorbed into P.  The
odd term s is set to 0 on the Nyquist row and column (where k and -k alias),
the usual convention for odd spectral derivatives; only an even side length
has a Nyquist line; R = I at k = 0.  Grids may be rectangular (ny x nx) and of
any side lengths.  Pixels are square, so mode (my, mx) of an ny x nx grid has
the wavevector (kx, ky) = 2 pi (mx / nx, my / ny) / pixel, the k of App. C.

Pins (what fixes this file independently of itself) live in
tests/test_oracle_pins.py: naive O(n^4) DFT, Parseval, unmasked closed form
S/(S+N), Woodbury agreement of the two dense Wiener-filter forms, exact central
differences of a quadratic, the lambda_min >= 1 certificate, analytic band
terms without a mask, the Fisher identity Cov(E) = F, the two-loop recursion
against the dense BFGS inverse update, strong-Wolfe steps, the envelope identity
d chi^2 / d log q_l = -2 Theta_fid,l E_l at the MAP, chi^2_min ~ chi-square(N_obs), the
unbiasedness of Theta_hat (exact b and F) for a rescaled true spectrum, and the leakage-bias form
of App. C against the full Fisher run where E and B do not mix; on rectangular and
odd grids the DFT plane wave, the rotation's shear of a plane-wave potential,
its k -> -k symmetry, the unmasked S/(S+N) MAP and exact central differences.
Parity unpinned: iteration counts and chi^2-versus-iteration curves, because the
paper gives them only as figures.
"""
from __future__ import annotations

import numpy as np

# ---------------------------------------------------------------------------
# Fourier machinery (full plane, unitary)
# ---------------------------------------------------------------------------


def dft2_naive(x: np.ndarray) -> np.ndarray:
    """Unitary 2-D DFT by the definition, O(ny^2 nx^2): X[ky,kx] =
    (ny nx)^-1/2 sum x[y,x] exp(-2 pi i (ky y / ny + kx x / nx)).  For pinning
    the FFT-based code; any side lengths."""
    ny, nx = x.shape[-2], x.shape[-1]
    out = np.zeros(x.shape, dtype=np.complex128)
    iy, ix = np.arange(ny), np.arange(nx)
    norm = np.sqrt(float(ny * nx))
    for ky in range(ny):
        ey = np.exp(-2j * np.pi * ky * iy / ny)
        for kx in range(nx):
            ex = np.exp(-2j * np.pi * kx * ix / nx)
            out[..., ky, kx] = np.einsum("...yx,y,x->...", x, ey, ex) / norm
    return out


def fft2u(x):
    return np.fft.fft2(x, norm="ortho")


def ifft2u(X):
    return np.fft.ifft2(X, norm="ortho")


def signed_modes(n: int, nx: int | None = None):
    """Integer mode numbers (my, mx) of an n x nx grid (nx = n by default)."""
    nx = n if nx is None else nx
    fy = np.fft.fftfreq(n, d=1.0 / n)
    fx = np.fft.fftfreq(nx, d=1.0 / nx)
    my, mx = np.meshgrid(fy, fx, indexing="ij")
    return my, mx


def ks_rotation(n: int, nx: int | None = None):
    """Per-mode Kaiser-Squires cosine and sine (App. C, E/B operator), full
    plane of an n x nx grid (nx = n by default): c = (kx^2 - ky^2)/k^2,
    s = 2 kx ky / k^2 at the mode's wavevector k ~ (mx / nx, my / n), here
    scaled by n nx to the integers (mx n, my nx).  The Nyquist line of an even
    side, where k and -k alias, gets s = 0; an odd side has none."""
    nx = n if nx is None else nx
    my, mx = signed_modes(n, nx)
    qx, qy = mx * n, my * nx
    k2 = qx * qx + qy * qy
    c = np.ones((n, nx))
    s = np.zeros((n, nx))
    nz = k2 > 0
    c[nz] = (qx[nz] ** 2 - qy[nz] ** 2) / k2[nz]
    s[nz] = 2.0 * qx[nz] * qy[nz] / k2[nz]
    nyq = ((nx % 2 == 0) & (np.abs(mx) == nx // 2)) | ((n % 2 == 0) & (np.abs(my) == n // 2))
    s[nyq] = 0.0
    return c, s


def apply_A(z: np.ndarray, P: np.ndarray) -> np.ndarray:
    """Signal map s = A z for a whitened real field z (C, ny, nx); P (C, ny, nx)."""
    C = z.shape[0]
    Z = fft2u(z) * np.sqrt(P)
    if C == 2:
        c, s = ks_rotation(z.shape[-2], z.shape[-1])
        Z = np.stack([c * Z[0] - s * Z[1], s * Z[0] + c * Z[1]])
    x = ifft2u(Z)
    return x.real


def apply_At(x: np.ndarray, P: np.ndarray) -> np.ndarray:
    """Transpose of apply_A: A^T = U^-1 diag(sqrt P) R(k)^T U."""
    C = x.shape[0]
    X = fft2u(x)
    if C == 2:
        c, s = ks_rotation(x.shape[-2], x.shape[-1])
        X = np.stack([c * X[0] + s * X[1], -s * X[0] + c * X[1]])
    return ifft2u(X * np.sqrt(P)).real


def synthesize_data(z, noise, mask, P):
    """Step 2 of the paper's procedure (Sec. 2.5): d = M (A z + n)."""
    return (apply_A(z, P) + noise) * mask[None]


# ---------------------------------------------------------------------------
# Objective and gradient (Sec. 2.2, eq_chi and eq_cost)
# ---------------------------------------------------------------------------


def chi2(z, d, W, P) -> float:
    r = d - apply_A(z, P)
    return float(np.sum(z * z) + np.sum(r * W * r))


def grad(z, d, W, P) -> np.ndarray:
    r = d - apply_A(z, P)
    return 2.0 * (z - apply_At(W * r, P))


def chi2_dlogq(z, d, W, P, bands, n_bands):
    """d chi^2 / d log q_l when band l's power is scaled by q_l (S = sum_l q_l
    S_fid on band l, Sec. 2.3 eq. pilin), at the scale already folded into P:
    d sqrt(q P) / d log q = sqrt(q P) / 2 on band l, so dA/dlog q_l is A built
    with P/4 on band l and 0 elsewhere, and d chi^2 = -2 (W r).(dA z)."""
    r = d - apply_A(z, P)
    out = np.zeros(n_bands)
    for l in range(n_bands):
        dA_z = apply_A(z, np.where(bands == l, 0.25 * P, 0.0))
        out[l] = -2.0 * float(np.sum(W * r * dA_z))
    return out


def hess_vec(v, W, P) -> np.ndarray:
    """Full Hessian of chi^2 times v: 2 (I + A^T W A) v (twice eq_curv)."""
    return 2.0 * (v + apply_At(W * apply_A(v, P), P))


# ---------------------------------------------------------------------------
# Dense Wiener filter (App. A, eq. eq:wiener), small maps only
# ---------------------------------------------------------------------------


def dense_operator(P: np.ndarray) -> np.ndarray:
    """A as a dense (C ny nx) x (C ny nx) matrix, column j = A e_j."""
    C, ny, nx = P.shape
    N = C * ny * nx
    A = np.empty((N, N))
    e = np.zeros(N)
    for j in range(N):
        e[j] = 1.0
        A[:, j] = apply_A(e.reshape(C, ny, nx), P).ravel()
        e[j] = 0.0
    return A


def dense_wf_whitened(d, W, P, A=None):
    """Minimiser of chi^2 from the normal equations (I + A^T W A) z = A^T W d,
    solved by Cholesky.  Returns z* (C, n, n)."""
    A = dense_operator(P) if A is None else A
    w = W.ravel()
    H = np.eye(A.shape[0]) + A.T @ (w[:, None] * A)
    b = A.T @ (w * d.ravel())
    L = np.linalg.cholesky(H)
    z = np.linalg.solve(L.T, np.linalg.solve(L, b))
    return z.reshape(d.shape)


def dense_wf_covariance(d, mask, Ninv, P, A=None):
    """Paper's form s_hat = S R^dagger C^-1 d (App. A, eq:wiener) over the
    observed pixels only: S = A A^T (pixel signal covariance), R = mask
    selection, C = R S R^T + N.  Returns (x*, z*) with x* the Wiener-filtered
    signal map and z* = A^T R^T C^-1 d the same solution in whitened variables."""
    A = dense_operator(P) if A is None else A
    obs = np.broadcast_to(mask[None] == 1, d.shape).ravel()
    Ao = A[obs]
    Cmat = Ao @ Ao.T + np.diag(1.0 / Ninv.ravel()[obs])
    L = np.linalg.cholesky(Cmat)
    y = np.linalg.solve(L.T, np.linalg.solve(L, d.ravel()[obs]))
    S_cols = A @ Ao.T                      # S R^T = A A^T restricted to observed columns
    x = (S_cols @ y).reshape(d.shape)
    z = (Ao.T @ y).reshape(d.shape)
    return x, z


def chi2_min_dense(d, mask, Ninv, P, A=None) -> float:
    """Minimum of chi^2 = d_o^T C^-1 d_o (Woodbury on the normal equations)."""
    A = dense_operator(P) if A is None else A
    obs = np.broadcast_to(mask[None] == 1, d.shape).ravel()
    Ao = A[obs]
    Cmat = Ao @ Ao.T + np.diag(1.0 / Ninv.ravel()[obs])
    do = d.ravel()[obs]
    return float(do @ np.linalg.solve(Cmat, do))


# ---------------------------------------------------------------------------
# Textbook L-BFGS (Sec. 2.2: low-rank quasi-Newton; Nocedal & Wright,
# Numerical Optimization 2nd ed., Alg. 7.4 two-loop, Alg. 7.5 driver,
# Alg. 3.5 / 3.6 strong-Wolfe line search with zoom)
# ---------------------------------------------------------------------------


def _two_loop(g, S, Y):
    q = g.copy()
    alphas = []
    for s, y in zip(reversed(S), reversed(Y)):
        rho = 1.0 / np.dot(y, s)
        a = rho * np.dot(s, q)
        q -= a * y
        alphas.append((a, rho))
    if S:
        gamma = np.dot(S[-1], Y[-1]) / np.dot(Y[-1], Y[-1])
    else:
        gamma = 1.0
    r = gamma * q
    for (s, y), (a, rho) in zip(zip(S, Y), reversed(alphas)):
        b = rho * np.dot(y, r)
        r += s * (a - b)
    return -r


def _sufficient(f, f0, a, d0, c1, eps_f):
    """Armijo condition, relaxed by eps_f |f0| so that a step is not rejected
    when f changes by less than its own rounding error near the minimum (the
    approximate-Wolfe relaxation of Hager & Zhang, SIAM J. Optim. 16 (2005))."""
    return f <= f0 + c1 * a * d0 + eps_f * abs(f0)


def _zoom(phi, lo, hi, f0, d0, c1, c2, max_iter=60, eps_f=1e-14):
    a_lo, f_lo, d_lo = lo
    a_hi, f_hi, d_hi = hi
    for _ in range(max_iter):
        # cubic-free safeguarded quadratic interpolation from (a_lo, f_lo, d_lo) and f_hi
        da = a_hi - a_lo
        denom = 2.0 * (f_hi - f_lo - d_lo * da)
        a = a_lo - d_lo * da * da / denom if denom > 0 else 0.5 * (a_lo + a_hi)
        lo_b, hi_b = sorted((a_lo, a_hi))
        if not (lo_b + 0.1 * (hi_b - lo_b) <= a <= hi_b - 0.1 * (hi_b - lo_b)):
            a = 0.5 * (a_lo + a_hi)
        f, d, gvec = phi(a)
        if not _sufficient(f, f0, a, d0, c1, eps_f) or f > f_lo + eps_f * abs(f0):
            a_hi, f_hi, d_hi = a, f, d
        else:
            if abs(d) <= -c2 * d0:
                return a, f, gvec
            if d * (a_hi - a_lo) >= 0:
                a_hi, f_hi, d_hi = a_lo, f_lo, d_lo
            a_lo, f_lo, d_lo = a, f, d
    return a_lo, f_lo, None


def _line_search(fg, x, f0, g0, p, c1, c2, a_max=1e6, max_iter=40, eps_f=1e-14):
    d0 = float(np.dot(g0, p))
    cache = {}

    def phi(a):
        if a not in cache:
            f, g = fg(x + a * p)
            cache[a] = (f, float(np.dot(g, p)), g)
        return cache[a]

    a_prev, f_prev, d_prev = 0.0, f0, d0
    a = 1.0
    for i in range(max_iter):
        f, d, g = phi(a)
        if not _sufficient(f, f0, a, d0, c1, eps_f) or (i > 0 and f > f_prev + eps_f * abs(f0)):
            return _zoom(phi, (a_prev, f_prev, d_prev), (a, f, d), f0, d0, c1, c2)
        if abs(d) <= -c2 * d0:
            return a, f, g
        if d >= 0:
            return _zoom(phi, (a, f, d), (a_prev, f_prev, d_prev), f0, d0, c1, c2)
        a_prev, f_prev, d_prev = a, f, d
        a = min(2.0 * a, a_max)
    return a, f, g


def lbfgs(fg, x0, m=10, gtol_rel=1e-10, dchi2_abs=0.0, max_iter=10000,
          c1=1e-4, c2=0.9, callback=None):
    """Minimise f with L-BFGS.  fg(x) -> (f, grad).  Stops when
    ||g|| <= gtol_rel ||g0||, or |f_k - f_{k-1}| < dchi2_abs (the paper's
    Delta chi^2 rule, Sec. 3), or after max_iter iterations.
    Returns (x, info) with info = dict(iters, evals, f, gnorm_rel, history)."""
    x = np.array(x0, dtype=np.float64, copy=True).ravel()
    shape = np.shape(x0)
    evals = [0]

    def fgv(v):
        evals[0] += 1
        f, g = fg(v.reshape(shape))
        return f, np.asarray(g, dtype=np.float64).ravel()

    f, g = fgv(x)
    g0n = float(np.linalg.norm(g))
    S, Y = [], []
    hist = [f]
    it = 0
    status = "maxiter"
    if g0n == 0.0:
        status = "converged"
    while it < max_iter and status != "converged":
        p = _two_loop(g, S, Y)
        a, f_new, g_new = _line_search(fgv, x, f, g, p, c1, c2)
        if g_new is None:
            f_new, g_new = fgv(x + a * p)
        s = a * p
        y = g_new - g
        x = x + s
        sy = float(np.dot(s, y))
        if sy > 1e-12 * np.linalg.norm(s) * np.linalg.norm(y):
            S.append(s)
            Y.append(y)
            if len(S) > m:
                S.pop(0)
                Y.pop(0)
        df = abs(f_new - f)
        f, g = f_new, g_new
        it += 1
        hist.append(f)
        if callback is not None:
            callback(it, x, f, g)
        if np.linalg.norm(g) <= gtol_rel * g0n:
            status = "converged"
        elif dchi2_abs > 0 and df < dchi2_abs:
            status = "converged"
    info = dict(iters=it, evals=evals[0], f=f,
                gnorm_rel=float(np.linalg.norm(g)) / g0n if g0n else 0.0,
                status=status, history=np.array(hist))
    return x.reshape(shape), info


def map_solve(d, W, P, m=10, gtol_rel=1e-10, dchi2_abs=0.0, max_iter=10000, z0=None):
    """MAP field (Sec. 2.2) in whitened variables by textbook L-BFGS from z0 = 0
    (the start does not matter: the objective is strictly convex)."""
    z0 = np.zeros_like(d) if z0 is None else z0

    def fg(z):
        r = d - apply_A(z, P)
        return float(np.sum(z * z) + np.sum(r * W * r)), 2.0 * (z - apply_At(W * r, P))

    return lbfgs(fg, z0, m=m, gtol_rel=gtol_rel, dchi2_abs=dchi2_abs, max_iter=max_iter)


def exact_step(g, p, W, P):
    """Exact minimiser along p of the quadratic chi^2: -g.p / p.H p."""
    return -float(np.sum(g * p)) / float(np.sum(p * hess_vec(p, W, P)))


# ---------------------------------------------------------------------------
# Band powers (Sec. 2.3-2.5)
# ---------------------------------------------------------------------------


def theta_fid(P, bands, n_bands):
    """Theta_fid,l: mean of the fiducial P over the band's modes (Sec. 2.3,
    eq. pilin; the paper leaves the per-band normalisation open)."""
    out = np.zeros(n_bands)
    for l in range(n_bands):
        sel = bands == l
        out[l] = P[sel].mean()
    return out


def band_E(z, bands, theta, n_bands):
    """E_l = 1/2 sum_{k in l} s_k^2 / (Theta_fid,l S_fid,k) (Sec. 2.4, eq. el).
    In whitened variables s_k^2 / S_fid,k = |z_k|^2, summed over the full plane."""
    Z = fft2u(z)
    a2 = np.abs(Z) ** 2
    E = np.zeros(n_bands)
    for l in range(n_bands):
        E[l] = 0.5 * a2[bands == l].sum() / theta[l]
    return E


def band_signal(u, P, bands, band):
    """Field with the fiducial spectrum restricted to one band, from white noise u:
    U^-1 sqrt(P 1_band) U u (the extra signal Delta Theta_l' Pi_l' of eq. fisher
    with Delta Theta = Theta_fid)."""
    Pl = np.where(bands == band, P, 0.0)
    return apply_A(u, Pl)


def fisher_fill_columns(F, sampled):
    """Fisher columns of unsampled bands from the sampled ones (Sec. 3.1: the
    matrix is smooth and nearly translation invariant, so a few rows suffice and
    the rest are interpolated).  Reading: column l' between sampled s0 < l' < s1
    is F[l' + o][l'] = (1 - t) F[s0 + o][s0] + t F[s1 + o][s1] at every offset o,
    t = (l' - s0) / (s1 - s0); a term whose row s + o falls outside the matrix is
    dropped and the other weighted alone; before the first or after the last
    sampled column the nearest one is shifted.  sampled: ascending band ids."""
    nb = F.shape[0]
    G = F.copy()
    S = list(sampled)
    for lp in range(nb):
        if lp in S:
            continue
        lo = [s for s in S if s < lp]
        hi = [s for s in S if s > lp]
        if lo and hi:
            s0, s1 = lo[-1], hi[0]
            t = (lp - s0) / (s1 - s0)
            terms = [(1.0 - t, s0), (t, s1)]
        else:
            terms = [(1.0, lo[-1] if lo else hi[0])]
        for l in range(nb):
            o = l - lp
            acc, wsum = 0.0, 0.0
            for wt, sc in terms:
                if 0 <= sc + o < nb and wt > 0.0:
                    acc += wt * F[sc + o, sc]
                    wsum += wt
            G[l, lp] = acc / wsum if wsum > 0.0 else 0.0
    return G


def fisher_truncate(F, n_trunc, width):
    """Zero the Fisher terms far from the diagonal inside the leading n_trunc
    bands (App. C: the EE block, E bands first), |l - l'| > width."""
    G = F.copy()
    for l in range(min(n_trunc, F.shape[0])):
        for lp in range(min(n_trunc, F.shape[0])):
            if abs(l - lp) > width:
                G[l, lp] = 0.0
    return G


def bandpower_sims(d, mask, Ninv, P, bands, n_bands, z_sims, n_sims, u_fd,
                   m=10, gtol_rel=1e-10, max_iter=20000, fd_bands=None, trunc=(0, 0), leak_split=0):
    """Simulation estimates of Sec. 2.5 on one data map (C = 1, or C = 2 for the
    joint E/B case of App. C with separate band ids for the two channels).

    * E(d): eq. el on the MAP of the data.
    * b_l = mean_j E_l(MAP(d_j)), d_j = M (A z_j + n_j)        (eq. blmv)
    * F_ll' Delta Theta_l' = mean_j [E_l(MAP(d_j + delta_l'j)) - E_l(MAP(d_j))],
      delta_l'j = M A_l' u_l'j, Delta Theta_l' = Theta_fid,l'   (eq. fisher)
      with common random numbers: the j-th finite-difference map reuses d_j.
    * Theta_hat = Theta_fid + F^-1 (E - b)                      (eq. eq:wfmv)
    * cov = F^-1 (eq. eq:var), and the sample covariance of E over the sims.
    z_sims, n_sims: (J, C, n, n) white signal fields and noise realisations.
    u_fd: (n_bands, J_fd, C, n, n) white fields for the Fisher perturbations;
    J_fd <= J, and the j-th perturbation is added to sim j.  fd_bands: the bands
    given Fisher simulations (default all; u_fd then holds one row per listed
    band), the other columns from fisher_fill_columns.  trunc = (n_trunc,
    width): fisher_truncate before the inversion ((0, 0) = off).
    leak_split = L > 0: the leakage-bias alternative of App. C (E bands
    0..L-1, B bands L..n_bands-1).  The B power gets no per-band Fisher maps:
    one map per simulation j < J_fd adds the fiducial power of every B band at
    once, delta_Bj = M A_B u_Bj, and the B bands get only the diagonal response
    F_ll = mean_j [E_l(MAP(d_j + delta_Bj)) - E_l(MAP(d_j))] / Theta_fid,l.
    The cross blocks (E response to B power, B response to E power) are not
    estimated: the E-to-B leakage enters through b alone, the mean over
    simulations at the fiducial power, like the noise.  Per-band maps,
    fd_bands (all < L), the interpolation and trunc then concern the E block;
    u_fd holds one more row, the B fields, last.
    """
    W = mask[None] * Ninv
    theta = theta_fid(P, bands, n_bands)

    def E_of(data):
        z, _ = map_solve(data, W, P, m=m, gtol_rel=gtol_rel, max_iter=max_iter)
        return band_E(z, bands, theta, n_bands)

    E_d = E_of(d)
    J = z_sims.shape[0]
    sims = [synthesize_data(z_sims[j], n_sims[j], mask, P) for j in range(J)]
    E_s = np.array([E_of(sd) for sd in sims])
    b = E_s.mean(axis=0)
    J_fd = u_fd.shape[1]
    L = int(leak_split)
    nE = L if L > 0 else n_bands       # bands with per-band Fisher maps (all, or the E bands)
    fdb = list(range(nE)) if fd_bands is None else list(fd_bands)
    F = np.zeros((n_bands, n_bands))
    for k, lp in enumerate(fdb):
        acc = np.zeros(n_bands)
        for j in range(J_fd):
            delta = band_signal(u_fd[k, j], P, bands, lp) * mask[None]
            acc += E_of(sims[j] + delta) - E_s[j]
        F[:, lp] = acc / J_fd / theta[lp]
    if L > 0:
        F[L:, :L] = 0.0                  # B response to E power: left to b
        PB = np.where(bands >= L, P, 0.0)
        acc = np.zeros(n_bands)
        for j in range(J_fd):
            delta = apply_A(u_fd[len(fdb), j], PB) * mask[None]
            acc += E_of(sims[j] + delta) - E_s[j]
        for l in range(L, n_bands):
            F[l, l] = acc[l] / J_fd / theta[l]
    if len(fdb) < nE:
        F[:nE, :nE] = fisher_fill_columns(F[:nE, :nE], fdb)
    if trunc[0] > 0:
        F = fisher_truncate(F, trunc[0], trunc[1])
    Finv = np.linalg.inv(F)
    theta_hat = theta + Finv @ (E_d - b)
    covE = np.cov(E_s.T, ddof=1) if J > 1 else np.zeros((n_bands, n_bands))
    return dict(E=E_d, b=b, F=F, cov=Finv, theta_hat=theta_hat, theta_fid=theta,
                E_sims=E_s, cov_E=covE)


def bandpower_iterate(d, mask, Ninv, P0, bands, n_bands, z_sims, n_sims, u_fd, n_iter,
                      q_min=0.01, q_max=100.0, **kw):
    """Iterated fiducial (Sec. 2.3, after eq. pilin): estimate the band powers
    with the fiducial S_fid, move each band of S_fid to its estimate, S_fid <-
    S_fid * q_l on the modes of band l with q_l = Theta_hat_l / Theta_fid,l kept
    in [q_min, q_max] (the regularisation: no band power becomes zero or
    negative), and estimate again; n_iter estimates with the same random fields.
    Returns (list of the n_iter estimates, final fiducial P)."""
    P = np.array(P0, dtype=np.float64, copy=True)
    out = []
    for it in range(n_iter):
        r = bandpower_sims(d, mask, Ninv, P, bands, n_bands, z_sims, n_sims, u_fd, **kw)
        out.append(r)
        if it + 1 < n_iter:
            q = np.clip(r["theta_hat"] / r["theta_fid"], q_min, q_max)
            for l in range(n_bands):
                P = np.where(bands == l, P * q[l], P)
    return out, P


def exact_band_terms(mask, Ninv, P, bands, n_bands, A=None):
    """Exact noise bias and Fisher matrix by dense traces (App. A, eq.
    eq:wf_exact_f, first equality; Sec. 2.1 Q_l = dC/dTheta_l):
    C = M A A^T M^T + N,  Q_l = M A Pi_l A^T M^T / Theta_fid,l,
    b_l = 1/2 tr(C^-1 Q_l),  F_ll' = 1/2 tr(C^-1 Q_l C^-1 Q_l')."""
    A = dense_operator(P) if A is None else A
    obs = np.broadcast_to(mask[None] == 1, P.shape).ravel()
    Ao = A[obs]
    Cmat = Ao @ Ao.T + np.diag(1.0 / Ninv.ravel()[obs])
    Cinv = np.linalg.inv(Cmat)
    theta = theta_fid(P, bands, n_bands)
    Ms = []
    for l in range(n_bands):
        Al = dense_operator(np.where(bands == l, P, 0.0))[obs]
        Ql = (Al @ Al.T) / theta[l]
        Ms.append(Cinv @ Ql)
    b = np.array([0.5 * np.trace(M) for M in Ms])
    F = np.array([[0.5 * np.sum(Ms[i] * Ms[j].T) for j in range(n_bands)]
                  for i in range(n_bands)])
    return b, F, theta
