"""Shared test helpers: building the library on demand, moving seeded inputs
to the GPU, and comparing half-plane spectra with the oracle's pixel fields."""
import os

import numpy as np

from paper_1810_00503_gb300 import wf


def ensure_lib():
    if not os.path.exists(wf.LIB_PATH):
        from paper_1810_00503_gb300 import build
        build.build()
    return wf.lib()


def rfft_u(x):
    """Half-plane unitary spectrum of a real field (numpy rfft2, 'ortho')."""
    return np.fft.rfft2(x, norm="ortho")


def irfft_u(S, n, nx=None):
    return np.fft.irfft2(S, s=(n, n if nx is None else nx), norm="ortho")


def rel(a, b):
    a = np.asarray(a); b = np.asarray(b)
    den = np.linalg.norm(b.ravel())
    return np.linalg.norm((a - b).ravel()) / (den if den > 0 else 1.0)


def to_dev(a, dtype, dev="cuda"):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device=dev)


def make_problem(inputs, precision="fp64", d_list=None, lbfgs_m=10, shared_P=True):
    """Problem over a list of MapInputs of one shape.  Returns (problem, host arrays)
    where the host arrays are the exact (rounded) values the GPU sees, as float64."""
    import torch
    from oracle import wf_oracle as O
    fdt = torch.float64 if precision == "fp64" else torch.float32
    npdt = np.float64 if precision == "fp64" else np.float32
    ds, Ns, Ps, Ms = [], [], [], []
    for i, inp in enumerate(inputs):
        Pr = inp.P.astype(npdt).astype(np.float64)
        Nr = inp.Ninv.astype(npdt).astype(np.float64)
        d = O.synthesize_data(inp.z, inp.noise, inp.mask, inp.P) if d_list is None else d_list[i]
        ds.append(d.astype(npdt).astype(np.float64)); Ns.append(Nr); Ps.append(Pr); Ms.append(inp.mask)
    h1 = inputs[0].P.shape[-1] // 2 + 1  # half-plane columns
    d_t = to_dev(np.stack(ds), fdt)
    N_t = to_dev(np.stack(Ns), fdt)
    M_t = to_dev(np.stack(Ms), torch.uint8)
    if shared_P:
        P_t = to_dev(Ps[0][..., :h1], fdt)
    else:
        P_t = to_dev(np.stack(Ps)[..., :h1], fdt)
    prob = wf.Problem(d_t, M_t, N_t, P_t, precision=precision, lbfgs_m=lbfgs_m)
    host = dict(d=ds, Ninv=Ns, P=Ps, mask=Ms, W=[m[None] * N for m, N in zip(Ms, Ns)])
    return prob, host


def any_inputs(ny, nx, C, B, seed):
    """Seeded inputs on an ny x nx grid of any side lengths: real white fields
    z, masks (about 30% masked), inverse noise variances in [0.5, 1.5), a
    red power spectrum P ~ (|k| + 0.05)^-2 over the full plane (0 at k = 0;
    the second channel at 0.3 of the first), data d = M (A z + n) from the
    oracle, and the half-plane states s of independent white fields."""
    from oracle import wf_oracle as O
    rng = np.random.default_rng(seed)
    my, mx = O.signed_modes(ny, nx)
    k = np.sqrt((mx / nx) ** 2 + (my / ny) ** 2)
    P1 = np.where(k > 0, 1.0 / (k + 0.05) ** 2, 0.0) / (ny * nx) ** 0.5
    P = np.stack([P1, 0.3 * P1][:C])
    out = dict(P=P, z=[], d=[], mask=[], Ninv=[], f=[])
    for _ in range(B):
        z = rng.standard_normal((C, ny, nx))
        mask = (rng.random((ny, nx)) > 0.3).astype(np.uint8)
        Ninv = rng.random((C, ny, nx)) + 0.5
        noise = rng.standard_normal((C, ny, nx)) / np.sqrt(Ninv)
        out["z"].append(z)
        out["mask"].append(mask)
        out["Ninv"].append(Ninv)
        out["d"].append(O.synthesize_data(z, noise, mask, P))
        out["f"].append(rng.standard_normal((C, ny, nx)))
    return out
