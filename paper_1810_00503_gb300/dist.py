"""Band powers from simulations spread over several GPUs (one process each).

Each rank solves its own contiguous range of noise-bias simulations, and the
Fisher simulations that reuse them, with bandpower_estimate on its GPU.  The
ranks then combine (3 n_b + n_b^2) FP64 sums in one all-reduce (Sec. 2.5,
eq. blmv, fisher, eq:wfmv):
    b      = sum_j E_j / J
    F_ll'  = sum_j (E_l(d_l'j) - E_l(d_j)) / J_fd / Theta_fid,l'
    cov_E  = (sum_j E_j E_j^T - J b b^T) / (J - 1)
    Theta  = Theta_fid + F^-1 (E - b)
With the leakage-bias form of App. C (leak_split = L: E bands 0..L-1 with
per-band Fisher maps, one joint map of the B bands per Fisher simulation) the
Fisher sums have L + 1 rows, and F keeps the EE block and the B diagonal only;
with sampled Fisher columns (fd_bands) the sums have a row per sampled band and
the other columns are interpolated.  The sums and the estimator are the
library's (bandpower_sums, bandpower_combine); this module only splits the
simulations, all-reduces and marshals.  No data path crosses GPUs; only these
sums do.
"""
from __future__ import annotations

import numpy as np


def shard(n_total: int, world: int, rank: int) -> tuple[int, int]:
    """Contiguous [start, stop) range of simulation indices owned by `rank`."""
    base, extra = divmod(n_total, world)
    start = rank * base + min(rank, extra)
    return start, start + base + (1 if rank < extra else 0)


def assignment(n_sim: int, n_fd: int, world: int, rank: int):
    """Simulations owned by `rank`, in the local order bandpower_estimate needs:
    the Fisher simulation j reuses simulation j, so the simulations paired with
    Fisher maps (global 0 .. n_fd-1) are split evenly and listed first, then the
    rank's share of the others.  Returns (global simulation indices, (fd_lo, fd_hi))."""
    fd_lo, fd_hi = shard(n_fd, world, rank)
    o_lo, o_hi = shard(n_sim - n_fd, world, rank)
    sims = list(range(fd_lo, fd_hi)) + list(range(n_fd + o_lo, n_fd + o_hi))
    return sims, (fd_lo, fd_hi)


def fisher_rows(n_bands: int, leak_split: int = 0, fd_bands=None) -> int:
    """Fisher-map rows of a rank's run: one per band with Fisher maps (every
    band, the listed fd_bands, or the E bands), plus the joint B row of the
    leakage-bias form."""
    from . import wf
    return wf.fisher_rows(n_bands, leak_split, fd_bands)


def local_sums(E_maps: np.ndarray, n_sim: int, n_bands: int, n_fd: int, leak_split: int = 0,
               fd_bands=None) -> np.ndarray:
    """This rank's partial sums (the library's bandpower_sums) from its per-map
    band energies, rows ordered as bandpower_estimate writes them: data, n_sim
    simulations, then the Fisher maps."""
    from . import wf
    return wf.bandpower_sums(E_maps, n_sim, n_fd, fisher_rows(n_bands, leak_split, fd_bands))


def combine(total: np.ndarray, E_data: np.ndarray, theta_fid: np.ndarray, leak_split: int = 0,
            trunc=(0, 0), fd_bands=None) -> dict:
    """Band-power estimate from the all-reduced sums (the library's
    bandpower_combine, the code bandpower_estimate ends with)."""
    from . import wf
    return wf.bandpower_combine(total, E_data, theta_fid, leak_split=leak_split, fd_bands=fd_bands, trunc=trunc)


def reduce_bandpower(E_maps: np.ndarray, n_sim: int, n_bands: int, n_fd: int, theta_fid: np.ndarray,
                     group=None, leak_split: int = 0, trunc=(0, 0), fd_bands=None) -> dict:
    """All-reduce the rank's partial sums (torch.distributed, any backend) and
    combine them.  E_maps: this rank's per-map energies; the data map's row 0
    is taken from rank 0."""
    import torch
    import torch.distributed as dist
    part = torch.as_tensor(local_sums(E_maps, n_sim, n_bands, n_fd, leak_split, fd_bands), dtype=torch.float64)
    e0 = torch.as_tensor(E_maps[0], dtype=torch.float64).clone()
    if dist.is_available() and dist.is_initialized():
        dist.all_reduce(part, group=group)
        dist.broadcast(e0, src=0, group=group)
    return combine(part.numpy(), e0.numpy(), np.asarray(theta_fid, dtype=np.float64), leak_split, trunc, fd_bands)


def estimate_on_rank(d, mask, Ninv, P, band, n_bands, n_sim, n_fd, world, rank, seed, group=None, **opts):
    """One band-power estimate spread over `world` ranks, this rank's part:
    bandpower_estimate on the rank's simulations with fields drawn on its GPU
    (Philox keyed by each simulation's global index, so every simulation has
    the same fields whatever the split), then the all-reduce of the partial
    sums.  Returns (estimate, this rank's per-map stats); the estimate is the
    same on every rank and equals the single-process one."""
    from . import wf
    sims, (fd_lo, fd_hi) = assignment(n_sim, n_fd, world, rank)
    res, stats = wf.bandpower_estimate(d, mask, Ninv, P, band, n_bands, None, None, None, n_sim=len(sims),
                                       n_fd=fd_hi - fd_lo, sim_index=sims, seed=seed, **opts)
    est = reduce_bandpower(res["E_maps"], len(sims), n_bands, fd_hi - fd_lo, res["theta_fid"], group,
                           opts.get("leak_split", 0), opts.get("trunc", (0, 0)), opts.get("fd_bands"))
    return est, stats
