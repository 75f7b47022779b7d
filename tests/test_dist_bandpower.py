"""Multi-rank band powers on the CPU (gloo, world size 2): the sums each rank
contributes, all-reduced, give the same estimate as one process holding every
simulation.  The per-map band energies are synthetic here; no GPU is used."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_1810_00503_gb300 import dist as D


def _reference(E_all, n_sim, nb, n_fd, theta):
    Es = E_all[1:1 + n_sim]
    Ef = E_all[1 + n_sim:].reshape(nb, n_fd, nb)
    b = Es.mean(axis=0)
    F = np.zeros((nb, nb))
    for lp in range(nb):
        F[:, lp] = (Ef[lp] - Es[:n_fd]).mean(axis=0) / theta[lp]
    covE = np.cov(Es.T, ddof=1)
    return dict(bias=b, fisher=F, cov_E=covE, theta_hat=theta + np.linalg.solve(F, E_all[0] - b))


def _worker(rank, world, port, n_sim, nb, n_fd, E_all, theta, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sims, (fd_lo, fd_hi) = D.assignment(n_sim, n_fd, world, rank)
    Ef = E_all[1 + n_sim:].reshape(nb, n_fd, nb)[:, fd_lo:fd_hi]
    Es_local = E_all[[1 + j for j in sims]]
    rows = np.concatenate([E_all[:1], Es_local, Ef.reshape(-1, nb)])
    res = D.reduce_bandpower(rows, len(sims), nb, fd_hi - fd_lo, theta)
    out[rank] = {k: res[k] for k in ("bias", "fisher", "cov_E", "theta_hat")}
    dist.destroy_process_group()


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def test_assignment_pairs_fisher_maps_with_local_simulations():
    for n_sim, n_fd, w in ((10, 6, 2), (100, 20, 3), (7, 7, 4), (5, 1, 2)):
        seen = []
        for r in range(w):
            sims, (a, b) = D.assignment(n_sim, n_fd, w, r)
            assert sims[: b - a] == list(range(a, b))
            seen += sims
        assert sorted(seen) == list(range(n_sim))


def test_shard_covers_everything_once():
    for n in (1, 7, 100, 101):
        for w in (1, 2, 3, 8):
            ranges = [D.shard(n, w, r) for r in range(w)]
            idx = [i for a, b in ranges for i in range(a, b)]
            assert idx == list(range(n))


def test_two_rank_reduction_equals_single_process():
    rng = np.random.default_rng(3)
    n_sim, nb, n_fd = 10, 4, 6
    E_all = rng.uniform(0.5, 2.0, size=(1 + n_sim + nb * n_fd, nb))
    theta = rng.uniform(0.5, 1.5, size=nb)
    ref = _reference(E_all, n_sim, nb, n_fd, theta)
    single = D.combine(D.local_sums(E_all, n_sim, nb, n_fd), E_all[0], theta)
    for k in ref:
        assert np.allclose(single[k], ref[k], rtol=1e-12)
    mgr = mp.Manager()
    out = mgr.dict()
    port = _free_port()
    mp.start_processes(_worker, args=(2, port, n_sim, nb, n_fd, E_all, theta, out), nprocs=2,
                       start_method="spawn", join=True)
    for rank in (0, 1):
        for k in ref:
            assert np.allclose(out[rank][k], ref[k], rtol=1e-12, atol=1e-14), (rank, k)


@pytest.mark.parametrize("opt", [dict(fd_bands=[0, 2]), dict(leak_split=2)])
def test_rank_estimate_rejects_forms_the_reduction_does_not_cover(opt):
    """The reduction sums per-band Fisher maps of every band, so sampled
    Fisher columns and the leakage-bias form are refused before any work."""
    with pytest.raises(ValueError):
        D.estimate_on_rank(None, None, None, None, None, 4, 2, 1, 2, 0, 0, **opt)
