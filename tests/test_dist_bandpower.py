"""Multi-rank band powers on the CPU (gloo, world size 2): the sums each rank
contributes (the library's bandpower_sums), all-reduced and combined by the
library's bandpower_combine, give the same estimate as one process holding
every simulation, computed here independently with numpy (and the oracle's
Fisher-column interpolation).  The per-map band energies are synthetic; the
two host calls need no GPU."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from oracle import wf_oracle as O
from paper_1810_00503_gb300 import dist as D
from tests.helpers import ensure_lib


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ensure_lib()


def _reference(E_all, n_sim, nb, n_fd, theta, leak=0, trunc=(0, 0), fd_bands=None):
    nR = D.fisher_rows(nb, leak, fd_bands)
    cols = list(fd_bands) if fd_bands is not None else list(range(leak if leak else nb))
    Es = E_all[1:1 + n_sim]
    Ef = E_all[1 + n_sim:].reshape(nR, n_fd, nb)
    b = Es.mean(axis=0)
    F = np.zeros((nb, nb))
    for k in range(nR):
        resp = (Ef[k] - Es[:n_fd]).mean(axis=0)  # every band's response to Fisher row k
        if k >= len(cols):                        # joint B row: the B diagonal
            F[leak:, leak:] = np.diag(resp[leak:] / theta[leak:])
        elif not leak:
            F[:, cols[k]] = resp / theta[cols[k]]
        else:                                     # E column, E rows only
            F[:leak, cols[k]] = resp[:leak] / theta[cols[k]]
    if fd_bands is not None:
        lim = leak if leak else nb
        F[:lim, :lim] = O.fisher_fill_columns(F[:lim, :lim], cols)
    for l in range(trunc[0]):
        for lp in range(trunc[0]):
            if abs(l - lp) > trunc[1]:
                F[l, lp] = 0.0
    covE = np.cov(Es.T, ddof=1)
    return dict(bias=b, fisher=F, cov_E=covE, theta_hat=theta + np.linalg.solve(F, E_all[0] - b))


def _worker(rank, world, port, n_sim, nb, n_fd, E_all, theta, out, leak=0, trunc=(0, 0), fd_bands=None):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sims, (fd_lo, fd_hi) = D.assignment(n_sim, n_fd, world, rank)
    Ef = E_all[1 + n_sim:].reshape(D.fisher_rows(nb, leak, fd_bands), n_fd, nb)[:, fd_lo:fd_hi]
    Es_local = E_all[[1 + j for j in sims]]
    rows = np.concatenate([E_all[:1], Es_local, Ef.reshape(-1, nb)])
    res = D.reduce_bandpower(rows, len(sims), nb, fd_hi - fd_lo, theta, leak_split=leak, trunc=trunc,
                             fd_bands=fd_bands)
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


@pytest.mark.parametrize("leak,trunc,fdb", [(0, (0, 0), None), (2, (0, 0), None), (0, (3, 1), None),
                                             (3, (3, 0), None), (0, (0, 0), [0, 2, 4]), (3, (0, 0), [0, 2])])
def test_two_rank_reduction_equals_single_process(leak, trunc, fdb):
    """Plain, leakage-bias (E bands 0..leak-1, joint B row last), truncated and
    sampled-column forms: two gloo ranks give the single-process estimate."""
    rng = np.random.default_rng(3)
    n_sim, nb, n_fd = 10, 5, 6
    nR = D.fisher_rows(nb, leak, fdb)
    E_all = rng.uniform(0.5, 2.0, size=(1 + n_sim + nR * n_fd, nb))
    theta = rng.uniform(0.5, 1.5, size=nb)
    ref = _reference(E_all, n_sim, nb, n_fd, theta, leak, trunc, fdb)
    if leak:
        assert not ref["fisher"][:leak, leak:].any() and not ref["fisher"][leak:, :leak].any()
    single = D.combine(D.local_sums(E_all, n_sim, nb, n_fd, leak, fdb), E_all[0], theta, leak, trunc, fdb)
    for k in ref:
        assert np.allclose(single[k], ref[k], rtol=1e-12), k
    mgr = mp.Manager()
    out = mgr.dict()
    port = _free_port()
    mp.start_processes(_worker, args=(2, port, n_sim, nb, n_fd, E_all, theta, out, leak, trunc, fdb), nprocs=2,
                       start_method="spawn", join=True)
    for rank in (0, 1):
        for k in ref:
            assert np.allclose(out[rank][k], ref[k], rtol=1e-12, atol=1e-14), (rank, k)


def test_combine_refuses_inconsistent_inputs():
    """Counts and rules are checked on the host before any arithmetic."""
    from paper_1810_00503_gb300 import wf
    nb = 3
    S = np.zeros(wf.lib().bandpower_sums_len(nb, nb))
    with pytest.raises(wf.WfError, match="EINVAL"):  # J = 0 simulations
        wf.bandpower_combine(S, np.ones(nb), np.ones(nb))
    S[0], S[1] = 4.0, 5.0  # more Fisher simulations than simulations
    with pytest.raises(wf.WfError, match="EINVAL"):
        wf.bandpower_combine(S, np.ones(nb), np.ones(nb))
    S[1] = 2.0
    with pytest.raises(wf.WfError, match="EINVAL"):  # fd_bands not ascending
        wf.bandpower_combine(np.zeros(wf.lib().bandpower_sums_len(nb, 2)) + 1.0, np.ones(nb), np.ones(nb),
                             fd_bands=[2, 0])
    with pytest.raises(ValueError):  # sums of the wrong length for the rules
        wf.bandpower_combine(S, np.ones(nb), np.ones(nb), leak_split=1)
