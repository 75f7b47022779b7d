"""GPU MAP solves (device L-BFGS with exact line search) against the FP64 oracle.

Tolerances follow the stated targets: relative L2 error of s_MAP <= 1e-10 for
the FP64 path and <= 1e-4 for the mixed FP32/FP64 path.  The FP64 reference
is the dense Wiener filter (32^2) or the oracle's textbook L-BFGS driven to
||g|| / ||g0|| < 1e-11, whose own error is bounded by the certificate
||s - s*|| <= ||grad|| / 2 (the half-Hessian has lambda_min >= 1)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import wf_oracle as O  # noqa: E402
from paper_1810_00503_gb300 import synth, wf  # noqa: E402
from tests.helpers import ensure_lib, make_problem, rel, rfft_u, to_dev  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    ensure_lib()


def test_fp64_density_32_matches_dense_wiener_filter():
    inp = synth.density_small(32, seed=0)
    prob, host = make_problem([inp], "fp64")
    res = prob.solve(gtol_rel=1e-12, max_iter=5000)
    assert res.stats[0]["status"] == "WF_OK", res.stats
    zs = O.dense_wf_whitened(host["d"][0], host["W"][0], host["P"][0])
    err = rel(res.s[0].cpu().numpy(), rfft_u(zs))
    assert err <= 1e-10, err
    assert abs(res.stats[0]["chi2"] - O.chi2(zs, host["d"][0], host["W"][0], host["P"][0])) \
        <= 1e-10 * res.stats[0]["chi2"]
    assert res.stats[0]["gnorm_rel"] <= 1e-11


@pytest.mark.parametrize("C", [1, 2])
def test_fp64_unmasked_closed_form(C):
    n, sig2 = 64, 0.2
    inp = synth.density_small(n, seed=3) if C == 1 else synth.shear_eb(n, seed=3)
    inp.mask[:] = 1
    inp.Ninv[:] = 1.0 / sig2
    d = O.synthesize_data(inp.z, inp.noise, inp.mask, inp.P)
    prob, host = make_problem([inp], "fp64", d_list=[d])
    res = prob.solve(gtol_rel=1e-12, max_iter=3000)
    # per mode: s* = R^T-free closed form only for C = 1; for C = 2 the rotation is
    # orthogonal off the Nyquist lines, so use the dense-free oracle L-BFGS instead.
    if C == 1:
        zstar = O.ifft2u(np.sqrt(inp.P) * O.fft2u(d) / (inp.P + sig2)).real
    else:
        zstar, _ = O.map_solve(d, host["W"][0], host["P"][0], gtol_rel=1e-13, max_iter=3000)
    assert rel(res.s[0].cpu().numpy(), rfft_u(zstar)) <= 1e-10


def test_fp64_batch_of_maps_and_signal_map():
    maps = [synth.density_small(32, seed=s) for s in (1, 2, 3)]
    prob, host = make_problem(maps, "fp64")
    res = prob.solve(gtol_rel=1e-12, max_iter=5000, x_out=True)
    for b in range(3):
        zs = O.dense_wf_whitened(host["d"][b], host["W"][b], host["P"][b])
        assert rel(res.s[b].cpu().numpy(), rfft_u(zs)) <= 1e-10
        assert rel(res.x[b].cpu().numpy(), O.apply_A(zs, host["P"][b])) <= 1e-10


def test_fp64_shear_eb_64_matches_oracle_lbfgs():
    inp = synth.shear_eb(64, seed=7)
    prob, host = make_problem([inp], "fp64")
    res = prob.solve(gtol_rel=1e-12, max_iter=5000)
    zs, info = O.map_solve(host["d"][0], host["W"][0], host["P"][0], gtol_rel=1e-13, max_iter=5000)
    g = O.grad(zs, host["d"][0], host["W"][0], host["P"][0])
    assert 0.5 * np.linalg.norm(g) <= 1e-12 * np.linalg.norm(zs)  # oracle certified
    assert rel(res.s[0].cpu().numpy(), rfft_u(zs)) <= 1e-10


def test_mixed_density_256_within_1e4():
    inp = synth.density_projected(256, seed=1)
    prob, host = make_problem([inp], "mixed")
    res = prob.solve(gtol_rel=1e-6, max_iter=3000, refresh_every=64)
    zs, info = O.map_solve(host["d"][0], host["W"][0], host["P"][0], gtol_rel=1e-11, max_iter=5000)
    err = rel(res.s[0].cpu().numpy(), rfft_u(zs))
    assert err <= 1e-4, (err, res.stats)


def test_iteration_limit_and_warm_start():
    inp = synth.density_small(32, seed=4)
    prob, host = make_problem([inp], "fp64")
    res = prob.solve(gtol_rel=1e-14, max_iter=5)
    assert res.stats[0]["status"] == "WF_ENOTCONVERGED"
    assert res.stats[0]["iters"] == 5
    full = prob.solve(gtol_rel=1e-12, max_iter=5000)
    # gtol_rel is relative to the starting gradient, so a warm start is tested
    # with the Delta chi^2 rule: chi^2 no longer changes after the first step.
    warm = prob.solve(s0=full.s, gtol_rel=0.0, dchi2_abs=1e-9, max_iter=5000)
    assert warm.stats[0]["iters"] <= 2
    assert rel(warm.s[0].cpu().numpy(), full.s[0].cpu().numpy()) <= 1e-11


def test_delta_chi2_rule_stops_early():
    inp = synth.density_small(32, seed=5)
    prob, host = make_problem([inp], "fp64")
    loose = prob.solve(gtol_rel=0.0, dchi2_abs=0.1, max_iter=5000)
    tight = prob.solve(gtol_rel=1e-12, max_iter=5000)
    assert loose.stats[0]["status"] == "WF_OK"
    assert loose.stats[0]["iters"] < tight.stats[0]["iters"]
    assert loose.stats[0]["chi2"] - tight.stats[0]["chi2"] < 1.0


def test_graphs_and_plain_launches_agree():
    inp = synth.density_small(64, seed=6)
    prob, host = make_problem([inp], "fp64")
    a = prob.solve(gtol_rel=1e-10, max_iter=2000, use_graphs=1, check_every=8)
    b = prob.solve(gtol_rel=1e-10, max_iter=2000, use_graphs=0, check_every=8)
    assert a.stats[0]["iters"] == b.stats[0]["iters"]
    assert rel(a.s[0].cpu().numpy(), b.s[0].cpu().numpy()) <= 1e-13


def test_heterogeneous_batch_solved_together():
    # maps of uneven size (one problem per shape), solved concurrently; each map
    # agrees with the oracle's own L-BFGS minimiser.
    from paper_1810_00503_gb300 import wf
    maps = synth.hetero_batch(count=9, seed=4, sizes=(64, 128, 256))
    groups = {}
    for m in maps:
        groups.setdefault(m.n, []).append(m)
    probs, hosts, order = [], [], []
    for n in sorted(groups):
        pr, ho = make_problem(groups[n], "fp64", shared_P=False)
        probs.append(pr); hosts.append(ho); order.append(n)
    res = wf.solve_many(probs, gtol_rel=1e-11, max_iter=20000)
    for r, ho, n in zip(res, hosts, order):
        assert all(s["status"] == "WF_OK" for s in r.stats), r.stats
        b = 0
        zs, info = O.map_solve(ho["d"][b], ho["W"][b], ho["P"][b], gtol_rel=1e-12, max_iter=20000)
        assert rel(r.s[b].cpu().numpy(), rfft_u(zs)) <= 1e-9, n


@pytest.mark.parametrize("case", ["all_masked", "zero_data", "zero_power"])
def test_degenerate_problems(case):
    # Degenerate cases of the method: with no observed pixel, no data or no
    # signal power the MAP field is 0 and the solver stops at once.
    n = 32
    inp = synth.density_small(n, seed=2)
    d = O.synthesize_data(inp.z, inp.noise, inp.mask, inp.P)
    if case == "all_masked":
        inp.mask[:] = 0
        inp.Ninv[:] = 0.0
        d = d * 0.0
    elif case == "zero_data":
        d = d * 0.0
    else:
        inp.P[:] = 0.0
    prob, host = make_problem([inp], "fp64", d_list=[d])
    res = prob.solve(gtol_rel=1e-10, max_iter=100)
    assert res.stats[0]["status"] == "WF_OK"
    assert res.stats[0]["iters"] == 0
    assert np.abs(res.s[0].cpu().numpy()).max() == 0.0


def test_mixed_cmb_256_within_1e4():
    # CMB-like red spectrum (the paper's hardest conditioning) in FP32 fields with
    # FP64 reductions and periodic true-gradient refresh.
    inp = synth.cmb_patch(256, seed=3)
    prob, host = make_problem([inp], "mixed")
    res = prob.solve(gtol_rel=1e-7, max_iter=20000, refresh_every=100)
    zs, info = O.map_solve(host["d"][0], host["W"][0], host["P"][0], gtol_rel=1e-11, max_iter=20000)
    err = rel(res.s[0].cpu().numpy(), rfft_u(zs))
    assert err <= 1e-4, (err, res.stats)


def test_mixed_shear_eb_256_within_1e4():
    inp = synth.shear_eb(256, seed=2)
    prob, host = make_problem([inp], "mixed")
    res = prob.solve(gtol_rel=1e-7, max_iter=20000, refresh_every=100)
    zs, info = O.map_solve(host["d"][0], host["W"][0], host["P"][0], gtol_rel=1e-11, max_iter=20000)
    err = rel(res.s[0].cpu().numpy(), rfft_u(zs))
    assert err <= 1e-4, (err, res.stats)


def test_wolfe_fp64_density_32_matches_dense_wiener_filter():
    inp = synth.density_small(32, seed=0)
    prob, host = make_problem([inp], "fp64")
    res = prob.solve(gtol_rel=1e-12, max_iter=5000, line_search=wf.WF_LS_WOLFE)
    assert res.stats[0]["status"] == "WF_OK", res.stats
    zs = O.dense_wf_whitened(host["d"][0], host["W"][0], host["P"][0])
    assert rel(res.s[0].cpu().numpy(), rfft_u(zs)) <= 1e-10


def test_wolfe_iterates_follow_the_textbook_search():
    """Five L-BFGS iterations with the strong Wolfe search: the device runs
    Alg. 3.5/3.6 on the closed-form line model, the oracle on true objective
    evaluations.  Both accept the same trial steps; inside a zoom the oracle's
    interpolated step carries the rounding of chi^2 differences (chi^2 ~ 1e3
    against changes a few orders smaller), so the iterates agree to ~1e-8,
    while one different accept/reject decision would move them by ~1e-2."""
    inp = synth.shear_eb(32, seed=4)
    prob, host = make_problem([inp], "fp64")
    for k in (1, 2, 5):
        res = prob.solve(gtol_rel=0.0, max_iter=k, line_search=wf.WF_LS_WOLFE, use_graphs=0)
        zk, info = O.map_solve(host["d"][0], host["W"][0], host["P"][0], gtol_rel=0.0, max_iter=k)
        assert info["iters"] == k and res.stats[0]["iters"] == k
        assert rel(res.s[0].cpu().numpy(), rfft_u(zk)) <= 1e-7, k


def test_wolfe_mixed_shear_eb_256_within_1e4():
    inp = synth.shear_eb(256, seed=2)
    prob, host = make_problem([inp], "mixed")
    res = prob.solve(gtol_rel=1e-6, max_iter=4000, refresh_every=64, line_search=wf.WF_LS_WOLFE)
    zs, info = O.map_solve(host["d"][0], host["W"][0], host["P"][0], gtol_rel=1e-11, max_iter=6000)
    assert rel(res.s[0].cpu().numpy(), rfft_u(zs)) <= 1e-4, res.stats


@pytest.mark.parametrize("bad", [dict(line_search=2), dict(line_search=1, c1=0.5, c2=0.4),
                                 dict(line_search=1, c1=0.0), dict(line_search=1, c2=1.0)])
def test_bad_line_search_options_rejected(bad):
    inp = synth.density_small(16, seed=1)
    prob, host = make_problem([inp], "fp64")
    with pytest.raises(wf.WfError, match="EINVAL"):
        prob.solve(max_iter=3, **bad)


def test_mixed_heterogeneous_batch_one_graph_each_size_certified():
    """One map of each size 64^2 .. 1024^2 of the heterogeneous workload, in
    mixed precision: the batch solve (one graph launch per round for all
    sizes) stops every map with WF_OK, and a refined solve warm-started from
    each batch solution is certified to 1e-4 by the oracle's gradient."""
    from tests.test_gpu_certified import oracle_cert, p_eff
    sizes = (64, 128, 256, 512, 1024)
    maps = synth.hetero_batch(count=24, seed=4, sizes=sizes)
    first = {}
    for m in maps:
        first.setdefault(m.n, m)
    assert sorted(first) == list(sizes)
    probs, hosts = [], []
    for n in sizes:
        pr, ho = make_problem([first[n]], "mixed")
        probs.append(pr)
        hosts.append(ho)
    res = wf.solve_many(probs, gtol_rel=1e-6, max_iter=20000, check_every=16, refresh_every=200)
    for r, n in zip(res, sizes):
        assert [s["status"] for s in r.stats] == ["WF_OK"], (n, r.stats)
    for p, r, ho, n in zip(probs, res, hosts, sizes):
        ref, cert = p.solve_refined(s0=r.s, cert_tol=1e-4, gtol_rel=1e-5, max_iter=20000)
        P = p_eff(ho["P"][0].astype(np.float32), n)
        c = oracle_cert(ref.s[0].cpu().numpy(), ho["d"][0], ho["W"][0], P, n)
        assert c <= 1e-4, (n, c, cert)
        s_ref = ref.s[0].cpu().numpy()
        assert rel(r.s[0].cpu().numpy().astype(np.complex128), s_ref) <= 1e-2, n
        p.close()
