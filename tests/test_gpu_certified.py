"""Certified accuracy of the MAP at the benchmarked configurations, with the
oracle's FP64 gradient deciding the error bound.

Certificate (Sec. 2.2 in whitened variables): the half-Hessian I + A^T W A of
chi^2 has every eigenvalue >= 1, so for any state s the exact MAP s* satisfies
|s - s*| <= |grad chi2(s)| / 2.  Evaluating the oracle's FP64 gradient at the
state the GPU returns therefore bounds its error without an oracle solve:
|grad| / 2 <= 1e-4 |s| proves the relative L2 error target of the FP32 path
(1e-4), to first order.

The oracle is handed exactly the problem the library solves: the FP32 values
of d and W, and the signal amplitude sqrt(P)/n rounded to FP32 as the library
stores it (P_eff = (n fl32(sqrt(P)/n))^2, an exact square in FP64).  On the
CMB workload the curvature reaches ~2e6, where a relative perturbation of the
operator of 3e-8 already moves |grad| / 2 by ~1e-4 |s| although it moves the
MAP itself by ~1e-7; that is also why the certified solve keeps its state in
FP64 (an FP32-rounded exact MAP has |grad| / 2 ~ 1.8e-4 |s| there)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import wf_oracle as O  # noqa: E402
from paper_1810_00503_gb300 import synth, wf  # noqa: E402
from tests.helpers import ensure_lib, make_problem  # noqa: E402

TOL = 1e-4


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    ensure_lib()


def p_eff(P32, n):
    """Per-mode power whose FP64 sqrt(P)/n equals the library's FP32 table."""
    sp = (np.sqrt(P32.astype(np.float64)) / n).astype(np.float32).astype(np.float64)
    return (n * sp) ** 2


def oracle_cert(s_half, d, W, P, n):
    """|grad chi2(s)| / (2 |s|) by the oracle, s a half-plane unitary spectrum."""
    z = np.fft.irfft2(np.asarray(s_half, dtype=np.complex128), s=(n, n), norm="ortho")
    g = O.grad(z, d, W, P)
    return 0.5 * np.linalg.norm(g) / np.linalg.norm(z)


def cmb_bench_maps(idx, n=1024, B=120):
    """Maps `idx` of the benchmark's batch: the 1024^2 CMB patch, 120 simulated
    data maps from torch's device generator seeded 1000 (signal then noise
    fields), as bench.py makes them."""
    dev = torch.device("cuda")
    inp = synth.cmb_patch(n, seed=3)
    g = torch.Generator(device=dev)
    g.manual_seed(1000)
    Ninv = torch.as_tensor(inp.Ninv, dtype=torch.float32, device=dev)
    mask = torch.as_tensor(inp.mask, dtype=torch.uint8, device=dev)
    P = torch.as_tensor(inp.P_half, dtype=torch.float32, device=dev)
    z = torch.randn(B, 1, n, n, generator=g, device=dev)
    sig = torch.where(Ninv > 0, torch.rsqrt(torch.clamp(Ninv, min=1e-30)), torch.zeros_like(Ninv))
    noise = torch.randn(B, 1, n, n, generator=g, device=dev) * sig
    k = len(idx)
    Nk = Ninv[None].expand(k, -1, -1, -1).contiguous()
    prob = wf.Problem(torch.zeros_like(Nk), mask, Nk, P, precision="mixed")
    d = prob.simulate(z[list(idx)].contiguous(), noise[list(idx)].contiguous())
    prob.set_data(d)
    del z, noise
    W = (inp.mask[None] * inp.Ninv.astype(np.float32)).astype(np.float64)
    host = dict(d=d.cpu().numpy().astype(np.float64), W=W, P=p_eff(inp.P.astype(np.float32), n))
    return prob, host


def test_refined_mixed_solve_certified_on_cmb_1024():
    """Maps 0, 57 and 119 of the benchmark's 120 x 1024^2 CMB batch, solved in
    mixed precision with FP64 refinement to the 1e-4 certificate; the oracle's
    gradient at the returned FP64 states confirms it, and the library's own
    certificate agrees with the oracle's."""
    idx = (0, 57, 119)
    n = 1024
    prob, host = cmb_bench_maps(idx)
    res, cert = prob.solve_refined(cert_tol=TOL, max_rounds=6, gtol_rel=1e-6, max_iter=20000, check_every=64)
    assert all(st["status"] == "WF_OK" for st in res.stats), res.stats
    for b in range(len(idx)):
        c = oracle_cert(res.s[b].cpu().numpy(), host["d"][b], host["W"], host["P"], n)
        assert c <= TOL, (idx[b], c, cert[b])
        assert abs(c - cert[b]) <= 1e-3 * c + 1e-12, (idx[b], c, cert[b])
        # the FP32 rounding of the certified state adds at most 2^-24 |s|
        assert res.stats[b]["chi2"] > 0
    prob.close()


def test_plain_mixed_solve_certified_on_shear_eb_512():
    """The 512^2 joint E/B workload solved by the plain mixed path (FP32 state,
    periodic FP32 refresh, |g| / |g0| < 1e-6): its returned FP32 state already
    passes the oracle's 1e-4 certificate (the E/B curvature is mild)."""
    n = 512
    inp = synth.shear_eb(n, seed=2)
    prob, host = make_problem([inp], "mixed")
    res = prob.solve(gtol_rel=1e-6, max_iter=20000, check_every=64, refresh_every=200)
    assert res.stats[0]["status"] == "WF_OK", res.stats
    P = p_eff(host["P"][0].astype(np.float32), n)
    c = oracle_cert(res.s[0].cpu().numpy(), host["d"][0], host["W"][0], P, n)
    assert c <= TOL, c
    res2, cert = prob.solve_refined(cert_tol=1e-6, max_rounds=6, gtol_rel=1e-6, max_iter=20000)
    c2 = oracle_cert(res2.s[0].cpu().numpy(), host["d"][0], host["W"][0], P, n)
    assert res2.stats[0]["status"] == "WF_OK" and c2 <= 1e-6, (c2, cert, res2.stats)
    prob.close()


def test_refined_fp64_problem_and_degenerate_maps():
    """The same call on an FP64 problem (FP64 inner rounds) certifies a 64^2
    E/B map far below 1e-4, and maps with zero data stop at s = 0 with a zero
    certificate after one outer evaluation."""
    n = 64
    inp = synth.shear_eb(n, seed=5)
    d0 = O.synthesize_data(inp.z, inp.noise, inp.mask, inp.P)
    prob, host = make_problem([inp, inp], "fp64", d_list=[d0, 0.0 * d0])
    res, cert = prob.solve_refined(cert_tol=1e-10, max_rounds=4, gtol_rel=1e-8, max_iter=5000)
    assert [st["status"] for st in res.stats] == ["WF_OK", "WF_OK"], res.stats
    c = oracle_cert(res.s[0].cpu().numpy(), host["d"][0], host["W"][0], host["P"][0], n)
    assert c <= 1e-10, (c, cert)
    assert cert[1] == 0.0 and np.abs(res.s[1].cpu().numpy()).max() == 0.0
    assert res.stats[1]["iters"] == 0
    zs, _ = O.map_solve(host["d"][0], host["W"][0], host["P"][0], gtol_rel=1e-13, max_iter=5000)
    s_ref = np.fft.rfft2(zs, norm="ortho")
    assert np.linalg.norm(res.s[0].cpu().numpy() - s_ref) <= 1e-9 * np.linalg.norm(s_ref)
    prob.close()


def test_refined_rejects_bad_arguments():
    inp = synth.density_small(16, seed=1)
    prob, _ = make_problem([inp], "mixed")
    for kw in (dict(cert_tol=0.0), dict(cert_tol=float("nan")), dict(max_rounds=0)):
        with pytest.raises(wf.WfError, match="EINVAL"):
            prob.solve_refined(**kw)
    prob.close()
