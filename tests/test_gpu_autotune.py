"""FFT-stage variants of the Hessian-vector pass and the autotuner that picks
among them.  Every variant computes the same operator (Eq. 4-5 through the
three FFT stages), so every forced variant must reach the oracle's MAP solution
to the same tolerance as the default one: 1e-10 relative L2 for FP64, 1e-4 for
the mixed path."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import wf_oracle as O  # noqa: E402
from paper_1810_00503_gb300 import synth, wf  # noqa: E402
from tests.helpers import ensure_lib, make_problem, rel, rfft_u  # noqa: E402

# column / row radix plan (0: large radix first, 1: ascending, 2: radix 32 for
# lengths 512 and 1024), inverse column stage (1 TMA, 2 ping-pong, 3 in-place),
# row stage (1 ping-pong, 2 in-place), column / row tile narrowing 1, 2, 4
VARIANTS = [1111, 1211, 2111, 2211, 3111, 3211, 1142, 2124, 3244, 1222, 2141, 3114,
            11111, 111111, 212111, 121142]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    ensure_lib()


def _valid(v):
    f, e = v // 100000, (v // 10000) % 10
    a, b, c, d = (v // 1000) % 10, (v // 100) % 10, (v // 10) % 10, v % 10
    return (f in (0, 1, 2) and e in (0, 1, 2) and a in (1, 2, 3) and b in (1, 2) and c in (1, 2, 4)
            and d in (1, 2, 4))


@pytest.fixture(scope="module")
def shear64():
    inp = synth.shear_eb(64, seed=11)
    _, host = make_problem([inp], "fp64")
    zs, _ = O.map_solve(host["d"][0], host["W"][0], host["P"][0], gtol_rel=1e-13, max_iter=5000)
    g = O.grad(zs, host["d"][0], host["W"][0], host["P"][0])
    assert 0.5 * np.linalg.norm(g) <= 1e-12 * np.linalg.norm(zs)  # oracle certified
    return inp, zs


@pytest.mark.parametrize("variant", VARIANTS)
def test_forced_variant_fp64_shear_eb_matches_oracle(shear64, variant):
    inp, zs = shear64
    prob, host = make_problem([inp, inp], "fp64")
    res = prob.solve(gtol_rel=1e-12, max_iter=5000, fft_variant=variant)
    assert prob.variant() == variant
    for b in range(2):
        assert res.stats[b]["status"] == "WF_OK", res.stats
        assert rel(res.s[b].cpu().numpy(), rfft_u(zs)) <= 1e-10
    # the objective pass on the chosen stages agrees with the oracle too
    chi2, grad = prob.eval(res.s.contiguous())
    c_ref = O.chi2(zs, host["d"][0], host["W"][0], host["P"][0])
    assert abs(chi2[0].item() - c_ref) <= 1e-10 * c_ref


@pytest.mark.parametrize("variant", [1111, 2211, 3124, 1242])
def test_forced_variant_mixed_density_128(variant):
    inp = synth.density_projected(128, seed=4)
    prob, host = make_problem([inp], "mixed")
    res = prob.solve(gtol_rel=1e-6, max_iter=3000, refresh_every=64, fft_variant=variant)
    assert res.stats[0]["status"] == "WF_OK", res.stats
    zs, _ = O.map_solve(host["d"][0], host["W"][0], host["P"][0], gtol_rel=1e-12, max_iter=5000)
    assert rel(res.s[0].cpu().numpy(), rfft_u(zs)) <= 1e-4


def test_autotune_picks_a_valid_variant_and_caches_it(shear64):
    inp, zs = shear64
    h = wf.Handle()
    probs = []
    for _ in range(2):  # same shape and batch size twice on one handle
        prob, _ = _on_handle(h, [inp, inp, inp])
        res = prob.solve(gtol_rel=1e-12, max_iter=5000)
        for b in range(3):
            assert rel(res.s[b].cpu().numpy(), rfft_u(zs)) <= 1e-10
        assert _valid(prob.variant()), prob.variant()
        probs.append(prob)
    assert probs[0].variant() == probs[1].variant()
    # autotune off: the built-in default (widest tiles, ping-pong rows)
    prob, _ = _on_handle(h, [inp])
    prob.solve(gtol_rel=1e-8, max_iter=2000, autotune=0)
    assert prob.variant() in (1111, 2111), prob.variant()
    # the history length is part of the tuned shape
    prob, _ = _on_handle(h, [inp, inp, inp])
    res = prob.solve(gtol_rel=1e-12, max_iter=5000, lbfgs_m=5)
    assert _valid(prob.variant()), prob.variant()
    for b in range(3):
        assert rel(res.s[b].cpu().numpy(), rfft_u(zs)) <= 1e-10


def _on_handle(h, inputs):
    """make_problem on an explicit handle."""
    from tests.helpers import to_dev
    n = inputs[0].n
    ds = [O.synthesize_data(i.z, i.noise, i.mask, i.P) for i in inputs]
    prob = wf.Problem(to_dev(np.stack(ds), torch.float64), to_dev(np.stack([i.mask for i in inputs]), torch.uint8),
                      to_dev(np.stack([i.Ninv for i in inputs]), torch.float64),
                      to_dev(inputs[0].P[..., : n // 2 + 1], torch.float64), precision="fp64", handle=h)
    return prob, ds


@pytest.mark.parametrize("bad", [5, 999, 4111, 1311, 1131, 1113, 10111, 31111, 301111, 1000000, -1111])
def test_bad_variant_codes_rejected(bad):
    inp = synth.density_small(32, seed=0)
    prob, _ = make_problem([inp], "fp64")
    with pytest.raises(wf.WfError) as ei:
        prob.solve(max_iter=10, fft_variant=bad)
    assert ei.value.status == 1  # WF_EINVAL


def _cmb_fp64(n, B):
    inp = synth.cmb_patch(n, seed=3)
    d = O.synthesize_data(inp.z, inp.noise, inp.mask, inp.P)
    prob, host = make_problem([inp] * B, "fp64", d_list=[d] * B)
    return prob, host


# Radix plans at the lengths where they differ: 512 (columns at n = 512, rows
# at n = 1024) and 1024 (columns at n = 1024); both column stages and the row
# stage, TMA-fed and ping-pong.
PLAN_VARIANTS = [201111, 221111, 111111, 222111, 122211, 211142]


@pytest.mark.parametrize("n", [512, 1024])
@pytest.mark.parametrize("variant", PLAN_VARIANTS)
def test_radix_plans_objective_matches_oracle(n, variant):
    # the objective pass runs on the problem's chosen stages: chi2 and gradient
    # at a random state against the oracle (FP64)
    prob, host = _cmb_fp64(n, 1)
    prob.solve(gtol_rel=1e-12, max_iter=2, fft_variant=variant)
    assert prob.variant() == variant
    z = synth.random_state(n, 1, seed=n + variant % 97)
    s = torch.as_tensor(rfft_u(z)[None], device="cuda")
    chi2, grad = prob.eval(s.contiguous())
    c_ref = O.chi2(z, host["d"][0], host["W"][0], host["P"][0])
    g_ref = O.grad(z, host["d"][0], host["W"][0], host["P"][0])
    assert abs(chi2[0].item() - c_ref) <= 1e-12 * c_ref
    # the library's gradient is the half-plane spectrum of the pixel gradient
    assert rel(grad[0].cpu().numpy(), rfft_u(g_ref)) <= 1e-11


@pytest.mark.parametrize("variant", PLAN_VARIANTS + [1142, 2124, 3111])
def test_radix_plans_iterate_like_the_default(variant):
    # the Hessian-vector stages of the iteration: three FP64 L-BFGS iterations
    # on two 1024^2 maps follow the default variant's iterates to rounding
    # (further on, rounding differences grow with the iteration count on this
    # ill-conditioned problem, as in any Krylov method)
    runs = []
    for v in (1111, variant):
        prob, _ = _cmb_fp64(1024, 2)
        res = prob.solve(gtol_rel=0.0, max_iter=3, check_every=1, fft_variant=v)
        runs.append(res.s.cpu().numpy())
    assert rel(runs[1], runs[0]) <= 1e-11
