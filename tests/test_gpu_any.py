"""Objective, gradient and Hessian-vector product on grids whose sides are not
powers of two (wf_eval_any: mixed-radix transforms with radix 2, 3, 4, 5 and 7
passes) against the FP64 oracle, which takes grids of any side lengths
(Sec. 2.2, eq_chi and eq_cost; the E/B rotation of App. C at the wavevector
(mx / nx, my / ny), sine 0 on the Nyquist line of an even side).

Shapes cover odd and even sides, every radix, one-pass and many-pass lengths,
narrow strips, column tiles with a ragged last tile, the 1024 limit and sizes
of the paper's kind that are not powers of two (360, 640, 768, 1000).
Tolerances as the power-of-two tests: FP64 fields and chi^2 1e-12 (relative
L2), mixed fields 2e-5 and chi^2 1e-5."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import wf_oracle as O  # noqa: E402
from paper_1810_00503_gb300 import synth, wf  # noqa: E402
from tests.helpers import any_inputs, ensure_lib, make_problem, rel, rfft_u, to_dev  # noqa: E402

TOL = {"fp64": dict(field=1e-12, chi2=1e-12), "mixed": dict(field=2e-5, chi2=1e-5)}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    ensure_lib()


def _run(ny, nx, C, B, precision, seed, hess=False):
    I = any_inputs(ny, nx, C, B, seed)
    wdt = torch.float64 if precision == "fp64" else torch.float32
    cdt = torch.complex128 if precision == "fp64" else torch.complex64
    npw = np.float64 if precision == "fp64" else np.float32
    npc = np.complex128 if precision == "fp64" else np.complex64
    h1 = nx // 2 + 1
    # the values the GPU sees, rounded to the working type, are what the oracle gets
    P = I["P"].astype(npw).astype(np.float64)
    Ninv = [a.astype(npw).astype(np.float64) for a in I["Ninv"]]
    d = [a.astype(npw).astype(np.float64) for a in I["d"]]
    S = np.stack([rfft_u(f) for f in I["f"]]).astype(npc)
    z = [np.fft.irfft2(S[b].astype(np.complex128), s=(ny, nx), norm="ortho") for b in range(B)]
    chi2, g = wf.eval_any(to_dev(S, cdt), to_dev(np.stack(I["mask"]), torch.uint8), to_dev(np.stack(Ninv), wdt),
                          to_dev(np.ascontiguousarray(P[..., :h1]), wdt),
                          d=None if hess else to_dev(np.stack(d), wdt))
    torch.cuda.synchronize()
    tol = TOL[precision]
    for b in range(B):
        W = I["mask"][b][None] * Ninv[b]
        if hess:
            rg = rfft_u(O.hess_vec(z[b], W, P))
            x = O.apply_A(z[b], P)
            rc = float(np.sum(z[b] * z[b]) + np.sum(x * W * x))
        else:
            rg = rfft_u(O.grad(z[b], d[b], W, P))
            rc = O.chi2(z[b], d[b], W, P)
        assert abs(chi2[b].item() - rc) <= tol["chi2"] * abs(rc), (b, chi2[b].item(), rc)
        assert rel(g[b].cpu().numpy(), rg) <= tol["field"], (b, rel(g[b].cpu().numpy(), rg))


CASES = [(2, 2, 1, 1, "fp64"), (3, 5, 1, 2, "fp64"), (5, 3, 2, 1, "fp64"), (6, 10, 2, 2, "fp64"),
         (9, 15, 1, 1, "fp64"), (12, 7, 2, 1, "fp64"), (7, 49, 2, 1, "fp64"), (30, 42, 1, 3, "fp64"),
         (42, 30, 2, 2, "fp64"), (96, 60, 1, 2, "fp64"), (60, 96, 2, 1, "fp64"), (343, 20, 1, 1, "fp64"),
         (20, 343, 2, 1, "fp64"), (1024, 6, 2, 1, "fp64"), (6, 1000, 2, 1, "fp64"), (360, 640, 2, 1, "fp64"),
         (1000, 1000, 1, 1, "fp64"),
         (15, 21, 2, 2, "mixed"), (100, 90, 1, 2, "mixed"), (360, 640, 2, 2, "mixed"), (768, 768, 1, 2, "mixed"),
         (1000, 360, 2, 1, "mixed"), (1024, 1000, 1, 1, "mixed")]


@pytest.mark.parametrize("ny,nx,C,B,precision", CASES)
def test_eval_any_matches_oracle(ny, nx, C, B, precision):
    _run(ny, nx, C, B, precision, seed=11 * ny + nx + C)


@pytest.mark.parametrize("ny,nx,C,precision", [(9, 15, 2, "fp64"), (60, 96, 1, "fp64"), (640, 360, 2, "mixed")])
def test_hess_vec_any_matches_oracle(ny, nx, C, precision):
    _run(ny, nx, C, 2, precision, seed=5 + ny, hess=True)


@pytest.mark.parametrize("n,C", [(64, 1), (128, 2)])
def test_eval_any_agrees_with_the_power_of_two_path(n, C):
    """On a power-of-two map both paths compute the same function: wf_eval
    (fused radix-2^k stages) and wf_eval_any agree to rounding in FP64."""
    inp = synth.density_small(n, seed=n) if C == 1 else synth.shear_eb(n, seed=n)
    prob, host = make_problem([inp, inp], "fp64")
    f = [synth.random_state(n, C, seed=s) for s in (1, 2)]
    s = to_dev(np.stack([rfft_u(x) for x in f]), torch.complex128)
    chi2, g = prob.eval(s)
    ca, ga = wf.eval_any(s, to_dev(np.stack(host["mask"]), torch.uint8), to_dev(np.stack(host["Ninv"]), torch.float64),
                         to_dev(np.ascontiguousarray(host["P"][0][..., : n // 2 + 1]), torch.float64),
                         d=to_dev(np.stack(host["d"]), torch.float64))
    torch.cuda.synchronize()
    prob.close()
    assert torch.allclose(ca, chi2, rtol=1e-13, atol=0)
    assert rel(ga.cpu().numpy(), g.cpu().numpy()) <= 1e-13


def test_eval_any_frees_its_scratch_and_respects_the_workspace_limit():
    big = wf.Handle()
    base = big.workspace_used()  # the handle's own twiddle tables
    small = wf.Handle(workspace_limit=base + 100 * 1024)
    I = any_inputs(300, 300, 1, 1, seed=1)
    s = to_dev(np.stack([rfft_u(f) for f in I["f"]]), torch.complex128)
    args = (to_dev(np.stack(I["mask"]), torch.uint8), to_dev(np.stack(I["Ninv"]), torch.float64),
            to_dev(np.ascontiguousarray(I["P"][..., :151]), torch.float64))
    with pytest.raises(wf.WfError, match="workspace limit"):
        wf.eval_any(s, *args, handle=small)  # 300 x 151 complex FP64 scratch: 725 KB
    assert small.workspace_used() == base
    wf.eval_any(s, *args, handle=big)
    assert big.workspace_used() == base
    small.close()
    big.close()
