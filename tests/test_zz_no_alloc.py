"""The allocation-free objective + gradient entry point (wf_eval_noalloc),
called through the C ABI, agrees with the regular wf_eval on two calls in a
row with different inputs, and with the FP64 oracle at its largest documented
batch (three 1024^2 maps in FP32).  Its scratch sits in a static device array
shared by all calls, so the second call also shows that the first call's
leftovers do not leak into its result.  The first call on a device writes the
twiddle tables into that array; a fresh process makes that first call on a
non-blocking side stream.  This file is collected last on purpose."""
import os
import subprocess
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import wf_oracle as O  # noqa: E402
from paper_1810_00503_gb300 import synth, wf  # noqa: E402
from tests.helpers import ensure_lib, make_problem, rel, rfft_u, to_dev  # noqa: E402

TOL = {"fp64": 1e-12, "mixed": 2e-5}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    ensure_lib()


def _case(n, C, B, seed, precision):
    inputs = [synth.density_small(n, seed=seed + b) if C == 1 else synth.shear_eb(n, seed=seed)
              for b in range(B)]
    prob, host = make_problem(inputs, precision, shared_P=True)
    wdt = torch.float64 if precision == "fp64" else torch.float32
    cdt = torch.complex128 if precision == "fp64" else torch.complex64
    d = to_dev(np.stack([dd * m[None] for dd, m in zip(host["d"], host["mask"])]), wdt)
    w = to_dev(np.stack(host["W"]), wdt)
    P = to_dev(host["P"][0][..., : n // 2 + 1], wdt)
    S = np.stack([rfft_u(synth.random_state(n, C, seed=seed + 50 + b)) for b in range(B)])
    s = to_dev(S, cdt)
    return prob, s, d, w, P


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_noalloc_matches_wf_eval_on_two_calls(precision):
    cases = [_case(256, 1, 2, 11, precision), _case(64, 2, 1, 23, precision)]
    for prob, s, d, w, P in cases:
        ref_c, ref_g = prob.eval(s)
        c, g = wf.eval_noalloc(s, d, w, P)
        torch.cuda.synchronize()
        assert rel(g.cpu().numpy(), ref_g.cpu().numpy()) <= TOL[precision]
        assert np.allclose(c.cpu().numpy(), ref_c.cpu().numpy(), rtol=TOL[precision], atol=0)


def test_noalloc_rejects_batches_beyond_its_scratch():
    dt = torch.float64
    n, C, B = 1024, 2, 1
    s = torch.zeros((B, C, n, n // 2 + 1), dtype=torch.complex128, device="cuda")
    d = torch.zeros((B, C, n, n), dtype=dt, device="cuda")
    P = torch.zeros((C, n, n // 2 + 1), dtype=dt, device="cuda")
    with pytest.raises(wf.WfError, match="EINVAL.*static"):
        wf.eval_noalloc(s, d, d, P)


def test_noalloc_matches_oracle_at_its_largest_batch():
    """Three 1024^2 CMB-like maps in FP32, the most the static scratch holds
    at that size, against the oracle's chi2 and gradient map by map."""
    n, B = 1024, 3
    inp = synth.cmb_patch(n, seed=3)
    rng = np.random.default_rng(5)
    W = (inp.mask[None] * inp.Ninv).astype(np.float32).astype(np.float64)
    P = inp.P.astype(np.float32).astype(np.float64)
    ds, ss = [], []
    for b in range(B):
        z = rng.standard_normal((1, n, n))
        noise = rng.standard_normal((1, n, n)) / np.sqrt(np.where(inp.Ninv > 0, inp.Ninv, 1.0))
        ds.append(O.synthesize_data(z, noise, inp.mask, inp.P).astype(np.float32).astype(np.float64))
        ss.append(rfft_u(rng.standard_normal((1, n, n))).astype(np.complex64).astype(np.complex128))
    d_t = to_dev(np.stack(ds), torch.float32)
    w_t = to_dev(np.broadcast_to(W, (B, 1, n, n)), torch.float32)
    P_t = to_dev(P[..., : n // 2 + 1], torch.float32)
    s_t = to_dev(np.stack(ss), torch.complex64)
    for call in range(2):
        c, g = wf.eval_noalloc(s_t, d_t, w_t, P_t)
        torch.cuda.synchronize()
        for b in range(B):
            z = np.fft.irfft2(ss[b], s=(n, n), norm="ortho")
            rc = O.chi2(z, ds[b], W, P)
            rg = rfft_u(O.grad(z, ds[b], W, P))
            assert abs(c[b].item() - rc) <= 1e-5 * abs(rc), (call, b)
            assert rel(g[b].cpu().numpy(), rg) <= TOL["mixed"], (call, b)


_FRESH = r"""
import sys
sys.path.insert(0, {root!r})
import numpy as np, torch
from oracle import wf_oracle as O
from paper_1810_00503_gb300 import synth, wf
from tests.helpers import rel, rfft_u, to_dev
n = 64
inp = synth.density_small(n, seed=9)
d = O.synthesize_data(inp.z, inp.noise, inp.mask, inp.P)
W = inp.mask[None] * inp.Ninv
z = synth.random_state(n, 1, seed=10)
side = torch.cuda.Stream()
with torch.cuda.stream(side):
    dt, wt = to_dev(d[None], torch.float64), to_dev(W[None], torch.float64)
    Pt = to_dev(inp.P[..., : n // 2 + 1], torch.float64)
    st = to_dev(rfft_u(z)[None], torch.complex128)
    c, g = wf.eval_noalloc(st, dt, wt, Pt, stream=side)
side.synchronize()
rc, rg = O.chi2(z, d, W, inp.P), rfft_u(O.grad(z, d, W, inp.P))
assert abs(c[0].item() - rc) <= 1e-12 * abs(rc), (c[0].item(), rc)
assert rel(g[0].cpu().numpy(), rg) <= 1e-12
print("fresh-process first call ok")
"""


def test_first_call_in_a_fresh_process_on_a_side_stream():
    """The first call on a device writes the twiddle tables, then waits for
    them; here it is issued on a non-blocking torch side stream, and its result
    must already match the oracle."""
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, "-c", _FRESH.format(root=root)], capture_output=True, text=True,
                         timeout=600, cwd=root)
    assert out.returncode == 0, out.stdout + out.stderr
