"""Checkpoint and resume of a solve (wf_solver_export / wf_solver_import): a
solve stopped, saved and resumed in a fresh problem on a fresh handle ends
with exactly the iterates of the uninterrupted solve, from a device or a host
copy of the checkpoint."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import wf_oracle as O  # noqa: E402
from paper_1810_00503_gb300 import synth, wf  # noqa: E402
from tests.helpers import ensure_lib, to_dev  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    ensure_lib()


def _problem(precision, handle=None, n=128):
    inp = synth.cmb_patch(n, seed=3)
    rng = np.random.default_rng(31)
    ds = []
    for _ in range(2):
        noise = rng.standard_normal((1, n, n)) / np.sqrt(np.where(inp.Ninv > 0, inp.Ninv, 1.0))
        ds.append(O.synthesize_data(rng.standard_normal((1, n, n)), noise, inp.mask, inp.P))
    dt = torch.float64 if precision == "fp64" else torch.float32
    return wf.Problem(to_dev(np.stack(ds), dt), to_dev(inp.mask, torch.uint8),
                      to_dev(np.broadcast_to(inp.Ninv, (2, 1, n, n)), dt), to_dev(inp.P_half, dt),
                      precision=precision, handle=handle)


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_resume_equals_uninterrupted(precision):
    opts = dict(gtol_rel=1e-9, max_iter=5000, refresh_every=50, check_every=8, history=16)
    pa = _problem(precision)
    pa.start(**opts)
    pa.step(37)
    ck = pa.export_state()
    ck_host = ck.cpu()
    pa.step(70)
    ra = pa.finish()
    for buf in (ck, ck_host):
        pb = _problem(precision, handle=wf.Handle())
        pb.import_state(buf)
        pb.step(70)
        rb = pb.finish()
        assert torch.equal(ra.s, rb.s)
        assert [s["iters"] for s in ra.stats] == [s["iters"] for s in rb.stats]
        assert [s["chi2"] for s in ra.stats] == [s["chi2"] for s in rb.stats]
        assert [s["fft_variant"] for s in ra.stats] == [s["fft_variant"] for s in rb.stats]
        pb.close()
    pa.close()


def test_import_refuses_other_shapes_and_garbage():
    pa = _problem("mixed", n=64)
    pa.start(gtol_rel=1e-6, max_iter=100)
    pa.step(3)
    ck = pa.export_state()
    other = _problem("fp64", n=64)
    with pytest.raises(wf.WfError, match="EINVAL"):
        other.import_state(ck)
    bigger = _problem("mixed", n=128)
    with pytest.raises(wf.WfError, match="EINVAL"):
        bigger.import_state(ck)
    with pytest.raises(wf.WfError, match="EINVAL"):
        pa.import_state(torch.zeros_like(ck))
    with pytest.raises(wf.WfError, match="EINVAL"):
        pa.import_state(ck[:100].clone())
    for p in (pa, other, bigger):
        p.close()
