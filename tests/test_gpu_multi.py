"""A heterogeneous batch in shared launches (wf_map_solve_many): when the
problems share the working type and the channel count, each L-BFGS iteration
of the whole batch is one set of seven launches whose blocks cover every
problem's own grid, every problem on the ping-pong stages with radix plan 0
and its own tuned tile widths (variant codes 21cd).  Every map must then end
exactly where its problem ends when solved alone with the same FFT-stage
variant: the same states bit for bit, the same iteration counts; and the
solutions must be the oracle's MAPs."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import wf_oracle as O  # noqa: E402
from paper_1810_00503_gb300 import synth, wf  # noqa: E402
from tests.helpers import ensure_lib, make_problem, rel, rfft_u  # noqa: E402

SHARED_VARIANT = 2111


def shared_kinds(v):
    """Variant code of the shared launches: ping-pong inverse column and row
    stages (a = 2, b = 1), radix plans 0, any tile widths."""
    return v // 10000 == 0 and (v // 100) % 100 == 21


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    ensure_lib()


def _problems(shapes, C, precision, seed):
    out = []
    for i, (ny, nx, B) in enumerate(shapes):
        maker = synth.density_small if C == 1 else synth.shear_eb
        inputs = [maker(ny, seed=seed + 10 * i + b, nx=nx) for b in range(B)]
        out.append(make_problem(inputs, precision, shared_P=(B == 1)))
    return out


@pytest.mark.parametrize("C,precision", [(1, "fp64"), (2, "fp64"), (1, "mixed"), (2, "mixed")])
def test_shared_launches_equal_each_problem_alone(C, precision):
    shapes = [(32, 32, 3), (64, 16, 2), (16, 128, 1), (128, 128, 2)]
    # no periodic refresh: alone, a refresh falls on its exact iteration, in a
    # batch at the next round boundary, so the iterates would differ by rounding
    opts = dict(gtol_rel=1e-9 if precision == "fp64" else 1e-5, max_iter=20000, check_every=8)
    probs = [p for p, _ in _problems(shapes, C, precision, seed=40)]
    together = wf.solve_many(probs, **opts)
    for p, r in zip(probs, together):
        v = r.stats[0]["fft_variant"]
        assert {s["fft_variant"] for s in r.stats} == {v} and shared_kinds(v), r.stats
        alone = p.solve(fft_variant=v, **opts)
        assert torch.equal(r.s, alone.s)
        assert [s["iters"] for s in r.stats] == [s["iters"] for s in alone.stats]
        assert [s["status"] for s in r.stats] == ["WF_OK"] * len(r.stats)
        p.close()


def test_shared_launches_reach_the_oracle_map():
    shapes = [(16, 16, 2), (32, 8, 1), (8, 64, 2)]
    made = _problems(shapes, 1, "fp64", seed=7)
    probs = [p for p, _ in made]
    res = wf.solve_many(probs, gtol_rel=1e-12, max_iter=20000, refresh_every=40, autotune=0)
    for (p, host), r in zip(made, res):
        assert {s["fft_variant"] for s in r.stats} == {SHARED_VARIANT}
        for b in range(p.B):
            zs = O.dense_wf_whitened(host["d"][b], host["W"][b], host["P"][b])
            assert rel(r.s[b].cpu().numpy(), rfft_u(zs)) <= 1e-10
        p.close()


def test_mixed_types_fall_back_to_a_branch_per_problem():
    """Problems of different working types cannot share launches: each then
    runs its own (tuned) kernels, and the batch still solves."""
    (p1, _), = _problems([(32, 32, 2)], 1, "fp64", seed=3)
    (p2, _), = _problems([(64, 64, 1)], 1, "mixed", seed=5)
    res = wf.solve_many([p1, p2], gtol_rel=1e-6, max_iter=20000)
    for r in res:
        assert all(s["status"] == "WF_OK" for s in r.stats), r.stats
    p1.close()
    p2.close()


def test_more_problems_than_shared_slots_and_mixed_channels_fall_back():
    """Nine problems (one more than a shared launch holds), and a pair with
    different channel counts, run a branch per problem: every map still
    solves, each problem on its own tuned variant."""
    shapes = [(16, 16, 1)] * 9
    made = _problems(shapes, 1, "fp64", seed=60)
    res = wf.solve_many([p for p, _ in made], gtol_rel=1e-10, max_iter=20000)
    for (p, host), r in zip(made, res):
        assert all(s["status"] == "WF_OK" for s in r.stats), r.stats
        zs = O.dense_wf_whitened(host["d"][0], host["W"][0], host["P"][0])
        assert rel(r.s[0].cpu().numpy(), rfft_u(zs)) <= 1e-8
        p.close()
    (p1, _), = _problems([(32, 32, 1)], 1, "mixed", seed=70)
    (p2, _), = _problems([(32, 64, 1)], 2, "mixed", seed=71)
    res = wf.solve_many([p1, p2], gtol_rel=1e-6, max_iter=20000)
    for r in res:
        assert all(s["status"] == "WF_OK" for s in r.stats), r.stats
    p1.close()
    p2.close()
