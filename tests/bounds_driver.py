"""Driver of the bounds-checked run (tests/test_gpu_debug_bounds.py runs it
in a child process with WF_LIB_PATH pointing at the bounds-checked library):
tiny square maps of every size and rectangular ones of both aspects up to the
extreme strips (8 x 1024, 1024 x 8), every channel count and precision,
through every entry point that launches the FFT stages, and short solves
under a covering set of FFT-stage variants; the mixed-radix objective on
sides that are not powers of two; prints one JSON line with the violation
count."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402
import torch  # noqa: E402

from oracle import wf_oracle as O  # noqa: E402
from paper_1810_00503_gb300 import synth, wf  # noqa: E402
from tests.helpers import make_problem, rel, rfft_u, to_dev  # noqa: E402


def main():
    out = {"lib": wf.LIB_PATH}
    selftest, first = wf.debug_bounds(mode=2)
    out["selftest"] = selftest
    out["selftest_first"] = first
    wf.debug_bounds(mode=1)  # clear
    worst = 0.0
    variants = [100000 * pl + 10000 * pl + 1000 * a + 100 * b + 11 * dv
                for a in (1, 2, 3) for b in (1, 2) for dv in (1, 4) for pl in (0, 1, 2)]
    runs = 0
    shapes = [(n, n) for n in (8, 16, 32, 64, 128)] + [(8, 64), (64, 8), (16, 256), (256, 32), (8, 1024),
                                                       (1024, 8)]
    for n, nx in shapes:
        for C in (1, 2):
            inp = synth.density_small(n, seed=n + C, nx=nx) if C == 1 else synth.shear_eb(n, seed=n + C, nx=nx)
            for prec in ("fp64", "mixed"):
                prob, host = make_problem([inp, inp], prec)
                cdt = torch.complex128 if prec == "fp64" else torch.complex64
                z = synth.random_state(n, C, seed=7, nx=nx)
                s = to_dev(np.stack([rfft_u(z)] * 2), cdt)
                chi2, g = prob.eval(s)
                ref = rfft_u(O.grad(z, host["d"][0], host["W"][0], host["P"][0]))
                worst = max(worst, rel(g[0].cpu().numpy(), ref))
                prob.hess_vec(s)
                prob.signal_map(s)
                band = to_dev(np.ascontiguousarray(synth.log_bands(n, 3, C=C, nx=nx)[..., : nx // 2 + 1]),
                              torch.int16)
                prob.eval_bands(s, band, 3 * C)
                prob.band_energy(s, band, torch.ones(3 * C, dtype=torch.float64, device="cuda"))
                wdt = torch.float64 if prec == "fp64" else torch.float32
                zz = to_dev(np.stack([z, z]), wdt)
                prob.simulate(zz, zz)
                if nx == n:  # the allocation-free call takes square maps
                    wf.eval_noalloc(s, to_dev(np.stack(host["d"]), wdt), to_dev(np.stack(host["W"]), wdt),
                                    to_dev(host["P"][0][..., : n // 2 + 1], wdt))
                for v in variants:
                    try:
                        prob.solve(gtol_rel=0.0, max_iter=6, fft_variant=v, check_every=2, refresh_every=3)
                    except wf.WfError as e:
                        out.setdefault("solve_errors", []).append([n, nx, C, prec, v, str(e)[:80]])
                    runs += 1
                prob.solve_refined(cert_tol=1e-3, max_rounds=2, gtol_rel=1e-3, max_iter=50)
                prob.start(gtol_rel=0.0, max_iter=20, check_every=4)
                prob.step(5)
                ck = prob.export_state()
                prob.import_state(ck)
                prob.step(5)
                prob.finish()
                prob.close()
    # heterogeneous batches in shared launches (square and rectangular shapes)
    for C in (1, 2):
        for prec in ("fp64", "mixed"):
            made = []
            for i, (n, nx) in enumerate([(8, 8), (16, 64), (64, 16), (32, 32)]):
                inp = synth.density_small(n, seed=i, nx=nx) if C == 1 else synth.shear_eb(n, seed=i, nx=nx)
                made.append(make_problem([inp, inp], prec)[0])
            try:
                wf.solve_many(made, gtol_rel=0.0, max_iter=12, check_every=4, refresh_every=5)
            except wf.WfError as e:
                out.setdefault("solve_errors", []).append(["many", C, prec, str(e)[:80]])
            runs += 1
            for p in made:
                p.close()
    # the mixed-radix objective on sides that are not powers of two (odd and
    # even sides, every radix, strips, the 1024 limit)
    from tests.helpers import any_inputs
    for ny, nx in [(2, 2), (3, 5), (7, 12), (30, 42), (96, 60), (343, 20), (1024, 6), (6, 1000)]:
        for C in (1, 2):
            for prec in ("fp64", "mixed"):
                I = any_inputs(ny, nx, C, 2, seed=ny + nx)
                wdt = torch.float64 if prec == "fp64" else torch.float32
                cdt = torch.complex128 if prec == "fp64" else torch.complex64
                s = to_dev(np.stack([rfft_u(f) for f in I["f"]]), cdt)
                args = (to_dev(np.stack(I["mask"]), torch.uint8), to_dev(np.stack(I["Ninv"]), wdt),
                        to_dev(np.ascontiguousarray(I["P"][..., : nx // 2 + 1]), wdt))
                wf.eval_any(s, *args, d=to_dev(np.stack(I["d"]), wdt))
                wf.eval_any(s, *args)
                runs += 1
    torch.cuda.synchronize()
    count, first = wf.debug_bounds(mode=0)
    out.update(violations=count, first=first, solves=runs, worst_grad_rel=worst)
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
