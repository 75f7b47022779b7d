"""The C-ABI library loads on a machine without a GPU and exports every entry
point declared in include/wf.h; host-only calls behave as documented."""
import ctypes
import os
import re

import pytest

from paper_1810_00503_gb300 import wf
from tests.helpers import ensure_lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "wf.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b((?:wf|bandpower)_[a-z_0-9]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    L = ensure_lib()
    names = declared_symbols()
    assert names, "no declarations found"
    for name in names:
        assert hasattr(L, name), f"{name} declared in wf.h but not exported"
    assert sorted(wf.EXPORTS) == names


def test_opts_default_and_last_error_need_no_gpu():
    L = ensure_lib()
    o = wf.WfOpts()
    L.wf_opts_default(ctypes.byref(o))
    assert (o.lbfgs_m, o.max_iter, o.gtol_rel, o.check_every, o.use_graphs) == (10, 10000, 1e-6, 16, 1)
    assert (o.line_search, o.c1, o.c2, o.seed) == (wf.WF_LS_EXACT, 1e-4, 0.9, 0)
    assert (o.spin_limit, o.inject_timeout_map, o.autotune, o.fft_variant) == (0, 0, 1, 0)
    assert ctypes.sizeof(o) == 104  # layout of wf_opts in include/wf.h
    assert isinstance(L.wf_last_error(), bytes)


def test_null_arguments_are_rejected_without_touching_the_device():
    L = ensure_lib()
    assert L.wf_create(None, 0) == 1
    assert b"null" in L.wf_last_error()
    out = ctypes.c_void_p()
    # null handle is rejected before any CUDA call
    assert L.wf_problem_create(None, None, 1, 32, 1, 1, 0, 10, None, ctypes.byref(out)) == 1
    assert L.wf_eval(None, None, None, None, None) == 1


@pytest.mark.parametrize("cname,pyname", [("wf_opts", "WfOpts"), ("wf_map", "WfMap"),
                                           ("wf_solve_stats", "WfSolveStats"),
                                           ("wf_bandpower_in", "WfBandpowerIn"),
                                           ("wf_bandpower_out", "WfBandpowerOut")])
def test_struct_layouts_match_the_header(cname, pyname):
    """Compile a tiny C program against include/wf.h and compare the size and
    field offsets of each struct the binding mirrors with the binding's."""
    import shutil
    import subprocess
    import tempfile
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    cls = getattr(wf, pyname)
    fields = [f[0] for f in cls._fields_]
    src = "#include <stdio.h>\n#include <stddef.h>\n#include \"wf.h\"\nint main(void){\n"
    src += f'printf("%zu\\n", sizeof({cname}));\n'
    for f in fields:
        src += f'printf("%zu\\n", offsetof({cname}, {f}));\n'
    src += "return 0;}\n"
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        exe = os.path.join(d, "t")
        open(c, "w").write(src)
        subprocess.check_call([cc, "-I", os.path.join(root, "include"), "-I", "/usr/local/cuda/include", c, "-o", exe])
        out = [int(x) for x in subprocess.check_output([exe]).split()]
    assert out[0] == ctypes.sizeof(cls)
    assert out[1:] == [getattr(cls, f).offset for f in fields]


def test_band_table_from_edges_matches_brute_force():
    """wf_band_table (host code in the library) against a loop over modes."""
    ensure_lib()
    import numpy as np
    for n, C, kscale in ((16, 1, 1.0), (32, 2, 0.5), (64, 1, 3.0)):
        edges = np.array([1.0, 2.5, 4.0, 7.5, 11.0, 20.0])
        got = wf.band_table(n, edges, C=C, kscale=kscale)
        want = np.full((C, n, n // 2 + 1), -1, dtype=np.int16)
        for j in range(n):
            ky = j if j < n // 2 else j - n
            for kx in range(n // 2 + 1):
                k = kscale * np.hypot(kx, ky)
                for lb in range(len(edges) - 1):
                    if edges[lb] <= k < edges[lb + 1]:
                        want[:, j, kx] = lb
        assert np.array_equal(got, want)
    with pytest.raises(wf.WfError, match="EINVAL"):
        wf.band_table(16, [2.0, 1.0])


def test_rect_band_table_uses_the_physical_wavevector():
    """wf_band_table_rect against a loop over modes with the wavevector of a
    mode of an ny x nx map of square pixels, N (mx / nx, my / ny) in units of
    the longer side's fundamental, N = max(ny, nx)."""
    ensure_lib()
    import numpy as np
    edges = np.array([1.1, 2.55, 4.05, 7.3, 11.2, 20.1])
    for ny, nx, C, kscale in ((16, 64, 2, 1.0), (32, 8, 1, 0.5), (8, 8, 1, 1.0), (6, 10, 1, 1.0), (12, 8, 2, 0.7)):
        got = wf.band_table(ny, edges, C=C, kscale=kscale, nx=nx)
        N = max(ny, nx)
        want = np.full((C, ny, nx // 2 + 1), -1, dtype=np.int16)
        for j in range(ny):
            my = j if j < ny // 2 else j - ny
            for kx in range(nx // 2 + 1):
                k = kscale * N * np.hypot(kx / nx, my / ny)
                for lb in range(len(edges) - 1):
                    if edges[lb] <= k < edges[lb + 1]:
                        want[:, j, kx] = lb
        assert np.array_equal(got, want), (ny, nx)
    with pytest.raises(wf.WfError, match="EINVAL"):
        wf.band_table(16, [1.0, 2.0], nx=7)


def test_binding_refuses_host_tensors_before_any_call():
    """The binding hands raw data pointers to the library, which reads them as
    device memory: host tensors are refused before a handle or a call is made
    (no GPU is needed to see it)."""
    torch = pytest.importorskip("torch")
    n, f64 = 16, torch.float64
    d = torch.zeros(1, 1, n, n, dtype=f64)
    mask = torch.ones(n, n, dtype=torch.uint8)
    P = torch.ones(1, n, n // 2 + 1, dtype=f64)
    with pytest.raises(TypeError, match="CUDA"):
        wf.Problem(d, mask, d + 1.0, P)
    band = torch.zeros(1, n, n // 2 + 1, dtype=torch.int16)
    with pytest.raises(TypeError, match="CUDA"):
        wf.bandpower_estimate(d[0], mask, d[0] + 1.0, P, band, 2, None, None, None, n_sim=2, n_fd=1)


def _stand_ins():
    """A non-null handle and non-null pointers for argument checks that return
    before the library reads the handle, reads a buffer or calls CUDA: the
    host buffer behind them is never touched on these paths."""
    buf = ctypes.create_string_buffer(1 << 16)
    return buf, ctypes.c_void_p(ctypes.addressof(buf)), ctypes.addressof(buf)


def test_problem_create_refuses_bad_arguments_before_device_work():
    L = ensure_lib()
    buf, h, addr = _stand_ins()
    maps = (wf.WfMap * 2)()
    for m in maps:
        m.d = m.mask = m.Ninv = m.P = addr
    out = ctypes.c_void_p(1)
    good = dict(count=1, n=16, C=1, dtype=wf.WF_F32, prec=wf.WF_MIXED, m=10)
    for bad in (dict(count=0), dict(n=12), dict(n=4), dict(n=2048), dict(C=3), dict(C=0), dict(dtype=2),
                dict(prec=2), dict(m=0), dict(m=33)):
        a = {**good, **bad}
        st = L.wf_problem_create(h, maps, a["count"], a["n"], a["C"], a["dtype"], a["prec"], a["m"], None,
                                 ctypes.byref(out))
        assert st == 1 and out.value is None, (bad, st)
    for ny, nx in ((16, 12), (12, 16), (4, 16), (16, 4), (16, 2048), (2048, 16), (0, 16)):
        st = L.wf_problem_create_rect(h, maps, 1, ny, nx, 1, wf.WF_F32, wf.WF_MIXED, 10, None, ctypes.byref(out))
        assert st == 1 and out.value is None and b"power of two" in L.wf_last_error(), (ny, nx)
    maps[1].Ninv = None
    assert L.wf_problem_create(h, maps, 2, 16, 1, wf.WF_F32, wf.WF_MIXED, 10, None, ctypes.byref(out)) == 1
    assert b"map 1" in L.wf_last_error()
    assert L.wf_problem_create_rect(h, maps, 2, 16, 64, 1, wf.WF_F32, wf.WF_MIXED, 10, None,
                                    ctypes.byref(out)) == 1
    assert b"map 1" in L.wf_last_error()


def test_bandpower_refuses_bad_arguments_before_device_work():
    """The band-power calls' argument rules, the leakage-bias ones included,
    checked through the C ABI on the host."""
    import numpy as np
    L = ensure_lib()
    buf, h, addr = _stand_ins()
    data = wf.WfMap(d=addr, mask=addr, Ninv=addr, P=addr)
    outs = {k: np.zeros(64 * 64 * 4) for k in ("theta_fid", "E", "bias", "fisher", "cov", "theta_hat", "cov_E")}
    bo = wf.WfBandpowerOut(**{k: v.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) for k, v in outs.items()})
    o = wf.WfOpts()
    L.wf_opts_default(ctypes.byref(o))
    fdb = (ctypes.c_int * 2)(0, 2)

    def estimate(C=2, **kw):
        f = dict(n_bands=4, n_sim=2, n_fd=1, leak_split=0, band=addr, z=None, noise=None, u=None,
                 sim_index=None, fd_bands=None, n_fd_bands=0, trunc_bands=0, trunc_width=0, out_on_device=0)
        f.update(kw)
        bi = wf.WfBandpowerIn(**f)
        return L.bandpower_estimate(h, ctypes.byref(data), 16, C, wf.WF_F32, wf.WF_MIXED, ctypes.byref(bi),
                                    ctypes.byref(o), ctypes.byref(bo), None)

    for C, kw, msg in [(2, dict(n_bands=0), b"n_bands"), (2, dict(n_bands=65), b"n_bands"),
                       (2, dict(n_sim=0), b"n_sim"), (2, dict(n_fd=3), b"n_fd"), (2, dict(band=None), b"band"),
                       (2, dict(z=addr), b"random fields"), (2, dict(trunc_bands=5), b"trunc"),
                       (2, dict(leak_split=4), b"leak_split"), (2, dict(leak_split=-1), b"leak_split"),
                       (1, dict(leak_split=2), b"leak_split"), (2, dict(leak_split=1, trunc_bands=2), b"trunc_bands"),
                       (2, dict(leak_split=2, fd_bands=ctypes.addressof(fdb), n_fd_bands=2), b"fd_bands"),
                       (2, dict(out_on_device=2), b"out_on_device")]:
        assert estimate(C, **kw) == 1, (C, kw)
        assert msg in L.wf_last_error(), (kw, L.wf_last_error())
    sims = (ctypes.c_longlong * 2)(0, 1)
    for n, C in ((0, 1), (12, 1), (2048, 1), (16, 0), (16, 3)):  # checked before any size arithmetic
        bi = wf.WfBandpowerIn(n_bands=4, n_sim=2, n_fd=1, band=addr, sim_index=ctypes.addressof(sims))
        st = L.bandpower_estimate(h, ctypes.byref(data), n, C, wf.WF_F32, wf.WF_MIXED, ctypes.byref(bi),
                                  ctypes.byref(o), ctypes.byref(bo), None)
        assert st == 1 and b"power of two" in L.wf_last_error(), (n, C, L.wf_last_error())
    bi = wf.WfBandpowerIn(n_bands=4, n_sim=2, n_fd=1, band=addr)
    for n_iter, qmin, qmax, msg in [(0, 0.1, 10.0, b"n_iter"), (2, 1.5, 10.0, b"q_min"), (2, 0.1, 0.5, b"q_min")]:
        st = L.bandpower_iterate(h, ctypes.byref(data), 16, 1, wf.WF_F32, wf.WF_MIXED, ctypes.byref(bi),
                                 ctypes.byref(o), n_iter, qmin, qmax, None, None, ctypes.byref(bo), None)
        assert st == 1 and msg in L.wf_last_error(), (n_iter, qmin, qmax, L.wf_last_error())
    st = L.bandpower_iterate(h, ctypes.byref(data), 0, 1, wf.WF_F32, wf.WF_MIXED, ctypes.byref(bi),
                             ctypes.byref(o), 2, 0.1, 10.0, None, None, ctypes.byref(bo), None)
    assert st == 1 and b"power of two" in L.wf_last_error(), L.wf_last_error()


def test_normal_draw_refuses_bad_arguments_on_the_host():
    L = ensure_lib()
    buf, h, addr = _stand_ins()
    assert L.wf_normal_draw(1, 0, 0, 10, wf.WF_F32, None, None) == 1
    assert b"null output" in L.wf_last_error()
    assert L.wf_normal_draw(1, 0, 0, 10, 7, addr, None) == 1
    assert b"dtype" in L.wf_last_error()
    assert L.wf_normal_draw(1, 0, 2 ** 64 - 5, 10, wf.WF_F32, addr, None) == 1
    assert b"overflows" in L.wf_last_error()


def test_eval_noalloc_refuses_bad_arguments_on_the_host():
    L = ensure_lib()
    buf, h, addr = _stand_ins()
    chi2 = (ctypes.c_double * 4)()
    other = ctypes.create_string_buffer(64)
    g = ctypes.addressof(other)
    ok = dict(s=addr, d=addr, w=addr, P=addr, n=16, C=1, count=1, prec=wf.WF_MIXED, grad=g)
    for bad, msg in [(dict(s=None), b"null"), (dict(grad=addr), b"alias"), (dict(n=12), b"power of two"),
                     (dict(n=2048), b"power of two"), (dict(C=3), b"C ="), (dict(count=0), b"count"),
                     (dict(prec=5), b"precision")]:
        a = {**ok, **bad}
        st = L.wf_eval_noalloc(a["s"], a["d"], a["w"], a["P"], a["n"], a["C"], a["count"], a["prec"], chi2,
                               a["grad"], None)
        assert st == 1 and msg in L.wf_last_error(), (bad, L.wf_last_error())


def test_eval_noalloc_binding_checks_every_tensor_before_the_library(monkeypatch):
    """The binding hands seven raw pointers to wf_eval_noalloc; a tensor of the
    wrong shape, dtype, layout or device would be read or written out of
    bounds.  Each such mismatch raises before the library is reached (the
    library loader is replaced by one that fails the test)."""
    torch = pytest.importorskip("torch")

    def no_lib():
        raise AssertionError("the library was called")

    monkeypatch.setattr(wf, "lib", no_lib)
    cpu = torch.device("cpu")
    B, C, n = 2, 1, 16
    f32, c64 = torch.float32, torch.complex64
    good = dict(s=torch.zeros(B, C, n, n // 2 + 1, dtype=c64), d=torch.zeros(B, C, n, n, dtype=f32),
                w=torch.zeros(B, C, n, n, dtype=f32), P=torch.zeros(C, n, n // 2 + 1, dtype=f32),
                chi2=torch.zeros(B, dtype=torch.float64), grad=torch.zeros(B, C, n, n // 2 + 1, dtype=c64))
    assert wf._noalloc_check(**good, device=cpu) == (B, C, n)
    bad = [("s", torch.zeros(B, C, n, n // 2 + 1, dtype=torch.complex128), TypeError),
           ("s", torch.zeros(B, C, n, n // 2, dtype=c64), ValueError),
           ("grad", torch.zeros(B + 1, C, n, n // 2 + 1, dtype=c64), ValueError),
           ("w", torch.zeros(B, C, n, n, dtype=torch.float64), TypeError),
           ("w", torch.zeros(B, C, n, 2 * n, dtype=f32)[..., ::2], ValueError),
           ("P", torch.zeros(2, n, n // 2 + 1, dtype=f32), ValueError),
           ("P", torch.zeros(C, n, n // 2 + 1, dtype=torch.float64), TypeError),
           ("chi2", torch.zeros(B, dtype=f32), TypeError),
           ("chi2", torch.zeros(B + 1, dtype=torch.float64), ValueError),
           ("d", torch.zeros(B, C, n, n // 2, dtype=f32), ValueError),
           ("s", torch.zeros(B, C, n, n // 2 + 1, dtype=c64, device="meta"), ValueError)]
    for name, t, exc in bad:
        with pytest.raises(exc):
            wf._noalloc_check(**{**good, name: t}, device=cpu)
    with pytest.raises(TypeError, match="CUDA"):  # host tensors never reach the library
        wf.eval_noalloc(good["s"], good["d"], good["w"], good["P"])


def test_eval_any_refuses_bad_arguments_on_the_host():
    """wf_eval_any checks its sizes, pointers and precision before it reads the
    handle, allocates or calls CUDA (stand-in pointers are never touched)."""
    L = ensure_lib()
    buf, h, addr = _stand_ins()
    other = ctypes.create_string_buffer(64)
    g = ctypes.addressof(other)
    ok = dict(h=h, B=1, C=1, ny=12, nx=20, prec=wf.WF_MIXED, d=addr, mask=addr, Ninv=addr, P=addr, s=addr, grad=g,
              chi2=addr)
    for bad, msg in [(dict(h=None), b"null"), (dict(mask=None), b"null"), (dict(chi2=None), b"null"),
                     (dict(grad=addr), b"alias"), (dict(B=0), b"count"), (dict(C=3), b"C ="),
                     (dict(prec=7), b"precision"), (dict(ny=11), b"prime factor"), (dict(nx=26), b"prime factor"),
                     (dict(ny=1), b"prime factor"), (dict(nx=1050), b"prime factor"),
                     (dict(ny=2048), b"prime factor")]:
        a = {**ok, **bad}
        st = L.wf_eval_any(a["h"], a["B"], a["C"], a["ny"], a["nx"], a["prec"], a["d"], a["mask"], a["Ninv"], a["P"],
                           a["s"], a["grad"], a["chi2"], None)
        assert st == 1 and msg in L.wf_last_error(), (bad, L.wf_last_error())


def test_eval_any_binding_checks_every_tensor_before_the_library(monkeypatch):
    """The binding hands eight raw pointers to wf_eval_any; each mismatch of
    shape, dtype, layout or device raises before the library is reached."""
    torch = pytest.importorskip("torch")

    def no_lib():
        raise AssertionError("the library was called")

    monkeypatch.setattr(wf, "lib", no_lib)
    cpu = torch.device("cpu")
    B, C, ny, nx = 2, 2, 12, 30
    h1 = nx // 2 + 1
    f32, c64 = torch.float32, torch.complex64
    good = dict(s=torch.zeros(B, C, ny, h1, dtype=c64), mask=torch.zeros(B, ny, nx, dtype=torch.uint8),
                Ninv=torch.zeros(B, C, ny, nx, dtype=f32), P=torch.zeros(C, ny, h1, dtype=f32),
                d=torch.zeros(B, C, ny, nx, dtype=f32), chi2=torch.zeros(B, dtype=torch.float64),
                grad=torch.zeros(B, C, ny, h1, dtype=c64))
    assert wf._any_check(**good, device=cpu) == (B, C, ny, nx)
    assert wf._any_check(**{**good, "d": None}, device=cpu) == (B, C, ny, nx)
    bad = [("s", torch.zeros(B, C, ny, h1, dtype=torch.complex128), TypeError),
           ("s", torch.zeros(B, C, ny, h1 - 1, dtype=c64), ValueError),
           ("grad", torch.zeros(B + 1, C, ny, h1, dtype=c64), ValueError),
           ("mask", torch.zeros(B, ny, nx, dtype=torch.bool), TypeError),
           ("mask", torch.zeros(B, C, ny, nx, dtype=torch.uint8), ValueError),
           ("d", torch.zeros(B, C, ny, nx, dtype=torch.float64), TypeError),
           ("d", torch.zeros(B, C, ny, 2 * nx, dtype=f32)[..., ::2], ValueError),
           ("P", torch.zeros(1, ny, h1, dtype=f32), ValueError),
           ("chi2", torch.zeros(B, dtype=f32), TypeError),
           ("s", torch.zeros(B, C, ny, h1, dtype=c64, device="meta"), ValueError)]
    for name, t, exc in bad:
        with pytest.raises(exc):
            wf._any_check(**{**good, name: t}, device=cpu)
    with pytest.raises(TypeError):
        wf.eval_any(good["s"], good["mask"], good["Ninv"], good["P"])  # host tensors: refused before any call
