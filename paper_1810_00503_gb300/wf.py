"""Thin Python binding of the C ABI in include/wf.h (ctypes; argument
marshalling only).  Device memory and streams come from PyTorch; every
computation runs in libwf.so.  Importing works without a GPU; the first call
that needs the library raises if libwf.so has not been built."""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
# WF_LIB_PATH selects another build of the library, e.g. the bounds-checked one.
LIB_PATH = os.environ.get("WF_LIB_PATH") or os.path.join(HERE, "libwf.so")

WF_FP64, WF_MIXED = 0, 1
WF_F32, WF_F64 = 0, 1
WF_LS_EXACT, WF_LS_WOLFE = 0, 1
STATUS = {0: "WF_OK", 1: "WF_EINVAL", 2: "WF_ENONFINITE", 3: "WF_ENOMEM", 4: "WF_ECUDA",
          5: "WF_ENOTCONVERGED", 6: "WF_ELINESEARCH", 7: "WF_ETIMEOUT"}

# Names declared in include/wf.h (checked against the header by the tests).
EXPORTS = ["wf_create", "wf_destroy", "wf_last_error", "wf_opts_default", "wf_problem_create",
           "wf_problem_destroy", "wf_problem_set_data", "wf_eval", "wf_hess_vec",
           "wf_signal_map", "wf_map_solve", "wf_simulate_data", "wf_band_energy",
           "wf_solver_start", "wf_solver_step", "wf_solver_finish", "wf_solver_profile",
           "wf_eval_noalloc", "bandpower_estimate", "wf_problem_set_band_scale", "wf_eval_bands",
           "wf_map_solve_many", "wf_normal_draw", "wf_workspace_used", "wf_band_table",
           "bandpower_iterate", "wf_problem_variant", "wf_alu_peak", "wf_solver_history",
           "wf_map_solve_refined", "bandpower_sums_len", "bandpower_sums", "bandpower_combine",
           "wf_solver_state_size", "wf_solver_export", "wf_solver_import", "wf_debug_bounds",
           "wf_problem_create_rect", "bandpower_estimate_rect", "bandpower_iterate_rect", "wf_band_table_rect",
           "wf_eval_any"]


class WfMap(ctypes.Structure):
    _fields_ = [("d", ctypes.c_void_p), ("mask", ctypes.c_void_p),
                ("Ninv", ctypes.c_void_p), ("P", ctypes.c_void_p)]


class WfOpts(ctypes.Structure):
    _fields_ = [("lbfgs_m", ctypes.c_int), ("max_iter", ctypes.c_int),
                ("gtol_rel", ctypes.c_double), ("dchi2_abs", ctypes.c_double),
                ("refresh_every", ctypes.c_int), ("check_every", ctypes.c_int),
                ("use_graphs", ctypes.c_int), ("stream", ctypes.c_void_p),
                ("line_search", ctypes.c_int), ("pad_", ctypes.c_int), ("c1", ctypes.c_double),
                ("c2", ctypes.c_double), ("seed", ctypes.c_ulonglong), ("spin_limit", ctypes.c_longlong),
                ("inject_timeout_map", ctypes.c_int), ("autotune", ctypes.c_int), ("fft_variant", ctypes.c_int),
                ("history", ctypes.c_int)]


class WfSolveStats(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("evals", ctypes.c_int), ("status", ctypes.c_int),
                ("fft_variant", ctypes.c_int), ("chi2", ctypes.c_double), ("gnorm_rel", ctypes.c_double)]


class WfBandpowerIn(ctypes.Structure):
    _fields_ = [("n_bands", ctypes.c_int), ("n_sim", ctypes.c_int), ("n_fd", ctypes.c_int),
                ("leak_split", ctypes.c_int), ("band", ctypes.c_void_p), ("z", ctypes.c_void_p),
                ("noise", ctypes.c_void_p), ("u", ctypes.c_void_p), ("sim_index", ctypes.c_void_p),
                ("fd_bands", ctypes.c_void_p), ("n_fd_bands", ctypes.c_int), ("trunc_bands", ctypes.c_int),
                ("trunc_width", ctypes.c_int), ("out_on_device", ctypes.c_int)]


class WfBandpowerOut(ctypes.Structure):
    _fields_ = [(k, ctypes.POINTER(ctypes.c_double)) for k in
                ("theta_fid", "E", "bias", "fisher", "cov", "theta_hat", "cov_E", "E_maps")]


class WfError(RuntimeError):
    """A failing call.  `result` holds the per-map outcome when the call still
    produced one (a solve in which some maps stopped with an error)."""

    def __init__(self, status, msg, result=None):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status
        self.result = result


_lib = None


def lib() -> ctypes.CDLL:
    """Load libwf.so; raises if it has not been built (no fallback exists)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"CUDA library missing: {LIB_PATH} (run paper_1810_00503_gb300.build.build())")
    L = ctypes.CDLL(LIB_PATH)
    vp, i, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    L.wf_last_error.restype = ctypes.c_char_p
    L.wf_create.argtypes = [ctypes.POINTER(vp), ctypes.c_size_t]
    L.wf_workspace_used.argtypes = [vp, ctypes.POINTER(ctypes.c_size_t)]
    L.wf_problem_variant.argtypes = [vp, ctypes.POINTER(i)]
    L.wf_alu_peak.argtypes = [i, ctypes.POINTER(d)]
    L.wf_solver_history.argtypes = [vp, ctypes.POINTER(d), ctypes.POINTER(i)]
    L.wf_band_table.argtypes = [i, i, ctypes.POINTER(d), i, d, vp]
    L.wf_band_table_rect.argtypes = [i, i, i, ctypes.POINTER(d), i, d, vp]
    L.wf_destroy.argtypes = [vp]
    L.wf_opts_default.argtypes = [ctypes.POINTER(WfOpts)]
    L.wf_opts_default.restype = None
    L.wf_problem_create.argtypes = [vp, ctypes.POINTER(WfMap), i, i, i, i, i, i, vp, ctypes.POINTER(vp)]
    L.wf_problem_create_rect.argtypes = [vp, ctypes.POINTER(WfMap), i, i, i, i, i, i, i, vp, ctypes.POINTER(vp)]
    L.wf_problem_destroy.argtypes = [vp]
    L.wf_problem_set_data.argtypes = [vp, vp, vp]
    L.wf_eval.argtypes = [vp, vp, vp, vp, vp]
    L.wf_hess_vec.argtypes = [vp, vp, vp, vp]
    L.wf_signal_map.argtypes = [vp, vp, vp, vp]
    L.wf_map_solve.argtypes = [vp, ctypes.POINTER(WfOpts), vp, vp, vp, ctypes.POINTER(WfSolveStats)]
    L.wf_map_solve_refined.argtypes = [vp, ctypes.POINTER(WfOpts), d, i, vp, vp, ctypes.POINTER(d),
                                       ctypes.POINTER(WfSolveStats)]
    L.wf_simulate_data.argtypes = [vp, vp, vp, vp, vp]
    L.wf_band_energy.argtypes = [vp, vp, vp, vp, i, vp, vp]
    L.wf_solver_start.argtypes = [vp, ctypes.POINTER(WfOpts), vp]
    L.wf_solver_step.argtypes = [vp, i, ctypes.POINTER(i)]
    L.wf_solver_finish.argtypes = [vp, vp, vp, ctypes.POINTER(WfSolveStats)]
    L.wf_solver_profile.argtypes = [vp, i, ctypes.POINTER(ctypes.c_float)]
    L.wf_eval_noalloc.argtypes = [vp, vp, vp, vp, i, i, i, i, vp, vp, vp]
    L.wf_eval_any.argtypes = [vp, i, i, i, i, i, vp, vp, vp, vp, vp, vp, vp, vp]
    L.wf_problem_set_band_scale.argtypes = [vp, vp, vp, i, vp]
    L.wf_eval_bands.argtypes = [vp, vp, vp, vp, vp, i, vp, vp]
    L.wf_map_solve_many.argtypes = [ctypes.POINTER(vp), i, ctypes.POINTER(WfOpts), ctypes.POINTER(vp),
                                    ctypes.POINTER(ctypes.POINTER(WfSolveStats))]
    L.bandpower_estimate.argtypes = [vp, ctypes.POINTER(WfMap), i, i, i, i, ctypes.POINTER(WfBandpowerIn),
                                     ctypes.POINTER(WfOpts), ctypes.POINTER(WfBandpowerOut),
                                     ctypes.POINTER(WfSolveStats)]
    L.bandpower_estimate_rect.argtypes = [vp, ctypes.POINTER(WfMap), i, i, i, i, i, ctypes.POINTER(WfBandpowerIn),
                                          ctypes.POINTER(WfOpts), ctypes.POINTER(WfBandpowerOut),
                                          ctypes.POINTER(WfSolveStats)]
    L.wf_normal_draw.argtypes = [ctypes.c_ulonglong, ctypes.c_uint, ctypes.c_ulonglong, ctypes.c_size_t, i, vp, vp]
    L.bandpower_iterate.argtypes = [vp, ctypes.POINTER(WfMap), i, i, i, i, ctypes.POINTER(WfBandpowerIn),
                                    ctypes.POINTER(WfOpts), i, d, d, vp, ctypes.POINTER(d),
                                    ctypes.POINTER(WfBandpowerOut), ctypes.POINTER(WfSolveStats)]
    L.bandpower_iterate_rect.argtypes = [vp, ctypes.POINTER(WfMap), i, i, i, i, i, ctypes.POINTER(WfBandpowerIn),
                                         ctypes.POINTER(WfOpts), i, d, d, vp, ctypes.POINTER(d),
                                         ctypes.POINTER(WfBandpowerOut), ctypes.POINTER(WfSolveStats)]
    L.bandpower_sums.argtypes = [ctypes.POINTER(d), i, i, i, i, ctypes.POINTER(d)]
    L.bandpower_combine.argtypes = [ctypes.POINTER(d), ctypes.POINTER(d), ctypes.POINTER(d),
                                    ctypes.POINTER(WfBandpowerIn), ctypes.POINTER(WfBandpowerOut)]
    L.bandpower_sums_len.argtypes = [i, i]
    L.wf_debug_bounds.argtypes = [ctypes.POINTER(ctypes.c_ulonglong), ctypes.POINTER(ctypes.c_longlong), i]
    L.wf_solver_state_size.argtypes = [vp, ctypes.POINTER(ctypes.c_size_t)]
    L.wf_solver_export.argtypes = [vp, vp, ctypes.c_size_t]
    L.wf_solver_import.argtypes = [vp, vp, ctypes.c_size_t, vp]
    for name in EXPORTS:
        if name not in ("wf_last_error", "wf_opts_default", "bandpower_sums_len"):
            getattr(L, name).restype = ctypes.c_int
    L.bandpower_sums_len.restype = ctypes.c_size_t
    _lib = L
    return L


def _check(status: int):
    if status != 0:
        raise WfError(status, lib().wf_last_error().decode())


def _ptr(t) -> int:
    return 0 if t is None else int(t.data_ptr())


def _need(t, name, shape=None, dtype=None):
    """Check a tensor before its data pointer goes to the library, which reads
    exactly the documented number of elements of the documented type from
    device memory: a contiguous CUDA tensor of that shape and dtype."""
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} has shape {tuple(t.shape)}, the call needs {tuple(shape)}")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"{name} has dtype {t.dtype}, the call needs {dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return t


def _stream(stream) -> int:
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return int(s.cuda_stream)


class Handle:
    """wf_create / wf_destroy.  workspace_limit: most device bytes the handle's
    problems and solvers may hold (0 = no limit)."""

    def __init__(self, workspace_limit=0):
        h = ctypes.c_void_p()
        _check(lib().wf_create(ctypes.byref(h), int(workspace_limit)))
        self._h = h

    def workspace_used(self):
        v = ctypes.c_size_t()
        _check(lib().wf_workspace_used(self._h, ctypes.byref(v)))
        return int(v.value)

    @property
    def ptr(self):
        return self._h

    def close(self):
        if self._h:
            lib().wf_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


_default_handle = None


def default_handle() -> Handle:
    global _default_handle
    if _default_handle is None:
        _default_handle = Handle()
    return _default_handle


@dataclass
class SolveResult:
    s: object
    x: object
    stats: list


def _noalloc_check(s, d, w, P, chi2, grad, device):
    """Argument rules of eval_noalloc, checked before any pointer reaches the
    library: d (B, C, n, n) float32 or float64 sets the shape and the working
    type; w like d; s and grad (B, C, n, n/2+1) of the matching complex type;
    P (C, n, n/2+1) like d; chi2 float64 (B,); all contiguous and on `device`."""
    import torch
    if not isinstance(d, torch.Tensor) or d.dim() != 4 or d.dtype not in (torch.float32, torch.float64):
        raise ValueError("d must be a float32 or float64 tensor of shape (B, C, n, n)")
    B, C, n, n2 = d.shape
    if n2 != n:
        raise ValueError(f"d has shape {tuple(d.shape)}: maps must be n x n")
    cdt = torch.complex128 if d.dtype == torch.float64 else torch.complex64
    spec = (B, C, n, n // 2 + 1)
    for t, name, shape, dtype in ((d, "d", (B, C, n, n), d.dtype), (w, "w", (B, C, n, n), d.dtype),
                                  (s, "s", spec, cdt), (grad, "grad", spec, cdt),
                                  (P, "P", (C, n, n // 2 + 1), d.dtype), (chi2, "chi2", (B,), torch.float64)):
        if not isinstance(t, torch.Tensor):
            raise TypeError(f"{name} must be a tensor")
        if t.device != device:
            raise ValueError(f"{name} is on {t.device}, the call runs on {device}")
        if tuple(t.shape) != tuple(shape):
            raise ValueError(f"{name} has shape {tuple(t.shape)}, the call needs {tuple(shape)}")
        if t.dtype != dtype:
            raise TypeError(f"{name} has dtype {t.dtype}, the call needs {dtype}")
        if not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
    return B, C, n


def eval_noalloc(s, d, w, P, chi2=None, grad=None, stream=None):
    """wf_eval_noalloc: objective + gradient without any device allocation in
    the library (scratch in a static device array).  s (B, C, n, n/2+1)
    complex, d and w (B, C, n, n), P (C, n, n/2+1), all CUDA tensors of the
    working type on the current device; chi2 and grad are written (allocated
    here by torch if not given, which is the caller's allocation, not the
    library's).  Every tensor is checked (device, shape, dtype, contiguity)
    before the library is called."""
    import torch
    if not isinstance(d, torch.Tensor) or not d.is_cuda:
        raise TypeError("d must be a CUDA tensor")
    dev = torch.device("cuda", torch.cuda.current_device())
    grad = torch.empty_like(s) if grad is None else grad
    chi2 = torch.empty(d.shape[0], dtype=torch.float64, device=d.device) if chi2 is None else chi2
    B, C, n = _noalloc_check(s, d, w, P, chi2, grad, dev)
    if s.data_ptr() == grad.data_ptr():
        raise ValueError("s and grad must not alias")
    precision = WF_FP64 if d.dtype == torch.float64 else WF_MIXED
    _check(lib().wf_eval_noalloc(_ptr(s), _ptr(d), _ptr(w), _ptr(P), n, C, B, precision, _ptr(chi2),
                                 _ptr(grad), _stream(stream)))
    return chi2, grad


def _any_check(s, mask, Ninv, P, d, chi2, grad, device):
    """Argument rules of eval_any, checked before any pointer reaches the
    library: Ninv (B, C, ny, nx) float32 or float64 sets the shape and the
    working type; d like Ninv or None; mask uint8 (B, ny, nx); s and grad
    (B, C, ny, nx/2+1) of the matching complex type; P (C, ny, nx/2+1) like
    Ninv; chi2 float64 (B,); all contiguous and on `device`."""
    import torch
    if not isinstance(Ninv, torch.Tensor) or Ninv.dim() != 4 or Ninv.dtype not in (torch.float32, torch.float64):
        raise ValueError("Ninv must be a float32 or float64 tensor of shape (B, C, ny, nx)")
    B, C, ny, nx = Ninv.shape
    cdt = torch.complex128 if Ninv.dtype == torch.float64 else torch.complex64
    spec = (B, C, ny, nx // 2 + 1)
    checks = [(Ninv, "Ninv", (B, C, ny, nx), Ninv.dtype), (mask, "mask", (B, ny, nx), torch.uint8),
              (s, "s", spec, cdt), (grad, "grad", spec, cdt), (P, "P", (C, ny, nx // 2 + 1), Ninv.dtype),
              (chi2, "chi2", (B,), torch.float64)]
    if d is not None:
        checks.append((d, "d", (B, C, ny, nx), Ninv.dtype))
    for t, name, shape, dtype in checks:
        if not isinstance(t, torch.Tensor):
            raise TypeError(f"{name} must be a tensor")
        if t.device != device:
            raise ValueError(f"{name} is on {t.device}, the call runs on {device}")
        if tuple(t.shape) != tuple(shape):
            raise ValueError(f"{name} has shape {tuple(t.shape)}, the call needs {tuple(shape)}")
        if t.dtype != dtype:
            raise TypeError(f"{name} has dtype {t.dtype}, the call needs {dtype}")
        if not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
    return B, C, ny, nx


def eval_any(s, mask, Ninv, P, d=None, handle=None, chi2=None, grad=None, stream=None):
    """wf_eval_any: objective and gradient on ny x nx maps whose sides have no
    prime factor above 7 (d None: the Hessian-vector product in grad).
    s (B, C, ny, nx/2+1) complex, mask uint8 (B, ny, nx), Ninv and d
    (B, C, ny, nx), P (C, ny, nx/2+1), all CUDA tensors of the working type
    (float64: FP64, float32: mixed) on the current device.  Every tensor is
    checked before the library is called.  Returns (chi2, grad)."""
    import torch
    if not isinstance(Ninv, torch.Tensor) or not Ninv.is_cuda:
        raise TypeError("Ninv must be a CUDA tensor")
    dev = torch.device("cuda", torch.cuda.current_device())
    grad = torch.empty_like(s) if grad is None else grad
    chi2 = torch.empty(Ninv.shape[0], dtype=torch.float64, device=Ninv.device) if chi2 is None else chi2
    B, C, ny, nx = _any_check(s, mask, Ninv, P, d, chi2, grad, dev)
    if s.data_ptr() == grad.data_ptr():
        raise ValueError("s and grad must not alias")
    h = handle if handle is not None else default_handle()
    precision = WF_FP64 if Ninv.dtype == torch.float64 else WF_MIXED
    _check(lib().wf_eval_any(h.ptr, B, C, ny, nx, precision, _ptr(d), _ptr(mask), _ptr(Ninv), _ptr(P), _ptr(s),
                             _ptr(grad), _ptr(chi2), _stream(stream)))
    return chi2, grad


def debug_bounds(mode=0):
    """wf_debug_bounds (bounds-checked build only): (violations, first) with
    first = (unit, source line, index, limit) of the first one or None."""
    cnt = ctypes.c_ulonglong()
    first = (ctypes.c_longlong * 4)(-1, -1, -1, -1)
    _check(lib().wf_debug_bounds(ctypes.byref(cnt), first, int(mode)))
    return int(cnt.value), (tuple(first) if cnt.value else None)


def solve_many(problems, stream=None, **opts):
    """wf_map_solve_many: solve several problems (one per map shape) at once.
    Returns one SolveResult per problem."""
    import torch
    o = WfOpts()
    lib().wf_opts_default(ctypes.byref(o))
    for k, v in opts.items():
        setattr(o, k, v)
    o.stream = _stream(stream)
    dev = torch.device("cuda", torch.cuda.current_device())
    outs = [torch.empty(p.spec_shape(), dtype=p._cplx(), device=dev) for p in problems]
    sts = [(WfSolveStats * p.B)() for p in problems]
    np_ = len(problems)
    parr = (ctypes.c_void_p * np_)(*[p._p.value for p in problems])
    oarr = (ctypes.c_void_p * np_)(*[_ptr(t) for t in outs])
    sarr = (ctypes.POINTER(WfSolveStats) * np_)(*[ctypes.cast(st, ctypes.POINTER(WfSolveStats)) for st in sts])
    status = lib().wf_map_solve_many(parr, np_, ctypes.byref(o), oarr, sarr)
    if status not in (0, 5):
        _check(status)
    return [SolveResult(s=t, x=None, stats=Problem._stats(st)) for t, st in zip(outs, sts)]


def alu_peak(dtype="f32"):
    """wf_alu_peak: measured FMA throughput of the current device, flop/s."""
    v = ctypes.c_double()
    _check(lib().wf_alu_peak(WF_F64 if dtype in ("f64", "fp64") else WF_F32, ctypes.byref(v)))
    return v.value


def band_table(n, edges, C=1, kscale=1.0, nx=None):
    """wf_band_table (wf_band_table_rect with nx): int16 numpy array
    (C, n, nx/2+1) of band ids from |k| edges (nx = n by default)."""
    e = np.ascontiguousarray(edges, dtype=np.float64)
    nx = n if nx is None else nx
    out = np.empty((C, n, nx // 2 + 1), dtype=np.int16)
    _check(lib().wf_band_table_rect(int(n), int(nx), int(C), e.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                    len(e) - 1, float(kscale), out.ctypes.data))
    return out


def normal_draw(seed, count, stream_id=0, offset=0, dtype=None, out=None, stream=None):
    """wf_normal_draw: `count` standard normal deviates of (seed, stream_id)
    starting at deviate `offset`, as a CUDA tensor (float64 by default)."""
    import torch
    if out is None:
        out = torch.empty(int(count), dtype=dtype or torch.float64, device="cuda")
    _check(lib().wf_normal_draw(int(seed), int(stream_id), int(offset), int(count),
                                WF_F64 if out.dtype == torch.float64 else WF_F32, _ptr(out), _stream(stream)))
    return out


def _bandpower_args(d, mask, Ninv, P, band, n_bands, z, noise, u, precision, stream, n_sim, n_fd, sim_index,
                    opts, fd_bands=None, trunc=(0, 0), out_on_device=False, leak_split=0):
    """ctypes arguments shared by bandpower_estimate and bandpower_iterate."""
    import torch
    _need(Ninv, "Ninv")
    if Ninv.dim() != 3 or Ninv.dtype not in (torch.float32, torch.float64):
        raise ValueError("Ninv must be a float32 or float64 (C, ny, nx) tensor")
    C, n, nx = Ninv.shape
    ddt = Ninv.dtype
    wdt = torch.float64 if precision == "fp64" else torch.float32
    _need(d, "d", (C, n, nx), ddt)
    _need(mask, "mask", (n, nx), torch.uint8)
    _need(P, "P", (C, n, nx // 2 + 1), ddt)
    _need(band, "band", (C, n, nx // 2 + 1), torch.int16)
    m = WfMap(d=_ptr(d), mask=_ptr(mask), Ninv=_ptr(Ninv), P=_ptr(P))
    nb = int(n_bands)
    J = int(z.shape[0]) if z is not None else int(n_sim)
    F = int(u.shape[1]) if u is not None else int(n_fd)
    for name, t in (("z", z), ("noise", noise)):  # all-or-none of the fields is the library's check
        if t is not None:
            _need(t, name, (J, C, n, nx), wdt)
    idx = None
    if sim_index is not None:
        idx = np.ascontiguousarray(sim_index, dtype=np.int64)
        if idx.shape != (J,):
            raise ValueError("sim_index needs one entry per simulation")
    fdb = None if fd_bands is None else np.ascontiguousarray(fd_bands, dtype=np.int32)
    L = int(leak_split)
    nR = ((L if L > 0 else nb) if fdb is None else int(fdb.size)) + (1 if L > 0 else 0)  # Fisher rows of u
    if u is not None and int(u.shape[0]) != nR:
        raise ValueError(f"u has {int(u.shape[0])} Fisher rows, the call needs {nR}")
    if u is not None:
        _need(u, "u", (nR, F, C, n, nx), wdt)
    bi = WfBandpowerIn(n_bands=nb, n_sim=J, n_fd=F, leak_split=L,
                       band=_ptr(band), z=_ptr(z), noise=_ptr(noise), u=_ptr(u),
                       sim_index=None if idx is None else idx.ctypes.data,
                       fd_bands=None if fdb is None else fdb.ctypes.data, n_fd_bands=0 if fdb is None else int(fdb.size),
                       trunc_bands=int(trunc[0]), trunc_width=int(trunc[1]), out_on_device=int(bool(out_on_device)))
    nmaps = 1 + J + nR * F
    sizes = (("theta_fid", nb), ("E", nb), ("bias", nb), ("fisher", nb * nb), ("cov", nb * nb),
             ("theta_hat", nb), ("cov_E", nb * nb), ("E_maps", nmaps * nb))
    if out_on_device:  # float64 CUDA tensors on the current device
        arrs = {k: torch.zeros(sz, dtype=torch.float64, device="cuda") for k, sz in sizes}
        ptrs = {k: ctypes.cast(ctypes.c_void_p(v.data_ptr()), ctypes.POINTER(ctypes.c_double)) for k, v in arrs.items()}
    else:
        arrs = {k: np.zeros(sz) for k, sz in sizes}
        ptrs = {k: v.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) for k, v in arrs.items()}
    bo = WfBandpowerOut(**ptrs)
    o = WfOpts()
    lib().wf_opts_default(ctypes.byref(o))
    for k, v in opts.items():
        setattr(o, k, v)
    o.stream = _stream(stream)
    st = (WfSolveStats * nmaps)()
    prec = WF_FP64 if precision == "fp64" else WF_MIXED
    dt = WF_F64 if Ninv.dtype == torch.float64 else WF_F32
    return dict(m=m, bi=bi, bo=bo, o=o, st=st, arrs=arrs, n=n, nx=nx, C=C, nb=nb, nmaps=nmaps, prec=prec, dt=dt,
                keep=(idx, fdb))


def _bandpower_result(a):
    arrs, nb = a["arrs"], a["nb"]
    for k in ("fisher", "cov", "cov_E"):
        arrs[k] = arrs[k].reshape(nb, nb)
    arrs["E_maps"] = arrs["E_maps"].reshape(a["nmaps"], nb)
    return arrs, Problem._stats(a["st"])


def bandpower_estimate(d, mask, Ninv, P, band, n_bands, z, noise, u, precision="fp64",
                       handle=None, stream=None, n_sim=None, n_fd=None, sim_index=None, fd_bands=None,
                       trunc=(0, 0), out_on_device=False, leak_split=0, **opts):
    """bandpower_estimate: band powers, noise bias, Fisher matrix and covariance
    of one data map from simulations (Sec. 2.4-2.5).  d, Ninv (C, ny, nx) and P
    (C, ny, nx/2+1) CUDA tensors of one float dtype; mask (ny, nx) uint8; band
    (C, ny, nx/2+1) int16; z, noise (n_sim, C, ny, nx), u (n_bands, n_fd, C, ny, nx)
    in the working type, or all three None with n_sim and n_fd given (the
    library then draws them from opts `seed`; sim_index gives the global index
    of each simulation, so that the draws do not depend on how simulations are
    split over calls).  fd_bands: the bands given Fisher maps (default all;
    the others' Fisher columns are interpolated, u then has one row per listed
    band); trunc = (n, w): zero F[l][l'] for l, l' < n with |l - l'| > w.
    leak_split = L > 0 (C = 2, E bands 0..L-1, B bands L..): the leakage-bias
    form of App. C, per-band Fisher maps for the E bands only, one joint map of
    all B bands per Fisher simulation giving the B bands' diagonal, no E-B
    cross terms; u then has the E rows and one more, the B fields.
    Returns (dict of numpy arrays, or float64 CUDA tensors with out_on_device,
    per-map stats)."""
    a = _bandpower_args(d, mask, Ninv, P, band, n_bands, z, noise, u, precision, stream, n_sim, n_fd, sim_index,
                        opts, fd_bands, trunc, out_on_device, leak_split)
    handle = handle or default_handle()
    status = lib().bandpower_estimate_rect(handle.ptr, ctypes.byref(a["m"]), a["n"], a["nx"], a["C"], a["dt"],
                                           a["prec"], ctypes.byref(a["bi"]), ctypes.byref(a["o"]),
                                           ctypes.byref(a["bo"]), a["st"])
    if status not in (0, 5):
        _check(status)
    return _bandpower_result(a)


def bandpower_iterate(d, mask, Ninv, P, band, n_bands, z, noise, u, n_iter=2, q_min=0.01, q_max=100.0,
                      precision="fp64", handle=None, stream=None, n_sim=None, n_fd=None, sim_index=None,
                      fd_bands=None, trunc=(0, 0), out_on_device=False, leak_split=0, **opts):
    """bandpower_iterate: n_iter estimates, the fiducial P moved to each estimate
    in between (Sec. 2.3).  Arguments as bandpower_estimate.  Returns (last
    estimate, per-map stats of the last run, Theta_hat of every estimate
    (n_iter, n_bands), final fiducial P as a CUDA tensor like P)."""
    import torch
    a = _bandpower_args(d, mask, Ninv, P, band, n_bands, z, noise, u, precision, stream, n_sim, n_fd, sim_index,
                        opts, fd_bands, trunc, out_on_device, leak_split)
    handle = handle or default_handle()
    hist = np.zeros((int(n_iter), a["nb"]))
    P_out = torch.empty_like(P)
    status = lib().bandpower_iterate_rect(handle.ptr, ctypes.byref(a["m"]), a["n"], a["nx"], a["C"], a["dt"],
                                          a["prec"], ctypes.byref(a["bi"]), ctypes.byref(a["o"]), int(n_iter),
                                          float(q_min), float(q_max), _ptr(P_out),
                                          hist.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                          ctypes.byref(a["bo"]), a["st"])
    if status not in (0, 5):
        _check(status)
    res, stats = _bandpower_result(a)
    return res, stats, hist, P_out


def fisher_rows(n_bands, leak_split=0, fd_bands=None):
    """Fisher-map rows of a band-power call (the rows of its u): the bands with
    per-band Fisher maps, plus the joint B row of the leakage-bias form."""
    L = int(leak_split)
    per_band = len(fd_bands) if fd_bands is not None else (L if L > 0 else int(n_bands))
    return per_band + (1 if L > 0 else 0)


def _dptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def bandpower_sums(E_maps, n_sim, n_fd, n_rows):
    """bandpower_sums: the partial-sum vector of one share of the simulations
    from its per-map band energies (rows: data, n_sim simulations, n_rows x
    n_fd Fisher maps).  Returns a float64 numpy vector; vectors of different
    shares add entry by entry."""
    E = np.ascontiguousarray(E_maps, dtype=np.float64)
    if E.ndim != 2 or E.shape[0] != 1 + int(n_sim) + int(n_rows) * int(n_fd):
        raise ValueError(f"E_maps has shape {E.shape}, expected (1 + n_sim + n_rows * n_fd, n_bands)")
    L = lib()
    out = np.zeros(L.bandpower_sums_len(E.shape[1], int(n_rows)))
    _check(L.bandpower_sums(_dptr(E), E.shape[1], int(n_sim), int(n_fd), int(n_rows), _dptr(out)))
    return out


def bandpower_combine(sums, E_data, theta_fid, leak_split=0, fd_bands=None, trunc=(0, 0)):
    """bandpower_combine: the band-power estimate from summed partial sums
    (host arrays in, numpy arrays out), with the Fisher-row rules of the
    contributing calls (leak_split, fd_bands, trunc)."""
    th = np.ascontiguousarray(theta_fid, dtype=np.float64)
    Ed = np.ascontiguousarray(E_data, dtype=np.float64)
    S = np.ascontiguousarray(sums, dtype=np.float64)
    nb = th.size
    L = lib()
    if Ed.shape != (nb,) or S.shape != (L.bandpower_sums_len(nb, fisher_rows(nb, leak_split, fd_bands)),):
        raise ValueError("E_data needs n_bands entries and sums the length of the rules' partial sums")
    fdb = None if fd_bands is None else np.ascontiguousarray(fd_bands, dtype=np.int32)
    rules = WfBandpowerIn(n_bands=nb, leak_split=int(leak_split),
                          fd_bands=None if fdb is None else fdb.ctypes.data,
                          n_fd_bands=0 if fdb is None else int(fdb.size), trunc_bands=int(trunc[0]),
                          trunc_width=int(trunc[1]), out_on_device=0)
    sizes = (("theta_fid", nb), ("E", nb), ("bias", nb), ("fisher", nb * nb), ("cov", nb * nb),
             ("theta_hat", nb), ("cov_E", nb * nb))
    arrs = {k: np.zeros(sz) for k, sz in sizes}
    bo = WfBandpowerOut(**{k: _dptr(v) for k, v in arrs.items()}, E_maps=None)
    _check(L.bandpower_combine(_dptr(S), _dptr(Ed), _dptr(th), ctypes.byref(rules), ctypes.byref(bo)))
    for k in ("fisher", "cov", "cov_E"):
        arrs[k] = arrs[k].reshape(nb, nb)
    return arrs


class Problem:
    """A prepared batch of maps of one shape (wf_problem_create_rect).

    d, Ninv: (B, C, ny, nx) CUDA tensors (square or not, sides powers of two);
    mask: (B, ny, nx) or (ny, nx) uint8; P: (B, C, ny, nx/2+1) or (C, ny, nx/2+1).  Floating inputs must share one dtype
    (float32 or float64).  precision: "fp64" or "mixed".  State arrays (s, grad,
    z, noise, outputs) use the working type: float64 for fp64, float32 for mixed."""

    def __init__(self, d, mask, Ninv, P, precision="fp64", lbfgs_m=10, handle=None, stream=None):
        import torch
        _need(Ninv, "Ninv")
        if Ninv.dim() != 4:
            raise ValueError("Ninv must have shape (B, C, ny, nx)")
        B, C, n, nx = Ninv.shape
        self.B, self.C, self.n, self.nx = B, C, n, nx
        dtype = Ninv.dtype
        if dtype not in (torch.float32, torch.float64):
            raise TypeError("inputs must be float32 or float64")
        if d is not None:
            _need(d, "d", (B, C, n, nx), dtype)
        _need(mask, "mask", (B, n, nx) if mask.dim() == 3 else (n, nx), torch.uint8)
        _need(P, "P", (B, C, n, nx // 2 + 1) if P.dim() == 4 else (C, n, nx // 2 + 1), dtype)
        self.handle = handle or default_handle()
        self.precision = WF_FP64 if precision == "fp64" else WF_MIXED
        self.wdtype = torch.float64 if self.precision == WF_FP64 else torch.float32
        masks = mask if mask.dim() == 3 else mask.unsqueeze(0).expand(B, n, nx)
        Ps = P if P.dim() == 4 else P.unsqueeze(0).expand(B, *P.shape)
        self._keep = (d, masks, Ninv, Ps)
        arr = (WfMap * B)()
        for b in range(B):
            arr[b].d = _ptr(d[b]) if d is not None else 0
            arr[b].mask = _ptr(masks[b])
            arr[b].Ninv = _ptr(Ninv[b])
            arr[b].P = _ptr(Ps[b])
        out = ctypes.c_void_p()
        _check(lib().wf_problem_create_rect(self.handle.ptr, arr, B, n, nx, C,
                                            WF_F64 if dtype == torch.float64 else WF_F32,
                                            self.precision, lbfgs_m, _stream(stream), ctypes.byref(out)))
        self._p = out
        self._keep = None

    def close(self):
        if getattr(self, "_p", None):
            lib().wf_problem_destroy(self._p)
            self._p = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # shapes -----------------------------------------------------------------
    def spec_shape(self):
        return (self.B, self.C, self.n, self.nx // 2 + 1)

    def pix_shape(self):
        return (self.B, self.C, self.n, self.nx)

    def _cplx(self):
        import torch
        return torch.complex128 if self.precision == WF_FP64 else torch.complex64

    def _spec(self, t):
        import torch
        if (not t.is_cuda or t.dtype != self._cplx() or tuple(t.shape) != self.spec_shape()
                or not t.is_contiguous()):
            raise ValueError(f"spectrum must be contiguous {self._cplx()} of shape {self.spec_shape()}")
        return t

    def history(self, cap):
        """wf_solver_history: per map a float64 array (n_b, 5) of (k, chi2,
        |g|/|g0|, alpha, evals), the last iterations of the solve started with
        history=cap."""
        out = np.empty((self.B, cap, 5), dtype=np.float64)
        counts = np.zeros(self.B, dtype=np.int32)
        _check(lib().wf_solver_history(self._p, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                       counts.ctypes.data_as(ctypes.POINTER(ctypes.c_int))))
        return [out[b, : counts[b]].copy() for b in range(self.B)]

    def variant(self):
        """FFT-stage variant in use (wf_opts.fft_variant encoding: 1000 a + 100 b + 10 c + d)."""
        v = ctypes.c_int()
        _check(lib().wf_problem_variant(self._p, ctypes.byref(v)))
        return v.value

    # calls --------------------------------------------------------------------
    def eval(self, s, grad=None, chi2=None, stream=None):
        import torch
        self._spec(s)
        grad = torch.empty_like(s) if grad is None else grad
        chi2 = torch.empty(self.B, dtype=torch.float64, device=s.device) if chi2 is None else chi2
        _check(lib().wf_eval(self._p, _ptr(s), _ptr(grad), _ptr(chi2), _stream(stream)))
        return chi2, grad

    def set_band_scale(self, band, q, stream=None):
        """wf_problem_set_band_scale: P <- q[band] P (band int16 (C, ny, nx/2+1),
        q float64 (n_b,) CUDA tensors)."""
        _check(lib().wf_problem_set_band_scale(self._p, _ptr(band), _ptr(q), int(q.numel()), _stream(stream)))

    def eval_bands(self, s, band, n_b, stream=None):
        """wf_eval_bands: (chi2, grad, d chi2 / d log q) at the current band scale."""
        import torch
        self._spec(s)
        grad = torch.empty_like(s)
        chi2 = torch.empty(self.B, dtype=torch.float64, device=s.device)
        dq = torch.empty((self.B, int(n_b)), dtype=torch.float64, device=s.device)
        _check(lib().wf_eval_bands(self._p, _ptr(s), _ptr(grad), _ptr(chi2), _ptr(band), int(n_b), _ptr(dq),
                                   _stream(stream)))
        return chi2, grad, dq

    def hess_vec(self, v, out=None, stream=None):
        import torch
        self._spec(v)
        out = torch.empty_like(v) if out is None else out
        _check(lib().wf_hess_vec(self._p, _ptr(v), _ptr(out), _stream(stream)))
        return out

    def signal_map(self, s, out=None, stream=None):
        import torch
        self._spec(s)
        out = torch.empty(self.pix_shape(), dtype=self.wdtype, device=s.device) if out is None else out
        _check(lib().wf_signal_map(self._p, _ptr(s), _ptr(out), _stream(stream)))
        return out

    def simulate(self, z, noise, out=None, stream=None):
        import torch
        for t in (z, noise):
            if (not t.is_cuda or t.dtype != self.wdtype or tuple(t.shape) != self.pix_shape()
                    or not t.is_contiguous()):
                raise ValueError("z and noise must be contiguous working-type CUDA pixel maps")
        out = torch.empty_like(z) if out is None else out
        _check(lib().wf_simulate_data(self._p, _ptr(z), _ptr(noise), _ptr(out), _stream(stream)))
        return out

    def set_data(self, d, stream=None):
        if not d.is_cuda or d.dtype != self.wdtype or tuple(d.shape) != self.pix_shape() or not d.is_contiguous():
            raise ValueError("d must be a contiguous working-type CUDA pixel map batch")
        _check(lib().wf_problem_set_data(self._p, _ptr(d), _stream(stream)))

    def band_energy(self, s, band, theta, out=None, stream=None):
        import torch
        self._spec(s)
        nb = int(theta.numel())
        out = torch.empty((self.B, nb), dtype=torch.float64, device=s.device) if out is None else out
        _check(lib().wf_band_energy(self._p, _ptr(s), _ptr(band), _ptr(theta), nb, _ptr(out),
                                    _stream(stream)))
        return out

    def _opts(self, stream, opts):
        o = WfOpts()
        lib().wf_opts_default(ctypes.byref(o))
        for k, v in opts.items():
            if not hasattr(o, k):
                raise TypeError(f"unknown option {k}")
            setattr(o, k, v)
        o.stream = _stream(stream)
        return o

    def start(self, s0=None, stream=None, **opts):
        """wf_solver_start: prepare an L-BFGS solve from s0 (None = 0)."""
        self._o = self._opts(stream, opts)
        _check(lib().wf_solver_start(self._p, ctypes.byref(self._o), _ptr(s0)))

    def step(self, n_iter, sync=True):
        """wf_solver_step: run n_iter iterations; returns the active count if sync."""
        na = ctypes.c_int(-1)
        _check(lib().wf_solver_step(self._p, int(n_iter), ctypes.byref(na) if sync else None))
        return na.value if sync else None

    def export_state(self, out=None):
        """wf_solver_state_size + wf_solver_export: the checkpoint of the started
        solve as a uint8 tensor (a CUDA tensor by default; pass a pinned or
        plain CPU uint8 tensor of at least that size to keep it on the host)."""
        import torch
        n = ctypes.c_size_t()
        _check(lib().wf_solver_state_size(self._p, ctypes.byref(n)))
        if out is None:
            out = torch.empty(int(n.value), dtype=torch.uint8, device="cuda")
        if out.dtype != torch.uint8 or not out.is_contiguous() or out.numel() < n.value:
            raise ValueError(f"checkpoint buffer must be a contiguous uint8 tensor of >= {n.value} bytes")
        _check(lib().wf_solver_export(self._p, _ptr(out), int(out.numel())))
        return out

    def import_state(self, buf, stream=None):
        """wf_solver_import: resume the solve held in a checkpoint buffer."""
        import torch
        if not isinstance(buf, torch.Tensor) or buf.dtype != torch.uint8 or not buf.is_contiguous():
            raise ValueError("checkpoint buffer must be a contiguous uint8 tensor")
        _check(lib().wf_solver_import(self._p, _ptr(buf), int(buf.numel()), _stream(stream)))

    def profile(self, n_iter):
        """wf_solver_profile: average ms of the six kernels of one iteration."""
        ms = (ctypes.c_float * 6)()
        _check(lib().wf_solver_profile(self._p, int(n_iter), ms))
        return list(ms)

    def finish(self, x_out=False):
        """wf_solver_finish: returns SolveResult."""
        import torch
        dev = torch.device("cuda", torch.cuda.current_device())
        s = torch.empty(self.spec_shape(), dtype=self._cplx(), device=dev)
        x = torch.empty(self.pix_shape(), dtype=self.wdtype, device=dev) if x_out else None
        st = (WfSolveStats * self.B)()
        status = lib().wf_solver_finish(self._p, _ptr(s), _ptr(x), st)
        res = SolveResult(s=s, x=x, stats=self._stats(st))
        if status not in (0, 5):
            raise WfError(status, lib().wf_last_error().decode(), res)
        return res

    @staticmethod
    def _stats(st):
        return [dict(iters=e.iters, evals=e.evals, status=STATUS.get(e.status, e.status),
                     chi2=e.chi2, gnorm_rel=e.gnorm_rel, fft_variant=e.fft_variant) for e in st]

    def solve_refined(self, cert_tol=1e-4, max_rounds=8, s0=None, stream=None, **opts):
        """wf_map_solve_refined: MAP solve to the certificate |grad|/2 <= cert_tol |s|
        with an FP64 state.  Returns (SolveResult with s complex128, certificates
        as a numpy array)."""
        import torch
        o = self._opts(stream, opts)
        if s0 is not None:
            self._spec(s0)
        dev = torch.device("cuda", torch.cuda.current_device())
        s = torch.empty(self.spec_shape(), dtype=torch.complex128, device=dev)
        cert = np.zeros(self.B, dtype=np.float64)
        st = (WfSolveStats * self.B)()
        status = lib().wf_map_solve_refined(self._p, ctypes.byref(o), float(cert_tol), int(max_rounds), _ptr(s0),
                                            _ptr(s), cert.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), st)
        res = SolveResult(s=s, x=None, stats=self._stats(st))
        if status not in (0, 5):
            raise WfError(status, lib().wf_last_error().decode(), res)
        return res, cert

    def solve(self, s0=None, x_out=False, stream=None, **opts):
        import torch
        o = WfOpts()
        lib().wf_opts_default(ctypes.byref(o))
        for k, v in opts.items():
            if not hasattr(o, k):
                raise TypeError(f"unknown option {k}")
            setattr(o, k, v)
        o.stream = _stream(stream)
        dev = torch.device("cuda", torch.cuda.current_device())
        s = torch.empty(self.spec_shape(), dtype=self._cplx(), device=dev)
        x = torch.empty(self.pix_shape(), dtype=self.wdtype, device=dev) if x_out else None
        st = (WfSolveStats * self.B)()
        status = lib().wf_map_solve(self._p, ctypes.byref(o), _ptr(s0), _ptr(s), _ptr(x), st)
        res = SolveResult(s=s, x=x, stats=self._stats(st))
        if status not in (0, 5):
            raise WfError(status, lib().wf_last_error().decode(), res)
        return res
