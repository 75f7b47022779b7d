"""Build the CUDA library libwf.so in-tree for sm_103a.

Each translation unit is compiled in parallel with nvcc, then linked into
paper_1810_00503_gb300/libwf.so (static CUDA runtime, no torch dependency).
Run ``python -m paper_1810_00503_gb300.build`` or call ``build()``.
"""
from __future__ import annotations

import os
import re
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OBJ = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libwf.so")
SOURCES = ["wf_api.cu", "wf_solve.cu", "wf_ops_f32.cu", "wf_ops_f64.cu", "wf_lbcol_f32.cu", "wf_lbcol_f64.cu",
           "wf_lbrow_f32.cu", "wf_lbrow_f64.cu", "wf_noalloc.cu", "wf_bandpower.cu", "wf_rng.cu", "wf_peak.cu",
           "wf_multi.cu", "wf_any.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2"]


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libwf.so")


def _compile(src: str, extra: list[str], obj_dir: str = OBJ) -> tuple[str, str]:
    obj = os.path.join(obj_dir, os.path.splitext(src)[0] + ".o")
    cmd = [_nvcc(), *ARCH, *FLAGS, *extra, "-c", os.path.join(CSRC, src), "-o", obj]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"nvcc failed on {src}:\n{res.stdout}\n{res.stderr}")
    return obj, res.stderr


def resources(log: str) -> list[dict]:
    """Per-kernel resources from ptxas -v output: for every entry function
    (mangled name) its registers, stack frame, spill store and load bytes and
    static shared memory."""
    out, cur, props = [], None, {}
    for line in log.splitlines():
        m = re.search(r"Compiling entry function '([^']+)'", line)
        if m:
            cur = {"kernel": m.group(1), "registers": 0, "stack": 0, "spill_stores": 0, "spill_loads": 0,
                   "smem": 0}
            out.append(cur)
            continue
        m = re.search(r"Function properties for (\S+)", line)
        if m:
            props = {"name": m.group(1)}
            continue
        m = re.search(r"(\d+) bytes stack frame, (\d+) bytes spill stores, (\d+) bytes spill loads", line)
        if m and cur is not None and props.get("name") == cur["kernel"]:
            cur["stack"], cur["spill_stores"], cur["spill_loads"] = (int(v) for v in m.groups())
            continue
        m = re.search(r"Used (\d+) registers", line)
        if m and cur is not None:
            cur["registers"] = int(m.group(1))
            sm = re.search(r"(\d+) bytes smem", line)
            cur["smem"] = int(sm.group(1)) if sm else 0
    return out


def _demangle(names: list[str]) -> list[str]:
    tool = shutil.which("c++filt")
    if not tool or not names:
        return names
    res = subprocess.run([tool], input="\n".join(names), capture_output=True, text=True)
    dem = res.stdout.splitlines() if res.returncode == 0 else []
    if len(dem) != len(names):
        return names
    return [d.split("(")[0].replace("void ", "", 1) for d in dem]


def resource_report() -> str:
    """Build with -Xptxas -v and return one line per kernel: source file,
    registers, stack frame, spill store / load bytes, static shared memory."""
    import io
    import contextlib
    buf = io.StringIO()
    with contextlib.redirect_stderr(buf):
        build(verbose=True)
    rows, src = [], None
    for part in re.split(r"^== (\S+)\n", buf.getvalue(), flags=re.M)[1:]:
        if src is None:
            src = part
            continue
        for r in resources(part):
            rows.append((src, r))
        src = None
    names = _demangle([r["kernel"] for _, r in rows])
    lines = [f"{'source':<18} {'kernel':<58} {'regs':>4} {'stack':>5} {'spill st/ld':>11} {'smem':>6}"]
    for (src, r), name in sorted(zip(rows, names), key=lambda t: (t[0][0], t[1])):
        lines.append(f"{src:<18} {name[:58]:<58} {r['registers']:>4} {r['stack']:>5} "
                     f"{str(r['spill_stores']) + '/' + str(r['spill_loads']):>11} {r['smem']:>6}")
    return "\n".join(lines)


DEBUG_OBJ = os.path.join(HERE, "_build_dbg")
DEBUG_LIB = os.path.join(HERE, "libwf_dbg.so")


def build(verbose: bool = False, extra: list[str] | None = None, debug_bounds: bool = False) -> str:
    """Compile every CUDA source and link libwf.so; returns the library path.
    verbose: pass -Xptxas -v and print its per-kernel resource report
    (registers, spill bytes, shared memory) for every source to stderr.
    debug_bounds: build the bounds-checked copy libwf_dbg.so instead
    (-DWF_DEBUG_BOUNDS; load it with WF_LIB_PATH)."""
    obj_dir, lib_path = (DEBUG_OBJ, DEBUG_LIB) if debug_bounds else (OBJ, LIB)
    os.makedirs(obj_dir, exist_ok=True)
    extra = list(extra or [])
    if debug_bounds:
        extra += ["-DWF_DEBUG_BOUNDS"]
    if verbose:
        extra += ["-Xptxas", "-v"]
    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        done = list(ex.map(lambda s: _compile(s, extra, obj_dir), SOURCES))
    objs = [o for o, _ in done]
    if verbose:
        for src, (_, log) in zip(SOURCES, done):
            sys.stderr.write(f"== {src}\n{log}")
    tmp = lib_path + ".tmp"
    cmd = [_nvcc(), *ARCH, "-shared", "-o", tmp, *objs]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"link failed:\n{res.stdout}\n{res.stderr}")
    os.replace(tmp, lib_path)
    return lib_path


if __name__ == "__main__":
    if "--resources" in sys.argv:
        print(resource_report())
    else:
        path = build(verbose="-v" in sys.argv)
        print(path)
