"""Build the CUDA library libtmg.so in-tree for sm_103a (nvcc, no cmake).

The translation units compile in parallel; the result lands in
``paper_1409_5254_gb300/_build/libtmg.so`` (git-ignored).
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libtmg.so")
# the debug build with bounds checks (-DTMG_BOUNDS, csrc/tmg_bounds.h)
OUT_BOUNDS = os.path.join(HERE, "_build_bounds")
LIB_BOUNDS = os.path.join(OUT_BOUNDS, "libtmg.so")
SOURCES = ["tmg_inst_f64_w21.cu", "tmg_inst_f32_w21.cu", "tmg_inst_f64_wide.cu", "tmg_inst_f32_wide.cu",
           "tmg_api.cu", "tmg_inst_f32.cu", "tmg_inst_f32_hi.cu", "tmg_inst_f64.cu", "tmg_inst_f64_hi.cu",
           "tmg_adjoint.cu", "tmg_batched.cu", "tmg_batched_hi.cu", "tmg_batched_wide.cu", "tmg_noalloc.cu", "tmg_heat.cu"]
HEADERS = ["tmg_kernels.cuh", "tmg_impl.cuh", "tmg_plan.h", "tmg_batched.cuh", "tmg_batched_host.h",
           "tmg_scan.cuh", "tmg_setup_math.h", "tmg_nvtx.h", "tmg_bounds.h"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-std=c++17", "-O3", "-lineinfo", "-Xcompiler", "-fPIC"]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    return "nvcc"


def _newest_input() -> float:
    paths = [os.path.join(CSRC, s) for s in SOURCES + HEADERS if os.path.exists(os.path.join(CSRC, s))]
    paths.append(os.path.join(HERE, "..", "include", "tmg.h"))
    return max(os.path.getmtime(p) for p in paths)


def build(force: bool = False, verbose: bool = False, bounds: bool = False) -> str:
    """Compile every translation unit and link libtmg.so; bounds=True builds
    the debug library with bounds checks into _build_bounds instead."""
    out, lib = (OUT_BOUNDS, LIB_BOUNDS) if bounds else (OUT, LIB)
    os.makedirs(out, exist_ok=True)
    if not force and os.path.exists(lib) and os.path.getmtime(lib) >= _newest_input():
        return lib
    nvcc = _nvcc()
    procs, objs = [], []
    for src in SOURCES:
        path = os.path.join(CSRC, src)
        if not os.path.exists(path):
            continue
        obj = os.path.join(out, src.replace(".cu", ".o"))
        objs.append(obj)
        cmd = [nvcc, *ARCH, *FLAGS, *(["-DTMG_BOUNDS"] if bounds else []), "-c", path, "-o", obj]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        procs.append((src, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    failed = []
    for src, p in procs:
        out, _ = p.communicate()
        if verbose or p.returncode != 0:
            sys.stderr.write(out.decode(errors="replace"))
        if p.returncode != 0:
            failed.append(src)
    if failed:
        raise RuntimeError(f"nvcc failed for {failed}")
    tmp = lib + f".tmp{os.getpid()}"
    subprocess.check_call([nvcc, *ARCH, "-shared", "-o", tmp, *objs])
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv, bounds="--bounds" in sys.argv))
