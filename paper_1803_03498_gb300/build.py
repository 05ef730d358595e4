"""Build libheom.so in-tree with nvcc for sm_103a (GB300).

Translation units are compiled in parallel, then linked into
``paper_1803_03498_gb300/_build/libheom.so``.  Rebuilds only what changed.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.environ.get("HEOM_CSRC_DIR") or os.path.join(HERE, "csrc")
OUT = os.environ.get("HEOM_BUILD_DIR") or os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libheom.so")
# the bounds-checked debug build (-DHEOM_DEBUG): every link record's neighbour, state and record range
# is checked in the stage kernels before use, and a failure is reported by heom_observables
DEBUG_OUT = os.path.join(HERE, "_build_debug")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
SOURCES = (["hierarchy.cpp", "heom_abi.cu", "propagate.cu", "tuner.cu", "batch.cu", "aux_kernels.cu", "heom_static.cu"]
           + [f"stage_{p}_{g}.cu" for p in ("fp64", "fp32", "head") for g in "abcd"]
           + ["stage_tc_a.cu", "stage_tc_b.cu", "vec_stage_g1.cu", "vec_stage_g2.cu", "vec_stage_g4.cu", "gen_stage.cu",
              "stage_col.cu", "stage_list_a.cu", "stage_list_b.cu", "stage_list_c.cu", "group.cu"])
HEADERS = ["hierarchy.h", "heom_internal.h", "heom_run.h", "stage_kernel.cuh", "stage_tc.cuh", "vec_kernel.cuh", "gen_kernel.cuh",
           "stage_col.cuh", "stage_list.cuh"]


def _nvcc():
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.isabs(c) and os.path.exists(c) or not os.path.isabs(c)):
            return c
    return "nvcc"


def _flags(debug=False):
    extra = os.environ.get("HEOM_NVCC_DEFINES", "").split()  # e.g. -DHEOM_STAGE_WARPS=8 (tuning builds)
    if debug:
        extra = extra + ["-DHEOM_DEBUG"]
    return ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
                   "-I", os.path.join(ROOT, "include"), "-I", os.path.join(HERE, "csrc"),
                   "--expt-relaxed-constexpr"] + extra


def _stale(obj, deps):
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(d) > t for d in deps)


def build(verbose: bool = False, jobs: int | None = None, debug: bool = False) -> str:
    """Compile and link libheom.so; debug=True builds the bounds-checked variant into _build_debug/
    (load it with HEOM_LIB=<path> in the environment).  Returns the library's path."""
    out = DEBUG_OUT if debug else OUT
    lib = os.path.join(out, "libheom.so")
    os.makedirs(out, exist_ok=True)
    nvcc = _nvcc()
    hdrs = [os.path.join(CSRC, h) for h in HEADERS] + [os.path.join(ROOT, "include", "heom.h")]
    objs, work = [], []
    for s in SOURCES:
        src = os.path.join(CSRC, s)
        obj = os.path.join(out, s + ".o")
        objs.append(obj)
        if _stale(obj, [src] + hdrs + [__file__]):
            cmd = [nvcc] + _flags(debug) + ["-c", src, "-o", obj]
            if s.endswith(".cpp"):
                cmd = [nvcc] + _flags(debug) + ["-x", "cu", "-c", src, "-o", obj]
            work.append(cmd)
    with cf.ThreadPoolExecutor(max_workers=jobs or max(1, min(len(work), os.cpu_count() or 1))) as ex:
        futs = [ex.submit(subprocess.run, cmd, capture_output=True, text=True) for cmd in work]
        for cmd, f in zip(work, futs):
            r = f.result()
            if verbose or r.returncode != 0:
                sys.stderr.write(" ".join(cmd) + "\n" + r.stdout + r.stderr)
            if r.returncode != 0:
                raise RuntimeError(f"nvcc failed: {cmd[-3]}")
    if work or not os.path.exists(lib) or _stale(lib, objs):
        tmp = lib + f".tmp{os.getpid()}"
        cmd = [nvcc] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            sys.stderr.write(" ".join(cmd) + "\n" + r.stdout + r.stderr)
            raise RuntimeError("link of libheom.so failed")
        os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv, debug="--debug" in sys.argv))
