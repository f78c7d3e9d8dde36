"""Builds ``liblpm.so`` (the CUDA library behind include/lpm.h) in-tree for sm_103a.

Each translation unit is compiled by nvcc in parallel, then linked into one shared
object next to this file. The static CUDA runtime is linked in, so the library only
needs the NVIDIA driver at run time.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "liblpm.so")
BUILD = os.path.join(HERE, "_build")
# The checked build: the same sources with every indexed access of the kernels tested
# against its array (a failed test sets the device error word; nothing traps), for
# verification runs in place of a memory checker.
OUT_CHECKED = os.path.join(HERE, "liblpm_checked.so")
BUILD_CHECKED = os.path.join(HERE, "_build_checked")
SOURCES = ["lpm_api.cu", "lpm_kernels.cu", "lpm_advance_b128.cu", "lpm_advance_b256.cu",
           "lpm_advance_b512.cu", "lpm_adjoint.cu", "lpm_noalloc.cu", "lpm_sort.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-Wall",
         "--expt-relaxed-constexpr", "-I", os.path.join(ROOT, "include")]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build liblpm.so")


def _stale(target: str, deps) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def _headers():
    hs = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    return hs + [os.path.join(ROOT, "include", "lpm.h")]


def build(force: bool = False, verbose: bool = False, extra=(), checked: bool = False) -> str:
    """Builds liblpm.so (or, with ``checked``, liblpm_checked.so) and returns its path."""
    out_lib, build_dir = (OUT_CHECKED, BUILD_CHECKED) if checked else (OUT, BUILD)
    if checked:
        extra = tuple(extra) + ("-DLPM_CHECKED=1",)
    os.makedirs(build_dir, exist_ok=True)
    cc = nvcc()
    hdrs = _headers()
    jobs = []
    objs = []
    for src in SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(build_dir, src.replace(".cu", ".o"))
        objs.append(o)
        if force or _stale(o, [s] + hdrs):
            cmd = [cc, *ARCH, *FLAGS, *extra, "-c", s, "-o", o]
            if verbose:
                cmd.insert(1, "-Xptxas=-v")
            jobs.append(cmd)

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        return cmd, r

    with cf.ThreadPoolExecutor(max_workers=max(1, len(jobs))) as ex:
        for cmd, r in ex.map(run, jobs):
            if verbose or r.returncode != 0:
                sys.stderr.write(r.stdout + r.stderr)
            if r.returncode != 0:
                raise RuntimeError(f"nvcc failed: {' '.join(cmd)}")
    if force or jobs or _stale(out_lib, objs):
        tmp = out_lib + f".{os.getpid()}.tmp"
        subprocess.check_call([cc, *ARCH, "-shared", "-o", tmp, *objs])
        os.replace(tmp, out_lib)
    return out_lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv,
                checked="--checked" in sys.argv))
