"""In-tree build of libsplat.so for sm_103a (nvcc, one object per .cu, compiled in parallel),
and of its checked variant libsplat_checked.so (SPLAT_CHECKED: every kernel index checked)."""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libsplat.so")
BUILD_CHECKED = os.path.join(HERE, "_build_checked")
LIB_CHECKED = os.path.join(HERE, "libsplat_checked.so")
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2"]


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return sorted(glob.glob(os.path.join(CSRC, "*.cuh")) + [os.path.join(HERE, "..", "include", "splat.h")])


def _stale(target: str, inputs) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(p) > t for p in inputs)


def lib_path(checked: bool = False) -> str:
    return LIB_CHECKED if checked else LIB


def build(force: bool = False, verbose: bool = False, checked: bool = False) -> str:
    """Compile every kernel source and link libsplat.so (with checked=True the checked
    build, libsplat_checked.so); returns the library path."""
    bdir, lib = (BUILD_CHECKED, LIB_CHECKED) if checked else (BUILD, LIB)
    flags = FLAGS + (["-DSPLAT_CHECKED"] if checked else [])
    os.makedirs(bdir, exist_ok=True)
    srcs = _sources()
    deps = _deps()
    objs = []
    jobs = []
    for s in srcs:
        o = os.path.join(bdir, os.path.basename(s) + ".o")
        objs.append(o)
        if force or _stale(o, [s] + deps):
            jobs.append((s, o))

    def compile_one(job):
        s, o = job
        tmp = o + f".tmp{os.getpid()}"
        cmd = [NVCC] + ARCH + flags + ["-c", s, "-o", tmp]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {s}:\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, o)
        if verbose:
            print("compiled", os.path.basename(s))

    if jobs:
        with cf.ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 4)) as ex:
            list(ex.map(compile_one, jobs))
    if force or jobs or _stale(lib, objs):
        tmp = lib + f".tmp{os.getpid()}"
        cmd = [NVCC] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(verbose=True))
    print(build(verbose=True, checked=True))
