"""Build the C-ABI CUDA library ``libhc.so`` in-tree for sm_103a.

Each ``csrc/*.cu`` translation unit compiles in parallel with
``nvcc -gencode arch=compute_103a,code=sm_103a``; the objects link into
``paper_1109_0545_gb300/_build/libhc.so`` against the shared CUDA runtime.  The build is
incremental on source modification times.  ``ptxas -v`` output (registers, spills) is
kept in ``_build/ptxas.log``.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(PKG, "_build")
INCLUDE = os.path.join(os.path.dirname(PKG), "include")
SO = os.path.join(BUILD, "libhc.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _deps() -> list[str]:
    return (glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h"))
            + glob.glob(os.path.join(INCLUDE, "*.h")))


def _compile(src: str, obj: str) -> str:
    cmd = [nvcc(), *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
           "-Xptxas", "-v", "-I", INCLUDE, "-c", src, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {os.path.basename(src)}:\n{r.stderr}")
    return r.stderr


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    srcs = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    newest_dep = max([os.path.getmtime(p) for p in _deps()] + [0.0])
    jobs = []
    for src in srcs:
        obj = os.path.join(BUILD, os.path.basename(src)[:-3] + ".o")
        stale = (force or not os.path.exists(obj) or os.path.getmtime(obj) < os.path.getmtime(src)
                 or os.path.getmtime(obj) < newest_dep)
        jobs.append((src, obj, stale))
    todo = [(s, o) for s, o, st in jobs if st]
    logs = []
    if todo:
        with cf.ThreadPoolExecutor(max_workers=min(len(todo), os.cpu_count() or 4)) as ex:
            for (src, _), log in zip(todo, ex.map(lambda so: _compile(*so), todo)):
                logs.append(f"== {os.path.basename(src)}\n{log}")
        for (src, _), log in zip(todo, logs):
            name = os.path.basename(src)[:-3]
            with open(os.path.join(BUILD, f"{name}.ptxas.log"), "w") as fh:
                fh.write(log)
    objs = [o for _, o, _ in jobs]
    if todo or not os.path.exists(SO):
        tmp = SO + f".{os.getpid()}.tmp"
        cmd = [nvcc(), *ARCH, "-shared", "-cudart", "shared", "-o", tmp, *objs]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stderr}")
        os.replace(tmp, SO)
    if verbose:
        print("\n".join(logs))
    return SO


if __name__ == "__main__":
    print(build(verbose=True))
