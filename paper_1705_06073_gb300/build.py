"""Build the CUDA library liblse.so for sm_103a (GB300) in-tree.

Each translation unit is compiled in parallel with nvcc and linked into
``_build/liblse.so`` next to this file.  Only ``-gencode
arch=compute_103a,code=sm_103a`` is emitted: the library is GB300-only.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "liblse.so")
# (source, object, extra nvcc flags): lse_fit.cu builds as four units, one
# per kernel precision and one for its host code, so that they compile in
# parallel
UNITS = [("lse_api.cu", "lse_api.o", []), ("lse_grid.cu", "lse_grid.o", []),
         ("lse_noalloc.cu", "lse_noalloc.o", []), ("lse_serve.cu", "lse_serve.o", []),
         ("lse_semifast.cu", "lse_semifast.o", [])] + [
    ("lse_fit.cu", f"lse_fit{u}.o", [f"-DLSE_FIT_UNIT={u}"]) for u in range(4)]


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _cuda_lib_dir(nvcc: str) -> str:
    root = os.path.dirname(os.path.dirname(os.path.realpath(nvcc)))
    for sub in ("lib64", "lib", "targets/sbsa-linux/lib", "targets/x86_64-linux/lib"):
        d = os.path.join(root, sub)
        if os.path.exists(os.path.join(d, "libcudart.so")):
            return d
    return os.path.join(root, "lib64")


FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-lineinfo", "-std=c++17",
         "--extended-lambda", "-Xcompiler", "-fPIC", "-Xcompiler", "-fvisibility=hidden",
         "-Xptxas", "-warn-spills"]


def _newer(target: str, deps) -> bool:
    if not os.path.exists(target):
        return False
    t = os.path.getmtime(target)
    return all(os.path.getmtime(d) <= t for d in deps)


def build(verbose: bool = False, force: bool = False) -> str:
    nvcc = _nvcc()
    os.makedirs(OUT, exist_ok=True)
    headers = [os.path.join(SRC, f) for f in os.listdir(SRC) if f.endswith((".cuh", ".h"))]
    headers.append(os.path.join(os.path.dirname(HERE), "include", "lse.h"))
    objs, jobs = [], []
    for u, o, extra in UNITS:
        src = os.path.join(SRC, u)
        obj = os.path.join(OUT, o)
        objs.append(obj)
        if force or not _newer(obj, [src, *headers, __file__]):
            jobs.append([nvcc, *FLAGS, *extra, "-c", src, "-o", obj])
    if jobs:
        with cf.ThreadPoolExecutor(max_workers=len(jobs)) as ex:
            res = list(ex.map(lambda c: subprocess.run(c, capture_output=True, text=True), jobs))
        for cmd, r in zip(jobs, res):
            if verbose or r.returncode:
                sys.stderr.write(r.stdout + r.stderr)
            if r.returncode:
                raise RuntimeError("nvcc failed: " + " ".join(cmd))
    if force or jobs or not _newer(LIB, objs):
        libdir = _cuda_lib_dir(nvcc)
        cmd = [nvcc, "-shared", "-gencode", "arch=compute_103a,code=sm_103a", "-cudart", "shared",
               "-Xlinker", "-rpath=" + libdir, "-o", LIB, *objs]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode:
            sys.stderr.write(r.stdout + r.stderr)
            raise RuntimeError("link failed")
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv, force="-f" in sys.argv))
