"""Build libgpmg.so in place with nvcc for sm_103a (GB300).

Each translation unit compiles in parallel; geometry.cu and ghost3d.cu are
compiled with -fmad=false (their floating-point decisions must use
separately rounded operations).  The library links the CUDA runtime statically.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
OUT = os.path.join(HERE, "libgpmg.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
SOURCES = ["geometry.cu", "ops.cu", "coarse.cu", "solver.cu", "noalloc.cu", "cn.cu", "krylov.cu", "adjoint.cu",
           "probe.cu", "levelset.cu", "mac3d.cu", "ghost3d.cu"]
EXTRA = {"geometry.cu": ["-fmad=false"], "ghost3d.cu": ["-fmad=false"]}


def nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _stale(objs) -> bool:
    if not os.path.exists(OUT):
        return True
    t = os.path.getmtime(OUT)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(INCLUDE, "gpmg.h"), __file__]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    bdir = os.path.join(HERE, "_build")
    os.makedirs(bdir, exist_ok=True)
    objs = [os.path.join(bdir, s.replace(".cu", ".o")) for s in SOURCES]
    if not force and not _stale(objs):
        return OUT
    nv = nvcc()
    base = [nv, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE,
            "--expt-relaxed-constexpr", "-Xptxas", "-v" if verbose else "-O3"]

    def one(src_obj):
        src, obj = src_obj
        cmd = base + EXTRA.get(src, []) + ["-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (src, r.stdout, r.stderr))
        return r.stderr

    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        logs = list(ex.map(one, zip(SOURCES, objs)))
    if verbose:
        for lg in logs:
            sys.stderr.write(lg)
    tmp = OUT + ".%d.tmp" % os.getpid()
    r = subprocess.run([nv, *ARCH, "-shared", "-o", tmp, *objs], capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s\n%s" % (r.stdout, r.stderr))
    os.replace(tmp, OUT)
    return OUT


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
