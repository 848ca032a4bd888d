"""In-tree nvcc build of the CUDA library (sm_103a only).

`build_library()` compiles csrc/*.cu into _build/libtpflbm.so next to this file
and returns its path; it rebuilds only when a source is newer than the library.
"""
from __future__ import annotations

import glob
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
LIB = os.path.join(HERE, "_build", "libtpflbm.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def sources():
    return sorted(glob.glob(os.path.join(HERE, "csrc", "*.cu")))


def _deps():
    return sources() + sorted(glob.glob(os.path.join(HERE, "csrc", "*.cuh"))) + sorted(
        glob.glob(os.path.join(HERE, "csrc", "*.h"))) + sorted(glob.glob(os.path.join(ROOT, "include", "*.h")))


def build_library(force: bool = False, verbose: bool = False, out: str | None = None, defines=()) -> str:
    """Compile every csrc/*.cu (in parallel, one nvcc per file) and link the shared
    library.  `out` and `defines` (-D flags) serve tuning builds beside the default."""
    lib = out or LIB
    os.makedirs(os.path.dirname(lib), exist_ok=True)
    if not force and os.path.exists(lib):
        t = os.path.getmtime(lib)
        if all(os.path.getmtime(d) <= t for d in _deps()):
            return lib
    nvcc = os.environ.get("NVCC", "nvcc")
    flags = ["-O3", "-std=c++17", *ARCH, "-lineinfo", "-Xcompiler", "-fPIC", "-I", os.path.join(ROOT, "include"),
             *["-D" + d for d in defines]]
    if verbose:
        flags.insert(0, "-Xptxas=-v")
    objs = [os.path.splitext(lib)[0] + "." + os.path.splitext(os.path.basename(s))[0] + ".%d.o" % os.getpid()
            for s in sources()]
    procs = [subprocess.Popen([nvcc, *flags, "-c", "-o", o, src]) for src, o in zip(sources(), objs)]
    bad = [src for src, pr in zip(sources(), procs) if pr.wait() != 0]
    try:
        if bad:
            raise RuntimeError("nvcc failed on %s" % ", ".join(os.path.basename(b) for b in bad))
        tmp = lib + ".%d.tmp" % os.getpid()
        subprocess.run([nvcc, *ARCH, "-shared", "-o", tmp, *objs], check=True)
        os.replace(tmp, lib)
    finally:
        for o in objs:
            if os.path.exists(o):
                os.remove(o)
    return lib


if __name__ == "__main__":
    print(build_library(force=True, verbose=True))
